// rtlbfs_capi.cu -- the extern "C" entry points of include/rtlbfs.h: a
// single-cavity handle over the shared engine (one slot).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "rtlbfs.h"
#include "rtlbfs_engine.h"

using rtlbfs::Cavity;
using rtlbfs::CavityCtl;
using rtlbfs::Engine;

struct rtlbfs_ctx {
    Engine* eng = nullptr;
    int slot = 0;
    std::string err;
};

namespace {

int finish(rtlbfs_t h, int rc)
{
    if (rc != RTLBFS_OK && h && h->eng) h->err = h->eng->error();
    return rc;
}

int argfail(rtlbfs_t h, const char* msg)
{
    if (h) h->err = msg;
    return RTLBFS_ERR_ARG;
}

Cavity* cav(rtlbfs_t h) { return h && h->eng ? h->eng->cavity(h->slot) : nullptr; }

int status_to_rc(int status)
{
    switch (status) {
    case rtlbfs::kConverged: return RTLBFS_OK;
    case rtlbfs::kMaxSteps: return RTLBFS_ERR_NOT_CONVERGED;
    case rtlbfs::kDiverged: return RTLBFS_ERR_DIVERGED;
    default: return RTLBFS_ERR_NOT_CONVERGED;
    }
}

}  // namespace

extern "C" {

int rtlbfs_tanh_faces(int n, double L, double phi, double* out)
{
    if (n < 1 || !(L > 0.0) || !out) return RTLBFS_ERR_ARG;
    // Eq. 74
    for (int i = 0; i <= n; ++i) {
        const double s = (double)i / (double)n;
        out[i] = phi > 0.0 ? (std::tanh(phi) + std::tanh(2.0 * phi * (s - 0.5))) * L /
                                 (2.0 * std::tanh(phi))
                           : s * L;
    }
    return RTLBFS_OK;
}

int rtlbfs_create_mesh(int nx, int ny, const double* xf, const double* yf, int precision,
                       rtlbfs_t* out)
{
    if (!out) return RTLBFS_ERR_ARG;
    *out = nullptr;
    rtlbfs_ctx* h = new (std::nothrow) rtlbfs_ctx;
    if (!h) return RTLBFS_ERR_OOM;
    h->eng = new (std::nothrow) Engine(precision, 1);
    if (!h->eng) {
        delete h;
        return RTLBFS_ERR_OOM;
    }
    int rc = h->eng->init();
    if (rc == RTLBFS_OK) rc = h->eng->add(nx, ny, xf, yf, &h->slot);
    if (rc == RTLBFS_OK) rc = h->eng->set_conduction_state(h->slot);
    if (rc != RTLBFS_OK) {
        delete h->eng;
        delete h;
        return rc;
    }
    *out = h;
    return RTLBFS_OK;
}

int rtlbfs_create_strip(int nx, int ny_mesh, const double* xf, const double* yf, int j0, int j1,
                        int precision, rtlbfs_t* out)
{
    if (!out) return RTLBFS_ERR_ARG;
    *out = nullptr;
    rtlbfs_ctx* h = new (std::nothrow) rtlbfs_ctx;
    if (!h) return RTLBFS_ERR_OOM;
    h->eng = new (std::nothrow) Engine(precision, 1);
    if (!h->eng) {
        delete h;
        return RTLBFS_ERR_OOM;
    }
    int rc = h->eng->init();
    if (rc == RTLBFS_OK) rc = h->eng->add_strip(nx, ny_mesh, xf, yf, j0, j1, &h->slot);
    if (rc == RTLBFS_OK) rc = h->eng->set_conduction_state(h->slot);
    if (rc != RTLBFS_OK) {
        delete h->eng;
        delete h;
        return rc;
    }
    *out = h;
    return RTLBFS_OK;
}

int rtlbfs_strip_get_rows(rtlbfs_t h, int side, double* rows)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->get_rows(h->slot, side, 0, rows));
}

int rtlbfs_strip_set_halo(rtlbfs_t h, int side, const double* rows)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->set_rows(h->slot, side, 1, rows));
}

int rtlbfs_strip_rows(rtlbfs_t h, int side, int halo, int buffer, void** dev, size_t* bytes)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->strip_rows(h->slot, side, halo ? 1 : 0, buffer, dev, bytes));
}

int rtlbfs_residual_sums(rtlbfs_t h, double* sums, long* steps)
{
    if (!cav(h) || !sums) return RTLBFS_ERR_ARG;
    CavityCtl ctl;
    int rc = h->eng->read_ctl(h->slot, &ctl);
    if (rc) return finish(h, rc);
    for (int q = 0; q < 4; ++q) sums[q] = ctl.sums[q];
    if (steps) *steps = (long)ctl.steps;
    return RTLBFS_OK;
}

int rtlbfs_strip_pack(rtlbfs_t h, int side, int buffer, void* dev)
{
    if (!cav(h) || !dev) return RTLBFS_ERR_ARG;
    void* p = nullptr;
    size_t n = 0;
    int rc = h->eng->strip_rows(h->slot, side, 0, buffer, &p, &n);
    if (rc) return finish(h, rc);
    cudaError_t e = cudaMemcpyAsync(dev, p, n, cudaMemcpyDeviceToDevice, h->eng->stream());
    return e == cudaSuccess ? RTLBFS_OK : finish(h, h->eng->cuda_fail(e, "rtlbfs_strip_pack"));
}

int rtlbfs_strip_unpack(rtlbfs_t h, int side, int buffer, const void* dev)
{
    if (!cav(h) || !dev) return RTLBFS_ERR_ARG;
    void* p = nullptr;
    size_t n = 0;
    int rc = h->eng->strip_rows(h->slot, side, 1, buffer, &p, &n);
    if (rc) return finish(h, rc);
    cudaError_t e = cudaMemcpyAsync(p, dev, n, cudaMemcpyDeviceToDevice, h->eng->stream());
    return e == cudaSuccess ? RTLBFS_OK : finish(h, h->eng->cuda_fail(e, "rtlbfs_strip_unpack"));
}

int rtlbfs_current_buffer(rtlbfs_t h, int* buffer)
{
    if (!cav(h) || !buffer) return RTLBFS_ERR_ARG;
    CavityCtl ctl;
    int rc = h->eng->read_ctl(h->slot, &ctl);
    if (rc) return finish(h, rc);
    *buffer = ctl.cur & 1;
    return RTLBFS_OK;
}

int rtlbfs_set_params(rtlbfs_t h, double Ra, double Pr, double Ma, double dt)
{
    Cavity* c = cav(h);
    if (!c) return RTLBFS_ERR_ARG;
    if (!(Ra > 0 && Pr > 0 && Ma > 0) || !(dt >= 0)) return argfail(h, "Ra, Pr, Ma must be > 0, dt >= 0");
    c->from_ra = true;
    c->Ra = Ra;
    c->Pr = Pr;
    c->Ma = Ma;
    c->dt_auto = !(dt > 0);
    if (dt > 0) c->dt = dt;
    h->eng->touch(h->slot);
    return RTLBFS_OK;
}

int rtlbfs_set_params_ref(rtlbfs_t h, double Ra, double Pr, double Ma, double dt, double L,
                          double dT, double T_ref)
{
    Cavity* c = cav(h);
    if (!c) return RTLBFS_ERR_ARG;
    if (!(Ra > 0 && Pr > 0 && Ma > 0 && L > 0 && dT > 0) || !(dt >= 0))
        return argfail(h, "Ra, Pr, Ma, L, dT must be > 0, dt >= 0");
    c->from_ra = true;
    c->Ra = Ra;
    c->Pr = Pr;
    c->Ma = Ma;
    c->dt_auto = !(dt > 0);
    if (dt > 0) c->dt = dt;
    c->Lref = L;
    c->dT = dT;
    c->T_ref = T_ref;
    h->eng->touch(h->slot);
    return RTLBFS_OK;
}

int rtlbfs_set_lattice(rtlbfs_t h, double kappa)
{
    Cavity* c = cav(h);
    if (!c) return RTLBFS_ERR_ARG;
    if (!(kappa > 0)) return argfail(h, "kappa must be > 0");
    c->kappa = kappa;
    h->eng->touch(h->slot);
    return RTLBFS_OK;
}

int rtlbfs_set_bc(rtlbfs_t h, int side, int kind, double T_wall, double u_wall)
{
    Cavity* c = cav(h);
    if (!c) return RTLBFS_ERR_ARG;
    if (side < 0 || side > 3) return argfail(h, "side must be 0..3");
    if (kind < 0 || kind > 2) return argfail(h, "kind must be 0..2");
    if (c->kind[side] == rtlbfs::kHalo) return argfail(h, "that side of the strip is a halo side");
    c->kind[side] = kind;
    c->bcT[side] = T_wall;
    c->bcU[side] = u_wall;
    h->eng->touch(h->slot);
    return RTLBFS_OK;
}

int rtlbfs_set_body_force(rtlbfs_t h, double fx, double fy)
{
    Cavity* c = cav(h);
    if (!c) return RTLBFS_ERR_ARG;
    c->fx = fx;
    c->fy = fy;
    h->eng->touch(h->slot);
    return RTLBFS_OK;
}

int rtlbfs_set_physics(rtlbfs_t h, double nu, double chi, double beta_g)
{
    Cavity* c = cav(h);
    if (!c) return RTLBFS_ERR_ARG;
    if (!(nu > 0 && chi > 0)) return argfail(h, "nu and chi must be > 0");
    c->from_ra = false;
    c->nu = nu;
    c->chi = chi;
    c->beta_g = beta_g;
    h->eng->touch(h->slot);
    return RTLBFS_OK;
}

int rtlbfs_set_state(rtlbfs_t h, const double* rho, const double* u, const double* v,
                     const double* T)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->set_state(h->slot, rho, u, v, T));
}

int rtlbfs_get_state(rtlbfs_t h, double* rho, double* u, double* v, double* T)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->get_state(h->slot, rho, u, v, T));
}

size_t rtlbfs_state_raw_bytes(rtlbfs_t h)
{
    Cavity* c = cav(h);
    return c ? h->eng->record_bytes() * (size_t)c->nx * c->ny : 0;
}

int rtlbfs_get_state_raw(rtlbfs_t h, void* records, double* T_unit)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->get_records(h->slot, records, T_unit));
}

int rtlbfs_set_state_raw(rtlbfs_t h, const void* records, double T_unit)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->set_records(h->slot, records, T_unit));
}

int rtlbfs_step(rtlbfs_t h, long nsteps)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    if (nsteps < 0) return argfail(h, "nsteps must be >= 0");
    if (nsteps == 0) return RTLBFS_OK;
    int rc = h->eng->arm(h->slot, nsteps, -1.0);
    if (rc == RTLBFS_OK) rc = h->eng->launch_steps(nsteps);
    CavityCtl ctl;
    if (rc == RTLBFS_OK) rc = h->eng->read_ctl(h->slot, &ctl);
    if (rc != RTLBFS_OK) return finish(h, rc);
    if (ctl.status == rtlbfs::kDiverged) {
        h->err = "residual became non-finite";
        return RTLBFS_ERR_DIVERGED;
    }
    return RTLBFS_OK;
}

int rtlbfs_run_to_steady(rtlbfs_t h, double tol, long max_steps, double timeout_s,
                         long* steps_taken, double* residual)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    if (!(tol > 0) || max_steps < 0) return argfail(h, "tol must be > 0, max_steps >= 0");
    CavityCtl ctl;
    int rc = h->eng->read_ctl(h->slot, &ctl);
    if (rc) return finish(h, rc);
    const long long start = ctl.steps;
    rc = h->eng->arm(h->slot, max_steps, tol);
    if (rc) return finish(h, rc);
    const auto t0 = std::chrono::steady_clock::now();
    long long launched = 0;
    long long chunk = 256;
    int out = RTLBFS_ERR_NOT_CONVERGED;
    while (true) {
        const long long n = std::min<long long>(chunk, (long long)max_steps - launched);
        if (n > 0) {
            rc = h->eng->launch_steps(n);
            if (rc) return finish(h, rc);
            launched += n;
        }
        rc = h->eng->read_ctl(h->slot, &ctl);
        if (rc) return finish(h, rc);
        if (ctl.done || launched >= max_steps) {
            out = ctl.done ? status_to_rc(ctl.status) : RTLBFS_ERR_NOT_CONVERGED;
            if (max_steps == 0) out = RTLBFS_ERR_NOT_CONVERGED;
            break;
        }
        if (timeout_s > 0) {
            const double el =
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > timeout_s) {
                // stop the slot where it is
                h->eng->arm(h->slot, 0, -1.0);
                h->eng->read_ctl(h->slot, &ctl);
                out = RTLBFS_ERR_TIMEOUT;
                break;
            }
        }
        if (chunk < 4096) chunk *= 2;
    }
    if (steps_taken) *steps_taken = (long)(ctl.steps - start);
    if (residual) {
        residual[0] = ctl.res[0];
        residual[1] = ctl.res[1];
    }
    if (out == RTLBFS_ERR_DIVERGED) h->err = "residual became non-finite";
    if (out == RTLBFS_ERR_NOT_CONVERGED) h->err = "max_steps reached before tol";
    if (out == RTLBFS_ERR_TIMEOUT) h->err = "timeout";
    return out;
}

int rtlbfs_residual(rtlbfs_t h, double* res2, long* steps)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    CavityCtl ctl;
    int rc = h->eng->read_ctl(h->slot, &ctl);
    if (rc) return finish(h, rc);
    if (res2) {
        res2[0] = ctl.res[0];
        res2[1] = ctl.res[1];
    }
    if (steps) *steps = (long)ctl.steps;
    return RTLBFS_OK;
}

int rtlbfs_nusselt(rtlbfs_t h, int which, double* nu)
{
    if (!cav(h) || !nu) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->nusselt(h->slot, which, nu));
}

int rtlbfs_set_scheme(rtlbfs_t h, int scheme)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->set_scheme(scheme));
}

int rtlbfs_set_schedule(rtlbfs_t h, int kernel, int chunk_rows)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    int rc = h->eng->set_kernel(kernel);
    if (rc == RTLBFS_OK) rc = h->eng->set_chunk_rows(chunk_rows);
    return finish(h, rc);
}

int rtlbfs_debug_withhold_tile(rtlbfs_t h, int tile)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    if (tile < -1) return argfail(h, "tile must be >= -1");
    h->eng->set_withhold(tile);
    return RTLBFS_OK;
}

int rtlbfs_autotune(rtlbfs_t h, int steps, int* kernel, int* chunk_rows, double* ms_per_step)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->autotune(steps, kernel, chunk_rows, ms_per_step));
}

int rtlbfs_set_stream(rtlbfs_t h, void* stream)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->set_stream(static_cast<cudaStream_t>(stream)));
}

int rtlbfs_sync(rtlbfs_t h)
{
    if (!cav(h)) return RTLBFS_ERR_ARG;
    return finish(h, h->eng->sync());
}

const char* rtlbfs_last_error(rtlbfs_t h)
{
    if (!h) return "null handle";
    return h->err.c_str();
}

void rtlbfs_destroy(rtlbfs_t h)
{
    if (!h) return;
    delete h->eng;
    delete h;
}

long long rtlbfs_launch_count(void) { return rtlbfs::g_launches.load(); }

}  // extern "C"
