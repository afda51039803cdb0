// rtlbfs_batch.cu -- the batch C ABI (include/rtlbfs_batch.h) over the
// shared engine, and the continuous-batching request loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "rtlbfs.h"
#include "rtlbfs_batch.h"
#include "rtlbfs_engine.h"

using rtlbfs::Cavity;
using rtlbfs::CavityCtl;
using rtlbfs::Engine;

struct rtlbfs_batch_ctx {
    Engine* eng = nullptr;
    std::string err;
};

namespace {

int bfinish(rtlbfs_batch_t b, int rc)
{
    if (rc != RTLBFS_OK && b && b->eng) b->err = b->eng->error();
    return rc;
}

int slot_status(const CavityCtl& c)
{
    if (!c.done) return RTLBFS_SLOT_RUNNING;
    switch (c.status) {
    case rtlbfs::kConverged: return RTLBFS_SLOT_CONVERGED;
    case rtlbfs::kMaxSteps: return RTLBFS_SLOT_MAX_STEPS;
    case rtlbfs::kDiverged: return RTLBFS_SLOT_DIVERGED;
    default: return RTLBFS_SLOT_MAX_STEPS;  // idle: armed for 0 steps
    }
}

}  // namespace

extern "C" {

int rtlbfs_batch_create(int precision, int max_slots, rtlbfs_batch_t* out)
{
    if (!out || max_slots < 1) return RTLBFS_ERR_ARG;
    *out = nullptr;
    rtlbfs_batch_ctx* b = new (std::nothrow) rtlbfs_batch_ctx;
    if (!b) return RTLBFS_ERR_OOM;
    b->eng = new (std::nothrow) Engine(precision, max_slots);
    if (!b->eng) {
        delete b;
        return RTLBFS_ERR_OOM;
    }
    int rc = b->eng->init();
    if (rc) {
        delete b->eng;
        delete b;
        return rc;
    }
    *out = b;
    return RTLBFS_OK;
}

size_t rtlbfs_batch_bytes(int precision, int nx, int ny)
{
    if (nx < 1 || ny < 1) return 0;
    return Engine::bytes_for(precision, nx, ny);
}

int rtlbfs_batch_free_bytes(size_t* free_bytes, size_t* total_bytes)
{
    size_t f = 0, t = 0;
    if (cudaMemGetInfo(&f, &t) != cudaSuccess) return RTLBFS_ERR_CUDA;
    if (free_bytes) *free_bytes = f;
    if (total_bytes) *total_bytes = t;
    return RTLBFS_OK;
}

int rtlbfs_batch_add(rtlbfs_batch_t b, int nx, int ny, const double* xf, const double* yf,
                     double Ra, double Pr, double Ma, double dt, int* slot)
{
    if (!b || !slot) return RTLBFS_ERR_ARG;
    if (!(Ra > 0 && Pr > 0 && Ma > 0) || !(dt >= 0)) {
        b->err = "Ra, Pr, Ma must be > 0, dt >= 0";
        return RTLBFS_ERR_ARG;
    }
    int s = -1;
    int rc = b->eng->add(nx, ny, xf, yf, &s);
    if (rc) return bfinish(b, rc);
    Cavity* c = b->eng->cavity(s);
    c->from_ra = true;
    c->Ra = Ra;
    c->Pr = Pr;
    c->Ma = Ma;
    c->dt_auto = !(dt > 0);
    if (dt > 0) c->dt = dt;
    b->eng->touch(s);
    rc = b->eng->set_conduction_state(s);
    if (rc) {
        b->eng->remove(s);
        return bfinish(b, rc);
    }
    *slot = s;
    return RTLBFS_OK;
}

int rtlbfs_batch_set_bc(rtlbfs_batch_t b, int slot, int side, int kind, double T_wall,
                        double u_wall)
{
    if (!b) return RTLBFS_ERR_ARG;
    Cavity* c = b->eng->cavity(slot);
    if (!c || side < 0 || side > 3 || kind < 0 || kind > 2) return RTLBFS_ERR_ARG;
    c->kind[side] = kind;
    c->bcT[side] = T_wall;
    c->bcU[side] = u_wall;
    b->eng->touch(slot);
    return RTLBFS_OK;
}

int rtlbfs_batch_set_lattice(rtlbfs_batch_t b, int slot, double kappa)
{
    if (!b) return RTLBFS_ERR_ARG;
    Cavity* c = b->eng->cavity(slot);
    if (!c || !(kappa > 0)) return RTLBFS_ERR_ARG;
    c->kappa = kappa;
    b->eng->touch(slot);
    return RTLBFS_OK;
}

int rtlbfs_batch_set_state(rtlbfs_batch_t b, int slot, const double* rho, const double* u,
                           const double* v, const double* T)
{
    if (!b) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->set_state(slot, rho, u, v, T));
}

int rtlbfs_batch_get_state(rtlbfs_batch_t b, int slot, double* rho, double* u, double* v,
                           double* T)
{
    if (!b) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->get_state(slot, rho, u, v, T));
}

size_t rtlbfs_batch_state_raw_bytes(rtlbfs_batch_t b, int slot)
{
    if (!b) return 0;
    const rtlbfs::Cavity* c = b->eng->cavity(slot);  // null for a bad slot
    return c ? b->eng->record_bytes() * (size_t)c->nx * (size_t)c->ny : 0;
}

int rtlbfs_batch_get_state_raw(rtlbfs_batch_t b, int slot, void* records, double* T_unit)
{
    if (!b) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->get_records(slot, records, T_unit));
}

int rtlbfs_batch_set_state_raw(rtlbfs_batch_t b, int slot, const void* records, double T_unit)
{
    if (!b) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->set_records(slot, records, T_unit));
}

int rtlbfs_batch_get_states_raw(rtlbfs_batch_t b, int n, const int* slots, void* const* records,
                                double* T_units)
{
    if (!b) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->get_records_many(n, slots, records, T_units));
}

int rtlbfs_batch_set_states_raw(rtlbfs_batch_t b, int n, const int* slots,
                                const void* const* records, const double* T_units)
{
    if (!b) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->set_records_many(n, slots, records, T_units));
}

int rtlbfs_batch_arm(rtlbfs_batch_t b, int slot, double tol, long max_steps)
{
    if (!b || max_steps < 0) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->arm(slot, max_steps, tol > 0 ? tol : -1.0));
}

int rtlbfs_batch_arm_many(rtlbfs_batch_t b, int n, const int* slots, double tol, long max_steps)
{
    if (!b) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->arm_many(n, slots, max_steps, tol > 0 ? tol : -1.0));
}

int rtlbfs_batch_step(rtlbfs_batch_t b, long nsteps)
{
    if (!b || nsteps < 0) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->launch_steps(nsteps));
}

int rtlbfs_batch_poll(rtlbfs_batch_t b, int* status, long* steps, double* res2)
{
    if (!b) return RTLBFS_ERR_ARG;
    std::vector<CavityCtl> c;
    int rc = b->eng->read_ctls(c);
    if (rc) return bfinish(b, rc);
    for (int s = 0; s < b->eng->capacity(); ++s) {
        const bool act = b->eng->cavity(s) != nullptr;
        if (status) status[s] = act ? slot_status(c[s]) : RTLBFS_SLOT_EMPTY;
        if (steps) steps[s] = act ? (long)c[s].steps : 0;
        if (res2) {
            res2[2 * s] = act ? c[s].res[0] : NAN;
            res2[2 * s + 1] = act ? c[s].res[1] : NAN;
        }
    }
    return RTLBFS_OK;
}

int rtlbfs_batch_nusselt(rtlbfs_batch_t b, int slot, int which, double* nu)
{
    if (!b || !nu) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->nusselt(slot, which, nu));
}

int rtlbfs_batch_remove(rtlbfs_batch_t b, int slot)
{
    if (!b) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->remove(slot));
}

int rtlbfs_batch_set_schedule(rtlbfs_batch_t b, int kernel, int chunk_rows)
{
    if (!b || kernel == 2) return RTLBFS_ERR_ARG;
    int rc = b->eng->set_kernel(kernel);
    if (rc == RTLBFS_OK) rc = b->eng->set_chunk_rows(chunk_rows);
    return bfinish(b, rc);
}

int rtlbfs_batch_autotune(rtlbfs_batch_t b, int steps, int* kernel, int* chunk_rows,
                          double* ms_per_step)
{
    if (!b) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->autotune(steps, kernel, chunk_rows, ms_per_step));
}

int rtlbfs_batch_set_stream(rtlbfs_batch_t b, void* stream)
{
    if (!b) return RTLBFS_ERR_ARG;
    return bfinish(b, b->eng->set_stream(static_cast<cudaStream_t>(stream)));
}

int rtlbfs_batch_info(rtlbfs_batch_t b, long long* active_cells, int* active_slots, int* units)
{
    if (!b) return RTLBFS_ERR_ARG;
    long long cells = 0;
    int slots = 0;
    for (int s = 0; s < b->eng->capacity(); ++s)
        if (Cavity* c = b->eng->cavity(s)) {
            cells += (long long)c->nx * c->ny;
            ++slots;
        }
    if (active_cells) *active_cells = cells;
    if (active_slots) *active_slots = slots;
    if (units) *units = b->eng->active_tiles();
    return RTLBFS_OK;
}

const char* rtlbfs_batch_last_error(rtlbfs_batch_t b) { return b ? b->err.c_str() : "null batch"; }

void rtlbfs_batch_destroy(rtlbfs_batch_t b)
{
    if (!b) return;
    delete b->eng;
    delete b;
}

// ---------------------------------------------------------------------------
// request loop
// ---------------------------------------------------------------------------
int rtlbfs_serve(const rtlbfs_request* reqs, int nreq, const rtlbfs_serve_opts* opts,
                 rtlbfs_result* out, double* elapsed_s)
{
    if (!reqs || nreq < 0 || !opts || !out) return RTLBFS_ERR_ARG;
    if (opts->max_slots < 1 || opts->chunk_steps < 1 || opts->max_steps < 1 || !(opts->Ma > 0) ||
        !(opts->mem_fraction > 0) || opts->mem_fraction > 1.0)
        return RTLBFS_ERR_ARG;
    for (int k = 0; k < nreq; ++k) {
        out[k] = {-1.0, -1.0, 0, -1, NAN, NAN};
        if (reqs[k].n < 1 || !(reqs[k].Ra > 0) || !(reqs[k].Pr > 0)) return RTLBFS_ERR_ARG;
        if (k && reqs[k].t_arrive < reqs[k - 1].t_arrive) return RTLBFS_ERR_ARG;  // arrival order
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return RTLBFS_ERR_CUDA;
    const double budget = opts->mem_fraction * (double)free_b;
    Engine eng(opts->precision, opts->max_slots);
    int rc = eng.init();
    if (rc) return rc;
    std::vector<int> slot_req(opts->max_slots, -1);
    std::vector<size_t> slot_bytes(opts->max_slots, 0);
    double used = 0.0;
    int next = 0, active = 0, finished = 0;
    const auto t0 = std::chrono::steady_clock::now();
    auto now = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    std::vector<double> faces;
    std::vector<CavityCtl> ctl;
    while (finished < nreq) {
        const double t = now();
        if (opts->time_limit_s > 0 && t > opts->time_limit_s) break;
        // admit arrived requests in order while a slot and memory are free
        while (next < nreq && reqs[next].t_arrive <= t && active < opts->max_slots) {
            const rtlbfs_request& q = reqs[next];
            const size_t need = Engine::bytes_for(opts->precision, q.n, q.n);
            if (used + (double)need > budget && active > 0) break;  // wait for memory
            faces.resize(q.n + 1);
            for (int i = 0; i <= q.n; ++i) faces[i] = (double)i;
            int s = -1;
            rc = eng.add(q.n, q.n, faces.data(), faces.data(), &s);
            if (rc == RTLBFS_ERR_OOM && active > 0) break;
            if (rc) return rc;
            Cavity* c = eng.cavity(s);
            c->from_ra = true;
            c->Ra = q.Ra;
            c->Pr = q.Pr;
            c->Ma = opts->Ma;
            c->dt_auto = true;
            eng.touch(s);
            if ((rc = eng.set_conduction_state(s))) return rc;
            if ((rc = eng.arm(s, opts->max_steps, opts->tol > 0 ? opts->tol : -1.0))) return rc;
            slot_req[s] = next;
            slot_bytes[s] = need;
            used += (double)need;
            out[next].t_admit = now();
            ++active;
            ++next;
        }
        if (active == 0) {
            if (next >= nreq) break;
            const double wait = reqs[next].t_arrive - now();
            if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
            continue;
        }
        if ((rc = eng.launch_steps(opts->chunk_steps))) return rc;
        if ((rc = eng.read_ctls(ctl))) return rc;
        rtlbfs::Nvtx retire("rtlbfs: serve retire");
        for (int s = 0; s < opts->max_slots; ++s) {
            const int k = slot_req[s];
            if (k < 0 || !ctl[s].done) continue;
            rtlbfs_result& r = out[k];
            r.steps = (long)ctl[s].steps;
            r.status = slot_status(ctl[s]);
            double nh = NAN, nc = NAN;
            if (r.status != RTLBFS_SLOT_DIVERGED) {
                if ((rc = eng.nusselt(s, rtlbfs::kNuWest, &nh))) return rc;
                if ((rc = eng.nusselt(s, rtlbfs::kNuEast, &nc))) return rc;
            }
            r.nu_hot = nh;
            r.nu_cold = nc;
            if ((rc = eng.remove(s))) return rc;
            r.t_finish = now();
            used -= (double)slot_bytes[s];
            slot_req[s] = -1;
            slot_bytes[s] = 0;
            --active;
            ++finished;
        }
    }
    if (elapsed_s) *elapsed_s = now();
    return RTLBFS_OK;
}

// ---------------------------------------------------------------------------
// stability map
// ---------------------------------------------------------------------------
int rtlbfs_stability_map(int ncase, const int* n, const double* Ra, const double* kappa,
                         const double* dt, double Pr, double Ma, double tol, long max_steps,
                         int precision, int chunk_steps, int* status_out, long* steps_out,
                         double* elapsed_s)
{
    if (ncase < 0 || !n || !Ra || !kappa || !status_out || !steps_out || !(Pr > 0) ||
        !(Ma > 0) || max_steps < 1 || chunk_steps < 1)
        return RTLBFS_ERR_ARG;
    for (int k = 0; k < ncase; ++k) {
        if (n[k] < 1 || !(Ra[k] > 0) || !(kappa[k] > 0) || (dt && !(dt[k] >= 0)))
            return RTLBFS_ERR_ARG;
        status_out[k] = -1;
        steps_out[k] = 0;
    }
    const auto t0 = std::chrono::steady_clock::now();
    if (ncase == 0) {
        if (elapsed_s) *elapsed_s = 0.0;
        return RTLBFS_OK;
    }
    Engine eng(precision, ncase);
    int rc = eng.init();
    if (rc) return rc;
    std::vector<double> faces;
    std::vector<int> slot_of(ncase, -1);
    for (int k = 0; k < ncase; ++k) {
        faces.resize(n[k] + 1);
        for (int i = 0; i <= n[k]; ++i) faces[i] = (double)i;  // unit cells, L = n
        int s = -1;
        if ((rc = eng.add(n[k], n[k], faces.data(), faces.data(), &s))) return rc;
        Cavity* c = eng.cavity(s);
        c->from_ra = true;
        c->Ra = Ra[k];
        c->Pr = Pr;
        c->Ma = Ma;
        c->kappa = kappa[k];
        if (dt && dt[k] > 0) c->dt = dt[k];
        else c->dt_auto = true;
        eng.touch(s);
        if ((rc = eng.set_conduction_state(s))) return rc;
        if ((rc = eng.arm(s, max_steps, tol > 0 ? tol : -1.0))) return rc;
        slot_of[k] = s;
    }
    std::vector<CavityCtl> ctl;
    for (;;) {
        if ((rc = eng.launch_steps(chunk_steps))) return rc;
        if ((rc = eng.read_ctls(ctl))) return rc;
        bool all = true;
        for (int k = 0; k < ncase; ++k) all = all && ctl[slot_of[k]].done;
        if (all) break;
    }
    for (int k = 0; k < ncase; ++k) {
        status_out[k] = slot_status(ctl[slot_of[k]]);
        steps_out[k] = (long)ctl[slot_of[k]].steps;
    }
    if (elapsed_s)
        *elapsed_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return RTLBFS_OK;
}

}  // extern "C"
