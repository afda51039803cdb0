// rtlbfs_engine.cu -- host side of the solver: per-cavity mesh lines, device
// buffers, the tile list of the batched step kernel, CUDA graphs of step
// launches, run control and the FP64 reductions.
#include "rtlbfs_engine.h"
#include "rtlbfs_worklist.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "rtlbfs.h"

namespace rtlbfs {

std::atomic<long long> g_launches{0};

namespace {
constexpr int kGraphChunk = 64;  // step launches per captured graph
constexpr int kPersistChunk = 1 << 16;  // steps per persistent launch
constexpr int kPartialMax = 2048;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Width of cell i in [-2, n+1] of a line with walls or periodic ends
// (ghosts: a wall ghost has its partner's width; a periodic ghost the
// opposite cell's).
double line_width(const std::vector<double>& f, int i, bool periodic)
{
    const int n = (int)f.size() - 1;
    int k = i;
    if (periodic) {
        k = ((i % n) + n) % n;
    } else {
        if (i < 0) k = -1 - i;        // -1 -> 0, -2 -> 1 (beyond the ghost: unused)
        if (i >= n) k = 2 * n - 1 - i; // n -> n-1, n+1 -> n-2
        k = std::min(std::max(k, 0), n - 1);
    }
    return f[k + 1] - f[k];
}

// hw: widths of the cells beyond a halo end ({w(-1), w(-2)} for the low
// end, {w(n), w(n+1)} for the high end), null for a wall or periodic end.
template <typename R>
void build_lines(const Cavity& c, const std::vector<double>& f, bool periodic, double kappa,
                 double nu, double chi, double dt, std::vector<FaceLine<R>>& fl,
                 std::vector<CellLine<R>>& cl, const double* hw_lo = nullptr,
                 const double* hw_hi = nullptr)
{
    const int n = (int)f.size() - 1;
    (void)c;
    auto width = [&](int i) {
        if (i < 0 && i >= -2 && hw_lo) return hw_lo[-1 - i];
        if (i >= n && i <= n + 1 && hw_hi) return hw_hi[i - n];
        return line_width(f, i, periodic);
    };
    fl.resize(n + 1);
    for (int i = 0; i <= n; ++i) {
        const double wl = width(i - 1), wr = width(i);
        const double h = kappa * std::min(wl, wr);
        FaceLine<R> x;
        x.h = (R)h;
        x.cL = (R)(0.5 * wl - h);
        x.cR = (R)(h - 0.5 * wr);
        x.pad = (R)0;
        x.m_nu_2h = (R)(-nu / (2.0 * h));
        x.m_chi_2h = (R)(-chi / (2.0 * h));
        x.m_tf15 = (R)(1.0 - 3.0 * nu / h);
        x.m_tg15 = (R)(1.0 - 3.0 * chi / h);
        fl[i] = x;
    }
    cl.resize(n + 4);
    for (int i = -2; i <= n + 1; ++i) {
        const double w = width(i), wn = width(i + 1);
        CellLine<R> y;
        y.w = (R)w;
        y.is_next = (R)(1.0 / (w + wn));
        y.dt_w = (R)(dt / w);
        y.pad = (R)0;
        cl[i + 2] = y;
    }
}
}  // namespace

Engine::Engine(int precision, int capacity)
    : precision_(precision), capacity_(capacity),
      rsize_(precision == RTLBFS_FP64 ? sizeof(double) : sizeof(float))
{
}

Engine::~Engine()
{
    if (gexec_) cudaGraphExecDestroy(gexec_);
    // the caller's stream may be gone by now: wait for the device, free on
    // the engine's own stream
    cudaDeviceSynchronize();
    for (auto& c : slots_) {
        if (c.d_fields) cudaFreeAsync(c.d_fields, own_stream_);
        if (c.d_lines) cudaFreeAsync(c.d_lines, own_stream_);
    }
    if (own_stream_) cudaStreamSynchronize(own_stream_);
    if (pool_) cudaMemPoolDestroy(pool_);
    cudaFree(d_desc_);
    cudaFree(d_ctl_);
    cudaFree(d_tiles_);
    cudaFree(d_ntiles_);
    cudaFree(d_partial_);
    cudaFree(d_scalar_);
    cudaFree(d_stage_);
    cudaFree(d_slot_list_);
    cudaFree(d_run_list_);
    cudaFree(d_tstep_);
    cudaFree(d_pctl_);
    if (h_stalled_) cudaFreeHost(h_stalled_);
    if (h_scalar_) cudaFreeHost(h_scalar_);
    if (own_stream_) cudaStreamDestroy(own_stream_);
}

int Engine::fail(int code, const std::string& msg)
{
    err_ = msg;
    return code;
}

int Engine::cuda_fail(cudaError_t e, const char* what)
{
    err_ = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RTLBFS_ERR_OOM : RTLBFS_ERR_CUDA;
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

int Engine::init()
{
    if (precision_ != RTLBFS_FP64 && precision_ != RTLBFS_FP32)
        return fail(RTLBFS_ERR_ARG, "precision must be RTLBFS_FP64 or RTLBFS_FP32");
    if (capacity_ < 1) return fail(RTLBFS_ERR_ARG, "capacity must be >= 1");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev));
    CK(step_prepare(precision_));
    for (int h : kTileHeights) {
        if (!tile_height_ok(precision_, h)) continue;
        CK(step_occupancy(precision_, h, kSchemeRTLBFS, &occ_tile_[h]));
        if (occ_tile_[h] < 1) return fail(RTLBFS_ERR_CUDA, "step kernel does not fit on an SM");
    }
    CK(step_occupancy(precision_, kTileYDefault, kSchemeTLBFS, &occ_tlbfs_));
    if (occ_tlbfs_ < 1) return fail(RTLBFS_ERR_CUDA, "TLBFS step kernel does not fit on an SM");
    CK(persist_prepare(precision_));
    for (int h : kTileHeights) {
        if (!tile_height_ok(precision_, h)) continue;
        CK(persist_occupancy(precision_, h, &occ_persist_[h]));
    }
    CK(march_prepare(precision_));
    CK(march_occupancy(precision_, &occ_march_));
    if (occ_march_ < 1) return fail(RTLBFS_ERR_CUDA, "march kernel does not fit on an SM");
    CK(cudaStreamCreateWithFlags(&own_stream_, cudaStreamNonBlocking));
    stream_ = own_stream_;
    // cavities come and go (batches, the request loop): their memory comes
    // from a stream-ordered pool of this engine, which keeps freed blocks
    // for reuse instead of returning them (no device-wide synchronisation)
    {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        CK(cudaMemPoolCreate(&pool_, &props));
        uint64_t keep = ~0ull;
        CK(cudaMemPoolSetAttribute(pool_, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    slots_.resize(capacity_);
    h_desc_.resize(capacity_);
    std::memset(h_desc_.data(), 0, sizeof(CavityDesc) * capacity_);
    CK(cudaMalloc(&d_desc_, sizeof(CavityDesc) * capacity_));
    CK(cudaMalloc(&d_ctl_, sizeof(CavityRun) * capacity_));
    std::vector<CavityRun> c0(capacity_);
    for (auto& r : c0) {
        std::memset(&r, 0, sizeof(r));
        for (auto& c : r.h) {
            c.done = 1;
            c.tol = -1.0;
            c.res[0] = c.res[1] = INFINITY;
        }
    }
    CK(cudaMemcpy(d_ctl_, c0.data(), sizeof(CavityRun) * capacity_, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&d_ntiles_, sizeof(int)));
    CK(cudaMemset(d_ntiles_, 0, sizeof(int)));
    partial_cap_ = kPartialMax;
    CK(cudaMalloc(&d_partial_, sizeof(double) * partial_cap_));
    CK(cudaMalloc(&d_scalar_, sizeof(double) * 8));
    CK(cudaMallocHost(&h_scalar_, sizeof(double) * 8));
    CK(cudaMalloc(&d_pctl_, sizeof(PersistCtl)));
    CK(cudaMallocHost(&h_stalled_, sizeof(int)));
    return RTLBFS_OK;
}

size_t Engine::bytes_for(int precision, int nx, int ny)
{
    const size_t rs = precision == RTLBFS_FP64 ? 8 : 4;
    const size_t pitch = align_up((size_t)nx, 32);
    const size_t fields = 8 * rs * pitch * (size_t)ny;
    const size_t lines = (2 * (nx + ny) + 12) * (sizeof(FaceLine<double>) + sizeof(CellLine<double>)) + 8 * 256;
    return fields + lines;
}

Cavity* Engine::cavity(int slot)
{
    if (slot < 0 || slot >= capacity_ || !slots_[slot].active) return nullptr;
    return &slots_[slot];
}

int Engine::add(int nx, int ny, const double* xf, const double* yf, int* slot_out, int halo_rows)
{
    if (nx < 1 || ny < 1 || !xf || !yf) return fail(RTLBFS_ERR_ARG, "bad mesh size or null faces");
    if ((long long)nx * ny > (1LL << 31)) return fail(RTLBFS_ERR_ARG, "mesh too large");
    for (int i = 0; i < nx; ++i)
        if (!(xf[i + 1] > xf[i])) return fail(RTLBFS_ERR_ARG, "xf must be strictly ascending");
    for (int j = 0; j < ny; ++j)
        if (!(yf[j + 1] > yf[j])) return fail(RTLBFS_ERR_ARG, "yf must be strictly ascending");
    int slot = -1;
    for (int k = 0; k < capacity_; ++k)
        if (!slots_[k].active) {
            slot = k;
            break;
        }
    if (slot < 0) return fail(RTLBFS_ERR_STATE, "no free slot");
    Cavity c;
    c.nx = nx;
    c.ny = ny;
    c.pitch = (int)align_up((size_t)nx, 32);
    c.xf.assign(xf, xf + nx + 1);
    c.yf.assign(yf, yf + ny + 1);
    double wmin = 1e300;
    for (int i = 0; i < nx; ++i) wmin = std::min(wmin, xf[i + 1] - xf[i]);
    for (int j = 0; j < ny; ++j) wmin = std::min(wmin, yf[j + 1] - yf[j]);
    c.dt = 0.5 * wmin;
    c.Lref = 0.0;  // 0: the domain width in x
    c.halo_rows = halo_rows;
    c.fields_bytes = 8 * rsize_ * (size_t)c.pitch * (ny + 2 * halo_rows);
    // line layout: R lines, then FP64 lines, each block 256-byte aligned
    const size_t fr = precision_ == RTLBFS_FP64 ? sizeof(FaceLine<double>) : sizeof(FaceLine<float>);
    const size_t cr = precision_ == RTLBFS_FP64 ? sizeof(CellLine<double>) : sizeof(CellLine<float>);
    size_t off = 0;
    c.off_xl = off; off = align_up(off + fr * (nx + 1), 256);
    c.off_yl = off; off = align_up(off + fr * (ny + 1), 256);
    c.off_xc = off; off = align_up(off + cr * (nx + 4), 256);
    c.off_yc = off; off = align_up(off + cr * (ny + 4), 256);
    c.off_xld = off; off = align_up(off + sizeof(FaceLine<double>) * (nx + 1), 256);
    c.off_yld = off; off = align_up(off + sizeof(FaceLine<double>) * (ny + 1), 256);
    c.off_xcd = off; off = align_up(off + sizeof(CellLine<double>) * (nx + 4), 256);
    c.off_ycd = off; off = align_up(off + sizeof(CellLine<double>) * (ny + 4), 256);
    c.lines_bytes = off;
    cudaError_t e = cudaMallocFromPoolAsync(&c.d_fields, c.fields_bytes, pool_, stream_);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocFromPoolAsync(fields)");
    e = cudaMallocFromPoolAsync(&c.d_lines, c.lines_bytes, pool_, stream_);
    if (e != cudaSuccess) {
        cudaFreeAsync(c.d_fields, stream_);
        return cuda_fail(e, "cudaMallocFromPoolAsync(lines)");
    }
    e = cudaMemsetAsync(c.d_fields, 0, c.fields_bytes, stream_);
    if (e != cudaSuccess) {
        cudaFreeAsync(c.d_fields, stream_);
        cudaFreeAsync(c.d_lines, stream_);
        return cuda_fail(e, "cudaMemset(fields)");
    }
    c.active = true;
    c.dirty = true;
    slots_[slot] = std::move(c);
    tiles_dirty_ = true;
    // reset the slot's run control: nothing to do until armed
    CavityCtl z;
    std::memset(&z, 0, sizeof(z));
    z.done = 1;
    z.tol = -1.0;
    z.res[0] = z.res[1] = INFINITY;
    int rc = put_run(slot, z);
    if (rc) return rc;
    *slot_out = slot;
    return RTLBFS_OK;
}

int Engine::put_run(int slot, const CavityCtl& c)
{
    CavityRun r;
    std::memset(&r, 0, sizeof(r));
    r.h[0] = c;
    r.h[1] = c;
    // from pageable memory: staged before the call returns, ordered on the stream
    CK(cudaMemcpyAsync(&d_ctl_[slot], &r, sizeof(r), cudaMemcpyHostToDevice, stream_));
    return RTLBFS_OK;
}

int Engine::remove(int slot)
{
    Cavity* c = cavity(slot);
    if (!c) return fail(RTLBFS_ERR_ARG, "no such slot");
    // stream-ordered: released after the work already queued on the stream
    CK(cudaFreeAsync(c->d_fields, stream_));
    CK(cudaFreeAsync(c->d_lines, stream_));
    slots_[slot] = Cavity();
    tiles_dirty_ = true;
    return RTLBFS_OK;
}

void Engine::touch(int slot)
{
    if (Cavity* c = cavity(slot)) c->dirty = true;
}

int Engine::resolve_params(Cavity& c)
{
    const double L = c.Lref > 0.0 ? c.Lref : (c.xf.back() - c.xf.front());
    if (c.from_ra) {
        if (!(c.Ra > 0 && c.Pr > 0 && c.Ma > 0 && c.dT > 0))
            return fail(RTLBFS_ERR_ARG, "Ra, Pr, Ma and dT must be positive");
        const double Vc = c.Ma;  // V_c = Ma * c with c = 1
        c.nu = Vc * L * std::sqrt(c.Pr / c.Ra);
        c.chi = c.nu / c.Pr;
        c.beta_g = Vc * Vc / (c.dT * L);
    }
    if (!(c.nu > 0 && c.chi > 0)) return fail(RTLBFS_ERR_ARG, "nu and chi must be positive");
    if (c.dt_auto) {
        // explicit step limits: acoustic dt <= 0.5 w_min (c = 1), diffusive
        // dt <= 0.2 w_min^2 / max(nu, chi) -- about half the largest stable
        // step of the scheme measured on uniform meshes
        double wmin = 1e300;
        for (int i = 0; i < c.nx; ++i) wmin = std::min(wmin, c.xf[i + 1] - c.xf[i]);
        for (int j = 0; j < c.ny; ++j) wmin = std::min(wmin, c.yf[j + 1] - c.yf[j]);
        if (c.wmin_mesh > 0.0) wmin = c.wmin_mesh;  // a strip: the whole mesh's rule
        c.dt = std::min(0.5 * wmin, 0.2 * wmin * wmin / std::max(c.nu, c.chi));
    }
    if (!(c.dt > 0) || !(c.kappa > 0)) return fail(RTLBFS_ERR_ARG, "dt and kappa must be positive");
    const bool xp = c.kind[kSideW] == kPeriodic, xp2 = c.kind[kSideE] == kPeriodic;
    const bool yp = c.kind[kSideS] == kPeriodic, yp2 = c.kind[kSideN] == kPeriodic;
    if (xp != xp2 || yp != yp2)
        return fail(RTLBFS_ERR_ARG, "periodic sides must come in opposite pairs");
    if (c.kind[kSideW] == kHalo || c.kind[kSideE] == kHalo)
        return fail(RTLBFS_ERR_ARG, "halo sides are south or north sides of a row strip");
    if ((c.kind[kSideS] == kHalo || c.kind[kSideN] == kHalo) && c.halo_rows < 2)
        return fail(RTLBFS_ERR_ARG, "halo sides need a row strip (rtlbfs_create_strip)");
    return RTLBFS_OK;
}

int Engine::add_strip(int nx, int ny_mesh, const double* xf, const double* yf, int j0, int j1,
                      int* slot_out)
{
    if (!xf || !yf || nx < 1 || ny_mesh < 2 || j0 < 0 || j1 > ny_mesh || j1 - j0 < 2)
        return fail(RTLBFS_ERR_ARG, "a strip needs 0 <= j0, j1 <= ny, at least 2 rows");
    for (int j = 0; j < ny_mesh; ++j)
        if (!(yf[j + 1] > yf[j])) return fail(RTLBFS_ERR_ARG, "yf must be strictly ascending");
    int slot = -1;
    int rc = add(nx, j1 - j0, xf, yf + j0, &slot, 2);
    if (rc) return rc;
    Cavity& c = slots_[slot];
    auto w = [&](int j) { return yf[j + 1] - yf[j]; };
    if (j0 > 0) {  // rows j0 - 1, j0 - 2 of the mesh lie beyond the south side
        c.kind[kSideS] = kHalo;
        c.halo_w[0][0] = w(j0 - 1);
        c.halo_w[0][1] = j0 >= 2 ? w(j0 - 2) : w(j0 - 1);
    }
    if (j1 < ny_mesh) {  // rows j1, j1 + 1 beyond the north side
        c.kind[kSideN] = kHalo;
        c.halo_w[1][0] = w(j1);
        c.halo_w[1][1] = j1 + 1 < ny_mesh ? w(j1 + 1) : w(j1);
    }
    double wmin = 1e300;
    for (int i = 0; i < nx; ++i) wmin = std::min(wmin, xf[i + 1] - xf[i]);
    for (int j = 0; j < ny_mesh; ++j) wmin = std::min(wmin, w(j));
    c.wmin_mesh = wmin;
    c.dt = 0.5 * wmin;
    c.dirty = true;
    *slot_out = slot;
    return RTLBFS_OK;
}

int Engine::strip_rows(int slot, int side, int ghost, int buffer, void** ptr, size_t* bytes)
{
    Cavity* c = cavity(slot);
    if (!c) return fail(RTLBFS_ERR_ARG, "no such slot");
    if ((side != kSideS && side != kSideN) || buffer < 0 || buffer > 1 || !ptr || !bytes)
        return fail(RTLBFS_ERR_ARG, "side must be south or north, buffer 0 or 1");
    if (c->kind[side] != kHalo) return fail(RTLBFS_ERR_ARG, "that side is not a halo side");
    if (c->dirty) {
        int rc = upload_lines(slot);
        if (rc) return rc;
    }
    // first row of the pair: own rows 0, 1 / ny-2, ny-1; halo rows -2, -1 / ny, ny+1
    const int r = side == kSideS ? (ghost ? -2 : 0) : (ghost ? c->ny : c->ny - 2);
    const size_t row = 4 * rsize_ * (size_t)c->pitch;
    *ptr = static_cast<unsigned char*>(h_desc_[slot].f[buffer][0]) + (long long)r * (long long)row;
    *bytes = 2 * row;
    return RTLBFS_OK;
}

int Engine::get_rows(int slot, int side, int ghost, double* host)
{
    Nvtx range("rtlbfs: strip rows out");
    Cavity* c = cavity(slot);
    if (!c || !host) return fail(RTLBFS_ERR_ARG, "no such slot or null array");
    CavityCtl ctl;
    int rc = read_ctl(slot, &ctl);
    if (rc) return rc;
    void* p = nullptr;
    size_t bytes = 0;
    if ((rc = strip_rows(slot, side, ghost, ctl.cur & 1, &p, &bytes))) return rc;
    const size_t n = 2 * (size_t)c->nx;
    if (stage_cap_ < 4 * n) {
        cudaFree(d_stage_);
        d_stage_ = nullptr;
        CK(cudaMalloc(&d_stage_, sizeof(double) * 4 * n));
        stage_cap_ = 4 * n;
    }
    CK(launch_state_out(precision_, stream_, d_stage_, c->nx, 2, c->pitch, c->T_unit, p));
    g_launches++;
    double* dst[4] = {host, host + n, host + 2 * n, host + 3 * n};
    for (int k = 0; k < 4; ++k)
        CK(cudaMemcpyAsync(dst[k], d_stage_ + k * n, sizeof(double) * n, cudaMemcpyDeviceToHost,
                           stream_));
    CK(cudaStreamSynchronize(stream_));
    return RTLBFS_OK;
}

int Engine::set_rows(int slot, int side, int ghost, const double* host)
{
    Nvtx range("rtlbfs: strip halo in");
    Cavity* c = cavity(slot);
    if (!c || !host) return fail(RTLBFS_ERR_ARG, "no such slot or null array");
    CavityCtl ctl;
    int rc = read_ctl(slot, &ctl);
    if (rc) return rc;
    void* p = nullptr;
    size_t bytes = 0;
    if ((rc = strip_rows(slot, side, ghost, ctl.cur & 1, &p, &bytes))) return rc;
    const size_t n = 2 * (size_t)c->nx;
    if (stage_cap_ < 4 * n) {
        CK(cudaStreamSynchronize(stream_));
        cudaFree(d_stage_);
        d_stage_ = nullptr;
        CK(cudaMalloc(&d_stage_, sizeof(double) * 4 * n));
        stage_cap_ = 4 * n;
    }
    for (int k = 0; k < 4; ++k)
        CK(cudaMemcpyAsync(d_stage_ + k * n, host + k * n, sizeof(double) * n,
                           cudaMemcpyHostToDevice, stream_));
    int* d_bad = reinterpret_cast<int*>(d_scalar_ + 7);
    CK(cudaMemsetAsync(d_bad, 0, sizeof(int), stream_));
    CK(launch_state_in(precision_, stream_, d_stage_, c->nx, 2, c->pitch, c->T_unit, p, d_bad));
    g_launches++;
    int h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    if (h_bad)
        return fail(RTLBFS_ERR_ARG, "halo rows not representable in the FP32 fixed-point state");
    return RTLBFS_OK;
}

double Engine::temp_unit(const Cavity& c) const
{
    if (precision_ != RTLBFS_FP32) return 1.0;
    double m = std::max(std::fabs(c.T_ref - 0.5 * c.dT), std::fabs(c.T_ref + 0.5 * c.dT));
    for (int s = 0; s < 4; ++s)
        if (c.kind[s] == kDirichlet) m = std::max(m, std::fabs(c.bcT[s]));
    double u = 1.0;
    while ((m > 1.5 * u || c.state_Tmax > 1.9 * u) && u < 1e300) u *= 2.0;
    return u;
}

int Engine::upload_lines(int slot)
{
    Cavity& c = slots_[slot];
    int rc = resolve_params(c);
    if (rc) return rc;
    // a configuration that needs a larger temperature unit: the stored
    // temperatures of both buffers follow it (rounded to the new unit); the
    // unit never shrinks under a live state
    const double unit = temp_unit(c);
    if (unit > c.T_unit) {
        const int shift = (int)std::lround(std::log2(unit / c.T_unit));
        if (shift > 30) return fail(RTLBFS_ERR_ARG, "temperatures too large for the FP32 state");
        CK(launch_rescale_T(stream_, c.d_fields, 2LL * c.pitch * (c.ny + 2 * c.halo_rows), shift));
        g_launches++;
        c.T_unit = unit;
    }
    const double Tu = c.T_unit;
    const bool xp = c.kind[kSideW] == kPeriodic, yp = c.kind[kSideS] == kPeriodic;
    const double* hw_lo = c.kind[kSideS] == kHalo ? c.halo_w[0] : nullptr;
    const double* hw_hi = c.kind[kSideN] == kHalo ? c.halo_w[1] : nullptr;
    std::vector<unsigned char> buf(c.lines_bytes, 0);
    auto put = [&](size_t off, const void* src, size_t n) { std::memcpy(buf.data() + off, src, n); };
    {
        std::vector<FaceLine<double>> fx, fy;
        std::vector<CellLine<double>> cx, cy;
        build_lines<double>(c, c.xf, xp, c.kappa, c.nu, c.chi, c.dt, fx, cx);
        build_lines<double>(c, c.yf, yp, c.kappa, c.nu, c.chi, c.dt, fy, cy, hw_lo, hw_hi);
        put(c.off_xld, fx.data(), fx.size() * sizeof(fx[0]));
        put(c.off_yld, fy.data(), fy.size() * sizeof(fy[0]));
        put(c.off_xcd, cx.data(), cx.size() * sizeof(cx[0]));
        put(c.off_ycd, cy.data(), cy.size() * sizeof(cy[0]));
        if (precision_ == RTLBFS_FP64) {
            put(c.off_xl, fx.data(), fx.size() * sizeof(fx[0]));
            put(c.off_yl, fy.data(), fy.size() * sizeof(fy[0]));
            put(c.off_xc, cx.data(), cx.size() * sizeof(cx[0]));
            put(c.off_yc, cy.data(), cy.size() * sizeof(cy[0]));
        }
    }
    if (precision_ == RTLBFS_FP32) {
        std::vector<FaceLine<float>> fx, fy;
        std::vector<CellLine<float>> cx, cy;
        build_lines<float>(c, c.xf, xp, c.kappa, c.nu, c.chi, c.dt, fx, cx);
        build_lines<float>(c, c.yf, yp, c.kappa, c.nu, c.chi, c.dt, fy, cy, hw_lo, hw_hi);
        put(c.off_xl, fx.data(), fx.size() * sizeof(fx[0]));
        put(c.off_yl, fy.data(), fy.size() * sizeof(fy[0]));
        put(c.off_xc, cx.data(), cx.size() * sizeof(cx[0]));
        put(c.off_yc, cy.data(), cy.size() * sizeof(cy[0]));
    }
    // pageable source: staged before the call returns (buf may go out of
    // scope), copied in stream order after the work already queued
    CK(cudaMemcpyAsync(c.d_lines, buf.data(), c.lines_bytes, cudaMemcpyHostToDevice, stream_));

    CavityDesc& d = h_desc_[slot];
    std::memset(&d, 0, sizeof(d));
    d.nx = c.nx;
    d.ny = c.ny;
    d.pitch = c.pitch;
    // every temperature in the state's unit T_unit (buoyancy per unit of it)
    for (int s = 0; s < 4; ++s) {
        d.kind[s] = c.kind[s];
        d.bcT[s] = c.bcT[s] / Tu;
        d.bcU[s] = c.bcU[s];
    }
    d.tiles_x = (c.nx + kTileX - 1) / kTileX;
    d.tiles_y = (c.ny + tile_h_ - 1) / tile_h_;
    d.scheme = scheme_;
    d.ntiles = c.ntiles;  // work units of this cavity in the current list
    d.tile_begin = c.first_tile;
    d.beta_g = c.beta_g * Tu;
    d.T_ref = c.T_ref / Tu;
    d.fx = c.fx;
    d.fy = c.fy;
    d.dt = c.dt;
    d.dT = c.dT / Tu;
    d.nu = c.nu;
    d.chi = c.chi;
    d.f_beta_g = (float)d.beta_g;
    d.f_T_ref = (float)d.T_ref;
    d.f_fx = (float)c.fx;
    d.f_fy = (float)c.fy;
    d.f_dt = (float)c.dt;
    for (int s2 = 0; s2 < 4; ++s2) {
        d.f_bcU[s2] = (float)c.bcU[s2];
        d.f_bcT[s2] = (float)d.bcT[s2];
    }
    // cell records of one buffer (with a strip's halo rows below and above)
    const size_t rec = 4 * rsize_ * (size_t)c.pitch * (c.ny + 2 * c.halo_rows);
    const size_t row0 = 4 * rsize_ * (size_t)c.pitch * c.halo_rows;
    for (int b = 0; b < 2; ++b) {
        d.f[b][0] = static_cast<unsigned char*>(c.d_fields) + (size_t)b * rec + row0;
        d.f[b][1] = d.f[b][2] = d.f[b][3] = nullptr;
    }
    unsigned char* L = static_cast<unsigned char*>(c.d_lines);
    d.xline = L + c.off_xl;
    d.yline = L + c.off_yl;
    d.xcell = L + c.off_xc;
    d.ycell = L + c.off_yc;
    CK(cudaMemcpyAsync(&d_desc_[slot], &d, sizeof(d), cudaMemcpyHostToDevice, stream_));
    c.dirty = false;
    return RTLBFS_OK;
}

int Engine::set_scheme(int scheme)
{
    if (scheme != kSchemeRTLBFS && scheme != kSchemeTLBFS)
        return fail(RTLBFS_ERR_ARG, "scheme must be RTLBFS (0) or TLBFS (1)");
    if (scheme != scheme_) {
        scheme_ = scheme;
        if (gexec_) {
            cudaGraphExecDestroy(gexec_);
            gexec_ = nullptr;
        }
        tiles_dirty_ = true;
        for (auto& c : slots_)
            if (c.active) c.dirty = true;  // the scheme lives in the descriptor
    }
    if (scheme_ == kSchemeTLBFS) {  // tile kernel, default height
        kernel_ = 1;
        chunk_rows_ = kTileYDefault;
    }
    return RTLBFS_OK;
}

int Engine::set_kernel(int kind)
{
    if (kind < 0 || kind > 2) return fail(RTLBFS_ERR_ARG, "kernel kind must be 0, 1 or 2");
    if (scheme_ == kSchemeTLBFS && kind != 1)
        return fail(RTLBFS_ERR_ARG, "the TLBFS face stage runs on the tile kernel (1)");
    if (kind != kernel_) {
        kernel_ = kind;
        tiles_dirty_ = true;
        if (gexec_) {
            cudaGraphExecDestroy(gexec_);
            gexec_ = nullptr;
        }
    }
    return RTLBFS_OK;
}

int Engine::set_chunk_rows(int rows)
{
    if (rows < 0) return fail(RTLBFS_ERR_ARG, "chunk rows must be >= 0");
    if (scheme_ == kSchemeTLBFS && kernel_ == 1 && rows != 0 && rows != kTileYDefault)
        return fail(RTLBFS_ERR_ARG, "the TLBFS tile kernel has height 16 (or 0)");
    if (kernel_ >= 1 && rows != 0 && !tile_height_ok(precision_, rows))
        return fail(RTLBFS_ERR_ARG, precision_ == RTLBFS_FP64
                                        ? "FP64 tile height must be one of 16, 8, 4, 2 (or 0)"
                                        : "tile height must be one of 16, 14, 12, 10, 8, 4, 2 (or 0)");
    chunk_rows_ = rows;
    tiles_dirty_ = true;
    return RTLBFS_OK;
}

// Tile height for the current set of cavities: the tiles of one launch run
// about ceil(tiles / SMs) deep on the busiest SM, and a tile of height h
// costs its faces and gradient ring plus a fixed share (loads, barriers,
// the residual), in face-equivalents: 65 h + 32 + 0.25 * 34 (h + 2) + 300.
int Engine::pick_tile_height() const
{
    if (scheme_ == kSchemeTLBFS) return kTileYDefault;
    int best_h = kTileYDefault;
    double best = 1e300;
    for (int h : kTileHeights) {
        if (!tile_height_ok(precision_, h)) continue;
        long long tiles = 0;
        for (int s = 0; s < capacity_; ++s)
            if (slots_[s].active)
                tiles += (long long)((slots_[s].nx + kTileX - 1) / kTileX) *
                         ((slots_[s].ny + h - 1) / h);
        const double deep = (double)((tiles + sms_ - 1) / std::max(sms_, 1));
        const double cost = deep * (65.0 * h + 32.0 + 0.25 * 34.0 * (h + 2) + 300.0);
        if (cost < best * (1.0 - 1e-9)) {
            best = cost;
            best_h = h;
        }
    }
    return best_h;
}

int Engine::rebuild_tiles()
{
    std::vector<int4> t;
    if (kernel_ >= 1) {
        const int h = chunk_rows_ > 0 ? chunk_rows_ : pick_tile_height();
        if (h != tile_h_ && gexec_) {  // the graph baked the other tile kernel
            cudaGraphExecDestroy(gexec_);
            gexec_ = nullptr;
        }
        tile_h_ = h;
        for (int s = 0; s < capacity_; ++s) {
            Cavity& c = slots_[s];
            if (!c.active) continue;
            const int tx = (c.nx + kTileX - 1) / kTileX, ty = (c.ny + tile_h_ - 1) / tile_h_;
            c.first_tile = (int)t.size();
            c.ntiles = tx * ty;
            for (int j = 0; j < ty; ++j)
                for (int i = 0; i < tx; ++i) t.push_back(make_int4(s, i * kTileX, j * tile_h_, 0));
            // Tiles whose halo reaches past the mesh edge take the ghost-resolution
            // path and run longer: spaced evenly through the cavity's part of the
            // list, they are spread over the SMs instead of several landing on one.
            // The persistent kernel finds a tile's neighbours by its index in
            // row-major order: only the launch-per-step kernel takes the spread.
            if (kernel_ == 1) {
                const int nx = c.nx, ny = c.ny, th = tile_h_;
                spread_units(t, (std::size_t)c.first_tile, [=](const int4& u) {
                    return !(u.y >= 2 && u.z >= 2 && u.y + kTileX + 2 <= nx && u.z + th + 2 <= ny);
                });
            }
        }
    } else {
        // warp-marching units: strips of kStrip columns, chunks of H rows.
        // H: long enough to amortise each unit's 2-row prologue, short
        // enough that there are ~8 warps per SM of units to run.
        long long strip_rows = 0;
        for (int s = 0; s < capacity_; ++s)
            if (slots_[s].active)
                strip_rows += (long long)((slots_[s].nx + kStrip - 1) / kStrip) * slots_[s].ny;
        int H = chunk_rows_;
        if (H <= 0) {  // ~16 warps of units per SM, at least 16 rows each
            const long long target = (long long)sms_ * 16;
            H = (int)std::max<long long>(16, (strip_rows + target - 1) / std::max<long long>(target, 1));
            H = std::min(H, 64);
        }
        for (int s = 0; s < capacity_; ++s) {
            Cavity& c = slots_[s];
            if (!c.active) continue;
            const int strips = (c.nx + kStrip - 1) / kStrip;
            const int h = std::min(H, c.ny);
            const int chunks = (c.ny + h - 1) / h;
            c.first_tile = (int)t.size();
            c.ntiles = strips * chunks;
            for (int k = 0; k < chunks; ++k)
                for (int i = 0; i < strips; ++i)
                    t.push_back(make_int4(s, i * kStrip, k * h, std::min(c.ny, (k + 1) * h)));
        }
    }
    // the unit range of every cavity lives in its descriptor
    for (int s = 0; s < capacity_; ++s) {
        const Cavity& c = slots_[s];
        if (!c.active) continue;
        CavityDesc& d = h_desc_[s];
        d.ntiles = c.ntiles;
        d.tile_begin = c.first_tile;
        d.tiles_x = (c.nx + kTileX - 1) / kTileX;
        d.tiles_y = (c.ny + tile_h_ - 1) / tile_h_;
    }
    desc_dirty_ = true;
    if ((int)t.size() > tile_cap_) {
        CK(cudaStreamSynchronize(stream_));
        cudaFree(d_tiles_);
        d_tiles_ = nullptr;
        tile_cap_ = std::max<int>((int)t.size(), 2 * tile_cap_);
        CK(cudaMalloc(&d_tiles_, sizeof(int4) * tile_cap_));
        if (gexec_) {  // the graph baked the old tile pointer
            cudaGraphExecDestroy(gexec_);
            gexec_ = nullptr;
        }
    }
    // pageable sources, staged at the call; in stream order after the
    // launches already queued (which still read the old list)
    if (!t.empty())
        CK(cudaMemcpyAsync(d_tiles_, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice,
                           stream_));
    ntiles_ = (int)t.size();
    CK(cudaMemcpyAsync(d_ntiles_, &ntiles_, sizeof(int), cudaMemcpyHostToDevice, stream_));
    tiles_dirty_ = false;
    return RTLBFS_OK;
}

int Engine::prepare_launch()
{
    if (tiles_dirty_) {
        int rc = rebuild_tiles();
        if (rc) return rc;
    }
    for (int s = 0; s < capacity_; ++s)
        if (slots_[s].active && slots_[s].dirty) {
            int rc = upload_lines(s);
            if (rc) return rc;
        }
    if (desc_dirty_) {  // unit ranges of every cavity: one copy
        CK(cudaMemcpyAsync(d_desc_, h_desc_.data(), sizeof(CavityDesc) * capacity_,
                           cudaMemcpyHostToDevice, stream_));
        desc_dirty_ = false;
    }
    // persistent grid: every SM full, never more blocks than work units
    int want;
    if (kernel_ == 2) {
        int rc = persist_check();
        if (rc) return rc;
        if (ntiles_ > tstep_cap_) {
            CK(cudaStreamSynchronize(stream_));
            cudaFree(d_tstep_);
            d_tstep_ = nullptr;
            CK(cudaMalloc(&d_tstep_, sizeof(int) * ntiles_));
            tstep_cap_ = ntiles_;
        }
        want = ntiles_;
    } else if (kernel_ == 1) {
        const int occ = scheme_ == kSchemeTLBFS ? occ_tlbfs_ : occ_tile_[tile_h_];
        want = std::max(1, std::min(sms_ * occ, std::max(ntiles_, 1)));
    } else {
        const int wpb = kMarchThreads / 32;
        want = std::max(1, std::min(sms_ * occ_march_, (std::max(ntiles_, 1) + wpb - 1) / wpb));
    }
    if (want != grid_ && gexec_) {
        cudaGraphExecDestroy(gexec_);
        gexec_ = nullptr;
    }
    grid_ = want;
    return RTLBFS_OK;
}

int Engine::set_stream(cudaStream_t s)
{
    CK(cudaStreamSynchronize(stream_));
    stream_ = s ? s : own_stream_;
    return RTLBFS_OK;
}

int Engine::sync()
{
    CK(cudaStreamSynchronize(stream_));
    return RTLBFS_OK;
}

int Engine::set_state(int slot, const double* rho, const double* u, const double* v,
                      const double* T)
{
    Nvtx range("rtlbfs: state in");
    Cavity* c = cavity(slot);
    if (!c) return fail(RTLBFS_ERR_ARG, "no such slot");
    if (!rho || !u || !v || !T) return fail(RTLBFS_ERR_ARG, "null state array");
    const size_t n = (size_t)c->nx * c->ny;
    if (precision_ == RTLBFS_FP32) {
        // the new state replaces the old one: pick its temperature unit afresh
        double m = 0.0;
        for (size_t k = 0; k < n; ++k) m = std::max(m, std::fabs(T[k]));  // NaN: caught below
        c->state_Tmax = std::isfinite(m) ? m : 0.0;
        c->T_unit = temp_unit(*c);
        c->dirty = true;
    }
    if (c->dirty) {
        int rc = upload_lines(slot);
        if (rc) return rc;
    }
    if (stage_cap_ < 4 * n) {
        CK(cudaStreamSynchronize(stream_));
        cudaFree(d_stage_);
        d_stage_ = nullptr;
        CK(cudaMalloc(&d_stage_, sizeof(double) * 4 * n));
        stage_cap_ = 4 * n;
    }
    const double* src[4] = {rho, u, v, T};
    for (int k = 0; k < 4; ++k)
        CK(cudaMemcpyAsync(d_stage_ + k * n, src[k], sizeof(double) * n, cudaMemcpyHostToDevice,
                           stream_));
    const CavityDesc& d = h_desc_[slot];
    int* d_bad = reinterpret_cast<int*>(d_scalar_ + 7);
    CK(cudaMemsetAsync(d_bad, 0, sizeof(int), stream_));
    CK(launch_state_in(precision_, stream_, d_stage_, c->nx, c->ny, c->pitch, c->T_unit,
                       d.f[0][0], d_bad));
    g_launches++;
    int h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    CavityCtl z;
    std::memset(&z, 0, sizeof(z));
    z.cur = 0;
    z.done = 1;
    z.tol = -1.0;
    z.res[0] = z.res[1] = INFINITY;
    int rcz = put_run(slot, z);
    if (rcz) return rcz;
    if (h_bad)
        return fail(RTLBFS_ERR_ARG, "state not representable in the FP32 mode's fixed-point "
                                    "storage: NaN, |rho-1| >= 0.49, |u|,|v| >= 0.99 or "
                                    "|T| >= 1.98 T_unit");
    return RTLBFS_OK;
}

int Engine::get_state(int slot, double* rho, double* u, double* v, double* T)
{
    Nvtx range("rtlbfs: state out");
    Cavity* c = cavity(slot);
    if (!c) return fail(RTLBFS_ERR_ARG, "no such slot");
    if (!rho || !u || !v || !T) return fail(RTLBFS_ERR_ARG, "null state array");
    if (c->dirty) {
        int rc = upload_lines(slot);
        if (rc) return rc;
    }
    CavityCtl ctl;
    int rc = read_ctl(slot, &ctl);
    if (rc) return rc;
    const size_t n = (size_t)c->nx * c->ny;
    if (stage_cap_ < 4 * n) {
        cudaFree(d_stage_);
        d_stage_ = nullptr;
        CK(cudaMalloc(&d_stage_, sizeof(double) * 4 * n));
        stage_cap_ = 4 * n;
    }
    const CavityDesc& d = h_desc_[slot];
    CK(launch_state_out(precision_, stream_, d_stage_, c->nx, c->ny, c->pitch, c->T_unit,
                        d.f[ctl.cur & 1][0]));
    g_launches++;
    double* dst[4] = {rho, u, v, T};
    for (int k = 0; k < 4; ++k)
        CK(cudaMemcpyAsync(dst[k], d_stage_ + k * n, sizeof(double) * n, cudaMemcpyDeviceToHost,
                           stream_));
    CK(cudaStreamSynchronize(stream_));
    return RTLBFS_OK;
}

int Engine::get_records(int slot, void* host, double* T_unit)
{
    Nvtx range("rtlbfs: state records out");
    Cavity* c = cavity(slot);
    if (!c || !host) return fail(RTLBFS_ERR_ARG, "no such slot or null array");
    if (c->dirty) {
        int rc = upload_lines(slot);
        if (rc) return rc;
    }
    CavityCtl ctl;
    int rc = read_ctl(slot, &ctl);
    if (rc) return rc;
    const size_t rec = record_bytes();
    CK(cudaMemcpy2DAsync(host, rec * c->nx, h_desc_[slot].f[ctl.cur & 1][0], rec * c->pitch,
                         rec * c->nx, c->ny, cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    if (T_unit) *T_unit = c->T_unit;
    return RTLBFS_OK;
}

int Engine::set_records(int slot, const void* host, double T_unit)
{
    Nvtx range("rtlbfs: state records in");
    int rc = queue_set_records(slot, host, T_unit);
    if (rc) return rc;
    CK(cudaStreamSynchronize(stream_));
    return RTLBFS_OK;
}

int Engine::set_records_many(int n, const int* slots, const void* const* host,
                             const double* T_units)
{
    Nvtx range("rtlbfs: state records in, many");
    if (n < 0 || (n > 0 && (!slots || !host || !T_units)))
        return fail(RTLBFS_ERR_ARG, "null slot, record or unit array");
    for (int k = 0; k < n; ++k) {
        if (!cavity(slots[k]) || !host[k]) return fail(RTLBFS_ERR_ARG, "no such slot or null array");
        int e2 = 0;
        const double m = std::frexp(T_units[k], &e2);
        if (precision_ == RTLBFS_FP64 ? T_units[k] != 1.0 : !(T_units[k] >= 1.0 && m == 0.5))
            return fail(RTLBFS_ERR_ARG, "T_unit must be 1 (FP64) or a power of two >= 1 (FP32)");
    }
    int rc = grow_lists(n);
    if (rc) return rc;
    std::vector<CavityRun> runs(n);
    for (int k = 0; k < n; ++k) {
        rc = queue_set_records(slots[k], host[k], T_units[k], &runs[k]);
        if (rc) return rc;
    }
    // every slot's run record in two copies and one launch
    if (n > 0) {
        CK(cudaMemcpyAsync(d_slot_list_, slots, sizeof(int) * n, cudaMemcpyHostToDevice, stream_));
        CK(cudaMemcpyAsync(d_run_list_, runs.data(), sizeof(CavityRun) * n, cudaMemcpyHostToDevice,
                           stream_));
        CK(launch_put_runs(stream_, d_ctl_, d_slot_list_, d_run_list_, n));
        g_launches++;
    }
    CK(cudaStreamSynchronize(stream_));
    return RTLBFS_OK;
}

int Engine::grow_lists(int n)
{
    if (n <= list_cap_) return RTLBFS_OK;
    CK(cudaStreamSynchronize(stream_));
    cudaFree(d_slot_list_);
    cudaFree(d_run_list_);
    d_slot_list_ = nullptr;
    d_run_list_ = nullptr;
    list_cap_ = 0;
    CK(cudaMalloc(&d_slot_list_, sizeof(int) * n));
    CK(cudaMalloc(&d_run_list_, sizeof(CavityRun) * n));
    list_cap_ = n;
    return RTLBFS_OK;
}

int Engine::arm_many(int n, const int* slots, long long nsteps, double tol)
{
    if (n < 0 || (n > 0 && !slots)) return fail(RTLBFS_ERR_ARG, "null slot array");
    if (nsteps < 0) return fail(RTLBFS_ERR_ARG, "negative step count");
    for (int k = 0; k < n; ++k)
        if (!cavity(slots[k])) return fail(RTLBFS_ERR_ARG, "no such slot");
    if (n == 0) return RTLBFS_OK;
    int rc = grow_lists(n);
    if (rc) return rc;
    // copied from a pageable copy of the caller's array, which the runtime
    // stages before the call returns: the caller's array may be pinned, and
    // is free for reuse on return either way
    const std::vector<int> sl(slots, slots + n);
    CK(cudaMemcpyAsync(d_slot_list_, sl.data(), sizeof(int) * n, cudaMemcpyHostToDevice, stream_));
    CK(launch_arm_list(stream_, d_ctl_, d_slot_list_, n, nsteps, tol));
    g_launches++;
    return RTLBFS_OK;
}

int Engine::get_records_many(int n, const int* slots, void* const* host, double* T_units)
{
    Nvtx range("rtlbfs: state records out, many");
    if (n < 0 || (n > 0 && (!slots || !host)))
        return fail(RTLBFS_ERR_ARG, "null slot or record array");
    for (int k = 0; k < n; ++k)
        if (!cavity(slots[k]) || !host[k]) return fail(RTLBFS_ERR_ARG, "no such slot or null array");
    for (int k = 0; k < n; ++k)
        if (slots_[slots[k]].dirty) {
            int rc = upload_lines(slots[k]);
            if (rc) return rc;
        }
    std::vector<CavityCtl> ctl;
    int rc = read_ctls(ctl);  // the buffer of every slot's current state
    if (rc) return rc;
    const size_t rec = record_bytes();
    for (int k = 0; k < n; ++k) {
        const int slot = slots[k];
        const Cavity* c = &slots_[slot];
        CK(cudaMemcpy2DAsync(host[k], rec * c->nx, h_desc_[slot].f[ctl[slot].cur & 1][0],
                             rec * c->pitch, rec * c->nx, c->ny, cudaMemcpyDeviceToHost, stream_));
        if (T_units) T_units[k] = c->T_unit;
    }
    CK(cudaStreamSynchronize(stream_));
    return RTLBFS_OK;
}

// set_records without the final synchronisation: the copy from the host
// array is queued (pageable memory is staged before the copy call returns)
int Engine::queue_set_records(int slot, const void* host, double T_unit, CavityRun* run_out)
{
    Cavity* c = cavity(slot);
    if (!c || !host) return fail(RTLBFS_ERR_ARG, "no such slot or null array");
    int e2 = 0;
    const double m = std::frexp(T_unit, &e2);  // a power of two: m = 0.5
    if (precision_ == RTLBFS_FP64 ? T_unit != 1.0 : !(T_unit >= 1.0 && m == 0.5))
        return fail(RTLBFS_ERR_ARG, "T_unit must be 1 (FP64) or a power of two >= 1 (FP32)");
    c->state_Tmax = 0.0;
    // the records' unit; a configuration needing more rescales them.  In
    // the unit the slot already has, with its lines and descriptor current,
    // nothing needs uploading again (the unit was checked at that upload).
    if (T_unit != c->T_unit || c->dirty) {
        c->T_unit = T_unit;
        c->dirty = true;
        int rc = upload_lines(slot);
        if (rc) return rc;
    }
    const size_t rec = record_bytes();
    CK(cudaMemcpy2DAsync(h_desc_[slot].f[0][0], rec * c->pitch, host, rec * c->nx, rec * c->nx,
                         c->ny, cudaMemcpyHostToDevice, stream_));
    if (c->T_unit != T_unit) {  // the configuration asked for a larger unit
        const int shift = (int)std::lround(std::log2(c->T_unit / T_unit));
        CK(launch_rescale_T(stream_, h_desc_[slot].f[0][0], (long long)c->pitch * c->ny, shift));
        g_launches++;
    }
    CavityCtl z;
    std::memset(&z, 0, sizeof(z));
    z.cur = 0;
    z.done = 1;
    z.tol = -1.0;
    z.res[0] = z.res[1] = INFINITY;
    if (run_out) {  // the caller uploads the run record (set_records_many)
        std::memset(run_out, 0, sizeof(*run_out));
        run_out->h[0] = z;
        run_out->h[1] = z;
        return RTLBFS_OK;
    }
    return put_run(slot, z);
}

int Engine::set_conduction_state(int slot)
{
    Cavity* c = cavity(slot);
    if (!c) return fail(RTLBFS_ERR_ARG, "no such slot");
    // a new state from the configuration: its temperature unit afresh
    c->state_Tmax = 0.0;
    c->T_unit = temp_unit(*c);
    c->dirty = true;
    if (c->dirty) {
        int rc = upload_lines(slot);
        if (rc) return rc;
    }
    // rho = 1, u = v = 0, T linear in x between Dirichlet side walls (else
    // T_ref): one temperature per column, spread over the rows on the device
    std::vector<double> Tcol(c->nx, c->T_ref);
    if (c->kind[kSideW] == kDirichlet && c->kind[kSideE] == kDirichlet) {
        const double x0 = c->xf.front(), Lx = c->xf.back() - c->xf.front();
        for (int i = 0; i < c->nx; ++i) {
            const double s = (0.5 * (c->xf[i] + c->xf[i + 1]) - x0) / Lx;
            Tcol[i] = c->bcT[kSideW] + (c->bcT[kSideE] - c->bcT[kSideW]) * s;
        }
    }
    for (double& t : Tcol) t /= c->T_unit;  // exact: a power of two
    if (stage_cap_ < (size_t)c->nx) {
        CK(cudaStreamSynchronize(stream_));
        cudaFree(d_stage_);
        d_stage_ = nullptr;
        CK(cudaMalloc(&d_stage_, sizeof(double) * c->nx));
        stage_cap_ = c->nx;
    }
    CK(cudaMemcpyAsync(d_stage_, Tcol.data(), sizeof(double) * c->nx, cudaMemcpyHostToDevice,
                       stream_));
    CK(launch_conduction(precision_, stream_, d_stage_, c->nx, c->ny, c->pitch,
                         h_desc_[slot].f[0][0]));
    g_launches++;
    CavityCtl z;
    std::memset(&z, 0, sizeof(z));
    z.cur = 0;
    z.done = 1;
    z.tol = -1.0;
    z.res[0] = z.res[1] = INFINITY;
    return put_run(slot, z);
}

int Engine::arm(int slot, long long nsteps, double tol)
{
    if (!cavity(slot)) return fail(RTLBFS_ERR_ARG, "no such slot");
    if (nsteps < 0) return fail(RTLBFS_ERR_ARG, "negative step count");
    CK(launch_arm(stream_, d_ctl_, slot, nsteps, tol, 0));
    g_launches++;
    return RTLBFS_OK;
}

// The persistent tile kernel takes one RTLBFS cavity whose tiles are all
// resident at once and at least two cells wide and high (a tile's 2-cell
// halo then lies in the eight tiles around it).
int Engine::persist_check()
{
    persist_slot_ = -1;
    int active = 0, slot = -1;
    for (int s = 0; s < capacity_; ++s)
        if (slots_[s].active) {
            ++active;
            slot = s;
        }
    if (active != 1) return fail(RTLBFS_ERR_ARG, "the persistent kernel takes exactly one cavity");
    if (scheme_ != kSchemeRTLBFS)
        return fail(RTLBFS_ERR_ARG, "the persistent kernel runs the RTLBFS face stage only");
    const Cavity& c = slots_[slot];
    if (c.halo_rows)
        return fail(RTLBFS_ERR_ARG, "the persistent kernel takes whole meshes, not row strips");
    if ((c.nx % kTileX) == 1 || (c.ny % tile_h_) == 1)
        return fail(RTLBFS_ERR_ARG, "the persistent kernel needs tiles at least 2 cells wide");
    if ((long long)ntiles_ > (long long)sms_ * occ_persist_[tile_h_])
        return fail(RTLBFS_ERR_ARG, "the mesh has more tiles than fit on the GPU at once");
    persist_slot_ = slot;
    return RTLBFS_OK;
}

int Engine::launch_steps(long long launches)
{
    Nvtx range("rtlbfs: step launches");
    int rc = prepare_launch();
    if (rc) return rc;
    if (ntiles_ == 0 || launches <= 0) return RTLBFS_OK;
    if (kernel_ == 2) {
        // chunks of steps, one launch each; a wait that ran out is an error
        const Cavity& c = slots_[persist_slot_];
        for (long long left = launches; left > 0;) {
            const int n = (int)std::min<long long>(left, kPersistChunk);
            CK(cudaMemsetAsync(d_tstep_, 0, sizeof(int) * ntiles_, stream_));
            CK(cudaMemsetAsync(d_pctl_, 0, sizeof(PersistCtl), stream_));
            CK(launch_persist(precision_, tile_h_, ntiles_, stream_, &d_desc_[persist_slot_],
                              &d_ctl_[persist_slot_].h[0], d_tiles_ + c.first_tile, d_tstep_, d_pctl_,
                              n, withhold_));
            g_launches++;
            CK(cudaMemcpyAsync(h_stalled_, &d_pctl_->stalled, sizeof(int), cudaMemcpyDeviceToHost,
                               stream_));
            CK(cudaStreamSynchronize(stream_));
            if (*h_stalled_)
                return fail(RTLBFS_ERR_CUDA, "persistent step stalled: a bounded wait ran out");
            left -= n;
        }
        return RTLBFS_OK;
    }
    // launch k of this chain has parity k & 1 (graphs hold an even number
    // of launches); the chain ends with the stop test of its last step
    long long left = launches;
    int par = 0;
    auto launch = [&](cudaStream_t st, int p) {
        return kernel_ == 1 ? launch_step(precision_, tile_h_, scheme_, grid_, st, d_desc_, d_ctl_,
                                          d_tiles_, d_ntiles_, p)
                            : launch_march(precision_, grid_, st, d_desc_, d_ctl_, d_tiles_,
                                           d_ntiles_, p);
    };
    static_assert(kGraphChunk % 2 == 0, "graphs of an even number of launches");
    if (left >= kGraphChunk) {
        if (!gexec_) {
            cudaStream_t cs = nullptr;
            CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (int k = 0; k < kGraphChunk && e == cudaSuccess; ++k) e = launch(cs, k & 1);
                cudaError_t e2 = cudaStreamEndCapture(cs, &g);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec_, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) return cuda_fail(e, "capturing the step graph");
            gchunk_ = kGraphChunk;
        }
        while (left >= gchunk_) {
            Nvtx replay("rtlbfs: step graph replay");
            CK(cudaGraphLaunch(gexec_, stream_));
            g_launches += gchunk_;
            left -= gchunk_;
        }
    }
    for (; left > 0; --left) {
        CK(launch(stream_, par));
        par ^= 1;
        g_launches++;
    }
    CK(launch_finalize(stream_, d_ctl_, capacity_, par));
    g_launches++;
    return RTLBFS_OK;
}

int Engine::autotune(int steps, int* kernel_out, int* rows_out, double* ms_out)
{
    Nvtx range("rtlbfs: autotune");
    if (steps < 1) return fail(RTLBFS_ERR_ARG, "autotune needs steps >= 1");
    CK(cudaStreamSynchronize(stream_));
    // snapshot every active cavity's fields and the run control
    std::vector<void*> snap(capacity_, nullptr);
    std::vector<CavityRun> ctl_save(capacity_);
    CK(cudaMemcpy(ctl_save.data(), d_ctl_, sizeof(CavityRun) * capacity_, cudaMemcpyDeviceToHost));
    int maxny = 1;
    for (int s = 0; s < capacity_; ++s) {
        if (!slots_[s].active) continue;
        maxny = std::max(maxny, slots_[s].ny);
        cudaError_t e = cudaMalloc(&snap[s], slots_[s].fields_bytes);
        if (e != cudaSuccess) {
            for (void* p : snap) cudaFree(p);
            return cuda_fail(e, "autotune snapshot");
        }
        CK(cudaMemcpyAsync(snap[s], slots_[s].d_fields, slots_[s].fields_bytes,
                           cudaMemcpyDeviceToDevice, stream_));
    }
    struct Cand {
        int kernel, rows;
    };
    std::vector<Cand> cands;
    for (int h : kTileHeights)
        if (tile_height_ok(precision_, h) && (scheme_ == kSchemeRTLBFS || h == kTileYDefault))
            cands.push_back({1, h});
    // the persistent tile kernel, at each height whose tiles all fit at once
    // (engines of one slot only: a batch could grow past one cavity later)
    int active = 0, aslot = -1;
    for (int s = 0; s < capacity_; ++s)
        if (slots_[s].active) {
            ++active;
            aslot = s;
        }
    if (capacity_ == 1 && active == 1 && scheme_ == kSchemeRTLBFS && !slots_[aslot].halo_rows)
        for (int h : kTileHeights) {
            if (!tile_height_ok(precision_, h)) continue;
            const Cavity& c = slots_[aslot];
            const long long tiles =
                (long long)((c.nx + kTileX - 1) / kTileX) * ((c.ny + h - 1) / h);
            if ((c.nx % kTileX) != 1 && (c.ny % h) != 1 &&
                tiles <= (long long)sms_ * occ_persist_[h])
                cands.push_back({2, h});
        }
    for (int H : {8, 16, 32, 64, 128, 256}) {
        if (scheme_ == kSchemeTLBFS) break;
        if (H > maxny && H != 8) break;
        cands.push_back({0, H});
    }
    const int keep_kernel = kernel_, keep_rows = chunk_rows_;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    Cand pick = {keep_kernel, keep_rows};
    int rc = RTLBFS_OK;
    for (const Cand& c : cands) {
        if ((rc = set_kernel(c.kernel)) || (rc = set_chunk_rows(c.rows))) break;
        for (int s = 0; s < capacity_ && !rc; ++s)
            if (slots_[s].active) rc = arm(s, (long long)steps + 8, -1.0);
        if (rc || (rc = launch_steps(4))) break;
        cudaEventRecord(e0, stream_);
        if ((rc = launch_steps(steps))) break;
        cudaEventRecord(e1, stream_);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            pick = c;
        }
        // restore the snapshot before the next candidate
        for (int s = 0; s < capacity_; ++s)
            if (snap[s])
                cudaMemcpyAsync(slots_[s].d_fields, snap[s], slots_[s].fields_bytes,
                                cudaMemcpyDeviceToDevice, stream_);
        cudaMemcpyAsync(d_ctl_, ctl_save.data(), sizeof(CavityRun) * capacity_,
                        cudaMemcpyHostToDevice, stream_);
        cudaStreamSynchronize(stream_);
    }
    // final restore (also after an error)
    for (int s = 0; s < capacity_; ++s)
        if (snap[s])
            cudaMemcpyAsync(slots_[s].d_fields, snap[s], slots_[s].fields_bytes,
                            cudaMemcpyDeviceToDevice, stream_);
    cudaMemcpyAsync(d_ctl_, ctl_save.data(), sizeof(CavityRun) * capacity_, cudaMemcpyHostToDevice,
                    stream_);
    cudaStreamSynchronize(stream_);
    for (void* p : snap) cudaFree(p);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        set_kernel(keep_kernel);
        set_chunk_rows(keep_rows);
        return rc;
    }
    set_kernel(pick.kernel);
    set_chunk_rows(pick.rows);
    if (kernel_out) *kernel_out = pick.kernel;
    if (rows_out) *rows_out = pick.rows;
    if (ms_out) *ms_out = best / steps;
    return RTLBFS_OK;
}

int Engine::read_ctl(int slot, CavityCtl* out)
{
    if (slot < 0 || slot >= capacity_) return fail(RTLBFS_ERR_ARG, "no such slot");
    CK(cudaMemcpyAsync(out, &d_ctl_[slot].h[0], sizeof(CavityCtl), cudaMemcpyDeviceToHost,
                       stream_));
    CK(cudaStreamSynchronize(stream_));
    return RTLBFS_OK;
}

int Engine::read_ctls(std::vector<CavityCtl>& out)
{
    out.resize(capacity_);
    CK(cudaStreamSynchronize(stream_));
    // the tested header h[0] of every slot, in one strided copy
    CK(cudaMemcpy2D(out.data(), sizeof(CavityCtl), d_ctl_, sizeof(CavityRun), sizeof(CavityCtl),
                    capacity_, cudaMemcpyDeviceToHost));
    return RTLBFS_OK;
}

int Engine::nusselt(int slot, int which, double* out)
{
    Nvtx range("rtlbfs: Nusselt sum");
    Cavity* c = cavity(slot);
    if (!c) return fail(RTLBFS_ERR_ARG, "no such slot");
    if (which < kNuWest || which > kNuHalf) return fail(RTLBFS_ERR_ARG, "bad Nusselt selector");
    if (which == kNuHalf && (c->nx % 2)) return fail(RTLBFS_ERR_ARG, "Nu_1/2 needs nx even");
    if ((which == kNuSouth || which == kNuNorth) && c->kind[which] == kHalo)
        return fail(RTLBFS_ERR_ARG, "no wall on a strip's halo side");
    if (c->dirty) {  // the reduction reads this cavity's lines and descriptor
        int rc = upload_lines(slot);
        if (rc) return rc;
    }
    const CavityDesc& d = h_desc_[slot];
    unsigned char* L = static_cast<unsigned char*>(c->d_lines);
    NuLines ln;
    ln.xl = reinterpret_cast<const FaceLine<double>*>(L + c->off_xld);
    ln.yl = reinterpret_cast<const FaceLine<double>*>(L + c->off_yld);
    ln.xc = reinterpret_cast<const CellLine<double>*>(L + c->off_xcd);
    ln.yc = reinterpret_cast<const CellLine<double>*>(L + c->off_ycd);
    long long count;
    double scale = 1.0 / (c->chi * d.dT);  // dT in the state's temperature unit
    if (which == kNuWest || which == kNuEast || which == kNuHalf) count = c->ny;
    else if (which == kNuSouth || which == kNuNorth) count = c->nx;
    else {
        count = (long long)c->nx * c->ny;
        scale /= (c->xf.back() - c->xf.front());
    }
    CK(launch_nusselt(precision_, stream_, d_desc_, d_ctl_, slot, ln, which, count, scale,
                      d_partial_, partial_cap_, d_scalar_));
    g_launches += 2;
    CK(cudaMemcpyAsync(h_scalar_, d_scalar_, sizeof(double), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    *out = h_scalar_[0];
    return RTLBFS_OK;
}

}  // namespace rtlbfs
