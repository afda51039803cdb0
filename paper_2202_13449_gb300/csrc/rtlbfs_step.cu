// rtlbfs_step.cu -- the fused RTLBFS time step on sm_103a and the FP64
// reductions (Nusselt numbers), for any list of cavities ("batch").
//
// One launch advances every listed cavity by one explicit step (Section 3.2
// of arXiv 2202.13449).  Work unit: a tile of TX x TY cells of one cavity.
// Per tile, in shared memory:
//   1. the tile plus a 2-cell halo of (drho, u, v, T), with the boundary
//      ghosts materialised (mirror rules at walls, wrap at periodic sides);
//   2. Green-Gauss gradients (Eq. 55) with inverse-distance face values
//      (Eq. 56) on the tile plus a 1-cell ring; wall ghosts mirror their
//      partner's gradient;
//   3. every x- and y-face of the tile: 9-node lattice (Eq. 29), predictor
//      (Eqs. 46-48), corrector fluxes (Eqs. 57-59) -- face_flux();
//   4. the explicit update with the Boussinesq source (Eq. 64) and the
//      conservative -> primitive conversion;
//   5. the residual sums of the steady criterion; the last tile of a cavity
//      to finish turns them into (R_u, R_T), advances the step counter,
//      flips the buffer and decides whether the cavity is done.
// Face values and gradients never leave the SM; HBM sees one read and one
// write of the four fields per cell per step (halo re-reads hit L2).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "rtlbfs.h"
#include "rtlbfs_dev.cuh"
#include "rtlbfs_kernels.h"
#include "rtlbfs_tile.cuh"

namespace rtlbfs {

template <class P, int TX, int TY, int NT, int SCHEME>
__global__ void __launch_bounds__(NT, MinBlocks<P, NT>::value)
step_kernel(const CavityDesc* __restrict__ descs, CavityRun* __restrict__ runs,
            const int4* __restrict__ tiles, const int* __restrict__ ntiles_ptr, int par)
{
    using Sm = TileSmem<P, TX, TY, NT>;
    using S = typename P::S;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    Sm& sm = *reinterpret_cast<Sm*>(smem_raw);
    const int tid = threadIdx.x;
    // the tile list, the first tile's descriptor and mesh lines: written by
    // the host, not by the previous step, so fetched before the wait
    const int ntiles = *ntiles_ptr;
    if (blockIdx.x < ntiles) {
        const int4 tile = tiles[blockIdx.x];
        stage_tile(sm, &descs[tile.x], tile.y, tile.z);
    }
    chain_sync();

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tile = tiles[t];
        const int slot = tile.x, i0 = tile.y, j0 = tile.z;
        CavityRun* run = &runs[slot];
        // the stop test of the cavity's previous step (one thread; its first
        // tile also publishes the header for the next launch)
        if (tid == 0) {
            const CavityCtl d = run_head(run, par);
            if (t == descs[slot].tile_begin) run_publish(run, par, d);
            sm.plan[0] = d.done;
            sm.plan[1] = d.cur;
            sm.plan[2] = (int)(d.steps % 3);
        }
        __syncthreads();  // the plan (and, on the first tile, the staged descriptor and lines)
        const int done = sm.plan[0], cur = sm.plan[1], slot3 = sm.plan[2];
        if (done) {  // uniform across the block
            __syncthreads();  // everyone has read the plan before it is rewritten
            continue;
        }
        // the first tile uses what was staged; later tiles (batches) read
        // their descriptor in place and load their lines beside the state
        const bool first = t == (int)blockIdx.x;
        const CavityDesc* dp = first ? &sm.desc : &descs[slot];
        tile_step<P, TX, TY, NT, SCHEME, false>(sm, dp, i0, j0,
                                                static_cast<const Vec4<S>*>(dp->f[cur][0]),
                                                static_cast<Vec4<S>*>(dp->f[cur ^ 1][0]), first);
        __syncthreads();
        double a[4];
        if (tid < 32) tile_sums(sm, a);
        // the step's residual sums; the next launch tests them
        if (tid == 0)
            for (int q = 0; q < 4; ++q) atomicAdd(&run->acc[slot3][q], a[q]);
        __syncthreads();
    }
}

// The stop test of the last step of a chain of launches of parity par:
// both headers of every cavity become its tested header (host-readable).
__global__ void finalize_kernel(CavityRun* __restrict__ runs, int n, int par)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    CavityCtl d = run_head(&runs[s], par);
    if (d.res_stale) {  // (R_u, R_T) of the last tested step
        d.res[0] = r12(d.sums[0], d.sums[1]);
        d.res[1] = r12(d.sums[2], d.sums[3]);
        d.res_stale = 0;
    }
    runs[s].h[0] = d;
    runs[s].h[1] = d;
}

// ---------------------------------------------------------------------------
// FP64 evaluation straight from global memory (Nusselt reductions).
// ---------------------------------------------------------------------------
template <class P>
__device__ bool load_cell_d(const CavityDesc& d, int b, int gi, int gj, Vec4<double>& v)
{
    int si, sj, ms;
    if (!resolve_cell(d, gi, gj, si, sj, ms)) return false;
    const long long o = (long long)sj * d.pitch + si;
    const Vec4<typename P::S> x = P::load4(&d, b, o);
    v = {P::to_double(x.x, 0), P::to_double(x.y, 1), P::to_double(x.z, 2), P::to_double(x.w, 3)};
    if (ms >= 0) v = mirror_values<StoreD>(d, ms, v, 0.0);  // FP64, T absolute
    return true;
}

// Green-Gauss gradient (Eqs. 55-56) of cell (gi, gj) in FP64; a wall ghost
// mirrors its partner's.  xc/yc: FP64 cell lines (index i + 2).
template <class P>
__device__ void grad_d(const CavityDesc& d, int f, const CellLine<double>* xc,
                       const CellLine<double>* yc, int gi, int gj, Vec4<double>& gx,
                       Vec4<double>& gy)
{
    int si, sj, ms;
    gx = {0, 0, 0, 0};
    gy = gx;
    if (!resolve_cell(d, gi, gj, si, sj, ms)) return;
    int ci = gi, cj = gj;
    if (ms == kSideW) ci += 1;
    else if (ms == kSideE) ci -= 1;
    else if (ms == kSideS) cj += 1;
    else if (ms == kSideN) cj -= 1;
    Vec4<double> p = {0, 0, 0, 0}, e = p, w = p, n = p, s = p;
    load_cell_d<P>(d, f, ci, cj, p);
    load_cell_d<P>(d, f, ci + 1, cj, e);
    load_cell_d<P>(d, f, ci - 1, cj, w);
    load_cell_d<P>(d, f, ci, cj + 1, n);
    load_cell_d<P>(d, f, ci, cj - 1, s);
    gg_gradient<StoreD>(p, e, w, n, s, xc[ci + 2].is_next, xc[ci + 1].is_next, yc[cj + 2].is_next,
                        yc[cj + 1].is_next, gx, gy);
    if (ms >= 0) mirror_grad(d, ms, gx, gy);
}

// Energy flux (Eq. 59 brace) through x-face (i, j) (nd = 0) or y-face
// (nd = 1), in FP64.
template <class P>
__device__ double energy_flux_d(const CavityDesc& d, int f, const NuLines& ln, int nd, int i,
                                int j)
{
    const bool xper = d.kind[kSideW] == kPeriodic, yper = d.kind[kSideS] == kPeriodic;
    const int li = nd == 0 ? i - 1 : i, lj = nd == 0 ? j : j - 1;
    Vec4<double> vl = {0, 0, 0, 0}, vr = vl, gxl, gyl, gxr, gyr;
    load_cell_d<P>(d, f, li, lj, vl);
    load_cell_d<P>(d, f, i, j, vr);
    grad_d<P>(d, f, ln.xc, ln.yc, li, lj, gxl, gyl);
    grad_d<P>(d, f, ln.xc, ln.yc, i, j, gxr, gyr);
    CellNT<double> L, Rr;
    double Tbar;
    face_cells<double>(nd == 0, vl, vr, 0.0, gxl, gyl, gxr, gyr, L, Rr, Tbar);
    int wside = -1;
    if (nd == 0 && !xper) wside = i == 0 ? kSideW : (i == d.nx ? kSideE : -1);
    if (nd == 1 && !yper)
        wside = (j == 0 && d.kind[kSideS] != kHalo)
                    ? kSideS
                    : ((j == d.ny && d.kind[kSideN] != kHalo) ? kSideN : -1);
    const FaceLine<double> fl = nd == 0 ? ln.xl[i] : ln.yl[j];
    double F[4];
    const double keep = wside >= 0 ? 0.0 : 1.0, uw = wside >= 0 ? d.bcU[wside] : 0.0;
    if (d.scheme == 1) face_flux_tlbfs<double>(L, Rr, Tbar, fl, keep, uw, F);
    else face_flux<double>(L, Rr, Tbar, fl, keep, uw, F);
    return F[3];
}

// Sum over a block of up to 256 threads in FP64: warp shuffles, then the
// warps' sums by warp 0 (thread 0 holds the result).
__device__ __forceinline__ double block_sum_d(double v)
{
    __shared__ double wsum[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)((blockDim.x + 31) >> 5) ? wsum[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}

// Partial sums of a Nusselt number: one partial per block, in block order.
template <class P>
__global__ void __launch_bounds__(256)
nusselt_partial_kernel(const CavityDesc* __restrict__ descs, const CavityRun* __restrict__ runs,
                       int slot, NuLines ln, int which, double* __restrict__ partial)
{
    const CavityDesc& d = descs[slot];
    const int f = runs[slot].h[0].cur;  // buffer holding the current state
    long long count;
    if (which == kNuWest || which == kNuEast || which == kNuHalf) count = d.ny;
    else if (which == kNuSouth || which == kNuNorth) count = d.nx;
    else count = (long long)d.nx * d.ny;
    double s = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        if (which == kNuWest || which == kNuEast || which == kNuHalf) {
            const int i = which == kNuWest ? 0 : (which == kNuEast ? d.nx : d.nx / 2);
            const int j = (int)k;
            s += energy_flux_d<P>(d, f, ln, 0, i, j) * ln.yc[j + 2].w;
        } else if (which == kNuSouth || which == kNuNorth) {
            const int i = (int)k;
            const int j = which == kNuSouth ? 0 : d.ny;
            s += energy_flux_d<P>(d, f, ln, 1, i, j) * ln.xc[i + 2].w;
        } else {  // Eq. 69 integrand (u T - chi dT/dx) dV
            const int i = (int)(k % d.nx), j = (int)(k / d.nx);
            Vec4<double> p = {0, 0, 0, 0}, gx, gy;
            load_cell_d<P>(d, f, i, j, p);
            grad_d<P>(d, f, ln.xc, ln.yc, i, j, gx, gy);
            s += (p.y * p.w - d.chi * gx.w) * ln.xc[i + 2].w * ln.yc[j + 2].w;
        }
    }
    s = block_sum_d(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) sum_partials_kernel(const double* __restrict__ partial,
                                                           int n, double scale,
                                                           double* __restrict__ out)
{
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += partial[k];
    s = block_sum_d(s);
    if (threadIdx.x == 0) *out = s * scale;
}

// State conversion: FP64 host-layout staging (rho, u, v, T planes of n
// cells, row-major nx) <-> device storage (rho - 1, u, v, T with row pitch).
// T_unit: the temperature unit of the stored state (a power of two; 1 in
// FP64): the stored temperature is T / T_unit.
template <class P>
__global__ void state_in_kernel(const double* __restrict__ st, int nx, int ny, int pitch,
                                double T_unit, Vec4<typename P::S>* __restrict__ cells,
                                int* __restrict__ bad)
{
    const long long n = (long long)nx * ny;
    const double Tinv = 1.0 / T_unit;  // exact: a power of two
    bool b = false;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = k % nx, j = k / nx;
        const double x[4] = {st[k] - 1.0, st[n + k], st[2 * n + k], st[3 * n + k] * Tinv};
        for (int q = 0; q < 4; ++q) b = b || !P::representable(x[q], q);
        cells[(size_t)j * pitch + i] = {P::from_double(x[0], 0), P::from_double(x[1], 1),
                                        P::from_double(x[2], 2), P::from_double(x[3], 3)};
    }
    if (b) atomicOr(bad, 1);
}

template <class P>
__global__ void state_out_kernel(double* __restrict__ st, int nx, int ny, int pitch,
                                 double T_unit, const Vec4<typename P::S>* __restrict__ cells)
{
    const long long n = (long long)nx * ny;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = k % nx, j = k / nx;
        const Vec4<typename P::S> c = cells[(size_t)j * pitch + i];
        st[k] = 1.0 + P::to_double(c.x, 0);
        st[n + k] = P::to_double(c.y, 1);
        st[2 * n + k] = P::to_double(c.z, 2);
        st[3 * n + k] = P::to_double(c.w, 3) * T_unit;
    }
}

// Stored temperatures of `count` cell records divided by 2^shift (rounded
// to nearest): the state follows a temperature unit that grew by 2^shift.
__global__ void rescale_T_kernel(Vec4<int>* __restrict__ cells, long long count, int shift)
{
    const int half = 1 << (shift - 1);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x)
        cells[k].w = (int)(((long long)cells[k].w + half) >> shift);
}

template <class P>
__global__ void conduction_kernel(const double* __restrict__ Tcol, int nx, int ny, int pitch,
                                  Vec4<typename P::S>* __restrict__ cells)
{
    const long long n = (long long)nx * ny;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = k % nx, j = k / nx;
        cells[(size_t)j * pitch + i] = {P::from_double(0.0, 0), P::from_double(0.0, 1),
                                        P::from_double(0.0, 2), P::from_double(Tcol[i], 3)};
    }
}

// Arm the run control of one cavity: take `nsteps` more steps (stop early
// when max(R_u, R_T) < tol, tol < 0: never).  Runs on a tested header
// (pend = 0: after finalize_kernel or a state upload).
__global__ void arm_kernel(CavityRun* runs, const int* __restrict__ slot_list, int n, int slot,
                           long long nsteps, double tol, int reset_counter)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    CavityRun* r = &runs[slot_list ? slot_list[k] : slot];
    CavityCtl c = r->h[0];
    if (reset_counter) {
        c.steps = 0;
        c.res[0] = c.res[1] = INFINITY;
        for (int q = 0; q < 4; ++q) c.sums[q] = 0.0;
        c.res_stale = 0;
    }
    c.max_steps = c.steps + nsteps;
    c.tol = tol;
    c.status = kRunning;
    c.done = nsteps > 0 ? 0 : 1;
    c.pend = 0;
    r->h[0] = c;
    r->h[1] = c;
    for (int k = 0; k < 3; ++k)
        for (int q = 0; q < 4; ++q) r->acc[k][q] = 0.0;
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
template <class P, int TY, int SCHEME = 0>
struct TileKernel {
    static constexpr int NT = TileThreads<P, TY>::value;
    static constexpr size_t smem = sizeof(TileSmem<P, kTileX, TY, NT>);
    static constexpr auto fn = step_kernel<P, kTileX, TY, NT, SCHEME>;
    static cudaError_t prepare()
    {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        // all of the unified L1/shared array to shared memory: occupancy is
        // bounded by the tile buffers, and global loads are streamed once
        return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    static cudaError_t occupancy(int* blocks)
    {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, NT, smem);
    }
    static cudaError_t launch(int grid, cudaStream_t s, const CavityDesc* descs, CavityRun* runs,
                              const int4* tiles, const int* ntiles, int par)
    {
        return launch_chained(fn, grid, NT, smem, s, descs, runs, tiles, ntiles, par);
    }
};

// Call op on the compiled tile kernel of (precision, tile_h, scheme); the
// TLBFS face stage is compiled for the default tile height.
template <class Op>
static cudaError_t with_tile_kernel(int precision, int tile_h, int scheme, Op op)
{
    if (scheme == 1) {
        if (tile_h != kTileYDefault) return cudaErrorInvalidValue;
        if (precision == 0) return op(TileKernel<StoreD, kTileYDefault, 1>());
        return op(TileKernel<StoreQ, kTileYDefault, 1>());
    }
    if (scheme != 0) return cudaErrorInvalidValue;
    if (precision == 0) {
        switch (tile_h) {
        case 16: return op(TileKernel<StoreD, 16>());
        case 8: return op(TileKernel<StoreD, 8>());
        case 4: return op(TileKernel<StoreD, 4>());
        case 2: return op(TileKernel<StoreD, 2>());
        default: return cudaErrorInvalidValue;
        }
    }
    switch (tile_h) {
    case 16: return op(TileKernel<StoreQ, 16>());
    case 14: return op(TileKernel<StoreQ, 14>());
    case 12: return op(TileKernel<StoreQ, 12>());
    case 10: return op(TileKernel<StoreQ, 10>());
    case 8: return op(TileKernel<StoreQ, 8>());
    case 4: return op(TileKernel<StoreQ, 4>());
    case 2: return op(TileKernel<StoreQ, 2>());
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t step_prepare(int precision)
{
    for (int h : kTileHeights) {
        if (!tile_height_ok(precision, h)) continue;
        cudaError_t e = with_tile_kernel(precision, h, 0, [](auto k) { return k.prepare(); });
        if (e != cudaSuccess) return e;
    }
    return with_tile_kernel(precision, kTileYDefault, 1, [](auto k) { return k.prepare(); });
}

cudaError_t step_occupancy(int precision, int tile_h, int scheme, int* blocks_per_sm)
{
    return with_tile_kernel(precision, tile_h, scheme,
                            [&](auto k) { return k.occupancy(blocks_per_sm); });
}

cudaError_t launch_step(int precision, int tile_h, int scheme, int grid, cudaStream_t s,
                        const CavityDesc* descs, CavityRun* runs, const int4* tiles,
                        const int* ntiles, int par)
{
    return with_tile_kernel(precision, tile_h, scheme, [&](auto k) {
        return k.launch(grid, s, descs, runs, tiles, ntiles, par);
    });
}

cudaError_t launch_finalize(cudaStream_t s, CavityRun* runs, int n, int par)
{
    finalize_kernel<<<(n + 127) / 128, 128, 0, s>>>(runs, n, par);
    return cudaGetLastError();
}

cudaError_t launch_nusselt(int precision, cudaStream_t s, const CavityDesc* descs,
                           const CavityRun* ctls, int slot, const NuLines& ln, int which,
                           long long count, double scale, double* partial, int max_blocks,
                           double* out)
{
    int blocks = (int)((count + 255) / 256);
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    if (precision == 0)
        nusselt_partial_kernel<StoreD><<<blocks, 256, 0, s>>>(descs, ctls, slot, ln, which, partial);
    else
        nusselt_partial_kernel<StoreQ><<<blocks, 256, 0, s>>>(descs, ctls, slot, ln, which, partial);
    sum_partials_kernel<<<1, 256, 0, s>>>(partial, blocks, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_state_in(int precision, cudaStream_t s, const double* st, int nx, int ny,
                            int pitch, double T_unit, void* cells, int* bad)
{
    const long long n = (long long)nx * ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (precision == 0)
        state_in_kernel<StoreD><<<blocks, 256, 0, s>>>(st, nx, ny, pitch, T_unit,
                                                       static_cast<Vec4<double>*>(cells), bad);
    else
        state_in_kernel<StoreQ><<<blocks, 256, 0, s>>>(st, nx, ny, pitch, T_unit,
                                                       static_cast<Vec4<int>*>(cells), bad);
    return cudaGetLastError();
}

cudaError_t launch_state_out(int precision, cudaStream_t s, double* st, int nx, int ny, int pitch,
                             double T_unit, const void* cells)
{
    const long long n = (long long)nx * ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (precision == 0)
        state_out_kernel<StoreD><<<blocks, 256, 0, s>>>(st, nx, ny, pitch, T_unit,
                                                        static_cast<const Vec4<double>*>(cells));
    else
        state_out_kernel<StoreQ><<<blocks, 256, 0, s>>>(st, nx, ny, pitch, T_unit,
                                                        static_cast<const Vec4<int>*>(cells));
    return cudaGetLastError();
}

cudaError_t launch_rescale_T(cudaStream_t s, void* cells, long long count, int shift)
{
    if (shift < 1 || shift > 30) return cudaErrorInvalidValue;
    int blocks = (int)((count + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    rescale_T_kernel<<<blocks, 256, 0, s>>>(static_cast<Vec4<int>*>(cells), count, shift);
    return cudaGetLastError();
}

cudaError_t launch_conduction(int precision, cudaStream_t s, const double* Tcol, int nx, int ny,
                              int pitch, void* cells)
{
    const long long n = (long long)nx * ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (precision == 0)
        conduction_kernel<StoreD><<<blocks, 256, 0, s>>>(Tcol, nx, ny, pitch,
                                                         static_cast<Vec4<double>*>(cells));
    else
        conduction_kernel<StoreQ><<<blocks, 256, 0, s>>>(Tcol, nx, ny, pitch,
                                                         static_cast<Vec4<int>*>(cells));
    return cudaGetLastError();
}

cudaError_t launch_arm(cudaStream_t s, CavityRun* ctls, int slot, long long nsteps, double tol,
                       int reset_counter)
{
    arm_kernel<<<1, 1, 0, s>>>(ctls, nullptr, 1, slot, nsteps, tol, reset_counter);
    return cudaGetLastError();
}

cudaError_t launch_arm_list(cudaStream_t s, CavityRun* ctls, const int* slots, int n,
                            long long nsteps, double tol)
{
    if (n <= 0) return cudaSuccess;
    arm_kernel<<<(n + 127) / 128, 128, 0, s>>>(ctls, slots, n, 0, nsteps, tol, 0);
    return cudaGetLastError();
}

// Run records of n slots from a device array (slot k's record is src[k]).
__global__ void put_runs_kernel(CavityRun* runs, const int* __restrict__ slots,
                                const CavityRun* __restrict__ src, int n)
{
    const int k = blockIdx.x;
    if (k >= n) return;
    const double* a = reinterpret_cast<const double*>(&src[k]);
    double* b = reinterpret_cast<double*>(&runs[slots[k]]);
    for (int w = threadIdx.x; w < (int)(sizeof(CavityRun) / sizeof(double)); w += blockDim.x)
        b[w] = a[w];
}

cudaError_t launch_put_runs(cudaStream_t s, CavityRun* ctls, const int* slots,
                            const CavityRun* src, int n)
{
    if (n <= 0) return cudaSuccess;
    put_runs_kernel<<<n, 32, 0, s>>>(ctls, slots, src, n);
    return cudaGetLastError();
}

}  // namespace rtlbfs

// ---------------------------------------------------------------------------
// Allocation-free Nusselt number (rtlbfs_nusselt_noalloc).
//
// For callers that must not allocate device memory at call time: a
// real-time loop, where cudaMalloc can block on the device or fail at an
// unpredictable moment, or a host that gives the library only a fixed pool
// of memory it owns, and keeps its fields in its own buffers.  The
// wall/average Nusselt reduction runs on caller-owned device fields with all
// of its working memory in one file-scope device array: the cavity
// descriptor, the FP64 mesh lines and the per-block partial sums.  Every GPU
// that loads the library holds this array (kNoAllocBytes, about 1.8 MB)
// until the process exits.
// ---------------------------------------------------------------------------
namespace rtlbfs {

extern std::atomic<long long> g_launches;

constexpr int kNoAllocMaxN = 8192;       // cells per side
constexpr int kNoAllocPartials = 1024;   // reduction blocks

struct NoAllocScratch {
    CavityDesc desc;
    CavityRun ctl;
    double xf[kNoAllocMaxN + 1];
    double yf[kNoAllocMaxN + 1];
    FaceLine<double> xl[kNoAllocMaxN + 1];
    FaceLine<double> yl[kNoAllocMaxN + 1];
    CellLine<double> xc[kNoAllocMaxN + 4];
    CellLine<double> yc[kNoAllocMaxN + 4];
    double partial[kNoAllocPartials];
};
constexpr size_t kNoAllocBytes = sizeof(NoAllocScratch);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// The caller's four separate FP64 arrays, rho (not rho - 1) in the first.
struct StoreRho : StoreD {
    static __host__ __device__ __forceinline__ double to_double(double s, int k)
    {
        return k == 0 ? s - 1.0 : s;
    }
    static __device__ __forceinline__ Vec4<double> load4(const CavityDesc* d, int b, size_t o)
    {
        return {static_cast<const double*>(d->f[b][0])[o], static_cast<const double*>(d->f[b][1])[o],
                static_cast<const double*>(d->f[b][2])[o], static_cast<const double*>(d->f[b][3])[o]};
    }
};

// Mesh lines of one axis from its face coordinates (the same formulas as
// the host-side line builder of the engine), in device memory.
__global__ void noalloc_lines_kernel(const double* __restrict__ f, int n, int periodic,
                                     double kappa, double nu, double chi,
                                     FaceLine<double>* __restrict__ fl,
                                     CellLine<double>* __restrict__ cl)
{
    auto width = [&](int i) {
        int k = i;
        if (periodic) {
            k = ((i % n) + n) % n;
        } else {
            if (i < 0) k = -1 - i;
            if (i >= n) k = 2 * n - 1 - i;
            k = min(max(k, 0), n - 1);
        }
        return f[k + 1] - f[k];
    };
    for (int i = threadIdx.x; i <= n; i += blockDim.x) {
        const double wl = width(i - 1), wr = width(i);
        const double h = kappa * fmin(wl, wr);
        FaceLine<double> x;
        x.h = h;
        x.cL = 0.5 * wl - h;
        x.cR = h - 0.5 * wr;
        x.m_nu_2h = -nu / (2.0 * h);
        x.m_chi_2h = -chi / (2.0 * h);
        x.m_tf15 = 1.0 - 3.0 * nu / h;
        x.m_tg15 = 1.0 - 3.0 * chi / h;
        x.pad = 0.0;
        fl[i] = x;
    }
    for (int i = (int)threadIdx.x - 2; i <= n + 1; i += blockDim.x) {
        const double w = width(i), wn = width(i + 1);
        CellLine<double> y;
        y.w = w;
        y.is_next = 1.0 / (w + wn);
        y.dt_w = 0.0;
        y.pad = 0.0;
        cl[i + 2] = y;
    }
}

// The call's descriptor, passed by value (no host staging of a stack
// object), and the run control the reduction reads (buffer 0 current).
__global__ void noalloc_setup_kernel(CavityDesc d, CavityDesc* __restrict__ desc,
                                     CavityRun* __restrict__ ctl)
{
    *desc = d;
    CavityRun c;
    memset(&c, 0, sizeof(c));
    *ctl = c;
}

namespace {
std::atomic<void*> g_noalloc_ptr[64];
}

}  // namespace rtlbfs

extern "C" int rtlbfs_nusselt_noalloc(int nx, int ny, const double* xf, const double* yf,
                                      const double* rho, const double* u, const double* v,
                                      const double* T, double nu, double chi, double kappa,
                                      double dT, const int* bc_kind, const double* bc_T,
                                      const double* bc_u, int which, double* nu_out,
                                      void* stream)
{
    using namespace rtlbfs;
    if (nx < 1 || ny < 1 || nx > kNoAllocMaxN || ny > kNoAllocMaxN) return RTLBFS_ERR_ARG;
    if (!xf || !yf || !rho || !u || !v || !T || !bc_kind || !bc_T || !bc_u || !nu_out)
        return RTLBFS_ERR_ARG;
    if (which < kNuWest || which > kNuHalf || (which == kNuHalf && (nx % 2))) return RTLBFS_ERR_ARG;
    if (!(nu > 0) || !(chi > 0) || !(kappa > 0) || !(dT > 0)) return RTLBFS_ERR_ARG;
    for (int i = 0; i < nx; ++i)
        if (!(xf[i + 1] > xf[i])) return RTLBFS_ERR_ARG;
    for (int j = 0; j < ny; ++j)
        if (!(yf[j + 1] > yf[j])) return RTLBFS_ERR_ARG;
    for (int s = 0; s < 4; ++s)
        if (bc_kind[s] < 0 || bc_kind[s] > 2) return RTLBFS_ERR_ARG;
    if ((bc_kind[0] == kPeriodic) != (bc_kind[1] == kPeriodic) ||
        (bc_kind[2] == kPeriodic) != (bc_kind[3] == kPeriodic))
        return RTLBFS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // once per device, with that device current: the scratch array's address
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RTLBFS_ERR_CUDA;
    void* base = g_noalloc_ptr[dev].load();
    if (!base) {
        if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || !base)
            return RTLBFS_ERR_CUDA;
        g_noalloc_ptr[dev].store(base);
    }
    NoAllocScratch* sc = static_cast<NoAllocScratch*>(base);

    // descriptor of the caller's cavity (fields used as buffer 0)
    CavityDesc d;
    std::memset(&d, 0, sizeof(d));
    d.nx = nx;
    d.ny = ny;
    d.pitch = nx;
    for (int s = 0; s < 4; ++s) {
        d.kind[s] = bc_kind[s];
        d.bcT[s] = bc_T[s];
        d.bcU[s] = bc_u[s];
    }
    d.nu = nu;
    d.chi = chi;
    d.dT = dT;
    d.f[0][0] = const_cast<double*>(rho);
    d.f[0][1] = const_cast<double*>(u);
    d.f[0][2] = const_cast<double*>(v);
    d.f[0][3] = const_cast<double*>(T);
    noalloc_setup_kernel<<<1, 1, 0, st>>>(d, &sc->desc, &sc->ctl);
    // the face coordinates are caller-owned pageable host memory: each copy
    // has read its source when it returns
    if (cudaMemcpyAsync(sc->xf, xf, sizeof(double) * (nx + 1), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(sc->yf, yf, sizeof(double) * (ny + 1), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return RTLBFS_ERR_CUDA;
    noalloc_lines_kernel<<<1, 256, 0, st>>>(sc->xf, nx, bc_kind[0] == kPeriodic, kappa, nu, chi,
                                            sc->xl, sc->xc);
    noalloc_lines_kernel<<<1, 256, 0, st>>>(sc->yf, ny, bc_kind[2] == kPeriodic, kappa, nu, chi,
                                            sc->yl, sc->yc);
    NuLines ln;
    ln.xl = sc->xl;
    ln.yl = sc->yl;
    ln.xc = sc->xc;
    ln.yc = sc->yc;
    long long count;
    double scale = 1.0 / (chi * dT);
    if (which == kNuWest || which == kNuEast || which == kNuHalf) count = ny;
    else if (which == kNuSouth || which == kNuNorth) count = nx;
    else {
        count = (long long)nx * ny;
        scale /= (xf[nx] - xf[0]);
    }
    int blocks = (int)((count + 255) / 256);
    blocks = blocks > kNoAllocPartials ? kNoAllocPartials : (blocks < 1 ? 1 : blocks);
    nusselt_partial_kernel<StoreRho><<<blocks, 256, 0, st>>>(&sc->desc, &sc->ctl, 0, ln, which,
                                                            sc->partial);
    sum_partials_kernel<<<1, 256, 0, st>>>(sc->partial, blocks, scale, nu_out);
    g_launches += 5;
    return cudaGetLastError() == cudaSuccess ? RTLBFS_OK : RTLBFS_ERR_CUDA;
}
