// rtlbfs_persist.cu -- the tile step of rtlbfs_step.cu in persistent form:
// one launch advances one cavity by many explicit time steps (arXiv
// 2202.13449, Section 3.2), with the same arithmetic (tile_step) and the
// same stop test after every step.
//
// Launch: cooperative, one block per tile, every tile resident at once.
// Each block loops over the steps of the launch.  Before step k it waits
// for the eight tiles around its own (with the periodic wrap) to have
// finished step k - 1: their cells are its halo, and once they are done
// with step k - 1 they no longer read the buffer step k overwrites.  There
// is no grid-wide barrier, so the blocks of an SM drift apart and overlap
// one another's load, face and update phases.
//
// Run control: the residual sums of step k go to slot k % 3 of
// PersistCtl; the last tile to finish step k finalises it exactly as the
// launch-per-step kernels do (R_u, R_T, step counter, current buffer, stop
// test) and publishes fin = k.  A block starts step k only once step k - 2
// is final, because step k overwrites the buffer that holds the state
// after step k - 2.  A block therefore runs at most one step past the last
// stop test.  A step taken after a stop is discarded (the finaliser skips
// it, and the current buffer still holds the state at the stop), so the run
// stops at the same step and state as the launch-per-step kernels.
//
// Every wait is bounded (about a second).  A block whose wait runs out
// marks the run stalled; the other blocks see the mark in their own waits
// and return, and the host reports an error.
#include <cuda_runtime.h>

#include "rtlbfs_dev.cuh"
#include "rtlbfs_kernels.h"
#include "rtlbfs_tile.cuh"

namespace rtlbfs {

namespace {

constexpr unsigned long long kWaitNs = 1000000000ull;  // a wait gives up after a second
constexpr long long kSpinLimit = 1LL << 24;  // and after this many tries in any case

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One warp waits until every lane's condition holds: *p >= v, or *q != 0
// when the lane passes q (lanes without a condition pass p = nullptr).
// False when the run has stalled: this wait ran out (it then marks
// *stalled) or another block's did.  The lanes poll in parallel, so a wait
// on nine flags costs one L2 round trip when they are already set.
__device__ bool warp_wait(const int* p, int v, const int* q, int* stalled)
{
    auto holds = [&]() { return p == nullptr || ld_acquire(p) >= v || (q && ld_acquire(q)); };
    const unsigned long long t0 = global_ns();
    bool ok = holds();
    for (long long it = 0; it < kSpinLimit; ++it) {
        if (__all_sync(0xffffffffu, ok)) return true;
        const int st = (threadIdx.x & 31) == 0 ? ld_acquire(stalled) : 0;
        if (__shfl_sync(0xffffffffu, st, 0)) return false;
        const bool late = (threadIdx.x & 31) == 0 && global_ns() - t0 > kWaitNs;
        if (__shfl_sync(0xffffffffu, (int)late, 0)) break;
        __nanosleep(64);
        if (!ok) ok = holds();
    }
    if ((threadIdx.x & 31) == 0) atomicExch(stalled, 1);
    return false;
}

}  // namespace

template <class P, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT, MinBlocks<P, NT>::value)
persist_kernel(const CavityDesc* __restrict__ dp, CavityCtl* __restrict__ ctl,
               const int4* __restrict__ tiles, int* __restrict__ tstep,
               PersistCtl* __restrict__ pc, int nsteps, int withhold)
{
    using Sm = TileSmem<P, TX, TY, NT>;
    using S = typename P::S;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    Sm& sm = *reinterpret_cast<Sm*>(smem_raw);
    const int tid = threadIdx.x, t = blockIdx.x, ntiles = gridDim.x;
    const int4 tile = tiles[t];
    const int i0 = tile.y, j0 = tile.z;
    stage_tile(sm, dp, i0, j0);  // descriptor and mesh lines: fixed for the launch
    const int ntx = dp->tiles_x, nty = dp->tiles_y;
    const int tix = t % ntx, tiy = t / ntx;
    const bool xper = dp->kind[kSideW] == kPeriodic, yper = dp->kind[kSideS] == kPeriodic;
    // the buffer holding the state at launch (no step of this launch is
    // final before every block has read it: each block's step 1 counts)
    const int c0 = *reinterpret_cast<volatile const int*>(&ctl->cur);

    // lane l < 8 of warp 0 watches the l-th of the (up to) eight tiles
    // around this one, lane 8 the last final step
    int nb = -1;
    if (tid < 8) {
        const int dx = (tid < 3 ? tid : tid < 5 ? (tid == 3 ? 0 : 2) : tid - 5) - 1;
        const int dy = (tid < 3 ? 0 : tid < 5 ? 1 : 2) - 1;
        int a = tix + dx, b = tiy + dy;
        bool ok = true;
        if (a < 0 || a >= ntx) {
            ok = xper;
            a = (a + ntx) % ntx;
        }
        if (b < 0 || b >= nty) {
            ok = ok && yper;
            b = (b + nty) % nty;
        }
        if (ok && b * ntx + a != t) nb = b * ntx + a;
    }

    for (int k = 1; k <= nsteps; ++k) {
        if (tid < 32) {
            // lanes 0-7: the neighbour has finished step k - 1, or the run
            // has stopped (a stop is final for a step before k, and a
            // neighbour that saw it has returned); lane 8: step k - 2 is
            // final, after which the stop flag below is the whole story
            const int* p = nullptr;
            const int* q = nullptr;
            int v = 0;
            if (tid < 8 && nb >= 0 && k >= 2) {
                p = &tstep[nb];
                v = k - 1;
                q = &ctl->done;
            } else if (tid == 8 && k >= 3) {
                p = &pc->fin;
                v = k - 2;
            }
            int go = warp_wait(p, v, q, &pc->stalled) ? 1 : -1;
            __syncwarp();  // the lanes' acquires before lane 0's reads
            if (tid == 0) {
                __threadfence();
                if (go == 1 && *reinterpret_cast<volatile const int*>(&ctl->done)) go = 0;
                sm.last = go;
            }
        }
        __syncthreads();
        if (sm.last != 1) break;  // uniform: stopped, or stalled
        const int rb = c0 ^ ((k - 1) & 1);  // buffer with the state after step k - 1
        tile_step<P, TX, TY, NT, 0, true>(sm, &sm.desc, i0, j0,
                                          static_cast<const Vec4<S>*>(dp->f[rb][0]),
                                          static_cast<Vec4<S>*>(dp->f[rb ^ 1][0]), true);
        __syncthreads();
        double a[4];
        if (tid < 32) tile_sums(sm, a);
        if (tid == 0) {
            double* acc = pc->acc[k % 3];
            for (int q = 0; q < 4; ++q) atomicAdd(&acc[q], a[q]);
            __threadfence();  // the tile's new state (all threads, before the barrier) and sums
            if (t != withhold) st_release(&tstep[t], k);
            const unsigned prev = atomicAdd(&pc->arrive[k % 3], 1u);
            if (prev == (unsigned)ntiles - 1u) {
                // last tile of step k: finalise it, unless the run stopped earlier
                __threadfence();
                volatile double* va = acc;
                if (!*reinterpret_cast<volatile int*>(&ctl->done)) {
                    const double su = va[0], du = va[1], sT = va[2], dT = va[3];
                    const double ru = du > 0.0 ? sqrt(su) / sqrt(du) : INFINITY;
                    const double rT = dT > 0.0 ? sqrt(sT) / sqrt(dT) : INFINITY;
                    ctl->res[0] = ru;
                    ctl->res[1] = rT;
                    ctl->steps += 1;
                    ctl->cur = rb ^ 1;
                    int status = kRunning;
                    if (isnan(ru) || isnan(rT) || isnan(su) || isnan(sT)) status = kDiverged;
                    else if (fmax(ru, rT) < ctl->tol) status = kConverged;
                    else if (ctl->steps >= ctl->max_steps) status = kMaxSteps;
                    ctl->status = status;
                    if (status != kRunning) ctl->done = 1;
                }
                for (int q = 0; q < 4; ++q) va[q] = 0.0;
                *reinterpret_cast<volatile unsigned*>(&pc->arrive[k % 3]) = 0u;
                __threadfence();
                st_release(&pc->fin, k);
            }
        }
    }
}

template <class P, int TY>
struct PersistKernel {
    static constexpr int NT = TileThreads<P, TY>::value;
    static constexpr size_t smem = sizeof(TileSmem<P, kTileX, TY, NT>);
    static constexpr auto fn = persist_kernel<P, kTileX, TY, NT>;
    static cudaError_t prepare()
    {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    static cudaError_t occupancy(int* blocks)
    {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, NT, smem);
    }
    static cudaError_t launch(int ntiles, cudaStream_t s, const CavityDesc* d, CavityCtl* c,
                              const int4* tiles, int* tstep, PersistCtl* pc, int nsteps,
                              int withhold)
    {
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)ntiles);
        cfg.blockDim = dim3((unsigned)NT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, fn, d, c, tiles, tstep, pc, nsteps, withhold);
    }
};

template <class Op>
static cudaError_t with_persist_kernel(int precision, int tile_h, Op op)
{
    if (precision == 0) {
        switch (tile_h) {
        case 16: return op(PersistKernel<StoreD, 16>());
        case 8: return op(PersistKernel<StoreD, 8>());
        case 4: return op(PersistKernel<StoreD, 4>());
        case 2: return op(PersistKernel<StoreD, 2>());
        default: return cudaErrorInvalidValue;
        }
    }
    switch (tile_h) {
    case 16: return op(PersistKernel<StoreQ, 16>());
    case 14: return op(PersistKernel<StoreQ, 14>());
    case 12: return op(PersistKernel<StoreQ, 12>());
    case 10: return op(PersistKernel<StoreQ, 10>());
    case 8: return op(PersistKernel<StoreQ, 8>());
    case 4: return op(PersistKernel<StoreQ, 4>());
    case 2: return op(PersistKernel<StoreQ, 2>());
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t persist_prepare(int precision)
{
    for (int h : kTileHeights) {
        if (!tile_height_ok(precision, h)) continue;
        cudaError_t e = with_persist_kernel(precision, h, [](auto k) { return k.prepare(); });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t persist_occupancy(int precision, int tile_h, int* blocks_per_sm)
{
    return with_persist_kernel(precision, tile_h,
                               [&](auto k) { return k.occupancy(blocks_per_sm); });
}

cudaError_t launch_persist(int precision, int tile_h, int ntiles, cudaStream_t s,
                           const CavityDesc* desc, CavityCtl* ctl, const int4* tiles, int* tstep,
                           PersistCtl* pc, int nsteps, int withhold)
{
    return with_persist_kernel(precision, tile_h, [&](auto k) {
        return k.launch(ntiles, s, desc, ctl, tiles, tstep, pc, nsteps, withhold);
    });
}

}  // namespace rtlbfs
