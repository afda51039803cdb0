// rtlbfs_kernels.h -- launchers of the device kernels (rtlbfs_step.cu) as
// seen from the host code of the library (rtlbfs_capi.cu).
#pragma once

#include <cuda_runtime.h>

#include "rtlbfs_dev.cuh"

namespace rtlbfs {

// Tiles of the shared-memory step kernel: kTileX = 32 columns by one of
// the compiled heights below, 16 threads per tile row (two cells per thread
// in the update).  The height is picked per cavity set so that the number of
// tiles fills the SMs evenly (a 512-row mesh in 16-row tiles leaves a third
// of the SMs one tile short); the low heights spread small meshes over many
// SMs, which matters most in FP64, where an SM does 2 FMAs per clock.
constexpr int kTileX = 32;
constexpr int kTileHeights[] = {16, 14, 12, 10, 8, 4, 2};
constexpr int kTileYDefault = 16;
inline bool tile_height_ok(int precision, int h)
{
    if (precision == 0) return h == 16 || h == 8 || h == 4 || h == 2;
    for (int t : kTileHeights)
        if (t == h) return true;
    return false;
}
#ifndef RTLBFS_MARCH_THREADS
#define RTLBFS_MARCH_THREADS 128
#endif
#ifndef RTLBFS_MARCH_MIN_BLOCKS_FP32
#define RTLBFS_MARCH_MIN_BLOCKS_FP32 4
#endif
constexpr int kMarchThreads = RTLBFS_MARCH_THREADS;  // 4 warps per block
constexpr int kMarchMinBlocksFP32 = RTLBFS_MARCH_MIN_BLOCKS_FP32;
constexpr int kStrip = 28;  // interior columns per warp (32 lanes - 2 x 2 halo)

constexpr int kNuWest = 0, kNuEast = 1, kNuSouth = 2, kNuNorth = 3, kNuAvg = 4, kNuHalf = 5;

// FP64 mesh lines of one cavity, for the FP64 reductions.
struct NuLines {
    const FaceLine<double>* xl;
    const FaceLine<double>* yl;
    const CellLine<double>* xc;
    const CellLine<double>* yc;
};

// tile_h: a height tile_height_ok accepts for the precision; scheme: the
// face stage, 0 RTLBFS, 1 TLBFS (tile height kTileYDefault only)
constexpr int kSchemeRTLBFS = 0, kSchemeTLBFS = 1;
cudaError_t step_prepare(int precision);
cudaError_t step_occupancy(int precision, int tile_h, int scheme, int* blocks_per_sm);
// par: parity of the launch within a chain of step launches (launch k of
// a chain reads run header k & 1 and writes the other, see CavityRun)
cudaError_t launch_step(int precision, int tile_h, int scheme, int grid, cudaStream_t s,
                        const CavityDesc* descs, CavityRun* runs, const int4* tiles,
                        const int* ntiles, int par);
cudaError_t march_prepare(int precision);
cudaError_t march_occupancy(int precision, int* blocks_per_sm);
cudaError_t launch_march(int precision, int grid, cudaStream_t s, const CavityDesc* descs,
                         CavityRun* runs, const int4* units, const int* nunits, int par);
// the stop test of the last step of a chain whose next launch would have
// parity par, for cavities 0..n-1: both headers become the tested header
cudaError_t launch_finalize(cudaStream_t s, CavityRun* runs, int n, int par);

// Run control of the persistent tile kernel (rtlbfs_persist.cu), zeroed
// before each launch: the residual sums and arrivals of step k in slot
// k % 3, the last step whose stop test is done, and the stall mark.
struct PersistCtl {
    int fin;
    int stalled;
    unsigned arrive[3];
    int pad;
    double acc[3][4];
};
// One cavity, one block per tile (ntiles of them, all resident: check
// persist_occupancy), nsteps steps; tiles: that cavity's tile list; tstep:
// ntiles ints zeroed before the launch.  withhold >= 0 (tests only): that
// tile never reports its progress, so the waits of its neighbours run out.
cudaError_t persist_prepare(int precision);
cudaError_t persist_occupancy(int precision, int tile_h, int* blocks_per_sm);
cudaError_t launch_persist(int precision, int tile_h, int ntiles, cudaStream_t s,
                           const CavityDesc* desc, CavityCtl* ctl, const int4* tiles, int* tstep,
                           PersistCtl* pc, int nsteps, int withhold);
cudaError_t launch_nusselt(int precision, cudaStream_t s, const CavityDesc* descs,
                           const CavityRun* runs, int slot, const NuLines& ln, int which,
                           long long count, double scale, double* partial, int max_blocks,
                           double* out);
// T_unit: temperature unit of the stored state (stored T = T / T_unit)
cudaError_t launch_state_in(int precision, cudaStream_t s, const double* st, int nx, int ny,
                            int pitch, double T_unit, void* cells, int* bad);
cudaError_t launch_state_out(int precision, cudaStream_t s, double* st, int nx, int ny,
                             int pitch, double T_unit, const void* cells);
// FP32 records: stored temperatures divided by 2^shift (1 <= shift <= 30)
cudaError_t launch_rescale_T(cudaStream_t s, void* cells, long long count, int shift);
// rho = 1, u = v = 0, T = Tcol[i] in every row (one buffer of cell records)
cudaError_t launch_conduction(int precision, cudaStream_t s, const double* Tcol, int nx, int ny,
                              int pitch, void* cells);
cudaError_t launch_arm(cudaStream_t s, CavityRun* runs, int slot, long long nsteps, double tol,
                       int reset_counter);
// arm_kernel over the n slots of a device array of slot indices
cudaError_t launch_arm_list(cudaStream_t s, CavityRun* runs, const int* slots, int n,
                            long long nsteps, double tol);
// runs[slots[k]] = src[k] for k < n (device arrays)
cudaError_t launch_put_runs(cudaStream_t s, CavityRun* runs, const int* slots,
                            const CavityRun* src, int n);

}  // namespace rtlbfs
