// rtlbfs_kernels.h -- launchers of the device kernels (rtlbfs_step.cu) as
// seen from the host code of the library (rtlbfs_capi.cu).
#pragma once

#include <cuda_runtime.h>

#include "rtlbfs_dev.cuh"

namespace rtlbfs {

#ifndef RTLBFS_STEP_THREADS
#define RTLBFS_STEP_THREADS 256
#endif
#ifndef RTLBFS_TILE_X
#define RTLBFS_TILE_X 32
#endif
#ifndef RTLBFS_TILE_Y
#define RTLBFS_TILE_Y 16
#endif
#ifndef RTLBFS_MIN_BLOCKS_FP32
#define RTLBFS_MIN_BLOCKS_FP32 4
#endif
constexpr int kStepThreads = RTLBFS_STEP_THREADS;  // threads of a step block
constexpr int kTileX = RTLBFS_TILE_X;              // cells of a tile along x
constexpr int kTileY = RTLBFS_TILE_Y;              // cells of a tile along y
constexpr int kMinBlocksFP32 = RTLBFS_MIN_BLOCKS_FP32;  // resident blocks per SM to aim for

#ifndef RTLBFS_PAIR_FACES
#define RTLBFS_PAIR_FACES 0  // 1: x- and y-face in one packed FP32x2 evaluation
#endif
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

size_t step_smem(int precision);
cudaError_t step_prepare(int precision);
cudaError_t step_occupancy(int precision, int* blocks_per_sm);
cudaError_t launch_step(int precision, int grid, cudaStream_t s, const CavityDesc* descs,
                        CavityCtl* ctls, const int4* tiles, const int* ntiles);
cudaError_t march_prepare(int precision);
cudaError_t march_occupancy(int precision, int* blocks_per_sm);
cudaError_t launch_march(int precision, int grid, cudaStream_t s, const CavityDesc* descs,
                         CavityCtl* ctls, const int4* units, const int* nunits);
cudaError_t launch_nusselt(int precision, cudaStream_t s, const CavityDesc* descs,
                           const CavityCtl* ctls, int slot, const NuLines& ln, int which,
                           long long count, double scale, double* partial, int max_blocks,
                           double* out);
cudaError_t launch_state_in(int precision, cudaStream_t s, const double* st, int nx, int ny,
                            int pitch, void* cells, int* bad);
cudaError_t launch_state_out(int precision, cudaStream_t s, double* st, int nx, int ny,
                             int pitch, const void* cells);
cudaError_t launch_arm(cudaStream_t s, CavityCtl* ctls, int slot, long long nsteps, double tol,
                       int reset_counter);

}  // namespace rtlbfs
