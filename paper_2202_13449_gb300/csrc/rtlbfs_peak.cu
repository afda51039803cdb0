// rtlbfs_peak.cu -- the FMA rates the rooflines are stated against
// (rtlbfs_measure.h): independent FMA chains on every SM, timed with CUDA
// events.
#include <cuda_runtime.h>

#include "rtlbfs.h"
#include "rtlbfs_measure.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// The chains start from the thread index and a runtime multiplier, so the
// compiler can neither fold nor drop them; one sum per block reaches memory.
template <typename T>
__global__ void __launch_bounds__(kThreads) fma_kernel(int reps, T a, T b, float* sink)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * b;
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-1.2345)) *sink = float(s);
}

__global__ void __launch_bounds__(kThreads) fma2_kernel(int reps, float a, float b, float* sink)
{
    float2 x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(float(threadIdx.x + c) * b, float(c) * b);
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -1.2345f) *sink = s;
}

}  // namespace

extern "C" int rtlbfs_fma_rate(int kind, int reps, double* fma_per_s, double* ms)
{
    if (kind < RTLBFS_RATE_FP32 || kind > RTLBFS_RATE_FP64 || reps < 1 || !fma_per_s || !ms)
        return RTLBFS_ERR_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RTLBFS_ERR_CUDA;
    cudaError_t e;
    if (kind == RTLBFS_RATE_FP32)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_kernel<float>, kThreads, 0);
    else if (kind == RTLBFS_RATE_FP32X2)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma2_kernel, kThreads, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_kernel<double>, kThreads, 0);
    if (e != cudaSuccess || per_sm < 1) return RTLBFS_ERR_CUDA;
    const int grid = sms * per_sm;
    float* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return RTLBFS_ERR_OOM;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    int rc = RTLBFS_OK;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) {
        rc = RTLBFS_ERR_CUDA;
    } else {
        auto launch = [&]() {
            if (kind == RTLBFS_RATE_FP32)
                fma_kernel<float><<<grid, kThreads>>>(reps, 0.999999f, 1e-7f, sink);
            else if (kind == RTLBFS_RATE_FP32X2)
                fma2_kernel<<<grid, kThreads>>>(reps, 0.999999f, 1e-7f, sink);
            else
                fma_kernel<double><<<grid, kThreads>>>(reps, 0.999999, 1e-7, sink);
        };
        launch();  // untimed: clocks up, code resident
        cudaEventRecord(t0);
        launch();
        cudaEventRecord(t1);
        float t = 0.0f;
        if (cudaEventSynchronize(t1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&t, t0, t1) != cudaSuccess || t <= 0.0f) {
            rc = RTLBFS_ERR_CUDA;
        } else {
            const double per_thread = (double)reps * kChains * (kind == RTLBFS_RATE_FP32X2 ? 2 : 1);
            *fma_per_s = per_thread * grid * kThreads / (t * 1e-3);
            *ms = t;
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(sink);
    return rc;
}
