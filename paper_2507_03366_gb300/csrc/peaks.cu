// peaks.cu -- FMA-chain kernels that measure the FP32 (scalar and packed
// f32x2) and FP64 FMA throughput of the GPU for the rooflines of the stage
// kernel (include/eulbfs_peaks.h).
#include <cuda_runtime.h>

#include "eulbfs.h"
#include "eulbfs_internal.h"
#include "eulbfs_peaks.h"

namespace eulbfs {
namespace {

constexpr int kChains = 32;        // independent FMA chains per thread (hides the FMA latency)
constexpr int kPeakThreads = 256;

__device__ __forceinline__ float fma_op(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_op(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 fma_op(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ float seed_of(float, int t, int k) { return 1e-3f * (float)(t & 63) + (float)k; }
__device__ __forceinline__ double seed_of(double, int t, int k) { return 1e-3 * (double)(t & 63) + (double)k; }
__device__ __forceinline__ float2 seed_of(float2, int t, int k) {
    return make_float2(1e-3f * (float)(t & 63) + (float)k, 1e-3f * (float)(t & 31) - (float)k);
}
__device__ __forceinline__ float sum_of(float a, float b) { return a + b; }
__device__ __forceinline__ double sum_of(double a, double b) { return a + b; }
__device__ __forceinline__ float2 sum_of(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// b and c are kernel arguments, so the compiler cannot fold the chains; the
// sum of the chains is stored by every thread, so none of them is dead.
template <class T>
__global__ void __launch_bounds__(kPeakThreads) fma_chain_kernel(T* out, long long iters, T b, T c) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed_of(T{}, threadIdx.x, k);
#pragma unroll 4
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma_op(a[k], b, c);
    }
    T s = a[0];
#pragma unroll
    for (int k = 1; k < kChains; ++k) s = sum_of(s, a[k]);
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int run_peak(long long iters, cudaStream_t st, T b, T c, double fma_per_lane, double* flops, double* ms,
             double* winst) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<T>, kPeakThreads, 0);
    if (e != cudaSuccess) return set_error(EULBFS_ECUDA, cudaGetErrorString(e));
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    T* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, sizeof(T) * (size_t)grid * kPeakThreads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        fma_chain_kernel<T><<<grid, kPeakThreads, 0, st>>>(out, iters, b, c);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return set_error(EULBFS_ECUDA, cudaGetErrorString(e));
    const double threads = (double)grid * kPeakThreads;
    const double fmas = threads * (double)kChains * (double)iters * fma_per_lane;
    *ms = t;
    *flops = 2.0 * fmas / (t * 1e-3);
    *winst = threads / 32.0 * (double)kChains * (double)iters / (t * 1e-3);
    return EULBFS_OK;
}

}  // namespace
}  // namespace eulbfs

extern "C" int eulbfs_peak_fma(int kind, long long iters, void* stream, double* flops_per_s, double* ms,
                               double* fma_warp_inst_per_s) {
    using namespace eulbfs;
    if (iters < 1 || !flops_per_s || !ms || !fma_warp_inst_per_s)
        return set_error(EULBFS_EINVAL, "iters must be >= 1 and the outputs non-null");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (kind) {
        case EULBFS_PEAK_FP32:
            return run_peak<float>(iters, st, 0.999999f, 1e-7f, 1.0, flops_per_s, ms, fma_warp_inst_per_s);
        case EULBFS_PEAK_FP32X2:
            return run_peak<float2>(iters, st, make_float2(0.999999f, 0.9999995f), make_float2(1e-7f, -1e-7f), 2.0,
                                    flops_per_s, ms, fma_warp_inst_per_s);
        case EULBFS_PEAK_FP64:
            return run_peak<double>(iters, st, 0.999999999, 1e-12, 1.0, flops_per_s, ms, fma_warp_inst_per_s);
        default:
            return set_error(EULBFS_EINVAL, "unknown peak kind");
    }
}
