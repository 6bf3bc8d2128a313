// gc_peak.cu -- fused multiply-add throughput of this GPU in FP32 and FP64: the peaks the
// push kernels are measured against (the FP32 push is bound by FP32 instruction issue, the
// plain FP64 push by the double-precision pipe). Each thread runs CH independent FMA chains
// on registers, enough resident warps per SM to hide the FMA latency; the launch is timed with
// CUDA events, best of ten.
#include <cuda_runtime.h>

#include "gc_internal.h"
#include "gcpush.h"

namespace {

constexpr int kChains = 8;

// written only if a chain's sum equals -1, which these inputs never give; the test keeps
// every chain live without a store per thread
__device__ float g_fma_sink_f;
__device__ double g_fma_sink_d;

template <typename T> __device__ __forceinline__ T *fma_sink();
template <> __device__ __forceinline__ float *fma_sink<float>() { return &g_fma_sink_f; }
template <> __device__ __forceinline__ double *fma_sink<double>() { return &g_fma_sink_d; }

constexpr int kBlock = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kBlock) fma_rate_kernel(int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += x[c];
    if (s == (T)-1)
        *fma_sink<T>() = s;
}

template <typename T>
int rate(int sms, int iters, cudaStream_t st, double *tflops)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GC_ERR_CUDA;
    }
    const int blocks = sms * kBlocksPerSM;
    const T a = (T)0.9999999, b = (T)1e-7;
    float best = 0.0f;
    int rc = GC_OK;
    for (int k = 0; k < 11 && rc == GC_OK; ++k) { // launch 0 warms up
        cudaEventRecord(e0, st);
        fma_rate_kernel<T><<<blocks, kBlock, 0, st>>>(iters, a, b);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = GC_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (k > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GC_OK || best <= 0.0f) return GC_ERR_CUDA;
    const double flop = 2.0 * kChains * (double)iters * blocks * kBlock;
    *tflops = flop / (best * 1e-3) / 1e12;
    return GC_OK;
}

} // namespace

extern "C" int gc_fma_peak(int device, double *fp32_tflops, double *fp64_tflops)
{
    if (!fp32_tflops || !fp64_tflops) {
        gcp::set_last_error("gc_fma_peak: null argument");
        return GC_ERR_INVALID;
    }
    int prev = 0, n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
        gcp::set_last_error("gc_fma_peak: no such device");
        return GC_ERR_INVALID;
    }
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t st = nullptr;
    int rc = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess ? GC_OK : GC_ERR_CUDA;
    // about 10 ms per launch at the nominal rates (80 TFLOP/s FP32, 1.2 TFLOP/s FP64); the
    // FP64 rate first, since the FP32 chains draw the GPU to its power limit and the clock
    // dip that follows would otherwise land on the FP64 launches
    if (rc == GC_OK) rc = rate<double>(sms, 1 << 11, st, fp64_tflops);
    if (rc == GC_OK) rc = rate<float>(sms, 1 << 17, st, fp32_tflops);
    if (st) cudaStreamDestroy(st);
    if (rc != GC_OK) {
        cudaGetLastError();
        gcp::set_last_error("gc_fma_peak: CUDA error in the rate kernels");
    }
    cudaSetDevice(prev);
    return rc;
}
