// lbm_peak_fma: the measured FMA throughput of the current GPU in FP32 or
// FP64, the denominator against which the arithmetic-bound kernels (the FP32
// heat kernel, the whole FP64 path) report their fraction.  Not part of the
// method.
//
// Every thread runs eight independent chains a <- a b + c with 0 < b < 1 and
// c > 0, so the values stay positive and finite and every iteration issues
// eight dependent-free FMAs; the grid fills every SM with 2048 threads.  One
// untimed launch, then one launch timed with CUDA events on a private stream.
#include <cuda_runtime.h>

#include <string>

#include "lbm.h"
#include "lbm_launch.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;
constexpr int kChains = 8;

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T *out, int iters, T b, T c) {
    T a[kChains];
    #pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = T(1e-3) * T(threadIdx.x + j + 1);
    #pragma unroll 8
    for (int i = 0; i < iters; i++) {
        #pragma unroll
        for (int j = 0; j < kChains; j++) a[j] = fma_rn(a[j], b, c);
    }
    T s = T(0);
    #pragma unroll
    for (int j = 0; j < kChains; j++) s += a[j];
    // never true (all chains stay positive); keeps the chains from being removed
    if (s < T(0)) out[blockIdx.x] = s;
}

template <class T>
int run(int device, int iters, double *tflops) {
    int prev = 0, dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&prev);
    dev = device >= 0 ? device : prev;
    if (e == cudaSuccess && dev != prev) e = cudaSetDevice(dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        if (dev != prev) cudaSetDevice(prev);
        lbmgb::set_global_error(std::string("lbm_peak_fma: no usable device: ") + cudaGetErrorString(e));
        return LBM_E_CUDA;
    }
    const int blocks = sms * kBlocksPerSM;
    T *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    e = cudaMalloc(&out, sizeof(T) * blocks);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        const T b = T(0.999999), c = T(1e-7);
        k_fma_chains<T><<<blocks, kThreads, 0, s>>>(out, iters, b, c);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            k_fma_chains<T><<<blocks, kThreads, 0, s>>>(out, iters, b, c);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    if (dev != prev) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        lbmgb::set_global_error(std::string("lbm_peak_fma: ") + cudaGetErrorString(e));
        return LBM_E_CUDA;
    }
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    *tflops = ms > 0.0f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_peak_fma(int32_t device, int32_t bits, int32_t iters, double *tflops) {
    if (!tflops || (bits != 32 && bits != 64) || iters < 1 || iters > (1 << 24)) {
        lbmgb::set_global_error("lbm_peak_fma: bits must be 32 or 64, iters in 1 .. 2^24, tflops not NULL");
        return LBM_E_INVAL;
    }
    return bits == 64 ? run<double>(device, iters, tflops) : run<float>(device, iters, tflops);
}
