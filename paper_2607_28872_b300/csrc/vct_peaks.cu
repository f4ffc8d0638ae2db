// FP32 and FP64 fused multiply-add throughput of this GPU, measured with a
// plain FMA loop (a measurement tool for the roofline of the pair-sum
// kernels; not part of the step's C ABI).  Built into libvct_peaks.so.
//
//   int vct_fma_peak(int fp64, int iters, double *tflops, double *ms)
//
// Runs one launch of 148 x 8 blocks of 256 threads, each thread carrying 8
// independent FMA chains for `iters` iterations (2 flops per FMA), timed
// with CUDA events after one untimed launch.  Returns 0, or the CUDA error.
#include <cuda_runtime.h>

namespace {

constexpr int CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_loop(int iters, T a, T b, T *out)
{
    T acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = T(threadIdx.x + c) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) acc[c] = fma(acc[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c];
    if (s == T(-12345.678)) out[blockIdx.x] = s;   // keeps the loop; never true in practice
}

template <typename T>
int run(int iters, double *tflops, double *ms_out)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    T *out = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(T) * blocks);
    if (e != cudaSuccess) return (int)e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a = 1 - 2^-20, b = 2^-20: each chain converges to 1 without overflow or denormals
    const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 1048576.0);
    k_fma_loop<T><<<blocks, threads>>>(iters, a, b, out);
    cudaEventRecord(e0);
    k_fma_loop<T><<<blocks, threads>>>(iters, a, b, out);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double flops = 2.0 * 16.0 * CHAINS * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    *ms_out = ms;
    return 0;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int vct_fma_peak(int fp64, int iters,
                                                                    double *tflops, double *ms)
{
    if (!tflops || !ms || iters <= 0) return -1;
    return fp64 ? run<double>(iters, tflops, ms) : run<float>(iters, tflops, ms);
}
