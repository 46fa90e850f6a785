// Pipe-peak microbenchmark: the FP32 FMA (scalar and packed FP32x2) and FP64
// FMA throughput of the GPU, measured with independent FMA chains (eight per
// thread, no memory traffic)
// over a grid of several blocks per SM, timed with CUDA events.  The integral
// kernels' roofline fractions are reported against these measured rates beside
// the nominal ones (unit counts times the clock).
#include <cuda_runtime.h>

#include "context.h"
#include "f2.cuh"

namespace pcm {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(int iters, T seed, T *__restrict__ out)
{
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed + (T)(threadIdx.x + i);
    const T m = (T)0.999999, c = (T)1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = a[i] * m + c;   // one FMA each
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == (T)-12345) out[0] = s;   // keeps the chains live; never true
}

__global__ void __launch_bounds__(256) fma2_chains_kernel(int iters, float seed, float *__restrict__ out)
{
    f2 a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = f2(seed + (float)(threadIdx.x + i));
    const f2 m(0.999999f), c(1e-7f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma2(a[i], m, c);   // one packed FMA (two lanes) each
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i].v.x + a[i].v.y;
    if (s == -12345.f) out[0] = s;   // keeps the chains live; never true
}

}  // namespace pcm

extern "C" int pcm_pipe_peak(int device, int which, double *tflops)
{
    using namespace pcm;
    if (!tflops || which < 0 || which > 2) {
        set_last_error("pcm_pipe_peak: which must be 0 (FP32), 1 (FP64) or 2 (packed FP32x2)");
        return PCM_ERR_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    void *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = PCM_OK;
    const int blocks = nsm * 8, threads = 256;
    const int iters = which == 1 ? 1 << 11 : 1 << 16;
    float ms = 0.f;
    if (cudaMalloc(&out, 16) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        set_last_error("pcm_pipe_peak: CUDA set-up failed");
        st = PCM_ERR_CUDA;
    } else {
        for (int rep = 0; rep < 2; ++rep) {   // the first launch warms up
            cudaEventRecord(e0);
            if (which == 0)
                fma_chains_kernel<float><<<blocks, threads>>>(iters, 1.f, (float *)out);
            else if (which == 1)
                fma_chains_kernel<double><<<blocks, threads>>>(iters, 1.0, (double *)out);
            else
                fma2_chains_kernel<<<blocks, threads>>>(iters, 1.f, (float *)out);
            cudaEventRecord(e1);
        }
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            !(ms > 0.f)) {
            set_last_error("pcm_pipe_peak: timing failed");
            st = PCM_ERR_CUDA;
        } else {
            const double flops = (which == 2 ? 4.0 : 2.0) * 8.0 * (double)iters * (double)blocks * threads;
            *tflops = flops / (ms * 1e-3) / 1e12;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    cudaSetDevice(prev);
    return st;
}
