// pcm_energy_noalloc: the solvation energy (A q, then three dot products)
// for callers that cannot allocate device memory.  Its scratch lives in a
// file-scope device array instead of buffers from cudaMalloc.
//
// Who needs it: a host program whose device memory is owned by its own
// allocator (a framework memory pool that has reserved the GPU, an embedded
// solver with a fixed memory budget) cannot let a library call cudaMalloc:
// the call may fail when the pool holds the memory, and cudaMalloc/cudaFree
// may synchronise the device in the middle of the caller's work.  Such a
// caller keeps A, B z, c and q in its own buffers and passes them in.
//
// Two kernels: the first writes y = A q into the scratch array (one warp per
// row), the second reads y back and forms q.y, Bz.q and c.q in one block in a
// fixed order, so the result does not depend on the first kernel's grid.
//
// The scratch array is part of the library's device image: every GPU that
// loads the library holds it (65536 doubles = 512 KiB) until the process
// exits.  All calls share it; each call writes every value of y it later
// reads, so nothing has to be cleared between calls, but two calls whose
// kernels overlap on the GPU (different streams, or another host thread)
// race on it and give wrong results.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "context.h"

namespace pcm {
namespace noalloc {

constexpr int MAX_M = 65536;          // largest number of surface points accepted (length of y)
constexpr int NT = 256;               // threads per block of the row kernel (one row per warp at a time)
constexpr int ROW_BLOCKS = 1024;      // most blocks of the row kernel (rows are grid-strided beyond)
constexpr int DOT_NT = 1024;          // threads of the single dot-product block
constexpr int MAX_DEVICES = 64;

// scratch: y = A q
static __device__ __align__(256) double g_scratch[MAX_M];

static std::mutex g_mu;
static double *g_scratch_addr[MAX_DEVICES];  // device address of g_scratch, per device

// y_row = sum_col A[row][col] q_col for rows b*8+w, b*8+w+8*nb, ... (warp w of block b)
__global__ void __launch_bounds__(NT) energy_rows_kernel(int M, int lda, const double *__restrict__ A,
                                                         const double *__restrict__ q, double *__restrict__ y)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int row = blockIdx.x * (NT / 32) + w; row < M; row += gridDim.x * (NT / 32)) {
        const double *a = A + (size_t)row * lda;
        double s = 0.0;
        for (int col = lane; col < M; col += 32) s = fma(a[col], q[col], s);
        s = warp_sum(s);
        if (lane == 0) y[row] = s;
    }
}

// E = (Bz)^T q + c^T q + q^T y / (2 f): each thread sums a strided slice,
// then warps and the block combine in a fixed order.
__global__ void __launch_bounds__(DOT_NT) energy_dots_kernel(int M, const double *__restrict__ y,
                                                             const double *__restrict__ Bz,
                                                             const double *__restrict__ c,
                                                             const double *__restrict__ q, double f,
                                                             double *__restrict__ E)
{
    double qAq = 0.0, bzq = 0.0, cq = 0.0;
    for (int k = threadIdx.x; k < M; k += DOT_NT) {
        const double qk = q[k];
        qAq = fma(qk, y[k], qAq);
        bzq = fma(Bz[k], qk, bzq);
        cq = fma(c[k], qk, cq);
    }
    qAq = warp_sum(qAq);
    bzq = warp_sum(bzq);
    cq = warp_sum(cq);
    __shared__ double sh[3][DOT_NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][w] = qAq;
        sh[1][w] = bzq;
        sh[2][w] = cq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < DOT_NT / 32; ++i)
            for (int j = 0; j < 3; ++j) t[j] += sh[j][i];
        *E = t[1] + t[2] + t[0] / (2.0 * f);
    }
}

// Device address of g_scratch on the current device, looked up once per
// device with that device current.  The address is kept for the life of the
// process: the library must not be used across a reset of the device
// (cudaDeviceReset), after which its device image may be loaded elsewhere.
static int scratch_address(double **out)
{
    int dev = -1;
    PCM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_last_error("pcm_energy_noalloc: device ordinal %d is outside 0..%d", dev, MAX_DEVICES - 1);
        return PCM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            set_last_error("pcm_energy_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                           cudaGetErrorString(e));
            return PCM_ERR_CUDA;
        }
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return PCM_OK;
}

}  // namespace noalloc
}  // namespace pcm

extern "C" int pcm_energy_noalloc(int M, const double *A, int lda, const double *Bz, const double *c,
                                  const double *q, double f, double *E, void *stream)
{
    using namespace pcm::noalloc;
    if (M < 1 || !A || !Bz || !c || !q || !E || lda < M || !(f > 0.0)) {
        pcm::set_last_error("pcm_energy_noalloc: bad arguments (M >= 1, lda >= M, f > 0, non-null pointers)");
        return PCM_ERR_ARG;
    }
    if (M > MAX_M) {
        pcm::set_last_error("pcm_energy_noalloc: M = %d exceeds the fixed scratch limit of %d surface points; "
                            "use pcm_energy", M, MAX_M);
        return PCM_ERR_ARG;
    }
    double *y = nullptr;
    int st = scratch_address(&y);
    if (st != PCM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = std::min(ROW_BLOCKS, (M + NT / 32 - 1) / (NT / 32));
    energy_rows_kernel<<<nb, NT, 0, s>>>(M, lda, A, q, y);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        energy_dots_kernel<<<1, DOT_NT, 0, s>>>(M, y, Bz, c, q, f, E);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        pcm::set_last_error("pcm_energy_noalloc: launch failed: %s", cudaGetErrorString(e));
        return PCM_ERR_CUDA;
    }
    return PCM_OK;
}
