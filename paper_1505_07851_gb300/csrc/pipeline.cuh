// Bulk copies from global into shared memory (cp.async.bulk, the TMA's
// non-tensor form) completed on mbarriers, and a ring of NSTAGE buffers with
// "full" barriers (the copy has landed) and "empty" barriers (every consumer
// warp is done with the buffer).  One thread (the producer) issues the copies;
// consumer warps wait only for the buffer they read next, so warps of a block
// may drift apart by up to NSTAGE - 1 tiles instead of meeting at a block
// barrier after every tile.
//
// Every wait is bounded: after a fixed number of polls it returns false, the
// caller sets the device error flag and stops, and the producer lets copies in
// flight land (again with a bounded wait) before its block ends.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pcm {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *mb, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mb)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mb, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mb)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mb)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mb)) : "memory");
}

// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mb)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(mb))
                 : "memory");
}

// Wait for the phase with the given parity to complete; false after a bounded
// number of polls (each poll may suspend the thread for a short while).
__device__ __forceinline__ bool mbar_wait(uint64_t *mb, uint32_t parity)
{
    const uint32_t a = smem_addr(mb);
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// A ring of NSTAGE shared buffers of BUF floats for a sequence of tiles.
// Tile j lives in buffer j % NSTAGE; it is that buffer's (j / NSTAGE)-th use.
template <int NSTAGE, int BUF>
struct TileRing {
    float buf[NSTAGE][BUF];
    uint64_t full[NSTAGE], empty[NSTAGE];

    // thread 0, before a __syncthreads
    __device__ __forceinline__ void init(uint32_t consumer_warps)
    {
        for (int b = 0; b < NSTAGE; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], consumer_warps);
        }
        mbar_init_fence();
    }
    // consumer: tile j has landed
    __device__ __forceinline__ bool wait_full(int j) { return mbar_wait(&full[j % NSTAGE], (uint32_t)((j / NSTAGE) & 1)); }
    // consumer warp (all lanes): done with tile j
    __device__ __forceinline__ void release(int j)
    {
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[j % NSTAGE]);
    }
    // producer: buffer of tile j is free (tile j - NSTAGE consumed); true at once for j < NSTAGE
    __device__ __forceinline__ bool wait_empty(int j)
    {
        if (j < NSTAGE) return true;
        return mbar_wait(&empty[j % NSTAGE], (uint32_t)((j / NSTAGE - 1) & 1));
    }
    __device__ __forceinline__ float *data(int j) { return &buf[j % NSTAGE][0]; }
    __device__ __forceinline__ uint64_t *full_bar(int j) { return &full[j % NSTAGE]; }
};

}  // namespace pcm
