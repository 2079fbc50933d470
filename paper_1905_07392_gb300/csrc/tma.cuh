// Tensor-memory-accelerator (TMA) tile loads into shared memory, completed on
// an mbarrier, for sm_100-class GPUs: inline PTX (`mbarrier.*`,
// `cp.async.bulk.tensor`) plus the host-side encoding of the tensor maps.
//
// Every wait here is bounded: try_wait_bounded gives up after a number of
// clock64 cycles and reports it, so that a kernel can record an error and
// return instead of spinning for ever.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ebv {

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes initialised barriers visible to the async (TMA) proxy.
__device__ inline void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses before later async-proxy
// (TMA) writes to the same memory.
__device__ inline void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ inline void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of `parity` to complete, for at most `limit` cycles of
// clock64; limit <= 0 gives up at once (a switch for tests of the timeout
// path).  Returns false if it gave up.
__device__ inline bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit)
{
    if (limit <= 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (clock64() - t0 < limit)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// One 4-D tile of the tensor map `tm` at element coordinates (c0..c3) into
// shared memory at `dst` (128-byte aligned); completes `bytes` on `bar`.
// Coordinates may be negative or past the end: those elements read as zero.
__device__ inline void tma_load_4d(void *dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Host: encodes a 4-D tiled tensor map (no swizzle, no interleave, zero fill
// out of bounds).  dims[0] is the innermost (contiguous) dimension; strides
// are the byte strides of dims 1..3.  Returns false if the driver entry point
// is missing or the encoding is refused (the caller then takes another path).
bool tma_encode_4d(CUtensorMap *tm, CUtensorMapDataType type, void *base, const uint64_t dims[4],
                   const uint64_t strides[3], const uint32_t box[4]);

}  // namespace ebv
