// tma_util.cuh -- shared-memory addresses, mbarriers with bounded waits and
// 3-D TMA tile loads used by the staged convolution kernels and the split
// evaluator's PSF stage.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace gbk {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Arms `bar` for `bytes` and loads the box at (x, y, z) of `tmap` into dst.
__device__ __forceinline__ void tma_load_slab(const CUtensorMap *tmap, float *dst, uint64_t *bar, int x, int y,
                                              int z, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Arms `bar` for `bytes` of transfers that the next tma_load_3d calls bring.
__device__ __forceinline__ void tma_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Loads the box at (x, y, z) of `tmap` into dst; completion is counted on
// `bar` (armed beforehand by tma_expect for the sum of the boxes' bytes).
__device__ __forceinline__ void tma_load_3d(const CUtensorMap *tmap, void *dst, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Copies `bytes` (a multiple of 16) from global src to shared dst, both
// 16-byte aligned (an untiled bulk copy); completion is counted on `bar`
// (armed beforehand by tma_expect for the sum of the copies' bytes).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "{\n .reg .u64 g;\n cvta.to.global.u64 g, %1;\n"
        " cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [g], %2, [%3];\n}" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait for the given phase; false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase, long limit)
{
    for (long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace gbk
