// Small helpers for the tcgen05 kernels: shared-memory addresses, UMMA
// shared-memory descriptors, TF32 rounding and bounded mbarrier waits.
#pragma once

#include <cstdint>

namespace slr {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version; no swizzle, base offset 0
    return d;
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
    return __uint_as_float(t);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` polls (the caller then reports
// kStatusTimeout and stops using the tensor core).
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, int limit) {
    for (int it = 0; it < limit; ++it)
        if (mbar_try_wait(addr, parity)) return true;
    return false;
}

}  // namespace tc
}  // namespace slr
