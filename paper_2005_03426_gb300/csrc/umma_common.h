// umma_common.h -- inline-PTX helpers shared by the tcgen05 kernels (k_umma.cu, k_ozaki.cu):
// shared-memory matrix descriptors, instruction descriptors, bounded mbarrier waits, cp.async.
#pragma once
#include <cstdint>

#define UM_WAIT_LIMIT (1u << 26)   // polls before a wait gives up (the kernel then reports an error)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 bytes apart
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
    d |= (uint64_t)(16u >> 4) << 16;                   // leading byte offset (unused for SW128 K-major)
    d |= (uint64_t)(1024u >> 4) << 32;                 // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                            // fixed 0b001 (tcgen05 descriptor)
    d |= (uint64_t)2 << 61;                            // swizzle mode: 128 B
    return d;
}

// instruction descriptor: D = F32, A/B type (kind::tf32: 2 = TF32; kind::f16: 1 = BF16),
// both K-major, M x N tile (M = 128; N a multiple of 16 up to 256)
__device__ __forceinline__ uint32_t umma_idesc_mn(int ab_type, uint32_t M, uint32_t N) {
    return (1u << 4) | ((uint32_t)ab_type << 7) | ((uint32_t)ab_type << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
__device__ __forceinline__ uint32_t umma_idesc(int ab_type) { return umma_idesc_mn(ab_type, 128u, 128u); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait for the phase with the given parity; false on time-out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < UM_WAIT_LIMIT; ++it) {
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

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(src_bytes)
                 : "memory");
}

