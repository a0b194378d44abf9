// Helpers for the tcgen05 (5th-generation tensor core) kernels: shared-memory operand layout and
// descriptors, instruction descriptor, FP16 hi/lo split, bounded mbarrier wait, and thin wrappers of
// the tcgen05 instructions used (inline PTX; sm_100-family only).
#pragma once

#include <cuda_fp16.h>

#include "fga_internal.cuh"

namespace fga {
namespace tc {

constexpr int KB = 32;                      // K extent of one staged operand block (elements)
constexpr long long SPIN_LIMIT = 1ll << 24; // bound of every mbarrier wait (try_wait iterations)

// byte offset of element (row, k) of a K-major no-swizzle operand with K extent KB:
// core matrix (row/8, k/8) at (row/8) * SBO + (k/8) * LBO, SBO = 4 * 128 B, LBO = 128 B
__device__ __forceinline__ uint32_t kmaj_off(int row, int k) {
    return (uint32_t)(((row >> 3) * (KB / 8) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// tcgen05 shared-memory matrix descriptor (no swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    const uint64_t lbo = 128, sbo = (KB / 8) * 128;
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(lbo >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;  // fixed constant 0b001 at bits 46-48
    return d;                // base offset 0, relative LBO, swizzle none
}

// the same with explicit byte offsets between K-adjacent (lbo) and row-adjacent (sbo) core matrices
// (multiples of 16 bytes; padded layouts spread one warp's stores over all banks)
__device__ __forceinline__ uint64_t smem_desc_lbo_sbo(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: D f32, A and B f16, both K-major, N and M
__device__ __forceinline__ uint32_t instr_desc(int n, int m) {
    uint32_t d = 0;
    d |= 1u << 4;                    // D format f32
    d |= 0u << 7;                    // A format f16
    d |= 0u << 10;                   // B format f16
    d |= (uint32_t)(n >> 3) << 17;   // N / 8
    d |= (uint32_t)(m >> 4) << 24;   // M / 16
    return d;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void split_store(unsigned char *hi_base, unsigned char *lo_base, uint32_t off, float x) {
    const __half h = __float2half_rn(x);
    const __half l = __float2half_rn(x - __half2float(h));
    *reinterpret_cast<__half *>(hi_base + off) = h;
    *reinterpret_cast<__half *>(lo_base + off) = l;
}

template <typename T> __device__ __forceinline__ float2 ld_c(const T *p);
template <> __device__ __forceinline__ float2 ld_c<double2>(const double2 *p) {
    const double2 v = *p;
    return make_float2((float)v.x, (float)v.y);
}
template <> __device__ __forceinline__ float2 ld_c<float2>(const float2 *p) { return *p; }

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < SPIN_LIMIT; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Give-up path of a CTA whose wait for a tcgen05.commit ran out: the MMAs of that commit may still be
// reading shared memory and writing tensor memory, so before the CTA frees its tensor memory and
// exits it waits once more, with a bound four times longer, for the same phase.  Returns whether the
// commit arrived; if it never does (the tensor pipe made no progress for 5 x SPIN_LIMIT polls) the CTA
// frees its columns anyway rather than hang the GPU.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
    for (int r = 0; r < 4; r++)
        if (mbar_wait(bar, parity)) return true;
    return false;
}

// 8 consecutive K elements (k % 8 == 0) of one row: one 16-byte store of their FP16 values
__device__ __forceinline__ void store8(unsigned char *base, uint32_t off, const __half h[8]) {
    uint4 v;
    v.x = (uint32_t)__half_as_ushort(h[0]) | ((uint32_t)__half_as_ushort(h[1]) << 16);
    v.y = (uint32_t)__half_as_ushort(h[2]) | ((uint32_t)__half_as_ushort(h[3]) << 16);
    v.z = (uint32_t)__half_as_ushort(h[4]) | ((uint32_t)__half_as_ushort(h[5]) << 16);
    v.w = (uint32_t)__half_as_ushort(h[6]) | ((uint32_t)__half_as_ushort(h[7]) << 16);
    *reinterpret_cast<uint4 *>(base + off) = v;
}
// hi/lo split of 8 values scaled by s, stored as two 16-byte rows (hi and lo operand copies); pairs of
// values are rounded to FP16 together (one f16x2 conversion per pair)
__device__ __forceinline__ void split8(unsigned char *hi, unsigned char *lo, uint32_t off, const float x[8], float s) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const float a = x[2 * q] * s, b = x[2 * q + 1] * s;
        const __half2 hh = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(hh);
        const __half2 ll = __floats2half2_rn(a - hf.x, b - hf.y);
        h[q] = *reinterpret_cast<const uint32_t *>(&hh);
        l[q] = *reinterpret_cast<const uint32_t *>(&ll);
    }
    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void alloc(uint32_t slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t tmem, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// 8 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void ld8(uint32_t taddr, float v[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = __uint_as_float(r[q]);
}

}  // namespace tc
}  // namespace fga
