// tcgen05.cuh -- the 5th-generation tensor-core building blocks of the spot kernels: shared-
// memory matrix descriptors (K-major, 128-byte swizzle), the kind::f16 instruction descriptor,
// the MMA issue and commit, bounded mbarrier waits, tensor-memory loads, and the split operand
// elements (BF16 hi/lo, or FP16 hi/lo with power-of-two scaling).  Inline PTX, sm_100 family.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace gbwfs {
namespace tc {

constexpr int kWaitLimit = 1 << 24;      // mbarrier polls before giving up


__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // SWIZZLE_128B
    return d;
}

// Instruction descriptor of kind::f16: A and B of format fmt (0 = FP16, 1 = BF16; both operands
// always the same type) -> F32, both K-major.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N, uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < kWaitLimit && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
    return done != 0;
}

// The same wait with the thread suspended while the phase is incomplete (a time hint of 1 ms per
// try), so that a waiting warp takes no issue slots from the warps that have work; gives up after
// 4096 tries (about 4 s).
__device__ __forceinline__ bool mbar_wait_suspend(uint64_t *mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < 4096 && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity), "r"(1000000u)
            : "memory");
    return done != 0;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

#define GBWFS_TMEM_LD16(r, addr)                                                                          \
    asm volatile(                                                                                         \
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), \
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),        \
          "=r"(r[15])                                                                                     \
        : "r"(addr))

#define GBWFS_TMEM_LD32(r, addr)                                                                          \
    asm volatile(                                                                                         \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"  \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                         \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), \
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),        \
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),      \
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),      \
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])                                                           \
        : "r"(addr))

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// byte offset of element k of row r in a 128-row x 64-element BF16 swizzled tile
__host__ __device__ inline uint32_t sw128_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + (k & 7) * 2);
}

// The operand element of the tensor-core products: BF16 (8-bit significand), or FP16 (11-bit)
// with a power-of-two scale per subaperture and operand that puts its largest magnitude in
// [2^13, 2^14), inside FP16's normal range.  x = hi + lo exactly in FP32; the MMAs take
// hi*hi + lo*hi + hi*lo.
template <bool kF16>
struct TcElt {
    static constexpr uint32_t fmt = 1;  // BF16
    static __device__ __forceinline__ void split(float x, float &hi, float &lo) {
        hi = __bfloat162float(__float2bfloat16_rn(x));
        lo = x - hi;
    }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&v);
    }
    static __device__ __forceinline__ uint16_t bits(float a) { return __bfloat16_as_ushort(__float2bfloat16_rn(a)); }
    // The split of a pair as packed words: hw = pack(hi a, hi b), lw = pack(lo a, lo b) -- the
    // words pack() gives on split()'s parts (rounding is idempotent, so pack(a, b) holds the hi
    // parts, which unpack exactly; x - hi is exact).
    static __device__ __forceinline__ void split2(float a, float b, uint32_t &hw, uint32_t &lw) {
        hw = pack(a, b);
        lw = pack(a - __uint_as_float(hw << 16), b - __uint_as_float(hw & 0xFFFF0000u));
    }
};
template <>
struct TcElt<true> {
    static constexpr uint32_t fmt = 0;  // FP16
    static __device__ __forceinline__ void split(float x, float &hi, float &lo) {
        hi = __half2float(__float2half_rn(x));
        lo = x - hi;
    }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __half2 v = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&v);
    }
    static __device__ __forceinline__ uint16_t bits(float a) { return __half_as_ushort(__float2half_rn(a)); }
    static __device__ __forceinline__ void split2(float a, float b, uint32_t &hw, uint32_t &lw) {
        hw = pack(a, b);
        const float2 h = __half22float2(*reinterpret_cast<const __half2 *>(&hw));
        lw = pack(a - h.x, b - h.y);
    }
};

__device__ __forceinline__ float warp_sum_tc(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The FP16 operand scale 2^e: x 2^e in [2^13, 2^14) for the largest magnitude x (e = 0 for
// x = 0; |e| <= 60).
__device__ __forceinline__ int f16_scale_exp(float mx) {
    if (!(mx > 0.0f)) return 0;
    const int ex = (int)((__float_as_uint(mx) >> 23) & 0xFFu) - 127;
    return max(-60, min(60, 13 - ex));
}

__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }  // |e| <= 126

}  // namespace tc
}  // namespace gbwfs
