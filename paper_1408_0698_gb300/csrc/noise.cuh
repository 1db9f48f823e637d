// noise.cuh -- detector noise of the Shack-Hartmann image (Sec. 4: the centroid
// is taken on the final noise-added image).
//
//   counts = Poisson(E) + read_noise * z
//
// Uniforms come from the counter-based generator Philox4x32-10 (Salmon,
// Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11),
// keyed by the 64-bit seed.  Pixels go in pairs (2m, 2m + 1) that share the
// counter (m, wfs << 16 | block, low word of bits(t), high word of bits(t)),
// so a frame's noise depends only on (seed, t, wfs, pixel) and never on the
// CTA, batch slot or launch that computes it.  Block 0's words 0 and 1 give the
// pair's two Box-Muller deviates (cos for the even pixel, sin for the odd one);
// word 2 + parity starts the pixel's Poisson draws, which continue with blocks
// 1 + parity, 3 + parity, ...
//
// Poisson: sequential-search inversion for E < 16 with the recurrence
// p_k = (p_{k-1} E) * RN(1/k); above, Hormann's transformed rejection with
// squeeze (PTRS, "The transformed rejection method for generating Poisson
// random variables", 1993).  The integer decisions are taken in FP32 with
// explicitly rounded operations (no contraction), so the operation order is
// fixed.  For E < 16 the search stops before k = 43 even at the largest
// uniform, so RN(1/k) fits a 64-entry table.
//
// Everything here works on values: no generator object lives in memory, so a
// warp can run the generator blocks of several pixels side by side.
#pragma once
#include <stdint.h>

namespace gbwfs {

constexpr int kRecipTable = 64;  // RN(1/k), k < 64 (entry 0 unused)

// Philox4x32-10 of counter (x0, x1, x2, x3) under key (k0, k1).
__device__ __forceinline__ uint4 philox4x32_10(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
        const uint32_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(x0, x1, x2, x3);
}

// 23 random bits plus one half: exact in FP32, strictly inside (0, 1).
__device__ __forceinline__ float philox_unit(uint32_t x) {
    return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

// The stream of one pixel pair.
struct PairStream {
    uint32_t k0, k1, pair, wfs, tlo, thi;
    __device__ __forceinline__ uint4 block(uint32_t b) const {
        return philox4x32_10(pair, (wfs << 16) | (b & 0xFFFFu), tlo, thi, k0, k1);
    }
};

__device__ __forceinline__ PairStream pair_stream(uint64_t seed, uint32_t pixel, uint32_t wfs,
                                                  uint32_t tlo, uint32_t thi) {
    PairStream q;
    q.k0 = (uint32_t)seed;
    q.k1 = (uint32_t)(seed >> 32);
    q.pair = pixel >> 1;
    q.wfs = wfs;
    q.tlo = tlo;
    q.thi = thi;
    return q;
}

// The pair's two read-noise deviates from block 0's first two words: r = sqrt(-2 ln u0) and
// the angle 2 pi u1, whose cosine and sine come from the hardware unit on 2 pi (u1 - 1/2) in
// (-pi, pi) with the signs flipped (absolute error ~4e-7, i.e. < 1e-5 electrons of read noise).
__device__ __forceinline__ void box_muller_pair(uint32_t w0, uint32_t w1, float &z_even, float &z_odd) {
    const float r = sqrtf(-2.0f * logf(philox_unit(w0)));
    float sn, cs;
    __sincosf(6.28318531f * (philox_unit(w1) - 0.5f), &sn, &cs);
    z_even = -r * cs;
    z_odd = -r * sn;
}

__device__ __forceinline__ float log_factorial_f32(float k) {
    if (k < 10.0f) {
        float s = 0.0f;
        for (int j = 2; j <= (int)k; ++j) s = __fadd_rn(s, logf((float)j));
        return s;
    }
    float x = __fadd_rn(k, 1.0f);
    float r = __fdiv_rn(1.0f, x);
    float corr = __fmul_rn(r, __fsub_rn(1.0f / 12.0f, __fmul_rn(__fmul_rn(r, r), 1.0f / 360.0f)));
    float v = __fsub_rn(__fmul_rn(__fsub_rn(x, 0.5f), logf(x)), x);
    return __fadd_rn(__fadd_rn(v, 0.918938533f), corr);
}

// Inversion for 0 < E < 16 with the first Poisson uniform u and p0 = exp(-E): the smallest k
// with u <= F_k, F_k = F_{k-1} + p_k, stopping early where F stops growing.  With TAB, rk[k]
// holds RN(1/k) for k < kRecipTable, and the loop takes two steps a trip (both steps' table
// entries loaded together, the second step's result dropped when the first stops): the search
// ends before k = 43 for every E < 16 (and only finite 0 < E < 16 reach it), so no read passes
// entry 43.  Otherwise 1/k is rounded on the spot.  Both forms take the same operations in the
// same order.
template <bool TAB>
__device__ __forceinline__ int poisson_inversion(float E, float u, float p0, const float *rk) {
    float p = p0, F = p0;
    if (TAB) {
        if (!(u > F)) return 0;
        for (int k = 1;; k += 2) {
            const float r1 = rk[k], r2 = rk[k + 1];
            const float p1 = __fmul_rn(__fmul_rn(p, E), r1);
            const float F1 = __fadd_rn(F, p1);
            const bool s1 = F1 == F || !(u > F1);
            const float p2 = __fmul_rn(__fmul_rn(p1, E), r2);
            const float F2 = __fadd_rn(F1, p2);
            const bool s2 = F2 == F1 || !(u > F2);
            if (s1) return k;
            if (s2) return k + 1;
            p = p2;
            F = F2;
        }
    }
    int k = 0;
    while (u > F) {
        k = k + 1;
        const float r = __frcp_rn((float)k);
        p = __fmul_rn(__fmul_rn(p, E), r);
        const float Fn = __fadd_rn(F, p);
        if (Fn == F) break;
        F = Fn;
    }
    return k;
}

// PTRS for E >= 16: draws word 2 + parity of block 0, then blocks 1 + parity, 3 + parity,
// ...  Rare for the workloads here, so it recomputes block 0 rather than keep it live.
// Inlined: callers give it a single call site (an out-of-line call would make every live
// register a spill).
__device__ __forceinline__ int poisson_ptrs(float E, const PairStream &q, int parity) {
    uint4 buf = q.block(0);
    uint32_t blk = 0;
    int pos = 2 + parity;
    auto next = [&]() {
        if (pos == 4) {
            blk = blk == 0 ? 1u + (uint32_t)parity : blk + 2u;
            buf = q.block(blk);
            pos = 0;
        }
        const uint32_t w = pos == 0 ? buf.x : pos == 1 ? buf.y : pos == 2 ? buf.z : buf.w;
        pos = blk == 0 ? 4 : pos + 1;
        return philox_unit(w);
    };
    float slam = __fsqrt_rn(E);
    float logE = logf(E);
    float b = __fadd_rn(0.931f, __fmul_rn(2.53f, slam));
    float a = __fadd_rn(-0.059f, __fmul_rn(0.02483f, b));
    float inv_alpha = __fadd_rn(1.1239f, __fdiv_rn(1.1328f, __fsub_rn(b, 3.4f)));
    float vr = __fsub_rn(0.9277f, __fdiv_rn(3.6224f, __fsub_rn(b, 2.0f)));
    for (int tries = 0; tries < 1024; ++tries) {
        float U = __fsub_rn(next(), 0.5f);
        float V = next();
        float us = __fsub_rn(0.5f, fabsf(U));
        float t1 = __fadd_rn(__fdiv_rn(__fmul_rn(2.0f, a), us), b);
        float kf = floorf(__fadd_rn(__fadd_rn(__fmul_rn(t1, U), E), 0.43f));
        if (us >= 0.07f && V <= vr) return (int)kf;
        if (kf < 0.0f || (us < 0.013f && V > us)) continue;
        float lhs = __fsub_rn(__fadd_rn(logf(V), logf(inv_alpha)),
                              logf(__fadd_rn(__fdiv_rn(a, __fmul_rn(us, us)), b)));
        float rhs = __fsub_rn(__fadd_rn(-E, __fmul_rn(kf, logE)), log_factorial_f32(kf));
        if (lhs <= rhs) return (int)kf;
    }
    return (int)floorf(E);
}

// Poisson count of a pixel of the given parity whose block 0 gave the inversion uniform u
// (word 2 + parity).
template <bool TAB>
__device__ __forceinline__ int poisson_count(float E, float u, float p0, const PairStream &q, int parity,
                                             const float *rk) {
    if (!(E > 0.0f)) return 0;
    if (E < 16.0f) return poisson_inversion<TAB>(E, u, p0, rk);
    return poisson_ptrs(E, q, parity);
}

// One detector pixel: Poisson photon count plus Gaussian read noise (forms its pair's block).
__device__ __forceinline__ float noise_pixel(float E, float read_noise, uint64_t seed,
                                             uint32_t pixel, uint32_t wfs, uint32_t tlo,
                                             uint32_t thi) {
    const PairStream q = pair_stream(seed, pixel, wfs, tlo, thi);
    const uint4 r = q.block(0);
    const int parity = (int)(pixel & 1u);
    float ze, zo;
    box_muller_pair(r.x, r.y, ze, zo);
    const int k = poisson_count<false>(E, philox_unit(parity ? r.w : r.z), expf(-E), q, parity, nullptr);
    return (float)k + read_noise * (parity ? zo : ze);
}

// Fills rk[0 .. kRecipTable) with RN(1/k) (entry 0 = 1); call from every thread of the block.
__device__ __forceinline__ void fill_recip_table(float *rk, int tid, int nthreads) {
    for (int i = tid; i < kRecipTable; i += nthreads) rk[i] = __frcp_rn((float)(i > 0 ? i : 1));
}

}  // namespace gbwfs
