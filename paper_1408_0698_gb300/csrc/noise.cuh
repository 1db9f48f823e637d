// noise.cuh -- detector noise of the Shack-Hartmann image (Sec. 4: the centroid
// is taken on the final noise-added image).
//
//   counts = Poisson(E) + read_noise * z
//
// Uniforms come from the counter-based generator Philox4x32-10 (Salmon,
// Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11),
// keyed by the 64-bit seed, with counter
//   (pixel, wfs << 16 | block, low word of bits(t), high word of bits(t)),
// so a frame's noise depends only on (seed, t, wfs, pixel) and never on the
// CTA, batch slot or launch that computes it.  Block 0's first two words feed
// Box-Muller read noise; the Poisson sampler starts at its third word and
// continues with blocks 1, 2, ...
//
// Poisson: sequential-search inversion for E < 16; above, Hormann's
// transformed rejection with squeeze (PTRS, "The transformed rejection method
// for generating Poisson random variables", 1993).  The integer decisions are
// taken in FP32 with explicitly rounded operations (no contraction), so the
// operation order is fixed.
#pragma once
#include <stdint.h>

namespace gbwfs {

struct Philox {
    uint32_t k0, k1, c0, c1, c2, c3;
    uint32_t r[4];
    int pos;

    __device__ __forceinline__ void block(uint32_t b) {
        uint32_t x0 = c0, x1 = (c1 & 0xFFFF0000u) | (b & 0xFFFFu), x2 = c2, x3 = c3;
        c1 = x1;
        uint32_t a0 = k0, a1 = k1;
#pragma unroll
        for (int i = 0; i < 10; ++i) {
            uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
            uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
            uint32_t y0 = hi1 ^ x1 ^ a0, y2 = hi0 ^ x3 ^ a1;
            x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
            a0 += 0x9E3779B9u;
            a1 += 0xBB67AE85u;
        }
        r[0] = x0; r[1] = x1; r[2] = x2; r[3] = x3;
    }
    __device__ __forceinline__ static float unit(uint32_t x) {
        // 23 random bits plus one half: exact in FP32, strictly inside (0, 1)
        return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f);
    }
    __device__ __forceinline__ float next() {
        if (pos == 4) {
            block((c1 & 0xFFFFu) + 1u);
            pos = 0;
        }
        return unit(r[pos++]);
    }
};

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

static __device__ __noinline__ int poisson_f32(float E, Philox &g) {
    if (!(E > 0.0f)) return 0;
    if (E < 16.0f) {
        float u = g.next();
        float p = expf(-E);
        float F = p;
        int k = 0;
        while (u > F) {
            k = k + 1;
            p = __fdiv_rn(__fmul_rn(p, E), (float)k);
            float Fn = __fadd_rn(F, p);
            if (Fn == F) break;
            F = Fn;
        }
        return k;
    }
    float slam = __fsqrt_rn(E);
    float logE = logf(E);
    float b = __fadd_rn(0.931f, __fmul_rn(2.53f, slam));
    float a = __fadd_rn(-0.059f, __fmul_rn(0.02483f, b));
    float inv_alpha = __fadd_rn(1.1239f, __fdiv_rn(1.1328f, __fsub_rn(b, 3.4f)));
    float vr = __fsub_rn(0.9277f, __fdiv_rn(3.6224f, __fsub_rn(b, 2.0f)));
    for (int tries = 0; tries < 1024; ++tries) {
        float U = __fsub_rn(g.next(), 0.5f);
        float V = g.next();
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

// One detector pixel: Poisson photon count plus Gaussian read noise.
__device__ __forceinline__ float noise_pixel(float E, float read_noise, uint64_t seed,
                                             uint32_t pixel, uint32_t wfs, uint32_t tlo,
                                             uint32_t thi) {
    Philox g;
    g.k0 = (uint32_t)seed;
    g.k1 = (uint32_t)(seed >> 32);
    g.c0 = pixel;
    g.c1 = wfs << 16;
    g.c2 = tlo;
    g.c3 = thi;
    g.block(0);
    float u1 = Philox::unit(g.r[0]), u2 = Philox::unit(g.r[1]);
    g.pos = 2;
    int k = poisson_f32(E, g);
    float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    return (float)k + read_noise * z;
}

}  // namespace gbwfs
