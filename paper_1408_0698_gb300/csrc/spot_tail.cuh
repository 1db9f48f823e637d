// spot_tail.cuh -- the stages of the 32-point spot kernels that follow the first
// transfer-domain stage, on the CUDA cores, for one subaperture owned by one warp
// (Sec. 4 LGS SH: elongation by the sodium kernel, binning, noise-added image,
// centroid).  Shared by the FP32 and tensor-core kernels.
//
//   M[dy][dx] = Kt[dy][dx] sum_k Ga(dy, k) T[k][dx]       (k = lane: a 32-point DFT)
//   Q[iy][dx] = sum_dy G(dy, iy) M[dy][dx]                 (an nd-point DFT over dy)
//   B[iy][ix] = Re sum_dx Q[iy][dx] G[dx][ix]              (lane = ix, half-warp = iy half)
// with Ga(dy, k) = exp(+2 pi i (k - cN) dy / N) = ph(dy) w^(k dy), w = exp(2 pi i / N),
// ph(dy) = exp(-2 pi i cN dy / N), and G(dy, i) = sum_{r<b} exp(-2 pi i (b i + r - cN) dy / N)
// (conjugated for dy < 0).  The sum over k is a DFT of each column across the lanes: radix 2,
// decimation in frequency, one shuffle per stage and component; lane i ends with frequency
// bitrev5(i).  Kt carries 1/N^2 and the Hermitian weight c_dx, so B is the binned elongated
// spot.  Since N = b nd, G(dy, i) = h(dy) v^(i dy) with h(dy) = sum_{r<b} exp(-2 pi i (r - cN)
// dy / N) and v = exp(-2 pi i / nd): Q is the nd-point DFT of m[j] = sum_{dy = j mod nd} h(dy)
// M[dy][dx].  The lanes i and i ^ 1 hold the frequencies f and f + 16 (the same j, since
// nd = 16), so one shuffle folds them, and the positions p = i >> 1 hold j = bitrev4(p): a
// decimation-in-time DFT across the positions ends with Q[p] in natural order, the even lane
// of each pair working the first column pairs and the odd lane the rest.  Then
// E = photons fill B / sum B, C = Poisson(E) + ron z (or E), and the centre of gravity.
#pragma once
#include "internal.h"
#include "noise.cuh"

namespace gbwfs {
namespace tail {

__device__ __forceinline__ void cmac(float2 &acc, const float2 a, const float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kFftTable = 10 * 32;  // float2: five stages of twiddles, ph h(dy), four more stages

// Per-lane DFT constants: entry s * 32 + lane (s < 5, span h = 16 >> s) is 1 for the upper
// lane of a butterfly and w^((lane mod h) 16 / h) for the lower; entry 5 * 32 + lane is
// ph(dy) h(dy) = sum_{r<2} exp(-2 pi i r dy / 32) of the lane's output frequency dy when
// |dy| < n, else 0; entry (6 + s) * 32 + lane (s < 4, span q = 2^s in positions p = lane >> 1)
// is 1 for the upper position of a butterfly and exp(-2 pi i (p mod q) / 2q) for the lower.
// Call from every thread of the block.
template <int n>
__device__ __forceinline__ void fill_fft_table(float2 *tab, int tid, int nthreads) {
    for (int i = tid; i < kFftTable; i += nthreads) {
        const int st = i >> 5, l = i & 31;
        float sn = 0.0f, cs = 1.0f;
        if (st < 5) {
            const int h = 16 >> st;
            if (l & h) sincospif((float)((l & (h - 1)) * (16 / h)) / 16.0f, &sn, &cs);
        } else if (st == 5) {
            const int f = (int)(__brev((unsigned)l) >> 27), dy = f < 16 ? f : f - 32;
            if (dy > -n && dy < n) {
                sincospif((float)(-dy) / 16.0f, &sn, &cs);  // exp(-2 pi i dy / 32)
                cs += 1.0f;
            } else {
                cs = 0.0f;
            }
        } else {
            const int q = 1 << (st - 6), p = l >> 1;
            if (p & q) sincospif((float)(-(p & (q - 1))) / (float)q, &sn, &cs);
        }
        tab[i] = make_float2(cs, sn);
    }
}

// Packed FP32x2 arithmetic (one instruction for two lanes of values, each rounded as the scalar
// operation): the column pairs (dx, dx + 1) of the tail travel together.
__device__ __forceinline__ float2 dup2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// T: this lane's row k = lane of the first stage (T[k][dx], dx < n), consumed.  fft: the
// table above.  Gt: [n][nd] G[d][i].  kt: the subaperture's K~ [2n-1][n] (global or shared
// memory).  Q is per-warp scratch ([nd][n/2], 16-byte aligned), each entry a column pair
// (re dx, re dx+1, im dx, im dx+1).
// On return Bv[j] = B[half * nd/2 + j][ix] for lane = half * 16 + ix.
template <int n, int nd>
__device__ __forceinline__ void lgs_binned(float2 (&T)[n], float4 *Q, const float2 *fft, const float2 *Gt,
                                           const float2 *kt, int lane, float (&Bv)[nd / 2]) {
    constexpr int P = n / 2, PH = (P + 1) / 2;
    static_assert(nd == 16, "the detector tile maps to 16 lanes x 2 half-warps");
    static_assert(n <= 16, "frequencies |dy| < n must be distinct modulo 32");
    static_assert(n % 2 == 0, "columns travel in pairs");
    // columns as pairs: Tr[c] = (re 2c, re 2c+1), Ti[c] = (im 2c, im 2c+1)
    float2 Tr[P], Ti[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
        Tr[c] = make_float2(T[2 * c].x, T[2 * c + 1].x);
        Ti[c] = make_float2(T[2 * c].y, T[2 * c + 1].y);
    }
    // M: DFT over the lanes, five radix-2 stages
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int h = 16 >> st;
        const float2 sg = dup2((lane & h) ? -1.0f : 1.0f);
        const float2 tw = fft[st * 32 + lane];
        const float2 twx = dup2(tw.x), twy = dup2(tw.y), ntwy = dup2(-tw.y);
#pragma unroll
        for (int c = 0; c < P; ++c) {
            const float2 tr = make_float2(__shfl_xor_sync(0xffffffffu, Tr[c].x, h),
                                          __shfl_xor_sync(0xffffffffu, Tr[c].y, h));
            const float2 ti = make_float2(__shfl_xor_sync(0xffffffffu, Ti[c].x, h),
                                          __shfl_xor_sync(0xffffffffu, Ti[c].y, h));
            const float2 sr = fma2(sg, Tr[c], tr), si = fma2(sg, Ti[c], ti);
            Tr[c] = fma2(si, ntwy, mul2(sr, twx));
            Ti[c] = fma2(si, twx, mul2(sr, twy));
        }
    }
    // h(dy) M[dy] for the lane's frequency (zero outside the band |dy| < n, through the table),
    // then folded with the lane holding dy -/+ 16
    {
        const int f = (int)(__brev((unsigned)lane) >> 27), dy = f < 16 ? f : f - 32;
        const int dyi = min(max(dy + n - 1, 0), 2 * n - 2);
        const float2 ph = fft[5 * 32 + lane];
        const float2 phx = dup2(ph.x), phy = dup2(ph.y), nphy = dup2(-ph.y);
#pragma unroll
        for (int c = 0; c < P; ++c) {
            const float2 xr = fma2(Ti[c], nphy, mul2(Tr[c], phx));
            const float2 xi = fma2(Ti[c], phx, mul2(Tr[c], phy));
            const float2 k0 = kt[dyi * n + 2 * c], k1 = kt[dyi * n + 2 * c + 1];
            const float2 kr = make_float2(k0.x, k1.x), ki = make_float2(k0.y, k1.y);
            const float2 mr = fma2(xi, make_float2(-ki.x, -ki.y), mul2(xr, kr));
            const float2 mi = fma2(xi, kr, mul2(xr, ki));
            Tr[c] = __fadd2_rn(mr, make_float2(__shfl_xor_sync(0xffffffffu, mr.x, 1),
                                               __shfl_xor_sync(0xffffffffu, mr.y, 1)));
            Ti[c] = __fadd2_rn(mi, make_float2(__shfl_xor_sync(0xffffffffu, mi.x, 1),
                                               __shfl_xor_sync(0xffffffffu, mi.y, 1)));
        }
    }
    // Q: a 16-point DFT across the positions p = lane >> 1 (input bit-reversed, output in
    // natural order), four radix-2 decimation-in-time stages; the even lane of a position
    // takes the column pairs [0, PH), the odd lane the rest
    const int par = lane & 1;
    float2 Wr[PH], Wi[PH];
#pragma unroll
    for (int j = 0; j < PH; ++j) {
        const int c1 = PH + j;
        const float2 zr = c1 < P ? Tr[c1 < P ? c1 : 0] : make_float2(0.0f, 0.0f);
        const float2 zi = c1 < P ? Ti[c1 < P ? c1 : 0] : make_float2(0.0f, 0.0f);
        Wr[j] = par ? zr : Tr[j];
        Wi[j] = par ? zi : Ti[j];
    }
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        const int q = 1 << st;
        const float2 sg = dup2(((lane >> 1) & q) ? -1.0f : 1.0f);
        const float2 tw = fft[(6 + st) * 32 + lane];
        const float2 twx = dup2(tw.x), twy = dup2(tw.y), ntwy = dup2(-tw.y);
#pragma unroll
        for (int j = 0; j < PH; ++j) {
            // the lower position's value times its twiddle; then upper = own + partner's,
            // lower = partner's - own
            float2 vr = Wr[j], vi = Wi[j];
            if (st > 0) {  // the first stage's twiddles are all 1
                vr = fma2(Wi[j], ntwy, mul2(Wr[j], twx));
                vi = fma2(Wi[j], twx, mul2(Wr[j], twy));
            }
            const float2 pr = make_float2(__shfl_xor_sync(0xffffffffu, vr.x, 2 * q),
                                          __shfl_xor_sync(0xffffffffu, vr.y, 2 * q));
            const float2 pi = make_float2(__shfl_xor_sync(0xffffffffu, vi.x, 2 * q),
                                          __shfl_xor_sync(0xffffffffu, vi.y, 2 * q));
            Wr[j] = fma2(sg, vr, pr);
            Wi[j] = fma2(sg, vi, pi);
        }
    }
    const int ix = lane & 15, half = lane >> 4;
    __syncwarp();  // earlier reads of the scratch by other lanes are done
    {
        const int iy = lane >> 1;
#pragma unroll
        for (int j = 0; j < PH; ++j) {
            const int c = par ? PH + j : j;
            if (c < P) Q[iy * P + c] = make_float4(Wr[j].x, Wr[j].y, Wi[j].x, Wi[j].y);
        }
    }
    __syncwarp();
    // B[iy][ix] for iy in this half: Re sum_dx Q[iy][dx] G[dx][ix], even and odd columns summed
    // apart
    float2 gcx[P], ngcy[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
        const float2 g0 = Gt[(2 * c) * nd + ix], g1 = Gt[(2 * c + 1) * nd + ix];
        gcx[c] = make_float2(g0.x, g1.x);
        ngcy[c] = make_float2(-g0.y, -g1.y);
    }
#pragma unroll
    for (int j = 0; j < nd / 2; ++j) {
        const int iy = half * (nd / 2) + j;
        float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < P; ++c) {
            const float4 qv = Q[iy * P + c];
            s = fma2(make_float2(qv.x, qv.y), gcx[c], fma2(make_float2(qv.z, qv.w), ngcy[c], s));
        }
        Bv[j] = s.x + s.y;
    }
}

// NGS: b x b binning of the spot image rows Iw ([32][33] floats).
template <int nd>
__device__ __forceinline__ void ngs_binned(const float *Iw, int lane, float (&Bv)[nd / 2]) {
    constexpr int N = 32, b = N / nd;
    const int ix = lane & 15, half = lane >> 4;
#pragma unroll
    for (int j = 0; j < nd / 2; ++j) {
        const int iy = half * (nd / 2) + j;
        float s = 0.0f;
        if (ix < nd) {
#pragma unroll
            for (int r = 0; r < b; ++r)
#pragma unroll
                for (int c = 0; c < b; ++c) s += Iw[(b * iy + r) * (N + 1) + b * ix + c];
        }
        Bv[j] = s;
    }
}

// Photometry: ev[j] = E of detector row half * nd/2 + j, column ix (lane = half * 16 + ix),
// E = photons fill B / sum B.
template <int nd>
__device__ __forceinline__ void expected(const float (&Bv)[nd / 2], const WfsDesc &W, int v, int lane,
                                         float (&ev)[nd / 2]) {
    constexpr int J = nd / 2;
    const int ix = lane & 15;
    float sb = 0.0f;
    if (ix < nd) {
#pragma unroll
        for (int j = 0; j < J; ++j) sb += Bv[j];
    }
    sb = warp_sum(sb);
    const float scale = sb > 0.0f ? W.photons * __ldg(W.fill + v) / sb : 0.0f;
#pragma unroll
    for (int j = 0; j < J; ++j) ev[j] = scale * Bv[j];
}

// Stores E of subaperture v to D.st_E (when given).
template <int nd>
__device__ __forceinline__ void store_expected(const float (&ev)[nd / 2], const WfsDesc &W, const InstDyn &D,
                                               int v, int lane) {
    constexpr int nd2 = nd * nd, J = nd / 2;
    const int ix = lane & 15, half = lane >> 4;
    if (!D.st_E || ix >= nd) return;
    float *st_E = D.st_E + W.det_off + (size_t)v * nd2;
#pragma unroll
    for (int j = 0; j < J; ++j) st_E[(half * J + j) * nd + ix] = ev[j];
}

// Noise and the centroid of subaperture v of WFS W from its expected image ev (the layout of
// expected()); lane 0 writes the slopes.  rk: RN(1/k) table (fill_recip_table) in shared
// memory.  One generator block per pixel pair; each exchange between the lane pair is followed
// by both pixels' inversion searches, and the rare pixels with E >= 16 go last through one PTRS
// call site.
template <int nd>
__device__ __forceinline__ void noise_centroid(const float (&ev)[nd / 2], const WfsDesc &W, const InstDyn &D,
                                               uint64_t seed, int v, int lane, const float *rk) {
    constexpr int nd2 = nd * nd, J = nd / 2;
    static_assert(nd == 16, "pixel pairs are the lane pairs (ix, ix + 1) of a 16-lane row");
    const int ix = lane & 15, half = lane >> 4;
    const float cd = 0.5f * (float)(nd - 1);
    const uint32_t tlo = (uint32_t)__double_as_longlong(D.t);
    const uint32_t thi = (uint32_t)((unsigned long long)__double_as_longlong(D.t) >> 32);
    float *st_C = D.st_C ? D.st_C + W.det_off : nullptr;
    float sc = 0.0f, sx = 0.0f, sy = 0.0f;
    if (ix < nd) {
        float cv[J];
        if (D.noise) {
            // Pixel pairs (2m, 2m + 1) are the lanes (ix, ix + 1) of one row: the even lane
            // forms the pair blocks of its first J/2 rows, the odd lane those of its last J/2,
            // and each hands its partner that pixel's deviate and uniform; rows m and
            // m + J/2 are then sampled together.
            const uint32_t pix0 = (uint32_t)(v * nd2 + half * J * nd + ix);
            const int par = ix & 1;
            uint32_t big = 0;
            float z[J];
#pragma unroll
            for (int m = 0; m < J / 2; ++m) {
                const uint32_t pix = pix0 + (uint32_t)((par * (J / 2) + m) * nd);
                const uint4 r = pair_stream(seed, pix, (uint32_t)W.gs_index, tlo, thi).block(0);
                float ze, zd;
                box_muller_pair(r.x, r.y, ze, zd);
                const float zr = __shfl_xor_sync(0xffffffffu, par ? ze : zd, 1);
                const float ur = __shfl_xor_sync(0xffffffffu, philox_unit(par ? r.z : r.w), 1);
                const float zo = par ? zd : ze, uo = philox_unit(par ? r.w : r.z);
                z[m] = par ? zr : zo;
                z[m + J / 2] = par ? zo : zr;
                const float ua = par ? ur : uo, ub = par ? uo : ur;
                const float ea = ev[m], eb = ev[m + J / 2];
                int ka = 0, kb = 0;
                if (ea >= 16.0f) big |= 1u << m;
                else if (ea > 0.0f) ka = poisson_inversion<true>(ea, ua, expf(-ea), rk);
                if (eb >= 16.0f) big |= 1u << (m + J / 2);
                else if (eb > 0.0f) kb = poisson_inversion<true>(eb, ub, expf(-eb), rk);
                cv[m] = (float)ka + W.read_noise * z[m];
                cv[m + J / 2] = (float)kb + W.read_noise * z[m + J / 2];
            }
            while (big) {  // PTRS: one call site, rare
                const int j = __ffs(big) - 1;
                big &= big - 1;
                float e = 0.0f, zj = 0.0f;
#pragma unroll
                for (int jj = 0; jj < J; ++jj)
                    if (jj == j) {
                        e = ev[jj];
                        zj = z[jj];
                    }
                const PairStream q = pair_stream(seed, pix0 + (uint32_t)(j * nd), (uint32_t)W.gs_index, tlo, thi);
                const float c = (float)poisson_ptrs(e, q, par) + W.read_noise * zj;
#pragma unroll
                for (int jj = 0; jj < J; ++jj)
                    if (jj == j) cv[jj] = c;
            }
        } else {
#pragma unroll
            for (int j = 0; j < J; ++j) cv[j] = ev[j];
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int iy = half * J + j, o = iy * nd + ix;
            if (st_C) st_C[(size_t)v * nd2 + o] = cv[j];
            sc += cv[j];
            sx = fmaf((float)ix - cd, cv[j], sx);
            sy = fmaf((float)iy - cd, cv[j], sy);
        }
    }
    sc = warp_sum(sc);
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) {
        const bool ok = sc > 0.0f;
        float *sl = D.slopes + W.slope_off;
        sl[2 * v] = ok ? sx / sc : 0.0f;
        sl[2 * v + 1] = ok ? sy / sc : 0.0f;
    }
}

// Photometry, noise and the centroid in one pass (the spot kernel completes the measurement);
// with split, only the expected image is stored and the noise kernel completes it.
template <int nd>
__device__ __forceinline__ void finish(const float (&Bv)[nd / 2], const WfsDesc &W, const InstDyn &D,
                                       uint64_t seed, int v, int lane, const float *rk, bool split) {
    float ev[nd / 2];
    expected<nd>(Bv, W, v, lane, ev);
    store_expected<nd>(ev, W, D, v, lane);
    if (!split) noise_centroid<nd>(ev, W, D, seed, v, lane, rk);
}

// ---- any DFT size (N <= 32) and detector tile: the same stages as direct sums over the warp's
// rows in shared memory, in the order of the FP32 generic kernel; the noise pixel by pixel.

// Ta: [N][n|1] the first stage (row k, column dx).  kt: the subaperture's K~ [2n-1][n].  Ga:
// [n][N] Ga[d][k] = exp(+2 pi i (k - cN) d / N) (conjugated for d < 0).  G: [n][nd] G[d][i].
// M [2n-1][n], P [2n-1][nd] complex and B [nd][nd] real are the warp's scratch; B holds the
// binned elongated spot on return.
template <int n, int N, int nd>
__device__ __forceinline__ void lgs_direct(const float2 *Ta, float2 *M, float2 *P, float *B, const float2 *kt,
                                           const float2 *Ga, const float2 *G, int lane) {
    constexpr int D2 = 2 * n - 1, no = n | 1;
    // M[dy][dx] = Kt[dy][dx] sum_k Ga[dy][k] Ta[k][dx]
    for (int o = lane; o < D2 * n; o += 32) {
        const int dyi = o / n, dx = o - dyi * n, dy = dyi - (n - 1);
        const float2 *ga = Ga + (dy >= 0 ? dy : -dy) * N;
        const float sg = dy >= 0 ? 1.0f : -1.0f;
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll 8
        for (int k = 0; k < N; ++k) {
            float2 gg = ga[k];
            gg.y *= sg;
            cmac(acc, gg, Ta[k * no + dx]);
        }
        const float2 kv = kt[o];
        M[o] = make_float2(acc.x * kv.x - acc.y * kv.y, acc.x * kv.y + acc.y * kv.x);
    }
    __syncwarp();
    // P[dy][ix] = sum_dx M[dy][dx] G[dx][ix]
    for (int o = lane; o < D2 * nd; o += 32) {
        const int dyi = o / nd, ix = o - dyi * nd;
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int dx = 0; dx < n; ++dx) cmac(acc, M[dyi * n + dx], G[dx * nd + ix]);
        P[o] = acc;
    }
    __syncwarp();
    // B[iy][ix] = Re sum_dy G[iy][dy] P[dy][ix]
    for (int o = lane; o < nd * nd; o += 32) {
        const int iy = o / nd, ix = o - iy * nd;
        float sum = 0.0f;
#pragma unroll
        for (int dyi = 0; dyi < D2; ++dyi) {
            const int dy = dyi - (n - 1);
            float2 gg = G[(dy >= 0 ? dy : -dy) * nd + iy];
            if (dy < 0) gg.y = -gg.y;
            const float2 pv = P[dyi * nd + ix];
            sum = fmaf(gg.x, pv.x, fmaf(-gg.y, pv.y, sum));
        }
        B[o] = sum;
    }
    __syncwarp();
}

// NGS: b x b binning of the spot image rows I ([N][N + 1] floats) into B [nd][nd].
template <int N, int nd>
__device__ __forceinline__ void ngs_direct(const float *I, float *B, int lane) {
    constexpr int b = N / nd;
    for (int o = lane; o < nd * nd; o += 32) {
        const int iy = o / nd, ix = o - iy * nd;
        float sum = 0.0f;
#pragma unroll
        for (int r = 0; r < b; ++r)
#pragma unroll
            for (int c = 0; c < b; ++c) sum += I[(b * iy + r) * (N + 1) + b * ix + c];
        B[o] = sum;
    }
    __syncwarp();
}

// Photometry, noise (pixel by pixel) and the centroid of subaperture v from its binned image B
// [nd][nd] in the warp's shared memory; lane 0 writes the slopes.
template <int nd>
__device__ __forceinline__ void finish_direct(const float *B, const WfsDesc &W, const InstDyn &D, uint64_t seed,
                                              int v, int lane) {
    constexpr int nd2 = nd * nd;
    float sb = 0.0f;
    for (int o = lane; o < nd2; o += 32) sb += B[o];
    sb = warp_sum(sb);
    const float scale = sb > 0.0f ? W.photons * __ldg(W.fill + v) / sb : 0.0f;
    const float cd = 0.5f * (float)(nd - 1);
    const uint32_t tlo = (uint32_t)__double_as_longlong(D.t);
    const uint32_t thi = (uint32_t)((unsigned long long)__double_as_longlong(D.t) >> 32);
    float *st_E = D.st_E ? D.st_E + W.det_off + (size_t)v * nd2 : nullptr;
    float *st_C = D.st_C ? D.st_C + W.det_off + (size_t)v * nd2 : nullptr;
    float sc = 0.0f, sx = 0.0f, sy = 0.0f;
    for (int o = lane; o < nd2; o += 32) {
        const int iy = o / nd, ix = o - iy * nd;
        const float e = scale * B[o];
        const float c = D.noise ? noise_pixel(e, W.read_noise, seed, (uint32_t)(v * nd2 + o), (uint32_t)W.gs_index,
                                              tlo, thi)
                                : e;
        if (st_E) st_E[o] = e;
        if (st_C) st_C[o] = c;
        sc += c;
        sx = fmaf((float)ix - cd, c, sx);
        sy = fmaf((float)iy - cd, c, sy);
    }
    sc = warp_sum(sc);
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) {
        const bool ok = sc > 0.0f;
        float *sl = D.slopes + W.slope_off;
        sl[2 * v] = ok ? sx / sc : 0.0f;
        sl[2 * v + 1] = ok ? sy / sc : 0.0f;
    }
}

}  // namespace tail
}  // namespace gbwfs
