// k_sh_n32.cu -- the FP32 spot kernel specialised for a 32-point DFT (the ELT
// LGS geometry: n = 10 pupil pixels, N = 32, 16x16 detector pixels).
//
// Same arithmetic as k_sh.cu (Sec. 4 LGS SH: spot by DFT, sodium elongation,
// binning, noise, centroid), mapped so that one warp owns one subaperture and
// lane k owns DFT row k:
//   U[k][q]  = sum_p F[k][p] X[p][q]                 (lane k, registers)
//   Y[k][m]  = sum_q U[k][q] F[m][q],  I = |Y|^2       (lane k, m looped)
//   Ta[k][dx] = sum_m I[k][m] Ga[dx][m]               (fused: I never stored)
//   M[dy][dx] = Kt[dy][dx] sum_k Ga[dy][k] Ta[k][dx]  (2x2 register tiles)
//   P[dy][ix] = sum_dx M[dy][dx] G[dx][ix]            (lane = ix, half-warp = dy half)
//   B[iy][ix] = Re sum_dy G[dy][iy] P[dy][ix]         (half-warp partials + one shuffle)
// then photometry, noise and the centroid with warp reductions.  All sizes are
// compile-time constants.
#include "internal.h"
#include "noise.cuh"

namespace gbwfs {

namespace {

__device__ __forceinline__ void cmac2(float2 &acc, const float2 a, const float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int n, int nd>
struct N32Layout {
    static constexpr int N = 32, D2 = 2 * n - 1, NO = n | 1, GAK = 33;
    // per-CTA tables (float2 units)
    static constexpr int oFk = 0;                 // [p][k]   F[k][p]      (lane-k column)
    static constexpr int oFm = oFk + n * N;        // [m][q]   F[m][q]      (broadcast rows)
    static constexpr int oGam = oFm + N * n;       // [m][dx]  Ga[dx][m]    (broadcast rows)
    static constexpr int oGak = oGam + N * n;      // [d][GAK] Ga[d][k]     (padded rows)
    static constexpr int oG = oGak + n * GAK;      // [d][nd]  G[d][i]
    static constexpr int table = oG + n * nd;
    // per-warp scratch (float2 units)
    static constexpr int wX = 0;                   // [p][q]
    static constexpr int wTa = wX + n * n;         // [k][NO]
    static constexpr int wM = wTa + N * NO;        // [dyi][n]
    static constexpr int wI = wM + D2 * n;         // [k][N+1] floats (NGS binning only)
    static constexpr int warp = wI + (N * (N + 1) + 1) / 2;
};

}  // namespace

template <int n, int nd>
__global__ void __launch_bounds__(256, 2) k_sh_n32(const __grid_constant__ ShArgs a) {
    using Lay = N32Layout<n, nd>;
    constexpr int N = 32, D2 = Lay::D2, NO = Lay::NO, GAK = Lay::GAK, b = N / nd;
    constexpr int nd2 = nd * nd;
    static_assert(nd <= 32 && nd2 % 32 == 0, "detector tile must split evenly over a warp");
    extern __shared__ __align__(16) float2 sm2[];
    float2 *Fk = sm2 + Lay::oFk, *Fm = sm2 + Lay::oFm, *Gam = sm2 + Lay::oGam;
    float2 *Gak = sm2 + Lay::oGak, *Gt = sm2 + Lay::oG;
    // global tables: F[q*N + m] = F[m][q]; Ga[d*N + k]; G[d*nd + i]
    for (int i = threadIdx.x; i < n * N; i += blockDim.x) {
        const int q = i / N, m = i - q * N;
        const float2 f = a.F[i];
        Fk[q * N + m] = f;          // [p][k] with p = q, k = m
        Fm[m * n + q] = f;          // [m][q]
        const int d = q, k = m;     // Ga has the same [d][k] shape
        const float2 g = a.Ga[i];
        Gam[k * n + d] = g;
        Gak[d * GAK + k] = g;
    }
    for (int i = threadIdx.x; i < n * nd; i += blockDim.x) Gt[i] = a.G[i];
    __syncthreads();

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float2 *X = sm2 + Lay::table + wib * Lay::warp + Lay::wX;
    float2 *Ta = sm2 + Lay::table + wib * Lay::warp + Lay::wTa;
    float2 *Mw = sm2 + Lay::table + wib * Lay::warp + Lay::wM;
    float *Iw = reinterpret_cast<float *>(sm2 + Lay::table + wib * Lay::warp + Lay::wI);

    const float cd = 0.5f * (float)(nd - 1);
    const int ix = lane & 15, half = lane >> 4;

    for (int g = blockIdx.x * nw + wib; g < a.total; g += gridDim.x * nw) {
        const WfsDesc &W = a.wfs[find_wfs(a.wfs, a.n_wfs, g)];
        const InstDyn &D = a.dyn[W.inst];
        const uint64_t seed = a.inst[W.inst].seed;
        const uint32_t tlo = (uint32_t)__double_as_longlong(D.t);
        const uint32_t thi = (uint32_t)((unsigned long long)__double_as_longlong(D.t) >> 32);
        const int v = g - W.subap_begin;
        float *st_E = D.st_E ? D.st_E + W.det_off : nullptr;
        float *st_C = D.st_C ? D.st_C + W.det_off : nullptr;
        __syncwarp();

        // field, piston-free
        const float *opd = D.opd + W.opd_off + (size_t)v * (n * n);
        const uint32_t *mk = W.mask + (size_t)v * a.mask_words;
        const float ref = __ldg(opd);
        for (int i = lane; i < n * n; i += 32) {
            const bool lit = (__ldg(mk + (i >> 5)) >> (i & 31)) & 1u;
            float s, c;
            sincosf(W.k_phase * (__ldg(opd + i) - ref), &s, &c);
            X[i] = lit ? make_float2(c, s) : make_float2(0.0f, 0.0f);
        }
        __syncwarp();

        // U[k][q], k = lane
        float2 U[n];
#pragma unroll
        for (int q = 0; q < n; ++q) U[q] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int p = 0; p < n; ++p) {
            const float2 f = Fk[p * N + lane];
#pragma unroll
            for (int q = 0; q < n; ++q) cmac2(U[q], f, X[p * n + q]);
        }

        // Y, I and the first inverse-transform stage, row by row
        float2 T[n];
#pragma unroll
        for (int d = 0; d < n; ++d) T[d] = make_float2(0.0f, 0.0f);
        float *stI = D.st_I ? D.st_I + W.int_off + (size_t)v * (N * N) + lane * N : nullptr;
#pragma unroll 2
        for (int m = 0; m < N; ++m) {
            float2 y = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int q = 0; q < n; ++q) cmac2(y, U[q], Fm[m * n + q]);
            const float in = fmaf(y.x, y.x, y.y * y.y);
            if (stI) stI[m] = in;
            if (W.is_lgs) {
#pragma unroll
                for (int d = 0; d < n; ++d) {
                    const float2 ga = Gam[m * n + d];
                    T[d].x = fmaf(in, ga.x, T[d].x);
                    T[d].y = fmaf(in, ga.y, T[d].y);
                }
            } else {
                Iw[lane * (N + 1) + m] = in;
            }
        }

        float Bv[nd / 2];  // B[iy][ix] for iy = half*(nd/2) + j
        if (W.is_lgs) {
#pragma unroll
            for (int d = 0; d < n; ++d) Ta[lane * NO + d] = T[d];
            __syncwarp();
            // M = Kt * (Ga_y Ta): 2x2 tiles over (dy pair, dx pair)
            const float2 *kt = W.ktil + (size_t)v * (D2 * n);
            constexpr int DYP = (D2 + 1) / 2, DXP = (n + 1) / 2, TASKS = DYP * DXP;
            for (int task = lane; task < TASKS; task += 32) {
                const int dyp = task / DXP, dxp = task - dyp * DXP;
                const int dyi0 = 2 * dyp, dx0 = 2 * dxp;
                const int dy0 = dyi0 - (n - 1), dy1 = dy0 + 1;
                const bool has_dy1 = dyi0 + 1 < D2, has_dx1 = dx0 + 1 < n;
                const float2 *g0 = Gak + (dy0 >= 0 ? dy0 : -dy0) * GAK;
                const float2 *g1 = Gak + (dy1 >= 0 ? dy1 : -dy1) * GAK;
                const float s0 = dy0 >= 0 ? 1.0f : -1.0f, s1 = dy1 >= 0 ? 1.0f : -1.0f;
                float2 c00 = make_float2(0.f, 0.f), c01 = c00, c10 = c00, c11 = c00;
#pragma unroll 4
                for (int k = 0; k < N; ++k) {
                    float2 ga0 = g0[k], ga1 = g1[k];
                    ga0.y *= s0;
                    ga1.y *= s1;
                    const float2 t0 = Ta[k * NO + dx0];
                    const float2 t1 = has_dx1 ? Ta[k * NO + dx0 + 1] : make_float2(0.f, 0.f);
                    cmac2(c00, ga0, t0);
                    cmac2(c01, ga0, t1);
                    cmac2(c10, ga1, t0);
                    cmac2(c11, ga1, t1);
                }
                auto put = [&](int dyi, int dx, float2 c) {
                    const float2 kv = __ldg(kt + dyi * n + dx);
                    Mw[dyi * n + dx] = make_float2(c.x * kv.x - c.y * kv.y, c.x * kv.y + c.y * kv.x);
                };
                put(dyi0, dx0, c00);
                if (has_dx1) put(dyi0, dx0 + 1, c01);
                if (has_dy1) {
                    put(dyi0 + 1, dx0, c10);
                    if (has_dx1) put(dyi0 + 1, dx0 + 1, c11);
                }
            }
            __syncwarp();
            // P for this half's dy rows, then partial B over those rows
            constexpr int HALF_DY = (D2 + 1) / 2;
            const int dyi_begin = half * HALF_DY;
            float2 Gc[n];
#pragma unroll
            for (int d = 0; d < n; ++d) Gc[d] = ix < nd ? Gt[d * nd + ix] : make_float2(0.f, 0.f);
            float Bp[nd];
#pragma unroll
            for (int i = 0; i < nd; ++i) Bp[i] = 0.0f;
#pragma unroll
            for (int j = 0; j < HALF_DY; ++j) {
                const int dyi = dyi_begin + j;
                if (dyi < D2) {
                    float2 p = make_float2(0.f, 0.f);
#pragma unroll
                    for (int d = 0; d < n; ++d) cmac2(p, Mw[dyi * n + d], Gc[d]);
                    const int dy = dyi - (n - 1);
                    const float2 *gr = Gt + (dy >= 0 ? dy : -dy) * nd;
                    const float sg = dy >= 0 ? 1.0f : -1.0f;
#pragma unroll
                    for (int i = 0; i < nd; ++i) {
                        const float2 gv = gr[i];
                        Bp[i] = fmaf(gv.x, p.x, fmaf(-sg * gv.y, p.y, Bp[i]));
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < nd; ++i) Bp[i] += __shfl_xor_sync(0xffffffffu, Bp[i], 16);
#pragma unroll
            for (int j = 0; j < nd / 2; ++j) Bv[j] = half ? Bp[nd / 2 + j] : Bp[j];
        } else {
            __syncwarp();
#pragma unroll
            for (int j = 0; j < nd / 2; ++j) {
                const int iy = half * (nd / 2) + j;
                float s = 0.0f;
#pragma unroll
                for (int r = 0; r < b; ++r)
#pragma unroll
                    for (int c = 0; c < b; ++c) s += Iw[(b * iy + r) * (N + 1) + b * ix + c];
                Bv[j] = s;
            }
        }

        // photometry, noise, centroid (lane holds column ix, rows half*nd/2 ...)
        float sb = 0.0f;
        if (ix < nd) {
#pragma unroll
            for (int j = 0; j < nd / 2; ++j) sb += Bv[j];
        }
        sb = warp_sum(sb);
        const float scale = sb > 0.0f ? W.photons * __ldg(W.fill + v) / sb : 0.0f;
        float sc = 0.0f, sx = 0.0f, sy = 0.0f;
        if (ix < nd) {
#pragma unroll
            for (int j = 0; j < nd / 2; ++j) {
                const int iy = half * (nd / 2) + j, o = iy * nd + ix;
                const float e = scale * Bv[j];
                const float c = D.noise ? noise_pixel(e, W.read_noise, seed, (uint32_t)(v * nd2 + o),
                                                      (uint32_t)W.gs_index, tlo, thi)
                                        : e;
                if (st_E) st_E[(size_t)v * nd2 + o] = e;
                if (st_C) st_C[(size_t)v * nd2 + o] = c;
                sc += c;
                sx = fmaf((float)ix - cd, c, sx);
                sy = fmaf((float)iy - cd, c, sy);
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
}

namespace {
template <int n, int nd>
cudaError_t shape_n32(const ShArgs &a, LaunchShape *out) {
    using Lay = N32Layout<n, nd>;
    const int warps = (a.cta_warps == 4 || a.cta_warps == 8) ? a.cta_warps : 8;
    const size_t smem = (size_t)(Lay::table + warps * Lay::warp) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_sh_n32<n, nd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = (a.total + warps - 1) / warps;
    const int cap = a.grid_cap > 0 ? a.grid_cap : 152 * 2 * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    out->func = (const void *)k_sh_n32<n, nd>;
    out->grid = dim3(blocks);
    out->block = dim3(warps * 32);
    out->smem = smem;
    return cudaSuccess;
}
}  // namespace

bool sh_n32_supported(int n, int N, int nd) {
    return N == 32 && ((n == 10 && nd == 16) || (n == 8 && nd == 16));
}

cudaError_t n32_launch_shape(const ShArgs &a, LaunchShape *out) {
    if (a.n == 10 && a.nd == 16) return shape_n32<10, 16>(a, out);
    if (a.n == 8 && a.nd == 16) return shape_n32<8, 16>(a, out);
    return cudaErrorInvalidValue;
}

}  // namespace gbwfs
