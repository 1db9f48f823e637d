// k_sh_n32.cu -- the FP32 spot kernel specialised for a 32-point DFT (the ELT
// LGS geometry: n = 10 pupil pixels, N = 32, 16x16 detector pixels).
//
// Same arithmetic as k_sh.cu (Sec. 4 LGS SH: spot by DFT, sodium elongation,
// binning, noise, centroid), mapped so that one warp owns one subaperture and
// lane k owns DFT row k:
//   U[k][q]  = sum_p F[k][p] X[p][q]                 (lanes k, k + 16: even and odd p)
//   Y[k][m]  = sum_q U[k][q] F[m][q],  I = |Y|^2       (lane k, columns m + 8j together)
//   Ta[k][dx] = sum_m I[k][m] Ga[dx][m]               (fused: I never stored)
//   M[dy][dx] = Kt[dy][dx] sum_k Ga[dy][k] Ta[k][dx]  (DFT across the lanes)
//   Q[iy][dx] = sum_dy G[dy][iy] M[dy][dx]            (16-point DFT across the lane pairs)
//   B[iy][ix] = Re sum_dx Q[iy][dx] G[dx][ix]         (lane = ix, half-warp = iy half)
// then photometry, noise and the centroid with warp reductions.  All sizes are
// compile-time constants.
//
// The per-slice variant (kSlices, launched with ShArgs::slice_opd_stride) runs the LGS per-slice
// model (Sec. 4: one wavefront and one spot per sodium sub-layer, piled up with the profile
// weights): the projection has made one OPD per slice (the layers through the slice's cone);
// per slice the warp adds the slice's geometric term, and the weighted spots are summed in the
// warp's shared rows before the first inverse-transform stage T.
#include "internal.h"
#include "noise.cuh"
#include "spot_tail.cuh"

namespace gbwfs {

namespace {

__device__ __forceinline__ void cmac2(float2 &acc, const float2 a, const float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

// The first transfer-domain stage for the columns (m, m + 8, m + 16, m + 24) of a 32-point
// row: Ga[d][m + 8j] = i^(jd) Ga[d][m], so T[d] += (sum_j i^(jd) I[m + 8j]) Ga[d][m], whose
// coefficient is real for even d (I0 + I1 + I2 + I3 or I0 - I1 + I2 - I3) and complex for odd d
// ((I0 - I2) +/- i (I1 - I3)).  ga: Ga[.][m] for d < n.
template <int n>
__device__ __forceinline__ void ta_quad(float2 (&T)[n], const float (&iv)[4], const float2 *ga) {
    const float P = iv[0] + iv[2], M = iv[0] - iv[2], Q = iv[1] + iv[3], R = iv[1] - iv[3];
    const float V0 = P + Q, V2 = P - Q;
#pragma unroll
    for (int d = 0; d < n; ++d) {
        const float2 g = ga[d];
        if ((d & 3) == 0 || (d & 3) == 2) {
            const float V = (d & 3) == 0 ? V0 : V2;
            T[d].x = fmaf(V, g.x, T[d].x);
            T[d].y = fmaf(V, g.y, T[d].y);
        } else {
            const float Ri = (d & 3) == 1 ? R : -R;  // V = M + i Ri
            T[d].x = fmaf(M, g.x, fmaf(-Ri, g.y, T[d].x));
            T[d].y = fmaf(M, g.y, fmaf(Ri, g.x, T[d].y));
        }
    }
}

template <int n, int nd, bool kSlices = false>
struct N32Layout {
    static constexpr int N = 32, D2 = 2 * n - 1;
    // per-CTA tables (float2 units)
    static constexpr int oFk = 0;                 // [p][k]   F[k][p]      (lane-k column)
    static constexpr int oFm = oFk + n * N;        // [m][q]   F[m][q]      (broadcast rows)
    static constexpr int oGam = oFm + N * n;       // [m][dx]  Ga[dx][m]    (broadcast rows)
    static constexpr int oFft = oGam + N * n;      // lane-DFT twiddles and phases (tail::fill_fft_table)
    static constexpr int oG = oFft + tail::kFftTable;  // [d][nd]  G[d][i]
    static constexpr int oRk = oG + n * nd;         // RN(1/k) for the Poisson inversion (floats)
    static constexpr int table = oRk + kRecipTable / 2;
    // per-warp scratch (float2 units)
    static constexpr int wX = 0;                   // [p][q]
    static constexpr int wTa = wX + n * n;         // Q: [nd][n]
    static constexpr int wI = wTa + nd * n;        // [k][N+1] floats (NGS binning only)
    static constexpr int warp = wI + (N * (N + 1) + 1) / 2;
    static_assert(table % 2 == 0 && warp % 2 == 0 && wTa % 2 == 0,
                  "16-byte aligned column-pair scratch");
};

}  // namespace

template <int n, int nd, bool kSlices>
__global__ void __launch_bounds__(256, 2) k_sh_n32(const __grid_constant__ ShArgs a) {
    using Lay = N32Layout<n, nd, kSlices>;
    constexpr int N = 32, D2 = Lay::D2;
    constexpr int nd2 = nd * nd;
    static_assert(nd <= 32 && nd2 % 32 == 0, "detector tile must split evenly over a warp");
    extern __shared__ __align__(16) float2 sm2[];
    float2 *Fk = sm2 + Lay::oFk, *Fm = sm2 + Lay::oFm, *Gam = sm2 + Lay::oGam;
    float2 *fft = sm2 + Lay::oFft, *Gt = sm2 + Lay::oG;
    // global tables: F[q*N + m] = F[m][q]; Ga[d*N + k]; G[d*nd + i]
    for (int i = threadIdx.x; i < n * N; i += blockDim.x) {
        const int q = i / N, m = i - q * N;
        const float2 f = a.F[i];
        Fk[q * N + m] = f;          // [p][k] with p = q, k = m
        Fm[m * n + q] = f;          // [m][q]
        const int d = q, k = m;     // Ga has the same [d][k] shape
        const float2 g = a.Ga[i];
        Gam[k * n + d] = g;
    }
    for (int i = threadIdx.x; i < n * nd; i += blockDim.x) Gt[i] = a.G[i];
    float *rk = reinterpret_cast<float *>(sm2 + Lay::oRk);
    fill_recip_table(rk, threadIdx.x, blockDim.x);
    tail::fill_fft_table<n>(fft, threadIdx.x, blockDim.x);
    __syncthreads();
    wait_prior_grid();
    if (a.split_noise) allow_dependent_grid();  // the noise kernel may take SMs as CTAs retire

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float2 *X = sm2 + Lay::table + wib * Lay::warp + Lay::wX;
    float2 *Ta = sm2 + Lay::table + wib * Lay::warp + Lay::wTa;
    float *Iw = reinterpret_cast<float *>(sm2 + Lay::table + wib * Lay::warp + Lay::wI);

    // Work split: each warp starts with subaperture blockIdx.x * nw + wib; with a.work, lane 0
    // draws one ticket per iteration (issued at the top, used at the bottom).
    const int nwarps = gridDim.x * nw;
    for (int g = blockIdx.x * nw + wib; g < a.total;) {
        int ticket = 0;
        if (a.work && lane == 0) ticket = atomicAdd(a.work, 1);
        const WfsDesc &W = a.wfs[find_wfs(a.wfs, a.n_wfs, g)];
        const InstDyn &D = a.dyn[W.inst];
        const uint64_t seed = a.inst[W.inst].seed;
        const uint32_t tlo = (uint32_t)__double_as_longlong(D.t);
        const uint32_t thi = (uint32_t)((unsigned long long)__double_as_longlong(D.t) >> 32);
        const int v = g - W.subap_begin;
        __syncwarp();
        if (!guard(v >= 0 && v < W.n_valid, a.status)) {  // uniform over the warp
            g = a.work ? nwarps + __shfl_sync(0xffffffffu, ticket, 0) : g + nwarps;
            continue;
        }

        const SliceDesc *SD = kSlices ? W.slices : nullptr;
        const int n_sl = SD ? SD->n : 1;
        const uint32_t *mk = W.mask + (size_t)v * a.mask_words;
        float2 T[n];
#pragma unroll
        for (int d = 0; d < n; ++d) T[d] = make_float2(0.0f, 0.0f);
        float *stI = D.st_I ? D.st_I + W.int_off + (size_t)v * (N * N) + lane * N : nullptr;
        // per-slice model: the slice's geometric term k_s ((x - r_b).(r_b - r_L) + 1/2 |x - r_b|^2)
        // about the subaperture centre r_b, added to the slice's projected OPD
        float ebx = 0.0f, eby = 0.0f, dxp = 0.0f;
        if (SD) {
            const InstDesc &I = a.inst[W.inst];
            const int id = __ldg(W.subap + v), sy = id / W.n_sub, sx = id - sy * W.n_sub;
            const float half = 0.5f * (float)(W.n_sub * n - 1), c0 = 0.5f * (float)(n - 1);
            dxp = (float)(W.pupil_dx_over_ds * I.ds);
            ebx = ((float)(sx * n) + c0 - half) * dxp - (float)W.launch_x;
            eby = ((float)(sy * n) + c0 - half) * dxp - (float)W.launch_y;
        }
        for (int sl = 0; sl < n_sl; ++sl) {
            const float *opd = D.opd + W.opd_off + (size_t)sl * a.slice_opd_stride + (size_t)v * (n * n);
            const float ks = SD ? SD->k[sl] : 0.0f;
            auto geo = [&](int i) -> float {
                const int pp = i / n, qq = i - pp * n;
                const float ux = ((float)qq - 0.5f * (float)(n - 1)) * dxp;
                const float uy = ((float)pp - 0.5f * (float)(n - 1)) * dxp;
                return ks * fmaf(ux, ebx, fmaf(uy, eby, 0.5f * fmaf(ux, ux, uy * uy)));
            };
            // field, piston-free
            const float ref = __ldg(opd) + (kSlices ? geo(0) : 0.0f);
            // all of the lane's loads first (element i = lane + 32 m, mask word m)
            constexpr int kFw = (n * n + 31) / 32;
            float o[kFw];
            uint32_t mw[kFw];
#pragma unroll
            for (int m = 0; m < kFw; ++m) {
                o[m] = lane + 32 * m < n * n ? __ldg(opd + lane + 32 * m) : 0.0f;
                mw[m] = __ldg(mk + m);
            }
#pragma unroll
            for (int m = 0; m < kFw; ++m) {
                const int i = lane + 32 * m;
                if (i < n * n) {
                    const bool lit = (mw[m] >> lane) & 1u;
                    float s, c;
                    field_phasor(W.k_phase * ((o[m] + (kSlices ? geo(i) : 0.0f)) - ref), s, c);
                    X[i] = lit ? make_float2(c, s) : make_float2(0.0f, 0.0f);
                }
            }
            __syncwarp();

            // U[k][q], k = lane.  F[k + 16][p] = F[k][p] (-1)^p i^(n-1): the lane k < 16 sums the
            // even p and the lane k + 16 the odd p, both with row k of F; after one exchange
            // U[k] = E + O and U[k + 16] = i^(n-1) (E - O)
            float2 U[n];
#pragma unroll
            for (int q = 0; q < n; ++q) U[q] = make_float2(0.0f, 0.0f);
            const bool upper = lane >= N / 2;
            const int k16 = lane & (N / 2 - 1);
#pragma unroll
            for (int j = 0; j < n / 2; ++j) {
                const int p = 2 * j + (upper ? 1 : 0);
                const float2 f = Fk[p * N + k16];
#pragma unroll
                for (int q = 0; q < n; ++q) cmac2(U[q], f, X[p * n + q]);
            }
            {
                constexpr float sr = ((n - 1) % 4 == 1) ? 1.0f : -1.0f;  // i^(n-1) = sr i
#pragma unroll
                for (int q = 0; q < n; ++q) {
                    const float ox = __shfl_xor_sync(0xffffffffu, U[q].x, N / 2);
                    const float oy = __shfl_xor_sync(0xffffffffu, U[q].y, N / 2);
                    if (upper) {
                        const float dx = ox - U[q].x, dy = oy - U[q].y;
                        U[q] = make_float2(-sr * dy, sr * dx);
                    } else {
                        U[q] = make_float2(U[q].x + ox, U[q].y + oy);
                    }
                }
            }

            // Y, I (times the slice's weight) and the first inverse-transform stage, by column
            // quadruples (m, m + 8, m + 16, m + 24): F[m + 8j][q] = F[m][q] (-i)^(jq) exp(i pi j cn / 2),
            // so |Y[m + 8j]| = |T_j| with T_j = sum_r (-i)^(jr) S_r, S_r the sum over q = r mod 4
            // (a 4-point DFT of the S_r); Ta adds the quadruple through ta_quad
            const float wsl = SD ? SD->w[sl] : 1.0f;
#pragma unroll 2
            for (int m = 0; m < N / 4; ++m) {
                float2 S[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) S[r] = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int q = 0; q < n; ++q) cmac2(S[q & 3], U[q], Fm[m * n + q]);
                const float2 A = make_float2(S[0].x + S[2].x, S[0].y + S[2].y);
                const float2 B = make_float2(S[0].x - S[2].x, S[0].y - S[2].y);
                const float2 C = make_float2(S[1].x + S[3].x, S[1].y + S[3].y);
                const float2 Dd = make_float2(S[1].x - S[3].x, S[1].y - S[3].y);
                // T0 = A + C, T1 = B - i D, T2 = A - C, T3 = B + i D
                const float2 Tq[4] = {make_float2(A.x + C.x, A.y + C.y), make_float2(B.x + Dd.y, B.y - Dd.x),
                                      make_float2(A.x - C.x, A.y - C.y), make_float2(B.x - Dd.y, B.y + Dd.x)};
                float iv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    iv[j] = fmaf(Tq[j].x, Tq[j].x, Tq[j].y * Tq[j].y);
                    if (SD) iv[j] *= wsl;
                }
                if (stI) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) stI[m + 8 * j] = sl == 0 ? iv[j] : stI[m + 8 * j] + iv[j];
                }
                if (kSlices) {
                    // the slices' spots summed in the warp's rows; T once after the last slice
                    float *ir = Iw + lane * (N + 1) + m;
#pragma unroll
                    for (int j = 0; j < 4; ++j) ir[8 * j] = sl == 0 ? iv[j] : ir[8 * j] + iv[j];
                } else if (W.is_lgs) {
                    ta_quad<n>(T, iv, Gam + m * n);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) Iw[lane * (N + 1) + m + 8 * j] = iv[j];
                }
            }
            __syncwarp();  // X and the slice's OPD are rewritten by the next slice
        }
        if (kSlices && W.is_lgs) {
#pragma unroll 2
            for (int m = 0; m < N / 4; ++m) {
                float iv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) iv[j] = Iw[lane * (N + 1) + m + 8 * j];
                ta_quad<n>(T, iv, Gam + m * n);
            }
        }

        float Bv[nd / 2];  // B[iy][ix] for iy = half*(nd/2) + j
        if (W.is_lgs) {
            tail::lgs_binned<n, nd>(T, reinterpret_cast<float4 *>(Ta), fft, Gt,
                                       W.ktil + (size_t)v * (D2 * n), lane, Bv);
        } else {
            __syncwarp();
            tail::ngs_binned<nd>(Iw, lane, Bv);
        }
        tail::finish<nd>(Bv, W, D, seed, v, lane, rk, a.split_noise != 0);
        g = a.work ? nwarps + __shfl_sync(0xffffffffu, ticket, 0) : g + nwarps;
    }
    if (a.work) {
        // every ticket of this CTA was drawn before the barrier; the last CTA to get here leaves
        // the counters at zero for the next launch
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(a.work + 1, 1) == (int)gridDim.x - 1) {
                a.work[0] = 0;
                a.work[1] = 0;
            }
        }
    }
}

namespace {
template <int n, int nd, bool kSlices>
cudaError_t shape_n32_k(const ShArgs &a, LaunchShape *out) {
    using Lay = N32Layout<n, nd, kSlices>;
    const int warps = (a.cta_warps == 4 || a.cta_warps == 8) ? a.cta_warps : 8;
    const size_t smem = (size_t)(Lay::table + warps * Lay::warp) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_sh_n32<n, nd, kSlices>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = (a.total + warps - 1) / warps;
    const int cap = a.grid_cap > 0 ? a.grid_cap : 152 * 2 * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    out->func = (const void *)k_sh_n32<n, nd, kSlices>;
    out->grid = dim3(blocks);
    out->block = dim3(warps * 32);
    out->smem = smem;
    return cudaSuccess;
}

// ShArgs::slice_opd_stride selects the per-slice variant.
template <int n, int nd>
cudaError_t shape_n32(const ShArgs &a, LaunchShape *out) {
    return a.slice_opd_stride > 0 ? shape_n32_k<n, nd, true>(a, out) : shape_n32_k<n, nd, false>(a, out);
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
