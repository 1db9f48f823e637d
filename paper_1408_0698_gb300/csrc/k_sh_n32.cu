// k_sh_n32.cu -- the FP32 spot kernel specialised for a 32-point DFT (the ELT
// LGS geometry: n = 10 pupil pixels, N = 32, 16x16 detector pixels).
//
// Same arithmetic as k_sh.cu (Sec. 4 LGS SH: spot by DFT, sodium elongation,
// binning, noise, centroid), mapped so that one warp owns one subaperture and
// lane k owns DFT row k:
//   U[k][q]  = sum_p F[k][p] X[p][q]                 (lanes k, k + 16: even and odd p)
//   Y[k][m]  = sum_q U[k][q] F[m][q],  I = |Y|^2       (lane k, column pairs m, m + 16)
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
            // pairs (m, m + 16): F[m + 16][q] = F[m][q] (-1)^q i^(n-1), so Y[m] = E + O and
            // |Y[m + 16]| = |E - O| with E, O the sums over the even and the odd q; and
            // Ga[d][m + 16] = (-1)^d Ga[d][m], so the pair adds (I[m] +/- I[m + 16]) Ga[d][m]
            const float wsl = SD ? SD->w[sl] : 1.0f;
#pragma unroll 2
            for (int m = 0; m < N / 2; ++m) {
                float2 e = make_float2(0.0f, 0.0f), o = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int q = 0; q < n; q += 2) {
                    cmac2(e, U[q], Fm[m * n + q]);
                    cmac2(o, U[q + 1], Fm[m * n + q + 1]);
                }
                const float2 yl = make_float2(e.x + o.x, e.y + o.y), yh = make_float2(e.x - o.x, e.y - o.y);
                float il = fmaf(yl.x, yl.x, yl.y * yl.y), ih = fmaf(yh.x, yh.x, yh.y * yh.y);
                if (SD) {
                    il *= wsl;
                    ih *= wsl;
                }
                if (stI) {
                    stI[m] = sl == 0 ? il : stI[m] + il;
                    stI[m + N / 2] = sl == 0 ? ih : stI[m + N / 2] + ih;
                }
                if (kSlices) {
                    // the slices' spots summed in the warp's rows; T once after the last slice
                    float *ir = Iw + lane * (N + 1) + m;
                    ir[0] = sl == 0 ? il : ir[0] + il;
                    ir[N / 2] = sl == 0 ? ih : ir[N / 2] + ih;
                } else if (W.is_lgs) {
                    const float sp = il + ih, sm = il - ih;
#pragma unroll
                    for (int d = 0; d < n; ++d) {
                        const float2 ga = Gam[m * n + d];
                        const float in = (d & 1) ? sm : sp;
                        T[d].x = fmaf(in, ga.x, T[d].x);
                        T[d].y = fmaf(in, ga.y, T[d].y);
                    }
                } else {
                    Iw[lane * (N + 1) + m] = il;
                    Iw[lane * (N + 1) + m + N / 2] = ih;
                }
            }
            __syncwarp();  // X and the slice's OPD are rewritten by the next slice
        }
        if (kSlices && W.is_lgs) {
#pragma unroll 2
            for (int m = 0; m < N / 2; ++m) {
                const float il = Iw[lane * (N + 1) + m], ih = Iw[lane * (N + 1) + m + N / 2];
                const float sp = il + ih, sm = il - ih;
#pragma unroll
                for (int d = 0; d < n; ++d) {
                    const float2 ga = Gam[m * n + d];
                    const float in = (d & 1) ? sm : sp;
                    T[d].x = fmaf(in, ga.x, T[d].x);
                    T[d].y = fmaf(in, ga.y, T[d].y);
                }
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
