// k_sh_tc.cu -- the spot kernel with the DFT contraction on the 5th-generation
// tensor cores (tcgen05, BF16 hi/lo split with three products, FP32
// accumulation in tensor memory; or the same with FP16 hi/lo and per-subaperture
// power-of-two operand scaling), for 32-point DFT geometries with n <= 10.
//
// Arithmetic (Sec. 4 LGS SH: spot by DFT, sodium elongation, binning, noise,
// centroid) is that of k_sh.cu; only the two contractions whose second operand
// is a constant matrix shared by all subapertures run on the tensor cores:
//
//   Y = U F^T   rows (subaperture b, DFT row k): M = 4 x 32 = 128, N = 64
//               (re/im x 32 columns), K = [U_hi | U_lo | U_hi] x [F_hi; F_hi; F_lo]
//               = 3 x 2n (complex as real pairs), zero-padded to 64
//   Ta = I Ga^T rows (b, k): M = 128, N = 32 (re/im x 16 dx), K = [I_hi | I_lo]
//               x [Ga_hi; Ga_hi] (64) then [I_hi | I_lo] x [Ga_lo; 0] (64)
//
// Each BF16 pair (x_hi, x_lo = bf16(x - x_hi)) carries ~16 significant bits; the
// dropped lo*lo products are ~2^-16 of each term.  An FP16 pair carries ~22 bits once the
// operand is scaled into FP16's normal range (TcElt).  Operands live in shared memory
// in the 128-byte-swizzled K-major layout (8-row x 128-byte atoms); one elected
// thread issues the MMAs and commits them to an mbarrier; every wait is bounded
// and a timeout is reported in the status word (the kernel then frees its tensor
// memory and returns).  U = F X, the column transform, binning, photometry,
// noise and the centroid run on the CUDA cores exactly as in the FP32 kernels.
//
// CTA = two warpgroups (4 warps each); warp w of a warpgroup owns subaperture 4g + w of its
// group g and its lane k owns DFT row k, which is also TMEM lane 32 w + k of both accumulators.
//
// The per-slice variant (k_sh_tc_sl, launched with ShArgs::slice_opd_stride) runs the LGS
// per-slice model (Sec. 4: one wavefront and one spot per sodium sub-layer, piled up with the
// profile weights): the projection has made one OPD per slice (the layers through the slice's
// cone); per slice the warp adds the slice's geometric term, forms U, and the warpgroup's
// Y = U F^T runs on the tensor cores; the weighted |Y|^2 of the slices are summed in the warp's
// shared rows, which then feed Ta = I Ga^T.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <string.h>

#include <vector>

#include "internal.h"
#include "noise.cuh"
#include "spot_tail.cuh"
#include "tcgen05.cuh"

namespace gbwfs {

namespace {

using namespace tc;

constexpr int kWG = 2;                   // independent warpgroups per CTA
constexpr int kTcThreads = 128 * kWG;
constexpr uint32_t kTmemCols = 128 * kWG;  // per warpgroup: D1 columns [0, 64), D2 [64, 96)
// The field X of one subaperture in the warp's scratch as column pairs: entry [p][q/2] holds
// (re q, re q+1, im q, im q+1) of row p (q even).
template <int n>
__device__ __forceinline__ void store_field(float4 *X4, int i, float c, float s) {
    const int p = i / n, q = i - p * n;
    float *e = reinterpret_cast<float *>(X4 + p * (n / 2) + (q >> 1)) + (q & 1);
    e[0] = c;
    e[2] = s;
}

// U[q] = sum_p F[k][p] X[p][q] for this lane's DFT row k (lanes k >= N get zeros).  The rows k
// and k + N/2 share F up to a sign and a quarter turn: F[k + N/2][p] = F[k][p] (-1)^p i^(n-1)
// (n even), so of each such pair the lane k sums the even p, E = sum F[k][p] X[p][q], and the
// lane k + N/2 the odd p, O, both with row k of F; after one exchange U[k] = E + O and
// U[k + N/2] = i^(n-1) (E - O).  Two columns per packed FP32x2 FMA (each half rounded as fmaf);
// per p, re += -f.im x.im then f.re x.re, im += f.im x.re then f.re x.im.  Call from the whole
// warp.
template <int n, int N>
__device__ __forceinline__ void field_rows(const float2 *Fk, const float4 *X4, int lane, float2 (&U)[n]) {
    constexpr int H = N / 2, P = n / 2;
    static_assert(n % 2 == 0 && N % 2 == 0, "even/odd halves of the rows and of the columns");
    const bool upper = lane >= H && lane < N;
    const int k = lane < N ? (upper ? lane - H : lane) : 0;
    float2 ur[P], ui[P];
#pragma unroll
    for (int c = 0; c < P; ++c) ur[c] = ui[c] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int p = 2 * j + (upper ? 1 : 0);
        const float2 f = Fk[p * N + k];
        const float2 fx = make_float2(f.x, f.x), fy = make_float2(f.y, f.y), nfy = make_float2(-f.y, -f.y);
#pragma unroll
        for (int c = 0; c < P; ++c) {
            const float4 x = X4[p * P + c];
            const float2 xr = make_float2(x.x, x.y), xi = make_float2(x.z, x.w);
            ur[c] = __ffma2_rn(fx, xr, __ffma2_rn(nfy, xi, ur[c]));
            ui[c] = __ffma2_rn(fx, xi, __ffma2_rn(fy, xr, ui[c]));
        }
    }
    // lower lane: own + partner's = E + O; upper: partner's - own = E - O, then times
    // i^(n-1) = s i (s = +1 for n = 2 mod 4, -1 for n = 0 mod 4): (re, im) -> (-s im, s re)
    const int src = lane < N ? (upper ? lane - H : lane + H) : lane;
    const float sg = upper ? -1.0f : 1.0f;
    constexpr float s = ((n - 1) % 4 == 1) ? 1.0f : -1.0f;
    const float2 sg2 = make_float2(sg, sg);
    const float2 A = upper ? make_float2(0.0f, 0.0f) : make_float2(1.0f, 1.0f);
    const float2 B = upper ? make_float2(-s, -s) : make_float2(0.0f, 0.0f);
    const float2 Cc = upper ? make_float2(s, s) : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int c = 0; c < P; ++c) {
        const float2 pr = make_float2(__shfl_sync(0xffffffffu, ur[c].x, src), __shfl_sync(0xffffffffu, ur[c].y, src));
        const float2 pi = make_float2(__shfl_sync(0xffffffffu, ui[c].x, src), __shfl_sync(0xffffffffu, ui[c].y, src));
        const float2 vr = __ffma2_rn(sg2, ur[c], pr), vi = __ffma2_rn(sg2, ui[c], pi);
        ur[c] = __ffma2_rn(vr, A, __fmul2_rn(vi, B));
        ui[c] = __ffma2_rn(vi, A, __fmul2_rn(vr, Cc));
    }
    const bool row = lane < N;
#pragma unroll
    for (int c = 0; c < P; ++c) {
        U[2 * c] = row ? make_float2(ur[c].x, ui[c].x) : make_float2(0.0f, 0.0f);
        U[2 * c + 1] = row ? make_float2(ur[c].y, ui[c].y) : make_float2(0.0f, 0.0f);
    }
}

template <int n, int N_, int nd, bool kSlices = false, bool kMmaU = false, int WG = kWG>
struct TcLayout {
    static constexpr int N = N_, D2 = 2 * n - 1, no = n | 1;
    // N = 32 with a 16 x 16 detector: the elongation stage as a DFT across the 32 lanes and
    // the noise in its own pass; other sizes: the stages as direct sums over the warp's rows
    static constexpr bool kLane = N == 32 && nd == 16;
    // byte offsets; tensor-core tiles first (1024-aligned)
    static constexpr int oB1 = 0;                  // 64 rows x 128 B: [F_hi; F_hi; F_lo] blocks
    static constexpr int oB2h = oB1 + 8192;        // 32 rows x 128 B: [Ga_hi; Ga_hi]
    static constexpr int oB2l = oB2h + 4096;       // 32 rows x 128 B: [Ga_lo; 0]
    // with U = F X as an MMA: 128 rows x 128 B, F's rows [F_hi | F_lo | F_hi] for each of the
    // four subapertures of a group
    static constexpr int oA0 = oB2l + 4096;
    // per warpgroup, 128 rows x 128 B: the fields [X_hi | X_hi | X_lo] of the group's four
    // subapertures (U = F X as an MMA), then [U_hi | U_lo | U_hi] for the DFT's second MMA,
    // then (after it has completed) [I_hi | I_lo] for the transfer-function MMA
    static constexpr int oA = oA0 + (kMmaU ? 16384 : 0);
    static constexpr int oTab = oA + 16384 * WG;  // CUDA-core tables (float2)
    static constexpr int tFk = 0;                  // [p][k]  F[k][p] (U = F X on the CUDA cores)
    static constexpr int tFft = tFk + (kMmaU ? 0 : n * N);  // lane-DFT twiddles and phases (tail::fill_fft_table)
    static constexpr int tG = tFft + (kLane ? tail::kFftTable : 0);  // [d][nd] G[d][i]
    static constexpr int tGa = tG + n * nd;        // [d][k] Ga (direct-sum stages only)
    static constexpr int tRk = tGa + (kLane ? 0 : n * N);  // RN(1/k) for the Poisson inversion (floats)
    static constexpr int tEnd = tRk + kRecipTable / 2;
    static constexpr int oWarp = (oTab + tEnd * 8 + 15) / 16 * 16;  // per-warp scratch (float2)
    static constexpr int even(int x) { return (x + 1) & ~1; }
    // 32-lane path: the NGS image rows (wI) alias the LGS scratch (wQ); X and Q hold column
    // pairs, 16-byte aligned
    static constexpr int wX = 0, wQ = wX + n * n;
    // direct-sum path: Ta [N][no] over the consumed field X, then M [D2][n], P [D2][nd], B
    // [nd][nd] floats; an NGS's image rows [N][N + 1] floats over X, then B
    static constexpr int wTa = 0, wMg = even(n * n > N * no ? n * n : N * no), wP = wMg + D2 * n,
                         wB = kLane ? 0 : wP + D2 * nd;
    static constexpr int wI = kLane ? wQ : 0, wBn = even((N * (N + 1) + 1) / 2);
    static_assert(wQ % 2 == 0, "16-byte aligned column-pair scratch");
    static constexpr int lgs_end = kLane ? wQ + nd * n : even(wB + (nd * nd + 1) / 2);
    static constexpr int ngs_end = kLane ? wI + (N * (N + 1) + 1) / 2 : wBn + (nd * nd + 1) / 2;
    // an LGS subaperture's elongation table K~ ([2n-1][n] complex), staged by cp.async at the
    // top of a group and read by the elongation stage; it may overlap the NGS rows, which an LGS
    // subaperture never writes (a warp's copies land before its next NGS image)
    static constexpr int wKt = lgs_end;
    static constexpr int base_warp = even(wKt + D2 * n > ngs_end ? wKt + D2 * n : ngs_end);
    // per-slice variant: the summed spot rows use the NGS rows (wI; K~ is staged after them)
    static constexpr int warp = base_warp;
    // per warpgroup: 2 mbarriers (0), flag (16), next group (20), the first-stage mbarrier (24);
    // per-slice variant: the slice counts of its 4 warps (32)
    static constexpr int misc = kSlices ? 48 : 32;
    static constexpr int oMisc = oWarp + 4 * WG * warp * 8;
    static constexpr int bytes = oMisc + misc * WG + 16;
};

}  // namespace

template <int n, int N, int nd, bool kF16, bool kMmaU, int WG>
__global__ void __launch_bounds__(128 * WG, WG == 1 ? 3 : 2) k_sh_tc(const __grid_constant__ ShArgs a) {
    using Lay = TcLayout<n, N, nd, false, kMmaU, WG>;
    // warpgroups per CTA (the tile shape the tuner picks): their threads and tensor-memory columns
    constexpr int kWG = WG, kTcThreads = 128 * WG;
    constexpr uint32_t kTmemCols = 128 * WG;
    using E = TcElt<kF16>;
    constexpr bool kLane = Lay::kLane;
    constexpr int D2 = Lay::D2, nd2 = nd * nd;
    static_assert(6 * n <= 64 && n <= 16, "the split DFT operand must fit one 64-element K atom");
    static_assert(N <= 32 && N >= 2 * n - 1, "one DFT row per lane; the autocorrelation fits the grid");
    static_assert(n % 2 == 0 && Lay::wKt % 2 == 0 && Lay::warp % 2 == 0 && Lay::oWarp % 16 == 0,
                  "16-byte aligned K~ staging");
    static_assert(!kLane || nd2 % 32 == 0, "detector tile must split evenly over a warp");
    static_assert(N % nd == 0 && nd % 2 == 0, "whole binning blocks; even detector rows");
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sB1 = smem + Lay::oB1, *sB2h = smem + Lay::oB2h, *sB2l = smem + Lay::oB2l;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int wg = wib >> 2, wq = wib & 3;  // warpgroup, warp within it (= TMEM lane quarter)
    uint8_t *sA1 = smem + Lay::oA + 16384 * wg, *sA2 = sA1, *sB0 = sA1, *sA0 = smem + Lay::oA0;
    float2 *tab = reinterpret_cast<float2 *>(smem + Lay::oTab);
    float2 *Fk = tab + Lay::tFk, *fft = tab + Lay::tFft, *Gt = tab + Lay::tG;
    float2 *Gat = tab + Lay::tGa;
    float *rk = reinterpret_cast<float *>(tab + Lay::tRk);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + Lay::oMisc + 32 * wg);
    int *sflag = reinterpret_cast<int *>(smem + Lay::oMisc + 32 * wg + 16);
    int *snext = reinterpret_cast<int *>(smem + Lay::oMisc + 32 * wg + 20);  // next group (dynamic split)
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + Lay::oMisc + 32 * kWG);
    const uint32_t bar_id = 1 + wg;
    auto wg_sync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(128) : "memory"); };
    // constant operand tiles (pre-swizzled on the host) and CUDA-core tables
    {
        const uint4 *src1 = reinterpret_cast<const uint4 *>(a.tc_B1);
        const uint4 *src2 = reinterpret_cast<const uint4 *>(a.tc_B2h);
        const uint4 *src3 = reinterpret_cast<const uint4 *>(a.tc_B2l);
        for (int i = tid; i < 8192 / 16; i += kTcThreads) reinterpret_cast<uint4 *>(sB1)[i] = src1[i];
        for (int i = tid; i < 4096 / 16; i += kTcThreads) {
            reinterpret_cast<uint4 *>(sB2h)[i] = src2[i];
            reinterpret_cast<uint4 *>(sB2l)[i] = src3[i];
        }
        if constexpr (kMmaU) {
            // F's rows for the first MMA, and the field tiles cleared once: their K columns past
            // 6n meet zeros of F's tile, so they must never hold a NaN pattern
            const uint4 *src0 = reinterpret_cast<const uint4 *>(a.tc_A0);
            for (int i = tid; i < 16384 / 16; i += kTcThreads) reinterpret_cast<uint4 *>(sA0)[i] = src0[i];
            for (int i = tid; i < 16384 * kWG / 16; i += kTcThreads)
                reinterpret_cast<uint4 *>(smem + Lay::oA)[i] = make_uint4(0u, 0u, 0u, 0u);
        } else {
            for (int i = tid; i < n * N; i += kTcThreads) {
                const int p = i / N, k = i - p * N;
                Fk[p * N + k] = a.F[i];  // F[q*N + m] = F[m][q]: row index = p, column = k
            }
        }
        if constexpr (kLane) tail::fill_fft_table<n>(fft, tid, kTcThreads);
        else
            for (int i = tid; i < n * N; i += kTcThreads) Gat[i] = a.Ga[i];
        for (int i = tid; i < n * nd; i += kTcThreads) Gt[i] = a.G[i];
        fill_recip_table(rk, tid, kTcThreads);
    }
    if (wib == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (wq == 0 && lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
        if constexpr (kMmaU) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[3])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *sflag = 0;
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem_all = *tslot;
    wait_prior_grid();
    if (a.split_noise) allow_dependent_grid();  // the noise kernel may take SMs as CTAs retire
    const uint32_t tmem = tmem_all + 128u * wg;  // this warpgroup's columns
    const uint32_t t_row = tmem + ((uint32_t)(wq * 32) << 16);
    constexpr uint32_t idesc1 = tc_idesc(128, 64, E::fmt), idesc2 = tc_idesc(128, 32, E::fmt);
    constexpr uint32_t idesc0 = tc_idesc(128, 128, E::fmt);

    float4 *X4 = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(smem + Lay::oWarp) + wib * Lay::warp + Lay::wX);
    float2 *Qw = reinterpret_cast<float2 *>(smem + Lay::oWarp) + wib * Lay::warp + Lay::wQ;
    float2 *Kts = reinterpret_cast<float2 *>(smem + Lay::oWarp) + wib * Lay::warp + Lay::wKt;
    float *Iw = reinterpret_cast<float *>(reinterpret_cast<float2 *>(smem + Lay::oWarp) + wib * Lay::warp + Lay::wI);
    const int row = wq * 32 + lane;  // this thread's row of the MMA tiles and TMEM lane
    const int groups = (a.total + 3) / 4;
    const bool issuer = wq == 0 && lane == 0;
    uint32_t phase = 0;

    // Work split: each warpgroup starts with group blockIdx.x * kWG + wg; with a.work the
    // issuer then draws one ticket per iteration (issued at the top, published before the first
    // warpgroup barrier, read after it), so CTAs that start late take fewer groups.
    const int nwg = gridDim.x * kWG;
    int grp_next = 0;
    for (int grp = blockIdx.x * kWG + wg; grp < groups; grp = grp_next) {
        int ticket = 0;
        if (a.work && issuer) ticket = atomicAdd(a.work, 1);
        const int g = 4 * grp + wq;
        bool active = g < a.total;
        const WfsDesc &W = a.wfs[active ? find_wfs(a.wfs, a.n_wfs, g) : 0];
        const InstDyn &D = a.dyn[W.inst];
        const int v = active ? g - W.subap_begin : 0;
        active = active && guard(v >= 0 && v < W.n_valid, a.status);
        if (active && W.is_lgs) {
            // K~ of this subaperture: (2n-1) n complex = 16-byte chunks (n even)
            const float4 *src = reinterpret_cast<const float4 *>(W.ktil + (size_t)v * (D2 * n));
            for (int c = lane; c < D2 * n / 2; c += 32) {
                const uint32_t dst = smem_u32(reinterpret_cast<float4 *>(Kts) + c);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + c) : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }

        float2 U[n];
#pragma unroll
        for (int q = 0; q < n; ++q) U[q] = make_float2(0.0f, 0.0f);
        if constexpr (kMmaU) {
            // the field straight into this subaperture's rows of the first MMA's B tile:
            // pixel (p, q) -> row q: [X_hi | X_hi | X_lo] of (re p, -im p); row n + q: of (im p,
            // re p); U = F X lands in TMEM columns 32 wq + (q, n + q) of the warp's lanes
            if (active) {
                const float *opd = D.opd + W.opd_off + (size_t)v * (n * n);
                const uint32_t *mk = W.mask + (size_t)v * a.mask_words;
                const float ref = __ldg(opd);
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
                        float sn, cs;
                        field_phasor(W.k_phase * (o[m] - ref), sn, cs);
                        const int p = i / n, q = i - p * n;
                        float rh, rl, ih, il;
                        E::split(lit ? cs : 0.0f, rh, rl);
                        E::split(lit ? sn : 0.0f, ih, il);
                        const uint16_t brh = E::bits(rh), brl = E::bits(rl), bih = E::bits(ih), bil = E::bits(il);
                        const int r0 = wq * 32 + q, r1 = r0 + n;
                        uint8_t *b0 = sB0, *b1 = sB0;
                        auto st = [](uint8_t *base, int r, int k, uint16_t v16) {
                            *reinterpret_cast<uint16_t *>(base + sw128_off(r, k)) = v16;
                        };
                        // K = t 2n + c n + p; t = 0, 1 take the hi part, t = 2 the lo part
                        st(b0, r0, p, brh);
                        st(b0, r0, 2 * n + p, brh);
                        st(b0, r0, 4 * n + p, brl);
                        st(b0, r0, n + p, bih ^ 0x8000u);
                        st(b0, r0, 3 * n + p, bih ^ 0x8000u);
                        st(b0, r0, 5 * n + p, bil ^ 0x8000u);
                        st(b1, r1, p, bih);
                        st(b1, r1, 2 * n + p, bih);
                        st(b1, r1, 4 * n + p, bil);
                        st(b1, r1, n + p, brh);
                        st(b1, r1, 3 * n + p, brh);
                        st(b1, r1, 5 * n + p, brl);
                    }
                }
            }
            if (a.work && issuer) *snext = nwg + ticket;
            fence_async_smem();
            fence_before_sync();
            wg_sync();
            fence_after_sync();
            grp_next = a.work ? *snext : grp + nwg;
            if (*sflag) break;
            if (issuer) {
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    mma_f16(tmem, sw128_desc(smem_u32(sA0) + 32 * s), sw128_desc(smem_u32(sB0) + 32 * s), idesc0, s > 0);
                mma_commit(&mbar[3]);
            }
            if (!mbar_wait(&mbar[3], phase)) *sflag = 1;
            fence_after_sync();
            {
                uint32_t r[16], r2[16];
                GBWFS_TMEM_LD16(r, t_row + 32 * wq);
                GBWFS_TMEM_LD16(r2, t_row + 32 * wq + 16);
                tmem_wait_ld();
                auto col = [&](int j) { return __uint_as_float(j < 16 ? r[j] : r2[j - 16]); };
                if (active && (N == 32 || lane < N)) {
#pragma unroll
                    for (int q = 0; q < n; ++q) U[q] = make_float2(col(q), col(n + q));
                }
            }
        } else if (active) {
            // field and U = F X (CUDA cores)
            const float *opd = D.opd + W.opd_off + (size_t)v * (n * n);
            const uint32_t *mk = W.mask + (size_t)v * a.mask_words;
            const float ref = __ldg(opd);
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
                    field_phasor(W.k_phase * (o[m] - ref), s, c);
                    store_field<n>(X4, i, lit ? c : 0.0f, lit ? s : 0.0f);
                }
            }
            __syncwarp();
            field_rows<n, N>(Fk, X4, lane, U);  // DFT rows k >= N are zero
        }
        // FP16: U times 2^eu (exact), eu from the subaperture's largest component
        int eu = 0;
        if constexpr (kF16) {
            float mx = 0.0f;
#pragma unroll
            for (int q = 0; q < n; ++q) mx = fmaxf(mx, fmaxf(fabsf(U[q].x), fabsf(U[q].y)));
            eu = f16_scale_exp(warp_max(mx));
            const float su = pow2f(eu);
#pragma unroll
            for (int q = 0; q < n; ++q) U[q] = make_float2(U[q].x * su, U[q].y * su);
        }
        // A1 row: [U_hi | U_lo | U_hi | 0], each block (re q = 0..n-1, im q = 0..n-1); word w of
        // a block holds its elements (2w, 2w + 1)
        {
            uint32_t hw[n], lw[n];
#pragma unroll
            for (int i = 0; i < n / 2; ++i) {
                E::split2(U[2 * i].x, U[2 * i + 1].x, hw[i], lw[i]);
                E::split2(U[2 * i].y, U[2 * i + 1].y, hw[n / 2 + i], lw[n / 2 + i]);
            }
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) {
                uint32_t wds[4];
#pragma unroll
                for (int e2 = 0; e2 < 4; ++e2) {
                    const int w = ch * 4 + e2, t = w / n, j = w % n;
                    wds[e2] = w >= 3 * n ? 0u : (t == 1 ? lw[j] : hw[j]);
                }
                *reinterpret_cast<uint4 *>(sA1 + sw128_off(row, ch * 8)) = make_uint4(wds[0], wds[1], wds[2], wds[3]);
            }
        }
        if (!kMmaU && a.work && issuer) *snext = nwg + ticket;
        fence_async_smem();
        fence_before_sync();
        wg_sync();
        fence_after_sync();
        if (!kMmaU) grp_next = a.work ? *snext : grp + nwg;
        if (*sflag) break;  // a previous wait timed out (uniform: read after the barrier)
        if (issuer) {
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mma_f16(tmem, sw128_desc(smem_u32(sA1) + 32 * s), sw128_desc(smem_u32(sB1) + 32 * s), idesc1, s > 0);
            mma_commit(&mbar[0]);
        }
        if (!mbar_wait(&mbar[0], phase)) *sflag = 1;
        fence_after_sync();
        // Y row from TMEM -> I = |Y|^2 -> second operand row [I_hi | I_lo], 16 columns at a time.
        // FP16: Y carries 2^eu, so the intensity is |Y|^2 2^-2eu (exact); the operand takes
        // |Y|^2 2^ei, ei from a first pass over the warp's rows.
        int ei = 0;
        if constexpr (kF16) {
            float mx = 0.0f;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t r[16], r2[16];
                GBWFS_TMEM_LD16(r, t_row + 16 * hh);
                GBWFS_TMEM_LD16(r2, t_row + 32 + 16 * hh);
                tmem_wait_ld();
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    const float yr = __uint_as_float(r[m]), yi = __uint_as_float(r2[m]);
                    mx = fmaxf(mx, fmaf(yr, yr, yi * yi));
                }
            }
            ei = f16_scale_exp(warp_max(mx));
        }
        {
            float *dstI = (active && D.st_I && lane < N) ? D.st_I + W.int_off + (size_t)v * (N * N) + lane * N : nullptr;
            const float uy = kF16 ? pow2f(-eu) : 1.0f, si = kF16 ? pow2f(ei) : 1.0f;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t r[16], r2[16];
                GBWFS_TMEM_LD16(r, t_row + 16 * hh);
                GBWFS_TMEM_LD16(r2, t_row + 32 + 16 * hh);
                tmem_wait_ld();
                float I[16], Iop[16];  // the intensity, and the operand value
#pragma unroll
                for (int m = 0; m < 16; m += 2) {  // column pairs: each half as fmaf(yr, yr, yi * yi)
                    const float2 yr = make_float2(__uint_as_float(r[m]), __uint_as_float(r[m + 1]));
                    const float2 yi = make_float2(__uint_as_float(r2[m]), __uint_as_float(r2[m + 1]));
                    const float2 y2 = __ffma2_rn(yr, yr, __fmul2_rn(yi, yi));
                    const float2 iv = kF16 ? __fmul2_rn(__fmul2_rn(y2, make_float2(uy, uy)), make_float2(uy, uy)) : y2;
                    const float2 ov = kF16 ? __fmul2_rn(y2, make_float2(si, si)) : y2;
                    I[m] = iv.x;
                    I[m + 1] = iv.y;
                    Iop[m] = ov.x;
                    Iop[m + 1] = ov.y;
                }
                if (dstI) {
#pragma unroll
                    for (int m = 0; m < 16; ++m)
                        if (16 * hh + m < N) dstI[16 * hh + m] = I[m];
                }
                if (active && !W.is_lgs && lane < N) {
#pragma unroll
                    for (int m = 0; m < 16; ++m)
                        if (16 * hh + m < N) Iw[lane * (N + 1) + 16 * hh + m] = I[m];
                }
#pragma unroll
                for (int c2 = 0; c2 < 2; ++c2) {
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        E::split2(Iop[c2 * 8 + 2 * e2], Iop[c2 * 8 + 2 * e2 + 1], hw[e2], lw[e2]);
                    }
                    *reinterpret_cast<uint4 *>(sA2 + sw128_off(row, (2 * hh + c2) * 8)) =
                        make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4 *>(sA2 + sw128_off(row, (4 + 2 * hh + c2) * 8)) =
                        make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
            }
        }
        fence_async_smem();
        fence_before_sync();
        wg_sync();
        fence_after_sync();
        if (*sflag) break;
        if (issuer) {
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mma_f16(tmem + 64, sw128_desc(smem_u32(sA2) + 32 * s), sw128_desc(smem_u32(sB2h) + 32 * s), idesc2, s > 0);
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mma_f16(tmem + 64, sw128_desc(smem_u32(sA2) + 32 * s), sw128_desc(smem_u32(sB2l) + 32 * s), idesc2, 1);
            mma_commit(&mbar[1]);
        }
        if (!mbar_wait(&mbar[1], phase)) *sflag = 1;
        fence_after_sync();
        float2 T[n];  // row k = lane of the first inverse stage (LGS)
        {
            uint32_t r[32];
            GBWFS_TMEM_LD32(r, t_row + 64);
            tmem_wait_ld();
#pragma unroll
            for (int d = 0; d < n; ++d) T[d] = make_float2(__uint_as_float(r[d]), __uint_as_float(r[16 + d]));
            if constexpr (kF16) {
                // T carries 2^(ei + 2 eu): three exact power-of-two factors
                const float ti = pow2f(-ei), tu = pow2f(-eu);
#pragma unroll
                for (int d = 0; d < n; ++d) T[d] = make_float2(T[d].x * ti * tu * tu, T[d].y * ti * tu * tu);
            }
        }
        phase ^= 1u;
        fence_before_sync();  // TMEM reads of this group precede the next group's MMAs
        if (!active) continue;
        __syncwarp();

        // remaining stages on the CUDA cores (per warp)
        if constexpr (kLane) {
            float Bv[nd / 2];
            if (W.is_lgs) {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
                __syncwarp();
                tail::lgs_binned<n, nd>(T, reinterpret_cast<float4 *>(Qw), fft, Gt,
                                        Kts, lane, Bv);
            } else
                tail::ngs_binned<nd>(Iw, lane, Bv);
            tail::finish<nd>(Bv, W, D, a.inst[W.inst].seed, v, lane, rk, a.split_noise != 0);
        } else {
            float2 *wbase = reinterpret_cast<float2 *>(smem + Lay::oWarp) + wib * Lay::warp;
            float *Bw;
            if (W.is_lgs) {
                float2 *Ta = wbase + Lay::wTa;
                if (lane < N) {
#pragma unroll
                    for (int d = 0; d < n; ++d) Ta[lane * Lay::no + d] = T[d];
                }
                asm volatile("cp.async.wait_group 0;" ::: "memory");
                __syncwarp();
                Bw = reinterpret_cast<float *>(wbase + Lay::wB);
                tail::lgs_direct<n, N, nd>(Ta, wbase + Lay::wMg, wbase + Lay::wP, Bw, Kts, Gat, Gt, lane);
            } else {
                __syncwarp();
                Bw = reinterpret_cast<float *>(wbase + Lay::wBn);
                tail::ngs_direct<N, nd>(Iw, Bw, lane);
            }
            tail::finish_direct<nd>(Bw, W, D, a.inst[W.inst].seed, v, lane);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy outlives the CTA
    fence_before_sync();
    __syncthreads();
    if (*sflag && issuer && a.status) atomicCAS(a.status, 0, 5 /* WFS_ETIMEOUT */);
    if (a.work && tid == 0) {
        // every ticket of this CTA was drawn before the barrier above; the last CTA to get here
        // leaves the counters at zero for the next launch
        __threadfence();
        if (atomicAdd(a.work + 1, 1) == (int)gridDim.x - 1) {
            a.work[0] = 0;
            a.work[1] = 0;
        }
    }
    fence_after_sync();
    if (wib == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_all), "r"(kTmemCols));
}

// The per-slice variant (see the file comment).
template <int n, int nd, bool kF16>
__global__ void __launch_bounds__(kTcThreads, 2) k_sh_tc_sl(const __grid_constant__ ShArgs a) {
    constexpr bool kSlices = true;
    using Lay = TcLayout<n, 32, nd, kSlices, false, kWG>;
    using E = TcElt<kF16>;
    constexpr int N = 32, D2 = Lay::D2, nd2 = nd * nd;
    static_assert(6 * n <= 64 && n <= 16, "the split DFT operand must fit one 64-element K atom");
    static_assert(n % 2 == 0 && Lay::wKt % 2 == 0 && Lay::warp % 2 == 0 && Lay::oWarp % 16 == 0,
                  "16-byte aligned K~ staging");
    static_assert(nd <= 32 && nd2 % 32 == 0, "detector tile must split evenly over a warp");
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sB1 = smem + Lay::oB1, *sB2h = smem + Lay::oB2h, *sB2l = smem + Lay::oB2l;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int wg = wib >> 2, wq = wib & 3;  // warpgroup, warp within it (= TMEM lane quarter)
    uint8_t *sA1 = smem + Lay::oA + 16384 * wg, *sA2 = sA1;
    float2 *tab = reinterpret_cast<float2 *>(smem + Lay::oTab);
    float2 *Fk = tab + Lay::tFk, *fft = tab + Lay::tFft, *Gt = tab + Lay::tG;
    float *rk = reinterpret_cast<float *>(tab + Lay::tRk);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + Lay::oMisc + Lay::misc * wg);
    int *sflag = reinterpret_cast<int *>(smem + Lay::oMisc + Lay::misc * wg + 16);
    int *snext = reinterpret_cast<int *>(smem + Lay::oMisc + Lay::misc * wg + 20);  // next group (dynamic split)
    int *snsl = reinterpret_cast<int *>(smem + Lay::oMisc + Lay::misc * wg + 32);   // slices per warp (kSlices)
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + Lay::oMisc + Lay::misc * kWG);
    const uint32_t bar_id = 1 + wg;
    auto wg_sync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(128) : "memory"); };
    // constant operand tiles (pre-swizzled on the host) and CUDA-core tables
    {
        const uint4 *src1 = reinterpret_cast<const uint4 *>(a.tc_B1);
        const uint4 *src2 = reinterpret_cast<const uint4 *>(a.tc_B2h);
        const uint4 *src3 = reinterpret_cast<const uint4 *>(a.tc_B2l);
        for (int i = tid; i < 8192 / 16; i += kTcThreads) reinterpret_cast<uint4 *>(sB1)[i] = src1[i];
        for (int i = tid; i < 4096 / 16; i += kTcThreads) {
            reinterpret_cast<uint4 *>(sB2h)[i] = src2[i];
            reinterpret_cast<uint4 *>(sB2l)[i] = src3[i];
        }
        for (int i = tid; i < n * N; i += kTcThreads) {
            const int p = i / N, k = i - p * N;
            Fk[p * N + k] = a.F[i];  // F[q*N + m] = F[m][q]: row index = p, column = k
        }
        tail::fill_fft_table<n>(fft, tid, kTcThreads);
        for (int i = tid; i < n * nd; i += kTcThreads) Gt[i] = a.G[i];
        fill_recip_table(rk, tid, kTcThreads);
    }
    if (wib == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (wq == 0 && lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *sflag = 0;
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem_all = *tslot;
    wait_prior_grid();
    if (a.split_noise) allow_dependent_grid();  // the noise kernel may take SMs as CTAs retire
    const uint32_t tmem = tmem_all + 128u * wg;  // this warpgroup's columns
    const uint32_t t_row = tmem + ((uint32_t)(wq * 32) << 16);
    constexpr uint32_t idesc1 = tc_idesc(128, 64, E::fmt), idesc2 = tc_idesc(128, 32, E::fmt);

    float4 *X4 = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(smem + Lay::oWarp) + wib * Lay::warp + Lay::wX);
    float2 *Qw = reinterpret_cast<float2 *>(smem + Lay::oWarp) + wib * Lay::warp + Lay::wQ;
    float2 *Kts = reinterpret_cast<float2 *>(smem + Lay::oWarp) + wib * Lay::warp + Lay::wKt;
    float *Iw = reinterpret_cast<float *>(reinterpret_cast<float2 *>(smem + Lay::oWarp) + wib * Lay::warp + Lay::wI);
    const int row = wq * 32 + lane;  // this thread's row of the MMA tiles and TMEM lane
    const int groups = (a.total + 3) / 4;
    const bool issuer = wq == 0 && lane == 0;
    uint32_t phase = 0, phase0 = 0;  // mbarrier parities: [1] once per group, [0] once per slice

    // Work split: each warpgroup starts with group blockIdx.x * kWG + wg; with a.work the
    // issuer then draws one ticket per iteration (issued at the top, published before the first
    // warpgroup barrier, read after it), so CTAs that start late take fewer groups.
    const int nwg = gridDim.x * kWG;
    int grp_next = 0;
    for (int grp = blockIdx.x * kWG + wg; grp < groups; grp = grp_next) {
        int ticket = 0;
        if (a.work && issuer) ticket = atomicAdd(a.work, 1);
        const int g = 4 * grp + wq;
        bool active = g < a.total;
        const WfsDesc &W = a.wfs[active ? find_wfs(a.wfs, a.n_wfs, g) : 0];
        const InstDyn &D = a.dyn[W.inst];
        const int v = active ? g - W.subap_begin : 0;
        active = active && guard(v >= 0 && v < W.n_valid, a.status);
        // K~ of this subaperture: (2n-1) n complex = 16-byte chunks (n even); the per-slice
        // variant stages it after its slices, whose summed rows share the space
        auto stage_ktil = [&]() {
            const float4 *src = reinterpret_cast<const float4 *>(W.ktil + (size_t)v * (D2 * n));
            for (int c = lane; c < D2 * n / 2; c += 32) {
                const uint32_t dst = smem_u32(reinterpret_cast<float4 *>(Kts) + c);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + c) : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        if (!kSlices && active && W.is_lgs) stage_ktil();

        // slices: one for the elongation-kernel model; the warpgroup runs the largest count of
        // its four subapertures (a subaperture with fewer adds nothing in the extra ones)
        const SliceDesc *SD = (kSlices && active) ? W.slices : nullptr;
        const int my_n = SD ? SD->n : 1;
        int n_sl = 1;
        if (kSlices) {
            if (lane == 0) snsl[wq] = my_n;
            wg_sync();
            n_sl = max(max(snsl[0], snsl[1]), max(snsl[2], snsl[3]));
        }
        bool quit = false;
        for (int sl = 0; sl < n_sl; ++sl) {
            // field and U = F X (CUDA cores)
            float2 U[n];
#pragma unroll
            for (int q = 0; q < n; ++q) U[q] = make_float2(0.0f, 0.0f);
            if (active && sl < my_n) {
                // the slice's OPD (projected through its cone) plus its geometric term
                // k_s ((x - r_b).(r_b - r_L) + 1/2 |x - r_b|^2) about the subaperture centre r_b
                const float *opd = D.opd + W.opd_off + (size_t)sl * a.slice_opd_stride + (size_t)v * (n * n);
                float ebx = 0.0f, eby = 0.0f, dxp = 0.0f, ks = 0.0f;
                if (SD) {
                    const InstDesc &I = a.inst[W.inst];
                    const int id = __ldg(W.subap + v), sy = id / W.n_sub, sx = id - sy * W.n_sub;
                    const float half = 0.5f * (float)(W.n_sub * n - 1), c0 = 0.5f * (float)(n - 1);
                    dxp = (float)(W.pupil_dx_over_ds * I.ds);
                    ebx = ((float)(sx * n) + c0 - half) * dxp - (float)W.launch_x;
                    eby = ((float)(sy * n) + c0 - half) * dxp - (float)W.launch_y;
                    ks = SD->k[sl];
                }
                auto geo = [&](int i) -> float {
                    const int pp = i / n, qq = i - pp * n;
                    const float ux = ((float)qq - 0.5f * (float)(n - 1)) * dxp;
                    const float uy = ((float)pp - 0.5f * (float)(n - 1)) * dxp;
                    return ks * fmaf(ux, ebx, fmaf(uy, eby, 0.5f * fmaf(ux, ux, uy * uy)));
                };
                const uint32_t *mk = W.mask + (size_t)v * a.mask_words;
                const float ref = __ldg(opd) + geo(0);
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
                        field_phasor(W.k_phase * ((o[m] + geo(i)) - ref), s, c);
                        store_field<n>(X4, i, lit ? c : 0.0f, lit ? s : 0.0f);
                    }
                }
                __syncwarp();
                field_rows<n, N>(Fk, X4, lane, U);
            }
            // FP16: U times 2^eu (exact), eu from the slice's largest component
            int eu = 0;
            if constexpr (kF16) {
                float mx = 0.0f;
#pragma unroll
                for (int q = 0; q < n; ++q) mx = fmaxf(mx, fmaxf(fabsf(U[q].x), fabsf(U[q].y)));
                eu = f16_scale_exp(warp_max(mx));
                const float su = pow2f(eu);
#pragma unroll
                for (int q = 0; q < n; ++q) U[q] = make_float2(U[q].x * su, U[q].y * su);
            }
            // A1 row: [U_hi | U_lo | U_hi | 0], each block (re q = 0..n-1, im q = 0..n-1); word w of
            // a block holds its elements (2w, 2w + 1)
            {
                uint32_t hw[n], lw[n];
#pragma unroll
                for (int i = 0; i < n / 2; ++i) {
                    E::split2(U[2 * i].x, U[2 * i + 1].x, hw[i], lw[i]);
                    E::split2(U[2 * i].y, U[2 * i + 1].y, hw[n / 2 + i], lw[n / 2 + i]);
                }
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) {
                    uint32_t wds[4];
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        const int w = ch * 4 + e2, t = w / n, j = w % n;
                        wds[e2] = w >= 3 * n ? 0u : (t == 1 ? lw[j] : hw[j]);
                    }
                    *reinterpret_cast<uint4 *>(sA1 + sw128_off(row, ch * 8)) = make_uint4(wds[0], wds[1], wds[2], wds[3]);
                }
            }
            if (sl == 0 && a.work && issuer) *snext = nwg + ticket;
            fence_async_smem();
            fence_before_sync();
            wg_sync();
            fence_after_sync();
            if (sl == 0) grp_next = a.work ? *snext : grp + nwg;
            if (*sflag) {  // a previous wait timed out (uniform: read after the barrier)
                quit = true;
                break;
            }
            if (issuer) {
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    mma_f16(tmem, sw128_desc(smem_u32(sA1) + 32 * s), sw128_desc(smem_u32(sB1) + 32 * s), idesc1, s > 0);
                mma_commit(&mbar[0]);
            }
            // the elongation-kernel model completes mbar[0] once per group like mbar[1]
            if (!mbar_wait(&mbar[0], kSlices ? phase0 : phase)) *sflag = 1;
            if (kSlices) phase0 ^= 1u;
            fence_after_sync();
            // Y row from TMEM -> I = |Y|^2; the elongation-kernel model writes the second operand
            // row [I_hi | I_lo] at once, the per-slice model adds w_s I into the warp's rows
            {
                float *dstI = (active && D.st_I && (!kSlices || sl == n_sl - 1))
                                  ? D.st_I + W.int_off + (size_t)v * (N * N) + lane * N
                                  : nullptr;
                const float wsl = (SD && sl < my_n) ? SD->w[sl] : (kSlices && sl > 0 ? 0.0f : 1.0f);
                const float uy = kF16 ? pow2f(-eu) : 1.0f;  // FP16: Y carries 2^eu
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    uint32_t r[16], r2[16];
                    GBWFS_TMEM_LD16(r, t_row + 16 * hh);
                    GBWFS_TMEM_LD16(r2, t_row + 32 + 16 * hh);
                    tmem_wait_ld();
                    float I[16];
#pragma unroll
                    for (int m = 0; m < 16; m += 2) {  // column pairs: each half as fmaf(yr, yr, yi * yi)
                        const float2 yr = make_float2(__uint_as_float(r[m]), __uint_as_float(r[m + 1]));
                        const float2 yi = make_float2(__uint_as_float(r2[m]), __uint_as_float(r2[m + 1]));
                        const float2 y2 = __ffma2_rn(yr, yr, __fmul2_rn(yi, yi));
                        const float2 iv = kF16 ? __fmul2_rn(__fmul2_rn(y2, make_float2(uy, uy)), make_float2(uy, uy)) : y2;
                        I[m] = iv.x;
                        I[m + 1] = iv.y;
                    }
                    if (kSlices) {
                        float *ir = Iw + lane * (N + 1) + 16 * hh;
#pragma unroll
                        for (int m = 0; m < 16; ++m) {
                            const float tot = sl == 0 ? wsl * I[m] : fmaf(wsl, I[m], ir[m]);
                            ir[m] = tot;
                            if (dstI) dstI[16 * hh + m] = tot;
                        }
                        continue;
                    }
                    if (dstI) {
#pragma unroll
                        for (int m = 0; m < 16; ++m) dstI[16 * hh + m] = I[m];
                    }
                    if (active && !W.is_lgs) {
#pragma unroll
                        for (int m = 0; m < 16; ++m) Iw[lane * (N + 1) + 16 * hh + m] = I[m];
                    }
#pragma unroll
                    for (int c2 = 0; c2 < 2; ++c2) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int e2 = 0; e2 < 4; ++e2) {
                            E::split2(I[c2 * 8 + 2 * e2], I[c2 * 8 + 2 * e2 + 1], hw[e2], lw[e2]);
                        }
                        *reinterpret_cast<uint4 *>(sA2 + sw128_off(row, (2 * hh + c2) * 8)) =
                            make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4 *>(sA2 + sw128_off(row, (4 + 2 * hh + c2) * 8)) =
                            make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
            }
            fence_before_sync();  // these TMEM reads precede the next slice's MMA
            __syncwarp();         // the warp's rows are complete before the next slice adds to them
        }
        if (quit) break;
        int ei = 0;  // FP16: the second operand carries 2^ei
        if (kSlices) {
            // the summed rows -> second operand row [I_hi | I_lo] (after the last slice's MMA), then
            // the K~ staging, which reuses their space
            if constexpr (kF16) {
                float mx = 0.0f;
#pragma unroll
                for (int c = 0; c < N; ++c) mx = fmaxf(mx, Iw[lane * (N + 1) + c]);
                ei = f16_scale_exp(warp_max(mx));
            }
            const float si = kF16 ? pow2f(ei) : 1.0f;
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int e2 = 0; e2 < 4; ++e2) {
                    const float i0 = Iw[lane * (N + 1) + c4 * 8 + 2 * e2], i1 = Iw[lane * (N + 1) + c4 * 8 + 2 * e2 + 1];
                    E::split2(kF16 ? i0 * si : i0, kF16 ? i1 * si : i1, hw[e2], lw[e2]);
                }
                *reinterpret_cast<uint4 *>(sA2 + sw128_off(row, c4 * 8)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4 *>(sA2 + sw128_off(row, (4 + c4) * 8)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            __syncwarp();
            if (active && W.is_lgs) stage_ktil();
        }
        fence_async_smem();
        fence_before_sync();
        wg_sync();
        fence_after_sync();
        if (*sflag) break;
        if (issuer) {
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mma_f16(tmem + 64, sw128_desc(smem_u32(sA2) + 32 * s), sw128_desc(smem_u32(sB2h) + 32 * s), idesc2, s > 0);
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mma_f16(tmem + 64, sw128_desc(smem_u32(sA2) + 32 * s), sw128_desc(smem_u32(sB2l) + 32 * s), idesc2, 1);
            mma_commit(&mbar[1]);
        }
        if (!mbar_wait(&mbar[1], phase)) *sflag = 1;
        fence_after_sync();
        float2 T[n];  // row k = lane of the first inverse stage (LGS)
        {
            uint32_t r[32];
            GBWFS_TMEM_LD32(r, t_row + 64);
            tmem_wait_ld();
#pragma unroll
            for (int d = 0; d < n; ++d) T[d] = make_float2(__uint_as_float(r[d]), __uint_as_float(r[16 + d]));
            if constexpr (kF16) {
                const float ti = pow2f(-ei);
#pragma unroll
                for (int d = 0; d < n; ++d) T[d] = make_float2(T[d].x * ti, T[d].y * ti);
            }
        }
        phase ^= 1u;
        fence_before_sync();  // TMEM reads of this group precede the next group's MMAs
        if (!active) continue;
        __syncwarp();

        // remaining stages on the CUDA cores (per warp)
        float Bv[nd / 2];
        if (W.is_lgs) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncwarp();
            tail::lgs_binned<n, nd>(T, reinterpret_cast<float4 *>(Qw), fft, Gt, Kts,
                                    lane, Bv);
        } else
            tail::ngs_binned<nd>(Iw, lane, Bv);
        tail::finish<nd>(Bv, W, D, a.inst[W.inst].seed, v, lane, rk, a.split_noise != 0);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy outlives the CTA
    fence_before_sync();
    __syncthreads();
    if (*sflag && issuer && a.status) atomicCAS(a.status, 0, 5 /* WFS_ETIMEOUT */);
    if (a.work && tid == 0) {
        // every ticket of this CTA was drawn before the barrier above; the last CTA to get here
        // leaves the counters at zero for the next launch
        __threadfence();
        if (atomicAdd(a.work + 1, 1) == (int)gridDim.x - 1) {
            a.work[0] = 0;
            a.work[1] = 0;
        }
    }
    fence_after_sync();
    if (wib == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_all), "r"(kTmemCols));
}

// ---------------------------------------------------------------- wait check
// One CTA waits on an mbarrier that nothing will ever arrive on, with a short bound, then
// reports WFS_ETIMEOUT in *status: the same bounded wait the spot kernel uses, exercised
// without faulting or hanging the GPU.
__global__ void k_wait_check(int *status, int limit) {
    __shared__ __align__(8) uint64_t mb;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mb)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(&mb)), "r"(0)
            : "memory");
    __syncthreads();
    if (threadIdx.x == 0) *status = done ? 0 : 5 /* WFS_ETIMEOUT */;
}

cudaError_t launch_wait_check(int *status, int limit, cudaStream_t s) {
    k_wait_check<<<1, 32, 0, s>>>(status, limit);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- host side

namespace {

uint16_t bf16_bits(float f) {  // round to nearest even (finite inputs)
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_float(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

template <int n, int N, int nd, bool kSlices, bool kF16, bool kMmaU, int WG = kWG>
cudaError_t shape_tc_k(const ShArgs &a, LaunchShape *out) {
    using Lay = TcLayout<n, N, nd, kSlices, kSlices ? false : kMmaU, WG>;
    const void *f;
    if constexpr (kSlices) f = (const void *)k_sh_tc_sl<n, nd, kF16>;
    else f = (const void *)k_sh_tc<n, N, nd, kF16, kMmaU, WG>;
    const int smem = Lay::bytes;  // no static shared memory: the dynamic base is 1024-aligned
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int groups = (a.total + 3) / 4;
    const int cta_groups = (groups + WG - 1) / WG;
    // resident CTAs per SM: two of two warpgroups or three of one (shared memory); their tensor
    // memory (4 x 128 or 3 x 128 columns) always fits
    const int per_sm = WG == 1 ? 3 : 2;
    const int cap = a.grid_cap > 0 && a.grid_cap < 152 * per_sm ? a.grid_cap : 152 * per_sm;
    int blocks = cta_groups < cap ? cta_groups : cap;
    if (blocks < 1) blocks = 1;
    out->func = f;
    out->grid = dim3(blocks);
    out->block = dim3(128 * WG);
    out->smem = smem;
    return cudaSuccess;
}

// ShArgs::slice_opd_stride selects the per-slice variant (32-point geometries only);
// ShArgs::mma_u the variant with U = F X as an MMA.
template <int n, int N, int nd>
cudaError_t shape_tc(const ShArgs &a, LaunchShape *out, bool f16) {
    if constexpr (N == 32 && nd == 16) {
        if (a.slice_opd_stride > 0)
            return f16 ? shape_tc_k<n, N, nd, true, true, false>(a, out) : shape_tc_k<n, N, nd, true, false, false>(a, out);
    } else {
        if (a.slice_opd_stride > 0) return cudaErrorInvalidValue;
    }
    if (a.mma_u)
        return f16 ? shape_tc_k<n, N, nd, false, true, true>(a, out) : shape_tc_k<n, N, nd, false, false, true>(a, out);
    // ShArgs::cta_warps = 4: one warpgroup per CTA (else two)
    if (a.cta_warps == 4)
        return f16 ? shape_tc_k<n, N, nd, false, true, false, 1>(a, out) : shape_tc_k<n, N, nd, false, false, false, 1>(a, out);
    return f16 ? shape_tc_k<n, N, nd, false, true, false>(a, out) : shape_tc_k<n, N, nd, false, false, false>(a, out);
}

}  // namespace

// The geometries with a tensor-core spot kernel: 32-point DFTs with a 16 x 16 detector (n = 8
// or 10), and the other DFT sizes of the configured sensors -- 16-point (n = 8, 8 x 8
// detector) and 24-point (n = 6, 12 x 12 detector).
bool sh_tc_supported(int n, int N, int nd) {
    return (N == 32 && nd == 16 && (n == 10 || n == 8)) || (N == 16 && n == 8 && nd == 8) ||
           (N == 24 && n == 6 && nd == 12);
}

// The per-slice LGS variant exists for the 32-point tensor-core geometries.
bool sh_tc_slices_supported(int n, int N, int nd) { return N == 32 && nd == 16 && (n == 10 || n == 8); }

// Operand tiles of the two constant matrices, already in the swizzled shared layout, in BF16 or
// FP16 (hi = the element's rounding of the value, lo = that of the remainder).
void build_tc_tiles(int n, int N, const double *F_re64, const double *F_im64, const double *Ga_re64,
                    const double *Ga_im64, bool f16, std::vector<uint8_t> &B1, std::vector<uint8_t> &B2h,
                    std::vector<uint8_t> &B2l, std::vector<uint8_t> &A0) {
    A0.assign(16384, 0);
    B1.assign(8192, 0);
    B2h.assign(4096, 0);
    B2l.assign(4096, 0);
    auto bits = [f16](float v) -> uint16_t {
        if (!f16) return bf16_bits(v);
        const __half h = __float2half_rn(v);
        uint16_t u;
        memcpy(&u, &h, 2);
        return u;
    };
    auto rounded = [f16](float v) -> float {
        return f16 ? __half2float(__float2half_rn(v)) : bf16_float(bf16_bits(v));
    };
    auto put = [&](std::vector<uint8_t> &t, int r, int k, float v) {
        const uint16_t h = bits(v);
        memcpy(t.data() + sw128_off(r, k), &h, 2);
    };
    // B1[row = c' * 32 + m][K = t * 2n + c * n + q]
    for (int cp = 0; cp < 2; ++cp)
        for (int m = 0; m < N; ++m)
            for (int t = 0; t < 3; ++t)
                for (int c = 0; c < 2; ++c)
                    for (int q = 0; q < n; ++q) {
                        const double fr = F_re64[q * N + m], fi = F_im64[q * N + m];
                        double val;
                        if (c == 0 && cp == 0) val = fr;
                        else if (c == 1 && cp == 0) val = -fi;
                        else if (c == 0 && cp == 1) val = fi;
                        else val = fr;
                        const float hi = rounded((float)val);
                        const float lo = (float)(val - (double)hi);
                        put(B1, cp * 32 + m, t * 2 * n + c * n + q, t == 2 ? lo : hi);
                    }
    // A0[row = b * 32 + k][K = t * 2n + c * n + p]: F[k][p] (c = 0 real, 1 imaginary) as
    // [F_hi | F_lo | F_hi], the same for the four subapertures b of a group; rows k >= N zero
    for (int b = 0; b < 4; ++b)
        for (int k = 0; k < N; ++k)
            for (int t = 0; t < 3; ++t)
                for (int c = 0; c < 2; ++c)
                    for (int p = 0; p < n; ++p) {
                        const double val = c == 0 ? F_re64[p * N + k] : F_im64[p * N + k];
                        const float hi = rounded((float)val);
                        const float lo = (float)(val - (double)hi);
                        put(A0, b * 32 + k, t * 2 * n + c * n + p, t == 1 ? lo : hi);
                    }
    // B2h[row = c'' * 16 + dx][K = h * 32 + m] = Ga_hi, B2l = [Ga_lo; 0]
    for (int cpp = 0; cpp < 2; ++cpp)
        for (int dx = 0; dx < n; ++dx)
            for (int m = 0; m < N; ++m) {
                const double val = cpp == 0 ? Ga_re64[dx * N + m] : Ga_im64[dx * N + m];
                const float hi = rounded((float)val);
                const float lo = (float)(val - (double)hi);
                put(B2h, cpp * 16 + dx, m, hi);
                put(B2h, cpp * 16 + dx, 32 + m, hi);
                put(B2l, cpp * 16 + dx, m, lo);
            }
}

cudaError_t tc_launch_shape(const ShArgs &a, LaunchShape *out, bool f16) {
    if (a.N == 32 && a.n == 10 && a.nd == 16) return shape_tc<10, 32, 16>(a, out, f16);
    if (a.N == 32 && a.n == 8 && a.nd == 16) return shape_tc<8, 32, 16>(a, out, f16);
    if (a.N == 16 && a.n == 8 && a.nd == 8) return shape_tc<8, 16, 8>(a, out, f16);
    if (a.N == 24 && a.n == 6 && a.nd == 12) return shape_tc<6, 24, 12>(a, out, f16);
    return cudaErrorInvalidValue;
}

}  // namespace gbwfs
