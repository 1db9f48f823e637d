// k_sh_tc64.cu -- the spot kernel of the 64-point DFT geometry with a 32 x 32 detector (the
// 2x2 NGS sensors: 32 x 32 pupil pixels per subaperture, zero-padded to 64) with both DFT
// contractions on the tensor cores (Sec. 4: spot by FFT, the image composed on the detector,
// noise added, centroid taken; Sec. 2: "FFT (actually DFT)").
//
//   U = F X     rows (subaperture b, DFT row k), M = 2 x 64 = 128: A = F's rows (the same for
//               both subapertures) as [F_hi | F_lo | F_hi], B = the two fields as
//               [X_hi | X_hi | X_lo] (rows: re and im output columns of each subaperture),
//               N = 2 x 64, K = 3 x 64 (three 64-element atoms)
//   Y = U F^T   rows (b, k): A = [U_hi | U_lo | U_hi], B = [F_hi; F_hi; F_lo] (rows: re and im
//               output columns), N = 128, K = 3 x 64
//
// with FP32 accumulation in tensor memory (BF16 hi/lo, or FP16 hi/lo with the subaperture's U
// scaled by a power of two into FP16's normal range).  Then I = |Y|^2, 2 x 2 binning, the
// photometry, the noise pixel by pixel and the centre of gravity on the CUDA cores, in the order
// of the FP32 generic kernel.  One warpgroup per CTA, two subapertures per step; thread t owns
// DFT row t mod 64 of subaperture t / 64, which is also TMEM lane t.  Every mbarrier wait is
// bounded; a timeout is recorded in the status word and the CTA frees its tensor memory.
//
// With ShArgs::project the kernel projects its subapertures' OPD from the screens itself (the
// arithmetic of the projection kernel: FP64 layer offsets, bilinear samples summed over the
// layers in order, the uplink tilt; the OPD also goes to dyn.opd): a few NGS subapertures on a
// side stream then take their SMs with one launch at the start of a frame instead of queueing a
// projection behind the large one.
#include <string.h>

#include <vector>

#include "internal.h"
#include "noise.cuh"
#include "proj_math.cuh"
#include "tcgen05.cuh"

namespace gbwfs {

namespace {

using namespace tc;

constexpr int kT64Threads = 128;
constexpr int kT64N = 64, kT64n = 32, kT64nd = 32;
constexpr int kAtom = 16384;  // one 128-row x 64-element K atom (128-byte rows, swizzled)

struct T64Layout {
    static constexpr int oA0 = 0;              // 3 atoms: F's rows for U = F X
    static constexpr int oB1 = oA0 + 3 * kAtom;  // 3 atoms: [F_hi; F_hi; F_lo] for Y = U F^T
    static constexpr int oT = oB1 + 3 * kAtom;   // 3 atoms: the fields, then [U_hi | U_lo | U_hi]
    static constexpr int oI = oT + 3 * kAtom;    // the two spots' rows [64][65] floats
    static constexpr int oRed = oI + 2 * kT64N * (kT64N + 1) * 4;  // per-warp partial sums (4 x 4 floats)
    static constexpr int oMisc = oRed + 4 * 4 * 4;                  // 2 mbarriers, flag, TMEM slot
    static constexpr int oLo = oMisc + 32;                          // layer offsets of the two subapertures
    static constexpr int bytes = oLo + 2 * kMaxProjLayers * (int)sizeof(LayerOffs) + 16;
};

}  // namespace

template <bool kF16>
__global__ void __launch_bounds__(kT64Threads, 1) k_sh_tc64(const __grid_constant__ ShArgs a) {
    using Lay = T64Layout;
    using E = TcElt<kF16>;
    constexpr int N = kT64N, n = kT64n, nd = kT64nd, nn = n * n, nd2 = nd * nd;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA0 = smem + Lay::oA0, *sB1 = smem + Lay::oB1, *sT = smem + Lay::oT;
    float *Iw = reinterpret_cast<float *>(smem + Lay::oI);
    float *red = reinterpret_cast<float *>(smem + Lay::oRed);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + Lay::oMisc);
    int *sflag = reinterpret_cast<int *>(smem + Lay::oMisc + 16);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + Lay::oMisc + 20);
    float *sref = reinterpret_cast<float *>(smem + Lay::oMisc + 24);  // a self-projected subaperture's piston (x2)
    LayerOffs *slo = reinterpret_cast<LayerOffs *>(smem + Lay::oLo);
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int b = tid >> 6, k = tid & 63;  // subaperture of the step, DFT row (= TMEM lane tid)
    {
        const uint4 *s0 = reinterpret_cast<const uint4 *>(a.tc_A0);
        const uint4 *s1 = reinterpret_cast<const uint4 *>(a.tc_B1);
        for (int i = tid; i < 3 * kAtom / 16; i += kT64Threads) {
            reinterpret_cast<uint4 *>(sA0)[i] = s0[i];
            reinterpret_cast<uint4 *>(sB1)[i] = s1[i];
            // the operand tile starts cleared: no NaN pattern may ever meet a zero of F's tile
            reinterpret_cast<uint4 *>(sT)[i] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    if (wib == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *sflag = 0;
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t t_row = tmem + ((uint32_t)(wib * 32) << 16);
    wait_prior_grid();
    constexpr uint32_t idesc = tc_idesc(128, 128, E::fmt);
    auto sync_all = [&]() {
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
    };
    // the operand element at (row r, K = 64 t + kk) of a three-atom tile
    auto at = [](uint8_t *base, int t, int r, int kk) { return base + t * kAtom + sw128_off(r, kk); };
    uint32_t phase = 0;
    const int steps = (a.total + 1) / 2;
    for (int st = blockIdx.x; st < steps; st += gridDim.x) {
        const int g = 2 * st + b;
        bool active = g < a.total;
        const WfsDesc &W = a.wfs[active ? find_wfs(a.wfs, a.n_wfs, g) : 0];
        const InstDyn &D = a.dyn[W.inst];
        const int v = active ? g - W.subap_begin : 0;
        active = active && guard(v >= 0 && v < W.n_valid, a.status);
        // the subaperture's OPD: from the projection, or projected here (16 pixels per thread)
        float o[nn / 64];
        float ref = 0.0f;
        if (a.project) {
            const InstDesc &I = a.inst[W.inst];
            const int L = proj_layers(I, D);
            if (active)
                for (int l = k; l < L; l += 64) slo[b * kMaxProjLayers + l] = layer_offsets(I, W, D.t, l);
            __syncthreads();
            if (active) {
                const int S = I.S;
                const bool pow2 = (S & (S - 1)) == 0;
                const int id = __ldg(W.subap + v), sy = id / W.n_sub, sx = id - sy * W.n_sub;
                const float half = 0.5f * (float)(W.n_sub * n - 1);
                const LayerOffs *lo = slo + b * kMaxProjLayers;
                float *out = D.opd + W.opd_off + (size_t)v * nn;
                // layers outside, the thread's 16 pixels inside: every tap of a layer in flight at once
#pragma unroll
                for (int m = 0; m < nn / 64; ++m) o[m] = 0.0f;
                for (int l = 0; l < L; ++l) {
                    const LayerOffs L0 = lo[l];
                    const float *scr = layer_screen(I, D, l);
#pragma unroll
                    for (int m = 0; m < nn / 64; ++m) {
                        const int i = k + 64 * m, pp = i >> 5, qq = i & 31;
                        const float xr = (float)(sx * n + qq) - half, yr = (float)(sy * n + pp) - half;
                        int ou, ov, i0, i1, j0, j1;
                        float fx, gy;
                        screen_offset(L0.c, L0.cl, L0.fu, xr, ou, fx);
                        screen_offset(L0.c, L0.cl, L0.fv, yr, ov, gy);
                        wrap_pair(L0.bu + ou, S, pow2, i0, i1);
                        wrap_pair(L0.bv + ov, S, pow2, j0, j1);
                        if (!guard(i0 >= 0 && i1 < S && i1 >= 0 && j0 >= 0 && j1 < S && j1 >= 0 && i0 < S && j0 < S,
                                   a.status))
                            continue;
                        const float *r0 = scr + (size_t)j0 * S, *r1 = scr + (size_t)j1 * S;
                        const float s00 = __ldg(r0 + i0), s01 = __ldg(r0 + i1);
                        const float s10 = __ldg(r1 + i0), s11 = __ldg(r1 + i1);
                        const float top = fmaf(fx, s01 - s00, s00);
                        const float bot = fmaf(fx, s11 - s10, s10);
                        o[m] += fmaf(gy, bot - top, top);
                    }
                }
#pragma unroll
                for (int m = 0; m < nn / 64; ++m) {
                    const int i = k + 64 * m, pp = i >> 5, qq = i & 31;
                    const float xr = (float)(sx * n + qq) - half, yr = (float)(sy * n + pp) - half;
                    if (W.uplink) o[m] += fmaf(W.uplink->x, xr, W.uplink->y * yr);
                    out[i] = o[m];
                }
                if (k == 0) sref[b] = o[0];
            }
            __syncthreads();
            ref = sref[b];
        } else if (active) {
            const float *opd = D.opd + W.opd_off + (size_t)v * nn;
            ref = __ldg(opd);
#pragma unroll
            for (int m = 0; m < nn / 64; ++m) o[m] = __ldg(opd + k + 64 * m);
        }
        // the field of subaperture b into its rows of the first MMA's B tile: pixel (p, q) ->
        // row 64 b + q: [X_hi | X_hi | X_lo] of (re p, -im p); row 64 b + 32 + q: of (im p, re p)
        if (active) {
            const uint32_t *mk = W.mask + (size_t)v * a.mask_words;
#pragma unroll
            for (int m = 0; m < nn / 64; ++m) {
                const int i = k + 64 * m, p = i >> 5, q = i & 31;
                const bool lit = (__ldg(mk + (i >> 5)) >> (i & 31)) & 1u;
                float sn, cs;
                field_phasor(W.k_phase * (o[m] - ref), sn, cs);
                float rh, rl, ih, il;
                E::split(lit ? cs : 0.0f, rh, rl);
                E::split(lit ? sn : 0.0f, ih, il);
                const uint16_t brh = E::bits(rh), brl = E::bits(rl), bih = E::bits(ih), bil = E::bits(il);
                const int r0 = 64 * b + q, r1 = r0 + 32;
                auto put = [&](int t, int r, int kk, uint16_t v16) { *reinterpret_cast<uint16_t *>(at(sT, t, r, kk)) = v16; };
                put(0, r0, p, brh);
                put(1, r0, p, brh);
                put(2, r0, p, brl);
                put(0, r0, 32 + p, bih ^ 0x8000u);
                put(1, r0, 32 + p, bih ^ 0x8000u);
                put(2, r0, 32 + p, bil ^ 0x8000u);
                put(0, r1, p, bih);
                put(1, r1, p, bih);
                put(2, r1, p, bil);
                put(0, r1, 32 + p, brh);
                put(1, r1, 32 + p, brh);
                put(2, r1, 32 + p, brl);
            }
        }
        sync_all();
        if (*sflag) break;
        if (tid == 0) {
#pragma unroll
            for (int t = 0; t < 3; ++t)
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    mma_f16(tmem, sw128_desc(smem_u32(sA0) + t * kAtom + 32 * s),
                            sw128_desc(smem_u32(sT) + t * kAtom + 32 * s), idesc, (t | s) > 0);
            mma_commit(&mbar[0]);
        }
        if (!mbar_wait(&mbar[0], phase)) *sflag = 1;
        fence_after_sync();
        // this thread's row of U: columns 64 b + q (re) and 64 b + 32 + q (im)
        float ur[n], ui[n];
        {
            uint32_t r[16];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                GBWFS_TMEM_LD16(r, t_row + 64 * b + 16 * h);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = 16 * h + j;
                    if (c < 32) ur[c] = __uint_as_float(r[j]);
                    else ui[c - 32] = __uint_as_float(r[j]);
                }
            }
        }
        // FP16: U times 2^eu (exact), eu from the subaperture's largest component (its two warps)
        int eu = 0;
        if constexpr (kF16) {
            float mx = 0.0f;
#pragma unroll
            for (int q = 0; q < n; ++q) mx = fmaxf(mx, fmaxf(fabsf(ur[q]), fabsf(ui[q])));
            mx = warp_max(mx);
            if (lane == 0) red[wib] = mx;
            __syncthreads();
            eu = f16_scale_exp(fmaxf(red[2 * b], red[2 * b + 1]));
            const float su = pow2f(eu);
#pragma unroll
            for (int q = 0; q < n; ++q) {
                ur[q] *= su;
                ui[q] *= su;
            }
        }
        // the second MMA's A row (b, k): atom t holds (re q, im q) as hi, lo, hi
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
                const int c0 = ch * 8 + 2 * e2, c1 = c0 + 1;
                E::split2(c0 < 32 ? ur[c0] : ui[c0 - 32], c1 < 32 ? ur[c1] : ui[c1 - 32], hw[e2], lw[e2]);
            }
            *reinterpret_cast<uint4 *>(at(sT, 0, tid, ch * 8)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(at(sT, 1, tid, ch * 8)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            *reinterpret_cast<uint4 *>(at(sT, 2, tid, ch * 8)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        }
        sync_all();
        if (*sflag) break;
        if (tid == 0) {
#pragma unroll
            for (int t = 0; t < 3; ++t)
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    mma_f16(tmem, sw128_desc(smem_u32(sT) + t * kAtom + 32 * s),
                            sw128_desc(smem_u32(sB1) + t * kAtom + 32 * s), idesc, (t | s) > 0);
            mma_commit(&mbar[1]);
        }
        if (!mbar_wait(&mbar[1], phase)) *sflag = 1;
        fence_after_sync();
        phase ^= 1u;
        // I = |Y|^2 of row k (Y carries 2^eu in FP16: the intensity is exact times 2^-2eu)
        {
            const float uy = kF16 ? pow2f(-eu) : 1.0f;
            float *dstI = (active && D.st_I) ? D.st_I + W.int_off + (size_t)v * (N * N) + k * N : nullptr;
            float *irow = Iw + (size_t)b * N * (N + 1) + k * (N + 1);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t r[16], r2[16];
                GBWFS_TMEM_LD16(r, t_row + 16 * h);
                GBWFS_TMEM_LD16(r2, t_row + 64 + 16 * h);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float yr = __uint_as_float(r[j]), yi = __uint_as_float(r2[j]);
                    const float y2 = fmaf(yr, yr, yi * yi);
                    const float iv = kF16 ? y2 * uy * uy : y2;
                    irow[16 * h + j] = iv;
                    if (dstI) dstI[16 * h + j] = iv;
                }
            }
        }
        fence_before_sync();  // TMEM reads of this step precede the next step's MMAs
        __syncthreads();
        // binning, photometry, noise and centroid of subaperture b by its 64 threads
        const float *Ib = Iw + (size_t)b * N * (N + 1);
        float bv[nd2 / 64];
        float sb = 0.0f;
#pragma unroll
        for (int j = 0; j < nd2 / 64; ++j) {
            const int o = k + 64 * j, iy = o / nd, ix = o - iy * nd;
            float s2 = 0.0f;
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c) s2 += Ib[(2 * iy + r) * (N + 1) + 2 * ix + c];
            bv[j] = s2;
            sb += s2;
        }
        auto pair_sum = [&](float x, int slot) -> float {
            x = warp_sum_tc(x);
            if (lane == 0) red[4 * slot + wib] = x;
            __syncthreads();
            return red[4 * slot + 2 * b] + red[4 * slot + 2 * b + 1];
        };
        sb = pair_sum(sb, 1);
        const float scale = (active && sb > 0.0f) ? W.photons * __ldg(W.fill + v) / sb : 0.0f;
        const float cd = 0.5f * (float)(nd - 1);
        const uint32_t tlo = (uint32_t)__double_as_longlong(D.t);
        const uint32_t thi = (uint32_t)((unsigned long long)__double_as_longlong(D.t) >> 32);
        const uint64_t seed = a.inst[W.inst].seed;
        float *st_E = (active && D.st_E) ? D.st_E + W.det_off + (size_t)v * nd2 : nullptr;
        float *st_C = (active && D.st_C) ? D.st_C + W.det_off + (size_t)v * nd2 : nullptr;
        float sc = 0.0f, sx = 0.0f, sy = 0.0f;
        if (active) {
#pragma unroll 4
            for (int j = 0; j < nd2 / 64; ++j) {
                const int o = k + 64 * j, iy = o / nd, ix = o - iy * nd;
                const float e = scale * bv[j];
                const float c = D.noise ? noise_pixel(e, W.read_noise, seed, (uint32_t)(v * nd2 + o),
                                                      (uint32_t)W.gs_index, tlo, thi)
                                        : e;
                if (st_E) st_E[o] = e;
                if (st_C) st_C[o] = c;
                sc += c;
                sx = fmaf((float)ix - cd, c, sx);
                sy = fmaf((float)iy - cd, c, sy);
            }
        }
        sc = pair_sum(sc, 2);
        sx = pair_sum(sx, 3);
        sy = pair_sum(sy, 0);
        if (active && k == 0) {
            const bool ok = sc > 0.0f;
            float *sl = D.slopes + W.slope_off;
            sl[2 * v] = ok ? sx / sc : 0.0f;
            sl[2 * v + 1] = ok ? sy / sc : 0.0f;
        }
        __syncthreads();  // the spot rows and partial sums are reused by the next step
    }
    fence_before_sync();
    __syncthreads();
    if (*sflag && tid == 0 && a.status) atomicCAS(a.status, 0, 5 /* WFS_ETIMEOUT */);
    fence_after_sync();
    if (wib == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

// ---------------------------------------------------------------- host side

namespace {

template <bool kF16>
cudaError_t shape_tc64_k(const ShArgs &a, LaunchShape *out) {
    const void *f = (const void *)k_sh_tc64<kF16>;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, T64Layout::bytes);
    if (e != cudaSuccess) return e;
    const int steps = (a.total + 1) / 2;
    const int cap = a.grid_cap > 0 && a.grid_cap < 152 ? a.grid_cap : 152;
    out->func = f;
    out->grid = dim3(steps < cap ? (steps > 0 ? steps : 1) : cap);
    out->block = dim3(kT64Threads);
    out->smem = T64Layout::bytes;
    return cudaSuccess;
}

}  // namespace

bool sh_tc64_supported(int n, int N, int nd) { return n == kT64n && N == kT64N && nd == kT64nd; }

cudaError_t tc64_launch_shape(const ShArgs &a, LaunchShape *out, bool f16) {
    if (!sh_tc64_supported(a.n, a.N, a.nd) || a.slice_opd_stride > 0) return cudaErrorInvalidValue;
    return f16 ? shape_tc64_k<true>(a, out) : shape_tc64_k<false>(a, out);
}

// The two constant operand tiles of the 64-point kernel (three atoms each), in BF16 or FP16:
// A0[row b * 64 + k][K = 64 t + 32 c + p] = F[k][p] (c = 0 real, 1 imaginary) as hi, lo, hi;
// B1[row 64 c' + m][K = 64 t + 32 c + q]: for the real output column (c' = 0) F_re[m][q] (c = 0)
// and -F_im[m][q] (c = 1), for the imaginary one F_im and F_re, as hi, hi, lo.
void build_tc64_tiles(const double *F_re64, const double *F_im64, bool f16, std::vector<uint8_t> &A0,
                      std::vector<uint8_t> &B1) {
    constexpr int N = kT64N, n = kT64n;
    A0.assign(3 * kAtom, 0);
    B1.assign(3 * kAtom, 0);
    auto bits = [f16](float v) -> uint16_t {
        if (!f16) {
            uint32_t u;
            memcpy(&u, &v, 4);
            u += 0x7FFFu + ((u >> 16) & 1u);
            return (uint16_t)(u >> 16);
        }
        const __half h = __float2half_rn(v);
        uint16_t u;
        memcpy(&u, &h, 2);
        return u;
    };
    auto rounded = [&](float v) -> float {
        const uint16_t h = bits(v);
        if (f16) {
            __half hh;
            memcpy(&hh, &h, 2);
            return __half2float(hh);
        }
        const uint32_t u = (uint32_t)h << 16;
        float f;
        memcpy(&f, &u, 4);
        return f;
    };
    auto put = [&](std::vector<uint8_t> &t, int atom, int r, int kk, float v) {
        const uint16_t h = bits(v);
        memcpy(t.data() + atom * kAtom + sw128_off(r, kk), &h, 2);
    };
    for (int bb = 0; bb < 2; ++bb)
        for (int k = 0; k < N; ++k)
            for (int c = 0; c < 2; ++c)
                for (int p = 0; p < n; ++p) {
                    const double val = c == 0 ? F_re64[p * N + k] : F_im64[p * N + k];
                    const float hi = rounded((float)val), lo = (float)(val - (double)hi);
                    put(A0, 0, 64 * bb + k, 32 * c + p, hi);
                    put(A0, 1, 64 * bb + k, 32 * c + p, lo);
                    put(A0, 2, 64 * bb + k, 32 * c + p, hi);
                }
    for (int cp = 0; cp < 2; ++cp)
        for (int m = 0; m < N; ++m)
            for (int c = 0; c < 2; ++c)
                for (int q = 0; q < n; ++q) {
                    const double fr = F_re64[q * N + m], fi = F_im64[q * N + m];
                    const double val = cp == 0 ? (c == 0 ? fr : -fi) : (c == 0 ? fi : fr);
                    const float hi = rounded((float)val), lo = (float)(val - (double)hi);
                    put(B1, 0, 64 * cp + m, 32 * c + q, hi);
                    put(B1, 1, 64 * cp + m, 32 * c + q, hi);
                    put(B1, 2, 64 * cp + m, 32 * c + q, lo);
                }
}

}  // namespace gbwfs
