// k_project.cu -- layered frozen-flow projection (Sec. 4 "Open Loop
// generation": the layers' screens are piled up, each shifted for the star's
// direction and for the temporal evolution; for an LGS the pupil projection
// shrinks with altitude, c = 1 - h / range).  No Fresnel propagation.
//
// For pupil pixel x (metres from the pupil centre) and layer l the sampled
// screen coordinate, in screen pixels from the screen origin, is
//     u = S/2 + (c_l x + theta h_l - (x0_l + v_l t)) / ds
// split as  u = [S/2 + (theta h_l - x0_l - v_l t)/ds]  +  c_l (dx/ds) j'
// where j' is the pixel's half-integer column offset from the pupil centre.
// The first (time-dependent, possibly large) term is evaluated once per CTA
// in FP64 and split into an integer base (mod S) and an FP32 fraction.  The
// per-pixel term uses FP32 only: the scale c_l dx/ds is held as two floats
// (hi + lo) and the product with j' is split exactly with an FMA, so the
// fractional coordinate is accurate to ~1e-7 px even 400 px from the centre.
// This keeps long runs (large v t) exact to FP64 rounding.
//
// Output layout: per WFS, [n_valid][n][n] (subaperture-tiled), so the spot
// kernel reads each subaperture's n*n OPD as one contiguous block.
#include "internal.h"

namespace gbwfs {

constexpr int kProjThreads = 256;

__global__ void __launch_bounds__(kProjThreads) k_project(const __grid_constant__ ProjArgs a) {
    __shared__ int s_bu[kMaxLayers], s_bv[kMaxLayers];
    __shared__ float s_fu[kMaxLayers], s_fv[kMaxLayers], s_c[kMaxLayers], s_cl[kMaxLayers];

    // the WFS owning this CTA: last entry whose first CTA is <= blockIdx.x
    int lo = 0, hi = a.n_wfs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.wfs[mid].proj_block_begin <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const WfsDesc &W = a.wfs[lo];
    const InstDesc &I = a.inst[W.inst];
    const InstDyn &D = a.dyn[W.inst];
    const int S = I.S;

    if ((int)threadIdx.x < I.n_layers) {
        const int l = threadIdx.x;
        const double h = I.alt[l];
        const double c = W.is_lgs ? 1.0 - h / W.range_m : 1.0;
        const double inv_ds = 1.0 / I.ds;
        const double ou = 0.5 * S + (W.theta_x * h - (I.x0[l] + I.vx[l] * D.t)) * inv_ds;
        const double ov = 0.5 * S + (W.theta_y * h - (I.y0[l] + I.vy[l] * D.t)) * inv_ds;
        const double bu = floor(ou), bv = floor(ov);
        s_fu[l] = (float)(ou - bu);
        s_fv[l] = (float)(ov - bv);
        // base index mod S (exact: bu, bv are integers well inside 2^53)
        long long iu = (long long)bu % S, iv = (long long)bv % S;
        if (iu < 0) iu += S;
        if (iv < 0) iv += S;
        s_bu[l] = (int)iu;
        s_bv[l] = (int)iv;
        const double cs = c * W.pupil_dx_over_ds;
        s_c[l] = (float)cs;
        s_cl[l] = (float)(cs - (double)s_c[l]);
    }
    __syncthreads();

    // each thread: one 2x2 block of pupil pixels (rows p, p+1; columns q, q+1) of one subaperture
    const int n = W.n, nn = n * n, nb = (n + 1) >> 1, nbb = nb * nb;
    const int blk = ((int)blockIdx.x - W.proj_block_begin) * kProjThreads + threadIdx.x;
    if (blk >= W.n_valid * nbb) return;
    const int v = blk / nbb, r = blk - v * nbb, bp = r / nb, bq = r - bp * nb;
    const int p0 = 2 * bp, q0 = 2 * bq;
    const int id = __ldg(W.subap + v);
    const int sy = id / W.n_sub, sx = id - sy * W.n_sub;
    const float half = 0.5f * (float)(W.n_sub * n - 1);
    float xr[2], yr[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        xr[j] = (float)(sx * n + q0 + j) - half;  // exact half-integers
        yr[j] = (float)(sy * n + p0 + j) - half;
    }
    float acc[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    const bool pow2 = (S & (S - 1)) == 0;
    for (int l = 0; l < I.n_layers; ++l) {
        const float ch = s_c[l], cl = s_cl[l];
        const float *scr = D.screens + (size_t)l * S * S;
        int ci0[2], ci1[2];
        float fx[2];
        const float *row0[2], *row1[2];
        float gy[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            // c * x = ph + pl exactly (to FP32 rounding of the small part)
            const float ph = __fmul_rn(ch, xr[j]), pl = fmaf(ch, xr[j], -ph) + cl * xr[j];
            const float ih = floorf(ph);
            const float ru = ((ph - ih) + pl) + s_fu[l];  // in [-eps, 2)
            const float iu = floorf(ru);
            fx[j] = ru - iu;
            int i0 = s_bu[l] + (int)ih + (int)iu;
            const float qh = __fmul_rn(ch, yr[j]), ql = fmaf(ch, yr[j], -qh) + cl * yr[j];
            const float jh = floorf(qh);
            const float rv = ((qh - jh) + ql) + s_fv[l];
            const float jv = floorf(rv);
            gy[j] = rv - jv;
            int j0 = s_bv[l] + (int)jh + (int)jv;
            int i1, j1;
            if (pow2) {
                i0 &= S - 1;
                j0 &= S - 1;
                i1 = (i0 + 1) & (S - 1);
                j1 = (j0 + 1) & (S - 1);
            } else {
                // |c x / ds| < S is enforced when the handle is created: one wrap suffices
                i0 += (i0 < 0) ? S : 0;
                i0 -= (i0 >= S) ? S : 0;
                j0 += (j0 < 0) ? S : 0;
                j0 -= (j0 >= S) ? S : 0;
                i1 = (i0 + 1 == S) ? 0 : i0 + 1;
                j1 = (j0 + 1 == S) ? 0 : j0 + 1;
            }
            ci0[j] = i0;
            ci1[j] = i1;
            row0[j] = scr + (size_t)j0 * S;
            row1[j] = scr + (size_t)j1 * S;
        }
#pragma unroll
        for (int a2 = 0; a2 < 2; ++a2)      // row of the block
#pragma unroll
            for (int b2 = 0; b2 < 2; ++b2) {  // column of the block
                const float s00 = __ldg(row0[a2] + ci0[b2]), s01 = __ldg(row0[a2] + ci1[b2]);
                const float s10 = __ldg(row1[a2] + ci0[b2]), s11 = __ldg(row1[a2] + ci1[b2]);
                const float top = fmaf(fx[b2], s01 - s00, s00);
                const float bot = fmaf(fx[b2], s11 - s10, s10);
                acc[a2][b2] += fmaf(gy[a2], bot - top, top);
            }
    }
    float *opd = D.opd + W.opd_off + (size_t)v * nn;
#pragma unroll
    for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
        for (int b2 = 0; b2 < 2; ++b2)
            if (p0 + a2 < n && q0 + b2 < n) opd[(p0 + a2) * n + q0 + b2] = acc[a2][b2];
}

int project_blocks(int n_valid, int n) {
    const int nb = (n + 1) / 2;
    return (n_valid * nb * nb + kProjThreads - 1) / kProjThreads;
}

cudaError_t launch_project(const ProjArgs &a, int total_blocks, cudaStream_t s) {
    if (total_blocks <= 0) return cudaSuccess;
    k_project<<<total_blocks, kProjThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t project_launch_shape(int total_blocks, LaunchShape *out) {
    out->func = (const void *)k_project;
    out->grid = dim3(total_blocks > 0 ? total_blocks : 1);
    out->block = dim3(kProjThreads);
    out->smem = 0;
    return cudaSuccess;
}

}  // namespace gbwfs
