// proj_direct.cuh -- the projection's direct-gather form (Sec. 4 "Open Loop generation": the
// layers' screens, shifted for the star's direction and the wind and shrunk by the LGS cone,
// summed by bilinear interpolation): one thread per 2x2 block of pupil pixels, every tap read
// from the screens in global memory.  Used where the pupil samples the screens more coarsely than
// one screen pixel (no shared-memory tile pays) and by the allocation-free entry point.  The
// per-tap arithmetic and its order are those of the tiled forms, so every form gives the same
// OPD bit for bit.
#pragma once
#include "internal.h"
#include "proj_math.cuh"

namespace gbwfs {

// Block bid (kThreads 2x2 blocks) of WFS W; s_off: the WFS's layer offsets; tid < kThreads.
template <int kThreads>
__device__ __forceinline__ void project_direct(const ProjArgs &a, const WfsDesc &W, const InstDesc &I,
                                               const InstDyn &D, const LayerOffs *s_off, int bid, int tid) {
    const int S = I.S;
    const bool pow2 = (S & (S - 1)) == 0;
    // each thread: one 2x2 block of pupil pixels (rows p, p+1; columns q, q+1) of one subaperture
    const int n = W.n, nn = n * n, nb = (n + 1) >> 1, nbb = nb * nb;
    const int blk = (bid - W.proj_block_begin) * kThreads + tid;
    if (blk >= W.n_valid * nbb) return;
    const int v = blk / nbb, r = blk - v * nbb, bp = r / nb, bq = r - bp * nb;
    if (!guard(v < W.n_valid, a.status)) return;
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
    const int L = proj_layers(I, D);
    for (int l = 0; l < L; ++l) {
        const LayerOffs lo = s_off[l];
        const float *scr = layer_screen(I, D, l);
        int ci0[2], ci1[2];
        float fx[2];
        const float *row0[2], *row1[2];
        float gy[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            int ou, ov, j0, j1;
            screen_offset(lo.c, lo.cl, lo.fu, xr[j], ou, fx[j]);
            screen_offset(lo.c, lo.cl, lo.fv, yr[j], ov, gy[j]);
            wrap_pair(lo.bu + ou, S, pow2, ci0[j], ci1[j]);
            wrap_pair(lo.bv + ov, S, pow2, j0, j1);
            if (!guard(ci0[j] >= 0 && ci0[j] < S && ci1[j] >= 0 && ci1[j] < S && j0 >= 0 && j0 < S && j1 >= 0 && j1 < S,
                       a.status)) {
                ci0[j] = ci1[j] = j0 = j1 = 0;  // a checked build reads a valid sample instead
            }
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
    float2 up = make_float2(0.0f, 0.0f);
    if (W.uplink) {
        wait_prior_grid();
        up = *W.uplink;
    }
#pragma unroll
    for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
        for (int b2 = 0; b2 < 2; ++b2)
            if (p0 + a2 < n && q0 + b2 < n)
                opd[(p0 + a2) * n + q0 + b2] = acc[a2][b2] + fmaf(up.x, xr[b2], up.y * yr[a2]);
}

}  // namespace gbwfs
