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

constexpr int kTilePixels = 4096;                         // pupil pixels per tiled CTA
constexpr int kTilePx = kTilePixels / kProjThreads;       // per thread

__device__ __forceinline__ int wrap_index(int i, int S, bool pow2) {
    if (pow2) return i & (S - 1);
    int r = i % S;
    return r < 0 ? r + S : r;
}

__global__ void __launch_bounds__(kProjThreads) k_project(const __grid_constant__ ProjArgs a) {
    allow_dependent_grid();  // every CTA of this grid is resident or done: the spot kernel may start
    __shared__ int s_bu[kMaxLayers], s_bv[kMaxLayers];
    __shared__ float s_fu[kMaxLayers], s_fv[kMaxLayers], s_c[kMaxLayers], s_cl[kMaxLayers];

    // the WFS owning this CTA: last entry whose first CTA is <= bid
    const int bid = (int)blockIdx.x + a.block_base;
    int lo = 0, hi = a.n_wfs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.wfs[mid].proj_block_begin <= bid) lo = mid;
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

    const bool pow2 = (S & (S - 1)) == 0;
    if (W.tiled) {
        // one run of consecutive subapertures of one subaperture row; each layer's screen
        // footprint is staged in shared memory (cp.async, double-buffered so the next layer
        // streams in while this one is interpolated); coordinates come from per-column and
        // per-row tables (a pixel's screen column depends on its pupil column only)
        extern __shared__ float psm[];
        const int4 sg = W.segs[bid - W.proj_block_begin];  // sy, v_first, count, sx0
        const int n = W.n, nn = n * n, ncol = sg.z * n;
        const int box_floats = ((a.box_cap - ((4 * (ncol + n) + 3) & ~3)) / 2) & ~3;
        float2 *tab[2] = {reinterpret_cast<float2 *>(psm), reinterpret_cast<float2 *>(psm) + (ncol + n)};
        const int box_off = (4 * (ncol + n) + 3) & ~3;  // 16-byte aligned boxes
        float *boxb[2] = {psm + box_off, psm + box_off + (box_floats & ~3)};
        const float half = 0.5f * (float)(W.n_sub * n - 1);
        // thread -> (pupil row p, columns ch + k nch, k < kTilePx): lanes of a warp take
        // consecutive columns of one row, so their table and box reads fall in distinct banks
        const int nch = (ncol + kTilePx - 1) / kTilePx, ntask = n * nch;  // ntask <= kProjThreads
        const bool has_task = (int)threadIdx.x < ntask;
        const int p = has_task ? (int)threadIdx.x / nch : 0, ch = (int)threadIdx.x - p * nch;
        float acc[kTilePx];
#pragma unroll
        for (int k = 0; k < kTilePx; ++k) acc[k] = 0.0f;
        auto tables = [&](int l, float2 *t) {
            const float ch = s_c[l], cl = s_cl[l];
            for (int j = threadIdx.x; j < ncol + n; j += kProjThreads) {
                const bool col = j < ncol;
                const float xr = col ? (float)(sg.w * n + j) - half : (float)(sg.x * n + (j - ncol)) - half;
                const float ph = __fmul_rn(ch, xr), pl = fmaf(ch, xr, -ph) + cl * xr;
                const float ih = floorf(ph);
                const float ru = ((ph - ih) + pl) + (col ? s_fu[l] : s_fv[l]);
                const float iu = floorf(ru);
                t[j] = make_float2(__int_as_float((int)ih + (int)iu), ru - iu);
            }
        };
        // Box origin (relative to the layer base) and width, the origin rounded down so that
        // the box's first screen column is a multiple of 4 (16-byte copies when S % 4 == 0).
        const bool vec = (S & 3) == 0;
        auto box_geom = [&](int l, const float2 *t, int &bx0, int &by0, int &bw, int &bh) {
            bx0 = __float_as_int(t[0].x);
            by0 = __float_as_int(t[ncol].x);
            bw = __float_as_int(t[ncol - 1].x) - bx0 + 2;
            bh = __float_as_int(t[ncol + n - 1].x) - by0 + 2;
            if (vec) {
                const int off = wrap_index(s_bu[l] + bx0, S, pow2) & 3;
                bx0 -= off;
                bw = (bw + off + 3) & ~3;
            }
        };
        // returns false (for every thread) when the box would not fit
        auto issue_box = [&](int l, const float2 *t, float *box) -> bool {
            int bx0, by0, bw, bh;
            box_geom(l, t, bx0, by0, bw, bh);
            if (bw * bh > box_floats) return false;
            const float *scr = D.screens + (size_t)l * S * S;
            if (vec) {
                // one warp per box row, one lane per 16-byte chunk
                const int cw = bw >> 2, lane = threadIdx.x & 31, cbase = s_bu[l] + bx0;
                for (int r = threadIdx.x >> 5; r < bh; r += kProjThreads / 32) {
                    const float *srow = scr + (size_t)wrap_index(s_bv[l] + by0 + r, S, pow2) * S;
                    float *drow = box + r * bw;
                    for (int c4 = lane; c4 < cw; c4 += 32) {
                        const float *src = srow + wrap_index(cbase + 4 * c4, S, pow2);
                        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(drow + 4 * c4);
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
                    }
                }
            } else {
                for (int r = 0; r < bh; ++r) {
                    const float *grow = scr + (size_t)wrap_index(s_bv[l] + by0 + r, S, pow2) * S;
                    for (int c = threadIdx.x; c < bw; c += kProjThreads) {
                        const float *src = grow + wrap_index(s_bu[l] + bx0 + c, S, pow2);
                        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(box + r * bw + c);
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
                    }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            return true;
        };
        bool fits = true;
        tables(0, tab[0]);
        __syncthreads();
        fits = issue_box(0, tab[0], boxb[0]);
        for (int l = 0; l < I.n_layers && fits; ++l) {
            const int cur = l & 1, nxt = cur ^ 1;
            const bool more = l + 1 < I.n_layers;
            if (more) tables(l + 1, tab[nxt]);
            __syncthreads();
            bool fits_next = true;
            if (more) fits_next = issue_box(l + 1, tab[nxt], boxb[nxt]);
            if (more && fits_next)
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            else
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            const float2 *t = tab[cur];
            const float *box = boxb[cur];
            int bx0, by0, bw, bh;
            box_geom(l, t, bx0, by0, bw, bh);
            if (has_task) {
                const float2 rp = t[ncol + p];
                const float *brow = box + (__float_as_int(rp.x) - by0) * bw - bx0;
#pragma unroll
                for (int k = 0; k < kTilePx; ++k) {
                    const int j = ch + k * nch;
                    if (j < ncol) {
                        const float2 cj = t[j];
                        const float *b0 = brow + __float_as_int(cj.x);
                        const float s00 = b0[0], s01 = b0[1], s10 = b0[bw], s11 = b0[bw + 1];
                        const float top = fmaf(cj.y, s01 - s00, s00);
                        const float bot = fmaf(cj.y, s11 - s10, s10);
                        acc[k] += fmaf(rp.y, bot - top, top);
                    }
                }
            }
            __syncthreads();  // this layer's tables and box are free for layer l + 2
            fits = fits_next;
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (!fits && threadIdx.x == 0 && a.status) atomicCAS(a.status, 0, 6 /* WFS_EUNSUPPORTED */);
        if (has_task) {
            // column j = v n + q of the segment -> subaperture v, column q; j advances by nch
            float *opd = D.opd + W.opd_off + (size_t)sg.y * nn + p * n;
            const int dv = nch / n, dq = nch - dv * n;
            int v = ch / n, q = ch - v * n;
#pragma unroll
            for (int k = 0; k < kTilePx; ++k) {
                if (ch + k * nch < ncol) opd[v * nn + q] = acc[k];
                q += dq;
                v += dv;
                if (q >= n) {
                    q -= n;
                    ++v;
                }
            }
        }
        return;
    }

    // each thread: one 2x2 block of pupil pixels (rows p, p+1; columns q, q+1) of one subaperture
    const int n = W.n, nn = n * n, nb = (n + 1) >> 1, nbb = nb * nb;
    const int blk = (bid - W.proj_block_begin) * kProjThreads + threadIdx.x;
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

int segment_max_count(int n) {
    // a segment of c subaperture columns has n rows x ceil(c n / kTilePx) column sets, one
    // per thread
    int c = 1;
    while (n * (((c + 1) * n + kTilePx - 1) / kTilePx) <= kProjThreads) ++c;
    return c;
}

int project_blocks(const WfsDesc &d) {
    if (d.tiled) return d.n_segs;
    const int nb = (d.n + 1) / 2;
    return (d.n_valid * nb * nb + kProjThreads - 1) / kProjThreads;
}

int project_box_floats(const WfsDesc &d) {
    if (!d.tiled) return 0;
    // two sets of coordinate tables (2 x (ncol + n) float2) and two boxes of at most
    // (ncol + 2) x (n + 2) screen pixels (one per layer in flight)
    return 4 * (d.seg_cols + d.n) + 4 + 2 * ((d.seg_cols + 9) * (d.n + 3) + 4);
}

void build_segments(const std::vector<int32_t> &ids, int n_sub, int max_count, std::vector<int4> &segs,
                    int *max_run) {
    segs.clear();
    *max_run = 0;
    for (size_t v = 0; v < ids.size(); ++v) {
        const int sy = ids[v] / n_sub, sx = ids[v] - sy * n_sub;
        if (!segs.empty()) {
            int4 &b = segs.back();
            if (b.x == sy && b.w + b.z == sx && b.z < max_count) {
                ++b.z;
                if (b.z > *max_run) *max_run = b.z;
                continue;
            }
        }
        segs.push_back(make_int4(sy, (int)v, 1, sx));
        if (*max_run < 1) *max_run = 1;
    }
}

cudaError_t launch_project(const ProjArgs &a, int total_blocks, cudaStream_t s) {
    if (total_blocks <= 0) return cudaSuccess;
    LaunchShape sh;
    cudaError_t e = project_launch_shape(a, total_blocks, &sh);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(sh.func, sh.grid, sh.block, args, sh.smem, s);
}

cudaError_t project_launch_shape(const ProjArgs &a, int total_blocks, LaunchShape *out) {
    const size_t smem = (size_t)a.box_cap * sizeof(float) + (a.box_cap ? 64 : 0);
    cudaError_t e = cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    out->func = (const void *)k_project;
    out->grid = dim3(total_blocks > 0 ? total_blocks : 1);
    out->block = dim3(kProjThreads);
    out->smem = smem;
    return cudaSuccess;
}

}  // namespace gbwfs
