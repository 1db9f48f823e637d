// k_project.cu -- layered frozen-flow projection (Sec. 4 "Open Loop generation": the layers'
// screens are piled up, each shifted for the star's direction and for the temporal evolution;
// for an LGS the pupil projection shrinks with altitude, c = 1 - h / range).  No Fresnel
// propagation.  The coordinate arithmetic (FP64 per-layer offsets, FP32 per-pixel term with an
// exact two-float split) is in proj_math.cuh; it keeps long runs (large v t) exact to FP64
// rounding and the fractional coordinate accurate to ~1e-7 px.
//
// Output layout: per WFS, [n_valid][n][n] (subaperture-tiled), so the spot kernel reads each
// subaperture's n*n OPD as one contiguous block.
#include <algorithm>
#include <mutex>

#include "internal.h"
#include "proj_direct.cuh"
#include "proj_math.cuh"

namespace gbwfs {

constexpr int kProjThreads = 256;

constexpr int kTilePixels = 4096;                         // pupil pixels per tiled CTA
constexpr int kTilePx = kTilePixels / kProjThreads;       // per thread

__device__ __forceinline__ int wrap_index(int i, int S, bool pow2) {
    if (pow2) return i & (S - 1);
    int r = i % S;
    return r < 0 ? r + S : r;
}

constexpr int kOffsTable = 96;  // layer offsets a CTA keeps for every (WFS, layer) of its launch

// One projection block (a tiled segment, or kProjThreads 2x2 pixel blocks); every thread of
// the CTA calls it (its shared memory is free again once all threads have returned).  tab: the
// CTA's layer offsets; with all_offs, entry w * max_layers + l for every WFS w of the launch
// (filled once at the start of the kernel), else entries 0 .. L of the WFS last_wfs (refilled
// when a block belongs to another WFS).
__device__ __forceinline__ void project_one(const ProjArgs &a, const int bid, int &last_wfs, LayerOffs *tab,
                                            bool all_offs) {

    // the WFS owning this block: last entry whose first block is <= bid
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

    const LayerOffs *s_off = all_offs ? tab + lo * a.max_layers : tab;
    if (!all_offs && lo != last_wfs) {  // uniform: last_wfs was written before the caller's barrier
        if ((int)threadIdx.x < proj_layers(I, D)) tab[threadIdx.x] = layer_offsets(I, W, D.t, threadIdx.x);
        __syncthreads();
        if (threadIdx.x == 0) last_wfs = lo;  // read again only after the caller's barrier
    }

    const bool pow2 = (S & (S - 1)) == 0;
    if (W.tiled) {
        // One run of consecutive subapertures of one subaperture row.  Each layer's screen
        // footprint is staged in shared memory by cp.async; coordinates come from per-column
        // and per-row tables (a pixel's screen column depends on its pupil column only).
        // Tables and boxes are triple-buffered: in iteration l the CTA fills buffer
        // (l + 1) mod 3, last read by layer l - 2, which every thread finished before the
        // previous barrier; so one barrier per layer suffices (box l landed, tables l visible).
        extern __shared__ float psm[];
        __shared__ int4 s_geom[kMaxProjLayers];  // per layer: box origin (bx0, by0) and size (bw, bh)
        const int4 sg = W.segs[bid - W.proj_block_begin];  // sy, v_first, count, sx0
        const int n = W.n, nn = n * n, ncol = sg.z * n, L = proj_layers(I, D);
        const int tab_floats = (6 * (ncol + n) + 3) & ~3;  // three tables, 16-byte aligned boxes
        const int box_floats = ((a.box_cap - tab_floats) / 3) & ~3;
        // buffer i: tables at tab0 + i (ncol + n), box at box0 + i box_floats
        float2 *const tab0 = reinterpret_cast<float2 *>(psm);
        float *const box0 = psm + tab_floats;
        const float half = 0.5f * (float)(W.n_sub * n - 1);
        // thread -> (pupil row p, columns ch + k nch, k < kTilePx): lanes of a warp take
        // consecutive columns of one row, so their table and box reads fall in distinct banks
        const int nch = (ncol + kTilePx - 1) / kTilePx, ntask = n * nch;  // ntask <= kProjThreads
        const bool has_task = (int)threadIdx.x < ntask;
        const int p = has_task ? (int)threadIdx.x / nch : 0, ch = (int)threadIdx.x - p * nch;
        // acc[k / 2] holds the pixels k (x) and k + 1 (y), summed with packed FP32x2 operations
        // (each half rounded as the scalar operation)
        static_assert(kTilePx % 2 == 0, "pixels travel in pairs");
        float2 acc[kTilePx / 2];
#pragma unroll
        for (int k = 0; k < kTilePx / 2; ++k) acc[k] = make_float2(0.0f, 0.0f);
        // table entry j of layer l (column j < ncol, else row j - ncol): integer screen offset
        // from the layer base (as float bits) and the fraction
        auto coord = [&](int l, int j) -> float2 {
            const bool col = j < ncol;
            const float xr = col ? (float)(sg.w * n + j) - half : (float)(sg.x * n + (j - ncol)) - half;
            int off;
            float frac;
            screen_offset(s_off[l].c, s_off[l].cl, col ? s_off[l].fu : s_off[l].fv, xr, off, frac);
            return make_float2(__int_as_float(off), frac);
        };
        auto tables = [&](int l, float2 *t) {
            for (int j = threadIdx.x; j < ncol + n; j += kProjThreads) t[j] = coord(l, j);
        };
        // Box origin (relative to the layer base) and size, the origin rounded down so that the
        // box's first screen column is a multiple of 4: 16-byte copies when the layer's rows start
        // on 16-byte boundaries (S % 4 == 0 and a 16-byte-aligned layer base), else 4-byte copies.
        auto layer_vec = [&](int l) {
            return (S & 3) == 0 && (reinterpret_cast<uintptr_t>(layer_screen(I, D, l)) & 15) == 0;
        };
        if ((int)threadIdx.x < L) {
            const int l = threadIdx.x;
            const bool vec = layer_vec(l);
            int bx0 = __float_as_int(coord(l, 0).x), by0 = __float_as_int(coord(l, ncol).x);
            int bw = __float_as_int(coord(l, ncol - 1).x) - bx0 + 2;
            const int bh = __float_as_int(coord(l, ncol + n - 1).x) - by0 + 2;
            if (vec) {
                const int off = wrap_index(s_off[l].bu + bx0, S, pow2) & 3;
                bx0 -= off;
                bw = (bw + off + 3) & ~3;
            }
            s_geom[l] = make_int4(bx0, by0, bw, bh);
        }
        // returns false (for every thread) when the box would not fit
        auto issue_box = [&](int l, float *box) -> bool {
            const int4 gm = s_geom[l];
            const int bx0 = gm.x, by0 = gm.y, bw = gm.z, bh = gm.w;
            if (bw * bh > box_floats) return false;
            const float *scr = layer_screen(I, D, l);
            if (layer_vec(l)) {
                // one warp per box row, one lane per 16-byte chunk
                const int cw = bw >> 2, lane = threadIdx.x & 31, cbase = s_off[l].bu + bx0;
                for (int r = threadIdx.x >> 5; r < bh; r += kProjThreads / 32) {
                    const float *srow = scr + (size_t)wrap_index(s_off[l].bv + by0 + r, S, pow2) * S;
                    float *drow = box + r * bw;
                    for (int c4 = lane; c4 < cw; c4 += 32) {
                        if (!guard(r * bw + 4 * c4 + 3 < box_floats, a.status)) continue;
                        const float *src = srow + wrap_index(cbase + 4 * c4, S, pow2);
                        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(drow + 4 * c4);
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
                    }
                }
            } else {
                for (int r = 0; r < bh; ++r) {
                    const float *grow = scr + (size_t)wrap_index(s_off[l].bv + by0 + r, S, pow2) * S;
                    for (int c = threadIdx.x; c < bw; c += kProjThreads) {
                        if (!guard(r * bw + c < box_floats, a.status)) continue;
                        const float *src = grow + wrap_index(s_off[l].bu + bx0 + c, S, pow2);
                        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(box + r * bw + c);
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
                    }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            return true;
        };
        tables(0, tab0);
        __syncthreads();  // geometry of every layer, tables of layer 0
        bool fits = issue_box(0, box0);
        for (int l = 0; l < L && fits; ++l) {
            const int cur = l % 3, nxt = (l + 1) % 3;
            const bool more = l + 1 < L;
            bool fits_next = true;
            if (more) {
                tables(l + 1, tab0 + nxt * (ncol + n));
                fits_next = issue_box(l + 1, box0 + nxt * box_floats);
            }
            if (more && fits_next)
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            else
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            const float2 *t = tab0 + cur * (ncol + n);
            const float *box = box0 + cur * box_floats;
            const int4 gm = s_geom[l];
            const int bw = gm.z;
            if (has_task) {
                const float2 rp = t[ncol + p];
                const float *brow = box + (__float_as_int(rp.x) - gm.y) * bw - gm.x;
                const float2 gy = make_float2(rp.y, rp.y), m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
                for (int k = 0; k < kTilePx; k += 2) {
                    const int j = ch + k * nch, j2 = j + nch;
                    if (j2 < ncol) {
                        // two pixels: x - y as fma(y, -1, x) is the rounded difference
                        const float2 ca = t[j], cb = t[j2];
                        const float *b0 = brow + __float_as_int(ca.x), *b1 = brow + __float_as_int(cb.x);
                        if (!guard(b0 >= box && b0 + bw + 1 < box + box_floats && b1 >= box &&
                                       b1 + bw + 1 < box + box_floats,
                                   a.status))
                            continue;
                        const float2 fx = make_float2(ca.y, cb.y);
                        const float2 s00 = make_float2(b0[0], b1[0]), s01 = make_float2(b0[1], b1[1]);
                        const float2 s10 = make_float2(b0[bw], b1[bw]), s11 = make_float2(b0[bw + 1], b1[bw + 1]);
                        const float2 top = __ffma2_rn(fx, __ffma2_rn(s00, m1, s01), s00);
                        const float2 bot = __ffma2_rn(fx, __ffma2_rn(s10, m1, s11), s10);
                        acc[k / 2] = __fadd2_rn(acc[k / 2], __ffma2_rn(gy, __ffma2_rn(top, m1, bot), top));
                    } else if (j < ncol) {
                        const float2 cj = t[j];
                        const float *b0 = brow + __float_as_int(cj.x);
                        if (!guard(b0 >= box && b0 + bw + 1 < box + box_floats, a.status)) continue;
                        const float s00 = b0[0], s01 = b0[1], s10 = b0[bw], s11 = b0[bw + 1];
                        const float top = fmaf(cj.y, s01 - s00, s00);
                        const float bot = fmaf(cj.y, s11 - s10, s10);
                        acc[k / 2].x += fmaf(rp.y, bot - top, top);
                    }
                }
            }
            fits = fits_next;
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (!fits && threadIdx.x == 0 && a.status) atomicCAS(a.status, 0, 6 /* WFS_EUNSUPPORTED */);
        if (has_task) {
            // column j = v n + q of the segment -> subaperture v, column q; j advances by nch
            float *opd = D.opd + W.opd_off + (size_t)sg.y * nn + p * n;
            const int dv = nch / n, dq = nch - dv * n;
            int v = ch / n, q = ch - v * n;
            // the uplink tip-tilt as a plane over the pupil (zero when off); the uplink kernel may
            // still be running (programmatic dependent launch): wait for it first
            float2 up = make_float2(0.0f, 0.0f);
            if (W.uplink) {
                wait_prior_grid();
                up = *W.uplink;
            }
            const float row_tilt = up.y * ((float)(sg.x * n + p) - half);
#pragma unroll
            for (int k = 0; k < kTilePx; ++k) {
                const float xr = (float)(sg.w * n + ch + k * nch) - half;
                if (ch + k * nch < ncol) opd[v * nn + q] = (k & 1 ? acc[k / 2].y : acc[k / 2].x) + fmaf(up.x, xr, row_tilt);
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

    project_direct<kProjThreads>(a, W, I, D, s_off, bid, threadIdx.x);
}

// Blocks 0 .. n_blocks of this launch.  Each CTA starts with block blockIdx.x; with a.work the
// grid holds only as many CTAs as fit at once and each draws its next block from the ticket
// counter (issued at the top, consumed after the block), so CTAs that start late take fewer
// blocks and no partial last wave is left; the last CTA to finish resets the counter.
__global__ void __launch_bounds__(kProjThreads, 3) k_project(const __grid_constant__ ProjArgs a) {
    allow_dependent_grid();  // every CTA of this grid is resident or done: the spot kernel may start
    __shared__ int s_next, s_last_wfs;
    __shared__ LayerOffs s_tab[kOffsTable];
    // the layer offsets of every (WFS, layer) of this launch, once per CTA, when they fit
    const bool all_offs = a.n_wfs * a.max_layers <= kOffsTable;
    if (all_offs) {
        for (int i = threadIdx.x; i < a.n_wfs * a.max_layers; i += blockDim.x) {
            const int w = i / a.max_layers, l = i - w * a.max_layers;
            const WfsDesc &W = a.wfs[w];
            const InstDesc &I = a.inst[W.inst];
            if (l < proj_layers(I, a.dyn[W.inst])) s_tab[i] = layer_offsets(I, W, a.dyn[W.inst].t, l);
        }
    }
    if (threadIdx.x == 0) s_last_wfs = -1;
    __syncthreads();
    int blk = blockIdx.x;
    while (blk < a.n_blocks) {
        int ticket = 0;
        if (a.work && threadIdx.x == 0) ticket = atomicAdd(a.work, 1);
        project_one(a, blk + a.block_base, s_last_wfs, s_tab, all_offs);
        __syncthreads();  // the block's shared memory is free; orders s_next
        if (a.work) {
            if (threadIdx.x == 0) s_next = (int)gridDim.x + ticket;
            __syncthreads();
            blk = s_next;
        } else {
            blk += gridDim.x;
        }
    }
    if (a.work && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.work + 1, 1) == (int)gridDim.x - 1) {
            a.work[0] = 0;
            a.work[1] = 0;
        }
    }
}

int segment_max_count(int n) {
    // a segment of c subaperture columns spans c n pupil columns: at most two per consumer thread
    // of the bulk-copy projection (256 threads; row groups of whole warps over half the columns,
    // at most 16 rows per thread), and n rows x ceil(c n / kTilePx) column sets <= kProjThreads
    // for the cp.async form, which takes the same segments
    auto ok = [&](int c) {
        const int ncol = c * n, Tg = ((ncol + 1) / 2 + 31) & ~31;
        if (Tg > 256) return false;
        const int G = std::min(n, 256 / Tg), RG = (n + G - 1) / G;
        return RG <= 16 && n * ((ncol + kTilePx - 1) / kTilePx) <= kProjThreads;
    };
    int c = 1;
    while (ok(c + 1)) ++c;
    return c;
}

int project_blocks(const WfsDesc &d) {
    if (d.tiled) return d.n_segs;
    const int nb = (d.n + 1) / 2;
    return (d.n_valid * nb * nb + kProjThreads - 1) / kProjThreads;
}

int project_box_floats(const WfsDesc &d) {
    if (!d.tiled) return 0;
    // three sets of coordinate tables (3 x (ncol + n) float2) and three boxes of at most
    // (ncol + 2) x (n + 2) screen pixels (padded for the 16-byte alignment)
    return 6 * (d.seg_cols + d.n) + 4 + 3 * ((d.seg_cols + 9) * (d.n + 3) + 4);
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
    // longest runs first: with the projection's ticket order the short ones fill the tail
    std::stable_sort(segs.begin(), segs.end(), [](const int4 &x, const int4 &y) { return x.z > y.z; });
}

cudaError_t launch_project(const ProjArgs &a, int total_blocks, cudaStream_t s, bool after_uplink) {
    if (total_blocks <= 0) return cudaSuccess;
    LaunchShape sh;
    cudaError_t e = project_launch_shape(a, total_blocks, &sh);
    if (e != cudaSuccess) return e;
    ProjArgs b = a;
    b.n_blocks = total_blocks;
    void *args[] = {(void *)&b};
    if (!after_uplink) return cudaLaunchKernel(sh.func, sh.grid, sh.block, args, sh.smem, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = sh.grid;
    cfg.blockDim = sh.block;
    cfg.dynamicSmemBytes = sh.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, sh.func, args);
}

cudaError_t project_launch_shape(const ProjArgs &a, int total_blocks, LaunchShape *out) {
    // screen boxes moved by the bulk-copy unit where the launch's screens allow it
    if (a.stage_cap > 0) return project_bulk_launch_shape(a, total_blocks, out);
    const size_t smem = (size_t)a.box_cap * sizeof(float) + (a.box_cap ? 64 : 0);
    // the kernel's dynamic shared-memory limit is process-wide: only ever raise it, so that a
    // smaller request (the direct-gather launches ask for none) cannot lower it between another
    // thread's setting and its launch
    cudaError_t e = cudaSuccess;
    {
        static std::mutex m;
        static size_t raised[64] = {};  // per device ordinal
        int d = 0;
        if ((e = cudaGetDevice(&d)) != cudaSuccess) return e;
        std::lock_guard<std::mutex> lk(m);
        if (d < 0 || d >= 64 || smem > raised[d]) {
            if ((e = cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
                return e;
            if (d >= 0 && d < 64) raised[d] = smem;
        }
    }
    int grid = total_blocks > 0 ? total_blocks : 1;
    if (a.work) {
        // resident capacity for this shared-memory size (cached per thread)
        static thread_local size_t c_smem = (size_t)-1;
        static thread_local int c_dev = -1, c_cap = 0;
        int dev = 0;
        cudaGetDevice(&dev);
        if (smem != c_smem || dev != c_dev) {
            int per_sm = 0, sms = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project, kProjThreads, smem)) != cudaSuccess ||
                (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return e;
            c_smem = smem;
            c_dev = dev;
            c_cap = per_sm * sms;
        }
        if (c_cap > 0 && grid > c_cap) grid = c_cap;
    }
    out->func = (const void *)k_project;
    out->grid = dim3(grid);
    out->block = dim3(kProjThreads);
    out->smem = smem;
    return cudaSuccess;
}

}  // namespace gbwfs
