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
#include "proj_math.cuh"

namespace gbwfs {

constexpr int kProjThreads = 256;

constexpr int kProjWarps = kProjThreads / 32;
constexpr int kRowChunk = 16;   // pupil rows a warp accumulates at once (n <= 16: all of them)
constexpr int kUnitCols = 32;   // pupil columns of a dense unit: one per lane

__device__ __forceinline__ int wrap_index(int i, int S, bool pow2) {
    if (pow2) return i & (S - 1);
    int r = i % S;
    return r < 0 ? r + S : r;
}

constexpr int kOffsTable = 96;  // layer offsets a CTA keeps for every (WFS, layer) of its launch

// Work units.  Launch block b of a WFS holds up to kProjWarps warp units: for a WFS sampled
// densely (pupil pitch <= screen pitch) block b is a run of consecutive valid subapertures of
// one subaperture row (a segment of at most kProjWarps * 32 pupil columns), and unit (b, w) is
// its columns [32 w, 32 w + 32) over the segment's n pupil rows; otherwise unit (b, w) is 32
// threads of 2 x 2 pupil pixels each.  Every warp takes units from the ticket counter.

// Dense unit: lane = pupil column j of the segment.  Per layer, each lane finds its column's
// screen coordinate (integer offset and fraction; the arithmetic of proj_math.cuh); the pupil
// rows' coordinates are warp-uniform and go through a small per-warp table.  A screen row is
// read once per layer as two coalesced loads per lane, (s[cb + lane], s[cb + lane + 1]) from
// lane 0's column cb, and each lane takes its two taps from lane i0 = its column - cb by
// shuffles.  With a scale c dx/ds <= 1 consecutive pupil rows advance by at most one screen row,
// so the pair (top row, bottom row) carries over and only the new bottom row is read; the next
// row is fetched one step ahead.  The per-pixel arithmetic and the order of the layer sum are
// those of the direct gathers below, so both forms give the same OPD bit for bit.
__device__ __forceinline__ void project_dense(const ProjArgs &a, const WfsDesc &W, const InstDesc &I,
                                              const InstDyn &D, const LayerOffs *offs, const int4 sg, int chunk,
                                              int4 *rows) {
    const int lane = threadIdx.x & 31;
    const int n = W.n, nn = n * n, S = I.S, ncol = sg.z * n;
    const int j = chunk * kUnitCols + lane;
    const bool live = j < ncol;
    const bool pow2 = (S & (S - 1)) == 0;
    const float half = 0.5f * (float)(W.n_sub * n - 1);
    const float xr = (float)(sg.w * n + j) - half;
    const int L = proj_layers(I, D);
    float2 up = make_float2(0.0f, 0.0f);
    bool up_read = false;
    for (int p0 = 0; p0 < n; p0 += kRowChunk) {
        const int nr = min(kRowChunk, n - p0);
        float acc[kRowChunk];
#pragma unroll
        for (int p = 0; p < kRowChunk; ++p) acc[p] = 0.0f;
        for (int l = 0; l < L; ++l) {
            const LayerOffs lo = offs[l];
            const float *scr = layer_screen(I, D, l);
            // this lane's column
            int offc;
            float fx;
            screen_offset(lo.c, lo.cl, lo.fu, xr, offc, fx);
            const int colabs = lo.bu + offc;
            const int cb = __shfl_sync(0xffffffffu, colabs, 0);
            const int i0 = colabs - cb;
            const int c0 = wrap_index(cb + lane, S, pow2), c1 = wrap_index(cb + lane + 1, S, pow2);
            // the rows' coordinates: lane p < nr takes pupil row p0 + p
            if (lane < nr) {
                const float yr = (float)(sg.x * n + p0 + lane) - half;
                int offr;
                float gy;
                screen_offset(lo.c, lo.cl, lo.fv, yr, offr, gy);
                rows[lane] = make_int4(wrap_index(lo.bv + offr, S, pow2), offr, __float_as_int(gy), 0);
            }
            __syncwarp();
            // every live lane's two taps lie within the warp's 32-column window (scale <= 1);
            // otherwise (not met by the dense geometries) this layer gathers directly
            const bool window = __all_sync(0xffffffffu, !live || (i0 >= 0 && i0 < 32));
            const int src = i0 & 31;
            auto taps = [&](int row) -> float2 {
                const float *r = scr + (size_t)row * S;
                const float x0 = __ldg(r + c0), x1 = __ldg(r + c1);
                return make_float2(__shfl_sync(0xffffffffu, x0, src), __shfl_sync(0xffffffffu, x1, src));
            };
            auto taps_direct = [&](int row) -> float2 {
                const float *r = scr + (size_t)row * S;
                const int d0 = wrap_index(colabs, S, pow2), d1 = wrap_index(colabs + 1, S, pow2);
                return make_float2(__ldg(r + d0), __ldg(r + d1));
            };
            if (window) {
                int4 rw = rows[0];
                int cur = rw.y;  // the top row's offset
                float2 top = taps(rw.x), bot = taps(wrap_index(rw.x + 1, S, pow2));
                int nxt = wrap_index(rw.x + 2, S, pow2);
                float pf0 = __ldg(scr + (size_t)nxt * S + c0), pf1 = __ldg(scr + (size_t)nxt * S + c1);
#pragma unroll
                for (int p = 0; p < kRowChunk; ++p) {
                    if (p < nr) {
                        if (p > 0) {
                            rw = rows[p];
                            const int d = rw.y - cur;
                            if (d == 1) {
                                top = bot;
                                bot = make_float2(__shfl_sync(0xffffffffu, pf0, src), __shfl_sync(0xffffffffu, pf1, src));
                                nxt = wrap_index(rw.x + 2, S, pow2);
                                pf0 = __ldg(scr + (size_t)nxt * S + c0);
                                pf1 = __ldg(scr + (size_t)nxt * S + c1);
                            } else if (d != 0) {
                                top = taps(rw.x);
                                bot = taps(wrap_index(rw.x + 1, S, pow2));
                                nxt = wrap_index(rw.x + 2, S, pow2);
                                pf0 = __ldg(scr + (size_t)nxt * S + c0);
                                pf1 = __ldg(scr + (size_t)nxt * S + c1);
                            }
                            cur = rw.y;
                        }
                        const float gy = __int_as_float(rw.z);
                        const float t = fmaf(fx, top.y - top.x, top.x);
                        const float b = fmaf(fx, bot.y - bot.x, bot.x);
                        acc[p] += fmaf(gy, b - t, t);
                    }
                }
            } else {
#pragma unroll
                for (int p = 0; p < kRowChunk; ++p) {
                    if (p < nr) {
                        const int4 rw = rows[p];
                        const float2 top = taps_direct(rw.x), bot = taps_direct(wrap_index(rw.x + 1, S, pow2));
                        const float gy = __int_as_float(rw.z);
                        const float t = fmaf(fx, top.y - top.x, top.x);
                        const float b = fmaf(fx, bot.y - bot.x, bot.x);
                        acc[p] += fmaf(gy, b - t, t);
                    }
                }
            }
            __syncwarp();  // the row table is rewritten by the next layer
        }
        // the uplink tip-tilt as a plane over the pupil (zero when off); the uplink kernel may
        // still be running (programmatic dependent launch): wait for it first
        if (W.uplink && !up_read) {
            wait_prior_grid();
            up = *W.uplink;
            up_read = true;
        }
        if (live) {
            const int v = sg.y + j / n, q = j - (j / n) * n;
            if (guard(v < W.n_valid, a.status)) {
                float *opd = D.opd + W.opd_off + (size_t)v * nn + q;
#pragma unroll
                for (int p = 0; p < kRowChunk; ++p)
                    if (p < nr) {
                        const float row_tilt = up.y * ((float)(sg.x * n + p0 + p) - half);
                        opd[(p0 + p) * n] = acc[p] + fmaf(up.x, xr, row_tilt);
                    }
            }
        }
    }
}

// Sparse unit: each thread one 2 x 2 block of pupil pixels (rows p, p+1; columns q, q+1) of one
// subaperture, gathered directly from the screens.
__device__ __forceinline__ void project_sparse(const ProjArgs &a, const WfsDesc &W, const InstDesc &I,
                                               const InstDyn &D, const LayerOffs *s_off, int blk) {
    const int S = I.S;
    const bool pow2 = (S & (S - 1)) == 0;
    const int n = W.n, nn = n * n, nb = (n + 1) >> 1, nbb = nb * nb;
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

// Units 0 .. n_blocks * kProjWarps of this launch (unit u = (block u / kProjWarps, warp unit
// u % kProjWarps)).  Each warp starts with unit blockIdx.x * kProjWarps + its warp; with a.work
// it then draws its next unit from the ticket counter (so warps that start late take fewer
// units and no partial last wave is left), and the last warp to finish resets the counter.
__global__ void __launch_bounds__(kProjThreads, 3) k_project(const __grid_constant__ ProjArgs a) {
    allow_dependent_grid();  // every CTA of this grid is resident or done: the spot kernel may start
    __shared__ LayerOffs s_tab[kOffsTable];
    __shared__ LayerOffs s_wtab[kProjWarps][kMaxProjLayers];
    __shared__ int4 s_rows[kProjWarps][kRowChunk];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
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
    __syncthreads();
    const int n_units = a.n_blocks * kProjWarps;
    int last_wfs = -1;
    int u = blockIdx.x * kProjWarps + wib;
    while (u < n_units) {
        int ticket = 0;
        if (a.work && lane == 0) ticket = atomicAdd(a.work, 1);
        const int bid = u / kProjWarps + a.block_base, unit = u - (u / kProjWarps) * kProjWarps;
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
        const LayerOffs *offs = all_offs ? s_tab + lo * a.max_layers : s_wtab[wib];
        if (!all_offs && lo != last_wfs) {
            for (int l = lane; l < proj_layers(I, D); l += 32) s_wtab[wib][l] = layer_offsets(I, W, D.t, l);
            __syncwarp();
            last_wfs = lo;
        }
        if (W.tiled) {
            const int4 sg = W.segs[bid - W.proj_block_begin];
            if (unit * kUnitCols < sg.z * W.n) project_dense(a, W, I, D, offs, sg, unit, s_rows[wib]);
        } else {
            project_sparse(a, W, I, D, offs, (bid - W.proj_block_begin) * kProjThreads + unit * 32 + lane);
        }
        if (a.work) {
            ticket = __shfl_sync(0xffffffffu, ticket, 0);
            u = (int)gridDim.x * kProjWarps + ticket;
        } else {
            u += (int)gridDim.x * kProjWarps;
        }
    }
    if (a.work && lane == 0) {
        __threadfence();
        if (atomicAdd(a.work + 1, 1) == (int)gridDim.x * kProjWarps - 1) {
            a.work[0] = 0;
            a.work[1] = 0;
        }
    }
}

int segment_max_count(int n) {
    // a segment of c subaperture columns is c n pupil columns: at most one 32-column unit per warp
    return std::max(1, kProjWarps * kUnitCols / n);
}

int project_blocks(const WfsDesc &d) {
    if (d.tiled) return d.n_segs;
    const int nb = (d.n + 1) / 2;
    return (d.n_valid * nb * nb + kProjThreads - 1) / kProjThreads;
}

int project_box_floats(const WfsDesc &) {
    return 0;  // the projection stages nothing in dynamic shared memory
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
