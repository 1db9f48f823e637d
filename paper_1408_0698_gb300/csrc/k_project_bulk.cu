// k_project_bulk.cu -- the layered frozen-flow projection (Sec. 4 "Open Loop generation": each
// layer's screen shifted for the star's direction and the wind, shrunk by the LGS cone
// c = 1 - h / range, and the layers summed by bilinear interpolation) with the screen boxes moved
// by the bulk-copy unit.
//
// A CTA is two producer warps and eight consumer warps.  The producers walk the CTA's blocks
// (tickets as in k_project) layer by layer, taking alternate stages: per (block, layer) the
// producer computes the box of screen pixels the block's taps touch and the box rows of its
// pupil rows, writes them into one of kStages stage slots, and issues one cp.async.bulk per box
// row (two where the row crosses the periodic screen's edge) that completes on the slot's
// mbarrier.  The consumers wait for the slot, interpolate, and hand the slot back through a
// second mbarrier.  No CTA-wide barrier runs between layers, and no consumer spends instructions
// on the copies.
//
// Consumer thread = two pupil columns of a run of consecutive subapertures, half a run apart (so
// the lanes of a warp read consecutive box columns), and a group of the run's rows.  Going down a
// column, pupil row p + 1 falls on the same screen row pair as row p or one row lower (the cone
// factor is at most one for a tiled WFS), so a row's lower interpolated tap pair is the next row's
// upper pair and is reused, not reloaded; the two columns share the row bookkeeping and travel as
// packed FP32x2 operations (each half rounded as the scalar operation).  The per-tap arithmetic
// and its order are those of k_project and of the direct gathers, so the OPD is the same bit for
// bit.
#include <climits>
#include <mutex>

#include "internal.h"
#include "proj_direct.cuh"
#include "proj_math.cuh"
#include "tcgen05.cuh"

namespace gbwfs {

namespace {

constexpr int kConsumerWarps = 8;
constexpr int kConsumers = 32 * kConsumerWarps;  // = the direct-gather block size
constexpr int kProducers = 2;                    // producer warps, taking alternate stages
constexpr int kBulkThreads = kConsumers + 32 * kProducers;
constexpr int kStages = 4;
constexpr int kRowsPerThread = 16;    // pupil rows a consumer thread keeps in registers
constexpr int kBulkOffsTable = 512;   // (WFS, layer) offsets a CTA keeps for its whole launch
constexpr int kBeginCache = 1024;     // WFS first-block indices a CTA keeps in shared memory

static_assert(kConsumers == 256, "direct-gather blocks are 256 2x2 pixel blocks");

// One stage slot.  The header travels as 16-byte words (written by the producer's lane 0, read
// by the consumers as whole words).
struct __align__(16) StageMeta {
    int4 h0;          // blk (-1: no more blocks for this CTA), wfs entry, layer l, layers L
    int4 h1;          // kind (1: a direct-gather block, offs_all holds its layers' offsets; 2: a
                      // box whose consecutive pupil rows lie 0 or 1 box rows apart; 0: another
                      // box), fits (0: no box this stage), box first column bx0 (from the layer
                      // base, 16-byte aligned in the screen), box width bw (floats)
    int4 h2;          // box height bh, subaperture side n, pupil columns of the run, bits of the
                      // pupil centre (n_sub n - 1) / 2
    int4 seg;         // the run {sy, first valid index, count, sx of first}
    float *opd;       // OPD of the run's first subaperture
    const float2 *uplink;
    float4 off;       // layer l's column offset terms: c, cl, fu, -
    // pupil row p: byte offset of its lower box row (row + 1) in the box (int bits) and the
    // interpolation fraction; and its box row
    float2 rows[kMaxNPix];
    int row_idx[kMaxNPix];
    LayerOffs offs_all[kMaxProjLayers];
};

__device__ __forceinline__ int wrap_idx(int i, int S, bool pow2) {
    if (pow2) return i & (S - 1);
    const int r = i % S;
    return r < 0 ? r + S : r;
}

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_u32(m)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(m)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(m)), "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) that
// completes on mbarrier m.  Not multicast: the destination is this CTA's own shared memory.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(tc::smem_u32(m))
                 : "memory");
}

// Bilinear taps of two columns (a, b) on one box row: (s[ca], s[cb]) and (s[ca + 1], s[cb + 1]),
// interpolated across with the columns' fractions (x - y as fma(y, -1, x): the rounded difference).
__device__ __forceinline__ float2 lerp_row(const float *row, int ca, int cb, float2 fx) {
    const float2 s0 = make_float2(row[ca], row[cb]), s1 = make_float2(row[ca + 1], row[cb + 1]);
    return __ffma2_rn(fx, __ffma2_rn(s0, make_float2(-1.0f, -1.0f), s1), s0);
}

// Shared memory of one CTA: kStages boxes of stage_cap floats, then the stage slots, their
// mbarriers (full: the producer's arrival plus the copies' bytes; empty: one arrival per consumer
// warp), the launch's layer-offset table and the WFS first-block cache, when they fit.
struct BulkSmem {
    size_t meta, full, empty, tab, begin, total;
};

__host__ __device__ inline BulkSmem bulk_smem_layout(int stage_cap, int n_wfs, int max_layers) {
    BulkSmem s;
    size_t o = (size_t)kStages * stage_cap * sizeof(float);
    o = (o + 15) & ~(size_t)15;
    s.meta = o;
    o += kStages * sizeof(StageMeta);
    s.full = o;
    o += kStages * sizeof(uint64_t);
    s.empty = o;
    o += kStages * sizeof(uint64_t);
    s.tab = o;
    if (n_wfs * max_layers <= kBulkOffsTable) o += (size_t)n_wfs * max_layers * sizeof(LayerOffs);
    o = (o + 15) & ~(size_t)15;
    s.begin = o;
    if (n_wfs <= kBeginCache) o += (size_t)n_wfs * sizeof(int);
    s.total = (o + 15) & ~(size_t)15;
    return s;
}

}  // namespace

namespace {

// Producer warp `pw` of kProducers: both walk every (block, layer) of the CTA's blocks in the same
// order and producer pw stages those whose stage index is pw modulo kProducers, then (the one whose
// turn it is) the end stage.  Producer 0 draws the block tickets and hands each to the others
// through tk[] and a named barrier.
__device__ __forceinline__ void bulk_producer(const ProjArgs &a, float *boxes, StageMeta *meta, uint64_t *full,
                                              uint64_t *empty, const LayerOffs *tab, const int *begin,
                                              volatile int *tk, int pw) {
    const int lane = threadIdx.x & 31;
    int stage = 0;
    int blk = blockIdx.x;
    bool ok = true;
    int nb = 0;  // blocks walked
    // the slot of stage st, once the consumers have handed it back
    auto acquire = [&](int st) -> StageMeta * {
        const int b = st % kStages;
        if (st >= kStages && !tc::mbar_wait_suspend(&empty[b], (uint32_t)((st / kStages) - 1) & 1u)) {
            if (lane == 0 && a.status) atomicCAS(a.status, 0, 5 /* WFS_ETIMEOUT */);
            return nullptr;
        }
        return &meta[b];
    };
    // a producer whose wait gave up (ok = false) stops staging but keeps walking the blocks, so
    // that the other producers never wait at the ticket barrier for it
    while (blk < a.n_blocks) {
        int ticket = 0;
        if (a.work) {
            if (pw == 0 && lane == 0) tk[nb & 1] = atomicAdd(a.work, 1);
            asm volatile("bar.sync 1, %0;" ::"r"(32 * kProducers) : "memory");
            ticket = tk[nb & 1];
        }
        ++nb;
        const int bid = blk + a.block_base;
        // the WFS owning this block: last entry whose first block is <= bid
        int lo = 0, hi = a.n_wfs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const int bb = begin ? begin[mid] : a.wfs[mid].proj_block_begin;
            if (bb <= bid) lo = mid;
            else hi = mid - 1;
        }
        const WfsDesc &W = a.wfs[lo];
        const InstDesc &I = a.inst[W.inst];
        const InstDyn &D = a.dyn[W.inst];
        const int L = proj_layers(I, D);
        const LayerOffs *wt = tab ? tab + lo * a.max_layers : nullptr;
        if (!W.tiled) {
            StageMeta *m = (ok && stage % kProducers == pw) ? acquire(stage) : nullptr;
            if (!m) {
                if (ok && stage % kProducers == pw) ok = false;
                ++stage;
                blk = a.work ? (int)gridDim.x + ticket : blk + (int)gridDim.x;
                continue;
            }
            if (!wt)
                for (int l = lane; l < L; l += 32) m->offs_all[l] = layer_offsets(I, W, D.t, l);
            if (lane == 0) {
                m->h0 = make_int4(bid, lo, 0, L);
                m->h1 = make_int4(1, 0, 0, 0);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[stage % kStages]);
            ++stage;
        } else {
            const int S = I.S, n_lay = I.n_layers;
            const bool pow2 = (S & (S - 1)) == 0;
            const size_t SS = (size_t)S * S;
            const float *const scr0 = D.screens, *const dm0 = D.dm;
            const int4 sg = W.segs[bid - W.proj_block_begin];
            const int n = W.n, ncol = sg.z * n;
            const float half = 0.5f * (float)(W.n_sub * n - 1);
            const long long opd = (long long)(D.opd + W.opd_off + (size_t)sg.y * n * n);
            const long long uplink = (long long)W.uplink;
            // one coordinate per lane: lane p < n the run's pupil row p; lanes 30 and 31 its first
            // and last pupil columns (a second pass for them when n > 30)
            const bool row_lane = lane < n;
            const float x_row = (float)(sg.x * n + (row_lane ? lane : 0)) - half;
            const float x_col = (float)(sg.w * n + ((lane & 1) ? ncol - 1 : 0)) - half;
            for (int l = 0; l < L; ++l) {
                StageMeta *m = (ok && stage % kProducers == pw) ? acquire(stage) : nullptr;
                if (!m) {
                    if (ok && stage % kProducers == pw) ok = false;
                    ++stage;
                    continue;
                }
                const int b = stage % kStages;
                const LayerOffs o = wt ? wt[l] : layer_offsets(I, W, D.t, l);
                int off, c0, c1;
                float fr;
                if (n <= 30) {
                    const bool col_lane = lane >= 30;
                    screen_offset(o.c, o.cl, col_lane ? o.fu : o.fv, col_lane ? x_col : x_row, off, fr);
                    c0 = __shfl_sync(0xffffffffu, off, 30);
                    c1 = __shfl_sync(0xffffffffu, off, 31);
                } else {
                    screen_offset(o.c, o.cl, o.fv, x_row, off, fr);
                    int oc;
                    float fc;
                    screen_offset(o.c, o.cl, o.fu, x_col, oc, fc);
                    c0 = __shfl_sync(0xffffffffu, oc, 0);
                    c1 = __shfl_sync(0xffffffffu, oc, 1);
                }
                const int up_off = __shfl_up_sync(0xffffffffu, off, 1);
                const bool unit = __all_sync(0xffffffffu, !row_lane || lane == 0 || (unsigned)(off - up_off) <= 1u);
                const int by0 = __reduce_min_sync(0xffffffffu, row_lane ? off : INT_MAX);
                const int by1 = __reduce_max_sync(0xffffffffu, row_lane ? off : INT_MIN);
                int bx0 = c0, bw = c1 - c0 + 2;
                const int bh = by1 - by0 + 2;
                const int al = wrap_idx(o.bu + bx0, S, pow2) & 3;  // first column on a 16-byte boundary
                bx0 -= al;
                bw = (bw + al + 3) & ~3;
                const float *scr = l < n_lay ? scr0 + (size_t)l * SS : dm0 + (size_t)(l - n_lay) * SS;
                const bool fits = c1 >= c0 && bw * bh <= a.stage_cap && bw <= S && bh <= S && (S & 3) == 0 &&
                                  (reinterpret_cast<uintptr_t>(scr) & 15) == 0;
                if (row_lane) {
                    m->rows[lane] = make_float2(__int_as_float((off - by0 + 1) * bw * 4), fr);
                    m->row_idx[lane] = off - by0;
                }
                if (lane == 0) {
                    m->h0 = make_int4(bid, lo, l, L);
                    m->h1 = make_int4(unit ? 2 : 0, fits ? 1 : 0, bx0, bw);
                    m->h2 = make_int4(bh, n, ncol, __float_as_int(half));
                    m->seg = sg;
                    *reinterpret_cast<longlong2 *>(&m->opd) = make_longlong2(opd, uplink);
                    m->off = make_float4(o.c, o.cl, o.fu, 0.0f);
                    if (!fits && a.status) atomicCAS(a.status, 0, 6 /* WFS_EUNSUPPORTED */);
                }
                __syncwarp();
                if (lane == 0) {
                    if (fits) mbar_arrive_expect_tx(&full[b], (uint32_t)(bw * bh) * 4u);
                    else mbar_arrive(&full[b]);
                }
                __syncwarp();
                if (fits) {
                    const int cb = wrap_idx(o.bu + bx0, S, pow2);
                    float *box = boxes + (size_t)b * a.stage_cap;
                    for (int r = lane; r < bh; r += 32) {
                        const float *srow = scr + (size_t)wrap_idx(o.bv + by0 + r, S, pow2) * S;
                        float *drow = box + r * bw;
                        if (cb + bw <= S) {
                            bulk_copy_g2s(drow, srow + cb, (uint32_t)bw * 4u, &full[b]);
                        } else {  // the row crosses the screen's periodic edge
                            const int w1 = S - cb;
                            bulk_copy_g2s(drow, srow + cb, (uint32_t)w1 * 4u, &full[b]);
                            bulk_copy_g2s(drow + w1, srow, (uint32_t)(bw - w1) * 4u, &full[b]);
                        }
                    }
                }
                ++stage;
            }
        }
        blk = a.work ? (int)gridDim.x + ticket : blk + (int)gridDim.x;
    }
    if (ok && stage % kProducers == pw) {
        StageMeta *m = acquire(stage);
        if (m) {
            if (lane == 0) m->h0 = make_int4(-1, 0, 0, 0);
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[stage % kStages]);
        }
    }
    // the last CTA to draw past the end resets the ticket pair for the next launch
    if (a.work && pw == 0 && lane == 0) {
        __threadfence();
        if (atomicAdd(a.work + 1, 1) == (int)gridDim.x - 1) {
            a.work[0] = 0;
            a.work[1] = 0;
        }
    }
}

}  // namespace

namespace {

// R consecutive pupil rows of two columns whose box rows step by 0 or 1: straight-line code (no
// branch between rows), so the taps of later rows load while earlier rows are interpolated.  A
// step of 0 keeps the row pair (its lower pair is recomputed from the same taps: the same value);
// a step of 1 makes the lower pair the upper one.  pa, pb: the box bytes at the two columns;
// bw4: a box row in bytes.
__device__ __forceinline__ float2 lerp_at(const char *pa, const char *pb, int off, float2 fx) {
    const float *ra = reinterpret_cast<const float *>(pa + off), *rb = reinterpret_cast<const float *>(pb + off);
    const float2 s0 = make_float2(ra[0], rb[0]), s1 = make_float2(ra[1], rb[1]);
    return __ffma2_rn(fx, __ffma2_rn(s0, make_float2(-1.0f, -1.0f), s1), s0);
}

template <int R>
__device__ __forceinline__ void rows_unit(float2 (&acc)[kRowsPerThread], const float2 *rows, const char *pa,
                                          const char *pb, int bw4, float2 fx) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    float2 rp[R];
#pragma unroll
    for (int i = 0; i < R; ++i) rp[i] = rows[i];
    int prev = __float_as_int(rp[0].x);
    float2 top = lerp_at(pa, pb, prev - bw4, fx);
    float2 bot = lerp_at(pa, pb, prev, fx);
    acc[0] = __fadd2_rn(acc[0], __ffma2_rn(make_float2(rp[0].y, rp[0].y), __ffma2_rn(top, m1, bot), top));
#pragma unroll
    for (int i = 1; i < R; ++i) {
        const int off = __float_as_int(rp[i].x);
        const float2 nb = lerp_at(pa, pb, off, fx);
        const bool same = off == prev;
        top = make_float2(same ? top.x : bot.x, same ? top.y : bot.y);
        bot = nb;
        prev = off;
        acc[i] = __fadd2_rn(acc[i], __ffma2_rn(make_float2(rp[i].y, rp[i].y), __ffma2_rn(top, m1, bot), top));
    }
}

// The consumer warps: every stage the producer stages, until its end stage.
__device__ __forceinline__ void bulk_consumers(const ProjArgs &a, const float *boxes, const StageMeta *meta,
                                               uint64_t *full, uint64_t *empty, const LayerOffs *tab) {
    const int tid = threadIdx.x, lane = tid & 31;
    const float2 m1 = make_float2(-1.0f, -1.0f);
    float2 acc[kRowsPerThread];
    int p0 = 0, np = 0, n = 0, t = 0, Tg = 32, sgx = 0;
    bool b_on = false;
    float half = 0.0f;
    float2 xr = make_float2(0.0f, 0.0f);
    for (int stage = 0;; ++stage) {
        const int b = stage % kStages;
        if (!tc::mbar_wait_suspend(&full[b], (uint32_t)(stage / kStages) & 1u)) {
            if (lane == 0 && a.status) atomicCAS(a.status, 0, 5 /* WFS_ETIMEOUT */);
            return;
        }
        const StageMeta &m = meta[b];
        const int4 h0 = m.h0;
        if (h0.x < 0) return;
        const int4 h1 = m.h1;
        if (h1.x == 1) {
            const WfsDesc &W = a.wfs[h0.y];
            const InstDesc &I = a.inst[W.inst];
            const InstDyn &D = a.dyn[W.inst];
            project_direct<kConsumers>(a, W, I, D, tab ? tab + h0.y * a.max_layers : m.offs_all, h0.x, tid);
        } else {
            const int4 h2 = m.h2;
            if (h0.z == 0) {
                // this thread's columns t and t + Tg of the run and rows [p0, p0 + np): G row groups,
                // each of Tg threads (whole warps, at least half the run's columns)
                const int4 sg = m.seg;
                const int ncol = h2.z;
                n = h2.y;
                half = __int_as_float(h2.w);
                sgx = sg.x;
                Tg = (((ncol + 1) >> 1) + 31) & ~31;
                const int G = min(n, kConsumers / Tg), RG = (n + G - 1) / G;
                const int g = tid / Tg;
                t = tid - g * Tg;
                p0 = g * RG;
                np = (g < G && t < ncol && guard(RG <= kRowsPerThread, a.status)) ? max(0, min(RG, n - p0)) : 0;
                b_on = t + Tg < ncol;
                xr = make_float2((float)(sg.w * n + t) - half, (float)(sg.w * n + t + Tg) - half);
#pragma unroll
                for (int i = 0; i < kRowsPerThread; ++i) acc[i] = make_float2(0.0f, 0.0f);
            }
            if (np > 0 && h1.y) {
                const float4 of = m.off;
                int oa, ob;
                float fa, fb;
                screen_offset(of.x, of.y, of.z, xr.x, oa, fa);
                screen_offset(of.x, of.y, of.z, xr.y, ob, fb);
                const int bw = h1.w, bh = h2.x;
                // box columns, kept inside the box (column b of a thread past the run's end is
                // computed and dropped)
                guard(oa - h1.z >= 0 && oa - h1.z + 1 < bw, a.status);
                const int ca = min(max(oa - h1.z, 0), bw - 2), cb = min(max(ob - h1.z, 0), bw - 2);
                const float2 fx = make_float2(fa, fb);
                const float *box = boxes + (size_t)b * a.stage_cap;
                if (h1.x == 2) {
                    const char *pa = reinterpret_cast<const char *>(box + ca), *pb = reinterpret_cast<const char *>(box + cb);
                    switch (np) {
#define GBWFS_ROWS_CASE(R) \
    case R: rows_unit<R>(acc, m.rows + p0, pa, pb, bw * 4, fx); break;
                        GBWFS_ROWS_CASE(1) GBWFS_ROWS_CASE(2) GBWFS_ROWS_CASE(3) GBWFS_ROWS_CASE(4)
                        GBWFS_ROWS_CASE(5) GBWFS_ROWS_CASE(6) GBWFS_ROWS_CASE(7) GBWFS_ROWS_CASE(8)
                        GBWFS_ROWS_CASE(9) GBWFS_ROWS_CASE(10) GBWFS_ROWS_CASE(11) GBWFS_ROWS_CASE(12)
                        GBWFS_ROWS_CASE(13) GBWFS_ROWS_CASE(14) GBWFS_ROWS_CASE(15) GBWFS_ROWS_CASE(16)
#undef GBWFS_ROWS_CASE
                        default: break;
                    }
                } else {
                float2 rp = m.rows[p0];
                int prev = m.row_idx[p0];
                guard(prev >= 0 && prev + 1 < bh, a.status);
                float2 top = lerp_row(box + prev * bw, ca, cb, fx);
                float2 bot = lerp_row(box + (prev + 1) * bw, ca, cb, fx);
                acc[0] = __fadd2_rn(acc[0], __ffma2_rn(make_float2(rp.y, rp.y), __ffma2_rn(top, m1, bot), top));
#pragma unroll
                for (int i = 1; i < kRowsPerThread; ++i) {
                    if (i < np) {
                        rp = m.rows[p0 + i];
                        const int ry = m.row_idx[p0 + i];
                        guard(ry >= 0 && ry + 1 < bh, a.status);
                        const int d = ry - prev;  // the same for the whole warp (its rows are its group's)
                        if (d == 1) {
                            // one screen row lower: the lower pair becomes the upper one
                            top = bot;
                            bot = lerp_row(box + (ry + 1) * bw, ca, cb, fx);
                        } else if (d != 0) {
                            top = lerp_row(box + ry * bw, ca, cb, fx);
                            bot = lerp_row(box + (ry + 1) * bw, ca, cb, fx);
                        }
                        prev = ry;
                        acc[i] = __fadd2_rn(acc[i], __ffma2_rn(make_float2(rp.y, rp.y), __ffma2_rn(top, m1, bot), top));
                    }
                }
                }
            }
            if (h0.z == h0.w - 1 && np > 0) {
                // the uplink tip-tilt as a plane over the pupil (zero when off); the uplink kernel
                // may still be running (programmatic dependent launch): wait for it first
                float2 up = make_float2(0.0f, 0.0f);
                if (m.uplink) {
                    wait_prior_grid();
                    up = *m.uplink;
                }
                const int va = t / n, vb = (t + Tg) / n;
                float *oa = m.opd + (size_t)va * n * n + (t - va * n);
                float *ob = m.opd + (size_t)vb * n * n + (t + Tg - vb * n);
#pragma unroll
                for (int i = 0; i < kRowsPerThread; ++i)
                    if (i < np) {
                        const int p = p0 + i;
                        const float yr = (float)(sgx * n + p) - half;
                        oa[p * n] = acc[i].x + fmaf(up.x, xr.x, up.y * yr);
                        if (b_on) ob[p * n] = acc[i].y + fmaf(up.x, xr.y, up.y * yr);
                    }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
    }
}

}  // namespace

__global__ void __launch_bounds__(kBulkThreads, 2) k_project_bulk(const __grid_constant__ ProjArgs a) {
    allow_dependent_grid();  // every CTA of this grid is resident or done: the spot kernel may start
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ int s_tk[2];
    const BulkSmem L = bulk_smem_layout(a.stage_cap, a.n_wfs, a.max_layers);
    float *boxes = reinterpret_cast<float *>(bsm);
    StageMeta *meta = reinterpret_cast<StageMeta *>(bsm + L.meta);
    uint64_t *full = reinterpret_cast<uint64_t *>(bsm + L.full);
    uint64_t *empty = reinterpret_cast<uint64_t *>(bsm + L.empty);
    const bool all_offs = a.n_wfs * a.max_layers <= kBulkOffsTable;
    LayerOffs *tab = all_offs ? reinterpret_cast<LayerOffs *>(bsm + L.tab) : nullptr;
    int *begin = a.n_wfs <= kBeginCache ? reinterpret_cast<int *>(bsm + L.begin) : nullptr;
    if (all_offs) {
        for (int i = threadIdx.x; i < a.n_wfs * a.max_layers; i += blockDim.x) {
            const int w = i / a.max_layers, l = i - w * a.max_layers;
            const WfsDesc &W = a.wfs[w];
            const InstDesc &I = a.inst[W.inst];
            if (l < proj_layers(I, a.dyn[W.inst])) tab[i] = layer_offsets(I, W, a.dyn[W.inst].t, l);
        }
    }
    if (begin)
        for (int i = threadIdx.x; i < a.n_wfs; i += blockDim.x) begin[i] = a.wfs[i].proj_block_begin;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x >= kConsumers)
        bulk_producer(a, boxes, meta, full, empty, tab, begin, s_tk, (threadIdx.x - kConsumers) >> 5);
    else
        bulk_consumers(a, boxes, meta, full, empty, tab);
}

int project_stage_floats(const WfsDesc &d) {
    // a box of at most (run columns + 8) x (n + 3) screen pixels: the run's extent on the screen
    // (cone factor <= 1) plus the bilinear neighbour and up to three columns of 16-byte alignment
    if (!d.tiled) return 0;
    return (((d.seg_cols + 8) * (d.n + 3)) + 3) & ~3;
}

cudaError_t project_bulk_launch_shape(const ProjArgs &a, int total_blocks, LaunchShape *out) {
    const size_t smem = bulk_smem_layout(a.stage_cap, a.n_wfs, a.max_layers).total;
    // the kernel's dynamic shared-memory limit is process-wide: only ever raised
    cudaError_t e = cudaSuccess;
    {
        static std::mutex m;
        static size_t raised[64] = {};  // per device ordinal
        int d = 0;
        if ((e = cudaGetDevice(&d)) != cudaSuccess) return e;
        std::lock_guard<std::mutex> lk(m);
        if (d < 0 || d >= 64 || smem > raised[d]) {
            if ((e = cudaFuncSetAttribute(k_project_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess)
                return e;
            if (d >= 0 && d < 64) raised[d] = smem;
        }
    }
    int grid = total_blocks > 0 ? total_blocks : 1;
    if (a.work) {
        static thread_local size_t c_smem = (size_t)-1;
        static thread_local int c_dev = -1, c_cap = 0;
        int dev = 0;
        cudaGetDevice(&dev);
        if (smem != c_smem || dev != c_dev) {
            int per_sm = 0, sms = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project_bulk, kBulkThreads, smem)) !=
                    cudaSuccess ||
                (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return e;
            c_smem = smem;
            c_dev = dev;
            c_cap = per_sm * sms;
        }
        if (c_cap > 0 && grid > c_cap) grid = c_cap;
    }
    out->func = (const void *)k_project_bulk;
    out->grid = dim3(grid);
    out->block = dim3(kBulkThreads);
    out->smem = smem;
    return cudaSuccess;
}

}  // namespace gbwfs
