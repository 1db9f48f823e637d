// api.cu -- the C ABI of include/gbwfs.h: handle lifecycle, validation, the
// static tables of the measurement, and the per-frame launches.
//
// Static tables built once per handle (Sec. 4 LGS SH: the WF is split into
// subapertures; the spot of each is a DFT; the sodium slices shift and weight
// the spot and a Gaussian gives its physical extent):
//   - valid subaperture ids and lit fractions, and each subaperture's lit-pixel
//     bits, from the pixel-centre pupil test eps D/2 <= r <= D/2 in FP64;
//   - per geometry, the centred DFT matrix F and the transfer-domain matrices
//     Ga (autocorrelation) and G (binning) in FP64, stored FP32;
//   - per LGS subaperture, the elongation transfer function (device FP64).
// Per frame: one projection launch for all guide stars, then one spot launch
// per geometry.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gbwfs.h"
#include "internal.h"

namespace {
// One NVTX range per public compute call, in the domain "gbwfs", so that a profiler groups each
// call's kernels under its name (e.g. ncu --nvtx --nvtx-include "gbwfs@wfs_measure/").  NVTX is
// header-only; without a tool attached each push and pop is a test of a null function pointer.
nvtxDomainHandle_t nvtx_domain() {
    static const nvtxDomainHandle_t d = nvtxDomainCreateA("gbwfs");
    return d;
}
struct NvtxRange {
    explicit NvtxRange(const char *name) {
        nvtxEventAttributes_t a{};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(nvtx_domain(), &a);
    }
    ~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

using namespace gbwfs;

namespace {

thread_local std::string tl_error;

struct GeomDev {
    wfs_geometry g{};
    int mask_words = 0;
    float2 *F = nullptr, *Ga = nullptr, *G = nullptr;
    uint8_t *tcB1 = nullptr, *tcB2h = nullptr, *tcB2l = nullptr;  // BF16X3 operand tiles
    uint8_t *tcA0 = nullptr;                                        // first-stage operand tile
};

// One spot launch: consecutive entries of a WFS table sharing a kernel class.
struct SpotGroup {
    int geom = 0;            // geometry index (in the owning handle)
    int first = 0, count = 0, total = 0;
    int kind = 0;            // SpotKind
    int grid_cap = 0, cta_warps = 0;
    int proj_base = 0, proj_count = 0;  // this group's projection blocks
    // LGS per-slice model: the group runs a per-slice spot kernel (the 32-point kernels' variants
    // after a projection of every (WFS, slice) pair, else the self-projecting generic kernel); the
    // kind and launch shape of the elongation-kernel model are kept to restore it
    bool per_slice = false;
    int base_kind = 0, base_grid_cap = 0, base_cta_warps = 0;
    // 32-point kernels: the per-slice OPDs come from one projection of every (WFS, slice) pair
    bool sl_projected = false;
    WfsDesc *d_sl_wfs = nullptr;
    int sl_count = 0, sl_blocks = 0;
};

int spot_kind(const wfs_geometry &g) {
    if (g.precision == WFS_PREC_BF16X3) return kSpotTc;
    if (g.precision == WFS_PREC_FP16S) return kSpotTcF16;
    return sh_n32_supported(g.n_pix_sub, g.n_fft, g.n_det) ? kSpotN32 : kSpotGeneric;
}

struct GsDev {
    wfs_guide_star gs{};
    std::vector<double> na_alt, na_w;
    int n_valid = 0;
    std::vector<int32_t> ids;
    std::vector<float> fill;
    int32_t *d_ids = nullptr;
    uint32_t *d_mask = nullptr;
    float *d_fill = nullptr;
    float2 *d_ktil = nullptr;
    float2 *d_ktil_g = nullptr;  // per-slice model: the Gaussian extent alone
    int4 *d_segs = nullptr;
    int n_segs = 0, seg_cols = 0, tiled = 0;
    double up_diam = 0.0;   // LGS uplink beam diameter (0: off)
    int up_n = 0;
    size_t slope_off = 0, opd_off = 0, int_off = 0, det_off = 0;
};

}  // namespace

struct wfs_ctx {
    // work tables: one instance, WFS entries grouped by geometry
    InstDesc inst_host{};
    InstDesc *d_inst = nullptr;
    std::vector<WfsDesc> wfs_host;
    WfsDesc *d_wfs = nullptr;
    std::vector<SpotGroup> groups;
    int proj_blocks = 0, proj_box = 0;
    int proj_stage = 0;                 // bulk-copy projection box floats (-1: that form is off)
    bool screens_host_mapped = false;   // the screens of the current call are mapped host memory
    wfs_telescope tel{};
    std::vector<GeomDev> geoms;
    std::vector<GsDev> gs;
    int n_layers = 0, S = 0;
    double ds = 0.0;
    std::vector<double> alt, vx, vy, x0, y0;
    uint64_t seed = 0;
    int noise = 0;
    int device = 0;
    float *d_opd = nullptr;
    size_t opd_total = 0, int_total = 0, det_total = 0;
    int total_valid = 0;
    int *d_status = nullptr;
    int *d_work = nullptr;  // ticket counters: a pair per spot group, then a pair per group's projection
    float *d_E = nullptr;   // expected images of the split noise pass (det_total floats)
    // host-buffer path: two staging buffer sets used alternately, uploads on a copy stream
    float *d_screens_stage[2] = {nullptr, nullptr};
    float *d_slopes_stage[2] = {nullptr, nullptr};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
    unsigned long long host_calls = 0;
    unsigned long long host_h2d = 0, host_d2h = 0;  // bytes the last host-buffer call copied
    // rectangle copies of mapped pinned host screens: task tables (pinned host, device) per set
    HostRowTask *h_tasks[2] = {nullptr, nullptr};
    HostRowTask *d_tasks[2] = {nullptr, nullptr};
    int task_cap = 0;
    cudaStream_t last_stream = nullptr;
    std::string err;
    // side streams for the spot launches of the second and later geometries
    std::vector<cudaStream_t> side;
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_measured = nullptr;  // recorded at the end of each measurement (one stream at a time)
    std::vector<cudaEvent_t> ev_join;
    // kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;      // pool of event pairs
    std::vector<int> ev_kind;         // kernel kind of each recorded pair
    std::vector<std::string> kinds;   // kernel names
    size_t ev_used = 0;
    bool ev_overflow = false;
    wfs_loop_ctx *loop = nullptr;     // attached closed loop (at most one)
    float2 *d_uplink = nullptr;       // per guide star: uplink tilt per pupil pixel (x, y)
    double2 *d_uplink_part = nullptr; // per (WFS, layer) deflection
    int *d_uplink_count = nullptr;    // per WFS: layers done (zero between launches)
    int n_uplink = 0;                 // guide stars with the uplink tip-tilt on
    bool per_slice = false;           // LGS per-slice model on
    SliceDesc *d_slices = nullptr;    // per guide star (LGS entries used)
    float *d_opd_sl = nullptr;        // per-slice OPDs: slice s at s * opd_total
    cudaEvent_t ev_uplink = nullptr;  // after the uplink kernel: side groups with the uplink wait on it
};

// A closed loop attached to a handle: the mirrors, their coefficients, actuator commands and
// correction layers ([n_dm][S][S], zero outside each mirror's window).
struct LoopDm {
    wfs_dm d{};
    int mode0 = 0;                    // first coefficient of this mirror
    int x0 = 0, y0 = 0, w = 0, h = 0;  // window of the grid its influence functions reach
    float *act = nullptr;             // [n_act * n_act]
};

// Scratch of the push-pull calibration: kMaxInstances copies of one guide star's WFS entry
// (instance i = mode k of the chunk pushed (i = 2k) or pulled (i = 2k + 1)), each with its own
// mirror layer, OPD, expected images and slopes.
struct CalibScratch {
    int gs = -1, kind = 0, geom = 0, group = 0, nv = 0, blocks_per_wfs = 0;
    size_t opd_stride = 0, det_stride = 0;
    WfsDesc *d_wfs = nullptr;        // [kMaxInstances]
    InstDesc *d_inst = nullptr;      // [n_dm][kMaxInstances]: a mirror as the only layer
    float *opd = nullptr, *E = nullptr, *slopes = nullptr, *layers = nullptr;
    int *work = nullptr;             // ticket pairs: projection, spot kernel
    int cur_dm = -1;                 // mirror whose windows the layer buffers hold
};

struct wfs_loop_ctx {
    CalibScratch cal;
    wfs_handle h = nullptr;
    std::vector<LoopDm> dms;
    int n_modes = 0, n_slopes = 0;
    const float *cm = nullptr, *gain = nullptr;  // caller-owned
    float *coeffs = nullptr;          // [n_modes]
    float *layers = nullptr;          // [n_dm][S][S]
    cudaEvent_t ev_done = nullptr;    // end of the loop's last enqueued work
    cudaStream_t last_stream = nullptr;
};

// Loops stepped together: they share the control matrix and the mirrors' modal bases, which
// the reconstruction and the actuator commands then read once for up to kMaxGemvVec loops.
struct wfs_loop_batch_ctx {
    std::vector<wfs_loop> loops;
};

// A batch: the instances' work tables merged, WFS entries grouped by kernel class
// (kind, n, N, nd) across instances, replayed as one CUDA graph (projection node, then one
// spot node per class in parallel) whose kernel parameters are rewritten per call.
constexpr int kBatchSlots = 8;  // concurrent subset calls per batch (one per stream)

struct BatchClass {
    int kind = 0;
    const GeomDev *geom = nullptr;   // geometry tables (those of the first handle in the class)
    int first = 0, count = 0, total = 0;
    int grid_cap = 0, cta_warps = 0;
    std::string key;
};

struct wfs_batch_ctx {
    std::vector<wfs_handle> hs;
    int device = 0;
    InstDesc *d_inst = nullptr;
    WfsDesc *d_wfs = nullptr;
    std::vector<WfsDesc> wfs_host;
    std::vector<BatchClass> classes;
    int proj_blocks = 0, proj_box = 0;
    int proj_stage = 0;                 // bulk-copy projection box floats (-1: that form is off)
    int graph_stage = 0;                // the projection form the graph was built with
    ProjArgs *pa = nullptr;          // parameter blocks the graph nodes point to
    std::vector<ShArgs *> sa;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t proj_node = nullptr;
    std::vector<cudaGraphNode_t> spot_nodes;  // per class (null when the class is empty)
    std::vector<cudaGraphNode_t> noise_nodes; // per class (null unless the class splits its noise pass)
    int use_graph = 1;
    // subset calls: per slot, a pinned staging table, its device copy and a copy-done event
    struct Slot {
        WfsDesc *h = nullptr;
        WfsDesc *d = nullptr;
        cudaEvent_t copied = nullptr;
    };
    std::vector<Slot> slots;
    // dynamic work counters: one pair per class for graph / direct launches, then one pair per
    // (subset slot, class)
    int *d_work = nullptr;
};

namespace {

wfs_status fail(wfs_handle h, wfs_status st, const std::string &msg) {
    tl_error = msg;
    if (h) h->err = msg;
    return st;
}

wfs_status cuda_fail(wfs_handle h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? WFS_ENOMEM : WFS_ECUDA, m);
}

bool is_finite(double x) { return std::isfinite(x); }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// The bulk-copy projection's box floats for WFS d on screens of side S: 0 for a WFS without
// tiles, -1 where its boxes cannot move by bulk copies (rows not a whole number of 16-byte units,
// or a box wider than the screen).
int bulk_stage_floats(const WfsDesc &d, int S) {
    if (!d.tiled) return 0;
    if (S % 4 || d.seg_cols + 8 > S || d.n + 3 > S) return -1;
    return project_stage_floats(d);
}

// Folds one WFS's value into a launch's: the largest box, or -1 once any WFS cannot use the form.
void merge_stage(int &acc, int v) {
    if (acc < 0 || v < 0) acc = -1;
    else if (v > acc) acc = v;
}

constexpr size_t kMaxTimedLaunches = 65536;

int kind_index(wfs_ctx *h, const std::string &name) {
    for (size_t i = 0; i < h->kinds.size(); ++i)
        if (h->kinds[i] == name) return (int)i;
    h->kinds.push_back(name);
    return (int)h->kinds.size() - 1;
}

// Records the start event of a timed launch; returns the pair slot or -1.
long timed_begin(wfs_ctx *h, const std::string &name, cudaStream_t s) {
    if (!h->timing) return -1;
    if (h->ev_used >= kMaxTimedLaunches) {
        h->ev_overflow = true;
        return -1;
    }
    const size_t slot = h->ev_used++;
    while (h->ev.size() < 2 * (slot + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            h->ev_used--;
            return -1;
        }
        h->ev.push_back(e);
    }
    if (h->ev_kind.size() <= slot) h->ev_kind.resize(slot + 1);
    h->ev_kind[slot] = kind_index(h, name);
    cudaEventRecord(h->ev[2 * slot], s);
    return (long)slot;
}

void timed_end(wfs_ctx *h, long slot, cudaStream_t s) {
    if (slot >= 0) cudaEventRecord(h->ev[2 * slot + 1], s);
}

// Pixel-centre pupil test on the Np x Np grid of pitch D / Np.
bool pupil_lit(double D, double eps, int Np, int i, int j) {
    const double dx = D / Np;
    const double x = (j - (Np - 1) / 2.0) * dx;
    const double y = (i - (Np - 1) / 2.0) * dx;
    const double r2 = x * x + y * y;
    const double ro = D / 2.0, ri = eps * D / 2.0;
    return (r2 <= ro * ro) && (r2 >= ri * ri);
}

// exp(-2 pi i a / N) for a a multiple of 1/4 (exact reduction mod N first).
void cexp_minus(double a, int N, double *re, double *im) {
    a = std::fmod(a, (double)N);
    const double ang = -2.0 * M_PI * a / N;
    *re = std::cos(ang);
    *im = std::sin(ang);
}

void build_geom_tables(const wfs_geometry &g, std::vector<float2> &F, std::vector<float2> &Ga,
                       std::vector<float2> &G, std::vector<double> &F64, std::vector<double> &Ga64) {
    const int n = g.n_pix_sub, N = g.n_fft, nd = g.n_det, b = N / nd;
    const double cN = (N - 1) / 2.0, cn = (n - 1) / 2.0;
    F.resize((size_t)n * N);
    Ga.resize((size_t)n * N);
    G.resize((size_t)n * nd);
    F64.resize((size_t)2 * n * N);   // re block then im block, [q][m]
    Ga64.resize((size_t)2 * n * N);  // re block then im block, [d][k]
    for (int q = 0; q < n; ++q)
        for (int m = 0; m < N; ++m) {
            double re, im;
            cexp_minus((m - cN) * (q - cn), N, &re, &im);
            F[(size_t)q * N + m] = make_float2((float)re, (float)im);
            F64[(size_t)q * N + m] = re;
            F64[(size_t)n * N + q * N + m] = im;
        }
    for (int d = 0; d < n; ++d)
        for (int k = 0; k < N; ++k) {
            double re, im;
            cexp_minus(-(k - cN) * d, N, &re, &im);  // exp(+2 pi i (k - cN) d / N)
            Ga[(size_t)d * N + k] = make_float2((float)re, (float)im);
            Ga64[(size_t)d * N + k] = re;
            Ga64[(size_t)n * N + d * N + k] = im;
        }
    for (int d = 0; d < n; ++d)
        for (int i = 0; i < nd; ++i) {
            double sr = 0.0, si = 0.0;
            for (int r = 0; r < b; ++r) {
                double re, im;
                cexp_minus((b * i + r - cN) * d, N, &re, &im);
                sr += re;
                si += im;
            }
            G[(size_t)d * nd + i] = make_float2((float)sr, (float)si);
        }
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
    if (src.empty()) {
        *dst = nullptr;
        return cudaSuccess;
    }
    cudaError_t e = cudaMalloc((void **)dst, src.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void release(wfs_ctx *h) {
    cudaFree(h->d_uplink);
    cudaFree(h->d_slices);
    h->d_slices = nullptr;
    cudaFree(h->d_opd_sl);
    h->d_opd_sl = nullptr;
    for (SpotGroup &G : h->groups) {
        cudaFree(G.d_sl_wfs);
        G.d_sl_wfs = nullptr;
    }
    cudaFree(h->d_uplink_part);
    cudaFree(h->d_uplink_count);
    if (h->ev_uplink) cudaEventDestroy(h->ev_uplink);
    h->d_uplink = nullptr;
    for (auto &g : h->geoms) {
        cudaFree(g.F);
        cudaFree(g.Ga);
        cudaFree(g.G);
        cudaFree(g.tcB1);
        cudaFree(g.tcA0);
        cudaFree(g.tcB2h);
        cudaFree(g.tcB2l);
    }
    for (auto &s : h->gs) {
        cudaFree(s.d_ids);
        cudaFree(s.d_mask);
        cudaFree(s.d_fill);
        cudaFree(s.d_ktil);
        cudaFree(s.d_ktil_g);
        cudaFree(s.d_segs);
    }
    cudaFree(h->d_opd);
    cudaFree(h->d_status);
    cudaFree(h->d_work);
    cudaFree(h->d_E);
    cudaFree(h->d_inst);
    cudaFree(h->d_wfs);
    for (int i = 0; i < 2; ++i) {
        cudaFree(h->d_screens_stage[i]);
        cudaFree(h->d_slopes_stage[i]);
        if (h->h_tasks[i]) cudaFreeHost(h->h_tasks[i]);
        cudaFree(h->d_tasks[i]);
        if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
        if (h->ev_done[i]) cudaEventDestroy(h->ev_done[i]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
    for (cudaStream_t st : h->side) cudaStreamDestroy(st);
    h->side.clear();
    for (cudaEvent_t e : h->ev_join) cudaEventDestroy(e);
    h->ev_join.clear();
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    h->ev_fork = nullptr;
    if (h->ev_measured) cudaEventDestroy(h->ev_measured);
    h->ev_measured = nullptr;
}

wfs_status validate(const wfs_telescope *tel, int n_gs, const wfs_guide_star *gs, int n_geom,
                    const wfs_geometry *geom, const wfs_layers *L) {
    auto bad = [](const std::string &m) { return fail(nullptr, WFS_EINVAL, m); };
    if (!tel || !gs || !geom || !L) return bad("null description pointer");
    if (!(tel->diameter_m > 0) || !is_finite(tel->diameter_m)) return bad("telescope diameter must be > 0");
    if (!(tel->obstruction >= 0 && tel->obstruction < 1)) return bad("obstruction must be in [0, 1)");
    if (n_gs < 1 || n_gs > kMaxGuideStars) return bad("n_gs must be in [1, 32]");
    if (n_geom < 1 || n_geom > kMaxGuideStars) return bad("n_geom must be in [1, 32]");
    for (int i = 0; i < n_geom; ++i) {
        const wfs_geometry &g = geom[i];
        if (g.n_sub < 1 || g.n_sub > 4096) return bad("geometry " + std::to_string(i) + ": n_sub out of range");
        if (g.n_pix_sub < 1 || g.n_pix_sub > kMaxNPix) return bad("geometry " + std::to_string(i) + ": n_pix_sub must be in [1, 32]");
        if (g.n_fft < g.n_pix_sub || g.n_fft > kMaxN) return bad("geometry " + std::to_string(i) + ": n_fft must be in [n_pix_sub, 64]");
        if (g.n_det < 1 || g.n_fft % g.n_det) return bad("geometry " + std::to_string(i) + ": n_fft must be a multiple of n_det");
        if (!(g.valid_fill > 0 && g.valid_fill <= 1)) return bad("geometry " + std::to_string(i) + ": valid_fill must be in (0, 1]");
        if (g.precision != WFS_PREC_FP32 && g.precision != WFS_PREC_BF16X3 && g.precision != WFS_PREC_FP16S)
            return bad("geometry " + std::to_string(i) + ": unknown precision");
    }
    if (L->n_layers < 1 || L->n_layers > kMaxLayers) return bad("n_layers must be in [1, 32]");
    if (L->screen_size < 2 || L->screen_size > (1 << 16)) return bad("screen_size out of range");
    if (!(L->screen_dx_m > 0) || !is_finite(L->screen_dx_m)) return bad("screen_dx_m must be > 0");
    if (!L->alt_m || !L->wind_vx_mps || !L->wind_vy_mps || !L->x0_m || !L->y0_m) return bad("null layer array");
    for (int l = 0; l < L->n_layers; ++l)
        if (!is_finite(L->alt_m[l]) || L->alt_m[l] < 0 || !is_finite(L->wind_vx_mps[l]) || !is_finite(L->wind_vy_mps[l]) ||
            !is_finite(L->x0_m[l]) || !is_finite(L->y0_m[l]))
            return bad("layer " + std::to_string(l) + ": bad altitude, wind or offset");
    for (int i = 0; i < n_gs; ++i) {
        const wfs_guide_star &s = gs[i];
        const std::string who = "guide star " + std::to_string(i) + ": ";
        if (s.geometry_index < 0 || s.geometry_index >= n_geom) return bad(who + "bad geometry_index");
        const wfs_geometry &g = geom[s.geometry_index];
        if (!(s.wavelength_m > 0) || !is_finite(s.wavelength_m)) return bad(who + "wavelength must be > 0");
        if (!(s.photons_per_subap >= 0) || !is_finite(s.photons_per_subap)) return bad(who + "photons must be >= 0");
        if (!(s.read_noise_e >= 0) || !is_finite(s.read_noise_e)) return bad(who + "read noise must be >= 0");
        if (!is_finite(s.theta_x_rad) || !is_finite(s.theta_y_rad)) return bad(who + "bad direction");
        double cmax = 1.0;
        if (s.is_lgs) {
            if (!(s.range_m > 0) || !is_finite(s.range_m)) return bad(who + "LGS range must be finite and > 0");
            if (!(s.spot_fwhm_rad > 0) || !is_finite(s.spot_fwhm_rad)) return bad(who + "LGS spot_fwhm_rad must be > 0");
            if (s.n_na < 1 || s.n_na > kMaxNaSlices || !s.na_alt_m || !s.na_weight) return bad(who + "n_na must be in [1, 16]");
            double wsum = 0;
            for (int k = 0; k < s.n_na; ++k) {
                if (!(s.na_alt_m[k] > 0) || !is_finite(s.na_alt_m[k]) || !(s.na_weight[k] >= 0) || !is_finite(s.na_weight[k]))
                    return bad(who + "bad sodium slice");
                wsum += s.na_weight[k];
            }
            if (!(wsum > 0)) return bad(who + "sodium weights sum to zero");
            if (!is_finite(s.launch_x_m) || !is_finite(s.launch_y_m)) return bad(who + "bad launch position");
            if (g.n_fft < 2 * g.n_pix_sub - 1)
                return fail(nullptr, WFS_EUNSUPPORTED, who + "LGS elongation needs n_fft >= 2 n_pix_sub - 1");
            for (int l = 0; l < L->n_layers; ++l)
                if (!(L->alt_m[l] < s.range_m)) return bad(who + "layer above the LGS range");
        }
        // footprint: |c x / ds| + 2 < S so that one periodic wrap suffices
        const int Np = g.n_sub * g.n_pix_sub;
        const double half = 0.5 * Np * (tel->diameter_m / Np) * cmax / L->screen_dx_m;
        if (half + 2.0 >= L->screen_size) return bad(who + "pupil footprint larger than the screen");
    }
    return WFS_OK;
}

// Geometry tables of a spot launch.
void fill_geom_args(ShArgs &sa, const GeomDev &G) {
    sa.n = G.g.n_pix_sub;
    sa.N = G.g.n_fft;
    sa.nd = G.g.n_det;
    sa.mask_words = G.mask_words;
    sa.F = G.F;
    sa.Ga = G.Ga;
    sa.G = G.G;
    sa.tc_B1 = G.tcB1;
    sa.tc_A0 = G.tcA0;
    // the first DFT stage (U = F X) of the tensor-core kernels on the CUDA cores (default, the
    // faster form) or as a third MMA (GBWFS_TC_MMA_U=1); both meet the same parity bars
    const char *mu = getenv("GBWFS_TC_MMA_U");
    sa.mma_u = (mu && mu[0] == '1') ? 1 : 0;
    sa.tc_B2h = G.tcB2h;
    sa.tc_B2l = G.tcB2l;
}

const char *kind_name(int kind) {
    return kind == kSpotTc      ? "spot_tc_bf16x3_N"
           : kind == kSpotTcF16 ? "spot_tc_fp16s_N"
           : kind == kSpotN32   ? "spot_n32_fp32_N"
                                : "spot_fp32_N";
}

// dm_layers / n_dm: the correction layers of a closed loop's mirrors, summed after the
// screens (none for an open-loop measurement).
wfs_status measure_impl(wfs_handle h, const float *screens, double t, float *slopes,
                        const wfs_stage_out *st, cudaStream_t stream, const float *dm_layers = nullptr,
                        int n_dm = 0) {
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    if (!screens || !slopes) return fail(h, WFS_EINVAL, "null screens or slopes pointer");
    if (!is_finite(t)) return fail(h, WFS_EINVAL, "t must be finite");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != h->device) return fail(h, WFS_EINVAL, "current device differs from the handle's device");
    // one stream at a time: the handle's scratch (OPD, expected images) belongs to the work in
    // flight on the stream of the previous call
    if (stream != h->last_stream && cudaEventQuery(h->ev_measured) == cudaErrorNotReady)
        return fail(h, WFS_EBUSY, "handle busy on another stream (its previous measurement is still running)");
    h->last_stream = stream;
    InstDyn dyn;
    memset(&dyn, 0, sizeof dyn);
    dyn.screens = screens;
    dyn.opd = (st && st->opd) ? st->opd : h->d_opd;
    dyn.slopes = slopes;
    dyn.st_I = st ? st->intensity : nullptr;
    dyn.st_E = (st && st->expected) ? st->expected : h->d_E;  // the split noise pass reads E back
    dyn.st_C = st ? st->counts : nullptr;
    dyn.t = t;
    dyn.noise = h->noise;
    dyn.dm = dm_layers;
    dyn.n_dm = n_dm;

    static thread_local ProjArgs pa;
    cudaError_t e;
    pa.inst = h->d_inst;
    pa.n_inst = 1;
    pa.box_cap = h->proj_box;
    // the bulk-copy form reads 16-byte rows of device memory
    pa.stage_cap = (h->proj_stage > 0 && !h->screens_host_mapped && aligned16(screens) &&
                    (n_dm == 0 || aligned16(dm_layers)))
                       ? h->proj_stage
                       : 0;
    pa.max_layers = h->inst_host.n_layers + n_dm;
    pa.status = h->d_status;
    pa.dyn[0] = dyn;
    // projection of a contiguous range of the WFS table (a group's WFSs, or all of them)
    auto project = [&](const SpotGroup &G, cudaStream_t ls) -> cudaError_t {
        const int blocks = G.proj_count;
        if (blocks <= 0) return cudaSuccess;
        pa.wfs = h->d_wfs + G.first;
        pa.n_wfs = G.count;
        pa.block_base = G.proj_base;
        pa.work = h->d_work + 2 * (h->groups.size() + 1) + 2 * (&G - h->groups.data());
        long slot = timed_begin(h, "project", ls);
        cudaError_t err = launch_project(pa, blocks, ls, ls == stream && h->n_uplink > 0 && !h->timing);
        timed_end(h, slot, ls);
        return err;
    };

    // The largest group runs on the caller's stream; each other group (a few CTAs: the NGS of
    // an LGS system) runs its own projection and spot kernel on a side stream forked at the
    // start of the call, so that its work can overlap the large projection, and is joined
    // before the call returns.  (A higher priority for the side streams made the frame slower:
    // their CTAs then displace the large projection's.)
    size_t big = 0;
    for (size_t j = 1; j < h->groups.size(); ++j)
        if (h->groups[j].total > h->groups[big].total) big = j;
    static thread_local ShArgs sa;
    // project_mode: 0 = a projection launch precedes, 1 = self-projecting on a side stream,
    // 2 = self-projecting on the caller's stream
    // slice_stride > 0: the per-slice 32-point kernels read slice s of the OPDs from d_opd_sl
    auto launch_group = [&](const SpotGroup &G, cudaStream_t ls, bool after_project, int project_mode,
                            long long slice_stride = 0) -> cudaError_t {
        memset(&sa, 0, offsetof(ShArgs, dyn));
        fill_geom_args(sa, h->geoms[G.geom]);
        sa.inst = h->d_inst;
        sa.wfs = h->d_wfs + G.first;
        sa.n_wfs = G.count;
        sa.total = G.total;
        sa.status = h->d_status;
        sa.grid_cap = G.grid_cap;
        sa.cta_warps = G.cta_warps;
        sa.n_inst = 1;
        sa.work = h->d_work + 2 * (&G - h->groups.data());
        sa.project = project_mode;
        sa.split_noise = splits_noise(G.kind, sa.N, sa.nd) ? 1 : 0;
        sa.slice_opd_stride = slice_stride;
        sa.dyn[0] = dyn;
        if (slice_stride > 0) sa.dyn[0].opd = h->d_opd_sl;
        long sl = timed_begin(h, kind_name(G.kind) + std::to_string(sa.N), ls);
        cudaError_t err = launch_spot(G.kind, sa, ls, after_project && !h->timing);
        timed_end(h, sl, ls);
        if (err == cudaSuccess && sa.split_noise) {
            long sn = timed_begin(h, "noise_cog", ls);
            err = launch_noise_cog(sa, ls, !h->timing);
            timed_end(h, sn, ls);
        }
        return err;
    };
    // the side groups fork before the uplink kernel; a side group holding a WFS with the uplink
    // on also waits for it (the projections add the uplink tilt)
    const bool forks = h->groups.size() > 1;
    if (forks && (e = cudaEventRecord(h->ev_fork, stream)) != cudaSuccess) return cuda_fail(h, e, "fork");
    if (h->n_uplink > 0) {
        long slot = timed_begin(h, "uplink", stream);
        e = launch_uplink(h->d_inst, h->d_wfs, (int)h->wfs_host.size(), h->inst_host.n_layers, h->d_uplink_part,
                          h->d_uplink_count, &dyn, stream);
        timed_end(h, slot, stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "uplink launch");
        if ((e = cudaEventRecord(h->ev_uplink, stream)) != cudaSuccess) return cuda_fail(h, e, "uplink event");
    }
    size_t k = 0;
    for (size_t j = 0; j < h->groups.size(); ++j) {
        const SpotGroup &G = h->groups[j];
        if (j == big || G.total == 0) continue;
        if (k >= h->side.size()) return fail(h, WFS_EINVAL, "internal: missing side stream");
        cudaStream_t ss = h->side[k];
        if ((e = cudaStreamWaitEvent(ss, h->ev_fork, 0)) != cudaSuccess) return cuda_fail(h, e, "fork wait");
        bool needs_uplink = false;
        for (int q = 0; q < G.count; ++q) needs_uplink |= h->wfs_host[G.first + q].uplink != nullptr;
        if (needs_uplink && (e = cudaStreamWaitEvent(ss, h->ev_uplink, 0)) != cudaSuccess)
            return cuda_fail(h, e, "uplink wait");
        // a generic-kernel group (a few NGS subapertures) projects inside its spot kernel: one
        // launch that starts with the call and owns its SMs only while it runs
        const bool fused = G.kind == kSpotGeneric || G.per_slice || (is_tc(G.kind) && h->geoms[G.geom].g.n_fft == 64);
        if (!fused && (e = project(G, ss)) != cudaSuccess) return cuda_fail(h, e, "projection launch");
        if ((e = launch_group(G, ss, !fused && G.proj_count > 0, fused ? 1 : 0)) != cudaSuccess)
            return cuda_fail(h, e, "spot launch");
        if ((e = cudaEventRecord(h->ev_join[k], ss)) != cudaSuccess) return cuda_fail(h, e, "join");
        ++k;
    }
    if (!h->groups.empty()) {
        const SpotGroup &G = h->groups[big];
        if (G.per_slice && G.sl_projected) {
            // the per-slice model: one projection of every (WFS, slice) pair into the slice OPDs,
            // then the 32-point kernel's per-slice variant
            pa.wfs = G.d_sl_wfs;
            pa.n_wfs = G.sl_count;
            pa.block_base = 0;
            pa.work = h->d_work + 2 * (h->groups.size() + 1) + 2 * big;
            pa.dyn[0].opd = h->d_opd_sl;
            long slot = timed_begin(h, "project", stream);
            e = launch_project(pa, G.sl_blocks, stream, h->n_uplink > 0 && !h->timing);
            timed_end(h, slot, stream);
            pa.dyn[0].opd = dyn.opd;
            if (e != cudaSuccess) return cuda_fail(h, e, "projection launch");
            const bool copies = st && st->opd;  // the OPD stage: the first slice's OPDs
            for (int q = 0; copies && q < G.count; ++q) {
                const WfsDesc &d = h->wfs_host[G.first + q];
                if ((e = cudaMemcpyAsync(st->opd + d.opd_off, h->d_opd_sl + d.opd_off,
                                         sizeof(float) * (size_t)d.n_valid * d.n * d.n, cudaMemcpyDeviceToDevice,
                                         stream)) != cudaSuccess)
                    return cuda_fail(h, e, "OPD stage copy");
            }
            if (G.total > 0 && (e = launch_group(G, stream, !copies, 0, (long long)h->opd_total)) != cudaSuccess)
                return cuda_fail(h, e, "spot launch");
        } else if (G.per_slice) {
            // the per-slice model projects one wavefront per sodium slice inside the spot kernel
            if (G.total > 0 && (e = launch_group(G, stream, false, 2)) != cudaSuccess)
                return cuda_fail(h, e, "spot launch");
        } else {
            // with a single group this projects every WFS (blocks 0 .. proj_blocks)
            if ((e = project(G, stream)) != cudaSuccess)
                return cuda_fail(h, e, "projection launch");
            if (G.total > 0 && (e = launch_group(G, stream, G.proj_count > 0, 0)) != cudaSuccess)
                return cuda_fail(h, e, "spot launch");
        }
    }
    for (size_t j = 0; j < k; ++j)
        if ((e = cudaStreamWaitEvent(stream, h->ev_join[j], 0)) != cudaSuccess) return cuda_fail(h, e, "join wait");
    if ((e = cudaEventRecord(h->ev_measured, stream)) != cudaSuccess) return cuda_fail(h, e, "completion event");
    return WFS_OK;
}

// Slice tables of every LGS (weights, curvatures, per-layer cones including any mirror layers),
// uploaded to h->d_slices.
wfs_status refresh_slices(wfs_handle h) {
    if (!h->per_slice) return WFS_OK;
    std::vector<SliceDesc> sd(h->gs.size());
    memset(sd.data(), 0, sizeof(SliceDesc) * sd.size());
    for (size_t g = 0; g < h->gs.size(); ++g) {
        const GsDev &G = h->gs[g];
        if (!G.gs.is_lgs) continue;
        const wfs_geometry &geo = h->geoms[G.gs.geometry_index].g;
        const double r = (h->tel.diameter_m / (geo.n_sub * geo.n_pix_sub)) / h->ds;
        SliceDesc &d = sd[g];
        d.n = (int)G.na_alt.size();
        for (int s = 0; s < d.n; ++s) {
            d.w[s] = (float)G.na_w[s];
            d.k[s] = (float)(1.0 / G.gs.range_m - 1.0 / G.na_alt[s]);
            for (int l = 0; l < kMaxProjLayers; ++l) {
                const double c = (1.0 - h->inst_host.alt[l] / G.na_alt[s]) * r;
                d.c[s][l].x = (float)c;
                d.c[s][l].y = (float)(c - (double)d.c[s][l].x);
            }
        }
    }
    cudaError_t e = cudaMemcpy(h->d_slices, sd.data(), sizeof(SliceDesc) * sd.size(), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? WFS_OK : cuda_fail(h, e, "slice tables");
}

// 32-point kernels read per-slice OPDs made by one projection launch over copies of the WFS
// entries whose range is the slice altitude (the cone) and whose OPD goes to slice s; the copies
// follow the work table (rebuilt when it changes, e.g. the uplink switch).
wfs_status build_slice_projection(wfs_handle h) {
    cudaError_t e;
    for (SpotGroup &G : h->groups) {
        cudaFree(G.d_sl_wfs);
        G.d_sl_wfs = nullptr;
        if (!G.sl_projected) continue;
        std::vector<WfsDesc> t;
        int blocks = 0;
        for (int q = 0; q < G.count; ++q) {
            const WfsDesc &d0 = h->wfs_host[G.first + q];
            const GsDev &gd = h->gs[d0.gs_index];
            const size_t ns = d0.is_lgs ? gd.na_alt.size() : 1;
            for (size_t sl = 0; sl < ns; ++sl) {
                WfsDesc d = d0;
                if (d0.is_lgs) d.range_m = gd.na_alt[sl];
                d.opd_off = d0.opd_off + (long long)(sl * h->opd_total);
                d.proj_block_begin = blocks;
                blocks += project_blocks(d);
                t.push_back(d);
            }
        }
        G.sl_count = (int)t.size();
        G.sl_blocks = blocks;
        if ((e = upload(&G.d_sl_wfs, t)) != cudaSuccess) return cuda_fail(h, e, "slice projection table");
        if (!h->d_opd_sl) {
            size_t n_max = 1;
            for (const GsDev &gd : h->gs)
                if (gd.gs.is_lgs) n_max = std::max(n_max, gd.na_alt.size());
            if ((e = cudaMalloc(&h->d_opd_sl, sizeof(float) * h->opd_total * n_max)) != cudaSuccess)
                return cuda_fail(h, e, "slice OPDs");
        }
    }
    return WFS_OK;
}

// Actuator commands (modal base times the mirror's coefficients) and correction layer of every
// mirror of the loop, on stream s.
// Layer arguments of mirror M with commands act_scale * act[i * act_stride].
DmLayerArgs dm_layer_args(wfs_handle h, const LoopDm &M, const float *act, int act_stride, float act_scale,
                          float *layer) {
    DmLayerArgs a{};
    a.act = act;
    a.act_stride = act_stride;
    a.act_scale = act_scale;
    a.n_act = M.d.n_act;
    a.support = M.d.support;
    const double r = h->ds / M.d.pitch_m;
    a.r_hi = (float)r;
    a.r_lo = (float)(r - (double)a.r_hi);
    a.c_int = (M.d.n_act - 1) / 2;
    a.c_frac = (M.d.n_act - 1) % 2 ? 0.5f : 0.0f;
    a.log2k = (float)std::log2(M.d.coupling);
    const double edge = std::pow(M.d.coupling, (double)M.d.support * M.d.support);
    a.edge = (float)edge;
    a.inv_norm = (float)(1.0 / (1.0 - edge));
    a.S = h->S;
    a.x0 = M.x0;
    a.y0 = M.y0;
    a.w = M.w;
    a.h = M.h;
    a.layer = layer;
    return a;
}

wfs_status loop_rebuild(wfs_loop lp, cudaStream_t s) {
    wfs_handle h = lp->h;
    const size_t SS = (size_t)h->S * h->S;
    static thread_local DmLayerBatch batch;
    batch.n = (int)lp->dms.size();
    for (size_t d = 0; d < lp->dms.size(); ++d) {
        const LoopDm &M = lp->dms[d];
        GemvArgs g{M.d.m2a, M.d.n_act * M.d.n_act, M.d.n_modes, lp->coeffs + M.mode0, M.act, nullptr, nullptr};
        long sl = timed_begin(h, "dm_actuators", s);
        cudaError_t e = launch_gemv(g, s);
        timed_end(h, sl, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "actuator launch");
        batch.l[d] = dm_layer_args(h, M, M.act, 1, 1.0f, lp->layers + d * SS);
    }
    long sl = timed_begin(h, "dm_layer", s);
    cudaError_t e = launch_dm_layers(batch, s);
    timed_end(h, sl, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "mirror layer launch");
    return WFS_OK;
}

void calib_free(CalibScratch &c) {
    cudaFree(c.d_wfs);
    cudaFree(c.d_inst);
    cudaFree(c.opd);
    cudaFree(c.E);
    cudaFree(c.slopes);
    cudaFree(c.layers);
    cudaFree(c.work);
    c = CalibScratch{};
}

// Builds the calibration scratch for guide star gs (kept until another star is calibrated).
wfs_status calib_prepare(wfs_loop lp, int gs) {
    wfs_handle h = lp->h;
    CalibScratch &c = lp->cal;
    if (c.gs == gs) return WFS_OK;
    cudaDeviceSynchronize();  // the previous star's scratch may still be in use
    calib_free(c);
    int k = -1;
    for (size_t i = 0; i < h->wfs_host.size(); ++i)
        if (h->wfs_host[i].gs_index == gs) k = (int)i;
    if (k < 0) return fail(h, WFS_EINVAL, "internal: guide star not in the work table");
    int grp = -1;
    for (size_t g = 0; g < h->groups.size(); ++g)
        if (k >= h->groups[g].first && k < h->groups[g].first + h->groups[g].count) grp = (int)g;
    if (grp < 0) return fail(h, WFS_EINVAL, "internal: guide star in no spot group");
    const WfsDesc base = h->wfs_host[k];
    const GeomDev &G = h->geoms[h->groups[grp].geom];
    c.kind = h->groups[grp].kind;
    c.geom = h->groups[grp].geom;
    c.group = grp;
    c.nv = base.n_valid;
    c.blocks_per_wfs = project_blocks(base);
    c.opd_stride = (size_t)c.nv * base.n * base.n;
    c.det_stride = (size_t)c.nv * G.g.n_det * G.g.n_det;
    std::vector<WfsDesc> w(kMaxInstances, base);
    for (int i = 0; i < kMaxInstances; ++i) {
        w[i].inst = i;
        w[i].opd_off = w[i].slope_off = w[i].int_off = w[i].det_off = 0;
        w[i].uplink = nullptr;  // no turbulence: no uplink tilt
        w[i].proj_block_begin = i * c.blocks_per_wfs;
        w[i].subap_begin = i * c.nv;
    }
    const int n_dm = (int)lp->dms.size();
    std::vector<InstDesc> in((size_t)n_dm * kMaxInstances);
    for (int d = 0; d < n_dm; ++d) {
        InstDesc I = h->inst_host;
        I.n_layers = 0;  // the mirror is the only layer (InstDyn::n_dm = 1)
        I.alt[0] = lp->dms[d].d.alt_m;
        I.vx[0] = I.vy[0] = I.x0[0] = I.y0[0] = 0.0;
        for (int i = 0; i < kMaxInstances; ++i) in[(size_t)d * kMaxInstances + i] = I;
    }
    const size_t SS = (size_t)h->S * h->S;
    cudaError_t e;
    auto bail = [&](cudaError_t err, const char *what) {
        calib_free(c);
        return cuda_fail(h, err, what);
    };
    if ((e = cudaMalloc(&c.d_wfs, sizeof(WfsDesc) * kMaxInstances)) != cudaSuccess) return bail(e, "calibration table");
    if ((e = cudaMalloc(&c.d_inst, sizeof(InstDesc) * in.size())) != cudaSuccess) return bail(e, "calibration table");
    if ((e = cudaMalloc(&c.opd, sizeof(float) * c.opd_stride * kMaxInstances)) != cudaSuccess ||
        (e = cudaMalloc(&c.E, sizeof(float) * c.det_stride * kMaxInstances)) != cudaSuccess ||
        (e = cudaMalloc(&c.slopes, sizeof(float) * 2 * c.nv * kMaxInstances)) != cudaSuccess ||
        (e = cudaMalloc(&c.layers, sizeof(float) * SS * kMaxInstances)) != cudaSuccess ||
        (e = cudaMalloc(&c.work, sizeof(int) * 4)) != cudaSuccess)
        return bail(e, "calibration scratch");
    if ((e = cudaMemcpy(c.d_wfs, w.data(), sizeof(WfsDesc) * kMaxInstances, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c.d_inst, in.data(), sizeof(InstDesc) * in.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(c.work, 0, sizeof(int) * 4)) != cudaSuccess)
        return bail(e, "calibration tables");
    c.gs = gs;
    c.cur_dm = -1;
    return WFS_OK;
}

void loop_free(wfs_loop lp) {
    calib_free(lp->cal);
    for (LoopDm &M : lp->dms) cudaFree(M.act);
    cudaFree(lp->coeffs);
    cudaFree(lp->layers);
    if (lp->ev_done) cudaEventDestroy(lp->ev_done);
    delete lp;
}

// One stream at a time for the loop's own buffers (coefficients, commands, layers).
bool loop_busy(wfs_loop lp, cudaStream_t s) {
    return s != lp->last_stream && cudaEventQuery(lp->ev_done) == cudaErrorNotReady;
}

}  // namespace

void gbwfs::set_thread_error(const char *msg) { tl_error = msg ? msg : ""; }

wfs_status gbwfs::validate_description(const wfs_telescope *tel, int n_gs, const wfs_guide_star *gs, int n_geom,
                                       const wfs_geometry *geom, const wfs_layers *L) {
    return validate(tel, n_gs, gs, n_geom, geom, L);
}

extern "C" {

#ifdef GBWFS_CHECK
const char *wfs_version(void) { return "gbwfs 0.1 (sm_103a, bounds-checked)"; }
#else
const char *wfs_version(void) { return "gbwfs 0.1 (sm_103a)"; }
#endif

const char *wfs_last_error(wfs_handle h) { return h ? h->err.c_str() : tl_error.c_str(); }

wfs_status wfs_create(const wfs_telescope *tel, int n_gs, const wfs_guide_star *gs, int n_geom,
                      const wfs_geometry *geom, const wfs_layers *layers, uint64_t seed,
                      int noise_enable, wfs_handle *out) {
    if (!out) return fail(nullptr, WFS_EINVAL, "null output handle pointer");
    *out = nullptr;
    wfs_status st = validate(tel, n_gs, gs, n_geom, geom, layers);
    if (st != WFS_OK) return st;
    for (int i = 0; i < n_geom; ++i) {
        const wfs_geometry &g = geom[i];
        if (g.precision != WFS_PREC_BF16X3 && g.precision != WFS_PREC_FP16S) continue;
        const std::string who = "geometry " + std::to_string(i) + (g.precision == WFS_PREC_FP16S ? ": WFS_PREC_FP16S" : ": WFS_PREC_BF16X3");
        bool lgs = false;
        for (int w = 0; w < n_gs; ++w) lgs |= gs[w].geometry_index == i && gs[w].is_lgs;
        if (sh_tc64_supported(g.n_pix_sub, g.n_fft, g.n_det)) {
            if (lgs) return fail(nullptr, WFS_EUNSUPPORTED, who + " with n_fft = 64 is built for NGS sensors only");
        } else if (!sh_tc_supported(g.n_pix_sub, g.n_fft, g.n_det)) {
            return fail(nullptr, WFS_EUNSUPPORTED,
                        who + " is built for (n_pix_sub, n_fft, n_det) = (10, 32, 16), (8, 32, 16), (8, 16, 8), "
                              "(6, 24, 12) and (32, 64, 32) (NGS)");
        }
    }

    wfs_ctx *h = new wfs_ctx();
    h->tel = *tel;
    h->seed = seed;
    h->noise = noise_enable ? 1 : 0;
    h->n_layers = layers->n_layers;
    h->S = layers->screen_size;
    h->ds = layers->screen_dx_m;
    h->alt.assign(layers->alt_m, layers->alt_m + h->n_layers);
    h->vx.assign(layers->wind_vx_mps, layers->wind_vx_mps + h->n_layers);
    h->vy.assign(layers->wind_vy_mps, layers->wind_vy_mps + h->n_layers);
    h->x0.assign(layers->x0_m, layers->x0_m + h->n_layers);
    h->y0.assign(layers->y0_m, layers->y0_m + h->n_layers);
    cudaGetDevice(&h->device);

    cudaError_t e;
    h->geoms.resize(n_geom);
    for (int i = 0; i < n_geom; ++i) {
        GeomDev &G = h->geoms[i];
        G.g = geom[i];
        G.mask_words = (geom[i].n_pix_sub * geom[i].n_pix_sub + 31) / 32;
        std::vector<float2> F, Ga, Gb;
        std::vector<double> F64, Ga64;
        build_geom_tables(geom[i], F, Ga, Gb, F64, Ga64);
        if ((e = upload(&G.F, F)) != cudaSuccess || (e = upload(&G.Ga, Ga)) != cudaSuccess ||
            (e = upload(&G.G, Gb)) != cudaSuccess) {
            release(h);
            delete h;
            return cuda_fail(nullptr, e, "table upload");
        }
        if (geom[i].precision == WFS_PREC_BF16X3 || geom[i].precision == WFS_PREC_FP16S) {
            const int n = geom[i].n_pix_sub, N = geom[i].n_fft;
            std::vector<uint8_t> b1, b2h, b2l, a0;
            if (N == 64)
                build_tc64_tiles(F64.data(), F64.data() + (size_t)n * N, geom[i].precision == WFS_PREC_FP16S, a0, b1);
            else
                build_tc_tiles(n, N, F64.data(), F64.data() + (size_t)n * N, Ga64.data(), Ga64.data() + (size_t)n * N,
                               geom[i].precision == WFS_PREC_FP16S, b1, b2h, b2l, a0);
            if ((e = upload(&G.tcB1, b1)) != cudaSuccess || (e = upload(&G.tcB2h, b2h)) != cudaSuccess ||
                (e = upload(&G.tcA0, a0)) != cudaSuccess ||
                (e = upload(&G.tcB2l, b2l)) != cudaSuccess) {
                release(h);
                delete h;
                return cuda_fail(nullptr, e, "tensor-core tile upload");
            }
        }
    }
    h->gs.resize(n_gs);
    size_t slope = 0, opd = 0, inten = 0, det = 0;
    for (int w = 0; w < n_gs; ++w) {
        GsDev &s = h->gs[w];
        s.gs = gs[w];
        if (gs[w].is_lgs) {
            s.na_alt.assign(gs[w].na_alt_m, gs[w].na_alt_m + gs[w].n_na);
            s.na_w.assign(gs[w].na_weight, gs[w].na_weight + gs[w].n_na);
        }
        s.gs.na_alt_m = s.na_alt.empty() ? nullptr : s.na_alt.data();
        s.gs.na_weight = s.na_w.empty() ? nullptr : s.na_w.data();
        if (!gs[w].is_lgs) s.gs.n_na = 0;
        const wfs_geometry &g = geom[gs[w].geometry_index];
        const int n = g.n_pix_sub, Np = g.n_sub * n, mw = (n * n + 31) / 32;
        std::vector<uint32_t> mask;
        for (int sy = 0; sy < g.n_sub; ++sy)
            for (int sx = 0; sx < g.n_sub; ++sx) {
                std::vector<uint32_t> bits(mw, 0u);
                int c = 0;
                for (int p = 0; p < n; ++p)
                    for (int q = 0; q < n; ++q)
                        if (pupil_lit(tel->diameter_m, tel->obstruction, Np, sy * n + p, sx * n + q)) {
                            ++c;
                            bits[(p * n + q) >> 5] |= 1u << ((p * n + q) & 31);
                        }
                const double f = (double)c / ((double)n * n);
                if (f >= g.valid_fill) {
                    s.ids.push_back(sy * g.n_sub + sx);
                    s.fill.push_back((float)f);
                    mask.insert(mask.end(), bits.begin(), bits.end());
                }
            }
        s.n_valid = (int)s.ids.size();
        s.slope_off = slope;
        s.opd_off = opd;
        s.int_off = inten;
        s.det_off = det;
        slope += 2 * (size_t)s.n_valid;
        opd += (size_t)s.n_valid * n * n;
        inten += (size_t)s.n_valid * g.n_fft * g.n_fft;
        det += (size_t)s.n_valid * g.n_det * g.n_det;
        if ((e = upload(&s.d_ids, s.ids)) != cudaSuccess || (e = upload(&s.d_fill, s.fill)) != cudaSuccess ||
            (e = upload(&s.d_mask, mask)) != cudaSuccess) {
            release(h);
            delete h;
            return cuda_fail(nullptr, e, "subaperture table upload");
        }
        // shared-memory projection tiles when the pupil samples the screens no more coarsely
        // than one screen pixel (cone factor <= 1)
        s.tiled = (tel->diameter_m / Np) / layers->screen_dx_m <= 1.0 + 1e-12 && s.n_valid > 0;
        if (s.tiled) {
            std::vector<int4> segs;
            int run = 0;
            build_segments(s.ids, g.n_sub, segment_max_count(n), segs, &run);
            s.n_segs = (int)segs.size();
            s.seg_cols = run * n;
            if ((e = upload(&s.d_segs, segs)) != cudaSuccess) {
                release(h);
                delete h;
                return cuda_fail(nullptr, e, "projection tile upload");
            }
        }
        if (gs[w].is_lgs && s.n_valid > 0) {
            const size_t kt = (size_t)s.n_valid * (2 * n - 1) * n;
            if ((e = cudaMalloc(&s.d_ktil, kt * sizeof(float2))) != cudaSuccess) {
                release(h);
                delete h;
                return cuda_fail(nullptr, e, "elongation table allocation");
            }
            KtilArgs ka;
            memset(&ka, 0, sizeof ka);
            ka.subap = s.d_ids;
            ka.ktil = s.d_ktil;
            ka.n = n;
            ka.N = g.n_fft;
            ka.n_sub = g.n_sub;
            ka.n_valid = s.n_valid;
            ka.n_na = gs[w].n_na;
            ka.D = tel->diameter_m;
            ka.dx = tel->diameter_m / Np;
            ka.pix_rad = gs[w].wavelength_m / (g.n_fft * ka.dx);
            ka.sigma_px = gs[w].spot_fwhm_rad / (2.0 * std::sqrt(2.0 * std::log(2.0))) / ka.pix_rad;
            ka.launch_x = gs[w].launch_x_m;
            ka.launch_y = gs[w].launch_y_m;
            ka.h0 = gs[w].range_m;
            for (int k = 0; k < gs[w].n_na; ++k) {
                ka.alt[k] = gs[w].na_alt_m[k];
                ka.w[k] = gs[w].na_weight[k];
            }
            if ((e = launch_ktil(ka, 0)) != cudaSuccess) {
                release(h);
                delete h;
                return cuda_fail(nullptr, e, "elongation table launch");
            }
        }
    }
    // work tables: the instance (layers, seed) and the WFS entries grouped by geometry
    {
        InstDesc &I = h->inst_host;
        memset(&I, 0, sizeof I);
        I.n_layers = h->n_layers;
        I.S = h->S;
        I.ds = h->ds;
        for (int l = 0; l < h->n_layers; ++l) {
            I.alt[l] = h->alt[l];
            I.vx[l] = h->vx[l];
            I.vy[l] = h->vy[l];
            I.x0[l] = h->x0[l];
            I.y0[l] = h->y0[l];
        }
        I.seed = seed;
        int blocks = 0;
        for (int gi = 0; gi < n_geom; ++gi) {
            SpotGroup G;
            G.geom = gi;
            G.first = (int)h->wfs_host.size();
            G.proj_base = blocks;
            G.kind = spot_kind(geom[gi]);
            for (int w = 0; w < n_gs; ++w) {
                const GsDev &s = h->gs[w];
                if (s.gs.geometry_index != gi) continue;
                const wfs_geometry &g = geom[gi];
                WfsDesc d;
                memset(&d, 0, sizeof d);
                d.inst = 0;
                d.gs_index = w;
                d.n = g.n_pix_sub;
                d.n_sub = g.n_sub;
                d.n_valid = s.n_valid;
                d.is_lgs = s.gs.is_lgs;
                d.range_m = s.gs.range_m;
                d.theta_x = s.gs.theta_x_rad;
                d.theta_y = s.gs.theta_y_rad;
                d.pupil_dx_over_ds = (tel->diameter_m / (g.n_sub * g.n_pix_sub)) / h->ds;
                d.k_phase = (float)(2.0 * M_PI / s.gs.wavelength_m);
                d.photons = (float)s.gs.photons_per_subap;
                d.read_noise = (float)s.gs.read_noise_e;
                d.subap = s.d_ids;
                d.mask = s.d_mask;
                d.fill = s.d_fill;
                d.ktil = s.d_ktil;
                d.opd_off = (long long)s.opd_off;
                d.slope_off = (long long)s.slope_off;
                d.int_off = (long long)s.int_off;
                d.det_off = (long long)s.det_off;
                d.segs = s.d_segs;
                d.n_segs = s.n_segs;
                d.tiled = s.tiled;
                d.seg_cols = s.seg_cols;
                d.launch_x = s.gs.launch_x_m;
                d.launch_y = s.gs.launch_y_m;
                d.uplink = nullptr;
                d.proj_block_begin = blocks;
                blocks += project_blocks(d);
                if (project_box_floats(d) > h->proj_box) h->proj_box = project_box_floats(d);
                merge_stage(h->proj_stage, bulk_stage_floats(d, h->S));
                d.subap_begin = G.total;
                G.total += s.n_valid;
                h->wfs_host.push_back(d);
                ++G.count;
            }
            G.proj_count = blocks - G.proj_base;
            if (G.count) h->groups.push_back(G);
        }
        h->proj_blocks = blocks;
        if ((e = cudaMalloc(&h->d_inst, sizeof(InstDesc))) != cudaSuccess ||
            (e = cudaMemcpy(h->d_inst, &h->inst_host, sizeof(InstDesc), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = upload(&h->d_wfs, h->wfs_host)) != cudaSuccess) {
            release(h);
            delete h;
            return cuda_fail(nullptr, e, "work table upload");
        }
    }
    for (int i = 1; i < n_geom; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            if (st) cudaStreamDestroy(st);
            release(h);
            delete h;
            return cuda_fail(nullptr, e, "side stream creation");
        }
        h->side.push_back(st);
        h->ev_join.push_back(ev);
    }
    if ((e = cudaEventCreateWithFlags(&h->ev_measured, cudaEventDisableTiming)) != cudaSuccess ||
        (n_geom > 1 && (e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming)) != cudaSuccess)) {
        release(h);
        delete h;
        return cuda_fail(nullptr, e, "fork event creation");
    }
    h->total_valid = (int)(slope / 2);
    h->opd_total = opd;
    h->int_total = inten;
    h->det_total = det;
    if ((e = cudaMalloc(&h->d_opd, (opd ? opd : 1) * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_E, (det ? det : 1) * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_status, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(h->d_status, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_work, 4 * sizeof(int) * (h->groups.size() + 1))) != cudaSuccess ||
        (e = cudaMemset(h->d_work, 0, 4 * sizeof(int) * (h->groups.size() + 1))) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        release(h);
        delete h;
        return cuda_fail(nullptr, e, "handle allocation");
    }
    *out = h;
    return WFS_OK;
}

wfs_status wfs_destroy(wfs_handle h) {
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    cudaDeviceSynchronize();
    if (h->loop) wfs_loop_destroy(h->loop);
    release(h);
    delete h;
    return WFS_OK;
}

wfs_status wfs_measure(wfs_handle h, const float *screens, double t_s, float *slopes_out, void *stream) {
    const NvtxRange nvtx_range("wfs_measure");
    return measure_impl(h, screens, t_s, slopes_out, nullptr, (cudaStream_t)stream);
}

wfs_status wfs_measure_stages(wfs_handle h, const float *screens, double t_s, float *slopes_out,
                              const wfs_stage_out *stages, void *stream) {
    const NvtxRange nvtx_range("wfs_measure_stages");
    return measure_impl(h, screens, t_s, slopes_out, stages, (cudaStream_t)stream);
}

namespace {

// A run of whole rows of one layer copied host -> device: offset of its first element, rows.
struct ScreenRows {
    size_t off;
    int rows;
};

// The rows of the turbulent screens that a frame at time t reads (the host-buffer path copies
// only those).  Per layer, the union over the guide stars of the rows of the projected pupil
// square at every cone scale the star's model uses (1 for an NGS; 1 - h/range for an LGS, and
// 1 - h/h_s for each sodium slice of the per-slice model) and of the LGS uplink beam's disc,
// each widened by the bilinear tap and four rows of margin for rounding; as runs of rows (mod S,
// runs closer than 64 rows merged).  Whole rows are contiguous, so each run is one linear copy
// (rectangles of part rows went through the copy engines at a quarter of the linear rate).  The
// coordinates are the projection's and the uplink's (layer offsets in FP64).
void screen_rows(const wfs_ctx *h, double t, std::vector<ScreenRows> &out) {
    const int S = h->S;
    out.clear();
    std::vector<uint8_t> mr(S);
    std::vector<std::pair<int, int>> rr;
    auto mark = [S](std::vector<uint8_t> &m, double lo, double hi) {
        const long long a = (long long)std::floor(lo) - 4, b = (long long)std::floor(hi) + 5;
        if (b - a + 1 >= S) {
            std::fill(m.begin(), m.end(), (uint8_t)1);
            return;
        }
        for (long long i = a; i <= b; ++i) m[(size_t)(((i % S) + S) % S)] = 1;
    };
    auto runs = [S](const std::vector<uint8_t> &m, std::vector<std::pair<int, int>> &r) {
        r.clear();
        for (int i = 0; i < S;) {
            if (!m[i]) {
                ++i;
                continue;
            }
            int j = i;
            while (j < S && m[j]) ++j;
            if (!r.empty() && i - (r.back().first + r.back().second) <= 64)
                r.back().second = j - r.back().first;
            else
                r.push_back({i, j - i});
            i = j;
        }
    };
    for (int l = 0; l < h->n_layers; ++l) {
        std::fill(mr.begin(), mr.end(), (uint8_t)0);
        const double hl = h->alt[l], sy = h->y0[l] + h->vy[l] * t;
        for (const GsDev &G : h->gs) {
            const wfs_guide_star &g = G.gs;
            const wfs_geometry &geo = h->geoms[g.geometry_index].g;
            const int Np = geo.n_sub * geo.n_pix_sub;
            const double pdx = (h->tel.diameter_m / Np) / h->ds;  // pupil pitch in screen pixels
            const double ov = 0.5 * S + (g.theta_y_rad * hl - sy) / h->ds;
            auto pupil = [&](double c) {
                const double half = std::fabs(c) * pdx * 0.5 * (Np - 1);
                mark(mr, ov - half, ov + half);
            };
            if (!g.is_lgs) {
                pupil(1.0);
                continue;
            }
            pupil(1.0 - hl / g.range_m);
            if (h->per_slice)
                for (double hs : G.na_alt) pupil(1.0 - hl / hs);
            if (G.up_diam > 0.0 && hl < g.range_m) {
                const double cy = g.launch_y_m * (1.0 - hl / g.range_m) + g.theta_y_rad * hl;
                const double vv = 0.5 * S + (cy - sy) / h->ds, r = 0.5 * G.up_diam / h->ds;
                mark(mr, vv - r, vv + r);
            }
        }
        runs(mr, rr);
        for (const auto &a : rr) out.push_back({(size_t)l * S * S + (size_t)a.first * S, a.second});
    }
}

// The rectangles of the turbulent screens a frame at time t reads, as row bands for the gather
// kernel: per layer, each guide star's projected pupil square at every cone scale its model uses
// and its LGS uplink beam's disc (the coordinates of screen_rows), widened by the bilinear tap and
// four pixels of margin; the rows cut at the rectangles' row boundaries, and each band copies one
// column interval, the union of the rectangles covering it, split at the periodic edges.  Columns
// in 16-byte units.  Returns false where a rectangle spans the whole screen (the caller then
// copies rows).
bool screen_rects(const wfs_ctx *h, double t, std::vector<HostRowTask> &out) {
    const int S = h->S;
    out.clear();
    if (S % 4) return false;
    struct Rect {
        long long r0, r1, c0, c1;  // inclusive, unwrapped
    };
    std::vector<Rect> rects;
    std::vector<long long> cuts;
    for (int l = 0; l < h->n_layers; ++l) {
        rects.clear();
        const double hl = h->alt[l];
        const double sx = h->x0[l] + h->vx[l] * t, sy = h->y0[l] + h->vy[l] * t;
        auto add = [&](double cu, double cv, double hu, double hv) {
            rects.push_back({(long long)std::floor(cv - hv) - 4, (long long)std::floor(cv + hv) + 5,
                             (long long)std::floor(cu - hu) - 4, (long long)std::floor(cu + hu) + 5});
        };
        for (const GsDev &G : h->gs) {
            const wfs_guide_star &g = G.gs;
            const wfs_geometry &geo = h->geoms[g.geometry_index].g;
            const int Np = geo.n_sub * geo.n_pix_sub;
            const double pdx = (h->tel.diameter_m / Np) / h->ds;
            const double ou = 0.5 * S + (g.theta_x_rad * hl - sx) / h->ds;
            const double ov = 0.5 * S + (g.theta_y_rad * hl - sy) / h->ds;
            auto pupil = [&](double c) {
                const double half = std::fabs(c) * pdx * 0.5 * (Np - 1);
                add(ou, ov, half, half);
            };
            if (!g.is_lgs) {
                pupil(1.0);
                continue;
            }
            pupil(1.0 - hl / g.range_m);
            if (h->per_slice)
                for (double hs : G.na_alt) pupil(1.0 - hl / hs);
            if (G.up_diam > 0.0 && hl < g.range_m) {
                const double cx = g.launch_x_m * (1.0 - hl / g.range_m) + g.theta_x_rad * hl;
                const double cy = g.launch_y_m * (1.0 - hl / g.range_m) + g.theta_y_rad * hl;
                const double r = 0.5 * G.up_diam / h->ds;
                add(0.5 * S + (cx - sx) / h->ds, 0.5 * S + (cy - sy) / h->ds, r, r);
            }
        }
        // rows wrapped into [0, S): a rectangle crossing the edge splits in two
        std::vector<Rect> w;
        for (const Rect &r : rects) {
            if (r.r1 - r.r0 + 1 >= S || r.c1 - r.c0 + 1 >= S) return false;
            const long long sh = ((r.r0 % S) + S) % S - r.r0;
            const Rect q{r.r0 + sh, r.r1 + sh, r.c0, r.c1};
            if (q.r1 < S) {
                w.push_back(q);
            } else {
                w.push_back({q.r0, S - 1, q.c0, q.c1});
                w.push_back({0, q.r1 - S, q.c0, q.c1});
            }
        }
        cuts.clear();
        for (const Rect &r : w) {
            cuts.push_back(r.r0);
            cuts.push_back(r.r1 + 1);
        }
        std::sort(cuts.begin(), cuts.end());
        cuts.erase(std::unique(cuts.begin(), cuts.end()), cuts.end());
        for (size_t k = 0; k + 1 < cuts.size(); ++k) {
            const long long a = cuts[k], b = cuts[k + 1];  // rows [a, b)
            long long c0 = 0, c1 = -1;
            for (const Rect &r : w)
                if (r.r0 <= a && r.r1 >= b - 1) {
                    if (c1 < c0) {
                        c0 = r.c0;
                        c1 = r.c1;
                    } else {
                        c0 = std::min(c0, r.c0);
                        c1 = std::max(c1, r.c1);
                    }
                }
            if (c1 < c0) continue;
            if (c1 - c0 + 1 >= S) {
                c0 = 0;
                c1 = S - 1;
            }
            // columns wrapped into [0, S), in 16-byte units
            const long long sh = ((c0 % S) + S) % S - c0;
            const long long u0 = c0 + sh, u1 = c1 + sh;
            auto emit = [&](long long x0, long long x1) {
                const int q0 = (int)(x0 / 4), q1 = (int)(x1 / 4);
                const int begin = out.empty() ? 0 : out.back().row_begin + out.back().rows;
                out.push_back({(long long)l * S + a, (int)(b - a), q0, q1 - q0 + 1, begin});
            };
            if (u1 < S) {
                emit(u0, u1);
            } else {
                emit(u0, S - 1);
                emit(0, u1 - S);
            }
        }
    }
    return true;
}

}  // namespace

wfs_status wfs_host_transfer_bytes(wfs_handle h, uint64_t *h2d_bytes, uint64_t *d2h_bytes) {
    if (!h || !h2d_bytes || !d2h_bytes) return fail(h, WFS_EINVAL, "null argument");
    *h2d_bytes = h->host_h2d;
    *d2h_bytes = h->host_d2h;
    return WFS_OK;
}

wfs_status wfs_measure_host(wfs_handle h, const float *screens_host, double t_s, float *slopes_host,
                            void *stream) {
    const NvtxRange nvtx_range("wfs_measure_host");
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    if (!screens_host || !slopes_host) return fail(h, WFS_EINVAL, "null host buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nscr = (size_t)h->n_layers * h->S * h->S;
    const size_t nsl = 2 * (size_t)h->total_valid;
    cudaError_t e;
    if (!h->d_screens_stage[0]) {
        // staging screens start as NaN (all bits set), so a read outside the uploaded parts
        // shows in the results
        for (int i = 0; i < 2; ++i)
            if ((e = cudaMalloc(&h->d_screens_stage[i], nscr * sizeof(float))) != cudaSuccess ||
                (e = cudaMemset(h->d_screens_stage[i], 0xFF, nscr * sizeof(float))) != cudaSuccess ||
                (e = cudaMalloc(&h->d_slopes_stage[i], (nsl + 1) * sizeof(float))) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&h->ev_done[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(h, e, "host-path staging allocation");
        // the uploads (and the gather kernel that reads the mapped host screens) run beside the
        // previous frame's kernels; at the device's highest stream priority their thread blocks
        // take SM room first whenever a frame kernel's blocks retire
        int prio_low = 0, prio_high = 0;
        if ((e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high)) != cudaSuccess ||
            (e = cudaStreamCreateWithPriority(&h->copy_stream, cudaStreamNonBlocking, prio_high)) != cudaSuccess)
            return cuda_fail(h, e, "host-path copy stream");
    }
    if (s != h->last_stream && cudaEventQuery(h->ev_measured) == cudaErrorNotReady)
        return fail(h, WFS_EBUSY, "handle busy on another stream (its previous measurement is still running)");
    const int i = (int)(h->host_calls & 1);
    // the staging set is free once the frame that used it two calls ago has finished
    if (h->host_calls >= 2 && (e = cudaStreamWaitEvent(h->copy_stream, h->ev_done[i], 0)) != cudaSuccess)
        return cuda_fail(h, e, "host-path wait");
    // With GBWFS_HOST_ZERO_COPY=1, screens in pinned host memory that is mapped into the device's
    // address space (pinned allocations under unified addressing) are read in place by the kernels
    // instead of copying rows first.  Off by default: on the ELT frame the projection's gathers
    // over the host link made the frame 3x slower than the row copies (25.5 against 74.3 M
    // spots/s end to end).  Anything else (pageable memory) goes through the row copies below.
    {
        const char *zc = getenv("GBWFS_HOST_ZERO_COPY");
        cudaPointerAttributes pa;
        if (zc && zc[0] == '1' && cudaPointerGetAttributes(&pa, screens_host) == cudaSuccess &&
            pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr) {
            if (h->host_calls >= 2 && (e = cudaStreamWaitEvent(s, h->ev_done[i], 0)) != cudaSuccess)
                return cuda_fail(h, e, "host-path wait");
            h->screens_host_mapped = true;
            wfs_status st = measure_impl(h, static_cast<const float *>(pa.devicePointer), t_s, h->d_slopes_stage[i],
                                         nullptr, s);
            h->screens_host_mapped = false;
            if (st != WFS_OK) return st;
            if ((e = cudaMemcpyAsync(slopes_host, h->d_slopes_stage[i], nsl * sizeof(float), cudaMemcpyDeviceToHost,
                                     s)) != cudaSuccess ||
                (e = cudaEventRecord(h->ev_done[i], s)) != cudaSuccess)
                return cuda_fail(h, e, "slope download");
            ++h->host_calls;
            h->host_h2d = 0;  // nothing copied: the kernels read the screens in place
            h->host_d2h = nsl * sizeof(float);
            return WFS_OK;
        }
        cudaGetLastError();  // a failed attribute query of a pageable pointer leaves no error behind
    }
    // Screens in pinned host memory mapped into the device's address space: a gather kernel on
    // the copy stream copies the rectangles the frame reads (GBWFS_HOST_RECTS=0 turns this off;
    // pageable memory takes the row copies below).
    {
        const char *hr = getenv("GBWFS_HOST_RECTS");
        cudaPointerAttributes pa;
        std::vector<HostRowTask> tasks;
        if (!(hr && hr[0] == '0') && cudaPointerGetAttributes(&pa, screens_host) == cudaSuccess &&
            pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr &&
            (reinterpret_cast<uintptr_t>(pa.devicePointer) & 15) == 0 && screen_rects(h, t_s, tasks) &&
            !tasks.empty()) {
            if ((int)tasks.size() > h->task_cap) {
                const int cap = (int)tasks.size() * 2;
                for (int k = 0; k < 2; ++k) {
                    // the tables of both sets are free: their copies completed with the frames
                    // that used them
                    if (h->host_calls > 0 && (e = cudaEventSynchronize(h->ev_copied[k])) != cudaSuccess)
                        return cuda_fail(h, e, "host-path task table");
                    if (h->h_tasks[k]) cudaFreeHost(h->h_tasks[k]);
                    cudaFree(h->d_tasks[k]);
                    h->h_tasks[k] = nullptr;
                    h->d_tasks[k] = nullptr;
                    if ((e = cudaMallocHost(&h->h_tasks[k], cap * sizeof(HostRowTask))) != cudaSuccess ||
                        (e = cudaMalloc(&h->d_tasks[k], cap * sizeof(HostRowTask))) != cudaSuccess)
                        return cuda_fail(h, e, "host-path task table");
                }
                h->task_cap = cap;
            }
            // this set's host table was last read by the copy two calls ago
            if (h->host_calls >= 2 && (e = cudaEventSynchronize(h->ev_copied[i])) != cudaSuccess)
                return cuda_fail(h, e, "host-path task table");
            long long rows = 0, f4 = 0;
            for (const HostRowTask &k : tasks) {
                rows += k.rows;
                f4 += (long long)k.rows * k.c4_count;
            }
            memcpy(h->h_tasks[i], tasks.data(), tasks.size() * sizeof(HostRowTask));
            if ((e = cudaMemcpyAsync(h->d_tasks[i], h->h_tasks[i], tasks.size() * sizeof(HostRowTask),
                                     cudaMemcpyHostToDevice, h->copy_stream)) != cudaSuccess ||
                (e = launch_host_gather(static_cast<const float *>(pa.devicePointer), h->d_screens_stage[i],
                                        h->S, h->d_tasks[i], (int)tasks.size(), (int)rows, (long long)nscr,
                                        h->copy_stream)) !=
                    cudaSuccess ||
                (e = cudaEventRecord(h->ev_copied[i], h->copy_stream)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, h->ev_copied[i], 0)) != cudaSuccess)
                return cuda_fail(h, e, "screen gather");
            wfs_status st = measure_impl(h, h->d_screens_stage[i], t_s, h->d_slopes_stage[i], nullptr, s);
            if (st != WFS_OK) return st;
            if ((e = cudaMemcpyAsync(slopes_host, h->d_slopes_stage[i], nsl * sizeof(float), cudaMemcpyDeviceToHost,
                                     s)) != cudaSuccess ||
                (e = cudaEventRecord(h->ev_done[i], s)) != cudaSuccess)
                return cuda_fail(h, e, "slope download");
            ++h->host_calls;
            h->host_h2d = (unsigned long long)f4 * 16;
            h->host_d2h = nsl * sizeof(float);
            return WFS_OK;
        }
        cudaGetLastError();
    }
    // the rows of the screens this frame reads; the whole set when they cover most of it
    std::vector<ScreenRows> runs;
    screen_rows(h, t_s, runs);
    size_t part = 0;
    for (const ScreenRows &r : runs) part += (size_t)r.rows * h->S;
    if (part * 10 >= nscr * 9) {
        part = nscr;
        e = cudaMemcpyAsync(h->d_screens_stage[i], screens_host, nscr * sizeof(float), cudaMemcpyHostToDevice,
                            h->copy_stream);
    } else {
        e = cudaSuccess;
        for (size_t k = 0; k < runs.size() && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(h->d_screens_stage[i] + runs[k].off, screens_host + runs[k].off,
                                (size_t)runs[k].rows * h->S * sizeof(float), cudaMemcpyHostToDevice, h->copy_stream);
    }
    if (e != cudaSuccess || (e = cudaEventRecord(h->ev_copied[i], h->copy_stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, h->ev_copied[i], 0)) != cudaSuccess)
        return cuda_fail(h, e, "screen upload");
    wfs_status st = measure_impl(h, h->d_screens_stage[i], t_s, h->d_slopes_stage[i], nullptr, s);
    if (st != WFS_OK) return st;
    if ((e = cudaMemcpyAsync(slopes_host, h->d_slopes_stage[i], nsl * sizeof(float), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaEventRecord(h->ev_done[i], s)) != cudaSuccess)
        return cuda_fail(h, e, "slope download");
    ++h->host_calls;
    h->host_h2d = part * sizeof(float);
    h->host_d2h = nsl * sizeof(float);
    return WFS_OK;
}

wfs_status wfs_timing_enable(wfs_handle h, int enable) {
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    h->timing = enable != 0;
    return WFS_OK;
}

wfs_status wfs_timing_read(wfs_handle h, int max, wfs_kernel_time *out, int *n_out) {
    if (!h || !n_out || (max > 0 && !out)) return fail(h, WFS_EINVAL, "bad timing arguments");
    std::vector<double> tot(h->kinds.size(), 0.0);
    std::vector<int> cnt(h->kinds.size(), 0);
    for (size_t i = 0; i < h->ev_used; ++i) {
        cudaError_t e = cudaEventSynchronize(h->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(h, e, "timing event");
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(h, e, "timing elapsed");
        tot[h->ev_kind[i]] += ms;
        cnt[h->ev_kind[i]] += 1;
    }
    int k = 0;
    for (size_t i = 0; i < h->kinds.size(); ++i) {
        if (!cnt[i]) continue;
        if (k < max) {
            memset(&out[k], 0, sizeof(wfs_kernel_time));
            strncpy(out[k].name, h->kinds[i].c_str(), sizeof(out[k].name) - 1);
            out[k].launches = cnt[i];
            out[k].total_ms = tot[i];
        }
        ++k;
    }
    *n_out = k;
    const bool over = h->ev_overflow;
    h->ev_used = 0;
    h->ev_overflow = false;
    if (over) return fail(h, WFS_EBUSY, "more timed launches than the event pool holds");
    return WFS_OK;
}

wfs_status wfs_set_noise(wfs_handle h, int enable) {
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    h->noise = enable ? 1 : 0;
    return WFS_OK;
}

wfs_status wfs_num_valid(wfs_handle h, int gs, int *n) {
    if (!h || !n) return fail(h, WFS_EINVAL, "null argument");
    if (gs < 0 || gs >= (int)h->gs.size()) return fail(h, WFS_EINVAL, "guide star index out of range");
    *n = h->gs[gs].n_valid;
    return WFS_OK;
}

wfs_status wfs_total_valid(wfs_handle h, int *n) {
    if (!h || !n) return fail(h, WFS_EINVAL, "null argument");
    *n = h->total_valid;
    return WFS_OK;
}

wfs_status wfs_valid_map(wfs_handle h, int gs, int32_t *host_idx) {
    if (!h || !host_idx) return fail(h, WFS_EINVAL, "null argument");
    if (gs < 0 || gs >= (int)h->gs.size()) return fail(h, WFS_EINVAL, "guide star index out of range");
    const auto &ids = h->gs[gs].ids;
    if (!ids.empty()) memcpy(host_idx, ids.data(), ids.size() * sizeof(int32_t));
    return WFS_OK;
}

wfs_status wfs_layout(wfs_handle h, int gs, wfs_layout_info *out) {
    if (!h || !out) return fail(h, WFS_EINVAL, "null argument");
    if (gs < 0 || gs >= (int)h->gs.size()) return fail(h, WFS_EINVAL, "guide star index out of range");
    const GsDev &s = h->gs[gs];
    const wfs_geometry &g = h->geoms[s.gs.geometry_index].g;
    out->n_valid = s.n_valid;
    out->n = g.n_pix_sub;
    out->n_fft = g.n_fft;
    out->n_det = g.n_det;
    out->is_lgs = s.gs.is_lgs;
    out->slope_offset = s.slope_off;
    out->opd_offset = s.opd_off;
    out->intensity_offset = s.int_off;
    out->det_offset = s.det_off;
    return WFS_OK;
}

wfs_status wfs_sync_status(wfs_handle h) {
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    cudaError_t e = cudaStreamSynchronize(h->last_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronise");
    int v = 0;
    if ((e = cudaMemcpy(&v, h->d_status, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(h, e, "status read");
    if (v != 0) {
        cudaMemset(h->d_status, 0, sizeof(int));
        return fail(h, (wfs_status)v, "device reported status " + std::to_string(v));
    }
    return WFS_OK;
}

wfs_status wfs_check_bounded_wait(wfs_handle h, int polls, void *stream) {
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    if (polls < 1 || polls > (1 << 24)) return fail(h, WFS_EINVAL, "polls must be in [1, 2^24]");
    h->last_stream = (cudaStream_t)stream;
    cudaError_t e = launch_wait_check(h->d_status, polls, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "wait check launch");
    return WFS_OK;
}

wfs_status wfs_noise_apply(const float *expected, int n, float read_noise_e, uint64_t seed,
                           uint32_t wfs_index, double t_s, uint32_t pixel0, float *counts, void *stream) {
    const NvtxRange nvtx_range("wfs_noise_apply");
    if (!expected || !counts || n < 0) return fail(nullptr, WFS_EINVAL, "bad noise arguments");
    if (wfs_index >= (1u << 16)) return fail(nullptr, WFS_EINVAL, "wfs_index must be < 65536");
    if (!(read_noise_e >= 0) || !is_finite(t_s)) return fail(nullptr, WFS_EINVAL, "bad read noise or time");
    cudaError_t e = launch_noise(expected, n, read_noise_e, seed, wfs_index, t_s, pixel0, counts,
                                 (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "noise launch");
    return WFS_OK;
}

namespace {

void batch_free(wfs_batch b) {
    for (auto &sl : b->slots) {
        if (sl.copied) cudaEventDestroy(sl.copied);
        cudaFreeHost(sl.h);
        cudaFree(sl.d);
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_inst);
    cudaFree(b->d_wfs);
    cudaFree(b->d_work);
    delete b->pa;
    for (ShArgs *p : b->sa) delete p;
    delete b;
}

void batch_drop_graph(wfs_batch b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->proj_node = nullptr;
    b->spot_nodes.clear();
    b->noise_nodes.clear();
}

// Per-call parameters of every node.
wfs_status batch_fill(wfs_batch b, const float *const *screens, const double *t, float *const *slopes) {
    const int n = (int)b->hs.size();
    for (int i = 0; i < n; ++i) {
        if (!screens[i] || !slopes[i] || !is_finite(t[i]))
            return fail(nullptr, WFS_EINVAL, "batch: null buffer or non-finite time for instance " + std::to_string(i));
        InstDyn &d = b->pa->dyn[i];
        memset(&d, 0, sizeof d);
        d.screens = screens[i];
        d.opd = b->hs[i]->d_opd;
        d.slopes = slopes[i];
        d.t = t[i];
        d.noise = b->hs[i]->noise;
        d.st_E = b->hs[i]->d_E;
        b->hs[i]->last_stream = nullptr;
    }
    bool aligned = true;
    for (int i = 0; i < n; ++i) aligned = aligned && aligned16(screens[i]);
    b->pa->stage_cap = (b->proj_stage > 0 && aligned) ? b->proj_stage : 0;
    for (size_t c = 0; c < b->classes.size(); ++c) {
        ShArgs &a = *b->sa[c];
        memcpy(a.dyn, b->pa->dyn, sizeof(InstDyn) * n);
        a.grid_cap = b->classes[c].grid_cap;
        a.cta_warps = b->classes[c].cta_warps;
    }
    return WFS_OK;
}

cudaError_t batch_build_graph(wfs_batch b) {
    cudaError_t e;
    if ((e = cudaGraphCreate(&b->graph, 0)) != cudaSuccess) return e;
    b->graph_stage = b->pa->stage_cap;
    LaunchShape ps;
    project_launch_shape(*b->pa, b->proj_blocks, &ps);
    void *pargs[] = {(void *)b->pa};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)ps.func;
    kp.gridDim = ps.grid;
    kp.blockDim = ps.block;
    kp.sharedMemBytes = (unsigned)ps.smem;
    kp.kernelParams = pargs;
    if ((e = cudaGraphAddKernelNode(&b->proj_node, b->graph, nullptr, 0, &kp)) != cudaSuccess) return e;
    b->spot_nodes.assign(b->classes.size(), nullptr);
    b->noise_nodes.assign(b->classes.size(), nullptr);
    for (size_t c = 0; c < b->classes.size(); ++c) {
        if (b->classes[c].total <= 0) continue;
        LaunchShape sh;
        if ((e = spot_launch_shape(b->classes[c].kind, *b->sa[c], &sh)) != cudaSuccess) return e;
        void *sargs[] = {(void *)b->sa[c]};
        kp = cudaKernelNodeParams{};
        kp.func = (void *)sh.func;
        kp.gridDim = sh.grid;
        kp.blockDim = sh.block;
        kp.sharedMemBytes = (unsigned)sh.smem;
        kp.kernelParams = sargs;
        if ((e = cudaGraphAddKernelNode(&b->spot_nodes[c], b->graph, &b->proj_node, 1, &kp)) != cudaSuccess) return e;
        if (!b->sa[c]->split_noise) continue;
        if ((e = noise_cog_launch_shape(*b->sa[c], &sh)) != cudaSuccess) return e;
        kp = cudaKernelNodeParams{};
        kp.func = (void *)sh.func;
        kp.gridDim = sh.grid;
        kp.blockDim = sh.block;
        kp.sharedMemBytes = (unsigned)sh.smem;
        kp.kernelParams = sargs;
        if ((e = cudaGraphAddKernelNode(&b->noise_nodes[c], b->graph, &b->spot_nodes[c], 1, &kp)) != cudaSuccess)
            return e;
    }
    return cudaGraphInstantiate(&b->exec, b->graph, 0);
}

cudaError_t batch_update_graph(wfs_batch b) {
    cudaError_t e;
    LaunchShape ps;
    project_launch_shape(*b->pa, b->proj_blocks, &ps);
    void *pargs[] = {(void *)b->pa};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)ps.func;
    kp.gridDim = ps.grid;
    kp.blockDim = ps.block;
    kp.sharedMemBytes = (unsigned)ps.smem;
    kp.kernelParams = pargs;
    if ((e = cudaGraphExecKernelNodeSetParams(b->exec, b->proj_node, &kp)) != cudaSuccess) return e;
    for (size_t c = 0; c < b->classes.size(); ++c) {
        if (!b->spot_nodes[c]) continue;
        LaunchShape sh;
        if ((e = spot_launch_shape(b->classes[c].kind, *b->sa[c], &sh)) != cudaSuccess) return e;
        void *sargs[] = {(void *)b->sa[c]};
        kp = cudaKernelNodeParams{};
        kp.func = (void *)sh.func;
        kp.gridDim = sh.grid;
        kp.blockDim = sh.block;
        kp.sharedMemBytes = (unsigned)sh.smem;
        kp.kernelParams = sargs;
        if ((e = cudaGraphExecKernelNodeSetParams(b->exec, b->spot_nodes[c], &kp)) != cudaSuccess) return e;
        if (!b->noise_nodes[c]) continue;
        if ((e = noise_cog_launch_shape(*b->sa[c], &sh)) != cudaSuccess) return e;
        kp = cudaKernelNodeParams{};
        kp.func = (void *)sh.func;
        kp.gridDim = sh.grid;
        kp.blockDim = sh.block;
        kp.sharedMemBytes = (unsigned)sh.smem;
        kp.kernelParams = sargs;
        if ((e = cudaGraphExecKernelNodeSetParams(b->exec, b->noise_nodes[c], &kp)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t batch_launch_direct(wfs_batch b, cudaStream_t s) {
    cudaError_t e = launch_project(*b->pa, b->proj_blocks, s);
    if (e != cudaSuccess) return e;
    for (size_t c = 0; c < b->classes.size(); ++c) {
        if ((e = launch_spot(b->classes[c].kind, *b->sa[c], s)) != cudaSuccess) return e;
        if (b->sa[c]->split_noise && (e = launch_noise_cog(*b->sa[c], s, false)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---- tuning cache: lines "key grid_cap cta_warps" in the file named by GBWFS_TUNE_CACHE
std::string class_key(const BatchClass &c, int total) {
    int bucket = 1;
    while (bucket < total) bucket <<= 1;
    cudaDeviceProp p;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&p, dev);
    std::string name = p.name;
    for (char &ch : name)
        if (ch == ' ') ch = '_';
    return "kind" + std::to_string(c.kind) + "_n" + std::to_string(c.geom->g.n_pix_sub) + "_N" +
           std::to_string(c.geom->g.n_fft) + "_nd" + std::to_string(c.geom->g.n_det) + "_sub" +
           std::to_string(bucket) + "_" + name;
}

bool cache_lookup(const std::string &key, int *cap, int *warps) {
    const char *path = getenv("GBWFS_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char k[256];
    int a = 0, b = 0;
    bool found = false;
    while (fscanf(f, "%255s %d %d", k, &a, &b) == 3)
        if (key == k) {
            *cap = a;
            *warps = b;
            found = true;
        }
    fclose(f);
    return found;
}

void cache_store(const std::string &key, int cap, int warps) {
    const char *path = getenv("GBWFS_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d\n", key.c_str(), cap, warps);
    fclose(f);
}

}  // namespace

wfs_status wfs_batch_create(int n, const wfs_handle *hs, wfs_batch *out) {
    if (!out || !hs || n < 1) return fail(nullptr, WFS_EINVAL, "bad batch arguments");
    *out = nullptr;
    if (n > kMaxInstances) return fail(nullptr, WFS_EINVAL, "batch: more than 64 instances");
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return fail(nullptr, WFS_EINVAL, "null handle in batch");
        if (hs[i]->device != dev) return fail(nullptr, WFS_EINVAL, "batch handles must live on the current device");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(nullptr, WFS_EINVAL, "a handle appears twice in the batch");
        if (hs[i]->n_uplink > 0)
            return fail(nullptr, WFS_EUNSUPPORTED, "batch: a handle has the uplink tip-tilt on (not batched)");
        if (hs[i]->per_slice)
            return fail(nullptr, WFS_EUNSUPPORTED, "batch: a handle has the LGS per-slice model on (not batched)");
    }
    wfs_batch b = new wfs_batch_ctx();
    b->hs.assign(hs, hs + n);
    b->device = dev;
    // classes in order of first appearance; WFS entries of each class contiguous
    for (int i = 0; i < n; ++i)
        for (const SpotGroup &G : hs[i]->groups) {
            const wfs_geometry &g = hs[i]->geoms[G.geom].g;
            const std::string key = std::to_string(G.kind) + ":" + std::to_string(g.n_pix_sub) + ":" +
                                    std::to_string(g.n_fft) + ":" + std::to_string(g.n_det);
            size_t c = 0;
            while (c < b->classes.size() && b->classes[c].key != key) ++c;
            if (c == b->classes.size()) {
                BatchClass bc;
                bc.kind = G.kind;
                bc.geom = &hs[i]->geoms[G.geom];
                bc.key = key;
                b->classes.push_back(bc);
            }
        }
    std::vector<std::vector<WfsDesc>> per(b->classes.size());
    for (int i = 0; i < n; ++i)
        for (const SpotGroup &G : hs[i]->groups) {
            const wfs_geometry &g = hs[i]->geoms[G.geom].g;
            const std::string key = std::to_string(G.kind) + ":" + std::to_string(g.n_pix_sub) + ":" +
                                    std::to_string(g.n_fft) + ":" + std::to_string(g.n_det);
            size_t c = 0;
            while (b->classes[c].key != key) ++c;
            for (int k = 0; k < G.count; ++k) {
                WfsDesc d = hs[i]->wfs_host[G.first + k];
                d.inst = i;
                d.uplink = nullptr;  // batches measure without the uplink tip-tilt
                per[c].push_back(d);
            }
        }
    int blocks = 0;
    for (size_t c = 0; c < b->classes.size(); ++c) {
        BatchClass &bc = b->classes[c];
        bc.first = (int)b->wfs_host.size();
        for (WfsDesc d : per[c]) {
            d.subap_begin = bc.total;
            bc.total += d.n_valid;
            d.proj_block_begin = blocks;
            blocks += project_blocks(d);
            if (project_box_floats(d) > b->proj_box) b->proj_box = project_box_floats(d);
            merge_stage(b->proj_stage, bulk_stage_floats(d, hs[d.inst]->S));
            b->wfs_host.push_back(d);
            ++bc.count;
        }
        int cap = 0, warps = 0;
        if (cache_lookup(class_key(bc, bc.total), &cap, &warps)) {
            bc.grid_cap = cap;
            bc.cta_warps = warps;
        }
    }
    b->proj_blocks = blocks;
    std::vector<InstDesc> inst(n);
    for (int i = 0; i < n; ++i) inst[i] = hs[i]->inst_host;
    cudaError_t e;
    // spot counters (a pair per class, then per slot and class), then projection counters (the
    // graph's pair, then a pair per slot)
    const size_t proj_off = 2 * b->classes.size() * (1 + kBatchSlots);
    const size_t work_bytes = sizeof(int) * (proj_off + 2 * (1 + kBatchSlots) + 2);
    if ((e = upload(&b->d_inst, inst)) != cudaSuccess || (e = upload(&b->d_wfs, b->wfs_host)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_work, work_bytes)) != cudaSuccess || (e = cudaMemset(b->d_work, 0, work_bytes)) != cudaSuccess) {
        batch_free(b);
        return cuda_fail(nullptr, e, "batch table upload");
    }
    b->pa = new ProjArgs();
    memset(b->pa, 0, sizeof(ProjArgs));
    b->pa->inst = b->d_inst;
    b->pa->wfs = b->d_wfs;
    b->pa->n_wfs = (int)b->wfs_host.size();
    b->pa->n_inst = n;
    b->pa->box_cap = b->proj_box;
    b->pa->stage_cap = b->proj_stage > 0 ? b->proj_stage : 0;
    b->pa->n_blocks = b->proj_blocks;
    for (int i = 0; i < n; ++i) b->pa->max_layers = std::max(b->pa->max_layers, hs[i]->inst_host.n_layers);
    b->pa->work = b->d_work + 2 * b->classes.size() * (1 + kBatchSlots);
    b->pa->status = hs[0]->d_status;
    for (const BatchClass &bc : b->classes) {
        ShArgs *a = new ShArgs();
        memset(a, 0, sizeof(ShArgs));
        fill_geom_args(*a, *bc.geom);
        a->inst = b->d_inst;
        a->wfs = b->d_wfs + bc.first;
        a->n_wfs = bc.count;
        a->total = bc.total;
        a->status = hs[0]->d_status;
        a->n_inst = n;
        a->work = b->d_work + 2 * b->sa.size();
        a->split_noise = splits_noise(bc.kind, a->N, a->nd) ? 1 : 0;
        b->sa.push_back(a);
    }
    const char *g = getenv("GBWFS_BATCH_GRAPH");
    b->use_graph = !(g && g[0] == '0');
    *out = b;
    return WFS_OK;
}

wfs_status wfs_batch_measure(wfs_batch b, const float *const *screens, const double *t_s,
                             float *const *slopes_out, void *stream) {
    const NvtxRange nvtx_range("wfs_batch_measure");
    if (!b || !screens || !t_s || !slopes_out) return fail(nullptr, WFS_EINVAL, "bad batch arguments");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(nullptr, WFS_EINVAL, "current device differs from the batch's device");
    wfs_status st = batch_fill(b, screens, t_s, slopes_out);
    if (st != WFS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (!b->use_graph) {
        if ((e = batch_launch_direct(b, s)) != cudaSuccess) return cuda_fail(nullptr, e, "batch launch");
        return WFS_OK;
    }
    // the projection node's kernel follows the screens' alignment: a change rebuilds the graph
    if (b->exec && b->graph_stage != b->pa->stage_cap) batch_drop_graph(b);
    if (!b->exec) {
        if ((e = batch_build_graph(b)) != cudaSuccess) {
            batch_drop_graph(b);
            return cuda_fail(nullptr, e, "batch graph build");
        }
    } else if ((e = batch_update_graph(b)) != cudaSuccess) {
        return cuda_fail(nullptr, e, "batch graph update");
    }
    if ((e = cudaGraphLaunch(b->exec, s)) != cudaSuccess) return cuda_fail(nullptr, e, "batch graph launch");
    return WFS_OK;
}

wfs_status wfs_batch_measure_subset(wfs_batch b, int slot, int n_active, const int *active,
                                    const float *const *screens, const double *t_s, float *const *slopes_out,
                                    void *stream) {
    const NvtxRange nvtx_range("wfs_batch_measure_subset");
    if (!b || (n_active > 0 && (!active || !screens || !t_s || !slopes_out)) || n_active < 0)
        return fail(nullptr, WFS_EINVAL, "bad batch subset arguments");
    if (slot < 0 || slot >= kBatchSlots) return fail(nullptr, WFS_EINVAL, "batch subset slot out of range");
    const int n = (int)b->hs.size();
    if (n_active > n) return fail(nullptr, WFS_EINVAL, "more active instances than the batch holds");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(nullptr, WFS_EINVAL, "current device differs from the batch's device");
    std::vector<int> pos(n, -1);
    for (int j = 0; j < n_active; ++j) {
        const int i = active[j];
        if (i < 0 || i >= n || pos[i] >= 0) return fail(nullptr, WFS_EINVAL, "active instance out of range or repeated");
        if (!screens[j] || !slopes_out[j] || !is_finite(t_s[j]))
            return fail(nullptr, WFS_EINVAL, "batch subset: null buffer or non-finite time");
        pos[i] = j;
    }
    if (n_active == 0) return WFS_OK;
    cudaError_t e;
    if (b->slots.empty()) {
        b->slots.resize(kBatchSlots);
        const size_t cap = b->wfs_host.size() ? b->wfs_host.size() : 1;
        for (auto &sl : b->slots)
            if ((e = cudaMallocHost(&sl.h, cap * sizeof(WfsDesc))) != cudaSuccess ||
                (e = cudaMalloc(&sl.d, cap * sizeof(WfsDesc))) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(nullptr, e, "batch subset slot allocation");
    }
    auto &sl = b->slots[slot];
    // the previous upload from this slot's staging table must have been consumed
    if ((e = cudaEventSynchronize(sl.copied)) != cudaSuccess) return cuda_fail(nullptr, e, "slot wait");
    static thread_local ProjArgs pa;
    static thread_local ShArgs sa;
    memset(pa.dyn, 0, sizeof(InstDyn) * n);
    for (int i = 0; i < n; ++i)
        if (pos[i] >= 0) {
            InstDyn &d = pa.dyn[i];
            d.screens = screens[pos[i]];
            d.opd = b->hs[i]->d_opd;
            d.slopes = slopes_out[pos[i]];
            d.t = t_s[pos[i]];
            d.noise = b->hs[i]->noise;
            d.st_E = b->hs[i]->d_E;
        }
    int count = 0, blocks = 0, box = 0, stage = 0;
    bool aligned = true;
    for (int j = 0; j < n_active; ++j) aligned = aligned && aligned16(screens[j]);
    std::vector<int> cls_first(b->classes.size()), cls_count(b->classes.size()), cls_total(b->classes.size());
    for (size_t c = 0; c < b->classes.size(); ++c) {
        const BatchClass &bc = b->classes[c];
        cls_first[c] = count;
        cls_total[c] = 0;
        for (int k = 0; k < bc.count; ++k) {
            const WfsDesc &src = b->wfs_host[bc.first + k];
            if (pos[src.inst] < 0) continue;
            WfsDesc d = src;
            d.subap_begin = cls_total[c];
            cls_total[c] += d.n_valid;
            d.proj_block_begin = blocks;
            blocks += project_blocks(d);
            if (project_box_floats(d) > box) box = project_box_floats(d);
            merge_stage(stage, bulk_stage_floats(d, b->hs[src.inst]->S));
            sl.h[count++] = d;
        }
        cls_count[c] = count - cls_first[c];
    }
    if ((e = cudaMemcpyAsync(sl.d, sl.h, (size_t)count * sizeof(WfsDesc), cudaMemcpyHostToDevice,
                             (cudaStream_t)stream)) != cudaSuccess ||
        (e = cudaEventRecord(sl.copied, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(nullptr, e, "batch subset table upload");
    pa.inst = b->d_inst;
    pa.wfs = sl.d;
    pa.n_wfs = count;
    pa.block_base = 0;
    pa.max_layers = 0;
    for (size_t i = 0; i < b->hs.size(); ++i) pa.max_layers = std::max(pa.max_layers, b->hs[i]->inst_host.n_layers);
    pa.work = b->d_work + 2 * b->classes.size() * (1 + kBatchSlots) + 2 * (1 + (size_t)slot);
    pa.n_inst = n;
    pa.box_cap = box;
    pa.stage_cap = (stage > 0 && aligned) ? stage : 0;
    pa.status = b->hs[0]->d_status;
    if (blocks > 0 && (e = launch_project(pa, blocks, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(nullptr, e, "batch subset projection");
    for (size_t c = 0; c < b->classes.size(); ++c) {
        if (!cls_count[c] || !cls_total[c]) continue;
        const BatchClass &bc = b->classes[c];
        memset(&sa, 0, offsetof(ShArgs, dyn));
        fill_geom_args(sa, *bc.geom);
        sa.inst = b->d_inst;
        sa.wfs = sl.d + cls_first[c];
        sa.n_wfs = cls_count[c];
        sa.total = cls_total[c];
        sa.status = b->hs[0]->d_status;
        sa.grid_cap = bc.grid_cap;
        sa.cta_warps = bc.cta_warps;
        sa.n_inst = n;
        sa.work = b->d_work + 2 * (b->classes.size() * (1 + (size_t)slot) + c);
        sa.split_noise = splits_noise(bc.kind, sa.N, sa.nd) ? 1 : 0;
        memcpy(sa.dyn, pa.dyn, sizeof(InstDyn) * n);
        if ((e = launch_spot(bc.kind, sa, (cudaStream_t)stream)) != cudaSuccess)
            return cuda_fail(nullptr, e, "batch subset spot launch");
        if (sa.split_noise && (e = launch_noise_cog(sa, (cudaStream_t)stream, false)) != cudaSuccess)
            return cuda_fail(nullptr, e, "batch subset noise launch");
    }
    return WFS_OK;
}

wfs_status wfs_batch_tune(wfs_batch b, const float *const *screens, const double *t_s, float *const *slopes_out,
                          void *stream) {
    const NvtxRange nvtx_range("wfs_batch_tune");
    if (!b || !screens || !t_s || !slopes_out) return fail(nullptr, WFS_EINVAL, "bad batch arguments");
    wfs_status st = batch_fill(b, screens, t_s, slopes_out);
    if (st != WFS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = launch_project(*b->pa, b->proj_blocks, s)) != cudaSuccess) return cuda_fail(nullptr, e, "tune projection");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (size_t c = 0; c < b->classes.size(); ++c) {
        BatchClass &bc = b->classes[c];
        if (bc.total <= 0) continue;
        std::vector<std::pair<int, int>> cand;  // (grid cap, warps per CTA)
        if (bc.kind == kSpotN32) {
            for (int w : {4, 8})
                for (int m : {2, 4, 8, 16}) cand.push_back({152 * m * (8 / w), w});
        } else if (is_tc(bc.kind) && bc.geom->g.n_fft == 64) {
            for (int m : {1, 2}) cand.push_back({76 * m, 0});
        } else if (is_tc(bc.kind)) {
            // tile shape: two warpgroups (8 subapertures) per CTA, at most 2 CTAs per SM, or one
            // (4 subapertures) with up to 3 CTAs per SM; and the persistent grid size
            for (int m : {1, 2}) cand.push_back({152 * m, 8});
            for (int m : {1, 2, 3}) cand.push_back({152 * m, 4});
        } else {
            for (int m : {2, 4, 8, 32}) cand.push_back({152 * m, 0});
        }
        float best = 1e30f;
        std::pair<int, int> pick = cand[0];
        for (const auto &cw : cand) {
            ShArgs &a = *b->sa[c];
            a.grid_cap = cw.first;
            a.cta_warps = cw.second;
            if ((e = launch_spot(bc.kind, a, s)) != cudaSuccess) break;  // warm-up
            cudaEventRecord(e0, s);
            for (int r = 0; r < 5; ++r)
                if ((e = launch_spot(bc.kind, a, s)) != cudaSuccess) break;
            cudaEventRecord(e1, s);
            if (e != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                pick = cw;
            }
        }
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(nullptr, e, "tune launch");
        }
        bc.grid_cap = pick.first;
        bc.cta_warps = pick.second;
        b->sa[c]->grid_cap = pick.first;
        b->sa[c]->cta_warps = pick.second;
        cache_store(class_key(bc, bc.total), pick.first, pick.second);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    batch_drop_graph(b);  // the next measure captures the tuned shapes
    return WFS_OK;
}

wfs_status wfs_batch_info(wfs_batch b, int max, wfs_batch_class *out, int *n_out) {
    if (!b || !n_out || (max > 0 && !out)) return fail(nullptr, WFS_EINVAL, "bad batch arguments");
    int k = 0;
    for (const BatchClass &bc : b->classes) {
        if (k < max) {
            wfs_batch_class &o = out[k];
            o.kind = bc.kind;
            o.n_pix_sub = bc.geom->g.n_pix_sub;
            o.n_fft = bc.geom->g.n_fft;
            o.n_det = bc.geom->g.n_det;
            o.n_wfs = bc.count;
            o.n_subaps = bc.total;
            o.grid_cap = bc.grid_cap;
            o.cta_warps = bc.cta_warps;
        }
        ++k;
    }
    *n_out = k;
    return WFS_OK;
}

wfs_status wfs_batch_destroy(wfs_batch b) {
    if (!b) return fail(nullptr, WFS_EINVAL, "null batch");
    cudaDeviceSynchronize();
    batch_free(b);
    return WFS_OK;
}


wfs_status wfs_loop_create(wfs_handle h, int n_dm, const wfs_dm *dms, const float *cm, const float *gain,
                           wfs_loop *out) {
    if (!out) return fail(h, WFS_EINVAL, "null output loop pointer");
    *out = nullptr;
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    if (h->loop) return fail(h, WFS_EBUSY, "the handle already has a loop");
    if (n_dm < 1 || n_dm > kMaxDms || !dms) return fail(h, WFS_EINVAL, "n_dm must be in [1, 4] with a mirror array");
    if (!cm || !gain) return fail(h, WFS_EINVAL, "null control matrix or gain vector");
    double min_range = INFINITY;
    for (const GsDev &g : h->gs)
        if (g.gs.is_lgs) min_range = std::min(min_range, g.gs.range_m);
    long long n_modes = 0;
    for (int d = 0; d < n_dm; ++d) {
        const wfs_dm &m = dms[d];
        const std::string who = "mirror " + std::to_string(d) + ": ";
        if (m.n_act < 1 || m.n_act > 1024) return fail(h, WFS_EINVAL, who + "n_act must be in [1, 1024]");
        if (!is_finite(m.pitch_m) || !(m.pitch_m >= h->ds))
            return fail(h, WFS_EINVAL, who + "pitch_m must be at least the screen pitch");
        if (!is_finite(m.alt_m) || m.alt_m < 0 || !(m.alt_m < min_range))
            return fail(h, WFS_EINVAL, who + "alt_m must be >= 0 and below every LGS range");
        if (!(m.coupling > 0 && m.coupling < 1)) return fail(h, WFS_EINVAL, who + "coupling must be in (0, 1)");
        if (m.support < 1 || m.support > kMaxDmSupport) return fail(h, WFS_EINVAL, who + "support must be in [1, 8]");
        if (m.n_modes < 1 || !m.m2a) return fail(h, WFS_EINVAL, who + "n_modes must be >= 1 with a modal base");
        n_modes += m.n_modes;
    }
    if (n_modes > (1 << 24)) return fail(h, WFS_EINVAL, "more than 2^24 modes");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != h->device) return fail(h, WFS_EINVAL, "current device differs from the handle's device");

    wfs_loop lp = new wfs_loop_ctx;
    lp->h = h;
    lp->n_modes = (int)n_modes;
    lp->n_slopes = 2 * h->total_valid;
    lp->cm = cm;
    lp->gain = gain;
    const size_t SS = (size_t)h->S * h->S;
    cudaError_t e;
    auto bail = [&](cudaError_t err, const char *what) {
        loop_free(lp);
        return cuda_fail(h, err, what);
    };
    if ((e = cudaMalloc(&lp->coeffs, sizeof(float) * n_modes)) != cudaSuccess) return bail(e, "coefficients");
    if ((e = cudaMalloc(&lp->layers, sizeof(float) * SS * n_dm)) != cudaSuccess) return bail(e, "mirror layers");
    if ((e = cudaMemset(lp->coeffs, 0, sizeof(float) * n_modes)) != cudaSuccess ||
        (e = cudaMemset(lp->layers, 0, sizeof(float) * SS * n_dm)) != cudaSuccess)
        return bail(e, "loop buffers");
    if ((e = cudaEventCreateWithFlags(&lp->ev_done, cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");
    int mode0 = 0;
    for (int d = 0; d < n_dm; ++d) {
        LoopDm M;
        M.d = dms[d];
        M.mode0 = mode0;
        mode0 += M.d.n_modes;
        // pixels (i, j) whose distance to the nearest actuator along x or y is below the
        // support: |(j - S/2) ds| < (c + R) p, clipped to the grid
        const double reach = (0.5 * (M.d.n_act - 1) + M.d.support) * M.d.pitch_m / h->ds;
        const long long lo = std::max(0LL, (long long)std::floor(0.5 * h->S - reach));
        const long long hi = std::min((long long)h->S - 1, (long long)std::ceil(0.5 * h->S + reach));
        M.x0 = M.y0 = (int)lo;
        M.w = M.h = hi >= lo ? (int)(hi - lo + 1) : 0;
        const size_t na = (size_t)M.d.n_act * M.d.n_act;
        if ((e = cudaMalloc(&M.act, sizeof(float) * na)) != cudaSuccess ||
            (e = cudaMemset(M.act, 0, sizeof(float) * na)) != cudaSuccess) {
            if (M.act) cudaFree(M.act);
            return bail(e, "actuator commands");
        }
        lp->dms.push_back(M);
    }
    // the mirrors are layers n_layers .. n_layers + n_dm - 1 of the projection: no wind, no offset
    for (int d = 0; d < n_dm; ++d) {
        const int l = h->inst_host.n_layers + d;
        h->inst_host.alt[l] = dms[d].alt_m;
        h->inst_host.vx[l] = h->inst_host.vy[l] = 0.0;
        h->inst_host.x0[l] = h->inst_host.y0[l] = 0.0;
    }
    if ((e = cudaMemcpy(h->d_inst, &h->inst_host, sizeof(InstDesc), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "layer table");
    if (refresh_slices(h) != WFS_OK) {
        loop_free(lp);
        return WFS_ECUDA;
    }
    h->loop = lp;
    *out = lp;
    return WFS_OK;
}

wfs_status wfs_loop_step(wfs_loop lp, const float *screens, double t_s, float *slopes_out, void *stream) {
    const NvtxRange nvtx_range("wfs_loop_step");
    if (!lp) return fail(nullptr, WFS_EINVAL, "null loop");
    wfs_handle h = lp->h;
    const cudaStream_t s = (cudaStream_t)stream;
    if (loop_busy(lp, s)) return fail(h, WFS_EBUSY, "loop busy on another stream (its previous step is still running)");
    wfs_status st = measure_impl(h, screens, t_s, slopes_out, nullptr, s, lp->layers, (int)lp->dms.size());
    if (st != WFS_OK) return st;
    lp->last_stream = s;
    // the integrator: c += gain * (cm s)
    GemvArgs g{lp->cm, lp->n_modes, lp->n_slopes, slopes_out, nullptr, lp->gain, lp->coeffs};
    long sl = timed_begin(h, "reconstruct", s);
    cudaError_t e = launch_gemv(g, s);
    timed_end(h, sl, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "reconstruction launch");
    if ((st = loop_rebuild(lp, s)) != WFS_OK) return st;
    if ((e = cudaEventRecord(lp->ev_done, s)) != cudaSuccess) return cuda_fail(h, e, "completion event");
    return WFS_OK;
}

wfs_status wfs_loop_set_coeffs(wfs_loop lp, const float *coeffs, void *stream) {
    if (!lp) return fail(nullptr, WFS_EINVAL, "null loop");
    wfs_handle h = lp->h;
    const cudaStream_t s = (cudaStream_t)stream;
    if (loop_busy(lp, s)) return fail(h, WFS_EBUSY, "loop busy on another stream");
    lp->last_stream = s;
    const size_t bytes = sizeof(float) * lp->n_modes;
    cudaError_t e = coeffs ? cudaMemcpyAsync(lp->coeffs, coeffs, bytes, cudaMemcpyDeviceToDevice, s)
                           : cudaMemsetAsync(lp->coeffs, 0, bytes, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "coefficients");
    wfs_status st = loop_rebuild(lp, s);
    if (st != WFS_OK) return st;
    if ((e = cudaEventRecord(lp->ev_done, s)) != cudaSuccess) return cuda_fail(h, e, "completion event");
    return WFS_OK;
}

wfs_status wfs_loop_get_coeffs(wfs_loop lp, float *coeffs_out, void *stream) {
    if (!lp || !coeffs_out) return fail(lp ? lp->h : nullptr, WFS_EINVAL, "null loop or output");
    cudaError_t e = cudaMemcpyAsync(coeffs_out, lp->coeffs, sizeof(float) * lp->n_modes, cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? WFS_OK : cuda_fail(lp->h, e, "coefficients");
}

wfs_status wfs_loop_get_layer(wfs_loop lp, int d, float *layer_out, void *stream) {
    if (!lp || !layer_out || d < 0 || d >= (int)lp->dms.size())
        return fail(lp ? lp->h : nullptr, WFS_EINVAL, "bad loop, mirror index or output");
    const size_t SS = (size_t)lp->h->S * lp->h->S;
    cudaError_t e = cudaMemcpyAsync(layer_out, lp->layers + d * SS, sizeof(float) * SS, cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? WFS_OK : cuda_fail(lp->h, e, "mirror layer");
}

wfs_status wfs_loop_destroy(wfs_loop lp) {
    if (!lp) return fail(nullptr, WFS_EINVAL, "null loop");
    cudaEventSynchronize(lp->ev_done);
    lp->h->loop = nullptr;
    loop_free(lp);
    return WFS_OK;
}


wfs_status wfs_loop_calibrate(wfs_loop lp, int gs, double amplitude, float *im_out, void *stream) {
    const NvtxRange nvtx_range("wfs_loop_calibrate");
    if (!lp) return fail(nullptr, WFS_EINVAL, "null loop");
    wfs_handle h = lp->h;
    if (gs < 0 || gs >= (int)h->gs.size()) return fail(h, WFS_EINVAL, "guide star index out of range");
    if (!is_finite(amplitude) || amplitude == 0.0) return fail(h, WFS_EINVAL, "amplitude must be finite and non-zero");
    if (!im_out) return fail(h, WFS_EINVAL, "null output");
    const cudaStream_t s = (cudaStream_t)stream;
    if (loop_busy(lp, s)) return fail(h, WFS_EBUSY, "loop busy on another stream");
    if (h->per_slice) return fail(h, WFS_EUNSUPPORTED, "calibration with the LGS per-slice model is not built");
    wfs_status st = calib_prepare(lp, gs);
    if (st != WFS_OK) return st;
    lp->last_stream = s;
    CalibScratch &c = lp->cal;
    const SpotGroup &G = h->groups[c.group];
    const size_t SS = (size_t)h->S * h->S;
    const int n_slopes = 2 * c.nv;
    const int per_chunk = kMaxInstances / 2;
    static thread_local DmLayerBatch batch;
    static thread_local ProjArgs pa;
    static thread_local ShArgs sa;
    cudaError_t e;
    for (size_t d = 0; d < lp->dms.size(); ++d) {
        const LoopDm &M = lp->dms[d];
        if (c.cur_dm != (int)d) {  // other windows: clear what the previous mirror left
            if ((e = cudaMemsetAsync(c.layers, 0, sizeof(float) * SS * kMaxInstances, s)) != cudaSuccess)
                return cuda_fail(h, e, "calibration layers");
            c.cur_dm = (int)d;
        }
        for (int m0 = 0; m0 < M.d.n_modes; m0 += per_chunk) {
            const int K = std::min(per_chunk, M.d.n_modes - m0), ni = 2 * K;
            // instance 2k: +amplitude of mode m0 + k in the beam (coefficient -amplitude), 2k + 1: -amplitude
            batch.n = ni;
            for (int i = 0; i < ni; ++i)
                batch.l[i] = dm_layer_args(h, M, M.d.m2a + m0 + i / 2, M.d.n_modes,
                                           (float)((i & 1) ? amplitude : -amplitude), c.layers + i * SS);
            long sl = timed_begin(h, "dm_layer", s);
            e = launch_dm_layers(batch, s);
            timed_end(h, sl, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "calibration layers");
            InstDyn dyn;
            memset(&dyn, 0, sizeof dyn);
            dyn.n_dm = 1;
            pa.inst = c.d_inst + d * kMaxInstances;
            pa.wfs = c.d_wfs;
            pa.n_wfs = ni;
            pa.n_inst = ni;
            pa.box_cap = h->proj_box;
            pa.stage_cap = h->proj_stage > 0 ? h->proj_stage : 0;
            pa.block_base = 0;
            pa.max_layers = 1;
            pa.work = c.work;
            pa.status = h->d_status;
            for (int i = 0; i < ni; ++i) {
                dyn.dm = c.layers + i * SS;
                dyn.opd = c.opd + i * c.opd_stride;
                dyn.slopes = c.slopes + (size_t)i * n_slopes;
                dyn.st_E = c.E + i * c.det_stride;
                pa.dyn[i] = dyn;
            }
            sl = timed_begin(h, "project", s);
            e = launch_project(pa, ni * c.blocks_per_wfs, s);
            timed_end(h, sl, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "calibration projection");
            memset(&sa, 0, offsetof(ShArgs, dyn));
            fill_geom_args(sa, h->geoms[c.geom]);
            sa.inst = pa.inst;
            sa.wfs = c.d_wfs;
            sa.n_wfs = ni;
            sa.total = ni * c.nv;
            sa.status = h->d_status;
            sa.grid_cap = G.grid_cap;
            sa.cta_warps = G.cta_warps;
            sa.n_inst = ni;
            sa.work = c.work + 2;
            sa.project = 0;
            sa.split_noise = splits_noise(c.kind, sa.N, sa.nd) ? 1 : 0;
            memcpy(sa.dyn, pa.dyn, sizeof(InstDyn) * ni);
            sl = timed_begin(h, kind_name(c.kind) + std::to_string(sa.N), s);
            e = launch_spot(c.kind, sa, s, !h->timing);
            timed_end(h, sl, s);
            if (e == cudaSuccess && sa.split_noise) {
                sl = timed_begin(h, "noise_cog", s);
                e = launch_noise_cog(sa, s, !h->timing);
                timed_end(h, sl, s);
            }
            if (e != cudaSuccess) return cuda_fail(h, e, "calibration spot launch");
            sl = timed_begin(h, "push_pull_rows", s);
            e = launch_push_pull_rows(c.slopes, K, n_slopes, (float)(0.5 / amplitude),
                                      im_out + (size_t)(M.mode0 + m0) * n_slopes, s);
            timed_end(h, sl, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "interaction rows");
        }
    }
    if ((e = cudaEventRecord(lp->ev_done, s)) != cudaSuccess) return cuda_fail(h, e, "completion event");
    return WFS_OK;
}


wfs_status wfs_set_uplink(wfs_handle h, int gs, double diameter_m, int samples) {
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    if (gs < 0 || gs >= (int)h->gs.size()) return fail(h, WFS_EINVAL, "guide star index out of range");
    GsDev &g = h->gs[gs];
    const bool on = diameter_m > 0;
    if (!is_finite(diameter_m) || diameter_m < 0) return fail(h, WFS_EINVAL, "diameter_m must be finite and >= 0");
    if (on && !g.gs.is_lgs) return fail(h, WFS_EINVAL, "the uplink tip-tilt applies to laser guide stars only");
    if (on && (samples < 2 || samples > 64)) return fail(h, WFS_EINVAL, "samples must be in [2, 64]");
    if (on && diameter_m / samples < 1e-6) return fail(h, WFS_EINVAL, "uplink sample pitch below 1 micron");
    if (on && !(diameter_m < 0.5 * h->S * h->ds)) return fail(h, WFS_EINVAL, "uplink beam wider than half the screen");
    cudaError_t e;
    if (on && !h->d_uplink) {
        const size_t nw = h->wfs_host.size();
        if ((e = cudaMalloc(&h->d_uplink, sizeof(float2) * h->gs.size())) != cudaSuccess ||
            (e = cudaMemset(h->d_uplink, 0, sizeof(float2) * h->gs.size())) != cudaSuccess ||
            (e = cudaMalloc(&h->d_uplink_part, sizeof(double2) * nw * kMaxLayers)) != cudaSuccess ||
            (e = cudaMalloc(&h->d_uplink_count, sizeof(int) * nw)) != cudaSuccess ||
            (e = cudaMemset(h->d_uplink_count, 0, sizeof(int) * nw)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_uplink, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(h, e, "uplink buffer");
    }
    cudaEventSynchronize(h->ev_measured);  // the work table is read by the measurement in flight
    for (size_t k = 0; k < h->wfs_host.size(); ++k) {
        WfsDesc &d = h->wfs_host[k];
        if (d.gs_index != gs) continue;
        d.uplink = on ? h->d_uplink + gs : nullptr;
        d.up_diam = on ? diameter_m : 0.0;
        d.up_n = on ? samples : 0;
        if ((e = cudaMemcpy(h->d_wfs + k, &d, sizeof(WfsDesc), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(h, e, "work table");
    }
    if (on != (g.up_diam > 0)) h->n_uplink += on ? 1 : -1;
    g.up_diam = on ? diameter_m : 0.0;
    g.up_n = on ? samples : 0;
    if (h->per_slice) return build_slice_projection(h);  // the slice copies carry the uplink too
    return WFS_OK;
}


wfs_status wfs_set_lgs_model(wfs_handle h, int per_slice) {
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    if (per_slice != 0 && per_slice != 1) return fail(h, WFS_EINVAL, "model must be 0 (elongation kernel) or 1 (per slice)");
    if ((per_slice != 0) == h->per_slice) return WFS_OK;
    cudaEventSynchronize(h->ev_measured);  // the work tables are read by the measurement in flight
    cudaError_t e;
    if (per_slice) {
        if (!h->d_slices && (e = cudaMalloc(&h->d_slices, sizeof(SliceDesc) * h->gs.size())) != cudaSuccess)
            return cuda_fail(h, e, "slice tables");
        // the Gaussian extent alone: the elongation table of one slice at the focus
        for (size_t g = 0; g < h->gs.size(); ++g) {
            GsDev &G = h->gs[g];
            if (!G.gs.is_lgs || G.d_ktil_g || G.n_valid == 0) continue;
            const wfs_geometry &geo = h->geoms[G.gs.geometry_index].g;
            const int n = geo.n_pix_sub, Np = geo.n_sub * n;
            const size_t kt = (size_t)G.n_valid * (2 * n - 1) * n;
            if ((e = cudaMalloc(&G.d_ktil_g, kt * sizeof(float2))) != cudaSuccess) return cuda_fail(h, e, "Gaussian table");
            KtilArgs ka;
            memset(&ka, 0, sizeof ka);
            ka.subap = G.d_ids;
            ka.ktil = G.d_ktil_g;
            ka.n = n;
            ka.N = geo.n_fft;
            ka.n_sub = geo.n_sub;
            ka.n_valid = G.n_valid;
            ka.n_na = 1;
            ka.D = h->tel.diameter_m;
            ka.dx = h->tel.diameter_m / Np;
            ka.pix_rad = G.gs.wavelength_m / (geo.n_fft * ka.dx);
            ka.sigma_px = G.gs.spot_fwhm_rad / (2.0 * std::sqrt(2.0 * std::log(2.0))) / ka.pix_rad;
            ka.launch_x = G.gs.launch_x_m;
            ka.launch_y = G.gs.launch_y_m;
            ka.h0 = G.gs.range_m;
            ka.alt[0] = G.gs.range_m;
            ka.w[0] = 1.0;
            if ((e = launch_ktil(ka, 0)) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess)
                return cuda_fail(h, e, "Gaussian table");
        }
    }
    h->per_slice = per_slice != 0;
    if (per_slice && refresh_slices(h) != WFS_OK) {
        h->per_slice = false;
        return WFS_ECUDA;
    }
    for (SpotGroup &G : h->groups) {
        bool lgs = false;
        for (int q = 0; q < G.count; ++q) lgs |= h->wfs_host[G.first + q].is_lgs != 0;
        if (!lgs) continue;
        if (per_slice) {
            G.base_kind = G.kind;
            G.base_grid_cap = G.grid_cap;
            G.base_cta_warps = G.cta_warps;
            // the per-slice variant of the geometry's 32-point kernel (tensor-core or FP32) where
            // it has one, else the self-projecting generic kernel
            const wfs_geometry &geo = h->geoms[G.geom].g;
            if (!is_tc(G.kind) || !sh_tc_slices_supported(geo.n_pix_sub, geo.n_fft, geo.n_det))
                G.kind = sh_n32_supported(geo.n_pix_sub, geo.n_fft, geo.n_det) ? kSpotN32 : kSpotGeneric;
            G.grid_cap = G.cta_warps = 0;
        } else {
            G.kind = G.base_kind;
            G.grid_cap = G.base_grid_cap;
            G.cta_warps = G.base_cta_warps;
        }
        G.per_slice = per_slice != 0;
        for (int q = 0; q < G.count; ++q) {
            WfsDesc &d = h->wfs_host[G.first + q];
            if (!d.is_lgs) continue;
            const GsDev &gd = h->gs[d.gs_index];
            d.slices = per_slice ? h->d_slices + d.gs_index : nullptr;
            d.ktil = per_slice ? gd.d_ktil_g : gd.d_ktil;
        }
        G.sl_projected = per_slice && (is_tc(G.kind) || G.kind == kSpotN32);
    }
    if (build_slice_projection(h) != WFS_OK) return WFS_ECUDA;
    if ((e = cudaMemcpy(h->d_wfs, h->wfs_host.data(), sizeof(WfsDesc) * h->wfs_host.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_fail(h, e, "work table");
    return WFS_OK;
}


wfs_status wfs_loop_batch_create(int n, const wfs_loop *loops, wfs_loop_batch *out) {
    if (!out) return fail(nullptr, WFS_EINVAL, "null output pointer");
    *out = nullptr;
    if (n < 1 || n > kMaxInstances || !loops) return fail(nullptr, WFS_EINVAL, "n must be in [1, 64] with a loop array");
    for (int i = 0; i < n; ++i) {
        const wfs_loop a = loops[i], b = loops[0];
        if (!a) return fail(nullptr, WFS_EINVAL, "null loop in batch");
        for (int j = 0; j < i; ++j)
            if (loops[j] == a) return fail(nullptr, WFS_EINVAL, "a loop appears twice in the batch");
        bool same = a->cm == b->cm && a->n_modes == b->n_modes && a->n_slopes == b->n_slopes &&
                    a->dms.size() == b->dms.size() && a->h->S == b->h->S && a->h->device == b->h->device;
        for (size_t d = 0; same && d < a->dms.size(); ++d) {
            const wfs_dm &x = a->dms[d].d, &y = b->dms[d].d;
            same = x.n_act == y.n_act && x.pitch_m == y.pitch_m && x.alt_m == y.alt_m && x.coupling == y.coupling &&
                   x.support == y.support && x.n_modes == y.n_modes && x.m2a == y.m2a;
        }
        if (!same)
            return fail(nullptr, WFS_EINVAL, "loops of a batch share the control matrix, the slope count and the mirrors");
    }
    wfs_loop_batch b = new wfs_loop_batch_ctx;
    b->loops.assign(loops, loops + n);
    *out = b;
    return WFS_OK;
}

wfs_status wfs_loop_batch_step(wfs_loop_batch b, const float *const *screens, const double *t_s,
                               float *const *slopes_out, void *stream) {
    const NvtxRange nvtx_range("wfs_loop_batch_step");
    if (!b || !screens || !t_s || !slopes_out) return fail(nullptr, WFS_EINVAL, "bad batch arguments");
    const cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)b->loops.size();
    for (int i = 0; i < n; ++i) {
        if (!screens[i] || !slopes_out[i] || !is_finite(t_s[i]))
            return fail(nullptr, WFS_EINVAL, "batch: null buffer or non-finite time for loop " + std::to_string(i));
        if (loop_busy(b->loops[i], s)) return fail(b->loops[i]->h, WFS_EBUSY, "a loop of the batch is busy on another stream");
    }
    // the measurements, one loop after the other
    for (int i = 0; i < n; ++i) {
        wfs_loop lp = b->loops[i];
        wfs_status st = measure_impl(lp->h, screens[i], t_s[i], slopes_out[i], nullptr, s, lp->layers, (int)lp->dms.size());
        if (st != WFS_OK) return st;
        lp->last_stream = s;
    }
    const wfs_loop l0 = b->loops[0];
    wfs_handle h0 = l0->h;
    cudaError_t e;
    // the integrator, up to kMaxGemvVec loops per read of the control matrix
    for (int i0 = 0; i0 < n; i0 += kMaxGemvVec) {
        GemvMultiArgs g{};
        g.A = l0->cm;
        g.rows = l0->n_modes;
        g.cols = l0->n_slopes;
        g.nb = std::min(kMaxGemvVec, n - i0);
        for (int k = 0; k < g.nb; ++k) {
            const wfs_loop lp = b->loops[i0 + k];
            g.x[k] = slopes_out[i0 + k];
            g.y[k] = nullptr;
            g.gain[k] = lp->gain;
            g.c[k] = lp->coeffs;
        }
        long sl = timed_begin(h0, "reconstruct", s);
        e = launch_gemv_multi(g, s);
        timed_end(h0, sl, s);
        if (e != cudaSuccess) return cuda_fail(h0, e, "reconstruction launch");
    }
    // actuator commands per mirror (one read of its modal base per kMaxGemvVec loops), then every
    // loop's layers in launches of up to kMaxInstances
    for (size_t d = 0; d < l0->dms.size(); ++d) {
        const LoopDm &M = l0->dms[d];
        for (int i0 = 0; i0 < n; i0 += kMaxGemvVec) {
            GemvMultiArgs g{};
            g.A = M.d.m2a;
            g.rows = M.d.n_act * M.d.n_act;
            g.cols = M.d.n_modes;
            g.nb = std::min(kMaxGemvVec, n - i0);
            for (int k = 0; k < g.nb; ++k) {
                const wfs_loop lp = b->loops[i0 + k];
                g.x[k] = lp->coeffs + lp->dms[d].mode0;
                g.y[k] = lp->dms[d].act;
                g.gain[k] = nullptr;
                g.c[k] = nullptr;
            }
            long sl = timed_begin(h0, "dm_actuators", s);
            e = launch_gemv_multi(g, s);
            timed_end(h0, sl, s);
            if (e != cudaSuccess) return cuda_fail(h0, e, "actuator launch");
        }
    }
    static thread_local DmLayerBatch lb;
    lb.n = 0;
    auto flush_layers = [&]() -> cudaError_t {
        if (lb.n == 0) return cudaSuccess;
        long sl = timed_begin(h0, "dm_layer", s);
        cudaError_t err = launch_dm_layers(lb, s);
        timed_end(h0, sl, s);
        lb.n = 0;
        return err;
    };
    for (int i = 0; i < n; ++i) {
        const wfs_loop lp = b->loops[i];
        const size_t SS = (size_t)lp->h->S * lp->h->S;
        for (size_t d = 0; d < lp->dms.size(); ++d) {
            if (lb.n == kMaxInstances && (e = flush_layers()) != cudaSuccess) return cuda_fail(h0, e, "mirror layer launch");
            lb.l[lb.n++] = dm_layer_args(lp->h, lp->dms[d], lp->dms[d].act, 1, 1.0f, lp->layers + d * SS);
        }
    }
    if ((e = flush_layers()) != cudaSuccess) return cuda_fail(h0, e, "mirror layer launch");
    for (int i = 0; i < n; ++i)
        if ((e = cudaEventRecord(b->loops[i]->ev_done, s)) != cudaSuccess) return cuda_fail(b->loops[i]->h, e, "completion event");
    return WFS_OK;
}

wfs_status wfs_loop_batch_destroy(wfs_loop_batch b) {
    if (!b) return fail(nullptr, WFS_EINVAL, "null loop batch");
    delete b;
    return WFS_OK;
}

}  // extern "C"
