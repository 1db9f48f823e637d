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

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gbwfs.h"
#include "internal.h"

using namespace gbwfs;

namespace {

thread_local std::string tl_error;

struct GeomDev {
    wfs_geometry g{};
    int mask_words = 0;
    float2 *F = nullptr, *Ga = nullptr, *G = nullptr;
    uint8_t *tcB1 = nullptr, *tcB2h = nullptr, *tcB2l = nullptr;  // BF16X3 operand tiles
};

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
    size_t slope_off = 0, opd_off = 0, int_off = 0, det_off = 0;
};

}  // namespace

struct wfs_ctx {
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
    float *d_screens_stage = nullptr;
    float *d_slopes_stage = nullptr;
    cudaStream_t last_stream = nullptr;
    std::string err;
    // side streams for the spot launches of the second and later geometries
    std::vector<cudaStream_t> side;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    // kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;      // pool of event pairs
    std::vector<int> ev_kind;         // kernel kind of each recorded pair
    std::vector<std::string> kinds;   // kernel names
    size_t ev_used = 0;
    bool ev_overflow = false;
};

struct wfs_batch_ctx {
    std::vector<wfs_handle> hs;
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
    for (auto &g : h->geoms) {
        cudaFree(g.F);
        cudaFree(g.Ga);
        cudaFree(g.G);
        cudaFree(g.tcB1);
        cudaFree(g.tcB2h);
        cudaFree(g.tcB2l);
    }
    for (auto &s : h->gs) {
        cudaFree(s.d_ids);
        cudaFree(s.d_mask);
        cudaFree(s.d_fill);
        cudaFree(s.d_ktil);
    }
    cudaFree(h->d_opd);
    cudaFree(h->d_status);
    cudaFree(h->d_screens_stage);
    cudaFree(h->d_slopes_stage);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
    for (cudaStream_t st : h->side) cudaStreamDestroy(st);
    h->side.clear();
    for (cudaEvent_t e : h->ev_join) cudaEventDestroy(e);
    h->ev_join.clear();
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    h->ev_fork = nullptr;
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

wfs_status measure_impl(wfs_handle h, const float *screens, double t, float *slopes,
                        const wfs_stage_out *st, cudaStream_t stream) {
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    if (!screens || !slopes) return fail(h, WFS_EINVAL, "null screens or slopes pointer");
    if (!is_finite(t)) return fail(h, WFS_EINVAL, "t must be finite");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != h->device) return fail(h, WFS_EINVAL, "current device differs from the handle's device");
    h->last_stream = stream;
    float *opd = (st && st->opd) ? st->opd : h->d_opd;

    ProjArgs pa;
    memset(&pa, 0, sizeof pa);
    pa.screens = screens;
    pa.n_layers = h->n_layers;
    pa.S = h->S;
    pa.ds = h->ds;
    pa.t = t;
    for (int l = 0; l < h->n_layers; ++l) {
        pa.alt[l] = h->alt[l];
        pa.vx[l] = h->vx[l];
        pa.vy[l] = h->vy[l];
        pa.x0[l] = h->x0[l];
        pa.y0[l] = h->y0[l];
    }
    int blocks = 0;
    pa.n_wfs = (int)h->gs.size();
    for (size_t w = 0; w < h->gs.size(); ++w) {
        const GsDev &s = h->gs[w];
        const wfs_geometry &g = h->geoms[s.gs.geometry_index].g;
        ProjWfs &P = pa.w[w];
        P.subap = s.d_ids;
        P.opd = opd + s.opd_off;
        P.n = g.n_pix_sub;
        P.n_sub = g.n_sub;
        P.n_valid = s.n_valid;
        P.is_lgs = s.gs.is_lgs;
        P.range_m = s.gs.range_m;
        P.theta_x = s.gs.theta_x_rad;
        P.theta_y = s.gs.theta_y_rad;
        P.pupil_dx_over_ds = (h->tel.diameter_m / (g.n_sub * g.n_pix_sub)) / h->ds;
        P.block_begin = blocks;
        blocks += project_blocks(s.n_valid * g.n_pix_sub * g.n_pix_sub);
    }
    long slot = blocks > 0 ? timed_begin(h, "project", stream) : -1;
    cudaError_t e = launch_project(pa, blocks, stream);
    timed_end(h, slot, stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "projection launch");

    // The largest geometry runs on the caller's stream, launched last; the others run on side
    // streams forked after the projection (launched first, so their few CTAs are resident
    // before the large launch fills the GPU) and joined before the call returns.
    std::vector<ShArgs> jobs;
    jobs.reserve(h->geoms.size());
    for (size_t gi = 0; gi < h->geoms.size(); ++gi) {
        const GeomDev &G = h->geoms[gi];
        ShArgs sa;
        memset(&sa, 0, sizeof sa);
        sa.n = G.g.n_pix_sub;
        sa.N = G.g.n_fft;
        sa.nd = G.g.n_det;
        sa.mask_words = G.mask_words;
        sa.F = G.F;
        sa.Ga = G.Ga;
        sa.G = G.G;
        sa.tc_B1 = G.tcB1;
        sa.tc_B2h = G.tcB2h;
        sa.tc_B2l = G.tcB2l;
        sa.seed = h->seed;
        sa.noise = h->noise;
        sa.t = t;
        sa.status = h->d_status;
        int total = 0, nw = 0;
        for (size_t w = 0; w < h->gs.size(); ++w) {
            const GsDev &s = h->gs[w];
            if (s.gs.geometry_index != (int)gi) continue;
            ShWfs &W = sa.w[nw++];
            W.opd = opd + s.opd_off;
            W.mask = s.d_mask;
            W.fill = s.d_fill;
            W.ktil = s.d_ktil;
            W.slopes = slopes + s.slope_off;
            W.st_I = (st && st->intensity) ? st->intensity + s.int_off : nullptr;
            W.st_E = (st && st->expected) ? st->expected + s.det_off : nullptr;
            W.st_C = (st && st->counts) ? st->counts + s.det_off : nullptr;
            W.n_valid = s.n_valid;
            W.is_lgs = s.gs.is_lgs;
            W.gs_index = (int)w;
            W.subap_begin = total;
            W.k_phase = (float)(2.0 * M_PI / s.gs.wavelength_m);
            W.photons = (float)s.gs.photons_per_subap;
            W.read_noise = (float)s.gs.read_noise_e;
            total += s.n_valid;
        }
        if (!nw || !total) continue;
        sa.n_wfs = nw;
        sa.total = total;
        jobs.push_back(sa);
    }
    if (jobs.empty()) return WFS_OK;
    size_t big = 0;
    for (size_t j = 1; j < jobs.size(); ++j)
        if (jobs[j].total > jobs[big].total) big = j;
    auto prec_of = [&](const ShArgs &sa) {
        for (const GeomDev &G : h->geoms)
            if (G.F == sa.F) return G.g.precision;
        return (int)WFS_PREC_FP32;
    };
    auto launch_job = [&](const ShArgs &sa, cudaStream_t ls) -> cudaError_t {
        const int prec = prec_of(sa);
        std::string name;
        cudaError_t err;
        long sl;
        if (prec == WFS_PREC_BF16X3) {
            sl = timed_begin(h, "spot_tc_bf16x3_N" + std::to_string(sa.N), ls);
            err = launch_sh_tc(sa, ls);
        } else if (sh_n32_supported(sa.n, sa.N, sa.nd)) {
            sl = timed_begin(h, "spot_n32_fp32_N" + std::to_string(sa.N), ls);
            err = launch_sh_n32(sa, ls);
        } else {
            sl = timed_begin(h, "spot_fp32_N" + std::to_string(sa.N), ls);
            err = launch_sh_fp32(sa, ls);
        }
        timed_end(h, sl, ls);
        return err;
    };
    size_t k = 0;
    for (size_t j = 0; j < jobs.size(); ++j) {
        if (j == big) continue;
        if (k >= h->side.size()) return fail(h, WFS_EINVAL, "internal: missing side stream");
        if (k == 0 && (e = cudaEventRecord(h->ev_fork, stream)) != cudaSuccess) return cuda_fail(h, e, "fork");
        if ((e = cudaStreamWaitEvent(h->side[k], h->ev_fork, 0)) != cudaSuccess) return cuda_fail(h, e, "fork wait");
        if ((e = launch_job(jobs[j], h->side[k])) != cudaSuccess) return cuda_fail(h, e, "spot launch");
        if ((e = cudaEventRecord(h->ev_join[k], h->side[k])) != cudaSuccess) return cuda_fail(h, e, "join");
        ++k;
    }
    if ((e = launch_job(jobs[big], stream)) != cudaSuccess) return cuda_fail(h, e, "spot launch");
    for (size_t j = 0; j < k; ++j)
        if ((e = cudaStreamWaitEvent(stream, h->ev_join[j], 0)) != cudaSuccess) return cuda_fail(h, e, "join wait");
    return WFS_OK;
}

}  // namespace

void gbwfs::set_thread_error(const char *msg) { tl_error = msg ? msg : ""; }

extern "C" {

const char *wfs_version(void) { return "gbwfs 0.1 (sm_103a)"; }

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
        if (g.precision == WFS_PREC_FP16S)
            return fail(nullptr, WFS_EUNSUPPORTED, "geometry " + std::to_string(i) + ": WFS_PREC_FP16S is not built");
        if (g.precision == WFS_PREC_BF16X3 && !sh_tc_supported(g.n_pix_sub, g.n_fft, g.n_det))
            return fail(nullptr, WFS_EUNSUPPORTED,
                        "geometry " + std::to_string(i) +
                            ": WFS_PREC_BF16X3 is built for n_fft = 32 with (n_pix_sub, n_det) = (10, 16) or (8, 16)");
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
        if (geom[i].precision == WFS_PREC_BF16X3) {
            const int n = geom[i].n_pix_sub, N = geom[i].n_fft;
            std::vector<uint8_t> b1, b2h, b2l;
            build_tc_tiles(n, N, F64.data(), F64.data() + (size_t)n * N, Ga64.data(), Ga64.data() + (size_t)n * N,
                           b1, b2h, b2l);
            if ((e = upload(&G.tcB1, b1)) != cudaSuccess || (e = upload(&G.tcB2h, b2h)) != cudaSuccess ||
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
    if (n_geom > 1 && (e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming)) != cudaSuccess) {
        release(h);
        delete h;
        return cuda_fail(nullptr, e, "fork event creation");
    }
    h->total_valid = (int)(slope / 2);
    h->opd_total = opd;
    h->int_total = inten;
    h->det_total = det;
    if ((e = cudaMalloc(&h->d_opd, (opd ? opd : 1) * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_status, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(h->d_status, 0, sizeof(int))) != cudaSuccess ||
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
    release(h);
    delete h;
    return WFS_OK;
}

wfs_status wfs_measure(wfs_handle h, const float *screens, double t_s, float *slopes_out, void *stream) {
    return measure_impl(h, screens, t_s, slopes_out, nullptr, (cudaStream_t)stream);
}

wfs_status wfs_measure_stages(wfs_handle h, const float *screens, double t_s, float *slopes_out,
                              const wfs_stage_out *stages, void *stream) {
    return measure_impl(h, screens, t_s, slopes_out, stages, (cudaStream_t)stream);
}

wfs_status wfs_measure_host(wfs_handle h, const float *screens_host, double t_s, float *slopes_host,
                            void *stream) {
    if (!h) return fail(nullptr, WFS_EINVAL, "null handle");
    if (!screens_host || !slopes_host) return fail(h, WFS_EINVAL, "null host buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nscr = (size_t)h->n_layers * h->S * h->S;
    cudaError_t e;
    if (!h->d_screens_stage) {
        if ((e = cudaMalloc(&h->d_screens_stage, nscr * sizeof(float))) != cudaSuccess)
            return cuda_fail(h, e, "screen staging allocation");
        if ((e = cudaMalloc(&h->d_slopes_stage, (2 * (size_t)h->total_valid + 1) * sizeof(float))) != cudaSuccess)
            return cuda_fail(h, e, "slope staging allocation");
    }
    if ((e = cudaMemcpyAsync(h->d_screens_stage, screens_host, nscr * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(h, e, "screen upload");
    wfs_status st = measure_impl(h, h->d_screens_stage, t_s, h->d_slopes_stage, nullptr, s);
    if (st != WFS_OK) return st;
    if ((e = cudaMemcpyAsync(slopes_host, h->d_slopes_stage, 2 * (size_t)h->total_valid * sizeof(float),
                             cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(h, e, "slope download");
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

wfs_status wfs_noise_apply(const float *expected, int n, float read_noise_e, uint64_t seed,
                           uint32_t wfs_index, double t_s, uint32_t pixel0, float *counts, void *stream) {
    if (!expected || !counts || n < 0) return fail(nullptr, WFS_EINVAL, "bad noise arguments");
    if (wfs_index >= (1u << 16)) return fail(nullptr, WFS_EINVAL, "wfs_index must be < 65536");
    if (!(read_noise_e >= 0) || !is_finite(t_s)) return fail(nullptr, WFS_EINVAL, "bad read noise or time");
    cudaError_t e = launch_noise(expected, n, read_noise_e, seed, wfs_index, t_s, pixel0, counts,
                                 (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "noise launch");
    return WFS_OK;
}

wfs_status wfs_batch_create(int n, const wfs_handle *hs, wfs_batch *out) {
    if (!out || !hs || n < 1) return fail(nullptr, WFS_EINVAL, "bad batch arguments");
    for (int i = 0; i < n; ++i)
        if (!hs[i]) return fail(nullptr, WFS_EINVAL, "null handle in batch");
    wfs_batch b = new wfs_batch_ctx();
    b->hs.assign(hs, hs + n);
    *out = b;
    return WFS_OK;
}

wfs_status wfs_batch_measure(wfs_batch b, const float *const *screens, const double *t_s,
                             float *const *slopes_out, void *stream) {
    if (!b || !screens || !t_s || !slopes_out) return fail(nullptr, WFS_EINVAL, "bad batch arguments");
    for (size_t i = 0; i < b->hs.size(); ++i) {
        wfs_status st = measure_impl(b->hs[i], screens[i], t_s[i], slopes_out[i], nullptr, (cudaStream_t)stream);
        if (st != WFS_OK) return st;
    }
    return WFS_OK;
}

wfs_status wfs_batch_destroy(wfs_batch b) {
    if (!b) return fail(nullptr, WFS_EINVAL, "null batch");
    delete b;
    return WFS_OK;
}

}  // extern "C"
