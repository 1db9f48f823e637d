// static_scratch.cu -- wfs_measure_one_static: the measurement of one guide
// star for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed -- a real-time control loop that must not block on the allocator,
// a host that hands the library a fixed device budget it may not grow, or a
// plugin that only receives buffers from its host program.  Such callers
// cannot create a handle (wfs_create allocates the tables and the projected
// OPD buffer).  This entry point keeps everything the measurement needs
// between its kernels -- the subaperture tables, the DFT and binning
// matrices, the elongation table and the projected OPD -- in one file-scope
// __device__ array of WFS_STATIC_SCRATCH_BYTES, which exists for as long as
// the library is loaded, on every GPU that loads it.  It calls no cudaMalloc,
// cudaFree or other allocating routine; host-side staging uses fixed static
// arrays.
//
// It launches the kernels a handle holding the same guide star at index
// wfs_index launches -- the projection (here with direct gathers, which do
// the same per-tap arithmetic in the same order as the tiled form), the
// elongation table and the FP32 spot kernel -- so its slopes equal that
// handle's bit for bit.
//
// The device address of the array is looked up with cudaGetSymbolAddress on
// every call, with the caller's device current (no allocation; the address
// stays right if the device's context is torn down and made again).  The
// first call on a device may load the library's device code: make it before
// any stream capture.  The tables go up with cudaMemcpyAsync from static
// pageable host arrays: the copy reads them when it runs, the next call
// overwrites them, and the call may wait for the stream's earlier work before
// it returns.  All calls share the device array and the host staging: calls
// from several host threads, or calls whose GPU work overlaps (different
// streams without ordering), race.  Calls on one stream are ordered and safe.
// Nothing in the array needs to start at zero (every part is written before
// it is read) except the status word, which each call clears.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <string>

#include "../../include/gbwfs.h"
#include "internal.h"

using namespace gbwfs;

namespace {

constexpr int kStaticMaxValid = 8192;
constexpr int kStaticMaskWords = (kMaxNPix * kMaxNPix + 31) / 32;

__device__ __align__(256) unsigned char g_static_scratch[WFS_STATIC_SCRATCH_BYTES];

// host staging (fixed size, reused by every call)
int32_t h_ids[kStaticMaxValid];
float h_fill[kStaticMaxValid];
uint32_t h_mask[kStaticMaxValid * kStaticMaskWords];
float2 h_F[kMaxNPix * kMaxN], h_Ga[kMaxNPix * kMaxN], h_G[kMaxNPix * kMaxN];
InstDesc h_inst;
WfsDesc h_wfs;
ProjArgs h_pa;
ShArgs h_sa;
wfs_status st_fail(wfs_status st, const char *msg) {
    set_thread_error(msg);
    return st;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool lit_px(double D, double eps, int Np, int i, int j) {
    const double dx = D / Np;
    const double x = (j - (Np - 1) / 2.0) * dx;
    const double y = (i - (Np - 1) / 2.0) * dx;
    const double r2 = x * x + y * y;
    const double ro = D / 2.0, ri = eps * D / 2.0;
    return (r2 <= ro * ro) && (r2 >= ri * ri);
}

float2 cexp_neg(double a, int N) {  // exp(-2 pi i a / N), a a multiple of 1/4
    a = std::fmod(a, (double)N);
    const double ang = -2.0 * M_PI * a / N;
    return make_float2((float)std::cos(ang), (float)std::sin(ang));
}

}  // namespace

extern "C" wfs_status wfs_measure_one_static(const wfs_telescope *tel, const wfs_geometry *geom,
                                             const wfs_guide_star *gs, const wfs_layers *L,
                                             const float *screens, double t_s, uint64_t seed,
                                             uint32_t wfs_index, int noise_enable, float *slopes_out,
                                             int slopes_capacity, int *n_valid_out, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!tel || !geom || !gs || !L || !screens || !slopes_out || !n_valid_out)
        return st_fail(WFS_EINVAL, "wfs_measure_one_static: null argument");
    *n_valid_out = 0;
    // the checks of wfs_create on this one star and geometry, then the limits of this path
    wfs_guide_star gs1 = *gs;
    gs1.geometry_index = 0;
    if (wfs_status vs = validate_description(tel, 1, &gs1, 1, geom, L); vs != WFS_OK) return vs;
    const wfs_geometry &g = *geom;
    const int n = g.n_pix_sub, N = g.n_fft, nd = g.n_det;
    if (g.precision != WFS_PREC_FP32)
        return st_fail(WFS_EUNSUPPORTED, "wfs_measure_one_static: only WFS_PREC_FP32");
    if (!std::isfinite(t_s) || wfs_index >= (1u << 16))
        return st_fail(WFS_EINVAL, "wfs_measure_one_static: bad time or wfs_index");
    const int Np = g.n_sub * n;

    // the scratch array's device address on the current device
    void *addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_static_scratch);
    if (e != cudaSuccess || !addr) return st_fail(WFS_ECUDA, "wfs_measure_one_static: cudaGetSymbolAddress failed");
    unsigned char *base = (unsigned char *)addr;

    // valid subapertures and lit-pixel bits (FP64 pixel-centre test)
    const int mw = (n * n + 31) / 32;
    int nv = 0;
    for (int sy = 0; sy < g.n_sub; ++sy)
        for (int sx = 0; sx < g.n_sub; ++sx) {
            uint32_t bits[kStaticMaskWords] = {};
            int c = 0;
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q)
                    if (lit_px(tel->diameter_m, tel->obstruction, Np, sy * n + p, sx * n + q)) {
                        ++c;
                        bits[(p * n + q) >> 5] |= 1u << ((p * n + q) & 31);
                    }
            const double f = (double)c / ((double)n * n);
            if (f < g.valid_fill) continue;
            if (nv >= kStaticMaxValid)
                return st_fail(WFS_EINVAL, "wfs_measure_one_static: more than 8192 valid subapertures");
            h_ids[nv] = sy * g.n_sub + sx;
            h_fill[nv] = (float)f;
            memcpy(h_mask + (size_t)nv * mw, bits, mw * sizeof(uint32_t));
            ++nv;
        }
    if (nv > slopes_capacity)
        return st_fail(WFS_EINVAL, "wfs_measure_one_static: slopes_out holds fewer subapertures than are valid");

    // DFT, autocorrelation and binning matrices
    const double cN = (N - 1) / 2.0, cn = (n - 1) / 2.0;
    const int b = N / nd;
    for (int q = 0; q < n; ++q)
        for (int m = 0; m < N; ++m) h_F[q * N + m] = cexp_neg((m - cN) * (q - cn), N);
    for (int d = 0; d < n; ++d)
        for (int k = 0; k < N; ++k) h_Ga[d * N + k] = cexp_neg(-(k - cN) * d, N);
    for (int d = 0; d < n; ++d)
        for (int i = 0; i < nd; ++i) {
            double sr = 0.0, si = 0.0;
            for (int r = 0; r < b; ++r) {
                const double a = std::fmod((b * i + r - cN) * d, (double)N);
                sr += std::cos(-2.0 * M_PI * a / N);
                si += std::sin(-2.0 * M_PI * a / N);
            }
            h_G[d * nd + i] = make_float2((float)sr, (float)si);
        }

    // carve the scratch array
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t o_status = take(sizeof(int));
    const size_t o_inst = take(sizeof(InstDesc));
    const size_t o_wfs = take(sizeof(WfsDesc));
    const size_t o_ids = take((size_t)nv * sizeof(int32_t));
    const size_t o_fill = take((size_t)nv * sizeof(float));
    const size_t o_mask = take((size_t)nv * mw * sizeof(uint32_t));
    const size_t o_F = take((size_t)n * N * sizeof(float2));
    const size_t o_Ga = take((size_t)n * N * sizeof(float2));
    const size_t o_G = take((size_t)n * nd * sizeof(float2));
    const size_t o_kt = take(gs->is_lgs ? (size_t)nv * (2 * n - 1) * n * sizeof(float2) : 0);
    const size_t o_opd = take((size_t)nv * n * n * sizeof(float));
    if (off > (size_t)WFS_STATIC_SCRATCH_BYTES)
        return st_fail(WFS_EINVAL, "wfs_measure_one_static: this wavefront sensor needs more than "
                                   "WFS_STATIC_SCRATCH_BYTES of scratch");
    *n_valid_out = nv;
    if (nv == 0) return WFS_OK;

    if ((e = cudaMemsetAsync(base + o_status, 0, sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_ids, h_ids, (size_t)nv * sizeof(int32_t), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_fill, h_fill, (size_t)nv * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_mask, h_mask, (size_t)nv * mw * sizeof(uint32_t), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_F, h_F, (size_t)n * N * sizeof(float2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_Ga, h_Ga, (size_t)n * N * sizeof(float2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_G, h_G, (size_t)n * nd * sizeof(float2), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return st_fail(WFS_ECUDA, "wfs_measure_one_static: table upload failed");

    const int32_t *d_ids = (const int32_t *)(base + o_ids);
    float2 *d_kt = (float2 *)(base + o_kt);
    float *d_opd = (float *)(base + o_opd);
    const double dx = tel->diameter_m / Np;
    if (gs->is_lgs) {
        KtilArgs ka;
        memset(&ka, 0, sizeof ka);
        ka.subap = d_ids;
        ka.ktil = d_kt;
        ka.n = n;
        ka.N = N;
        ka.n_sub = g.n_sub;
        ka.n_valid = nv;
        ka.n_na = gs->n_na;
        ka.D = tel->diameter_m;
        ka.dx = dx;
        ka.pix_rad = gs->wavelength_m / (N * dx);
        ka.sigma_px = gs->spot_fwhm_rad / (2.0 * std::sqrt(2.0 * std::log(2.0))) / ka.pix_rad;
        ka.launch_x = gs->launch_x_m;
        ka.launch_y = gs->launch_y_m;
        ka.h0 = gs->range_m;
        for (int k = 0; k < gs->n_na; ++k) {
            ka.alt[k] = gs->na_alt_m[k];
            ka.w[k] = gs->na_weight[k];
        }
        if ((e = launch_ktil(ka, s)) != cudaSuccess) return st_fail(WFS_ECUDA, "wfs_measure_one_static: elongation table launch");
    }

    // work tables of this one instance and wavefront sensor
    memset(&h_inst, 0, sizeof h_inst);
    h_inst.n_layers = L->n_layers;
    h_inst.S = L->screen_size;
    h_inst.ds = L->screen_dx_m;
    for (int l = 0; l < L->n_layers; ++l) {
        h_inst.alt[l] = L->alt_m[l];
        h_inst.vx[l] = L->wind_vx_mps[l];
        h_inst.vy[l] = L->wind_vy_mps[l];
        h_inst.x0[l] = L->x0_m[l];
        h_inst.y0[l] = L->y0_m[l];
    }
    h_inst.seed = seed;
    memset(&h_wfs, 0, sizeof h_wfs);
    h_wfs.inst = 0;
    h_wfs.gs_index = (int)wfs_index;
    h_wfs.n = n;
    h_wfs.n_sub = g.n_sub;
    h_wfs.n_valid = nv;
    h_wfs.is_lgs = gs->is_lgs;
    h_wfs.range_m = gs->range_m;
    h_wfs.theta_x = gs->theta_x_rad;
    h_wfs.theta_y = gs->theta_y_rad;
    h_wfs.pupil_dx_over_ds = dx / L->screen_dx_m;
    h_wfs.k_phase = (float)(2.0 * M_PI / gs->wavelength_m);
    h_wfs.photons = (float)gs->photons_per_subap;
    h_wfs.read_noise = (float)gs->read_noise_e;
    h_wfs.subap = d_ids;
    h_wfs.mask = (const uint32_t *)(base + o_mask);
    h_wfs.fill = (const float *)(base + o_fill);
    h_wfs.ktil = gs->is_lgs ? d_kt : nullptr;
    h_wfs.proj_block_begin = 0;
    h_wfs.subap_begin = 0;
    if ((e = cudaMemcpyAsync(base + o_inst, &h_inst, sizeof h_inst, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_wfs, &h_wfs, sizeof h_wfs, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return st_fail(WFS_ECUDA, "wfs_measure_one_static: work table upload failed");
    const InstDesc *d_inst = (const InstDesc *)(base + o_inst);
    const WfsDesc *d_wfs = (const WfsDesc *)(base + o_wfs);
    InstDyn dyn;
    memset(&dyn, 0, sizeof dyn);
    dyn.screens = screens;
    dyn.opd = d_opd;
    dyn.slopes = slopes_out;
    dyn.t = t_s;
    dyn.noise = noise_enable ? 1 : 0;

    h_pa.inst = d_inst;
    h_pa.wfs = d_wfs;
    h_pa.n_wfs = 1;
    h_pa.n_inst = 1;
    h_pa.box_cap = 0;  // direct gathers: no projection tiles in the static scratch
    h_pa.stage_cap = 0;
    h_pa.block_base = 0;
    h_pa.work = nullptr;  // one CTA per block
    h_pa.max_layers = h_inst.n_layers;
    h_pa.status = (int *)(base + o_status);
    h_pa.dyn[0] = dyn;
    if ((e = launch_project(h_pa, project_blocks(h_wfs), s)) != cudaSuccess)
        return st_fail(WFS_ECUDA, "wfs_measure_one_static: projection launch");

    memset(&h_sa, 0, offsetof(ShArgs, dyn));
    h_sa.n = n;
    h_sa.N = N;
    h_sa.nd = nd;
    h_sa.mask_words = mw;
    h_sa.F = (const float2 *)(base + o_F);
    h_sa.Ga = (const float2 *)(base + o_Ga);
    h_sa.G = (const float2 *)(base + o_G);
    h_sa.inst = d_inst;
    h_sa.wfs = d_wfs;
    h_sa.n_wfs = 1;
    h_sa.total = nv;
    h_sa.status = (int *)(base + o_status);
    h_sa.n_inst = 1;
    h_sa.dyn[0] = dyn;
    const int kind = sh_n32_supported(n, N, nd) ? kSpotN32 : kSpotGeneric;
    if ((e = launch_spot(kind, h_sa, s)) != cudaSuccess)
        return st_fail(WFS_ECUDA, "wfs_measure_one_static: spot launch");
    return WFS_OK;
}
