// internal.h -- work tables, kernel argument blocks and launchers shared by the
// library's translation units (never installed; the public ABI is include/gbwfs.h).
//
// Every launch reads two device work tables: one InstDesc per instance (a handle:
// its turbulence layers and noise seed) and one WfsDesc per wavefront sensor (its
// static subaperture tables and its offsets into the instance's buffers).  Only the
// per-call values -- screens, output buffers, time, noise switch -- travel in the
// kernel parameters (InstDyn, one per instance), so a batch of uneven instances is
// one projection launch plus one spot launch per kernel class, and a captured graph
// is replayed by rewriting those parameters.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/gbwfs.h"

namespace gbwfs {

constexpr int kMaxGuideStars = 32;
constexpr int kMaxLayers = 32;         // turbulent layers of an instance
constexpr int kMaxDms = 4;             // deformable mirrors of a closed loop
constexpr int kMaxProjLayers = kMaxLayers + kMaxDms;  // layers a projection sums
constexpr int kMaxNaSlices = 16;
constexpr int kMaxN = 64;           // largest DFT size
constexpr int kMaxNPix = 32;        // largest subaperture side in pupil pixels
constexpr int kMaxInstances = 64;   // instances per launch (batch size limit)

struct InstDesc {                   // static per instance
    int n_layers, S;                // turbulent layers; mirror layers follow them (InstDyn::n_dm)
    double ds;
    double alt[kMaxProjLayers], vx[kMaxProjLayers], vy[kMaxProjLayers], x0[kMaxProjLayers],
        y0[kMaxProjLayers];
    uint64_t seed;
};

// LGS per-slice model of one WFS (Sec. 4: one projection and one spot per sodium sub-layer):
// per slice s its profile weight, its geometric curvature 1/h0 - 1/h_s, and per layer l the
// pupil-to-screen scale (1 - h_l / h_s) dx_pupil / ds as hi + lo.
struct SliceDesc {
    int n;
    float w[kMaxNaSlices], k[kMaxNaSlices];
    float2 c[kMaxNaSlices][kMaxProjLayers];
};

struct WfsDesc {                    // static per wavefront sensor
    int inst;                       // index into the launch's instance tables
    int gs_index;                   // guide-star index within its handle (noise counter)
    int n, n_sub, n_valid, is_lgs;
    double range_m, theta_x, theta_y;
    double pupil_dx_over_ds;        // pupil pitch / screen pitch
    float k_phase;                  // 2 pi / lambda
    float photons, read_noise;
    const int32_t *subap;           // [n_valid] ids sy * n_sub + sx
    const uint32_t *mask;           // [n_valid][mask_words] lit-pixel bits, bit p*n+q
    const float *fill;              // [n_valid]
    const float2 *ktil;             // [n_valid][(2n-1)*n] elongation transfer (LGS only)
    long long opd_off, slope_off, int_off, det_off;  // into the instance's buffers (floats)
    int proj_block_begin;           // first CTA of this WFS in the projection launch
    int subap_begin;                // first subaperture of this WFS in its spot launch
    // projection by shared-memory tiles (pupil pitch <= screen pitch): runs of consecutive
    // valid subapertures of one subaperture row, {sy, first valid index, count, sx of first}
    const int4 *segs;
    int n_segs, tiled, seg_cols;    // seg_cols: largest run width in pupil columns
    // LGS uplink tip-tilt (null: off): the kernel k_uplink writes the spot's deflection times
    // the pupil pitch (OPD per pupil pixel, x and y) here before the projection adds it
    float2 *uplink;
    double launch_x, launch_y, up_diam;
    int up_n;
    // LGS per-slice model (null: one projection and the elongation kernel); read by the per-slice
    // spot kernels, for which ktil holds the Gaussian extent alone
    const SliceDesc *slices;
};

struct InstDyn {                    // per call, per instance
    const float *screens;           // [L][S][S]
    const float *dm;                // [n_dm][S][S] mirror correction layers (closed loop), summed
                                    // after the screens as layers n_layers .. n_layers + n_dm - 1
    int n_dm;
    float *opd;                     // projected OPD, subaperture-tiled
    float *slopes;                  // [sum n_valid][2]
    float *st_I, *st_E, *st_C;      // optional stage outputs (null = not written)
    double t;
    int noise;
};

// ---------------------------------------------------------------- projection
struct ProjArgs {
    const InstDesc *inst;
    const WfsDesc *wfs;
    int n_wfs, n_inst;
    int box_cap;                    // floats of shared memory for tables and screen box
    int stage_cap;                  // floats of one screen box of the bulk-copy form (> 0: that
                                    // form runs; 0: the cp.async form or direct gathers)
    int block_base;                 // projection block of this launch's first block (a launch
                                    // may cover a contiguous range of the WFS table)
    int n_blocks;                   // blocks in this launch (set by the launcher)
    int max_layers;                 // largest n_layers + n_dm of the launch's instances
    int *work;                      // ticket counter pair {next, CTAs done}, zero between
                                    // launches, one launch at a time; null = one CTA per block
    int *status;                    // device status word (limit errors)
    InstDyn dyn[kMaxInstances];
};

// ---------------------------------------------------------------- spot / slopes
struct ShArgs {
    int n, N, nd, mask_words;
    const float2 *F;    // [n][N]  F^T: F[q*N + m] = exp(-2 pi i (m-cN)(q-cn)/N)
    const float2 *Ga;   // [n][N]  Ga[d*N + k] = exp(+2 pi i (k-cN) d / N), d = 0..n-1
    const float2 *G;    // [n][nd] G[d*nd + i] = sum_{r<b} exp(-2 pi i (b i + r - cN) d / N)
    const void *tc_B1, *tc_B2h, *tc_B2l;  // BF16X3 operand tiles (pre-swizzled)
    const void *tc_A0;                    // F's rows, four times over: the first DFT stage's operand
    int mma_u;                            // tensor-core kernels: U = F X as an MMA too (GBWFS_TC_MMA_U=1)
    const InstDesc *inst;
    const WfsDesc *wfs;  // this launch's WFS entries (subap_begin relative to them)
    int n_wfs, total;
    int *status;
    int grid_cap;        // maximum CTAs (0 = the launcher's default)
    int cta_warps;       // warps per CTA where the kernel allows a choice (0 = default)
    int n_inst;
    // Dynamic work split of the 32-point kernels: {next ticket, CTAs done}, zero between
    // launches (the last CTA to finish resets it), used by one launch at a time; null = a
    // static split.
    int *work;
    int project;         // generic and 64-point tensor-core kernels: 1 = project each subaperture's OPD from the screens
                         // itself (no separate projection launch; written to dyn.opd too) on a
                         // side stream, with the shared-memory reservation that keeps projection
                         // CTAs off its SMs; 2 = the same without the reservation
    // 32-point kernels, LGS per-slice model: slice s of a subaperture's OPD sits
    // s * slice_opd_stride floats after slice 0 (projected by k_project); 0 = one OPD
    long long slice_opd_stride;
    int split_noise;     // 32-point kernels: 1 = store the expected image (dyn.st_E, required)
                         // and stop; launch_noise_cog completes the measurement
    InstDyn dyn[kMaxInstances];
};

// ---------------------------------------------------------------- elongation tables
struct KtilArgs {
    const int32_t *subap;
    float2 *ktil;
    int n, N, n_sub, n_valid, n_na;
    double D, dx, pix_rad, sigma_px, launch_x, launch_y, h0;
    double alt[kMaxNaSlices], w[kMaxNaSlices];
};

// ---------------------------------------------------------------- closed loop
constexpr int kMaxDmSupport = 8;    // influence radius limit (pitches)

struct GemvArgs {                   // y = A x (rows x cols, row-major); c += gain * y if c
    const float *A;
    int rows, cols;
    const float *x;
    float *y;
    const float *gain;
    float *c;
};

// The same for nb <= kMaxGemvVec vectors sharing the matrix (read once): column b is computed
// in exactly the order of a single-vector launch.
constexpr int kMaxGemvVec = 4;  // 4 vectors: 80 registers, 3 CTAs per SM
struct GemvMultiArgs {
    const float *A;
    int rows, cols, nb;
    const float *x[kMaxGemvVec];
    float *y[kMaxGemvVec];
    const float *gain[kMaxGemvVec];
    float *c[kMaxGemvVec];
};

struct DmLayerArgs {                // one mirror's correction layer over a window of the grid
    const float *act;               // actuator commands: act_scale * act[(ay n_act + ax) act_stride]
    int act_stride;                 // 1 for a command vector, n_modes for a modal-base column
    float act_scale;
    int n_act, support;
    float r_hi, r_lo;               // screen pitch / actuator pitch as hi + lo (<= 1)
    int c_int;                      // (n_act - 1) / 2 = c_int + c_frac
    float c_frac;
    float log2k, edge, inv_norm;    // log2(coupling), coupling^(R^2), 1 / (1 - coupling^(R^2))
    int S, x0, y0, w, h;            // grid size and window (columns x0 .. x0 + w, rows y0 .. y0 + h)
    float *layer;                   // [S][S]
};

#ifdef __CUDACC__
// Bounds checks of the checked build (-DGBWFS_CHECK, a stand-in for a memory checker): guard
// records WFS_EBOUNDS (7) in the status word and returns false when ok is false, and the caller
// then skips the access; in the normal build it is the constant true and costs nothing.
__device__ __forceinline__ bool guard(bool ok, int *status) {
#ifdef GBWFS_CHECK
    if (!ok && status) atomicCAS(status, 0, 7);
    return ok;
#else
    (void)ok;
    (void)status;
    return true;
#endif
}

// The WFS of a launch that owns global subaperture g (binary search on subap_begin).
__device__ __forceinline__ int find_wfs(const WfsDesc *w, int n, int g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&w[mid].subap_begin) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
#endif

// A launch as a graph kernel node: function, grid, block, dynamic shared memory.
// exp(i phi) of the pupil field: Cody-Waite reduction (Cody and Waite, "Software Manual for
// the Elementary Functions", 1980) of phi to [-pi, pi] with 2 pi held as two floats (the FP32
// value of 2 pi and the remainder), then the hardware sine and cosine of the reduced argument.
// Absolute error about 1e-6 for the phases of a wavefront sensor (|phi| up to ~1e3).
__device__ __forceinline__ void field_phasor(float phi, float &s, float &c) {
    const float m = rintf(phi * 0.159154943f);  // round(phi / (2 pi))
    float r = fmaf(-m, 6.28318548f, phi);
    r = fmaf(-m, -1.74845553e-7f, r);
    __sincosf(r, &s, &c);
}

// Programmatic dependent launch: the projection lets the next grid on its stream start
// early; a spot kernel blocks here until the preceding grid has completed and its writes are
// visible (a no-op when the launch had no programmatic dependency).
__device__ __forceinline__ void allow_dependent_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

struct LaunchShape {
    const void *func;
    dim3 grid, block;
    size_t smem;
};

// Launchers (return the cudaGetLastError() of the launch).
// after_uplink: the launch follows the uplink kernel on s as a programmatic dependent launch
// (the projection waits for it before adding the uplink tilt).
cudaError_t launch_project(const ProjArgs &a, int total_blocks, cudaStream_t s, bool after_uplink = false);
cudaError_t project_launch_shape(const ProjArgs &a, int total_blocks, LaunchShape *out);
// CTAs the projection needs for one WFS.
int project_blocks(const WfsDesc &d);
// Shared-memory floats the WFS's screen box needs (0 when it is projected by direct gathers).
int project_box_floats(const WfsDesc &d);
// Floats of one screen box of the bulk-copy projection for WFS d (0: not tiled).
int project_stage_floats(const WfsDesc &d);
// The bulk-copy projection's launch (tiled blocks through screen boxes moved by the bulk-copy
// unit, direct-gather blocks as in k_project).
cudaError_t project_bulk_launch_shape(const ProjArgs &a, int total_blocks, LaunchShape *out);
// Runs of consecutive valid subapertures per subaperture row, at most max_count each.
void build_segments(const std::vector<int32_t> &ids, int n_sub, int max_count, std::vector<int4> &segs,
                    int *max_run);
// Largest run (in subapertures) of one projection tile for n x n-pixel subapertures.
int segment_max_count(int n);
cudaError_t launch_ktil(const KtilArgs &a, cudaStream_t s);
cudaError_t launch_noise(const float *E, int n, float ron, uint64_t seed, uint32_t wfs, double t,
                         uint32_t pixel0, float *C, cudaStream_t s);
// Spot kernels: kind 0 = generic FP32 (any geometry), 1 = FP32 specialised for N = 32,
// 2 = tensor core (BF16 x3) for N = 32, 3 = tensor core (scaled FP16 x3) for N = 32.
enum SpotKind { kSpotGeneric = 0, kSpotN32 = 1, kSpotTc = 2, kSpotTcF16 = 3 };
inline bool is_tc(int kind) { return kind == kSpotTc || kind == kSpotTcF16; }
bool sh_n32_supported(int n, int N, int nd);
bool sh_tc_supported(int n, int N, int nd);
bool sh_tc_slices_supported(int n, int N, int nd);
// The 64-point tensor-core kernel (32 x 32 pupil pixels, 32 x 32 detector; NGS only).
bool sh_tc64_supported(int n, int N, int nd);
// Shape of the launch (sets the kernel's dynamic shared-memory attribute).
cudaError_t spot_launch_shape(int kind, const ShArgs &a, LaunchShape *out);
// after_project: the launch follows the projection on stream s and may start (prologue only)
// before the projection has finished (programmatic dependent launch); the spot kernels wait
// for the preceding grid to complete before they read its output.
cudaError_t launch_spot(int kind, const ShArgs &a, cudaStream_t s, bool after_project = false);
// Noise and centroid of a 32-point group launched with split_noise (n_det = 16); after_spot:
// follows that spot kernel on s as a programmatic dependent launch.
cudaError_t launch_noise_cog(const ShArgs &a, cudaStream_t s, bool after_spot);
cudaError_t noise_cog_launch_shape(const ShArgs &a, LaunchShape *out);
// Whether a spot kind stores expected images and leaves noise and centroid to k_noise_cog.
// The 32-point kernels with a 16 x 16 detector leave the noise and the centroid to k_noise_cog.
inline bool splits_noise(int kind, int N, int nd) { return (kind == kSpotN32 || is_tc(kind)) && N == 32 && nd == 16; }
// Swizzled BF16 (f16: FP16) operand tiles of the two constant matrices (F^T blocks, Ga blocks),
// from FP64 tables laid out [q][m] (F) and [d][k] (Ga).
void build_tc_tiles(int n, int N, const double *F_re64, const double *F_im64, const double *Ga_re64,
                    const double *Ga_im64, bool f16, std::vector<uint8_t> &B1, std::vector<uint8_t> &B2h,
                    std::vector<uint8_t> &B2l, std::vector<uint8_t> &A0);
void build_tc64_tiles(const double *F_re64, const double *F_im64, bool f16, std::vector<uint8_t> &A0,
                      std::vector<uint8_t> &B1);
// Bounded mbarrier wait that is never satisfied; writes WFS_ETIMEOUT to *status.
cudaError_t launch_wait_check(int *status, int limit, cudaStream_t s);
// LGS uplink tip-tilt of every WFS of the table that has it on: one CTA per (WFS, turbulent
// layer); part [n_wfs][kMaxLayers] scratch, count [n_wfs] zero between launches.
cudaError_t launch_uplink(const InstDesc *inst, const WfsDesc *wfs, int n_wfs, int max_layers, double2 *part,
                          int *count, const InstDyn *dyn0, cudaStream_t s);
// Closed-loop kernels.
cudaError_t launch_gemv(const GemvArgs &a, cudaStream_t s);
cudaError_t launch_gemv_multi(const GemvMultiArgs &a, cudaStream_t s);
cudaError_t gemv_launch_shape(const GemvArgs &a, LaunchShape *out);
// Correction layers of n mirrors (or push-pull instances) in one launch, n <= kMaxInstances.
struct DmLayerBatch {
    int n;
    DmLayerArgs l[kMaxInstances];
};
cudaError_t launch_dm_layers(const DmLayerBatch &b, cudaStream_t s);
// IM rows of a push-pull chunk: im[k][j] = (s[2k][j] - s[2k+1][j]) / (2 amplitude) for k < n_modes,
// j < n_slopes, instance i's slopes at s + i * n_slopes.
cudaError_t launch_push_pull_rows(const float *s, int n_modes, int n_slopes, float inv_2a, float *im,
                                  cudaStream_t st);
// Sets the calling thread's message returned by wfs_last_error(NULL).
void set_thread_error(const char *msg);
// One band of screen rows the host-buffer path copies: rows [row, row + rows) of the [L * S]
// rows of the screens (one layer, no periodic wrap), 16-byte columns [c4_first, c4_first + c4_count).
struct HostRowTask {
    long long row;
    int rows;
    int c4_first;
    int c4_count;
    int row_begin;  // the band's first row in the flattened list of all bands' rows
};
// Copies the bands from mapped host screens (src, device-accessible) into the device screens dst.
cudaError_t launch_host_gather(const float *src, float *dst, int S, const HostRowTask *tasks, int n_tasks,
                               int total_rows, long long n_floats, cudaStream_t s);

// The argument checks of wfs_create (telescope, guide stars, geometries, layers); on failure
// the thread's error message says what is wrong.
wfs_status validate_description(const wfs_telescope *tel, int n_gs, const wfs_guide_star *gs, int n_geom,
                                const wfs_geometry *geom, const wfs_layers *L);

}  // namespace gbwfs
