/*
 * gbwfs.h -- C ABI of the GB300-native Shack-Hartmann wavefront-sensor
 * measurement library (libgbwfs.so).
 *
 * The library computes, on one GPU, the open-loop Shack-Hartmann measurement
 * of Arcidiacono et al., "End to end numerical simulations of the MAORY
 * multiconjugate adaptive optics system" (SPIE 2014):
 *
 *   Sec. 4 "Open Loop generation": the phase screens of the turbulent layers
 *     are piled up, each shifted for the star direction and for the temporal
 *     evolution (frozen flow); for a laser guide star the pupil footprint
 *     shrinks with layer altitude (cone effect).  No Fresnel propagation.
 *   Sec. 4 "LGS Shack Hartmann wavefront sensor": the wavefront is split into
 *     subapertures, each spot computed by FFT (a DFT, Sec. 2), the sodium
 *     layer's sub-layers shift the spot (tip-tilt) and are weighted by the
 *     sodium profile, the physical extent is a Gaussian convolution, the
 *     sub-layers are piled up, noise is added and the centroid gives the X and
 *     Y slopes (Sec. 3, closed-loop block: slopes are the WFS output).
 *
 * Conventions (all entry points):
 *   - Units: lengths in metres, angles in radians, time in seconds, OPD in
 *     metres, slopes in detector pixels.
 *   - Images: row index = y, column index = x, row-major.  Valid
 *     subapertures are ordered row-major (y, then x) over the n_sub x n_sub
 *     grid; a subaperture is valid when its lit-pixel fraction >= valid_fill.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device pointers are plain CUDA device addresses (for example
 *     torch.Tensor.data_ptr()); the caller keeps ownership of every buffer it
 *     passes and must keep it alive until the stream work completes.
 *   - Errors: argument errors are detected on the host before anything is
 *     enqueued and returned synchronously; the message is available from
 *     wfs_last_error().  Errors found by a kernel are written to a device
 *     status word that wfs_sync_status() reads back.
 *   - Threading: a handle may be used by one host thread at a time
 *     (thread-compatible, not thread-safe).  Different handles are
 *     independent.
 */
#ifndef GBWFS_H
#define GBWFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wfs_ctx *wfs_handle;
typedef struct wfs_batch_ctx *wfs_batch;
typedef struct wfs_loop_ctx *wfs_loop;
typedef struct wfs_loop_batch_ctx *wfs_loop_batch;

typedef enum {
    WFS_OK = 0,
    WFS_EINVAL = 1,       /* bad argument (see wfs_last_error) */
    WFS_ENOMEM = 2,       /* device or host allocation failed */
    WFS_ECUDA = 3,        /* a CUDA runtime call failed */
    WFS_EBUSY = 4,        /* handle in use */
    WFS_ETIMEOUT = 5,     /* a bounded device wait gave up */
    WFS_EUNSUPPORTED = 6, /* valid request this build does not implement */
    WFS_EBOUNDS = 7       /* the bounds-checked build (GBWFS_CHECK) met an out-of-range index
                             in a kernel and skipped that access (never in the normal build) */
} wfs_status;

/*
 * DFT arithmetic of a geometry (the rest of the path is FP32 throughout).  The two
 * tensor-core forms are built for n_fft = 32 with (n_pix_sub, n_det) = (10, 16) or
 * (8, 16); other geometries with them get WFS_EUNSUPPORTED from wfs_create.
 */
enum {
    WFS_PREC_FP32 = 0,    /* plain FP32 on the CUDA cores */
    WFS_PREC_BF16X3 = 1,  /* tensor cores, BF16 hi/lo split, 3 products, FP32 accumulate */
    WFS_PREC_FP16S = 2    /* tensor cores, FP16 hi/lo split, 3 products, FP32 accumulate;
                             each subaperture's operands are scaled by powers of two into
                             FP16's normal range (exact, undone after the products) */
};

/* Telescope pupil: circular, diameter D, central obstruction eps (fraction of D). */
typedef struct {
    double diameter_m;
    double obstruction;
} wfs_telescope;

/*
 * Shack-Hartmann geometry (Sec. 4 LGS SH: the WF is split into subapertures
 * and each spot is computed by a DFT).  The pupil is sampled on an
 * (n_sub*n_pix_sub)^2 grid of pitch D/(n_sub*n_pix_sub); each subaperture's
 * n_pix_sub^2 field is zero-padded to an n_fft^2 DFT and the intensity binned
 * to n_det^2 detector pixels.  Requires n_fft >= n_pix_sub, n_fft % n_det == 0,
 * n_pix_sub <= 32, n_fft <= 64; an LGS geometry also needs
 * n_fft >= 2*n_pix_sub - 1.
 */
typedef struct {
    int n_sub;
    int n_pix_sub;
    int n_fft;
    int n_det;
    double valid_fill;  /* valid-subaperture threshold on the lit fraction */
    int precision;      /* WFS_PREC_* */
} wfs_geometry;

/*
 * One guide star and its wavefront sensor.
 *   theta_*: direction of the star.  range_m: LGS focus / sodium centroid
 *   altitude (ignored for an NGS, which is at infinity).  launch_*: position
 *   of the LGS launch telescope in the pupil plane.  spot_fwhm_rad: FWHM of
 *   the Gaussian physical extent of the LGS spot (Sec. 4, must be > 0 for an
 *   LGS).  photons_per_subap: photons in a fully lit subaperture per frame.
 *   read_noise_e: detector read-noise sigma in electrons.  n_na sodium
 *   slices at altitudes na_alt_m with weights na_weight (the sodium profile,
 *   normalised by the library).  Arrays are copied by wfs_create.
 */
typedef struct {
    int is_lgs;
    double theta_x_rad, theta_y_rad;
    double range_m;
    double wavelength_m;
    double launch_x_m, launch_y_m;
    double spot_fwhm_rad;
    double photons_per_subap;
    double read_noise_e;
    int geometry_index;
    int n_na;
    const double *na_alt_m;
    const double *na_weight;
} wfs_guide_star;

/*
 * Turbulent layers (Sec. 4 Open Loop generation).  Each layer is a periodic
 * screen_size^2 OPD screen of pitch screen_dx_m at altitude alt_m, moving
 * with wind (vx, vy) from initial offset (x0, y0): at time t the point
 * sampled for pupil position x is screen position c*x + theta*h - (x0 + v t),
 * with c = 1 - h/range for an LGS and 1 for an NGS, relative to the screen
 * centre.  Arrays are copied by wfs_create.
 */
typedef struct {
    int n_layers;
    int screen_size;
    double screen_dx_m;
    const double *alt_m;
    const double *wind_vx_mps, *wind_vy_mps;
    const double *x0_m, *y0_m;
} wfs_layers;

/*
 * Optional per-stage device outputs of wfs_measure_stages (any may be NULL).
 * Each is the concatenation over guide stars, in guide-star order, of
 * n_valid_w blocks (offsets from wfs_layout):
 *   opd[n_valid][n*n]        projected OPD of each subaperture (m)
 *   intensity[n_valid][N*N]  spot |DFT|^2 before elongation
 *   expected[n_valid][nd*nd] expected detector counts (after elongation,
 *                            binning and photometry, before noise)
 *   counts[n_valid][nd*nd]   noisy counts (equal to expected without noise)
 */
typedef struct {
    float *opd;
    float *intensity;
    float *expected;
    float *counts;
} wfs_stage_out;

typedef struct {
    int n_valid, n, n_fft, n_det, is_lgs;
    size_t slope_offset;      /* in floats, into slopes_out (2 per subaperture) */
    size_t opd_offset;        /* in floats, into wfs_stage_out.opd */
    size_t intensity_offset;  /* in floats, into wfs_stage_out.intensity */
    size_t det_offset;        /* in floats, into wfs_stage_out.expected / counts */
} wfs_layout_info;

/*
 * wfs_create -- validate the description, build the valid-subaperture tables,
 * the pupil mask bits, the DFT and elongation tables, and allocate the
 * handle's device memory (cudaMalloc on the current device).  Host arrays are
 * copied.  seed keys the noise generator; noise_enable = 0 gives the expected
 * image (noise-free slopes).  On success *out owns all of it until
 * wfs_destroy.  Returns WFS_EINVAL (bad description), WFS_EUNSUPPORTED,
 * WFS_ENOMEM or WFS_ECUDA.
 */
wfs_status wfs_create(const wfs_telescope *tel, int n_gs, const wfs_guide_star *gs,
                      int n_geom, const wfs_geometry *geom, const wfs_layers *layers,
                      uint64_t seed, int noise_enable, wfs_handle *out);

/* Release everything the handle owns (synchronises the device first). */
wfs_status wfs_destroy(wfs_handle h);

/*
 * wfs_measure -- one frame at time t_s for every guide star of the handle.
 *   screens: device, float [n_layers][screen_size][screen_size], OPD (m).
 *   slopes_out: device, float [sum_w n_valid_w][2], (x, y) in detector pixels,
 *     guide stars concatenated in order.
 * Asynchronous on `stream`; no allocation, no host synchronisation; inputs
 * are not modified.  One stream at a time: the handle's device scratch belongs
 * to the work in flight, so a call on another stream while the previous
 * measurement is still running returns WFS_EBUSY (nothing is launched); calls
 * on the same stream are ordered by the stream.
 */
wfs_status wfs_measure(wfs_handle h, const float *screens, double t_s, float *slopes_out,
                       void *stream);

/* As wfs_measure, also writing the intermediate stages selected in *stages. */
wfs_status wfs_measure_stages(wfs_handle h, const float *screens, double t_s,
                              float *slopes_out, const wfs_stage_out *stages, void *stream);

/*
 * wfs_measure_host -- the same frame with HOST buffers: copies screens_host
 * (host, same layout as `screens`; pinned memory for asynchronous copies) to
 * the device, measures, and copies the slopes back to slopes_host.  Only the
 * parts of the screens the frame reads are copied: per layer, the areas covered
 * by the guide stars' projected pupils (every cone scale of the LGS model in
 * use) and LGS uplink beams at time t_s, plus a margin of a few pixels.  Pinned
 * memory mapped into the device's address space (pinned allocations under
 * unified addressing) is gathered rectangle by rectangle by a copy kernel
 * (GBWFS_HOST_RECTS=0 in the environment turns this off); otherwise whole
 * rows are copied (the whole set when those cover nine tenths of it).  The first
 * call allocates two sets of device staging buffers (screens and slopes) and a
 * copy stream that later calls reuse: successive calls alternate between the
 * sets and upload on the copy stream, so the next frame's upload overlaps this
 * frame's kernels.  With GBWFS_HOST_ZERO_COPY=1 in the environment, screens in
 * pinned host memory mapped into the device's address space are read in place
 * by the kernels and nothing is copied up (slower on the ELT frame than the
 * row copies; pageable memory always takes the copies).  Asynchronous on
 * `stream`: slopes_host is valid, and screens_host may be reused, after the
 * stream is synchronised.
 */
wfs_status wfs_measure_host(wfs_handle h, const float *screens_host, double t_s,
                            float *slopes_host, void *stream);

/*
 * wfs_host_transfer_bytes -- the bytes the handle's last wfs_measure_host call
 * copied host -> device (screen rows or rectangles; 0 when the kernels read the
 * screens in place) and device -> host (slopes); 0 and 0 before the first call.
 * WFS_EINVAL: a null argument.
 */
wfs_status wfs_host_transfer_bytes(wfs_handle h, uint64_t *h2d_bytes, uint64_t *d2h_bytes);

/* Switch the noise stage on or off for later calls. */
wfs_status wfs_set_noise(wfs_handle h, int enable);

/* Number of valid subapertures of guide star gs, and of all guide stars. */
wfs_status wfs_num_valid(wfs_handle h, int gs, int *n);
wfs_status wfs_total_valid(wfs_handle h, int *n);
/* Valid subaperture ids (sy * n_sub + sx) of guide star gs into host_idx[n_valid]. */
wfs_status wfs_valid_map(wfs_handle h, int gs, int32_t *host_idx);
/* Sizes and buffer offsets of guide star gs. */
wfs_status wfs_layout(wfs_handle h, int gs, wfs_layout_info *out);
/*
 * Synchronise the handle's last stream and read the device status word
 * (WFS_OK, or the first error a kernel recorded), then clear it.
 */
wfs_status wfs_sync_status(wfs_handle h);
/* Last error message of the handle (or, for h == NULL, of the calling thread). */
const char *wfs_last_error(wfs_handle h);

/*
 * wfs_noise_apply -- the noise stage alone (Sec. 4: "final noise-added
 * image"), the same device function the measurement uses:
 *   counts[i] = Poisson(expected[i]) + read_noise_e * z
 * with the uniforms drawn from Philox4x32-10 keyed by seed, counter
 * (pixel0 + i, wfs_index << 16 | block, bits of t_s).  expected and counts
 * are device float[n]; expected >= 0.
 */
wfs_status wfs_noise_apply(const float *expected, int n, float read_noise_e, uint64_t seed,
                           uint32_t wfs_index, double t_s, uint32_t pixel0, float *counts,
                           void *stream);

/*
 * Batching: several handles (uneven geometries, precisions, layer counts) measured
 * by one call.  wfs_batch_create keeps the handle pointers (they must outlive the
 * batch; at most 64, all on the current device, each at most once) and merges their
 * work tables: one projection launch covers every wavefront sensor of every
 * instance, and one persistent spot launch per kernel class (kernel kind, n_pix_sub,
 * n_fft, n_det) covers all subapertures of that class across instances.
 * wfs_batch_measure takes host arrays of n device screen pointers, n times and n
 * device slope buffers (laid out as for wfs_measure of each handle).  The first call
 * builds a CUDA graph (projection node, then the class nodes in parallel); later
 * calls rewrite the nodes' parameters and replay it (GBWFS_BATCH_GRAPH=0 in the
 * environment launches directly instead).  Results equal those of wfs_measure on
 * each handle.  The instances' projected OPD goes to each handle's own scratch, so
 * calls that involve the same handle must not overlap in time.  Asynchronous.
 */
wfs_status wfs_batch_create(int n, const wfs_handle *hs, wfs_batch *out);
wfs_status wfs_batch_measure(wfs_batch b, const float *const *screens, const double *t_s,
                             float *const *slopes_out, void *stream);
/*
 * wfs_batch_measure_subset -- continuous batching: measure only the n_active
 * instances listed in `active` (indices into the batch, each at most once), with
 * screens, t_s and slopes_out given per listed instance (arrays of n_active).  The
 * compacted work table is staged in pinned host memory of slot `slot`
 * (0 <= slot < 8) and copied on `stream`; calls using one slot must be issued on
 * one stream (they reuse its device table), and an instance must not be in two
 * calls whose GPU work overlaps (it owns one OPD scratch).  Launches directly
 * (no graph): one projection and one spot launch per kernel class present.
 * Results equal those of wfs_measure on each listed handle.
 */
wfs_status wfs_batch_measure_subset(wfs_batch b, int slot, int n_active, const int *active,
                                    const float *const *screens, const double *t_s,
                                    float *const *slopes_out, void *stream);
/*
 * Autotuner: times the candidate launch shapes of every kernel class on these inputs
 * (persistent grid size; warps per CTA for the FP32 32-point kernel), keeps the
 * fastest for later calls, and appends it to the file named by the environment
 * variable GBWFS_TUNE_CACHE (if set), from which wfs_batch_create reads earlier
 * choices.  Synchronises `stream`; leaves the slopes of one measurement in slopes_out.
 */
wfs_status wfs_batch_tune(wfs_batch b, const float *const *screens, const double *t_s,
                          float *const *slopes_out, void *stream);
/* Kernel classes of a batch (kind: 0 generic FP32, 1 FP32 N = 32, 2 tensor-core BF16x3). */
typedef struct {
    int kind, n_pix_sub, n_fft, n_det, n_wfs, n_subaps, grid_cap, cta_warps;
} wfs_batch_class;
wfs_status wfs_batch_info(wfs_batch b, int max, wfs_batch_class *out, int *n_out);
wfs_status wfs_batch_destroy(wfs_batch b);

/*
 * Kernel timing (measurement aid).  While enabled, every kernel launch of the
 * handle's later calls is bracketed by CUDA events recorded on the launch
 * stream.  wfs_timing_read synchronises those events, writes up to `max`
 * per-kernel totals (launch count and summed event time in milliseconds) to
 * out, sets *n_out to the number of distinct kernels, and resets the totals.
 * At most 65536 launches are recorded between two reads (WFS_EBUSY beyond).
 */
typedef struct {
    char name[48];
    int launches;
    double total_ms;
} wfs_kernel_time;

wfs_status wfs_timing_enable(wfs_handle h, int enable);
wfs_status wfs_timing_read(wfs_handle h, int max, wfs_kernel_time *out, int *n_out);

/*
 * wfs_measure_one_static -- one guide star's measurement without any device
 * allocation.  The paper has no counterpart; this entry point exists for
 * callers that cannot call cudaMalloc: a real-time control loop that must
 * not block on the allocator, a host program that gives the library a fixed
 * device budget, or a plugin that only receives buffers.  Such callers cannot
 * create a handle, because wfs_create allocates.
 *
 * Everything kept between the kernels (subaperture tables, DFT and binning
 * matrices, the LGS elongation table, the projected OPD) lives in one
 * file-scope device array of WFS_STATIC_SCRATCH_BYTES that every GPU loading
 * the library holds until the process exits.  No cudaMalloc, cudaFree or
 * other allocating routine is called; host staging uses fixed static arrays.
 * The description is checked as wfs_create checks it.  A guide star whose
 * tables would not fit, or with more than 8192 valid subapertures, is
 * rejected with WFS_EINVAL and a message from wfs_last_error(NULL).  Only
 * WFS_PREC_FP32 geometries are accepted (WFS_EUNSUPPORTED otherwise).
 *
 * Inputs and outputs as for wfs_measure with one guide star: screens (device
 * [n_layers][S][S]), slopes_out (device, room for slopes_capacity (x, y)
 * pairs); *n_valid_out receives the number of valid subapertures written.
 * wfs_index is the guide-star index used in the noise counter, so the slopes
 * equal, bit for bit, those of a handle whose guide star wfs_index is *gs.
 *
 * Every call looks up the array's device address with cudaGetSymbolAddress on
 * the current device.  The first call on a device may load the library's
 * device code: make it before any stream capture.  The tables are copied from
 * static pageable host arrays with cudaMemcpyAsync; the copy reads them when
 * it runs and the next call overwrites them, and the call may wait for the
 * stream's earlier work before it returns.  All calls share the device array
 * and the host staging, which keep the last call's contents: calls from
 * several host threads, or calls whose GPU work overlaps on different
 * streams, race.  Calls on one stream are ordered.  Otherwise asynchronous on
 * `stream`.
 */
#define WFS_STATIC_SCRATCH_BYTES (16u << 20)

wfs_status wfs_measure_one_static(const wfs_telescope *tel, const wfs_geometry *geom,
                                  const wfs_guide_star *gs, const wfs_layers *layers,
                                  const float *screens, double t_s, uint64_t seed,
                                  uint32_t wfs_index, int noise_enable, float *slopes_out,
                                  int slopes_capacity, int *n_valid_out, void *stream);

/*
 * wfs_check_bounded_wait -- failure-detection check: launches one CTA that waits on an
 * mbarrier nothing arrives on, for at most `polls` polls (the same bounded wait the
 * tensor-core spot kernel uses for its MMA completions), and records WFS_ETIMEOUT in the
 * handle's device status word, which the next wfs_sync_status returns.  The GPU is never
 * faulted or hung.  The paper has no counterpart (it is a property of this library).
 */
wfs_status wfs_check_bounded_wait(wfs_handle h, int polls, void *stream);

/*
 * Closed loop (Sec. 3 "The closed loop": the sensors compute the slopes of the
 * residual phase, the open-loop wavefront minus the deformable mirrors; the
 * slopes times the control matrix are the differential modal coefficients
 * added to those of the mirrors, a pure integrator; Sec. 3 "Influence function
 * and modal base": a mirror is a linear combination of a modal base defined
 * over its actuators' influence functions).
 *
 * A mirror (wfs_dm) is an n_act x n_act actuator grid at pitch pitch_m in its
 * conjugate plane at altitude alt_m, centred on the axis: actuator (ay, ax)
 * sits at ((ax - c) p, (ay - c) p), c = (n_act - 1) / 2.  Its influence
 * function is separable, w(u_x) w(u_y) with u in pitches and
 *     w(u) = max(0, k^(u^2) - k^(R^2)) / (1 - k^(R^2)),  k = coupling, R = support,
 * 1 on the actuator, about k at one pitch, 0 from R pitches on.  Its modal
 * base m2a (device, row-major [n_act * n_act][n_modes], actuator ay * n_act +
 * ax; metres of mirror shape per unit coefficient) maps its coefficients to
 * actuator commands.  The mirror enters the projection as one more layer at
 * alt_m, without wind, sampled on the screens' grid (pixel (i, j) at
 * ((j - S/2) ds, (i - S/2) ds)) and holding minus the mirror shape: the
 * sensors see the residual.  The cone and direction offsets are those of a
 * turbulent layer at that altitude.
 *
 * Step k (wfs_loop_step): the slopes s_k of the residual seen through the
 * mirrors of coefficients c_k (layout as for wfs_measure), then
 *     c_{k+1} = c_k + gain * (cm s_k)      (per mode, FP32)
 * with cm device row-major [n_modes][2 * total_valid] (n_modes = sum of the
 * mirrors' n_modes, mirror 0's modes first) and gain device [n_modes]; the
 * actuator commands m2a_d c_{k+1} and the mirrors' layers are rebuilt for step
 * k + 1.  So cm maps slopes to the coefficient change; with an interaction
 * matrix registered by applying each mode to the beam (slopes per unit
 * coefficient), cm = pinv(IM).
 *
 * wfs_loop_create attaches a loop to a handle (one loop per handle): it
 * validates (WFS_EINVAL: n_dm outside [1, 4], n_act outside [1, 1024], pitch
 * below the screen pitch, alt not finite or negative, alt not below every LGS range, coupling
 * outside (0, 1), support outside [1, 8], n_modes < 1, a null pointer; WFS_EBUSY
 * when the handle already has a loop), allocates the coefficients (zero),
 * the actuator commands and one S x S layer per mirror, and adds the mirrors'
 * altitudes to the handle's layer table.  m2a, cm and gain stay caller-owned
 * and must outlive the loop; their contents are read at each step.  The
 * handle keeps measuring open loop through wfs_measure.
 *
 * wfs_loop_step is asynchronous on `stream` like wfs_measure (same inputs,
 * same WFS_EBUSY rule for the handle and the loop).  wfs_loop_set_coeffs
 * copies n_modes coefficients from device memory (NULL = zeros) and rebuilds
 * the layers; wfs_loop_get_coeffs copies them to device memory; both are
 * asynchronous on `stream`.  wfs_loop_get_layer copies mirror d's S x S
 * correction layer (the one the next step uses) to device memory,
 * asynchronously on `stream`.  wfs_loop_destroy waits for the loop's work and frees
 * it; the handle stays valid.  The paper gives no influence function; the
 * truncated Gaussian is this library's choice.
 */
typedef struct {
    int n_act;
    double pitch_m;
    double alt_m;
    double coupling;
    int support;
    int n_modes;
    const float *m2a;
} wfs_dm;

wfs_status wfs_loop_create(wfs_handle h, int n_dm, const wfs_dm *dms, const float *cm,
                           const float *gain, wfs_loop *out);
wfs_status wfs_loop_step(wfs_loop lp, const float *screens, double t_s, float *slopes_out,
                         void *stream);
wfs_status wfs_loop_set_coeffs(wfs_loop lp, const float *coeffs, void *stream);
wfs_status wfs_loop_get_coeffs(wfs_loop lp, float *coeffs_out, void *stream);
wfs_status wfs_loop_get_layer(wfs_loop lp, int d, float *layer_out, void *stream);
wfs_status wfs_loop_destroy(wfs_loop lp);

/*
 * Batches of closed loops (Monte-Carlo runs of one system).  wfs_loop_batch_create
 * groups n <= 64 loops (each on its own handle) that share the control matrix
 * pointer, the slope count and the mirrors (same descriptions and modal-base
 * pointers); WFS_EINVAL otherwise.  It keeps the loop pointers (they must
 * outlive the batch).  wfs_loop_batch_step(b, screens[n], t_s[n],
 * slopes_out[n], stream) is equivalent, result for result, to wfs_loop_step of
 * each loop in order on `stream`: the measurements run one after the other,
 * then the control matrix and each modal base are read once per 4 loops (the
 * reconstruction and the actuator commands of up to 4 loops share one launch;
 * each loop's sums keep the single-loop order, so the results are bit for bit
 * those of separate steps), and all the loops' mirror layers are rebuilt in
 * launches of up to 64 layers.  Same WFS_EBUSY rule as wfs_loop_step for
 * every loop.  wfs_loop_batch_destroy frees the batch, not the loops.
 */
wfs_status wfs_loop_batch_create(int n, const wfs_loop *loops, wfs_loop_batch *out);
wfs_status wfs_loop_batch_step(wfs_loop_batch b, const float *const *screens, const double *t_s,
                               float *const *slopes_out, void *stream);
wfs_status wfs_loop_batch_destroy(wfs_loop_batch b);

/*
 * wfs_loop_calibrate -- push-pull registration of the interaction matrix of
 * guide star gs over all the loop's modes (Sec. 3 "The calibration of the
 * interaction matrices": the modes of the base register the slopes of the WFS;
 * Sec. 5: a modal push-pull scheme, 5000 modes of one LGS).  For each mode m
 * the star is measured with +amplitude of the mode in the beam (mirror
 * coefficient -amplitude, the other coefficients 0) and with -amplitude,
 * without turbulence, without noise, at t = 0, through the same projection
 * and spot kernels as wfs_loop_step; row m of im_out (device, row-major
 * [n_modes][2 n_valid_gs], x and y interleaved per subaperture as in
 * wfs_measure) is the difference over 2 amplitude: slopes per unit
 * coefficient, so that cm = pinv(im^T) restricted to that star's slopes.
 * Modes go 32 at a time (64 measurements per launch).  The first call for a
 * star allocates its scratch (64 layers of S x S floats plus the star's OPD,
 * expected images and slopes, 64 times) and synchronises the device; later
 * calls for the same star are asynchronous on `stream`.  The loop's
 * coefficients and layers are left unchanged.  WFS_EINVAL: gs out of range,
 * amplitude zero or not finite, null im_out.
 */
wfs_status wfs_loop_calibrate(wfs_loop lp, int gs, double amplitude, float *im_out, void *stream);

/*
 * wfs_set_uplink -- the LGS uplink tip-tilt (Sec. 4 "Open Loop generation":
 * the projection of the laser beam on the sodium layer is computed with the
 * spot shift induced by the tip-tilt integrated over the upward path).  For
 * laser guide star gs, a launch beam of diameter diameter_m runs from the
 * star's launch point on the ground to theta * range; at each turbulent layer
 * (not the loop's mirror layers) it is deflected by the least-squares plane
 * slope of the layer's OPD over its footprint (samples x samples points on a
 * square grid of pitch diameter_m / samples, those inside the disc, sampled
 * bilinearly like the projection at the frame's time), and the deflection acts
 * over the rest of the way up, times (range - h) / range.  The sum is the angle
 * by which the whole spot moves; every later measurement of the handle adds
 * it to the star's pupil OPD as a tilt (dx x + dy y), computed per frame by one
 * small kernel before the projection.  diameter_m = 0 turns it off (default).
 * Waits for the handle's measurement in flight, then updates its work table.
 * Batches measure without it: wfs_batch_create rejects a handle with it on
 * (WFS_EUNSUPPORTED).  WFS_EINVAL: gs out of range, an NGS with diameter_m > 0,
 * diameter_m negative, not finite or not below half the screen width,
 * samples outside [2, 64].  The paper gives
 * no beam size or fit; the plane fit over a disc is this library's reading.
 */
wfs_status wfs_set_uplink(wfs_handle h, int gs, double diameter_m, int samples);

/*
 * wfs_set_lgs_model -- how the handle's laser guide stars form their spots.
 * 0 (default): one projection with the cone to the star's range and the
 * sodium elongation as a convolution kernel (sum over slices of the profile
 * weight times the Gaussian extent shifted by the slice's offset), on the
 * geometry's spot kernel.  1: the paper's per-slice model (Sec. 4 "Open Loop
 * generation": one projection of the beam per sodium sub-layer, each with the
 * pupil projection of its altitude; "LGS Shack Hartmann wavefront sensor": for
 * each sub-layer its tip-tilt and defocus, the spot multiplied by the sodium
 * profile, a Gaussian for the physical extent, the sub-layer images piled up):
 * for slice s at altitude h_s, OPD_s = the layers seen with the cone
 * 1 - h_l / h_s (mirror layers included) plus the uplink tilt plus
 * 1/2 |x - r_L|^2 (1/h0 - 1/h_s) (h0 = the star's range, the focus; r_L the
 * launch point), one DFT per slice, I = sum_s w_s |DFT|^2, then the Gaussian
 * extent alone, binning, photometry, noise and centroid as in model 0.  It
 * runs on per-slice variants of the spot kernels (on the 32-point geometries
 * one projection launch makes every slice's OPD and the tensor-core BF16x3 or
 * FP32 kernel's variant reads them; other geometries use the generic FP32
 * kernel, which projects each slice itself; one DFT per slice: n_na times the
 * DFT work); the OPD stage output
 * holds the first slice's OPD without its geometric term.  Waits for the
 * handle's measurement in flight and updates its work tables (the first switch
 * to 1 also builds the Gaussian tables, synchronously).  Batches and
 * wfs_loop_calibrate do not support model 1 (WFS_EUNSUPPORTED).  WFS_EINVAL:
 * model not 0 or 1.
 */
wfs_status wfs_set_lgs_model(wfs_handle h, int per_slice);

/* Library version string. */
const char *wfs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GBWFS_H */
