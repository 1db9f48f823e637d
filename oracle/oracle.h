/*
 * oracle.h -- plain, slow FP64 CPU reference of the open-loop Shack-Hartmann
 * measurement (Arcidiacono et al., "End to end numerical simulations of the
 * MAORY multiconjugate adaptive optics system", SPIE 2014, Sec. 4 "Open Loop
 * generation" and "LGS Shack Hartmann wavefront sensor").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the two are written
 * independently from the paper and compared element by element.
 *
 * Every function is a direct transcription of a definition: brute-force
 * matrix DFT, direct periodic convolution, natural-order FP64 sums.  No
 * blocking, fusion or reordering.
 *
 * Parity pins: every function here is pinned by a test against a closed form,
 * an invariant or a brute-force computation (see tests/test_oracle_pins.py).
 */
#ifndef GBWFS_ORACLE_H
#define GBWFS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double diameter_m, obstruction;   /* telescope */
    int n_sub, n, N, n_det;           /* subaps across, px/subap, DFT size, det px/subap */
    double valid_fill;
} orc_wfs_geom;

typedef struct {
    int is_lgs;
    double theta_x, theta_y, range_m, wavelength_m;
    double launch_x, launch_y, spot_fwhm_rad, photons, read_noise;
    int n_na;
    const double *na_alt, *na_weight;
    double up_diameter;               /* LGS uplink beam diameter (m); 0 = no uplink tip-tilt */
    int up_samples;                   /* samples across the uplink beam */
    int slices;                       /* LGS model: 0 = one projection and the elongation kernel,
                                         1 = one wavefront and one DFT per sodium slice */
} orc_star;

typedef struct {
    int n_layers, S;
    double dx;
    const double *alt, *vx, *vy, *x0, *y0;
    int n_atm;                        /* turbulent layers (the first n_atm); the rest are mirror
                                         layers, which the uplink beam does not cross */
} orc_layers;

/* Pupil: binary mask from the pixel-centre test eps*D/2 <= r <= D/2. */
void orc_pupil_mask(double D, double eps, int Np, uint8_t *mask);
/* Valid subapertures (fill >= thr), row-major (y then x); returns the count. */
int orc_valid_subaps(double D, double eps, int n_sub, int n, double thr,
                     int32_t *idx, double *fill);
/* Periodic bilinear sample of one S x S screen at (u = column, v = row). */
double orc_bilinear(const float *scr, int S, double u, double v);
/* Layered, cone-compressed OPD along the star's line of sight at pupil (x, y), time t. */
double orc_opd(const orc_layers *L, const float *screens, const orc_star *gs,
               double x, double y, double t);
/* OPD on the whole Np x Np pupil grid of a geometry. */
void orc_project_grid(double D, int Np, const orc_layers *L, const float *screens,
                      const orc_star *gs, double t, double *opd);
/* LGS uplink tip-tilt (Sec. 4 Open Loop generation: the laser's projection on the sodium layer
   is shifted by the tip-tilt integrated over the upward path).  The beam, of diameter
   up_diameter, runs from the launch point (launch_x, launch_y) on the ground to theta * range on
   the sodium layer; at each turbulent layer it is deflected by the least-squares plane slope of
   the layer's OPD over its footprint (up_samples^2 points on a square grid of pitch
   up_diameter / up_samples, those inside the disc), and the deflection acts over the rest of the
   way up: (dx, dy) = sum_l slope_l (range - h_l) / range, the angle by which the whole spot moves.
   The measurement adds dx x + dy y to the pupil OPD.  Zero for an NGS or up_diameter = 0. */
void orc_uplink_tilt(const orc_layers *L, const float *screens, const orc_star *gs, double t,
                     double *dx, double *dy);
/* Centred 2-D DFT of an n x n field into N x N: Y = F X F^T. */
void orc_dft2(int n, int N, const double *xr, const double *xi, double *yr, double *yi);
/* Sodium elongation kernel (N x N, sums to one) of the subaperture centred at (rbx, rby). */
void orc_elong_kernel(int N, double pix_rad, double rbx, double rby, const orc_star *gs,
                      double *K);
/* Periodic convolution out = I (*) K on an N x N grid. */
void orc_convolve(int N, const double *I, const double *K, double *out);
/* The elongation kernel's convolution in separable form (per slice along rows then columns),
   equal to orc_elong_kernel + orc_convolve up to summation order. */
void orc_elong_convolve_separable(int N, double pix_rad, double rbx, double rby,
                                  const orc_star *gs, const double *I, double *out);
/* orc_measure_wfs's elongation: 0 = direct periodic convolution (default), 1 = separable. */
void orc_set_separable(int on);
/* b x b binning, b = N / nd. */
void orc_bin(int N, int nd, const double *I, double *B);
/* Philox4x32-10 block function. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* The inversion branch of the Poisson sampler (E < 16) on given uniforms u[0..n): k[i] is
   the count that the sampler returns for uniform u[i].  Exposed so that the sampler's exact
   distribution can be tabulated over every uniform the generator can yield. */
void orc_poisson_inversion_n(float E, int n, const float *u, int32_t *k);
/* One detector pixel's noisy count; *k_out receives the Poisson draw.  Pixels 2m and 2m + 1
   share Philox block 0 of counter m (read noise from its words 0-1, Poisson from word 2 or 3). */
double orc_noise_pixel(float E, float read_noise, uint64_t seed, uint32_t pixel,
                       uint32_t wfs, double t, int32_t *k_out);
void orc_noise_image(int n, const float *E, float read_noise, uint64_t seed, uint32_t wfs,
                     double t, uint32_t pixel0, double *C, int32_t *K);
/* Centre of gravity in detector pixels. */
void orc_cog(int nd, const double *C, double *sx, double *sy);

/*
 * LGS per-slice model (Sec. 4 "Open Loop generation": one projection of the beam per sodium
 * sub-layer, each with the pupil projection of its altitude; "LGS Shack Hartmann wavefront
 * sensor": per sub-layer the proper tip-tilt and defocus, the spot weighted by the sodium
 * profile, a Gaussian for the spot's physical extent, the sub-layer images piled up).  Slice s
 * at altitude h_s with weight w_s: OPD_s(x) = the layers projected with the cone 1 - h_l / h_s,
 * plus the uplink tilt, plus the slice's geometric term 1/2 |x - r_L|^2 (1/h0 - 1/h_s) (its
 * tip-tilt (r_b - r_L)(1/h0 - 1/h_s) at subaperture centre r_b, the elongation, and its
 * in-subaperture defocus), h0 = the star's range (the WFS focus); I = sum_s w_s |DFT(X_s)|^2,
 * then the Gaussian alone (the elongation kernel of one slice at h0).  The OPD stage output is
 * the first slice's OPD without its geometric term.
 *
 * One wavefront sensor, one time t.  sel lists indices into the valid-subap
 * list (NULL = all); every output is per selected subap and may be NULL
 * except slopes:  slopes[n_sel][2], opd[n_sel][n*n], I[n_sel][N*N],
 * Ie[n_sel][N*N] (after elongation), E[n_sel][nd*nd], C[n_sel][nd*nd].
 * Returns the number of valid subaps, or -1 on a bad argument.
 */
int orc_measure_wfs(const orc_wfs_geom *g, const orc_star *gs, int wfs_index,
                    const orc_layers *L, const float *screens, double t, uint64_t seed,
                    int noise, int n_sel, const int32_t *sel, double *slopes,
                    double *opd, double *I, double *Ie, double *E, double *C);

/*
 * Closed loop (Sec. 3 "Influence function and modal base", "The closed loop").
 * A deformable mirror is an n_act x n_act grid of actuators at pitch p (metres in
 * its conjugate plane at altitude alt_m), centred on the axis: actuator (ay, ax)
 * at ((ax - c) p, (ay - c) p), c = (n_act - 1) / 2.  Its influence function is
 * separable, w(u_x) w(u_y) with u in pitches and
 *     w(u) = max(0, k^(u^2) - k^(R^2)) / (1 - k^(R^2)),   k = coupling, R = support,
 * a Gaussian that is 1 on its actuator, ~k at one pitch and falls continuously to 0
 * at R pitches.  The mirror's correction layer is a screen on the atmospheric grid
 * (pixel (i, j) at x = (j - S/2) ds, y = (i - S/2) ds), the NEGATED mirror shape
 * -sum_a act[a] w w: the residual the sensors see is the open-loop wavefront minus
 * the mirror, so the layer enters the projection like one more turbulent layer at
 * alt_m with no wind.
 */
typedef struct {
    int n_act;
    double pitch_m, alt_m, coupling;
    int support;
} orc_dm;

/* Correction-layer value at (x, y) metres in the mirror's plane, act[ay * n_act + ax]. */
double orc_dm_value(const orc_dm *dm, const double *act, double x, double y);
/* The whole S x S correction layer (FP64 sums rounded to FP32, as screens are stored). */
void orc_dm_layer(const orc_dm *dm, const double *act, int S, double ds, float *layer);

int orc_num_threads(void);
void orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
