/*
 * oracle.c -- FP64 CPU reference of the open-loop Shack-Hartmann measurement.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library.  Independent of the
 * CUDA path (no shared code, header, table or constant).
 *
 * Paper: Arcidiacono et al. 2014 (MAORY E2E simulation).
 *   Sec. 4 "Open Loop generation": layers piled up, shifted for the star
 *     direction and the temporal evolution; for an LGS the pupil footprint
 *     shrinks with altitude (cone effect).
 *   Sec. 4 "LGS Shack Hartmann wavefront sensor": the WF is split into
 *     subapertures, each spot computed by FFT (Sec. 2: "FFT (actually DFT)"),
 *     sodium sub-layers with their tip-tilt shift weighted by the sodium
 *     profile, a Gaussian convolution for the physical spot extent, the
 *     sub-layers piled up, noise added, centroid taken to give X/Y slopes.
 *
 * Readings where the paper is silent are fixed in the design notes
 * (pixel-centre pupil, 0.5 fill threshold, centred DFT, periodic
 * minimum-image Gaussian kernel, periodic convolution, Philox/Poisson/
 * Box-Muller noise, CoG in detector pixels).
 *
 * Build with -ffp-contract=off: the Poisson decisions are taken in FP32 with
 * a fixed operation order, so no fused multiply-adds.  A count decided by a
 * floating-point comparison can only be compared draw by draw if both sides
 * decide in the same precision with the same roundings; the paper gives no
 * precision, so the decision is FP32.  The sampler's exact distribution over
 * every uniform is pinned against the exact Poisson CDF in the tests.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel loops (timing only; results do not depend on it). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---- pupil and subapertures (Sec. 2 pupil sampling; Sec. 4 subaperture split) ---- */

static int lit(double D, double eps, int Np, int i, int j)
{
    double dx = D / Np;
    double x = (j - (Np - 1) / 2.0) * dx;
    double y = (i - (Np - 1) / 2.0) * dx;
    double r2 = x * x + y * y;
    double ro = D / 2.0, ri = eps * D / 2.0;
    return (r2 <= ro * ro) && (r2 >= ri * ri);
}

void orc_pupil_mask(double D, double eps, int Np, uint8_t *mask)
{
    for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j)
            mask[(size_t)i * Np + j] = (uint8_t)lit(D, eps, Np, i, j);
}

int orc_valid_subaps(double D, double eps, int n_sub, int n, double thr, int32_t *idx,
                     double *fill)
{
    int Np = n_sub * n, count = 0;
    for (int sy = 0; sy < n_sub; ++sy)
        for (int sx = 0; sx < n_sub; ++sx) {
            int c = 0;
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q) c += lit(D, eps, Np, sy * n + p, sx * n + q);
            double f = (double)c / ((double)n * n);
            if (f >= thr) {
                if (idx) idx[count] = sy * n_sub + sx;
                if (fill) fill[count] = f;
                ++count;
            }
        }
    return count;
}

/* ---- projection (Sec. 4 Open Loop generation) ---- */

static int wrap(long long i, int S)
{
    long long r = i % S;
    return (int)(r < 0 ? r + S : r);
}

double orc_bilinear(const float *scr, int S, double u, double v)
{
    double iu = floor(u), iv = floor(v);
    double f = u - iu, g = v - iv;
    int i0 = wrap((long long)iu, S), i1 = wrap((long long)iu + 1, S);
    int j0 = wrap((long long)iv, S), j1 = wrap((long long)iv + 1, S);
    double s00 = scr[(size_t)j0 * S + i0], s01 = scr[(size_t)j0 * S + i1];
    double s10 = scr[(size_t)j1 * S + i0], s11 = scr[(size_t)j1 * S + i1];
    return (1 - f) * (1 - g) * s00 + f * (1 - g) * s01 + (1 - f) * g * s10 + f * g * s11;
}

double orc_opd(const orc_layers *L, const float *screens, const orc_star *gs, double x,
               double y, double t)
{
    double sum = 0.0;
    for (int l = 0; l < L->n_layers; ++l) {
        double h = L->alt[l];
        /* cone: a source at finite range sees the layer through a footprint
           shrunk by (1 - h / range) */
        double c = gs->is_lgs ? 1.0 - h / gs->range_m : 1.0;
        /* frozen flow: the screen moves by +v t, so the sample point moves by -v t */
        double u = L->S / 2.0 + (c * x + gs->theta_x * h - (L->x0[l] + L->vx[l] * t)) / L->dx;
        double v = L->S / 2.0 + (c * y + gs->theta_y * h - (L->y0[l] + L->vy[l] * t)) / L->dx;
        sum += orc_bilinear(screens + (size_t)l * L->S * L->S, L->S, u, v);
    }
    return sum;
}

void orc_project_grid(double D, int Np, const orc_layers *L, const float *screens,
                      const orc_star *gs, double t, double *opd)
{
    double dx = D / Np;
    for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j) {
            double x = (j - (Np - 1) / 2.0) * dx, y = (i - (Np - 1) / 2.0) * dx;
            opd[(size_t)i * Np + j] = orc_opd(L, screens, gs, x, y, t);
        }
}

/* ---- LGS uplink tip-tilt (Sec. 4 Open Loop generation) ---- */

void orc_uplink_tilt(const orc_layers *L, const float *screens, const orc_star *gs, double t,
                     double *dx, double *dy)
{
    *dx = *dy = 0.0;
    if (!gs->is_lgs || !(gs->up_diameter > 0) || gs->up_samples < 2) return;
    int n = gs->up_samples;
    double D = gs->up_diameter, H = gs->range_m;
    for (int l = 0; l < L->n_atm; ++l) {
        double h = L->alt[l];
        if (!(h < H)) continue;
        /* centre of the beam at the layer: from the launch point towards the spot */
        double cx = gs->launch_x * (1.0 - h / H) + gs->theta_x * h;
        double cy = gs->launch_y * (1.0 - h / H) + gs->theta_y * h;
        double sxv = 0.0, syv = 0.0, sxx = 0.0, syy = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double ox = (j - (n - 1) / 2.0) * D / n, oy = (i - (n - 1) / 2.0) * D / n;
                if (ox * ox + oy * oy > D * D / 4.0) continue;
                double u = L->S / 2.0 + (cx + ox - (L->x0[l] + L->vx[l] * t)) / L->dx;
                double v = L->S / 2.0 + (cy + oy - (L->y0[l] + L->vy[l] * t)) / L->dx;
                double val = orc_bilinear(screens + (size_t)l * L->S * L->S, L->S, u, v);
                sxv += ox * val;
                syv += oy * val;
                sxx += ox * ox;
                syy += oy * oy;
            }
        /* plane fit: the offsets sum to zero over the symmetric sample set, so the mean drops out */
        *dx += sxv / sxx * (H - h) / H;
        *dy += syv / syy * (H - h) / H;
    }
}

/* ---- spot by DFT (Sec. 4 LGS SH; Sec. 2 DFT) ---- */

/* F[k][p] = exp(-2 pi i (k - cN)(p - cn) / N), cN = (N-1)/2, cn = (n-1)/2 */
static void dft_matrix(int n, int N, double *fr, double *fi)
{
    double cN = (N - 1) / 2.0, cn = (n - 1) / 2.0;
    for (int k = 0; k < N; ++k)
        for (int p = 0; p < n; ++p) {
            double a = (k - cN) * (p - cn);     /* a multiple of 1/4: exact */
            a = fmod(a, (double)N);             /* exact reduction */
            double ang = -2.0 * M_PI * a / N;
            fr[k * n + p] = cos(ang);
            fi[k * n + p] = sin(ang);
        }
}

void orc_dft2(int n, int N, const double *xr, const double *xi, double *yr, double *yi)
{
    double *fr = malloc(sizeof(double) * N * n), *fi = malloc(sizeof(double) * N * n);
    double *ur = malloc(sizeof(double) * N * n), *ui = malloc(sizeof(double) * N * n);
    dft_matrix(n, N, fr, fi);
    /* U = F X  (N x n) */
    for (int k = 0; k < N; ++k)
        for (int q = 0; q < n; ++q) {
            double sr = 0, si = 0;
            for (int p = 0; p < n; ++p) {
                double a = fr[k * n + p], b = fi[k * n + p];
                double c = xr[p * n + q], d = xi[p * n + q];
                sr += a * c - b * d;
                si += a * d + b * c;
            }
            ur[k * n + q] = sr;
            ui[k * n + q] = si;
        }
    /* Y = U F^T  (N x N) */
    for (int k = 0; k < N; ++k)
        for (int m = 0; m < N; ++m) {
            double sr = 0, si = 0;
            for (int q = 0; q < n; ++q) {
                double a = ur[k * n + q], b = ui[k * n + q];
                double c = fr[m * n + q], d = fi[m * n + q];
                sr += a * c - b * d;
                si += a * d + b * c;
            }
            yr[k * N + m] = sr;
            yi[k * N + m] = si;
        }
    free(fr); free(fi); free(ur); free(ui);
}

/* ---- elongation (Sec. 4 LGS SH: sub-layer tip-tilt, profile weight, Gaussian) ---- */

static double min_image(double d, int N)
{
    return d - N * floor(d / N + 0.5);
}

void orc_elong_kernel(int N, double pix_rad, double rbx, double rby, const orc_star *gs,
                      double *K)
{
    double sigma = gs->spot_fwhm_rad / (2.0 * sqrt(2.0 * log(2.0))) / pix_rad;
    double h0 = gs->range_m, tot = 0.0;
    memset(K, 0, sizeof(double) * N * N);
    for (int s = 0; s < gs->n_na; ++s) {
        /* slice at h_s seen from the subaperture, relative to the focus at h0 */
        double k = 1.0 / h0 - 1.0 / gs->na_alt[s];
        double shx = (rbx - gs->launch_x) * k / pix_rad;
        double shy = (rby - gs->launch_y) * k / pix_rad;
        for (int p = 0; p < N; ++p)
            for (int q = 0; q < N; ++q) {
                double dy = min_image(p - shy, N), dx = min_image(q - shx, N);
                K[p * N + q] += gs->na_weight[s] * exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma));
            }
    }
    for (int i = 0; i < N * N; ++i) tot += K[i];
    for (int i = 0; i < N * N; ++i) K[i] /= tot;
}

/* The same elongated spot by the separable form: each slice's Gaussian is a product of a
   row and a column profile on the minimum-image distance, so the periodic convolution with
   K = sum_s w_s gy_s gx_s^T / Z is, per slice, a circular convolution along the columns
   and then along the rows (2 N^3 operations per slice instead of N^4).  Equal to
   orc_elong_kernel + orc_convolve up to the order of the sums. */
void orc_elong_convolve_separable(int N, double pix_rad, double rbx, double rby,
                                  const orc_star *gs, const double *I, double *out)
{
    double sigma = gs->spot_fwhm_rad / (2.0 * sqrt(2.0 * log(2.0))) / pix_rad;
    double h0 = gs->range_m, Z = 0.0;
    double *gy = malloc(sizeof(double) * N), *gx = malloc(sizeof(double) * N);
    double *T = malloc(sizeof(double) * N * N);
    for (int i = 0; i < N * N; ++i) out[i] = 0.0;
    for (int s = 0; s < gs->n_na; ++s) {
        double k = 1.0 / h0 - 1.0 / gs->na_alt[s];
        double shx = (rbx - gs->launch_x) * k / pix_rad;
        double shy = (rby - gs->launch_y) * k / pix_rad;
        double sy = 0.0, sx = 0.0;
        for (int p = 0; p < N; ++p) {
            double dy = min_image(p - shy, N), dx = min_image(p - shx, N);
            gy[p] = exp(-(dy * dy) / (2.0 * sigma * sigma));
            gx[p] = exp(-(dx * dx) / (2.0 * sigma * sigma));
            sy += gy[p];
            sx += gx[p];
        }
        Z += gs->na_weight[s] * sy * sx;
        /* along the rows: T[p][m] = sum_q I[p][q] gx[(m - q) mod N] */
        for (int p = 0; p < N; ++p)
            for (int m = 0; m < N; ++m) {
                double a = 0.0;
                for (int q = 0; q < N; ++q) a += I[p * N + q] * gx[(m - q + N) % N];
                T[p * N + m] = a;
            }
        /* along the columns, weighted: out[k][m] += w_s sum_p gy[(k - p) mod N] T[p][m] */
        for (int kk = 0; kk < N; ++kk)
            for (int m = 0; m < N; ++m) {
                double a = 0.0;
                for (int p = 0; p < N; ++p) a += gy[(kk - p + N) % N] * T[p * N + m];
                out[kk * N + m] += gs->na_weight[s] * a;
            }
    }
    for (int i = 0; i < N * N; ++i) out[i] /= Z;
    free(gy); free(gx); free(T);
}

/* Which elongation form orc_measure_wfs uses: 0 the direct periodic convolution (default,
   for parity), 1 the separable form (for timing). */
static int g_separable = 0;
void orc_set_separable(int on) { g_separable = on != 0; }

void orc_convolve(int N, const double *I, const double *K, double *out)
{
    for (int k = 0; k < N; ++k)
        for (int m = 0; m < N; ++m) {
            double s = 0.0;
            for (int p = 0; p < N; ++p)
                for (int q = 0; q < N; ++q)
                    s += I[p * N + q] * K[((k - p + N) % N) * N + ((m - q + N) % N)];
            out[k * N + m] = s;
        }
}

void orc_bin(int N, int nd, const double *I, double *B)
{
    int b = N / nd;
    for (int i = 0; i < nd; ++i)
        for (int j = 0; j < nd; ++j) {
            double s = 0.0;
            for (int r = 0; r < b; ++r)
                for (int c = 0; c < b; ++c) s += I[(b * i + r) * N + (b * j + c)];
            B[i * nd + j] = s;
        }
}

/* ---- noise (Sec. 4: "final noise-added image") ---- */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64
   multiplies; the key advances by the Weyl constants between rounds. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 23 random bits + 1/2, scaled: exactly representable, strictly inside (0, 1) */
static float unit_float(uint32_t x)
{
    return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

/* The uniforms of one pixel.  Pixels go in pairs (2m, 2m + 1) sharing block 0 of
   counter (m, wfs << 16 | block, bits(t)); a pixel of parity s draws word 2 + s of
   block 0 first, then all four words of blocks 1 + s, 3 + s, 5 + s, ... */
typedef struct {
    uint32_t key[2], ctr[4], buf[4];
    int pos, parity;
    uint32_t block;
} ustream;

static void us_block(ustream *s, uint32_t block)
{
    s->block = block;
    s->ctr[1] = (s->ctr[1] & 0xFFFF0000u) | (block & 0xFFFFu);
    orc_philox(s->ctr, s->key, s->buf);
}

static float us_next(ustream *s)
{
    if (s->pos == 4) {
        us_block(s, s->block == 0 ? 1u + (uint32_t)s->parity : s->block + 2u);
        s->pos = 0;
    }
    float u = unit_float(s->buf[s->pos]);
    s->pos = (s->block == 0) ? 4 : s->pos + 1;
    return u;
}

/* log(k!) in FP32: exact sum of logs below 10, Stirling's series above. */
static float log_factorial(float k)
{
    if (k < 10.0f) {
        float s = 0.0f;
        for (int j = 2; j <= (int)k; ++j) s = s + logf((float)j);
        return s;
    }
    float x = k + 1.0f;
    float r = 1.0f / x;
    float corr = r * (1.0f / 12.0f - (r * r) * (1.0f / 360.0f));
    return (x - 0.5f) * logf(x) - x + 0.918938533f + corr;
}

/* Inversion by sequential search (E < 16): the smallest k with u <= F_k, where
   F_k = sum_{j<=k} p_j, p_0 = exp(-E) and p_k = p_{k-1} E / k.  FP32, the recurrence
   evaluated as (p_{k-1} E) (1/k) with 1/k rounded to nearest: three IEEE roundings in
   a fixed order; the search also stops once F no longer grows.  For E < 16 it stops
   before k = 43 even at the largest uniform the stream yields. */
static int32_t poisson_inversion(float E, float u)
{
    float p = expf(-E);
    float F = p;
    int32_t k = 0;
    while (u > F) {
        k = k + 1;
        p = (p * E) * (1.0f / (float)k);
        float Fn = F + p;
        if (Fn == F) break;
        F = Fn;
    }
    return k;
}

void orc_poisson_inversion_n(float E, int n, const float *u, int32_t *k)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) k[i] = poisson_inversion(E, u[i]);
}

/* Poisson(E) in FP32: sequential-search inversion for E < 16, Hormann's
   transformed rejection (PTRS, 1993) for E >= 16. */
static int32_t poisson_f32(float E, ustream *s)
{
    if (!(E > 0.0f)) return 0;
    if (E < 16.0f) return poisson_inversion(E, us_next(s));
    float slam = sqrtf(E);
    float logE = logf(E);
    float b = 0.931f + 2.53f * slam;
    float a = -0.059f + 0.02483f * b;
    float inv_alpha = 1.1239f + 1.1328f / (b - 3.4f);
    float vr = 0.9277f - 3.6224f / (b - 2.0f);
    for (int tries = 0; tries < 1024; ++tries) {
        float U = us_next(s) - 0.5f;
        float V = us_next(s);
        float us = 0.5f - fabsf(U);
        float kf = floorf((2.0f * a / us + b) * U + E + 0.43f);
        if (us >= 0.07f && V <= vr) return (int32_t)kf;
        if (kf < 0.0f || (us < 0.013f && V > us)) continue;
        float lhs = logf(V) + logf(inv_alpha) - logf(a / (us * us) + b);
        float rhs = -E + kf * logE - log_factorial(kf);
        if (lhs <= rhs) return (int32_t)kf;
    }
    return (int32_t)floorf(E);
}

double orc_noise_pixel(float E, float read_noise, uint64_t seed, uint32_t pixel, uint32_t wfs,
                       double t, int32_t *k_out)
{
    ustream s;
    uint64_t tb;
    memcpy(&tb, &t, sizeof tb);
    s.key[0] = (uint32_t)seed;
    s.key[1] = (uint32_t)(seed >> 32);
    s.ctr[0] = pixel >> 1;
    s.ctr[1] = wfs << 16;
    s.ctr[2] = (uint32_t)tb;
    s.ctr[3] = (uint32_t)(tb >> 32);
    s.parity = (int)(pixel & 1u);
    us_block(&s, 0);
    /* block 0: words 0 and 1 give the pair's two Box-Muller deviates (cos for the even
       pixel, sin for the odd one); word 2 + parity starts this pixel's Poisson draws */
    double r = sqrt(-2.0 * log((double)unit_float(s.buf[0])));
    double th = 2.0 * M_PI * (double)unit_float(s.buf[1]);
    double z = r * (s.parity ? sin(th) : cos(th));
    s.pos = 2 + s.parity;
    int32_t k = poisson_f32(E, &s);
    if (k_out) *k_out = k;
    return (double)k + (double)read_noise * z;
}

void orc_noise_image(int n, const float *E, float read_noise, uint64_t seed, uint32_t wfs,
                     double t, uint32_t pixel0, double *C, int32_t *K)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        C[i] = orc_noise_pixel(E[i], read_noise, seed, pixel0 + (uint32_t)i, wfs, t,
                               K ? &K[i] : NULL);
}

/* ---- centroid (Sec. 3 closed loop: X and Y slopes; Sec. 4: centroid of the image) ---- */

void orc_cog(int nd, const double *C, double *sx, double *sy)
{
    double c = (nd - 1) / 2.0, s = 0.0, mx = 0.0, my = 0.0;
    for (int i = 0; i < nd; ++i)
        for (int j = 0; j < nd; ++j) {
            double v = C[i * nd + j];
            s += v;
            mx += (j - c) * v;
            my += (i - c) * v;
        }
    if (s > 0.0) {
        *sx = mx / s;
        *sy = my / s;
    } else {
        *sx = 0.0;
        *sy = 0.0;
    }
}

/* ---- deformable mirrors (Sec. 3 "Influence function and modal base") ---- */

/* Influence along one axis at u pitches: a Gaussian of value k at one pitch, lowered by its
   value at the support radius and renormalised, so that it reaches 0 continuously there. */
static double dm_axis(double u, double k, int R)
{
    double edge = pow(k, (double)R * R);
    double g = pow(k, u * u) - edge;
    return g > 0.0 ? g / (1.0 - edge) : 0.0;
}

double orc_dm_value(const orc_dm *dm, const double *act, double x, double y)
{
    double c = (dm->n_act - 1) / 2.0, sum = 0.0;
    /* actuators farther than the support contribute zero terms: visit the others only, in
       the natural (ay, ax) order */
    int ax0 = (int)floor(x / dm->pitch_m + c) - dm->support - 1, ax1 = ax0 + 2 * dm->support + 3;
    int ay0 = (int)floor(y / dm->pitch_m + c) - dm->support - 1, ay1 = ay0 + 2 * dm->support + 3;
    if (ax0 < 0) ax0 = 0;
    if (ay0 < 0) ay0 = 0;
    if (ax1 > dm->n_act - 1) ax1 = dm->n_act - 1;
    if (ay1 > dm->n_act - 1) ay1 = dm->n_act - 1;
    for (int ay = ay0; ay <= ay1; ++ay) {
        double wy = dm_axis(y / dm->pitch_m - (ay - c), dm->coupling, dm->support);
        for (int ax = ax0; ax <= ax1; ++ax) {
            double wx = dm_axis(x / dm->pitch_m - (ax - c), dm->coupling, dm->support);
            sum += act[(size_t)ay * dm->n_act + ax] * wx * wy;
        }
    }
    /* the mirror takes its shape out of the beam */
    return -sum;
}

void orc_dm_layer(const orc_dm *dm, const double *act, int S, double ds, float *layer)
{
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j)
            layer[(size_t)i * S + j] = (float)orc_dm_value(dm, act, (j - S / 2.0) * ds, (i - S / 2.0) * ds);
}

/* ---- one wavefront sensor ---- */

int orc_measure_wfs(const orc_wfs_geom *g, const orc_star *gs, int wfs_index,
                    const orc_layers *L, const float *screens, double t, uint64_t seed,
                    int noise, int n_sel, const int32_t *sel, double *slopes, double *opd_out,
                    double *I_out, double *Ie_out, double *E_out, double *C_out)
{
    if (g->n <= 0 || g->N < g->n || g->n_det <= 0 || g->N % g->n_det) return -1;
    int n = g->n, N = g->N, nd = g->n_det, Np = g->n_sub * g->n;
    int nv = orc_valid_subaps(g->diameter_m, g->obstruction, g->n_sub, n, g->valid_fill, NULL, NULL);
    int32_t *idx = malloc(sizeof(int32_t) * (nv > 0 ? nv : 1));
    double *fill = malloc(sizeof(double) * (nv > 0 ? nv : 1));
    orc_valid_subaps(g->diameter_m, g->obstruction, g->n_sub, n, g->valid_fill, idx, fill);
    if (!sel) n_sel = nv;
    double dx = g->diameter_m / Np;
    double pix_rad = gs->wavelength_m / (N * dx);
    double upx, upy;
    orc_uplink_tilt(L, screens, gs, t, &upx, &upy);

#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < n_sel; ++s) {
        int v = sel ? sel[s] : s;
        if (v < 0 || v >= nv) continue;
        int sy = idx[v] / g->n_sub, sx = idx[v] % g->n_sub;
        double *xr = calloc((size_t)n * n, sizeof(double)), *xi = calloc((size_t)n * n, sizeof(double));
        double *yr = malloc(sizeof(double) * N * N), *yi = malloc(sizeof(double) * N * N);
        double *I = malloc(sizeof(double) * N * N), *Ie = malloc(sizeof(double) * N * N);
        double *B = malloc(sizeof(double) * nd * nd), *C = malloc(sizeof(double) * nd * nd);
        const int per_slice = gs->is_lgs && gs->slices;
        const int ns = per_slice ? gs->n_na : 1;
        for (int k = 0; k < N * N; ++k) I[k] = 0.0;
        for (int sl = 0; sl < ns; ++sl) {
            /* the slice's source: the star's range replaced by the slice altitude (cone), and
               its geometric term relative to the focus at the star's range */
            orc_star src = *gs;
            double kgeo = 0.0, wsl = 1.0;
            if (per_slice) {
                src.range_m = gs->na_alt[sl];
                kgeo = 1.0 / gs->range_m - 1.0 / gs->na_alt[sl];
                wsl = gs->na_weight[sl];
            }
            /* field of the subaperture: a exp(i 2 pi OPD / lambda) */
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q) {
                    int i = sy * n + p, j = sx * n + q;
                    double x = (j - (Np - 1) / 2.0) * dx, y = (i - (Np - 1) / 2.0) * dx;
                    double o = orc_opd(L, screens, &src, x, y, t) + (upx * x + upy * y);
                    if (opd_out && sl == 0) opd_out[(size_t)s * n * n + p * n + q] = o;
                    if (per_slice) {
                        double ex = x - gs->launch_x, ey = y - gs->launch_y;
                        o += 0.5 * (ex * ex + ey * ey) * kgeo;
                    }
                    if (lit(g->diameter_m, g->obstruction, Np, i, j)) {
                        double phi = 2.0 * M_PI * o / gs->wavelength_m;
                        xr[p * n + q] = cos(phi);
                        xi[p * n + q] = sin(phi);
                    }
                }
            orc_dft2(n, N, xr, xi, yr, yi);
            /* the slice's spot weighted by the sodium profile, piled up */
            for (int k = 0; k < N * N; ++k) I[k] += wsl * (yr[k] * yr[k] + yi[k] * yi[k]);
        }
        if (gs->is_lgs) {
            double *K = malloc(sizeof(double) * N * N);
            double rbx = ((sx + 0.5) * n) * dx - g->diameter_m / 2.0;
            double rby = ((sy + 0.5) * n) * dx - g->diameter_m / 2.0;
            orc_star one = *gs;
            double h0 = gs->range_m, w1 = 1.0;
            if (per_slice) {
                /* the slices' offsets are in their wavefronts: the Gaussian extent alone */
                one.n_na = 1;
                one.na_alt = &h0;
                one.na_weight = &w1;
            }
            if (g_separable) {
                orc_elong_convolve_separable(N, pix_rad, rbx, rby, &one, I, Ie);
            } else {
                orc_elong_kernel(N, pix_rad, rbx, rby, &one, K);
                orc_convolve(N, I, K, Ie);
            }
            free(K);
        } else {
            memcpy(Ie, I, sizeof(double) * N * N);
        }
        orc_bin(N, nd, Ie, B);
        double sumB = 0.0;
        for (int k = 0; k < nd * nd; ++k) sumB += B[k];
        for (int k = 0; k < nd * nd; ++k)
            B[k] = sumB > 0.0 ? gs->photons * fill[v] * B[k] / sumB : 0.0;
        for (int k = 0; k < nd * nd; ++k) {
            if (noise)
                C[k] = orc_noise_pixel((float)B[k], (float)gs->read_noise, seed,
                                       (uint32_t)(v * nd * nd + k), (uint32_t)wfs_index, t, NULL);
            else
                C[k] = B[k];
        }
        orc_cog(nd, C, &slopes[2 * s], &slopes[2 * s + 1]);
        if (I_out) memcpy(I_out + (size_t)s * N * N, I, sizeof(double) * N * N);
        if (Ie_out) memcpy(Ie_out + (size_t)s * N * N, Ie, sizeof(double) * N * N);
        if (E_out) memcpy(E_out + (size_t)s * nd * nd, B, sizeof(double) * nd * nd);
        if (C_out) memcpy(C_out + (size_t)s * nd * nd, C, sizeof(double) * nd * nd);
        free(xr); free(xi); free(yr); free(yi); free(I); free(Ie); free(B); free(C);
    }
    free(idx);
    free(fill);
    return nv;
}
