/*
 * measure_frame.c -- one Shack-Hartmann frame through the C ABI from plain C99.
 *
 * The sensor: an 8 m telescope, one on-axis natural guide star at 700 nm (500 photons per
 * subaperture, 3 e- read noise), 20 x 20 subapertures of 8 x 8 pupil pixels, DFT padded to
 * 16 x 16, 8 x 8 detector pixels, FP32 arithmetic; one turbulent layer at the ground moving at
 * 10 m/s along x, a 256 x 256 screen of 0.05 m pixels.
 *
 * Usage: measure_frame SCREEN.f32 T_S SLOPES.f32 [NOISE]
 *   SCREEN.f32  256 * 256 float32 OPD samples in metres (row-major), read from a file
 *   T_S         frame time in seconds
 *   SLOPES.f32  output: n_valid * 2 float32 slopes in detector pixels (x, y per subaperture)
 *   NOISE       1 for Poisson and read noise (seed 1), default 0
 * Exit status 0 on success; otherwise the library's or CUDA's message goes to stderr.
 *
 * Build: gcc -std=c99 -I include measure_frame.c -L <dir of libgbwfs.so> -lgbwfs
 *        -I <CUDA include> -L <CUDA lib64> -lcudart
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "gbwfs.h"

enum { S = 256 };

static int cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return 0;
    fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
    return 1;
}

int main(int argc, char **argv) {
    if (argc < 4) {
        fprintf(stderr, "usage: %s SCREEN.f32 T_S SLOPES.f32 [NOISE]\n", argv[0]);
        return 2;
    }
    const double t = atof(argv[2]);
    const int noise = argc > 4 ? atoi(argv[4]) : 0;

    float *screen = (float *)malloc(sizeof(float) * S * S);
    FILE *f = fopen(argv[1], "rb");
    if (!screen || !f || fread(screen, sizeof(float), S * S, f) != (size_t)(S * S)) {
        fprintf(stderr, "cannot read %d floats from %s\n", S * S, argv[1]);
        return 2;
    }
    fclose(f);

    const wfs_telescope tel = {8.0, 0.0};
    const wfs_geometry geom = {20, 8, 16, 8, 0.5, WFS_PREC_FP32};
    wfs_guide_star ngs = {0};
    ngs.is_lgs = 0;
    ngs.range_m = INFINITY; /* at infinity */
    ngs.wavelength_m = 700e-9;
    ngs.photons_per_subap = 500.0;
    ngs.read_noise_e = 3.0;
    ngs.geometry_index = 0;
    const double alt = 0.0, vx = 10.0, vy = 0.0, x0 = 0.0, y0 = 0.0;
    const wfs_layers layers = {1, S, 0.05, &alt, &vx, &vy, &x0, &y0};

    wfs_handle h = NULL;
    wfs_status st = wfs_create(&tel, 1, &ngs, 1, &geom, &layers, 1, noise, &h);
    if (st != WFS_OK) {
        fprintf(stderr, "wfs_create: status %d: %s\n", (int)st, wfs_last_error(NULL));
        return 1;
    }
    int n = 0;
    wfs_total_valid(h, &n);

    float *d_screen = NULL, *d_slopes = NULL;
    float *slopes = (float *)malloc(sizeof(float) * 2 * (size_t)n);
    int rc = 1;
    if (cuda_check(cudaMalloc((void **)&d_screen, sizeof(float) * S * S), "cudaMalloc") ||
        cuda_check(cudaMalloc((void **)&d_slopes, sizeof(float) * 2 * (size_t)n), "cudaMalloc") ||
        cuda_check(cudaMemcpy(d_screen, screen, sizeof(float) * S * S, cudaMemcpyHostToDevice), "upload"))
        goto done;
    st = wfs_measure(h, d_screen, t, d_slopes, NULL);
    if (st != WFS_OK) {
        fprintf(stderr, "wfs_measure: status %d: %s\n", (int)st, wfs_last_error(h));
        goto done;
    }
    if (cuda_check(cudaMemcpy(slopes, d_slopes, sizeof(float) * 2 * (size_t)n, cudaMemcpyDeviceToHost), "download"))
        goto done;
    st = wfs_sync_status(h);
    if (st != WFS_OK) {
        fprintf(stderr, "device status %d: %s\n", (int)st, wfs_last_error(h));
        goto done;
    }
    f = fopen(argv[3], "wb");
    if (!f || fwrite(slopes, sizeof(float), 2 * (size_t)n, f) != 2 * (size_t)n) {
        fprintf(stderr, "cannot write %s\n", argv[3]);
        goto done;
    }
    fclose(f);
    printf("%d subapertures measured at t = %g s\n", n, t);
    rc = 0;
done:
    cudaFree(d_screen);
    cudaFree(d_slopes);
    wfs_destroy(h);
    free(slopes);
    free(screen);
    return rc;
}
