// internal.h -- kernel argument blocks and launchers shared by the library's
// translation units (never installed; the public ABI is include/gbwfs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace gbwfs {

constexpr int kMaxGuideStars = 32;
constexpr int kMaxLayers = 32;
constexpr int kMaxNaSlices = 16;
constexpr int kMaxN = 64;       // largest DFT size
constexpr int kMaxNPix = 32;    // largest subaperture side in pupil pixels

// ---------------------------------------------------------------- projection
struct ProjWfs {
    const int32_t *subap;   // valid subaperture ids, sy * n_sub + sx
    float *opd;             // [n_valid][n * n] output
    int n, n_sub, n_valid, is_lgs;
    double range_m, theta_x, theta_y;
    double pupil_dx_over_ds;  // pupil pitch / screen pitch
    int block_begin;          // first CTA of this WFS in the launch
};

struct ProjArgs {
    const float *screens;     // [L][S][S]
    int n_layers, S;
    double ds, t;
    double alt[kMaxLayers], vx[kMaxLayers], vy[kMaxLayers], x0[kMaxLayers], y0[kMaxLayers];
    int n_wfs;
    ProjWfs w[kMaxGuideStars];
};

// ---------------------------------------------------------------- spot / slopes
struct ShWfs {
    const float *opd;         // [n_valid][n*n]
    const uint32_t *mask;     // [n_valid][mask_words] lit-pixel bits, bit p*n+q
    const float *fill;        // [n_valid]
    const float2 *ktil;       // [n_valid][(2n-1)*n] elongation transfer (LGS only)
    float *slopes;            // [n_valid][2]
    float *st_I, *st_E, *st_C;  // optional stage outputs
    int n_valid, is_lgs, gs_index, subap_begin;
    float k_phase;            // 2 pi / lambda
    float photons, read_noise;
};

struct ShArgs {
    int n, N, nd, mask_words;
    const float2 *F;    // [n][N]  F^T: F[q*N + m] = exp(-2 pi i (m-cN)(q-cn)/N)
    const float2 *Ga;   // [n][N]  Ga[d*N + k] = exp(+2 pi i (k-cN) d / N), d = 0..n-1
    const float2 *G;    // [n][nd] G[d*nd + i] = sum_{r<b} exp(-2 pi i (b i + r - cN) d / N)
    int n_wfs, total;
    uint64_t seed;
    int noise;
    double t;
    int *status;
    // tensor-core operand tiles (BF16, pre-swizzled), used by the BF16X3 kernel only
    const void *tc_B1, *tc_B2h, *tc_B2l;
    ShWfs w[kMaxGuideStars];
};

// ---------------------------------------------------------------- elongation tables
struct KtilArgs {
    const int32_t *subap;
    float2 *ktil;
    int n, N, n_sub, n_valid, n_na;
    double D, dx, pix_rad, sigma_px, launch_x, launch_y, h0;
    double alt[kMaxNaSlices], w[kMaxNaSlices];
};

// Launchers (return the cudaGetLastError() of the launch).
cudaError_t launch_project(const ProjArgs &a, int total_blocks, cudaStream_t s);
// CTAs the projection needs for `pixels` pupil pixels of one WFS.
int project_blocks(int pixels);
cudaError_t launch_sh_fp32(const ShArgs &a, cudaStream_t s);
cudaError_t launch_ktil(const KtilArgs &a, cudaStream_t s);
// Compile-time specialised FP32 spot kernel for N = 32 geometries.
bool sh_n32_supported(int n, int N, int nd);
cudaError_t launch_sh_n32(const ShArgs &a, cudaStream_t s);
// Tensor-core (tcgen05, BF16 x3) spot kernel for N = 32 geometries with n <= 10.
bool sh_tc_supported(int n, int N, int nd);
cudaError_t launch_sh_tc(const ShArgs &a, cudaStream_t s);
// Swizzled BF16 operand tiles of the two constant matrices (F^T blocks, Ga blocks),
// from FP64 tables laid out [q][m] (F) and [d][k] (Ga).
void build_tc_tiles(int n, int N, const double *F_re64, const double *F_im64, const double *Ga_re64,
                    const double *Ga_im64, std::vector<uint8_t> &B1, std::vector<uint8_t> &B2h,
                    std::vector<uint8_t> &B2l);
cudaError_t launch_noise(const float *E, int n, float ron, uint64_t seed, uint32_t wfs, double t,
                         uint32_t pixel0, float *C, cudaStream_t s);
size_t sh_fp32_smem_bytes(int n, int N, int nd, int *team_threads, int *teams_per_cta);
// Sets the calling thread's message returned by wfs_last_error(NULL).
void set_thread_error(const char *msg);

}  // namespace gbwfs
