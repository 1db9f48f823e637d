// k_loop.cu -- the per-step kernels of the closed loop (Sec. 3 "The closed loop": the slopes
// times the control matrix are the differential modal coefficients added to the mirror's, a
// pure integrator; Sec. 3 "Influence function and modal base": a mirror is a combination of a
// modal base over its actuators' influence functions).
//
//   k_gemv      y = A x for a row-major FP32 matrix, optionally followed by the integrator
//               c += gain * y on the same rows.  Used for the reconstruction (A = control
//               matrix, x = slopes) and for the actuator commands (A = modal base, x = the
//               mirror's coefficients).  HBM-bound: the matrix is streamed once.
//   k_dm_layer  a mirror's correction layer (minus its shape) on the atmospheric screen grid,
//               over the window its influence functions reach.
#include "internal.h"
#include "proj_math.cuh"

namespace gbwfs {

namespace {
constexpr int kGemvThreads = 256;
constexpr int kGemvRows = 4;  // rows per CTA: each x chunk loaded serves four rows
}

// Four rows per CTA.  All threads walk the rows' 16-byte chunks in step, so each warp reads
// 512 contiguous bytes of every row per iteration (streaming loads: the matrix is read once),
// the NB vectors come through the read-only path; the CTA then reduces its partial sums in a
// fixed order.  Each (row, vector) pair accumulates in the same order whatever NB is, so a
// vector's result does not depend on the others it shares the launch with.
template <int NB, bool kVec>
__global__ void __launch_bounds__(kGemvThreads) k_gemv(const __grid_constant__ GemvMultiArgs a) {
    const int r0 = blockIdx.x * kGemvRows;
    float acc[kGemvRows][NB];
#pragma unroll
    for (int r = 0; r < kGemvRows; ++r)
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[r][b] = 0.0f;
    const float *rows[kGemvRows];
#pragma unroll
    for (int r = 0; r < kGemvRows; ++r) rows[r] = a.A + (size_t)min(r0 + r, a.rows - 1) * a.cols;
    if (kVec) {
        const int n4 = a.cols >> 2;
#pragma unroll 2
        for (int k = threadIdx.x; k < n4; k += kGemvThreads) {
            float4 xv[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) xv[b] = __ldg(reinterpret_cast<const float4 *>(a.x[b]) + k);
#pragma unroll
            for (int r = 0; r < kGemvRows; ++r) {
                const float4 v = __ldcs(reinterpret_cast<const float4 *>(rows[r]) + k);
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    acc[r][b] = fmaf(v.x, xv[b].x, acc[r][b]);
                    acc[r][b] = fmaf(v.y, xv[b].y, acc[r][b]);
                    acc[r][b] = fmaf(v.z, xv[b].z, acc[r][b]);
                    acc[r][b] = fmaf(v.w, xv[b].w, acc[r][b]);
                }
            }
        }
    } else {
        for (int k = threadIdx.x; k < a.cols; k += kGemvThreads) {
            float xv[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) xv[b] = __ldg(a.x[b] + k);
#pragma unroll
            for (int r = 0; r < kGemvRows; ++r) {
                const float v = __ldcs(rows[r] + k);
#pragma unroll
                for (int b = 0; b < NB; ++b) acc[r][b] = fmaf(v, xv[b], acc[r][b]);
            }
        }
    }
    __shared__ float part[kGemvThreads / 32][kGemvRows][NB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < kGemvRows; ++r)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            float v = acc[r][b];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) part[warp][r][b] = v;
        }
    __syncthreads();
    if (threadIdx.x < kGemvRows * NB) {
        const int r = threadIdx.x % kGemvRows, b = threadIdx.x / kGemvRows, row = r0 + r;
        float y = 0.0f;
#pragma unroll
        for (int w = 0; w < kGemvThreads / 32; ++w) y += part[w][r][b];
        if (row < a.rows) {
            if (a.y[b]) a.y[b][row] = y;
            if (a.c[b]) a.c[b][row] = fmaf(a.gain[b][row], y, a.c[b][row]);
        }
    }
}

namespace {
template <int NB>
const void *gemv_func(bool vec) {
    return vec ? (const void *)k_gemv<NB, true> : (const void *)k_gemv<NB, false>;
}
}  // namespace

cudaError_t launch_gemv_multi(const GemvMultiArgs &a, cudaStream_t s) {
    if (a.rows <= 0 || a.nb <= 0) return cudaSuccess;
    if (a.nb > kMaxGemvVec) return cudaErrorInvalidValue;
    const bool vec = (a.cols & 3) == 0 && ((uintptr_t)a.A & 15) == 0;
    bool aligned = true;
    for (int b = 0; b < a.nb; ++b) aligned = aligned && ((uintptr_t)a.x[b] & 15) == 0;
    if (vec && !aligned && a.nb > 1) {
        // a vector off the 16-byte grid: each vector alone, so that each keeps the summation
        // order a single-vector launch would give it
        for (int b = 0; b < a.nb; ++b) {
            GemvMultiArgs one = a;
            one.nb = 1;
            one.x[0] = a.x[b];
            one.y[0] = a.y[b];
            one.gain[0] = a.gain[b];
            one.c[0] = a.c[b];
            const cudaError_t e = launch_gemv_multi(one, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const void *f = nullptr;
    switch (a.nb) {
        case 1: f = gemv_func<1>(vec && aligned); break;
        case 2: f = gemv_func<2>(vec && aligned); break;
        case 3: f = gemv_func<3>(vec && aligned); break;
        default: f = gemv_func<4>(vec && aligned); break;
    }
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(f, dim3((a.rows + kGemvRows - 1) / kGemvRows), dim3(kGemvThreads), args, 0, s);
}

namespace {
GemvMultiArgs one_vector(const GemvArgs &a) {
    GemvMultiArgs m{};
    m.A = a.A;
    m.rows = a.rows;
    m.cols = a.cols;
    m.nb = 1;
    m.x[0] = a.x;
    m.y[0] = a.y;
    m.gain[0] = a.gain;
    m.c[0] = a.c;
    return m;
}
}  // namespace

cudaError_t gemv_launch_shape(const GemvArgs &a, LaunchShape *out) {
    const bool vec = (a.cols & 3) == 0 && ((uintptr_t)a.A & 15) == 0 && ((uintptr_t)a.x & 15) == 0;
    out->func = gemv_func<1>(vec);
    out->grid = dim3((a.rows + kGemvRows - 1) / kGemvRows);
    out->block = dim3(kGemvThreads);
    out->smem = 0;
    return cudaSuccess;
}

cudaError_t launch_gemv(const GemvArgs &a, cudaStream_t s) { return launch_gemv_multi(one_vector(a), s); }

// A CTA computes a 32-column x 64-row tile of the window in two separable passes: first
// T[ay][j] = sum_ax act[ay][ax] w(u_x(j) - ax) for the actuator rows the tile's rows reach, then
// layer[i][j] = -sum_ay w(u_y(i) - ay) T[ay][j].  A pixel's fractional actuator coordinate
// u = (j - S/2) ds / p + c comes from the projection's exact two-float product (ds / p held as
// hi + lo), split into an integer actuator and a fraction; the 2R + 2 actuators per axis around
// it get the weights w(u) = max(0, k^(u^2) - k^(R^2)) / (1 - k^(R^2)).  Actuators off the grid
// get weight zero (their index is clamped to a valid one).  The actuator pitch is at least the
// screen pitch, so the tile's 64 rows reach at most 64 + 2R + 2 actuator rows.
namespace {
constexpr int kDmTx = 32, kDmTy = 64;
constexpr int kDmW = 2 * kMaxDmSupport + 2;     // weights per pixel and axis
constexpr int kDmRows = kDmTy + kDmW;           // actuator rows a tile reaches
}

__device__ __forceinline__ void dm_axis_weights(const DmLayerArgs &a, int pix, int &base, float *w) {
    int off;
    float frac;
    screen_offset(a.r_hi, a.r_lo, a.c_frac, (float)(pix - a.S / 2), off, frac);
    base = off + a.c_int - a.support;  // first actuator of the 2R + 2
    const int nw = 2 * a.support + 2;
    for (int k = 0; k < nw; ++k) {
        const float u = frac + (float)(a.support - k);  // pixel minus actuator base + k, in pitches
        const float g = exp2f(u * u * a.log2k) - a.edge;
        const int ac = base + k;
        w[k] = (g > 0.0f && ac >= 0 && ac < a.n_act) ? g * a.inv_norm : 0.0f;
    }
}

// blockIdx.z: the layer of the batch; the grid covers the largest window, CTAs past a smaller
// one leave at once.
__global__ void __launch_bounds__(256) k_dm_layer(const __grid_constant__ DmLayerBatch b) {
    __shared__ float cw[kDmTx][kDmW], rw[kDmTy][kDmW], T[kDmRows][kDmTx];
    __shared__ int cb[kDmTx], rb[kDmTy];
    const DmLayerArgs &a = b.l[blockIdx.z];
    if ((int)blockIdx.x * kDmTx >= a.w || (int)blockIdx.y * kDmTy >= a.h) return;
    const int j0 = a.x0 + blockIdx.x * kDmTx, i0 = a.y0 + blockIdx.y * kDmTy;
    const int nw = 2 * a.support + 2;
    const int t = threadIdx.x;
    if (t < kDmTx) dm_axis_weights(a, j0 + t, cb[t], cw[t]);
    else if (t < kDmTx + kDmTy) dm_axis_weights(a, i0 + t - kDmTx, rb[t - kDmTx], rw[t - kDmTx]);
    __syncthreads();
    // pass 1: the actuator rows ay_lo .. ay_lo + nr - 1 the tile's rows reach
    const int ay_lo = rb[0];
    const int nr = min(rb[kDmTy - 1] + nw - ay_lo, kDmRows);
    for (int e = t; e < nr * kDmTx; e += 256) {
        const int r = e / kDmTx, jj = e - r * kDmTx;
        const int ay = ay_lo + r;
        float acc = 0.0f;
        if (ay >= 0 && ay < a.n_act) {
            const float *row = a.act + (size_t)ay * a.n_act * a.act_stride;
            for (int k = 0; k < nw; ++k) {
                const int ax = min(max(cb[jj] + k, 0), a.n_act - 1);
                acc = fmaf(__ldg(row + (size_t)ax * a.act_stride), cw[jj][k], acc);
            }
        }
        T[r][jj] = acc * a.act_scale;
    }
    __syncthreads();
    // pass 2: one column per lane, 8 rows per warp step
    const int jj = t & 31, j = j0 + jj;
    if (j >= a.x0 + a.w) return;
    for (int ii = t >> 5; ii < kDmTy; ii += 8) {
        const int i = i0 + ii;
        if (i >= a.y0 + a.h) break;
        const int r0 = rb[ii] - ay_lo;
        float sum = 0.0f;
        for (int k = 0; k < nw; ++k) sum = fmaf(rw[ii][k], T[r0 + k][jj], sum);
        a.layer[(size_t)i * a.S + j] = -sum;  // the mirror takes its shape out of the beam
    }
}

cudaError_t launch_dm_layers(const DmLayerBatch &b, cudaStream_t s) {
    if (b.n <= 0) return cudaSuccess;
    if (b.n > kMaxInstances) return cudaErrorInvalidValue;
    int gx = 0, gy = 0;
    for (int i = 0; i < b.n; ++i) {
        const DmLayerArgs &a = b.l[i];
        if (a.support < 1 || a.support > kMaxDmSupport || !(a.r_hi <= 1.0f) || a.w < 0 || a.h < 0)
            return cudaErrorInvalidValue;
        gx = max(gx, (a.w + kDmTx - 1) / kDmTx);
        gy = max(gy, (a.h + kDmTy - 1) / kDmTy);
    }
    if (gx == 0 || gy == 0) return cudaSuccess;
    void *args[] = {(void *)&b};
    return cudaLaunchKernel((const void *)k_dm_layer, dim3(gx, gy, b.n), dim3(256), args, 0, s);
}

__global__ void k_push_pull_rows(const float *__restrict__ s, int n_modes, int n_slopes, float inv_2a,
                                 float *__restrict__ im) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n_modes * n_slopes) return;
    const int k = (int)(e / n_slopes), j = (int)(e - (long long)k * n_slopes);
    const float *push = s + (size_t)(2 * k) * n_slopes, *pull = push + n_slopes;
    im[e] = (push[j] - pull[j]) * inv_2a;
}

cudaError_t launch_push_pull_rows(const float *s, int n_modes, int n_slopes, float inv_2a, float *im,
                                  cudaStream_t st) {
    const long long n = (long long)n_modes * n_slopes;
    if (n <= 0) return cudaSuccess;
    k_push_pull_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, n_modes, n_slopes, inv_2a, im);
    return cudaGetLastError();
}

}  // namespace gbwfs
