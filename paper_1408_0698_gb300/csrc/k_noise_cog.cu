// k_noise_cog.cu -- the detector noise and the centroid of the 32-point spot kernels' subapertures
// from their stored expected images (Sec. 4: the centroid is taken on the final noise-added
// image).  The spot kernels then stop after the photometry; this kernel gives the divergent
// Poisson searches warps of their own instead of holding a warpgroup's tensor-core pipeline in
// step with its slowest warp.  The arithmetic is the spot kernels' own (tail::noise_centroid on
// the same expected values), so the counts and slopes are those of the single-pass kernels.
//
// One warp per subaperture, eight per CTA; CTAs of launch order follow the spot kernel through
// a programmatic dependent launch and wait for it before reading the expected images.
#include "internal.h"
#include "noise.cuh"
#include "spot_tail.cuh"

namespace gbwfs {

namespace {
constexpr int kNcWarps = 8;
}

template <int nd>
__global__ void __launch_bounds__(32 * kNcWarps, 4) k_noise_cog(const __grid_constant__ ShArgs a) {
    __shared__ float rk[kRecipTable];
    fill_recip_table(rk, threadIdx.x, blockDim.x);
    __syncthreads();
    wait_prior_grid();
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * kNcWarps + (threadIdx.x >> 5);
    if (g >= a.total) return;
    const WfsDesc &W = a.wfs[find_wfs(a.wfs, a.n_wfs, g)];
    const InstDyn &D = a.dyn[W.inst];
    const int v = g - W.subap_begin;
    if (!guard(v >= 0 && v < W.n_valid, a.status)) return;
    constexpr int J = nd / 2;
    const int ix = lane & 15, half = lane >> 4;
    const float *E = D.st_E + W.det_off + (size_t)v * (nd * nd);
    float ev[J];
#pragma unroll
    for (int j = 0; j < J; ++j) ev[j] = E[(half * J + j) * nd + ix];
    tail::noise_centroid<nd>(ev, W, D, a.inst[W.inst].seed, v, lane, rk);
}

cudaError_t noise_cog_launch_shape(const ShArgs &a, LaunchShape *out) {
    if (a.nd != 16) return cudaErrorInvalidValue;
    out->func = (const void *)k_noise_cog<16>;
    out->grid = dim3((a.total + kNcWarps - 1) / kNcWarps);
    out->block = dim3(32 * kNcWarps);
    out->smem = 0;
    return cudaSuccess;
}

cudaError_t launch_noise_cog(const ShArgs &a, cudaStream_t s, bool after_spot) {
    if (a.total <= 0) return cudaSuccess;
    LaunchShape sh;
    cudaError_t e = noise_cog_launch_shape(a, &sh);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    if (!after_spot) return cudaLaunchKernel(sh.func, sh.grid, sh.block, args, sh.smem, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = sh.grid;
    cfg.blockDim = sh.block;
    cfg.dynamicSmemBytes = sh.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, sh.func, args);
}

}  // namespace gbwfs
