// k_uplink.cu -- the LGS uplink tip-tilt (Sec. 4 "Open Loop generation": the laser's
// projection on the sodium layer is computed with the spot shift induced by the tip-tilt
// integrated over the upward path), per frame, before the projection adds it to the pupil OPD.
#include "internal.h"
#include "proj_math.cuh"

namespace gbwfs {

// LGS uplink tip-tilt (Sec. 4 Open Loop generation: the laser's projection on the sodium layer
// is shifted by the tip-tilt integrated over the upward path).  CTA (w, l): WFS w of the table
// (those with the uplink on), turbulent layer l (mirror layers are not crossed).  The beam
// (diameter up_diam) runs from the launch point on the ground to theta * range; at the layer it
// is deflected by the plane-fit slope of the layer's OPD over its footprint, up_n^2 points on a
// square grid of pitch up_diam / up_n inside the disc, sampled like the projection (FP64 layer
// offset split into an integer base and an FP32 fraction); the deflection acts over the rest of
// the way up, (range - h) / range.  The sample set is symmetric, so the slope is
// sum(o v) / sum(o^2).  The last CTA of a WFS to finish adds the layers' parts in layer order
// (fixed-order sums throughout) and resets the WFS's counter.
__global__ void __launch_bounds__(256) k_uplink(const InstDesc *__restrict__ inst, const WfsDesc *__restrict__ wfs,
                                                double2 *part, int *count, const __grid_constant__ InstDyn d0) {
    allow_dependent_grid();  // the projection may start; it waits for this grid before adding the tilt
    const int wi = blockIdx.x, l = blockIdx.y;
    const WfsDesc &W = wfs[wi];
    if (!W.uplink || !W.is_lgs) return;
    const InstDesc &I = inst[W.inst];
    if (l >= I.n_layers) return;
    const int S = I.S, n = W.up_n, t = threadIdx.x;
    const bool pow2 = (S & (S - 1)) == 0;
    const double H = W.range_m, h = I.alt[l];
    // the layer's footprint geometry, once per CTA (FP64 is slow: one thread does it)
    __shared__ int s_iu, s_iv;
    __shared__ float s_fu, s_fv, s_pitch, s_r2, s_inv_ds;
    if (t == 0 && h < H) {
        const double cx = W.launch_x * (1.0 - h / H) + W.theta_x * h;
        const double cy = W.launch_y * (1.0 - h / H) + W.theta_y * h;
        const double ou = 0.5 * S + (cx - (I.x0[l] + I.vx[l] * d0.t)) / I.ds;
        const double ov = 0.5 * S + (cy - (I.y0[l] + I.vy[l] * d0.t)) / I.ds;
        const double bu = floor(ou), bv = floor(ov);
        s_fu = (float)(ou - bu);
        s_fv = (float)(ov - bv);
        long long iu = (long long)bu % S, iv = (long long)bv % S;
        if (iu < 0) iu += S;
        if (iv < 0) iv += S;
        s_iu = (int)iu;
        s_iv = (int)iv;
        s_pitch = (float)(W.up_diam / n);
        s_r2 = (float)(0.25 * W.up_diam * W.up_diam);
        s_inv_ds = (float)(1.0 / I.ds);
    }
    __syncthreads();
    // FP64 sums: the samples carry the layer's local piston, which the symmetric offsets cancel
    double sxv = 0.0, syv = 0.0, sxx = 0.0, syy = 0.0;
    if (h < H) {
        const int iu = s_iu, iv = s_iv;
        const float fu = s_fu, fv = s_fv, pitch = s_pitch, r2 = s_r2, inv_ds = s_inv_ds;
        const float *scr = d0.screens + (size_t)l * S * S;
        for (int e = t; e < n * n; e += 256) {
            const int i = e / n, j = e - i * n;
            const float ox = ((float)j - 0.5f * (float)(n - 1)) * pitch;
            const float oy = ((float)i - 0.5f * (float)(n - 1)) * pitch;
            if (ox * ox + oy * oy > r2) continue;
            const float u = fu + ox * inv_ds, v = fv + oy * inv_ds;
            const float uf = floorf(u), vf = floorf(v);
            int i0, i1, j0, j1;
            wrap_pair((int)iu + (int)uf, S, pow2, i0, i1);
            wrap_pair((int)iv + (int)vf, S, pow2, j0, j1);
            const float a = u - uf, b = v - vf;
            const float *r0 = scr + (size_t)j0 * S, *r1 = scr + (size_t)j1 * S;
            const float s00 = __ldg(r0 + i0), s01 = __ldg(r0 + i1), s10 = __ldg(r1 + i0), s11 = __ldg(r1 + i1);
            const float top = fmaf(a, s01 - s00, s00), bot = fmaf(a, s11 - s10, s10);
            const float val = fmaf(b, bot - top, top);
            sxv = fma((double)ox, (double)val, sxv);
            syv = fma((double)oy, (double)val, syv);
            sxx = fma((double)ox, (double)ox, sxx);
            syy = fma((double)oy, (double)oy, syy);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sxv += __shfl_xor_sync(0xffffffffu, sxv, o);
        syv += __shfl_xor_sync(0xffffffffu, syv, o);
        sxx += __shfl_xor_sync(0xffffffffu, sxx, o);
        syy += __shfl_xor_sync(0xffffffffu, syy, o);
    }
    __shared__ double red[4][8];
    __shared__ int s_last;
    if ((t & 31) == 0) {
        red[0][t >> 5] = sxv;
        red[1][t >> 5] = syv;
        red[2][t >> 5] = sxx;
        red[3][t >> 5] = syy;
    }
    __syncthreads();
    if (t == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        for (int w = 0; w < 8; ++w) {
            a0 += red[0][w];
            a1 += red[1][w];
            a2 += red[2][w];
            a3 += red[3][w];
        }
        const double arm = (H - h) / H;
        part[wi * kMaxLayers + l] = h < H ? make_double2(a0 / a2 * arm, a1 / a3 * arm) : make_double2(0.0, 0.0);
        __threadfence();
        s_last = atomicAdd(count + wi, 1) == I.n_layers - 1;
    }
    __syncthreads();
    if (s_last && t == 0) {
        __threadfence();
        double dx = 0.0, dy = 0.0;
        for (int k = 0; k < I.n_layers; ++k) {
            const double2 p = __ldcg(part + wi * kMaxLayers + k);
            dx += p.x;
            dy += p.y;
        }
        const double px = W.pupil_dx_over_ds * I.ds;  // pupil pitch (m)
        *W.uplink = make_float2((float)(dx * px), (float)(dy * px));
        count[wi] = 0;
    }
}

cudaError_t launch_uplink(const InstDesc *inst, const WfsDesc *wfs, int n_wfs, int max_layers, double2 *part,
                          int *count, const InstDyn *dyn0, cudaStream_t s) {
    if (n_wfs <= 0 || max_layers <= 0) return cudaSuccess;
    k_uplink<<<dim3(n_wfs, max_layers), 256, 0, s>>>(inst, wfs, part, count, *dyn0);
    return cudaGetLastError();
}

}  // namespace gbwfs
