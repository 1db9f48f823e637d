// proj_math.cuh -- the arithmetic of the layered frozen-flow projection shared by the
// projection kernel and the spot kernel that projects its own subapertures (Sec. 4 "Open Loop
// generation": the layers' screens are piled up, each shifted for the star's direction and the
// temporal evolution; for an LGS the footprint shrinks with altitude, c = 1 - h / range).
//
// For pupil pixel x (metres from the pupil centre) and layer l the sampled screen coordinate,
// in screen pixels from the screen origin, is
//     u = S/2 + (c_l x + theta h_l - (x0_l + v_l t)) / ds
// split as  u = [S/2 + (theta h_l - x0_l - v_l t)/ds]  +  c_l (dx/ds) j'
// where j' is the pixel's half-integer column offset from the pupil centre.  The first
// (time-dependent, possibly large) term is evaluated in FP64 and split into an integer base
// (mod S) and an FP32 fraction; the per-pixel term uses FP32 only, with the scale c_l dx/ds
// held as two floats (hi + lo) and its product with j' split exactly by an FMA.
#pragma once
#include "internal.h"

namespace gbwfs {

struct LayerOffs {
    int bu, bv;    // integer base of the layer's offset, mod S (columns, rows)
    float fu, fv;  // its fractional part
    float c, cl;   // c_l dx / ds as hi + lo
};

// Layers a projection of instance (I, D) sums: the turbulent screens, then the mirrors'
// correction layers.
__device__ __forceinline__ int proj_layers(const InstDesc &I, const InstDyn &D) { return I.n_layers + D.n_dm; }

// The S x S array of layer l.
__device__ __forceinline__ const float *layer_screen(const InstDesc &I, const InstDyn &D, int l) {
    const size_t SS = (size_t)I.S * I.S;
    return l < I.n_layers ? D.screens + (size_t)l * SS : D.dm + (size_t)(l - I.n_layers) * SS;
}

// Layer l's offsets for WFS W at time t (FP64).
__device__ __forceinline__ LayerOffs layer_offsets(const InstDesc &I, const WfsDesc &W, double t, int l) {
    const int S = I.S;
    const double h = I.alt[l];
    const double c = W.is_lgs ? 1.0 - h / W.range_m : 1.0;
    const double inv_ds = 1.0 / I.ds;
    const double ou = 0.5 * S + (W.theta_x * h - (I.x0[l] + I.vx[l] * t)) * inv_ds;
    const double ov = 0.5 * S + (W.theta_y * h - (I.y0[l] + I.vy[l] * t)) * inv_ds;
    const double bu = floor(ou), bv = floor(ov);
    LayerOffs o;
    o.fu = (float)(ou - bu);
    o.fv = (float)(ov - bv);
    // base index mod S (exact: bu, bv are integers well inside 2^53)
    long long iu = (long long)bu % S, iv = (long long)bv % S;
    if (iu < 0) iu += S;
    if (iv < 0) iv += S;
    o.bu = (int)iu;
    o.bv = (int)iv;
    const double cs = c * W.pupil_dx_over_ds;
    o.c = (float)cs;
    o.cl = (float)(cs - (double)o.c);
    return o;
}

// One screen coordinate of half-integer pupil offset x: the integer offset from the layer base
// (ih + iu) and the interpolation fraction.
__device__ __forceinline__ void screen_offset(float ch, float cl, float f, float x, int &off, float &frac) {
    // c * x = ph + pl exactly (to FP32 rounding of the small part)
    const float ph = __fmul_rn(ch, x), pl = fmaf(ch, x, -ph) + cl * x;
    const float ih = floorf(ph);
    const float r = ((ph - ih) + pl) + f;  // in [-eps, 2)
    const float ir = floorf(r);
    off = (int)ih + (int)ir;
    frac = r - ir;
}

// Screen index b + off and its successor, wrapped into [0, S).  |c x / ds| < S is enforced when
// the handle is created, so one wrap suffices.
__device__ __forceinline__ void wrap_pair(int i, int S, bool pow2, int &i0, int &i1) {
    if (pow2) {
        i0 = i & (S - 1);
        i1 = (i0 + 1) & (S - 1);
    } else {
        i += (i < 0) ? S : 0;
        i -= (i >= S) ? S : 0;
        i0 = i;
        i1 = (i0 + 1 == S) ? 0 : i0 + 1;
    }
}

}  // namespace gbwfs
