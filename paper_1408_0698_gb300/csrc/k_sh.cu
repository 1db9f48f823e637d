// k_sh.cu -- the Shack-Hartmann spot, elongation, binning, noise and
// centroid of every valid subaperture (Sec. 4 "LGS Shack Hartmann wavefront
// sensor"), plain-FP32 path on the CUDA cores.
//
// Per subaperture (one team of threads, everything in shared memory):
//   X  = a exp(i 2 pi (OPD - OPD_0) / lambda)          field (piston-free)
//   Y  = F X F^T,  F[k][p] = exp(-2 pi i (k-cN)(p-cn)/N) centred, zero-padded DFT
//   I  = |Y|^2
//   LGS: B = bin(I (*) K) computed exactly through the transfer function:
//        with A[d] = (1/N^2) sum_k I[k] exp(+2 pi i (k-cN).d/N)  (the spot's
//        autocorrelation; I is band-limited to |d| <= n-1 when N >= 2n-1),
//        B[i] = Re sum_{dy, dx>=0} c_dx A[d] Kt[d] G[iy][dy] G[ix][dx],
//        Kt[d] = sum_m K[m] exp(+2 pi i m.d/N), G[i][d] = sum_{r<b} w^{(b i+r-cN) d}
//        (w = exp(-2 pi i/N), c_0 = 1, c_dx>0 = 2 by Hermitian symmetry).
//        This equals binning the periodic convolution I (*) K exactly.
//   NGS: B = b x b binning of I.
//   E  = photons * fill * B / sum(B);  C = Poisson(E) + ron z  (or C = E)
//   slope = sum (x - c) C / sum C,  c = (nd-1)/2,  in detector pixels.
// The piston subtraction (OPD_0 = the subaperture's first OPD sample) leaves
// |Y|^2 unchanged exactly and keeps the FP32 phase small.
#include <string.h>

#include "internal.h"
#include "noise.cuh"
#include "proj_math.cuh"

namespace gbwfs {

__host__ __device__ inline int odd_up(int x) { return x | 1; }

// Shared-memory floats used by one team; the same formula sizes the launch.
__host__ __device__ inline int team_floats(int n, int N, int nd, int team) {
    const int D2 = 2 * n - 1;
    int ri = N * (N + 1);
    ri += ri & 1;
    int r1 = 2 * n * n;
    r1 = r1 > 2 * N * odd_up(n) ? r1 : 2 * N * odd_up(n);
    r1 = r1 > 2 * D2 * nd ? r1 : 2 * D2 * nd;
    int r2 = 2 * N * n;
    r2 = r2 > 2 * D2 * n ? r2 : 2 * D2 * n;
    r2 = r2 > nd * nd ? r2 : nd * nd;
    r2 += r2 & 1;
    const int red = 4 * (team / 32) + 4;
    return ri + r1 + r2 + red + 6 * kMaxProjLayers;  // then the layer offsets of a fused projection
}

template <int TEAM>
__device__ __forceinline__ void team_sync(int team) {
    if (TEAM == 32)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(TEAM) : "memory");
}

template <int TEAM>
__device__ __forceinline__ void team_sum3(float &x, float &y, float &z, float *red, int tid,
                                          int team) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
        z += __shfl_xor_sync(0xffffffffu, z, o);
    }
    if (TEAM > 32) {
        const int wi = tid >> 5;
        if ((tid & 31) == 0) {
            red[3 * wi] = x;
            red[3 * wi + 1] = y;
            red[3 * wi + 2] = z;
        }
        team_sync<TEAM>(team);
        x = y = z = 0.0f;
        for (int i = 0; i < TEAM / 32; ++i) {
            x += red[3 * i];
            y += red[3 * i + 1];
            z += red[3 * i + 2];
        }
        team_sync<TEAM>(team);
    }
}

__device__ __forceinline__ float2 cmac(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
    return acc;
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

template <int TEAM>
__global__ void __launch_bounds__(TEAM > 256 ? TEAM : 256) k_sh_fp32(const __grid_constant__ ShArgs a) {
    extern __shared__ __align__(16) float smem[];
    const int n = a.n, N = a.N, nd = a.nd, nn = n * n, D2 = 2 * n - 1, no = odd_up(n);
    float2 *sF = reinterpret_cast<float2 *>(smem);  // [q][m]
    float2 *sGa = sF + n * N;                       // [d][k]
    float2 *sG = sGa + n * N;                       // [d][i]
    for (int i = threadIdx.x; i < n * N; i += blockDim.x) {
        sF[i] = a.F[i];
        sGa[i] = a.Ga[i];
    }
    for (int i = threadIdx.x; i < n * nd; i += blockDim.x) sG[i] = a.G[i];
    __syncthreads();
    wait_prior_grid();

    const int team = threadIdx.x / TEAM, tid = threadIdx.x % TEAM;
    const int nteams = blockDim.x / TEAM;
    int ri = N * (N + 1);
    ri += ri & 1;
    int r1 = 2 * nn;
    r1 = max(r1, max(2 * N * no, 2 * D2 * nd));
    float *tb = reinterpret_cast<float *>(sG + n * nd) + (size_t)team * team_floats(n, N, nd, TEAM);
    float *I = tb;                                         // [k][N+1]
    float2 *X = reinterpret_cast<float2 *>(tb + ri);       // region 1: X, then Ta, then P
    float2 *Ta = X;                                        // [k][no]
    float2 *P = X;                                         // [dyi][nd]
    float2 *U = reinterpret_cast<float2 *>(tb + ri + r1);  // region 2: U, then M, then B
    float2 *M = U;                                         // [dyi][n]
    float *B = reinterpret_cast<float *>(U);               // [iy][ix]
    int r2 = max(2 * N * n, max(2 * D2 * n, nd * nd));
    r2 += r2 & 1;
    float *red = tb + ri + r1 + r2;

    const int nd2 = nd * nd;
    const float cd = 0.5f * (float)(nd - 1);

    for (int g = blockIdx.x * nteams + team; g < a.total; g += gridDim.x * nteams) {
        const WfsDesc &W = a.wfs[find_wfs(a.wfs, a.n_wfs, g)];
        const InstDyn &D = a.dyn[W.inst];
        const uint64_t seed = a.inst[W.inst].seed;
        const uint32_t tlo = (uint32_t)__double_as_longlong(D.t);
        const uint32_t thi = (uint32_t)((unsigned long long)__double_as_longlong(D.t) >> 32);
        const int v = g - W.subap_begin;
        if (!guard(v >= 0 && v < W.n_valid, a.status)) continue;  // uniform over the team
        float *st_I = D.st_I ? D.st_I + W.int_off : nullptr;
        float *st_E = D.st_E ? D.st_E + W.det_off : nullptr;
        float *st_C = D.st_C ? D.st_C + W.det_off : nullptr;
        team_sync<TEAM>(team);

        // field
        const float *opd = D.opd + W.opd_off + (size_t)v * nn;
        float *so = reinterpret_cast<float *>(U);  // a fused projection's OPD (U is written later)
        // LGS per-slice model (self-projecting launches only): one wavefront and one DFT per
        // sodium slice, the spots weighted by the profile and summed into I
        const SliceDesc *SD = (a.project && W.slices) ? W.slices : nullptr;
        const int n_sl = SD ? SD->n : 1;
        LayerOffs *lo = reinterpret_cast<LayerOffs *>(red + 4 * (TEAM / 32) + 4);
        if (a.project) {
            const InstDesc &I = a.inst[W.inst];
            const int L = proj_layers(I, D);
            for (int l = tid; l < L; l += TEAM) lo[l] = layer_offsets(I, W, D.t, l);
            team_sync<TEAM>(team);
        }
        for (int sl = 0; sl < n_sl; ++sl) {
            if (a.project) {
                // this subaperture's OPD straight from the screens: the arithmetic of the projection
                // kernel (layer offsets in FP64, bilinear samples summed over the layers in order);
                // a slice sees the layers through its own cone (the scale), the offsets are shared
                const InstDesc &I = a.inst[W.inst];
                const int L = proj_layers(I, D);
                const int S = I.S;
                const bool pow2 = (S & (S - 1)) == 0;
                const int id = __ldg(W.subap + v), sy = id / W.n_sub, sx = id - sy * W.n_sub;
                const float half = 0.5f * (float)(W.n_sub * n - 1);
                float *out = D.opd + W.opd_off + (size_t)v * nn;
                // the slice's geometric term 1/2 |x - r_L|^2 k_s relative to the subaperture centre r_b:
                // k_s ((x - r_b).(r_b - r_L) + 1/2 |x - r_b|^2)
                float ebx = 0.0f, eby = 0.0f, dxp = 0.0f, ks = 0.0f;
                if (SD) {
                    dxp = (float)(W.pupil_dx_over_ds * I.ds);
                    const float c0 = 0.5f * (float)(n - 1);
                    ebx = ((float)(sx * n) + c0 - half) * dxp - (float)W.launch_x;
                    eby = ((float)(sy * n) + c0 - half) * dxp - (float)W.launch_y;
                    ks = SD->k[sl];
                }
                for (int i = tid; i < nn; i += TEAM) {
                    const int pp = i / n, qq = i - pp * n;
                    const float xr = (float)(sx * n + qq) - half, yr = (float)(sy * n + pp) - half;
                    float acc = 0.0f;
                    for (int l = 0; l < L; ++l) {
                        const LayerOffs L0 = lo[l];
                        const float ch = SD ? SD->c[sl][l].x : L0.c, cl = SD ? SD->c[sl][l].y : L0.cl;
                        int ou, ov, i0, i1, j0, j1;
                        float fx, gy;
                        screen_offset(ch, cl, L0.fu, xr, ou, fx);
                        screen_offset(ch, cl, L0.fv, yr, ov, gy);
                        wrap_pair(L0.bu + ou, S, pow2, i0, i1);
                        wrap_pair(L0.bv + ov, S, pow2, j0, j1);
                        if (!guard(i0 >= 0 && i1 < S && i1 >= 0 && j0 >= 0 && j1 < S && j1 >= 0 && i0 < S && j0 < S,
                                   a.status))
                            continue;
                        const float *scr = layer_screen(I, D, l);
                        const float *r0 = scr + (size_t)j0 * S, *r1 = scr + (size_t)j1 * S;
                        const float s00 = __ldg(r0 + i0), s01 = __ldg(r0 + i1);
                        const float s10 = __ldg(r1 + i0), s11 = __ldg(r1 + i1);
                        const float top = fmaf(fx, s01 - s00, s00);
                        const float bot = fmaf(fx, s11 - s10, s10);
                        acc += fmaf(gy, bot - top, top);
                    }
                    if (W.uplink) acc += fmaf(W.uplink->x, xr, W.uplink->y * yr);
                    if (sl == 0) out[i] = acc;
                    if (SD) {
                        const float ux = ((float)qq - 0.5f * (float)(n - 1)) * dxp;
                        const float uy = ((float)pp - 0.5f * (float)(n - 1)) * dxp;
                        acc += ks * fmaf(ux, ebx, fmaf(uy, eby, 0.5f * fmaf(ux, ux, uy * uy)));
                    }
                    so[i] = acc;
                }
                team_sync<TEAM>(team);
            }
            const uint32_t *mk = W.mask + (size_t)v * a.mask_words;
            const float ref = a.project ? so[0] : __ldg(opd);
            for (int i = tid; i < nn; i += TEAM) {
                const bool lit = (__ldg(mk + (i >> 5)) >> (i & 31)) & 1u;
                float s, c;
                field_phasor(W.k_phase * ((a.project ? so[i] : __ldg(opd + i)) - ref), s, c);
                X[i] = lit ? make_float2(c, s) : make_float2(0.0f, 0.0f);
            }
            team_sync<TEAM>(team);
            // U = F X : U[k][q] = sum_p F[k][p] X[p][q]
            for (int o = tid; o < N * n; o += TEAM) {
                const int k = o / n, q = o - k * n;
                float2 acc = make_float2(0.0f, 0.0f);
                for (int p = 0; p < n; ++p) acc = cmac(acc, sF[p * N + k], X[p * n + q]);
                U[o] = acc;
            }
            team_sync<TEAM>(team);
            // I = |U F^T|^2, or the slices' sum of w_s |U F^T|^2
            const float wsl = SD ? SD->w[sl] : 1.0f;
            const bool last = sl == n_sl - 1;
            for (int o = tid; o < N * N; o += TEAM) {
                const int k = o / N, m = o - k * N;
                float2 acc = make_float2(0.0f, 0.0f);
                for (int q = 0; q < n; ++q) acc = cmac(acc, U[k * n + q], sF[q * N + m]);
                const float in = fmaf(acc.x, acc.x, acc.y * acc.y);
                const float tot = SD ? (sl == 0 ? wsl * in : fmaf(wsl, in, I[k * (N + 1) + m])) : in;
                I[k * (N + 1) + m] = tot;
                if (st_I && last) st_I[(size_t)v * N * N + o] = tot;
            }
            team_sync<TEAM>(team);
        }
        if (W.is_lgs) {
            // Ta[k][dx] = sum_m I[k][m] Ga[dx][m]
            for (int o = tid; o < N * n; o += TEAM) {
                const int dx = o / N, k = o - dx * N;
                float2 acc = make_float2(0.0f, 0.0f);
                const float *row = I + k * (N + 1);
                const float2 *ga = sGa + dx * N;
                for (int m = 0; m < N; ++m) {
                    const float iv = row[m];
                    const float2 gg = ga[m];
                    acc.x = fmaf(iv, gg.x, acc.x);
                    acc.y = fmaf(iv, gg.y, acc.y);
                }
                Ta[k * no + dx] = acc;
            }
            team_sync<TEAM>(team);
            // M[dy][dx] = Kt[dy][dx] * sum_k Ga[dy][k] Ta[k][dx]   (Ga[-d] = conj Ga[d])
            const float2 *kt = W.ktil + (size_t)v * D2 * n;
            for (int o = tid; o < D2 * n; o += TEAM) {
                const int dyi = o / n, dx = o - dyi * n, dy = dyi - (n - 1);
                const float2 *ga = sGa + (dy >= 0 ? dy : -dy) * N;
                const float sg = dy >= 0 ? 1.0f : -1.0f;
                float2 acc = make_float2(0.0f, 0.0f);
                for (int k = 0; k < N; ++k) {
                    float2 gg = ga[k];
                    gg.y *= sg;
                    acc = cmac(acc, gg, Ta[k * no + dx]);
                }
                const float2 kv = __ldg(kt + o);
                M[o] = make_float2(acc.x * kv.x - acc.y * kv.y, acc.x * kv.y + acc.y * kv.x);
            }
            team_sync<TEAM>(team);
            // P[dy][ix] = sum_dx M[dy][dx] G[ix][dx]
            for (int o = tid; o < D2 * nd; o += TEAM) {
                const int dyi = o / nd, ix = o - dyi * nd;
                float2 acc = make_float2(0.0f, 0.0f);
                for (int dx = 0; dx < n; ++dx) acc = cmac(acc, M[dyi * n + dx], sG[dx * nd + ix]);
                P[o] = acc;
            }
            team_sync<TEAM>(team);
            // B[iy][ix] = Re sum_dy G[iy][dy] P[dy][ix]
            for (int o = tid; o < nd2; o += TEAM) {
                const int iy = o / nd, ix = o - iy * nd;
                float s = 0.0f;
                for (int dyi = 0; dyi < D2; ++dyi) {
                    const int dy = dyi - (n - 1);
                    float2 gg = sG[(dy >= 0 ? dy : -dy) * nd + iy];
                    if (dy < 0) gg.y = -gg.y;
                    const float2 pv = P[dyi * nd + ix];
                    s = fmaf(gg.x, pv.x, fmaf(-gg.y, pv.y, s));
                }
                B[o] = s;
            }
        } else {
            const int b = N / nd;
            for (int o = tid; o < nd2; o += TEAM) {
                const int iy = o / nd, ix = o - iy * nd;
                float s = 0.0f;
                for (int r = 0; r < b; ++r)
                    for (int c = 0; c < b; ++c) s += I[(b * iy + r) * (N + 1) + b * ix + c];
                B[o] = s;
            }
        }
        team_sync<TEAM>(team);

        // photometry
        float sb = 0.0f, d1 = 0.0f, d2 = 0.0f;
        for (int o = tid; o < nd2; o += TEAM) sb += B[o];
        team_sum3<TEAM>(sb, d1, d2, red, tid, team);
        const float scale = sb > 0.0f ? W.photons * __ldg(W.fill + v) / sb : 0.0f;
        // noise and centroid
        float sc = 0.0f, sx = 0.0f, sy = 0.0f;
        for (int o = tid; o < nd2; o += TEAM) {
            const int iy = o / nd, ix = o - iy * nd;
            const float e = scale * B[o];
            const float c = D.noise ? noise_pixel(e, W.read_noise, seed, (uint32_t)(v * nd2 + o),
                                                  (uint32_t)W.gs_index, tlo, thi)
                                    : e;
            if (st_E) st_E[(size_t)v * nd2 + o] = e;
            if (st_C) st_C[(size_t)v * nd2 + o] = c;
            sc += c;
            sx = fmaf((float)ix - cd, c, sx);
            sy = fmaf((float)iy - cd, c, sy);
        }
        team_sum3<TEAM>(sc, sx, sy, red, tid, team);
        if (tid == 0) {
            const bool ok = sc > 0.0f;
            float *sl = D.slopes + W.slope_off;
            sl[2 * v] = ok ? sx / sc : 0.0f;
            sl[2 * v + 1] = ok ? sy / sc : 0.0f;
        }
    }
}

size_t sh_fp32_smem_bytes(int n, int N, int nd, int *team_threads, int *teams_per_cta) {
    // a warp per subaperture up to 32-point DFTs; larger DFTs get a 512-thread team each
    const int team = N > 32 ? 512 : 32;
    const size_t consts = (size_t)(2 * n * N + n * nd) * sizeof(float2);
    const size_t per = (size_t)team_floats(n, N, nd, team) * sizeof(float);
    int teams = team >= 256 ? 1 : 256 / team;
    while (teams > 1 && consts + teams * per > 200 * 1024) --teams;
    if (team_threads) *team_threads = team;
    if (teams_per_cta) *teams_per_cta = teams;
    return consts + teams * per;
}

namespace {
constexpr size_t kSelfProjectSmem = 160 * 1024;

cudaError_t generic_shape(const ShArgs &a, LaunchShape *out) {
    int team = 0, teams = 0;
    size_t smem = sh_fp32_smem_bytes(a.n, a.N, a.nd, &team, &teams);
    // A self-projecting launch (a few NGS subapertures beside a large projection) asks for
    // enough shared memory that no projection CTA (about 74 KB) fits on its SMs: it then runs
    // alone there and finishes early instead of being stretched across the projection, which
    // takes the freed SMs afterwards.
    if (a.project == 1 && smem < kSelfProjectSmem) smem = kSelfProjectSmem;
    int blocks = (a.total + teams - 1) / teams;
    const int cap = a.grid_cap > 0 ? a.grid_cap : 152 * 32;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const void *f = team == 32 ? (const void *)k_sh_fp32<32> : (const void *)k_sh_fp32<512>;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    out->func = f;
    out->grid = dim3(blocks);
    out->block = dim3(team * teams);
    out->smem = smem;
    return cudaSuccess;
}
}  // namespace

cudaError_t n32_launch_shape(const ShArgs &a, LaunchShape *out);
cudaError_t tc_launch_shape(const ShArgs &a, LaunchShape *out, bool f16);
cudaError_t tc64_launch_shape(const ShArgs &a, LaunchShape *out, bool f16);

cudaError_t spot_launch_shape(int kind, const ShArgs &a, LaunchShape *out) {
    switch (kind) {
        case kSpotGeneric: return generic_shape(a, out);
        case kSpotN32: return n32_launch_shape(a, out);
        case kSpotTc: return a.N == 64 ? tc64_launch_shape(a, out, false) : tc_launch_shape(a, out, false);
        case kSpotTcF16: return a.N == 64 ? tc64_launch_shape(a, out, true) : tc_launch_shape(a, out, true);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_spot(int kind, const ShArgs &a, cudaStream_t s, bool after_project) {
    if (a.total <= 0) return cudaSuccess;
    LaunchShape sh;
    cudaError_t e = spot_launch_shape(kind, a, &sh);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    if (!after_project) return cudaLaunchKernel(sh.func, sh.grid, sh.block, args, sh.smem, s);
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

// ---------------------------------------------------------------------------
// Elongation transfer table (static per subaperture; computed once, FP64).
// K[p][q] = sum_s w_s g_s(p - Dy_s) g_s(q - Dx_s), g(d) = exp(-d^2 / 2 sigma^2) with d
// the minimum-image periodic distance on the N grid; the slice shift seen by
// subaperture centre r_b from launch point r_L is (r_b - r_L)(1/h0 - 1/h_s)
// radians.  Kt[dy][dx] = c_dx / N^2 * sum_m K[m] exp(+2 pi i m.d / N) / sum K,
// factorised per slice: sum_s w_s gy~_s[dy] gx~_s[dx].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_ktil(const __grid_constant__ KtilArgs a) {
    __shared__ double gx[kMaxNaSlices][kMaxN], gy[kMaxNaSlices][kMaxN];
    __shared__ double2 tx[kMaxNaSlices][kMaxNPix], ty[kMaxNaSlices][2 * kMaxNPix - 1];
    __shared__ double s_norm;
    const int v = blockIdx.x;
    if (v >= a.n_valid) return;
    const int n = a.n, N = a.N, D2 = 2 * n - 1;
    const int id = a.subap[v];
    const int sy = id / a.n_sub, sx = id - sy * a.n_sub;
    const double rbx = ((sx + 0.5) * n) * a.dx - 0.5 * a.D;
    const double rby = ((sy + 0.5) * n) * a.dx - 0.5 * a.D;
    for (int i = threadIdx.x; i < a.n_na * N; i += blockDim.x) {
        const int s = i / N, q = i - s * N;
        const double kk = 1.0 / a.h0 - 1.0 / a.alt[s];
        const double shx = (rbx - a.launch_x) * kk / a.pix_rad;
        const double shy = (rby - a.launch_y) * kk / a.pix_rad;
        double dx = q - shx, dy = q - shy;
        dx -= N * floor(dx / N + 0.5);
        dy -= N * floor(dy / N + 0.5);
        const double two_s2 = 2.0 * a.sigma_px * a.sigma_px;
        gx[s][q] = exp(-dx * dx / two_s2);
        gy[s][q] = exp(-dy * dy / two_s2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double norm = 0.0;
        for (int s = 0; s < a.n_na; ++s) {
            double sxs = 0.0, sys = 0.0;
            for (int q = 0; q < N; ++q) {
                sxs += gx[s][q];
                sys += gy[s][q];
            }
            norm += a.w[s] * sxs * sys;
        }
        s_norm = norm;
    }
    for (int i = threadIdx.x; i < a.n_na * (n + D2); i += blockDim.x) {
        const int s = i / (n + D2), j = i - s * (n + D2);
        const bool isx = j < n;
        const int d = isx ? j : j - n - (n - 1);
        double re = 0.0, im = 0.0;
        for (int q = 0; q < N; ++q) {
            const int ph = ((q * d) % N + N) % N;  // exp(+2 pi i q d / N), exact reduction
            double sn, cs;
            sincospi(2.0 * ph / N, &sn, &cs);
            const double gv = isx ? gx[s][q] : gy[s][q];
            re += gv * cs;
            im += gv * sn;
        }
        if (isx)
            tx[s][j] = make_double2(re, im);
        else
            ty[s][j - n] = make_double2(re, im);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < D2 * n; o += blockDim.x) {
        const int dyi = o / n, dx = o - dyi * n;
        double re = 0.0, im = 0.0;
        for (int s = 0; s < a.n_na; ++s) {
            const double2 p = ty[s][dyi], q = tx[s][dx];
            re += a.w[s] * (p.x * q.x - p.y * q.y);
            im += a.w[s] * (p.x * q.y + p.y * q.x);
        }
        const double c = (dx == 0 ? 1.0 : 2.0) / ((double)N * N * s_norm);
        a.ktil[(size_t)v * D2 * n + o] = make_float2((float)(re * c), (float)(im * c));
    }
}

cudaError_t launch_ktil(const KtilArgs &a, cudaStream_t s) {
    if (a.n_valid <= 0) return cudaSuccess;
    k_ktil<<<a.n_valid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The noise stage alone, for element-wise checks of the generator.
// ---------------------------------------------------------------------------
__global__ void k_noise(const float *E, int n, float ron, uint64_t seed, uint32_t wfs,
                        uint32_t tlo, uint32_t thi, uint32_t pixel0, float *C) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) C[i] = noise_pixel(E[i], ron, seed, pixel0 + (uint32_t)i, wfs, tlo, thi);
}

cudaError_t launch_noise(const float *E, int n, float ron, uint64_t seed, uint32_t wfs, double t,
                         uint32_t pixel0, float *C, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    unsigned long long tb;
    memcpy(&tb, &t, sizeof tb);
    k_noise<<<(n + 255) / 256, 256, 0, s>>>(E, n, ron, seed, wfs, (uint32_t)tb,
                                            (uint32_t)(tb >> 32), pixel0, C);
    return cudaGetLastError();
}

}  // namespace gbwfs
