"""Pins of the FP64 oracle against what the mathematics and the physics fix.

Each test checks one oracle function against something other than itself: a
closed form (Dirichlet kernel), an independent library routine (numpy FFT), an
invariant (Parseval, energy conservation, mirror symmetry), an exact special case
(integer shifts, linear screens) or statistics.  Each is chosen so that a plausible
slip (dropped term, wrong sign or index, transposed operand) fails at least one.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1408_0698_gb300 import inputs

RNG = np.random.default_rng(12345)


def centred_dft_via_fft(X, N):
    """Centred DFT through numpy's FFT: Y[k] = e^{i..} FFT(X[p] w^{-cN p})[k] per axis."""
    n = X.shape[0]
    cN, cn = (N - 1) / 2.0, (n - 1) / 2.0
    p = np.arange(n)
    k = np.arange(N)
    mod = np.exp(2j * np.pi * cN * p / N)           # w^{-cN p}, w = e^{-2 pi i / N}
    Xm = X * mod[:, None] * mod[None, :]
    P = np.zeros((N, N), complex)
    P[:n, :n] = Xm
    F = np.fft.fft2(P)
    ph = np.exp(2j * np.pi * (k * cn - cN * cn) / N)  # w^{-k cn} w^{cN cn}
    return F * ph[:, None] * ph[None, :]


def dirichlet(u, n, N):
    """|sum_{q<n} e^{-2 pi i (q - cn) u / N}| for real u (closed form)."""
    u = np.asarray(u, float)
    s = np.sin(np.pi * u / N)
    out = np.where(np.abs(s) < 1e-300, float(n), np.sin(np.pi * n * u / N) / np.where(s == 0, 1, s))
    return out


# ---------------------------------------------------------------- P1, P2: the DFT

@pytest.mark.parametrize("n,N", [(2, 4), (3, 8), (4, 8), (5, 12), (8, 16), (6, 24)])
def test_dft_matches_numpy_fft(n, N):
    X = RNG.standard_normal((n, n)) + 1j * RNG.standard_normal((n, n))
    Y = oracle.dft2(X, N)
    Yf = centred_dft_via_fft(X, N)
    assert np.max(np.abs(Y - Yf)) <= 1e-12 * np.max(np.abs(Yf))


def test_dft_brute_force_tiny():
    n, N = 3, 5
    X = RNG.standard_normal((n, n)) + 1j * RNG.standard_normal((n, n))
    Y = oracle.dft2(X, N)
    # brute force with integer-shifted indices: (k-cN)(p-cn) expanded term by term
    cN, cn = (N - 1) / 2, (n - 1) / 2
    B = np.zeros((N, N), complex)
    for k in range(N):
        for m in range(N):
            acc = 0j
            for p in range(n):
                for q in range(n):
                    acc += X[p, q] * np.exp(-2j * np.pi * ((k - cN) * (p - cn) + (m - cN) * (q - cn)) / N)
            B[k, m] = acc
    assert np.allclose(Y, B, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,N", [(4, 8), (6, 24), (10, 32), (8, 16)])
def test_parseval(n, N):
    X = np.exp(1j * RNG.uniform(0, 2 * np.pi, (n, n))) * (RNG.uniform(size=(n, n)) > 0.3)
    Y = oracle.dft2(X, N)
    assert abs(np.sum(np.abs(Y) ** 2) - N * N * np.sum(np.abs(X) ** 2)) <= 1e-12 * N * N * n * n


# ---------------------------------------------------------------- P3, P4: flat and tilt

@pytest.mark.parametrize("n,N", [(8, 16), (10, 32), (6, 24)])
def test_flat_square_subap_is_dirichlet(n, N):
    X = np.ones((n, n), complex)
    I = np.abs(oracle.dft2(X, N)) ** 2
    u = np.arange(N) - (N - 1) / 2
    d = dirichlet(u, n, N) ** 2
    ref = d[:, None] * d[None, :]
    assert np.max(np.abs(I - ref)) <= 1e-10 * ref.max()


@pytest.mark.parametrize("ax,ay", [(0.37, -1.21), (2.0, 0.0), (-3.0, 1.0)])
def test_tilt_shifts_dirichlet(ax, ay):
    """phi = 2 pi (ax q + ay p)/N shifts the spot by (ax, ay) FFT px: closed form."""
    n, N = 8, 16
    p = np.arange(n)
    X = np.exp(2j * np.pi * (ay * p[:, None] + ax * p[None, :]) / N)
    I = np.abs(oracle.dft2(X, N)) ** 2
    u = np.arange(N) - (N - 1) / 2
    ref = (dirichlet(u - ay, n, N) ** 2)[:, None] * (dirichlet(u - ax, n, N) ** 2)[None, :]
    assert np.max(np.abs(I - ref)) <= 1e-10 * ref.max()
    if float(ax).is_integer() and float(ay).is_integer():
        I0 = np.abs(oracle.dft2(np.ones((n, n)), N)) ** 2
        assert np.allclose(I, np.roll(I0, (int(ay), int(ax)), axis=(0, 1)), rtol=0, atol=1e-10 * I0.max())


def test_flat_phase_gives_zero_slope_any_mask():
    cfg = inputs.config1()
    S = cfg.layers.screen_size
    r = oracle.measure_wfs(cfg, np.zeros((1, S, S), np.float32), 0, 0.0)
    assert np.max(np.abs(r["slopes"])) <= 1e-12


def _tilt_screen(S, ds, ax, ay):
    i = np.arange(S) * ds
    return (ax * i[None, :] + ay * i[:, None]).astype(np.float32)[None]


def test_tilt_slope_is_analytic_centroid():
    """End to end: a tilted wavefront on an interior (fully lit) NGS subap gives the CoG of
    the binned, shifted Dirichlet spot."""
    cfg = inputs.config1()
    g = cfg.geometries[0]
    S, ds = cfg.layers.screen_size, cfg.layers.screen_dx_m
    lam = cfg.stars[0].wavelength_m
    n, N, nd = g.n_pix_sub, g.n_fft, g.n_det
    dx = cfg.telescope.diameter_m / (g.n_sub * n)
    alpha_x, alpha_y = 0.8 * lam / (N * dx), -0.45 * lam / (N * dx)  # radians of tilt
    scr = _tilt_screen(S, ds, alpha_x, alpha_y)
    idx, fill = oracle.valid_subaps(cfg.telescope.diameter_m, 0.0, g.n_sub, n)
    interior = np.where(fill == 1.0)[0]
    r = oracle.measure_wfs(cfg, scr, 0, 0.0, sel=interior)
    ax, ay = alpha_x * N * dx / lam, alpha_y * N * dx / lam
    u = np.arange(N) - (N - 1) / 2
    I = (dirichlet(u - ay, n, N) ** 2)[:, None] * (dirichlet(u - ax, n, N) ** 2)[None, :]
    b = N // nd
    B = I.reshape(nd, b, nd, b).sum(axis=(1, 3))
    c = (nd - 1) / 2
    sx = np.sum((np.arange(nd)[None, :] - c) * B) / B.sum()
    sy = np.sum((np.arange(nd)[:, None] - c) * B) / B.sum()
    assert np.max(np.abs(r["slopes"][:, 0] - sx)) < 2e-6
    assert np.max(np.abs(r["slopes"][:, 1] - sy)) < 2e-6
    assert sx > 0 and sy < 0


# ---------------------------------------------------------------- P5: mirror symmetry

def test_mirror_and_transpose_symmetry():
    cfg = inputs.config1()
    g = cfg.geometries[0]
    S = cfg.layers.screen_size
    scr = inputs.make_screens(cfg.layers, 77)
    base = oracle.measure_wfs(cfg, scr, 0, 0.0)["slopes"]
    idx, _ = oracle.valid_subaps(cfg.telescope.diameter_m, 0.0, g.n_sub, g.n_pix_sub)
    pos = {int(v): k for k, v in enumerate(idx)}
    ns = g.n_sub
    # x -> -x: column i -> S - i (pixel centres sit half way between screen samples)
    mir = scr[:, :, (S - np.arange(S)) % S].copy()
    sm = oracle.measure_wfs(cfg, mir, 0, 0.0)["slopes"]
    for k, v in enumerate(idx):
        sy, sx = divmod(int(v), ns)
        j = pos[sy * ns + (ns - 1 - sx)]
        assert abs(sm[j, 0] + base[k, 0]) < 1e-9 and abs(sm[j, 1] - base[k, 1]) < 1e-9
    # transpose: swap x and y
    tr = np.ascontiguousarray(np.transpose(scr, (0, 2, 1)))
    st = oracle.measure_wfs(cfg, tr, 0, 0.0)["slopes"]
    for k, v in enumerate(idx):
        sy, sx = divmod(int(v), ns)
        j = pos[sx * ns + sy]
        assert abs(st[j, 0] - base[k, 1]) < 1e-9 and abs(st[j, 1] - base[k, 0]) < 1e-9


# ---------------------------------------------------------------- P6: elongation

def _one_slice_star(h0, h1, fwhm, launch=(0.0, 0.0)):
    return inputs.GuideStar(is_lgs=True, theta_x_rad=0, theta_y_rad=0, range_m=h0,
                            wavelength_m=589e-9, geometry_index=0, launch_x_m=launch[0],
                            launch_y_m=launch[1], spot_fwhm_rad=fwhm,
                            na_alt_m=np.array([h1]), na_weight=np.array([1.0]))


def test_elongation_integer_shift_is_roll():
    N = 16
    h0, h1 = 90e3, 100e3
    k = 1.0 / h0 - 1.0 / h1
    pix = 1e-6
    # choose subap centre so the shift is exactly (3, -2) FFT px
    rbx, rby = 3 * pix / k, -2 * pix / k
    star = _one_slice_star(h0, h1, 1e-3 * pix)  # sigma ~ 4e-4 px: a delta
    K = oracle.elong_kernel(N, pix, rbx, rby, star)
    assert abs(K.sum() - 1) < 1e-12
    I = RNG.uniform(size=(N, N))
    out = oracle.convolve(I, K)
    assert np.allclose(out, np.roll(I, (-2, 3), axis=(0, 1)), atol=1e-9)


def test_convolution_matches_fft_and_conserves_energy():
    N = 24
    cfg = inputs.config2()
    star = cfg.stars[1]
    K = oracle.elong_kernel(N, 7.36e-7, 2.5, -1.7, star)
    assert abs(K.sum() - 1) < 1e-12 and K.min() >= 0
    I = RNG.uniform(size=(N, N))
    out = oracle.convolve(I, K)
    ref = np.real(np.fft.ifft2(np.fft.fft2(I) * np.fft.fft2(K)))
    assert np.max(np.abs(out - ref)) < 1e-12 * np.abs(ref).max()
    assert abs(out.sum() - I.sum()) < 1e-11 * I.sum()


@pytest.mark.parametrize("N,shift", [(16, (0.3, -2.7)), (24, (5.5, 1.25)), (32, (-11.0, 7.4))])
def test_separable_elongation_equals_direct(N, shift):
    """The separable form (rows then columns, per slice) equals the elongation kernel's direct
    periodic convolution to rounding, for an elongation longer than the field (wrap)."""
    rng = np.random.default_rng(N)
    I = rng.random((N, N)) ** 3
    star = _one_slice_star(90e3, 90e3, 1.0 * 4.848e-6)
    star.na_alt_m = np.array([84e3, 88e3, 90e3, 93e3, 97e3])
    star.na_weight = np.array([0.1, 0.25, 0.3, 0.2, 0.15])
    star.launch_x_m, star.launch_y_m = 5.0, -2.0
    pix = 589e-9 / (N * 0.05)
    rbx, rby = 5.0 + shift[0], -2.0 + shift[1]
    K = oracle.elong_kernel(N, pix, rbx, rby, star)
    direct = oracle.convolve(I, K)
    sep = oracle.elong_convolve_separable(I, pix, rbx, rby, star)
    assert np.max(np.abs(sep - direct)) <= 1e-13 * np.abs(direct).max()


def test_measure_wfs_separable_equals_direct():
    """measure_wfs with the separable elongation (the timed CPU baseline) gives the stages and
    slopes of the direct form to rounding."""
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    sel = np.arange(0, 1264, 37, dtype=np.int32)
    a = oracle.measure_wfs(cfg, scr, 1, 0.01, sel=sel, stages=True)
    oracle.set_separable(True)
    try:
        b = oracle.measure_wfs(cfg, scr, 1, 0.01, sel=sel, stages=True)
    finally:
        oracle.set_separable(False)
    assert np.max(np.abs(a["Ie"] - b["Ie"])) <= 1e-12 * np.abs(a["Ie"]).max()
    assert np.max(np.abs(a["slopes"] - b["slopes"])) <= 1e-10


def test_elongation_centroid_and_antisymmetry():
    """Narrow slices, small shifts: the kernel's first moment is sum_s w_s Delta_s, and
    mirroring the subap about the launch point mirrors the kernel."""
    N = 32
    pix = 4e-7
    h, w = inputs.sodium_slices(90e3, 10e3, 8)
    star = inputs.GuideStar(True, 0, 0, 90e3, 589e-9, 0, launch_x_m=5.0, launch_y_m=0.0,
                            spot_fwhm_rad=4.0 * pix, na_alt_m=h, na_weight=w)
    rb = (4.0, 0.5)
    K = oracle.elong_kernel(N, pix, rb[0], rb[1], star)
    d = np.arange(N) - N * np.floor(np.arange(N) / N + 0.5)
    mx = np.sum(d[None, :] * K)
    my = np.sum(d[:, None] * K)
    kk = 1 / 90e3 - 1 / h
    ex = np.sum(w * (rb[0] - 5.0) * kk / pix)
    ey = np.sum(w * (rb[1] - 0.0) * kk / pix)
    assert abs(mx - ex) < 1e-6 and abs(my - ey) < 1e-6
    assert abs(ex) > 0.05  # the slices really are spread
    K2 = oracle.elong_kernel(N, pix, 2 * 5.0 - rb[0], -rb[1], star)
    flip = np.roll(K[::-1, ::-1], (1, 1), axis=(0, 1))  # index j -> -j mod N
    assert np.allclose(K2, flip, atol=1e-14)


# ---------------------------------------------------------------- P7: binning / photometry

def test_binning_and_photometry():
    I = RNG.uniform(size=(32, 32))
    B = oracle.bin_image(I, 16)
    assert np.allclose(B, I.reshape(16, 2, 16, 2).sum(axis=(1, 3)), atol=1e-13)
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, 5)
    g = cfg.geometries[0]
    _, fill = oracle.valid_subaps(8.0, 0.0, g.n_sub, g.n_pix_sub)
    for w in (0, 3):
        r = oracle.measure_wfs(cfg, scr, w, 0.01, stages=True)
        tot = r["E"].sum(axis=(1, 2))
        assert np.allclose(tot, cfg.stars[w].photons_per_subap * fill, rtol=1e-12)
        # Parseval through elongation: sum I' = sum I = N^2 * lit pixels
        lit = np.round(fill * g.n_pix_sub ** 2)
        assert np.allclose(r["Ie"].sum(axis=(1, 2)), g.n_fft ** 2 * lit, rtol=1e-11)


# ---------------------------------------------------------------- P8, P9, P12: projection

def _layers1(alt, S, ds, vx=0.0, vy=0.0):
    return inputs.Layers(alt_m=np.array([alt]), wind_vx_mps=np.array([vx]), wind_vy_mps=np.array([vy]),
                         x0_m=np.zeros(1), y0_m=np.zeros(1), screen_size=S, screen_dx_m=ds)


def test_projection_integer_offsets_copy_screen():
    cfg = inputs.config1()
    S = 256
    scr = RNG.standard_normal((1, S, S)).astype(np.float32)
    # pupil pixel centres sit at half-integer screen coordinates: shift the layer by half a px
    cfg.layers = _layers1(0.0, S, 0.05)
    cfg.layers.x0_m[:] = -0.025
    cfg.layers.y0_m[:] = -0.025
    opd = oracle.project_grid(cfg, scr, 0, 0.0)
    # u = 128 + (j - 79.5) + 0.5 = j + 49
    win = scr[0, 49:49 + 160, 49:49 + 160].astype(np.float64)
    assert np.max(np.abs(opd - win)) <= 1e-12 * np.abs(win).max()
    # periodic wrap: moving by a whole screen changes nothing
    cfg.layers.x0_m[:] = -0.025 + S * 0.05
    opd2 = oracle.project_grid(cfg, scr, 0, 0.0)
    assert np.max(np.abs(opd - opd2)) <= 1e-12 * np.abs(win).max()


def test_bilinear_exact_on_linear_screen():
    S = 64
    i = np.arange(S, dtype=np.float64)
    scr = (0.25 * i[None, :] - 0.5 * i[:, None] + 3.0).astype(np.float32)
    for u, v in [(10.3, 20.7), (33.01, 5.99), (0.5, 0.25)]:
        assert abs(oracle.bilinear(scr, u, v) - (0.25 * u - 0.5 * v + 3.0)) < 1e-12


def test_cone_scales_gradient():
    """A constant-gradient layer at altitude h seen from an LGS at range H: the sampled
    gradient is the screen's times c = 1 - h/H (closed form)."""
    S, ds, h, H = 512, 0.05, 8e3, 90e3
    g = 2e-7
    i = np.arange(S, dtype=np.float64) * ds
    scr = np.ascontiguousarray(np.broadcast_to(g * i[None, :], (S, S))).astype(np.float32)[None]
    cfg = inputs.config2()
    cfg.layers = _layers1(h, S, ds)
    star = cfg.stars[0]
    star.theta_x_rad = star.theta_y_rad = 0.0
    o1 = oracle.opd(cfg, scr, 0, -2.0, 0.3, 0.0)
    o2 = oracle.opd(cfg, scr, 0, 2.0, 0.3, 0.0)
    assert abs((o2 - o1) / 4.0 - g * (1 - h / H)) < 1e-6 * g
    ngs = cfg.stars[3]
    o1 = oracle.opd(cfg, scr, 3, -2.0, 0.3, 0.0)
    o2 = oracle.opd(cfg, scr, 3, 2.0, 0.3, 0.0)
    assert abs((o2 - o1) / 4.0 - g) < 1e-6 * g
    # direction: theta * h moves the footprint
    o2 = oracle.opd(cfg, scr, 0, 2.0, 0.3, 0.0)
    star.theta_x_rad = 1e-4
    o3 = oracle.opd(cfg, scr, 0, 2.0, 0.3, 0.0)
    assert abs((o3 - o2) - g * 1e-4 * h) < 1e-5 * g * 1e-4 * h


def test_frozen_flow_long_run_exact():
    """At t = 2 s with v = 10 m/s and 0.05 m px the footprint has moved by exactly 400 px:
    the OPD equals that of the screen rolled by 400 px."""
    cfg = inputs.config1()
    S = 1024
    cfg.layers = _layers1(0.0, S, 0.05, vx=10.0, vy=-5.0)
    scr = RNG.standard_normal((1, S, S)).astype(np.float32)
    o_t = oracle.project_grid(cfg, scr, 0, 2.0)
    rolled = np.roll(scr, (-200, 400), axis=(1, 2))
    o_0 = oracle.project_grid(cfg, rolled, 0, 0.0)
    assert np.max(np.abs(o_t - o_0)) <= 1e-12 * np.abs(o_0).max()


# ---------------------------------------------------------------- P10: noise

# Known-answer vectors of Philox4x32-10: Salmon, Moraes, Dror and Shaw, "Parallel random
# numbers: as easy as 1, 2, 3", SC'11; the vectors are the ones distributed with the authors'
# Random123 library (counter, key -> output; all-zero, all-ones, and the digits of pi).
PHILOX_KAT = [
    ([0x00000000, 0x00000000, 0x00000000, 0x00000000], [0x00000000, 0x00000000],
     [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF], [0xFFFFFFFF, 0xFFFFFFFF],
     [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
]


@pytest.mark.parametrize("ctr,key,expect", PHILOX_KAT)
def test_philox_known_answers(ctr, key, expect):
    """The generator is Philox4x32-10 exactly: a wrong multiplier, Weyl constant, round count
    or word permutation changes every output word of these published vectors."""
    assert [int(v) for v in oracle.philox(ctr, key)] == expect


def test_philox_uniformity_and_independence():
    n = 1 << 16
    vals = np.zeros((n, 4), np.uint32)
    for i in range(n):
        vals[i] = oracle.philox([i, 7, 0, 0], [0x1234, 0xABCD])
    u = (vals >> 9).astype(np.float64) / 2 ** 23
    h, _ = np.histogram(u.ravel(), bins=64, range=(0, 1))
    chi2 = np.sum((h - h.mean()) ** 2 / h.mean())
    assert chi2 < 130  # 63 dof, p ~ 1e-6
    # lanes uncorrelated; counter increments decorrelate
    cc = np.corrcoef(u.T)
    assert np.max(np.abs(cc - np.eye(4))) < 0.02
    assert abs(np.corrcoef(u[:-1, 0], u[1:, 0])[0, 1]) < 0.02
    # bits balanced
    bits = np.unpackbits(vals.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.002


@pytest.mark.parametrize("E", [0.3, 3.0, 12.0, 16.0, 40.0, 250.0])
def test_poisson_moments(E):
    n = 40000
    Earr = np.full(n, E, np.float32)
    C, K = oracle.noise_image(Earr, 0.0, 99, 1, 0.5)
    assert np.array_equal(C, K.astype(float))  # no read noise
    m, v = K.mean(), K.var()
    se = math.sqrt(E / n)
    assert abs(m - E) < 5 * se
    assert abs(v / E - 1) < 5 * math.sqrt(2.0 / n) + 0.01
    # pmf against the exact Poisson pmf (chi-square over the bulk)
    ks = np.arange(max(0, int(E - 4 * math.sqrt(E))), int(E + 4 * math.sqrt(E)) + 2)
    logp = np.array([-E + k * math.log(E) - math.lgamma(k + 1) for k in ks])
    expct = n * np.exp(logp)
    obs = np.array([(K == k).sum() for k in ks])
    keep = expct > 20
    chi2 = np.sum((obs[keep] - expct[keep]) ** 2 / expct[keep])
    assert chi2 < keep.sum() + 6 * math.sqrt(2 * keep.sum()) + 10


ALL_UNIFORMS = None


def _all_uniforms():
    """Every uniform the generator can yield: ((x >> 9) + 1/2) 2^-23 for the 2^23 values of
    x >> 9, each taken with the same probability (exact in FP32)."""
    global ALL_UNIFORMS
    if ALL_UNIFORMS is None:
        m = np.arange(1 << 23, dtype=np.float64)
        ALL_UNIFORMS = ((m + 0.5) / 2.0 ** 23).astype(np.float32)
    return ALL_UNIFORMS


@pytest.mark.parametrize("E", [1e-3, 0.05, 0.5, 1.0, 2.5, 5.0, 7.77, 10.0, 12.5, 15.0, 15.999])
def test_inversion_exact_distribution_is_poisson(E):
    """The sampler's inversion branch (E < 16, FP32 decisions) tabulated over every uniform
    the generator yields: its exact CDF P(K <= k) is the Poisson CDF of its mean within the
    FP32 rounding of the running sum, |P32 - F| <= (4k + 2) 2^-24 + 2^-23 (the recurrence
    p_k = p_{k-1} E / k costs three roundings a step, the running sum one more, the uniform
    grid 2^-23).  Tabulating every uniform resolves the rounding itself: any slip in the
    recurrence (an index, exp(-E), the stopping test) is off by orders of magnitude more.
    The same table bounds how often an exact-arithmetic decision on the same uniform would
    differ: at most the summed CDF gaps, under 1e-4 of the draws."""
    from scipy.stats import poisson

    E = np.float32(E)
    k = oracle.poisson_inversion(E, _all_uniforms())
    cnt = np.bincount(k)
    ks = np.arange(len(cnt))
    P32 = np.cumsum(cnt) / 2.0 ** 23
    F = poisson.cdf(ks, float(E))
    assert np.all(np.abs(P32 - F) <= (4 * ks + 2) * 2.0 ** -24 + 2.0 ** -23)
    # uniforms whose FP32 decision differs from the exact one lie between the two CDFs
    assert np.sum(np.abs(P32 - F)) < 1e-4
    # pmf mean equals E within the same rounding
    assert abs(np.sum(ks * cnt) / 2.0 ** 23 - float(E)) < 1e-4 * max(1.0, float(E))


@pytest.mark.parametrize("E", [16.0, 23.5, 80.0, 1000.0])
def test_ptrs_pmf_large_sample(E):
    """PTRS regime (E >= 16): 2^22 draws against the exact Poisson pmf, chi-square over the
    bins with more than 50 expected counts, and the mean and variance within 5 standard
    errors (Hormann 1993's transformed rejection is exact in exact arithmetic)."""
    n = 1 << 22
    _, K = oracle.noise_image(np.full(n, E, np.float32), 0.0, 2024, 6, 0.375)
    ks = np.arange(max(0, int(E - 6 * math.sqrt(E))), int(E + 6 * math.sqrt(E)) + 2)
    logp = np.array([-E + k * math.log(E) - math.lgamma(k + 1) for k in ks])
    expct = n * np.exp(logp)
    inside = (K >= ks[0]) & (K <= ks[-1])
    obs = np.bincount(K[inside] - ks[0], minlength=len(ks))
    keep = expct > 50
    chi2 = np.sum((obs[keep] - expct[keep]) ** 2 / expct[keep])
    dof = keep.sum()
    assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (chi2, dof)
    assert abs(K.mean() - E) < 5 * math.sqrt(E / n)
    assert abs(K.var() / E - 1) < 5 * math.sqrt(2.0 / n)


def test_inversion_search_length_bound():
    """The inversion recurrence (p E)(1/k) in FP32 ends (u <= F or F stops growing) before
    k = 43 for every E < 16, even at the largest uniform ((2^23 - 1 + 1/2) 2^-23): the
    spot kernels keep 1/k in a 64-entry table."""
    f = np.float32
    umax = f((float((1 << 23) - 1) + 0.5) / 8388608.0)

    def search(E):
        p = f(math.exp(-float(E)))
        F, k = p, 0
        while umax > F:
            k += 1
            p = f(f(p * E) * f(f(1.0) / f(k)))
            Fn = f(F + p)
            if Fn == F:
                break
            F = Fn
        return k

    Es = list(np.linspace(0.01, 15.999, 1600).astype(np.float32)) + [np.nextafter(f(16), f(0))]
    assert max(search(E) for E in Es) <= 42


@pytest.mark.parametrize("E", [3.0, 40.0])
def test_poisson_pair_members_independent(E):
    """Pixels 2m and 2m + 1 share one generator block (words 2 and 3 start their Poisson
    draws; above E = 16 their continuation blocks interleave): their counts are
    uncorrelated and equally distributed."""
    n = 60000
    C, K = oracle.noise_image(np.full(n, E, np.float32), 0.0, 17, 3, 0.125)
    ke, ko = K[0::2].astype(float), K[1::2].astype(float)
    assert abs(np.corrcoef(ke, ko)[0, 1]) < 0.02
    se = math.sqrt(E / (n // 2))
    assert abs(ke.mean() - E) < 5 * se and abs(ko.mean() - E) < 5 * se
    assert not np.array_equal(ke, ko)


def test_read_noise_gaussian():
    n = 50000
    C, K = oracle.noise_image(np.zeros(n, np.float32), 3.0, 5, 2, 0.0)
    assert np.all(K == 0)
    assert abs(C.mean()) < 5 * 3 / math.sqrt(n)
    assert abs(C.std() / 3.0 - 1) < 0.02
    # fourth moment of a Gaussian
    z = C / 3.0
    assert abs(np.mean(z ** 4) - 3) < 0.1
    # the pair's two Box-Muller deviates (cos and sin of one angle): independent, and
    # z_even^2 + z_odd^2 = -2 ln u is exponential with mean 2
    ze, zo = z[0::2], z[1::2]
    assert abs(np.corrcoef(ze, zo)[0, 1]) < 0.02
    assert abs(ze.std() - 1) < 0.02 and abs(zo.std() - 1) < 0.02
    r2 = ze ** 2 + zo ** 2
    assert abs(r2.mean() - 2) < 0.05 and abs(np.median(r2) - 2 * math.log(2)) < 0.05


def test_noise_is_counter_based():
    E = inputs.random_expected_image(4096, 3)
    C1, _ = oracle.noise_image(E, 3.0, 11, 4, 0.125)
    C2, _ = oracle.noise_image(E, 3.0, 11, 4, 0.125)
    C3, _ = oracle.noise_image(E, 3.0, 11, 4, 0.126)
    C4, _ = oracle.noise_image(E, 3.0, 11, 5, 0.125)
    assert np.array_equal(C1, C2)
    assert not np.array_equal(C1, C3) and not np.array_equal(C1, C4)


def test_slope_noise_variance_delta_method():
    """Photon + read noise on a fixed spot: the CoG variance matches the delta-method
    prediction sum((x - s)^2 (E + ron^2)) / (sum E)^2."""
    nd = 8
    rng = np.random.default_rng(0)
    y, x = np.mgrid[0:nd, 0:nd] - (nd - 1) / 2
    E = 500.0 * np.exp(-((x - 0.4) ** 2 + (y + 0.2) ** 2) / 2.0)
    E = (E / E.sum() * 500.0).astype(np.float32)
    ron = 1.0
    sx = []
    for rep in range(3000):
        C, _ = oracle.noise_image(E.ravel(), ron, 1, 0, float(rep) * 1e-3)
        sx.append(oracle.cog(C.reshape(nd, nd))[0])
    sx = np.array(sx)
    Ed = E.astype(float)
    s0 = np.sum(x * Ed) / Ed.sum()
    pred = np.sum((x - s0) ** 2 * (Ed + ron ** 2)) / Ed.sum() ** 2
    assert abs(sx.var() / pred - 1) < 0.1
    assert abs(sx.mean() - s0) < 5 * math.sqrt(pred / len(sx)) + 2e-3


# ---------------------------------------------------------------- subaperture counts

def test_valid_subap_counts():
    """Pupil split: valid-subaperture counts of the configured geometries (fill >= 0.5)."""
    assert len(oracle.valid_subaps(8.0, 0.0, 20, 8)[0]) == 316
    assert len(oracle.valid_subaps(8.0, 0.0, 40, 6)[0]) == 1264
    assert len(oracle.valid_subaps(39.0, 0.28, 80, 10)[0]) == 4632
    assert len(oracle.valid_subaps(39.0, 0.28, 2, 32)[0]) == 4
    # the pupil mask: area within one pixel ring of pi (D/2)^2 (1 - eps^2)
    m = oracle.pupil_mask(39.0, 0.28, 800)
    area = m.sum() * (39.0 / 800) ** 2
    exact = np.pi * (19.5 ** 2) * (1 - 0.28 ** 2)
    assert abs(area - exact) < 2 * np.pi * 19.5 * (39.0 / 800) * 1.3
    assert np.array_equal(m, m[::-1, :]) and np.array_equal(m, m.T)


# ---------------------------------------------------------------- golden fixtures

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _paper_sizes():
    out = {}
    for line in open(f"{GOLDEN}/paper_sizes.txt"):
        line = line.split("#")[0].split()
        if len(line) == 2:
            out[line[0]] = float(line[1])
    return out


def test_elt_workload_uses_the_paper_sizes():
    p = _paper_sizes()
    c3 = inputs.config3()
    g = c3.geometries[0]
    assert g.n_sub * g.n_pix_sub == p["pupil_px"] and g.n_sub == p["lgs_subaps"]
    assert abs(c3.telescope.diameter_m / (g.n_sub * g.n_pix_sub) - p["pupil_dx_m"]) < 1e-15
    assert sum(s.is_lgs for s in c3.stars) == p["n_lgs"]
    assert sum(not s.is_lgs for s in c3.stars) == p["n_ngs"]


def test_oracle_regression_fixtures():
    cfg = inputs.config1()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    ref = np.loadtxt(f"{GOLDEN}/config1_t0.003_slopes.txt")
    s = oracle.measure_wfs(cfg, scr, 0, 0.003)["slopes"]
    assert np.allclose(s, ref, rtol=0, atol=1e-12)
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    ref = np.loadtxt(f"{GOLDEN}/config2_lgs1_t0.01_slopes.txt")
    s = oracle.measure_wfs(cfg, scr, 1, 0.01, sel=ref[:, 0].astype(np.int32))["slopes"]
    assert np.allclose(s, ref[:, 1:], rtol=0, atol=1e-12)
    st = dataclasses.replace(cfg.stars[0], per_slice=True, uplink_diameter_m=0.5, uplink_samples=16)
    ref = np.loadtxt(f"{GOLDEN}/config2_lgs0_slices_uplink_t0.01_slopes.txt")
    s = oracle.measure_wfs(dataclasses.replace(cfg, stars=[st] + cfg.stars[1:]), scr, 0, 0.01,
                           sel=ref[:, 0].astype(np.int32))["slopes"]
    assert np.allclose(s, ref[:, 1:], rtol=0, atol=1e-12)
    cfg = inputs.config1()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    dm = inputs.Dm(21, 0.4, 0.0, 12)
    M = inputs.modal_base(dm, 5, amplitude_m=2e-8).astype(np.float64)
    cm = inputs.random_control_matrix(12, 2 * 316, seed=6, scale=0.5).astype(np.float64)
    ref = np.loadtxt(f"{GOLDEN}/config1_loop_step_coeffs.txt")
    _, c1 = oracle.loop_step(cfg, scr, 0.002, [dm], [M], cm, np.full(12, 0.4), ref[:, 0])
    assert np.allclose(c1, ref[:, 1], rtol=0, atol=1e-12)
    ref = np.loadtxt(f"{GOLDEN}/config1_interaction_rows.txt")
    im = oracle.interaction_matrix(cfg, 0, [dm], [M], 0.5, modes=[0, 5, 11])
    assert np.allclose(im.T, ref, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- closed loop: mirrors

def _poke(dm, ay, ax, v=1.0):
    a = np.zeros(dm.n_act * dm.n_act)
    a[ay * dm.n_act + ax] = v
    return a


def test_dm_poke_physics():
    """One actuator: the correction layer is minus a bump of height 1 on the actuator, the
    coupling at one pitch, symmetric, and zero from the support radius on."""
    dm = inputs.Dm(n_act=7, pitch_m=0.4, alt_m=0.0, n_modes=1, coupling=0.15, support=3)
    a = _poke(dm, 3, 3)
    v = lambda x, y: oracle.dm_value(dm, a, x, y)
    assert v(0, 0) == pytest.approx(-1.0, abs=1e-14)
    # coupling: the neighbour's influence relative to the actuator's, to within k^(R^2)
    for (x, y) in [(0.4, 0), (-0.4, 0), (0, 0.4), (0, -0.4)]:
        assert v(x, y) / v(0, 0) == pytest.approx(0.15, abs=0.15 ** 9)
    # separable (rank one) and even in x and y
    for x, y in [(0.13, 0.27), (0.5, -0.61), (-0.9, 0.05)]:
        assert v(x, y) * v(0, 0) == pytest.approx(v(x, 0) * v(0, y), rel=1e-12)
        assert v(-x, y) == pytest.approx(v(x, y), rel=1e-12)
        assert v(x, -y) == pytest.approx(v(x, y), rel=1e-12)
    # continuous fall to zero at the support radius, exactly zero beyond
    assert abs(v(3 * 0.4 - 1e-7, 0)) < 1e-6
    assert v(3 * 0.4 + 1e-9, 0) == 0.0 and v(0, -5 * 0.4) == 0.0
    # decreasing away from the actuator
    xs = np.linspace(0, 1.2, 25)
    vals = [-v(x, 0) for x in xs]
    assert all(b <= c for b, c in zip(vals[1:], vals[:-1]))


def test_dm_layer_grid_geometry():
    """Actuator (ay, ax) sits at ((ax - c) p, (ay - c) p) with pixel (i, j) at ((j - S/2) ds,
    (i - S/2) ds): a poke one actuator over moves the layer by p / ds pixels along that axis
    only; linear in the commands."""
    dm = inputs.Dm(n_act=9, pitch_m=0.4, alt_m=0.0, n_modes=1, coupling=0.2, support=2)
    S, ds = 64, 0.1                                   # pitch = 4 pixels
    L0 = oracle.dm_layer(dm, _poke(dm, 4, 4), S, ds)  # central actuator on pixel (32, 32)
    assert L0[32, 32] == np.float32(-1.0)
    assert np.unravel_index(np.argmin(L0), L0.shape) == (32, 32)
    Lx = oracle.dm_layer(dm, _poke(dm, 4, 6), S, ds)
    Ly = oracle.dm_layer(dm, _poke(dm, 1, 4), S, ds)
    np.testing.assert_array_equal(Lx, np.roll(L0, 8, axis=1))
    np.testing.assert_array_equal(Ly, np.roll(L0, -12, axis=0))
    rng = np.random.default_rng(5)
    a, b = rng.standard_normal(81), rng.standard_normal(81)
    La, Lb = oracle.dm_layer(dm, a, S, ds), oracle.dm_layer(dm, b, S, ds)
    Lab = oracle.dm_layer(dm, 2.0 * a - 0.5 * b, S, ds)
    np.testing.assert_allclose(Lab, 2.0 * La - 0.5 * Lb, atol=1e-6 * np.abs(Lab).max())
    # even n_act: the grid's centre falls between actuators
    dm8 = inputs.Dm(n_act=8, pitch_m=0.4, alt_m=0.0, n_modes=1, coupling=0.2, support=2)
    flat = oracle.dm_layer(dm8, np.ones(64), S, ds)
    np.testing.assert_allclose(flat[32, 32 - 2], flat[32, 32 + 2], rtol=1e-6)
    np.testing.assert_allclose(flat[32 - 6, 32], flat[32 + 6, 32], rtol=1e-6)


def _small_loop_cfg(is_lgs=False, alt=0.0):
    """4 m telescope, 10 x 10 subapertures of 8 px, N = 16, 8 x 8 detector pixels; one
    ground (or alt) layer without wind."""
    tel = inputs.Telescope(4.0, 0.0)
    geom = [inputs.Geometry(10, 8, 16, 8, 0.5, inputs.PREC_FP32)]
    if is_lgs:
        star = inputs._lgs(10 * inputs.ARCSEC, -5 * inputs.ARCSEC, 0.3, 0)
    else:
        star = inputs._ngs(5 * inputs.ARCSEC, 0.0, 700e-9, 0, photons=1000.0)
    lay = inputs.Layers(alt_m=np.array([alt]), wind_vx_mps=np.zeros(1), wind_vy_mps=np.zeros(1),
                        x0_m=np.zeros(1), y0_m=np.zeros(1), screen_size=128, screen_dx_m=0.05)
    return inputs.Config("loop_small", tel, geom, [star], lay, seed=7)


@pytest.mark.parametrize("is_lgs,alt", [(False, 0.0), (True, 0.0), (True, 6000.0)])
def test_dm_layer_equal_to_minus_screen_cancels_exactly(is_lgs, alt):
    """A mirror layer at the screen's altitude holding minus the screen leaves a flat
    wavefront: the slopes equal those of zero screens bit for bit (any slip in the mirror
    layer's cone, shift or sign breaks it)."""
    cfg = _small_loop_cfg(is_lgs, alt)
    scr = inputs.make_screens(cfg.layers, 3)
    dm = inputs.Dm(11, 0.4, alt, 1)
    cfg2, scr2 = oracle.with_dm_layers(cfg, scr, [dm], [-scr[0]])
    s = oracle.measure(cfg2, scr2, 0.0)
    s0 = oracle.measure(cfg, np.zeros_like(scr), 0.0)
    np.testing.assert_array_equal(s, s0)
    assert np.abs(oracle.measure(cfg, scr, 0.0)).max() > 0.05   # the screen alone is not flat


def test_closed_loop_integrator_corrects_a_static_modal_aberration():
    """Pure integrator with unit gains and CM = pinv(IM), IM registered by push-pull of each
    mode in the beam: a static aberration made of the mirror's modes is removed in one step
    (linear regime), and the next slopes are near zero.  A sign slip doubles the residual."""
    cfg = _small_loop_cfg()
    S, ds = cfg.layers.screen_size, cfg.layers.screen_dx_m
    dm = inputs.Dm(11, 0.4, 0.0, 8, coupling=0.15, support=3)
    M = inputs.modal_base(dm, 11, amplitude_m=1e-8).astype(np.float64)
    # interaction matrix: slopes per unit coefficient of +mode in the beam (= minus its layer)
    IM = oracle.interaction_matrix(cfg, 0, [dm], [M], 0.5).T
    CM = np.linalg.pinv(IM)
    c_star = np.random.default_rng(2).standard_normal(dm.n_modes)
    ol = -oracle.dm_layer(dm, M @ c_star, S, ds)[None]
    gain = np.ones(dm.n_modes)
    s0, c1 = oracle.loop_step(cfg, ol, 0.0, [dm], [M], CM, gain, np.zeros(dm.n_modes))
    assert np.linalg.norm(c1 - c_star) < 0.05 * np.linalg.norm(c_star)
    s1, c2 = oracle.loop_step(cfg, ol, 0.0, [dm], [M], CM, gain, c1)
    assert np.linalg.norm(s1) < 0.05 * np.linalg.norm(s0)
    assert np.linalg.norm(c2 - c_star) <= np.linalg.norm(c1 - c_star) + 1e-12
    # gains of zero leave the coefficients alone; a wrong sign makes the residual worse
    _, c_same = oracle.loop_step(cfg, ol, 0.0, [dm], [M], CM, 0 * gain, c1)
    np.testing.assert_array_equal(c_same, c1)
    sb, cb = oracle.loop_step(cfg, ol, 0.0, [dm], [M], -CM, gain, np.zeros(dm.n_modes))
    sb1, _ = oracle.loop_step(cfg, ol, 0.0, [dm], [M], CM, gain, cb)
    assert np.linalg.norm(sb1) > 1.5 * np.linalg.norm(s0)


def test_interaction_matrix_push_pull():
    """Push-pull rows: the mode put in the beam as a screen (minus its mirror layer) gives the
    same slopes through the plain measurement; the central difference is odd in the amplitude
    and converges (halving the amplitude changes it by O(a^2)); a pure actuator-space tilt of
    the mirror gives x slopes of one sign and no mean y slope."""
    cfg = _small_loop_cfg()
    S, ds = cfg.layers.screen_size, cfg.layers.screen_dx_m
    dm = inputs.Dm(11, 0.4, 0.0, 3)
    M = inputs.modal_base(dm, 4, amplitude_m=1e-8).astype(np.float64)
    xa = (np.arange(11) - 5) * 0.4
    M[:, 2] = np.tile(xa, 11) * 2e-8                           # tilt along x: act ~ x_a
    a = 0.5
    IM = oracle.interaction_matrix(cfg, 0, [dm], [M], a)
    beam = -oracle.dm_layer(dm, M[:, 0] * a, S, ds)            # +a of mode 0 in the beam
    ref = (oracle.measure(cfg, beam[None], 0.0) - oracle.measure(cfg, -beam[None], 0.0)).ravel() / (2 * a)
    np.testing.assert_allclose(IM[0], ref, rtol=0, atol=1e-12)
    IMn = oracle.interaction_matrix(cfg, 0, [dm], [M], -a)
    np.testing.assert_allclose(IMn, IM, rtol=0, atol=1e-12)
    IMh = oracle.interaction_matrix(cfg, 0, [dm], [M], a / 2)
    assert np.linalg.norm(IMh - IM) < 0.05 * np.linalg.norm(IM)
    tilt = IM[2].reshape(-1, 2)
    assert np.all(tilt[:, 0] > 0) and abs(tilt[:, 1].mean()) < 1e-3 * tilt[:, 0].mean()


# ---------------------------------------------------------------- LGS uplink tip-tilt

def _linear_layers_cfg(slopes_xy, alts, S=512, dx=0.05):
    """Screens that are exact planes a x + b y (metres of OPD per metre) around the pupil."""
    n = len(alts)
    lay = inputs.Layers(alt_m=np.array(alts, float), wind_vx_mps=np.full(n, 3.0), wind_vy_mps=np.full(n, -2.0),
                        x0_m=np.zeros(n), y0_m=np.zeros(n), screen_size=S, screen_dx_m=dx)
    j = (np.arange(S) - S / 2) * dx
    X, Y = np.meshgrid(j, j)
    scr = np.stack([(a * X + b * Y).astype(np.float32) for a, b in slopes_xy])
    return lay, scr


def test_uplink_tilt_of_planar_layers_is_exact():
    """Planar layers: the footprint plane fit returns each layer's gradient exactly, and the
    deflections add with the lever arm (H - h) / H; zero for an NGS, without a beam, and for
    layers at or above the sodium."""
    ab = [(2e-6, -1e-6), (-5e-7, 3e-6), (1e-6, 1e-6)]
    alts = [0.0, 8000.0, 15000.0]
    lay, scr = _linear_layers_cfg(ab, alts)
    star = inputs._lgs(20 * inputs.ARCSEC, 10 * inputs.ARCSEC, 0.7, 0)
    star.uplink_diameter_m, star.uplink_samples = 0.5, 16
    cfg = inputs.Config("up", inputs.Telescope(8.0, 0.0), [inputs.Geometry(10, 8, 16, 8)], [star], lay, seed=1)
    H = star.range_m
    dx, dy = oracle.uplink_tilt(cfg, scr, 0, 0.01)
    ex = sum(a * (H - h) / H for (a, _), h in zip(ab, alts))
    ey = sum(b * (H - h) / H for (_, b), h in zip(ab, alts))
    assert dx == pytest.approx(ex, rel=1e-6) and dy == pytest.approx(ey, rel=1e-6)
    star.uplink_diameter_m = 0.0
    assert oracle.uplink_tilt(cfg, scr, 0, 0.01) == (0.0, 0.0)
    ngs = inputs._ngs(0.0, 0.0, 700e-9, 0)
    ngs.uplink_diameter_m = 0.5
    cfg.stars = [ngs]
    assert oracle.uplink_tilt(cfg, scr, 0, 0.01) == (0.0, 0.0)


def test_uplink_tilt_equals_a_ground_tilt_layer():
    """The measurement adds the uplink tilt to the pupil OPD: the slopes equal those without
    uplink plus a ground layer that is exactly the plane dx x + dy y."""
    cfg = _small_loop_cfg(is_lgs=True)
    scr = inputs.make_screens(cfg.layers, 5)
    cfg.stars[0].uplink_diameter_m = 0.4
    cfg.stars[0].uplink_samples = 12
    dx, dy = oracle.uplink_tilt(cfg, scr, 0, 0.0)
    assert abs(dx) + abs(dy) > 1e-8
    s_up = oracle.measure(cfg, scr, 0.0)
    S, ds = cfg.layers.screen_size, cfg.layers.screen_dx_m
    j = (np.arange(S) - S / 2) * ds
    X, Y = np.meshgrid(j, j)
    plane = (dx * X + dy * Y).astype(np.float32)
    cfg_off = dataclasses.replace(cfg, stars=[dataclasses.replace(cfg.stars[0], uplink_diameter_m=0.0)])
    cfg2, scr2 = oracle.with_dm_layers(cfg_off, scr, [inputs.Dm(3, 1.0, 0.0, 1)], [plane])
    s_ref = oracle.measure(cfg2, scr2, 0.0)
    np.testing.assert_allclose(s_up, s_ref, rtol=0, atol=1e-6)
    assert np.abs(s_up - oracle.measure(cfg_off, scr, 0.0)).max() > 1e-3


# ---------------------------------------------------------------- LGS per-slice model

def _slice_cfg(alts_layers, S=256, dx=0.05, seed=9):
    """4 m telescope, 10 x 10 subapertures of 8 px (N = 16), one LGS 5 m launch, 3 slices."""
    tel = inputs.Telescope(4.0, 0.0)
    geom = [inputs.Geometry(10, 8, 16, 8, 0.5, inputs.PREC_FP32)]
    h, w = inputs.sodium_slices(90e3, 10e3, 3)
    star = inputs._lgs(15 * inputs.ARCSEC, -10 * inputs.ARCSEC, 0.6, 0, fwhm=1.0 * inputs.ARCSEC, na=(h, w))
    n = len(alts_layers)
    lay = inputs.Layers(alt_m=np.array(alts_layers, float), wind_vx_mps=np.full(n, 4.0), wind_vy_mps=np.zeros(n),
                        x0_m=np.zeros(n), y0_m=np.zeros(n), screen_size=S, screen_dx_m=dx,
                        weights=np.full(n, 1.0 / n))
    return inputs.Config("slices", tel, geom, [star], lay, seed=seed)


def test_per_slice_single_slice_at_focus_is_the_kernel_model():
    cfg = _slice_cfg([0.0, 7000.0])
    scr = inputs.make_screens(cfg.layers, 2)
    st = cfg.stars[0]
    one = dataclasses.replace(st, na_alt_m=np.array([st.range_m]), na_weight=np.array([1.0]))
    a = oracle.measure_wfs(dataclasses.replace(cfg, stars=[one]), scr, 0, 0.01, stages=True)
    b = oracle.measure_wfs(dataclasses.replace(cfg, stars=[dataclasses.replace(one, per_slice=True)]), scr, 0, 0.01,
                           stages=True)
    for k in ("slopes", "I", "Ie", "E"):
        np.testing.assert_array_equal(a[k], b[k])


def test_per_slice_slice_equals_cone_plus_geometric_screen():
    """One slice at h_s: the layers seen with the cone 1 - h/h_s and the slice's geometric
    term 1/2 |x - r_L|^2 (1/h0 - 1/h_s).  Built independently: a star at range h_s (cone, no
    offset) plus a ground screen holding that quadratic (bilinear at pixel centres adds only a
    constant) gives the same spot to FP32 rounding of the screen."""
    cfg = _slice_cfg([5000.0])
    scr = inputs.make_screens(cfg.layers, 4)
    st = cfg.stars[0]
    hs, h0 = 84e3, st.range_m
    sl = dataclasses.replace(st, na_alt_m=np.array([hs]), na_weight=np.array([1.0]), per_slice=True)
    a = oracle.measure_wfs(dataclasses.replace(cfg, stars=[sl]), scr, 0, 0.0, stages=True)
    ref_star = dataclasses.replace(st, range_m=hs, na_alt_m=np.array([hs]), na_weight=np.array([1.0]))
    S, ds = cfg.layers.screen_size, cfg.layers.screen_dx_m
    j = (np.arange(S) - S / 2) * ds
    X, Y = np.meshgrid(j, j)
    quad = 0.5 * ((X - st.launch_x_m) ** 2 + (Y - st.launch_y_m) ** 2) * (1 / h0 - 1 / hs)
    cfg2, scr2 = oracle.with_dm_layers(dataclasses.replace(cfg, stars=[ref_star]), scr,
                                       [inputs.Dm(3, 1.0, 0.0, 1)], [quad.astype(np.float32)])
    # the spot's physical extent is an angle: the Gaussian is the same for both stars
    b = oracle.measure_wfs(cfg2, scr2, 0, 0.0, stages=True)
    rel = np.abs(a["Ie"] - b["Ie"]).max() / np.abs(b["Ie"]).max()
    assert rel < 1e-5, rel
    np.testing.assert_allclose(a["slopes"], b["slopes"], atol=1e-5)
    # the quadratic moves the spot: without it the slopes differ
    c = oracle.measure_wfs(dataclasses.replace(cfg, stars=[ref_star]), scr, 0, 0.0)
    assert np.abs(c["slopes"] - a["slopes"]).max() > 0.05


def test_per_slice_pile_up_is_linear_in_the_profile():
    cfg = _slice_cfg([0.0, 7000.0])
    scr = inputs.make_screens(cfg.layers, 6)
    st = dataclasses.replace(cfg.stars[0], per_slice=True)
    wa = np.array([0.2, 0.0, 0.5])
    wb = np.array([0.0, 0.7, 0.1])
    Ie = lambda w: oracle.measure_wfs(dataclasses.replace(cfg, stars=[dataclasses.replace(st, na_weight=w)]),
                                      scr, 0, 0.0, stages=True)["Ie"]
    np.testing.assert_allclose(Ie(wa + wb), Ie(wa) + Ie(wb), rtol=0, atol=1e-12 * np.abs(Ie(wa + wb)).max())
    # and close to the elongation-kernel model (same slices, one projection)
    s_slice = oracle.measure_wfs(dataclasses.replace(cfg, stars=[st]), scr, 0, 0.0)["slopes"]
    s_kern = oracle.measure_wfs(cfg, scr, 0, 0.0)["slopes"]
    assert np.sqrt(np.mean((s_slice - s_kern) ** 2)) < 0.02
