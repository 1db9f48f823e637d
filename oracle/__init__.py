"""FP64 CPU oracle of the open-loop Shack-Hartmann measurement.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library (``paper_1408_0698_gb300``); both are written from the paper
(Arcidiacono et al. 2014, Sec. 4 "Open Loop generation" and "LGS Shack Hartmann
wavefront sensor") and compared element by element.

The arithmetic lives in ``oracle.c`` (plain C, FP64, brute-force definitions);
this module only builds it and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O3, OpenMP, no FP contraction; no machine-specific flags, so
    the x86 and Arm builds give the same results)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Geom(C.Structure):
    _fields_ = [("diameter_m", C.c_double), ("obstruction", C.c_double), ("n_sub", C.c_int),
                ("n", C.c_int), ("N", C.c_int), ("n_det", C.c_int), ("valid_fill", C.c_double)]


class _Star(C.Structure):
    _fields_ = [("is_lgs", C.c_int), ("theta_x", C.c_double), ("theta_y", C.c_double),
                ("range_m", C.c_double), ("wavelength_m", C.c_double), ("launch_x", C.c_double),
                ("launch_y", C.c_double), ("spot_fwhm_rad", C.c_double), ("photons", C.c_double),
                ("read_noise", C.c_double), ("n_na", C.c_int),
                ("na_alt", C.POINTER(C.c_double)), ("na_weight", C.POINTER(C.c_double)),
                ("up_diameter", C.c_double), ("up_samples", C.c_int), ("slices", C.c_int)]


class _Layers(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("S", C.c_int), ("dx", C.c_double),
                ("alt", C.POINTER(C.c_double)), ("vx", C.POINTER(C.c_double)),
                ("vy", C.POINTER(C.c_double)), ("x0", C.POINTER(C.c_double)),
                ("y0", C.POINTER(C.c_double)), ("n_atm", C.c_int)]


class _Dm(C.Structure):
    _fields_ = [("n_act", C.c_int), ("pitch_m", C.c_double), ("alt_m", C.c_double),
                ("coupling", C.c_double), ("support", C.c_int)]


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            L.orc_pupil_mask.argtypes = [C.c_double, C.c_double, C.c_int, C.POINTER(C.c_uint8)]
            L.orc_valid_subaps.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, _ip, _dp]
            L.orc_valid_subaps.restype = C.c_int
            L.orc_bilinear.argtypes = [_fp, C.c_int, C.c_double, C.c_double]
            L.orc_bilinear.restype = C.c_double
            L.orc_opd.argtypes = [C.POINTER(_Layers), _fp, C.POINTER(_Star), C.c_double, C.c_double, C.c_double]
            L.orc_opd.restype = C.c_double
            L.orc_project_grid.argtypes = [C.c_double, C.c_int, C.POINTER(_Layers), _fp, C.POINTER(_Star), C.c_double, _dp]
            L.orc_dft2.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp]
            L.orc_elong_kernel.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(_Star), _dp]
            L.orc_convolve.argtypes = [C.c_int, _dp, _dp, _dp]
            L.orc_elong_convolve_separable.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                                       C.POINTER(_Star), _dp, _dp]
            L.orc_elong_convolve_separable.restype = None
            L.orc_set_separable.argtypes = [C.c_int]
            L.orc_set_separable.restype = None
            L.orc_bin.argtypes = [C.c_int, C.c_int, _dp, _dp]
            L.orc_philox.argtypes = [_up, _up, _up]
            L.orc_poisson_inversion_n.argtypes = [C.c_float, C.c_int, _fp, _ip]
            L.orc_poisson_inversion_n.restype = None
            L.orc_noise_pixel.argtypes = [C.c_float, C.c_float, C.c_uint64, C.c_uint32, C.c_uint32, C.c_double, _ip]
            L.orc_noise_pixel.restype = C.c_double
            L.orc_noise_image.argtypes = [C.c_int, _fp, C.c_float, C.c_uint64, C.c_uint32, C.c_double, C.c_uint32, _dp, _ip]
            L.orc_cog.argtypes = [C.c_int, _dp, _dp, _dp]
            L.orc_measure_wfs.argtypes = [C.POINTER(_Geom), C.POINTER(_Star), C.c_int, C.POINTER(_Layers), _fp,
                                          C.c_double, C.c_uint64, C.c_int, C.c_int, _ip, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_measure_wfs.restype = C.c_int
            L.orc_dm_value.argtypes = [C.POINTER(_Dm), _dp, C.c_double, C.c_double]
            L.orc_dm_value.restype = C.c_double
            L.orc_dm_layer.argtypes = [C.POINTER(_Dm), _dp, C.c_int, C.c_double, _fp]
            L.orc_uplink_tilt.argtypes = [C.POINTER(_Layers), _fp, C.POINTER(_Star), C.c_double, _dp, _dp]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = None
        return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Keep:
    """Holds the numpy arrays that ctypes structs point into."""

    def __init__(self):
        self.refs = []

    def d(self, a):
        a = _f64(a)
        self.refs.append(a)
        return _ptr(a, _dp)


def _star(gs, keep):
    s = _Star()
    s.is_lgs = int(bool(gs.is_lgs))
    s.theta_x, s.theta_y = gs.theta_x_rad, gs.theta_y_rad
    s.range_m = gs.range_m if gs.is_lgs else math.inf
    s.wavelength_m = gs.wavelength_m
    s.launch_x, s.launch_y = gs.launch_x_m, gs.launch_y_m
    s.spot_fwhm_rad = gs.spot_fwhm_rad
    s.photons, s.read_noise = gs.photons_per_subap, gs.read_noise_e
    s.n_na = len(gs.na_alt_m) if gs.is_lgs else 0
    s.na_alt = keep.d(gs.na_alt_m if len(gs.na_alt_m) else [0.0])
    s.na_weight = keep.d(gs.na_weight if len(gs.na_weight) else [0.0])
    s.up_diameter = float(getattr(gs, "uplink_diameter_m", 0.0)) if gs.is_lgs else 0.0
    s.up_samples = int(getattr(gs, "uplink_samples", 0))
    s.slices = int(bool(getattr(gs, "per_slice", False))) if gs.is_lgs else 0
    return s


def _layers(lay, keep):
    L = _Layers()
    L.n_layers, L.S, L.dx = lay.n_layers, lay.screen_size, lay.screen_dx_m
    L.alt, L.vx, L.vy = keep.d(lay.alt_m), keep.d(lay.wind_vx_mps), keep.d(lay.wind_vy_mps)
    L.x0, L.y0 = keep.d(lay.x0_m), keep.d(lay.y0_m)
    L.n_atm = lay.n_layers - int(getattr(lay, "n_mirrors", 0))
    return L


def _geom(tel, g):
    G = _Geom()
    G.diameter_m, G.obstruction = tel.diameter_m, tel.obstruction
    G.n_sub, G.n, G.N, G.n_det, G.valid_fill = g.n_sub, g.n_pix_sub, g.n_fft, g.n_det, g.valid_fill
    return G


# ---------------------------------------------------------------- public wrappers

def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (timing only; results do not depend on it)."""
    lib().orc_set_threads(int(n))


def pupil_mask(D, eps, Np):
    m = np.zeros((Np, Np), dtype=np.uint8)
    lib().orc_pupil_mask(D, eps, Np, m.ctypes.data_as(C.POINTER(C.c_uint8)))
    return m


def valid_subaps(D, eps, n_sub, n, thr=0.5):
    cap = n_sub * n_sub
    idx = np.zeros(cap, dtype=np.int32)
    fill = np.zeros(cap, dtype=np.float64)
    c = lib().orc_valid_subaps(D, eps, n_sub, n, thr, _ptr(idx, _ip), _ptr(fill, _dp))
    return idx[:c].copy(), fill[:c].copy()


def bilinear(screen, u, v):
    s = np.ascontiguousarray(screen, dtype=np.float32)
    return lib().orc_bilinear(_ptr(s, _fp), s.shape[0], float(u), float(v))


def opd(cfg, screens, star_index, x, y, t):
    keep = _Keep()
    L = _layers(cfg.layers, keep)
    s = _star(cfg.stars[star_index], keep)
    sc = np.ascontiguousarray(screens, dtype=np.float32)
    return lib().orc_opd(C.byref(L), _ptr(sc, _fp), C.byref(s), x, y, t)


def project_grid(cfg, screens, star_index, t):
    gs = cfg.stars[star_index]
    g = cfg.geometries[gs.geometry_index]
    Np = g.n_sub * g.n_pix_sub
    keep = _Keep()
    L = _layers(cfg.layers, keep)
    s = _star(gs, keep)
    sc = np.ascontiguousarray(screens, dtype=np.float32)
    out = np.zeros((Np, Np), dtype=np.float64)
    lib().orc_project_grid(cfg.telescope.diameter_m, Np, C.byref(L), _ptr(sc, _fp), C.byref(s), t,
                           _ptr(out, _dp))
    return out


def dft2(X, N):
    X = np.asarray(X, dtype=np.complex128)
    n = X.shape[0]
    xr, xi = _f64(X.real), _f64(X.imag)
    yr = np.zeros((N, N)); yi = np.zeros((N, N))
    lib().orc_dft2(n, N, _ptr(xr, _dp), _ptr(xi, _dp), _ptr(yr, _dp), _ptr(yi, _dp))
    return yr + 1j * yi


def elong_kernel(N, pix_rad, rbx, rby, star):
    keep = _Keep()
    s = _star(star, keep)
    K = np.zeros((N, N))
    lib().orc_elong_kernel(N, pix_rad, rbx, rby, C.byref(s), _ptr(K, _dp))
    return K


def elong_convolve_separable(I, pix_rad, rbx, rby, star):
    """The elongation (kernel of elong_kernel, convolution of convolve) in separable form."""
    keep = _Keep()
    s = _star(star, keep)
    I = _f64(I)
    out = np.zeros_like(I)
    lib().orc_elong_convolve_separable(I.shape[0], pix_rad, rbx, rby, C.byref(s), _ptr(I, _dp), _ptr(out, _dp))
    return out


def set_separable(on: bool) -> None:
    """measure_wfs's elongation form: the direct periodic convolution (default, parity) or the
    separable form (timing)."""
    lib().orc_set_separable(int(bool(on)))


def convolve(I, K):
    I, K = _f64(I), _f64(K)
    out = np.zeros_like(I)
    lib().orc_convolve(I.shape[0], _ptr(I, _dp), _ptr(K, _dp), _ptr(out, _dp))
    return out


def bin_image(I, nd):
    I = _f64(I)
    B = np.zeros((nd, nd))
    lib().orc_bin(I.shape[0], nd, _ptr(I, _dp), _ptr(B, _dp))
    return B


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_ptr(c, _up), _ptr(k, _up), _ptr(o, _up))
    return o


def poisson_inversion(E, u):
    """The sampler's inversion branch (E < 16) on given FP32 uniforms: the counts it returns."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    k = np.empty(u.size, np.int32)
    lib().orc_poisson_inversion_n(float(E), u.size, _ptr(u, _fp), _ptr(k, _ip))
    return k


def noise_image(E, read_noise, seed, wfs, t, pixel0=0):
    E = np.ascontiguousarray(E, dtype=np.float32).ravel()
    Cc = np.zeros(E.size, dtype=np.float64)
    K = np.zeros(E.size, dtype=np.int32)
    lib().orc_noise_image(E.size, _ptr(E, _fp), float(read_noise), int(seed), int(wfs), float(t),
                          int(pixel0), _ptr(Cc, _dp), _ptr(K, _ip))
    return Cc, K


def cog(Cimg):
    Cimg = _f64(Cimg)
    sx, sy = C.c_double(), C.c_double()
    lib().orc_cog(Cimg.shape[0], _ptr(Cimg, _dp), C.byref(sx), C.byref(sy))
    return sx.value, sy.value


def measure_wfs(cfg, screens, star_index, t, seed=0, noise=False, sel=None, stages=False):
    """Measure one WFS; returns a dict with 'slopes' [n_sel, 2] and, with
    stages=True, 'opd', 'I', 'Ie', 'E', 'C' per selected subap."""
    gs = cfg.stars[star_index]
    g = cfg.geometries[gs.geometry_index]
    keep = _Keep()
    G = _geom(cfg.telescope, g)
    L = _layers(cfg.layers, keep)
    s = _star(gs, keep)
    sc = np.ascontiguousarray(screens, dtype=np.float32)
    if sel is None:
        nv = len(valid_subaps(cfg.telescope.diameter_m, cfg.telescope.obstruction, g.n_sub,
                              g.n_pix_sub, g.valid_fill)[0])
        n_sel, selp = nv, None
    else:
        sel = np.ascontiguousarray(sel, dtype=np.int32)
        n_sel, selp = len(sel), _ptr(sel, _ip)
    n, N, nd = g.n_pix_sub, g.n_fft, g.n_det
    out = {"slopes": np.zeros((n_sel, 2))}
    if stages:
        out["opd"] = np.zeros((n_sel, n, n))
        out["I"] = np.zeros((n_sel, N, N))
        out["Ie"] = np.zeros((n_sel, N, N))
        out["E"] = np.zeros((n_sel, nd, nd))
        out["C"] = np.zeros((n_sel, nd, nd))
    gp = lambda k: _ptr(out[k], _dp) if k in out else None
    rc = lib().orc_measure_wfs(C.byref(G), C.byref(s), star_index, C.byref(L), _ptr(sc, _fp), t,
                               int(seed), int(bool(noise)), n_sel, selp, gp("slopes"), gp("opd"),
                               gp("I"), gp("Ie"), gp("E"), gp("C"))
    if rc < 0:
        raise ValueError("oracle: bad geometry")
    return out


def measure(cfg, screens, t, seed=0, noise=False):
    """All guide stars of a configuration: slopes concatenated [sum_w n_valid_w, 2]."""
    return np.concatenate([measure_wfs(cfg, screens, w, t, seed, noise)["slopes"]
                           for w in range(len(cfg.stars))], axis=0)


# ---------------------------------------------------------------- closed loop
# Sec. 3 "Influence function and modal base" and "The closed loop": the mirrors are linear
# combinations of a modal base defined on their actuators; the sensors measure the open-loop
# wavefront minus the mirrors; the slopes times the control matrix are the differential
# coefficients added to the mirror's (pure integrator, one gain per mode).

def _dm(d):
    return _Dm(int(d.n_act), float(d.pitch_m), float(d.alt_m), float(d.coupling), int(d.support))


def dm_value(dm, act, x, y):
    """Correction-layer value (minus the mirror shape) at (x, y) metres in the mirror's plane."""
    a = _f64(np.asarray(act).ravel())
    D = _dm(dm)
    return lib().orc_dm_value(C.byref(D), _ptr(a, _dp), float(x), float(y))


def dm_layer(dm, act, S, ds):
    """[S, S] float32 correction layer of one mirror with actuator commands act [n_act^2]."""
    a = _f64(np.asarray(act).ravel())
    if a.size != dm.n_act * dm.n_act:
        raise ValueError("act must hold n_act^2 commands")
    out = np.zeros((S, S), dtype=np.float32)
    D = _dm(dm)
    lib().orc_dm_layer(C.byref(D), _ptr(a, _dp), int(S), float(ds), _ptr(out, _fp))
    return out


def with_dm_layers(cfg, screens, dms, layers):
    """The configuration and screens with each mirror's correction layer appended as one more
    layer at the mirror's altitude, without wind or initial offset."""
    lay = cfg.layers
    k = len(dms)
    z = np.zeros(k)
    lay2 = dataclasses.replace(
        lay, alt_m=np.concatenate([_f64(lay.alt_m), [float(d.alt_m) for d in dms]]),
        wind_vx_mps=np.concatenate([_f64(lay.wind_vx_mps), z]),
        wind_vy_mps=np.concatenate([_f64(lay.wind_vy_mps), z]),
        x0_m=np.concatenate([_f64(lay.x0_m), z]), y0_m=np.concatenate([_f64(lay.y0_m), z]),
        n_mirrors=int(getattr(lay, "n_mirrors", 0)) + k)
    cfg2 = dataclasses.replace(cfg, layers=lay2)
    scr = np.concatenate([np.asarray(screens, dtype=np.float32),
                          np.stack([np.asarray(l, dtype=np.float32) for l in layers])], axis=0)
    return cfg2, scr


def actuators(dms, m2a, coeffs):
    """Per mirror: its actuator commands m2a_d @ c_d, c_d its slice of the coefficient vector."""
    out, o = [], 0
    for d, M in zip(dms, m2a):
        M = _f64(M)
        out.append(M @ _f64(coeffs)[o:o + M.shape[1]])
        o += M.shape[1]
    return out


def loop_step(cfg, screens, t, dms, m2a, cm, gain, coeffs, seed=0, noise=False):
    """One integrator step: the slopes [n, 2] of the residual seen through the mirrors whose
    modal coefficients are ``coeffs``, and the next coefficients coeffs + gain * (cm @ s)."""
    S, ds = cfg.layers.screen_size, cfg.layers.screen_dx_m
    layers = [dm_layer(d, a, S, ds) for d, a in zip(dms, actuators(dms, m2a, coeffs))]
    cfg2, scr2 = with_dm_layers(cfg, screens, dms, layers)
    s = measure(cfg2, scr2, t, seed, noise)
    return s, _f64(coeffs) + _f64(gain) * (_f64(cm) @ s.ravel())


def interaction_matrix(cfg, star_index, dms, m2a, amplitude, modes=None):
    """Push-pull registration (Sec. 3 "The calibration of the interaction matrices"; Sec. 5: a
    modal push-pull scheme): for each mode m, the slopes of guide star ``star_index`` with
    +amplitude of the mode in the beam (mirror coefficient -amplitude) minus those with
    -amplitude, over 2 amplitude; no turbulence, no noise, t = 0.  Returns [len(modes), 2 n_valid]
    (row m: slopes x, y interleaved per subaperture)."""
    n = sum(M.shape[1] for M in m2a)
    modes = range(n) if modes is None else modes
    S, ds = cfg.layers.screen_size, cfg.layers.screen_dx_m
    empty = dataclasses.replace(cfg.layers, alt_m=np.zeros(0), wind_vx_mps=np.zeros(0),
                                wind_vy_mps=np.zeros(0), x0_m=np.zeros(0), y0_m=np.zeros(0), n_mirrors=0)
    cfg0 = dataclasses.replace(cfg, layers=empty)
    no_screens = np.zeros((0, S, S), np.float32)
    rows = []
    for m in modes:
        s = []
        for sign in (-1.0, 1.0):
            c = np.zeros(n)
            c[m] = sign * amplitude
            layers = [dm_layer(d, a, S, ds) for d, a in zip(dms, actuators(dms, m2a, c))]
            cfg2, scr2 = with_dm_layers(cfg0, no_screens, dms, layers)
            s.append(measure_wfs(cfg2, scr2, star_index, 0.0)["slopes"].ravel())
        rows.append((s[0] - s[1]) / (2.0 * amplitude))
    return np.array(rows)


def uplink_tilt(cfg, screens, star_index, t):
    """(dx, dy) radians: the LGS uplink tip-tilt that moves the whole spot."""
    keep = _Keep()
    L = _layers(cfg.layers, keep)
    s = _star(cfg.stars[star_index], keep)
    sc = np.ascontiguousarray(screens, dtype=np.float32)
    dx, dy = C.c_double(), C.c_double()
    lib().orc_uplink_tilt(C.byref(L), _ptr(sc, _fp), C.byref(s), float(t), C.byref(dx), C.byref(dy))
    return dx.value, dy.value
