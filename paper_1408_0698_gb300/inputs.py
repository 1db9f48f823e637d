"""Seeded synthetic inputs for the Shack-Hartmann measurement path.

This module is shared by the CUDA library's tests and benchmark and by the
FP64 oracle's tests.  It holds *no* arithmetic of the measurement itself
(no pupil mask, no projection, no DFT, no elongation, no noise, no
centroid): only

* the parameter sets of the workloads (telescope, guide stars, wavefront-sensor
  geometries, turbulence layers, sodium profile sampling), and
* the generation of frozen-flow phase screens from a von Karman power
  spectrum (Sec. 3, first block: screens are made by FFT from a Kolmogorov or
  von Karman phase spectrum), returned as FP32 optical path difference in
  metres.

Every generator takes an explicit seed; nothing depends on global state.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

ARCSEC = math.pi / 180.0 / 3600.0
#: Wavelength (m) at which r0 is quoted and at which screen phase is defined.
R0_WAVELENGTH = 500e-9
#: Sodium D2 line, the LGS wavelength.
LAMBDA_NA = 589e-9

PREC_FP32 = 0
PREC_BF16X3 = 1
PREC_FP16S = 2


@dataclass
class Telescope:
    diameter_m: float
    obstruction: float = 0.0


@dataclass
class Geometry:
    n_sub: int          # subapertures across the pupil
    n_pix_sub: int      # pupil pixels across one subaperture (n)
    n_fft: int          # padded DFT size (N)
    n_det: int          # detector pixels across one subaperture
    valid_fill: float = 0.5
    precision: int = PREC_FP32


@dataclass
class GuideStar:
    is_lgs: bool
    theta_x_rad: float
    theta_y_rad: float
    range_m: float                # math.inf for a natural guide star
    wavelength_m: float
    geometry_index: int
    photons_per_subap: float = 500.0
    read_noise_e: float = 3.0
    launch_x_m: float = 0.0
    launch_y_m: float = 0.0
    spot_fwhm_rad: float = 0.0
    na_alt_m: np.ndarray = field(default_factory=lambda: np.zeros(0))
    na_weight: np.ndarray = field(default_factory=lambda: np.zeros(0))
    uplink_diameter_m: float = 0.0   # LGS launch beam diameter; 0 = no uplink tip-tilt
    uplink_samples: int = 16         # samples across the launch beam
    per_slice: bool = False          # LGS: one wavefront and DFT per sodium slice


@dataclass
class Layers:
    alt_m: np.ndarray
    wind_vx_mps: np.ndarray
    wind_vy_mps: np.ndarray
    x0_m: np.ndarray
    y0_m: np.ndarray
    screen_size: int
    screen_dx_m: float
    # generation-only parameters (not part of the measurement)
    r0_m: float = 0.15
    L0_m: float = 25.0
    weights: np.ndarray = field(default_factory=lambda: np.ones(1))
    n_mirrors: int = 0   # trailing layers that are mirror correction layers (closed loop)

    @property
    def n_layers(self) -> int:
        return int(len(self.alt_m))


@dataclass
class Config:
    name: str
    telescope: Telescope
    geometries: List[Geometry]
    stars: List[GuideStar]
    layers: Layers
    seed: int
    dt_s: float = 1e-3
    steps: int = 10

    def with_precision(self, precision: int) -> "Config":
        c = dataclasses.replace(self)
        c.geometries = [dataclasses.replace(g, precision=precision) for g in self.geometries]
        return c


# ---------------------------------------------------------------------------
# Sodium profile sampling (input description of the LGS, Sec. 4 LGS SH:
# the sodium layer is cut into sub-layers weighted by its density profile).
# ---------------------------------------------------------------------------
def sodium_slices(h0_m: float = 90e3, fwhm_m: float = 10e3, n_slices: int = 8):
    """Gaussian sodium density sampled in ``n_slices`` equal slices spanning
    +-FWHM about the centroid; weights normalised to sum to one."""
    dh = 2.0 * fwhm_m / n_slices
    s = np.arange(n_slices, dtype=np.float64)
    h = h0_m + (s - (n_slices - 1) / 2.0) * dh
    sigma = fwhm_m / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    w = np.exp(-0.5 * ((h - h0_m) / sigma) ** 2)
    return h, w / w.sum()


def _ring(n: int, radius_rad: float, phase_deg: float = 0.0):
    out = []
    for k in range(n):
        a = math.radians(phase_deg + 360.0 * k / n)
        out.append((radius_rad * math.cos(a), radius_rad * math.sin(a), a))
    return out


def _lgs(theta_x, theta_y, azimuth, geom, launch_r=5.0, range_m=90e3, fwhm=1.0 * ARCSEC,
         photons=500.0, ron=3.0, na=None):
    h, w = na if na is not None else sodium_slices(range_m)
    return GuideStar(is_lgs=True, theta_x_rad=theta_x, theta_y_rad=theta_y, range_m=range_m,
                     wavelength_m=LAMBDA_NA, geometry_index=geom, photons_per_subap=photons,
                     read_noise_e=ron, launch_x_m=launch_r * math.cos(azimuth),
                     launch_y_m=launch_r * math.sin(azimuth), spot_fwhm_rad=fwhm,
                     na_alt_m=h.copy(), na_weight=w.copy())


def _ngs(theta_x, theta_y, wavelength, geom, photons=500.0, ron=3.0):
    return GuideStar(is_lgs=False, theta_x_rad=theta_x, theta_y_rad=theta_y, range_m=math.inf,
                     wavelength_m=wavelength, geometry_index=geom, photons_per_subap=photons,
                     read_noise_e=ron)


def _layers(alts, weights, r0, L0, S, dx, speed=10.0, dirs_deg=None):
    alts = np.asarray(alts, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    if dirs_deg is None:
        dirs_deg = [36.0 * l for l in range(len(alts))]
    d = np.radians(np.asarray(dirs_deg, dtype=np.float64))
    return Layers(alt_m=alts, wind_vx_mps=speed * np.cos(d), wind_vy_mps=speed * np.sin(d),
                  x0_m=np.zeros(len(alts)), y0_m=np.zeros(len(alts)), screen_size=S,
                  screen_dx_m=dx, r0_m=r0, L0_m=L0, weights=w)


# ---------------------------------------------------------------------------
# The five workloads.
# ---------------------------------------------------------------------------
def config1(precision: int = PREC_FP32) -> Config:
    """8 m, one on-axis NGS at 700 nm, 20x20 subaps of 8 px padded to 16, 8x8 det px."""
    tel = Telescope(8.0, 0.0)
    geom = [Geometry(20, 8, 16, 8, 0.5, precision)]
    stars = [_ngs(0.0, 0.0, 700e-9, 0, photons=500.0)]
    lay = _layers([0.0], [1.0], 0.15, 25.0, 256, 0.05, dirs_deg=[0.0])
    return Config("config1_ngs_20x20", tel, geom, stars, lay, seed=1000, dt_s=1e-3, steps=10)


def config2(precision: int = PREC_FP32) -> Config:
    """8 m MCAO: 3 LGS on a 60" ring + 1 on-axis NGS, 40x40 subaps of 6 px padded to 24."""
    tel = Telescope(8.0, 0.0)
    geom = [Geometry(40, 6, 24, 12, 0.5, precision)]
    stars = [_lgs(tx, ty, az, 0) for (tx, ty, az) in _ring(3, 60.0 * ARCSEC)]
    stars.append(_ngs(0.0, 0.0, 700e-9, 0, photons=500.0))
    lay = _layers([0.0, 4e3, 10e3], [0.6, 0.25, 0.15], 0.12, 25.0, 512, 8.0 / 240.0)
    return Config("config2_mcao_8m", tel, geom, stars, lay, seed=2000, dt_s=1e-3, steps=100)


def config3(precision: int = PREC_BF16X3, ngs_precision: int = PREC_FP32) -> Config:
    """ELT: 800x800 px pupil at 4.875e-2 m, obstruction 0.28; 6 LGS (80x80, n=10, N=32,
    16x16 det px) on a 45" ring; 3 H-band NGS 2x2 (n=32, N=64, 32x32 det px) on a 60" ring;
    10 layers 0-20 km.  `precision` is the LGS geometry's DFT arithmetic, `ngs_precision` the
    NGS geometry's (None: the same as the LGS).  The 12 NGS spots default to FP32: on their side
    stream the FP32 kernel's 512-thread teams finish them sooner than the 64-point tensor-core
    kernel's single warpgroup per two subapertures."""
    dx = 4.875e-2
    tel = Telescope(800 * dx, 0.28)
    geom = [Geometry(80, 10, 32, 16, 0.5, precision),
            Geometry(2, 32, 64, 32, 0.5, precision if ngs_precision is None else ngs_precision)]
    stars = [_lgs(tx, ty, az, 0) for (tx, ty, az) in _ring(6, 45.0 * ARCSEC)]
    stars += [_ngs(tx, ty, 1650e-9, 1, photons=5000.0) for (tx, ty, _) in _ring(3, 60.0 * ARCSEC)]
    alts = np.linspace(0.0, 20e3, 10)
    w = [0.5, 0.1, 0.08, 0.07, 0.06, 0.05, 0.045, 0.035, 0.03, 0.03]
    lay = _layers(alts, w, 0.157, 25.0, 2048, dx)
    return Config("config3_elt_6lgs_3ngs", tel, geom, stars, lay, seed=3000, dt_s=1e-3, steps=500)


#: Geometries drawn by the uneven-batch workload (n_sub, n, N, n_det).
BATCH_GEOMETRIES = [(2, 32, 64, 32), (10, 8, 16, 8), (40, 6, 24, 12), (80, 10, 32, 16)]


def config4_instances(n_instances: int = 64, seed: int = 4000,
                      precision: int = PREC_BF16X3) -> List[Config]:
    """Uneven batch: each instance is a one-WFS 8 m telescope whose geometry is drawn from
    BATCH_GEOMETRIES, with 1-10 layers, an LGS with probability 0.5 (never for 2x2)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        g = BATCH_GEOMETRIES[int(rng.integers(len(BATCH_GEOMETRIES)))]
        n_sub, n, N, nd = g
        D = 8.0
        dx = D / (n_sub * n)
        n_layers = int(rng.integers(1, 11))
        alts = np.sort(rng.uniform(0.0, 15e3, n_layers))
        alts[0] = 0.0
        w = rng.uniform(0.2, 1.0, n_layers)
        S = 1 << int(math.ceil(math.log2(max(64, 1.5 * (D / dx) + 64))))
        lay = _layers(alts, w, 0.12, 25.0, S, dx)
        lgs = (n_sub > 2) and bool(rng.integers(2))
        az = float(rng.uniform(0.0, 2 * math.pi))
        r = float(rng.uniform(0.0, 60.0)) * ARCSEC
        if lgs:
            star = _lgs(r * math.cos(az), r * math.sin(az), az, 0)
        else:
            star = _ngs(r * math.cos(az), r * math.sin(az), 700e-9, 0,
                        photons=5000.0 if n_sub == 2 else 500.0)
        out.append(Config(f"batch{i}_{n_sub}x{n_sub}_{'lgs' if lgs else 'ngs'}",
                          Telescope(D, 0.0), [Geometry(n_sub, n, N, nd, 0.5, precision)],
                          [star], lay, seed=seed + 1 + i))
    return out


# ---------------------------------------------------------------------------
# Deformable mirrors and control matrices of the closed loop (Sec. 2: ~5000 modes for
# the ground-layer mirror, ~1400 and ~1800 for two post-focal mirrors with a 1 m actuator
# pitch on the primary; Sec. 3: the mirrors are combinations of a modal base over their
# actuators, the control matrix maps slopes to modal coefficients).  Only descriptions
# and seeded random matrices here: the modal base and the control matrix are inputs.
# ---------------------------------------------------------------------------
@dataclass
class Dm:
    n_act: int           # actuators per side of the square grid (centred on the axis)
    pitch_m: float       # actuator pitch in the mirror's conjugate plane
    alt_m: float         # conjugation altitude
    n_modes: int
    coupling: float = 0.15   # influence at one pitch
    support: int = 3         # influence radius in pitches


def elt_dms() -> List[Dm]:
    """The three mirrors of the ELT workload: ground (81 x 81 at the subaperture pitch,
    5000 modes) and post-focal at 4 km (43 x 43, 1 m, 1400 modes) and 12.7 km (50 x 50,
    1 m, 1800 modes), each with n_act pitches covering the meta-pupil of the 160 arcsec field
    at its altitude."""
    return [Dm(81, 39.0 / 80.0, 0.0, 5000), Dm(43, 1.0, 4000.0, 1400), Dm(50, 1.0, 12700.0, 1800)]


def modal_base(dm: Dm, seed: int, amplitude_m: float = 1e-8) -> np.ndarray:
    """[n_act^2, n_modes] float32 synthetic modal base: independent Gaussian actuator
    patterns of rms ``amplitude_m`` per actuator (any base of the mirror's actuator space
    is admissible as an input)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((dm.n_act * dm.n_act, dm.n_modes)) * amplitude_m).astype(np.float32)


def random_control_matrix(n_modes: int, n_slopes: int, seed: int, scale: float = 1e-3) -> np.ndarray:
    """[n_modes, n_slopes] float32 synthetic control matrix (uniform in +-scale / sqrt(n_slopes)),
    a stand-in of the right size where no calibrated one is needed (timing)."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1.0, 1.0, (n_modes, n_slopes)) * (scale / math.sqrt(n_slopes))).astype(np.float32)


# ---------------------------------------------------------------------------
# von Karman phase screens (Sec. 3, atmospheric layers block).
# ---------------------------------------------------------------------------
def von_karman_screen(S: int, dx: float, r0: float, L0: float, rng: np.random.Generator):
    """One periodic S x S phase screen in radians at 500 nm.

    PSD Phi(k) = 0.023 r0^(-5/3) (k^2 + L0^-2)^(-11/6), k in cycles/m; each Fourier
    coefficient is complex Gaussian with variance Phi(k) dk^2 and the real part of the
    transform is kept, so the screen variance is sum(Phi dk^2) (piston removed).
    """
    dk = 1.0 / (S * dx)
    k = np.fft.fftfreq(S, d=dx)
    kx, ky = np.meshgrid(k, k, indexing="xy")
    psd = 0.023 * r0 ** (-5.0 / 3.0) * (kx * kx + ky * ky + L0 ** -2) ** (-11.0 / 6.0)
    psd[0, 0] = 0.0
    c = (rng.standard_normal((S, S)) + 1j * rng.standard_normal((S, S))) * np.sqrt(psd) * dk
    return np.real(np.fft.fft2(c))


def make_screens(layers: Layers, seed: int) -> np.ndarray:
    """[L][S][S] float32 OPD screens (metres), row index = y, column index = x."""
    rng = np.random.default_rng(seed)
    out = np.empty((layers.n_layers, layers.screen_size, layers.screen_size), dtype=np.float32)
    for l in range(layers.n_layers):
        r0_l = layers.r0_m * float(layers.weights[l]) ** (-3.0 / 5.0)
        phase = von_karman_screen(layers.screen_size, layers.screen_dx_m, r0_l, layers.L0_m, rng)
        out[l] = (phase * R0_WAVELENGTH / (2.0 * math.pi)).astype(np.float32)
    return out


def random_expected_image(n_pix: int, seed: int, max_mean: float = 60.0) -> np.ndarray:
    """Synthetic expected-count image for noise-stage tests: a mix of zeros, small means
    (inversion branch) and large means (rejection branch)."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(0.0, 1.0, n_pix) ** 3 * max_mean
    e[rng.uniform(size=n_pix) < 0.05] = 0.0
    return e.astype(np.float32)


CONFIGS = {1: config1, 2: config2, 3: config3}
