"""Pins of the synthetic-input generator (von Karman screens, workload parameters)."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_1408_0698_gb300 import inputs


def _structure_function(screens, lag):
    d = []
    for s in screens:
        d.append(np.mean((s[:, lag:] - s[:, :-lag]) ** 2))
        d.append(np.mean((s[lag:, :] - s[:-lag, :]) ** 2))
    return float(np.mean(d))


def test_von_karman_structure_function():
    """Empirical D(r) of FFT screens against (a) its exact expectation, the discrete PSD sum
    2 sum Phi dk^2 (1 - cos 2 pi k.r), and (b) the continuous von Karman integral
    4 pi int Phi(k) (1 - J0(2 pi k r)) k dk for r well above the pixel and well below L0."""
    S, dx, r0, L0 = 512, 0.05, 0.15, 25.0
    rng = np.random.default_rng(1)
    scr = [inputs.von_karman_screen(S, dx, r0, L0, rng) for _ in range(12)]
    k = np.fft.fftfreq(S, d=dx)
    kx, ky = np.meshgrid(k, k, indexing="xy")
    psd = 0.023 * r0 ** (-5 / 3) * (kx ** 2 + ky ** 2 + L0 ** -2) ** (-11 / 6)
    psd[0, 0] = 0
    dk = 1.0 / (S * dx)
    for lag in (4, 10, 20):
        r = lag * dx
        emp = _structure_function(scr, lag)
        exp_discrete = float(np.sum(psd * dk * dk * (2 - np.cos(2 * np.pi * kx * r) - np.cos(2 * np.pi * ky * r))))
        assert abs(emp / exp_discrete - 1) < 0.06, (lag, emp, exp_discrete)
        f = lambda kk: 0.023 * r0 ** (-5 / 3) * (kk * kk + L0 ** -2) ** (-11 / 6) * (1 - special.j0(2 * np.pi * kk * r)) * kk
        cont = 4 * np.pi * integrate.quad(f, 0, np.inf, limit=400)[0]
        assert abs(emp / cont - 1) < 0.15, (lag, emp, cont)
        # below the Kolmogorov law 6.88 (r/r0)^(5/3): the outer scale removes power
        assert 0.4 < emp / (6.88 * (r / r0) ** (5 / 3)) < 1.0


def test_screens_are_seeded_and_scaled():
    cfg = inputs.config2()
    a = inputs.make_screens(cfg.layers, 7)
    b = inputs.make_screens(cfg.layers, 7)
    c = inputs.make_screens(cfg.layers, 8)
    assert a.dtype == np.float32 and a.shape == (3, 512, 512)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # layer variance scales with the turbulence weight (r0_l = r0 w^-3/5  =>  var ~ w)
    v = a.reshape(3, -1).var(axis=1)
    w = cfg.layers.weights
    ratio = (v / w) / (v / w).mean()
    assert np.all(np.abs(ratio - 1) < 0.5)


def test_config_parameters():
    c3 = inputs.config3()
    assert abs(c3.telescope.diameter_m - 800 * 4.875e-2) < 1e-12
    assert sum(s.is_lgs for s in c3.stars) == 6 and sum(not s.is_lgs for s in c3.stars) == 3
    assert c3.layers.n_layers == 10 and abs(c3.layers.weights.sum() - 1) < 1e-12
    h, w = inputs.sodium_slices(90e3, 10e3, 8)
    assert len(h) == 8 and abs(w.sum() - 1) < 1e-12 and abs(np.sum(w * h) - 90e3) < 1e-6
    assert abs(h[-1] - h[0] - 17.5e3) < 1e-6
    radii = [math.hypot(s.theta_x_rad, s.theta_y_rad) / inputs.ARCSEC for s in c3.stars]
    assert np.allclose(radii[:6], 45.0) and np.allclose(radii[6:], 60.0)
    insts = inputs.config4_instances(64, 4000)
    assert len(insts) == 64
    assert not any(i.stars[0].is_lgs and i.geometries[0].n_sub == 2 for i in insts)
    assert {i.geometries[0].n_fft for i in insts} == {16, 24, 32, 64}


def test_mirror_inputs_of_the_elt_workload():
    """The ELT mirrors: 5000 + 1400 + 1800 = 8200 modes (the paper's M4 count on the ground
    mirror), the ground grid at the 80 x 80 subaperture pitch over 39 m, and each post-focal
    grid wide enough for the 160 arcsec field at its altitude; the modal bases and control
    matrices are seeded, of the stated shapes and amplitudes.  "Wide enough": n_act pitches (the
    actuator span plus half a pitch at each edge) cover the meta-pupil, D + field x altitude."""
    dms = inputs.elt_dms()
    assert [d.n_modes for d in dms] == [5000, 1400, 1800]
    assert sum(d.n_modes for d in dms) == 8200
    g = dms[0]
    assert g.n_act == 81 and g.alt_m == 0.0 and abs(g.pitch_m - 39.0 / 80) < 1e-12
    field = 160.0 / 3600.0 * math.pi / 180.0
    for d in dms[1:]:
        assert d.n_act * d.pitch_m >= 39.0 + field * d.alt_m
        assert d.n_modes <= d.n_act * d.n_act
    M = inputs.modal_base(g, 40, amplitude_m=2e-8)
    assert M.shape == (81 * 81, 5000) and M.dtype == np.float32
    assert abs(float(M.std()) / 2e-8 - 1) < 0.01
    np.testing.assert_array_equal(M, inputs.modal_base(g, 40, amplitude_m=2e-8))
    cm = inputs.random_control_matrix(300, 2000, seed=3, scale=0.5)
    assert cm.shape == (300, 2000) and cm.dtype == np.float32
    assert np.abs(cm).max() <= 0.5 / math.sqrt(2000) * (1 + 1e-6)
    np.testing.assert_array_equal(cm, inputs.random_control_matrix(300, 2000, seed=3, scale=0.5))
