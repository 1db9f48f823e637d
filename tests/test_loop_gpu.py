"""Closed loop on the GPU (wfs_loop_*) against the FP64 oracle.

Sec. 3 "The closed loop": the sensors measure the open-loop wavefront minus the
mirrors; slopes times the control matrix are added (per-mode gain) to the mirrors'
modal coefficients.  Bars: slopes as for the open-loop parity (<= 1e-3 detector-pixel
RMS, noise off); mirror layers <= 1e-5 of their largest magnitude (an FP32 modal sum of
the actuator commands, then <= (2R + 2)^2 FP32 products of influence weights made by
exp2f, against FP64); coefficients within the propagated slope bar,
|dc_m| <= gain_m * sum_k |cm_mk| * 5e-3 px, plus FP32 rounding of the product.
"""
import numpy as np
import pytest

import oracle
from paper_1408_0698_gb300 import inputs, native

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from _gpu import slope_rms  # noqa: E402

SLOPE_RMS = 1e-3
SLOPE_MAX = 5e-3
LAYER_REL = 1e-5


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _small_cfg(is_lgs=False):
    tel = inputs.Telescope(4.0, 0.0)
    geom = [inputs.Geometry(10, 8, 16, 8, 0.5, inputs.PREC_FP32)]
    star = (inputs._lgs(10 * inputs.ARCSEC, -5 * inputs.ARCSEC, 0.3, 0) if is_lgs
            else inputs._ngs(5 * inputs.ARCSEC, 0.0, 700e-9, 0, photons=1000.0))
    lay = inputs.Layers(alt_m=np.array([0.0]), wind_vx_mps=np.zeros(1), wind_vy_mps=np.zeros(1),
                        x0_m=np.zeros(1), y0_m=np.zeros(1), screen_size=128, screen_dx_m=0.05)
    return inputs.Config("loop_small", tel, geom, [star], lay, seed=7)


class _Loop:
    """A handle of cfg with a loop over mirrors dms (modal bases m2a, control matrix cm, gains)."""

    def __init__(self, cfg, dms, m2a, cm, gain, seed=0, noise=False):
        self.w = native.Wfs(cfg, seed=seed, noise=noise)
        self.m2a = [_dev(M) for M in m2a]
        self.cm = _dev(cm)
        self.gain = _dev(gain)
        structs = [native.wfs_dm(d.n_act, d.pitch_m, d.alt_m, d.coupling, d.support, d.n_modes,
                                 M.data_ptr()) for d, M in zip(dms, self.m2a)]
        self.lp = native.wfs_loop_create(self.w.h, structs, self.cm.data_ptr(), self.gain.data_ptr())
        self.n_modes = sum(d.n_modes for d in dms)
        self.S = cfg.layers.screen_size
        self.stream = torch.cuda.current_stream().cuda_stream

    def set_coeffs(self, c):
        ct = _dev(c)
        native.wfs_loop_set_coeffs(self.lp, self.w.h, ct.data_ptr(), self.stream)
        torch.cuda.synchronize()

    def coeffs(self):
        out = torch.zeros(self.n_modes, device="cuda")
        native.wfs_loop_get_coeffs(self.lp, self.w.h, out.data_ptr(), self.stream)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)

    def layer(self, d):
        out = torch.full((self.S, self.S), float("nan"), device="cuda")
        native.wfs_loop_get_layer(self.lp, self.w.h, d, out.data_ptr(), self.stream)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def step(self, screens_dev, t):
        s = torch.full((self.w.total, 2), float("nan"), device="cuda")
        native.wfs_loop_step(self.lp, self.w.h, screens_dev.data_ptr(), t, s.data_ptr(), self.stream)
        torch.cuda.synchronize()
        native.wfs_sync_status(self.w.h)
        return s.cpu().numpy().astype(np.float64)

    def close(self):
        native.wfs_loop_destroy(self.lp)
        self.w.close()


def _coeff_tol(cm, gain, steps):
    row_l1 = np.abs(np.asarray(cm, np.float32)).sum(axis=1, dtype=np.float64)
    return steps * np.abs(gain) * row_l1 * SLOPE_MAX + 1e-30


def test_mirror_layers_match_oracle():
    """Two mirrors (one above the ground) with random modal coefficients: the correction
    layers equal the oracle's, including the zeros outside each mirror's reach."""
    cfg = inputs.config2()
    S, ds = cfg.layers.screen_size, cfg.layers.screen_dx_m
    dms = [inputs.Dm(21, 0.4, 0.0, 30), inputs.Dm(13, 0.8, 8000.0, 12, coupling=0.3, support=2)]
    m2a = [inputs.modal_base(d, 100 + i) for i, d in enumerate(dms)]
    n = sum(d.n_modes for d in dms)
    L = _Loop(cfg, dms, m2a, np.zeros((n, 2 * 4 * 1264)), np.zeros(n))
    c = np.random.default_rng(1).standard_normal(n)
    L.set_coeffs(c)
    for d, (dm, a) in enumerate(zip(dms, oracle.actuators(dms, m2a, c))):
        ref = oracle.dm_layer(dm, a, S, ds)
        got = L.layer(d)
        scale = np.abs(ref).max()
        assert scale > 0
        assert np.abs(got - ref).max() <= LAYER_REL * scale, f"mirror {d}"
        # zero beyond the mirror's reach (R pitches past its outer actuators)
        S2, p, R = S // 2, dm.pitch_m, dm.support
        reach = ((dm.n_act - 1) / 2 + R) * p / ds
        far = np.abs(np.arange(S) - S2) > reach + 1
        assert np.all(got[far, :] == 0) and np.all(got[:, far] == 0)
        assert np.count_nonzero(got[~far][:, ~far]) > 0.5 * (~far).sum() ** 2
    L.close()


@pytest.mark.parametrize("which", ["ngs_small", "config2"])
def test_loop_steps_match_oracle(which):
    """Three integrator steps from random coefficients under frozen-flow turbulence: the
    slopes of each step and the coefficients after it follow the oracle's own chain."""
    if which == "ngs_small":
        cfg = _small_cfg()
        dms = [inputs.Dm(11, 0.4, 0.0, 16)]
    else:
        cfg = inputs.config2()
        dms = [inputs.Dm(21, 0.4, 0.0, 40), inputs.Dm(15, 0.7, 6000.0, 20)]
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    m2a = [inputs.modal_base(d, 7 + i, amplitude_m=2e-8) for i, d in enumerate(dms)]
    n = sum(d.n_modes for d in dms)
    rng = np.random.default_rng(3)
    w = native.Wfs(cfg)
    ns = 2 * w.total
    w.close()
    cm = inputs.random_control_matrix(n, ns, seed=9, scale=0.5)
    gain = rng.uniform(0.2, 0.6, n)
    c = rng.standard_normal(n)
    L = _Loop(cfg, dms, m2a, cm, gain)
    L.set_coeffs(c)
    scr_d = _dev(scr)
    c_ref = c.astype(np.float32).astype(np.float64)
    for k in range(3):
        t = 0.002 * k
        s_gpu = L.step(scr_d, t)
        s_ref, c_ref = oracle.loop_step(cfg, scr, t, dms, m2a, cm, gain, c_ref)
        assert slope_rms(s_gpu, s_ref) < SLOPE_RMS, f"step {k} slopes"
        assert np.abs(s_gpu - s_ref).max() < SLOPE_MAX, f"step {k} slopes (max)"
        c_gpu = L.coeffs()
        tol = _coeff_tol(cm, gain, k + 1) + 1e-5 * np.abs(c_ref)
        assert np.all(np.abs(c_gpu - c_ref) <= tol), f"step {k} coefficients"
    L.close()


def test_loop_corrects_static_modal_aberration():
    """Unit gains, CM = pinv(IM) with IM registered by push-pull in the oracle: one GPU step
    brings the coefficients to the aberration's and the next slopes near zero."""
    cfg = _small_cfg()
    S, ds = cfg.layers.screen_size, cfg.layers.screen_dx_m
    dm = inputs.Dm(11, 0.4, 0.0, 8)
    M = inputs.modal_base(dm, 11).astype(np.float64)
    IM = []
    for m in range(dm.n_modes):
        beam = -oracle.dm_layer(dm, M[:, m] * 0.5, S, ds)
        IM.append((oracle.measure(cfg, beam[None], 0.0) - oracle.measure(cfg, -beam[None], 0.0)).ravel())
    CM = np.linalg.pinv(np.array(IM).T)
    c_star = np.random.default_rng(2).standard_normal(dm.n_modes)
    ol = -oracle.dm_layer(dm, M @ c_star, S, ds)[None]
    L = _Loop(cfg, [dm], [M], CM, np.ones(dm.n_modes))
    ol_d = _dev(ol)
    s0 = L.step(ol_d, 0.0)
    c1 = L.coeffs()
    assert np.linalg.norm(c1 - c_star) < 0.05 * np.linalg.norm(c_star)
    s1 = L.step(ol_d, 0.0)
    assert np.linalg.norm(s1) < 0.05 * np.linalg.norm(s0)
    L.close()


def test_loop_busy_and_arguments():
    cfg = _small_cfg()
    dm = inputs.Dm(11, 0.4, 0.0, 4)
    M = _dev(inputs.modal_base(dm, 1))
    w = native.Wfs(cfg)
    cm = torch.zeros((4, 2 * w.total), device="cuda")
    g = torch.zeros(4, device="cuda")
    good = native.wfs_dm(11, 0.4, 0.0, 0.15, 3, 4, M.data_ptr())
    bad = [native.wfs_dm(0, 0.4, 0.0, 0.15, 3, 4, M.data_ptr()),
           native.wfs_dm(11, -1.0, 0.0, 0.15, 3, 4, M.data_ptr()),
           native.wfs_dm(11, 0.4, 0.0, 1.0, 3, 4, M.data_ptr()),
           native.wfs_dm(11, 0.4, 0.0, 0.15, 9, 4, M.data_ptr()),
           native.wfs_dm(11, 0.4, 0.0, 0.15, 3, 0, M.data_ptr()),
           native.wfs_dm(11, 0.4, 0.0, 0.15, 3, 4, None)]
    for b in bad:
        with pytest.raises(native.WfsError, match="WFS_EINVAL"):
            native.wfs_loop_create(w.h, [b], cm.data_ptr(), g.data_ptr())
    lp = native.wfs_loop_create(w.h, [good], cm.data_ptr(), g.data_ptr())
    with pytest.raises(native.WfsError, match="WFS_EBUSY"):
        native.wfs_loop_create(w.h, [good], cm.data_ptr(), g.data_ptr())
    out = torch.zeros((128, 128), device="cuda")
    with pytest.raises(native.WfsError, match="WFS_EINVAL"):
        native.wfs_loop_get_layer(lp, w.h, 1, out.data_ptr())
    # one stream at a time: a step queued behind a busy wait on s1 makes s2 wait its turn
    scr = _dev(np.zeros((1, 128, 128)))
    s = torch.zeros((w.total, 2), device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s1):
        torch.cuda._sleep(200_000_000)
        native.wfs_loop_step(lp, w.h, scr.data_ptr(), 0.0, s.data_ptr(), s1.cuda_stream)
    with pytest.raises(native.WfsError, match="WFS_EBUSY"):
        native.wfs_loop_step(lp, w.h, scr.data_ptr(), 0.0, s.data_ptr(), s2.cuda_stream)
    torch.cuda.synchronize()
    native.wfs_loop_destroy(lp)
    # the handle keeps measuring open loop and takes a new loop
    lp = native.wfs_loop_create(w.h, [good], cm.data_ptr(), g.data_ptr())
    w.close()  # destroys the attached loop too


def test_elt_loop_step_full_size():
    """The ELT frame (6 LGS BF16x3 + 3 NGS, 10 layers) with the three mirrors (5000 + 1400 +
    1800 modes) at full size, in the benchmark's launch configuration: one step from random
    coefficients; all slopes and all coefficients against the oracle."""
    cfg = inputs.config3()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    dms = inputs.elt_dms()
    m2a = [inputs.modal_base(d, 30 + i) for i, d in enumerate(dms)]
    n = sum(d.n_modes for d in dms)
    w = native.Wfs(cfg)
    ns = 2 * w.total
    w.close()
    cm = inputs.random_control_matrix(n, ns, seed=31)
    rng = np.random.default_rng(32)
    gain = rng.uniform(0.2, 0.6, n)
    c0 = rng.standard_normal(n)
    L = _Loop(cfg, dms, m2a, cm, gain)
    L.set_coeffs(c0)
    t = 0.137
    s_gpu = L.step(_dev(scr), t)
    c_gpu = L.coeffs()
    s_ref, c_ref = oracle.loop_step(cfg, scr, t, dms, m2a, cm, gain, c0.astype(np.float32).astype(np.float64))
    assert slope_rms(s_gpu, s_ref) < SLOPE_RMS
    assert np.abs(s_gpu - s_ref).max() < SLOPE_MAX
    tol = _coeff_tol(cm, gain, 1) + 1e-5 * np.abs(c_ref)
    assert np.all(np.abs(c_gpu - c_ref) <= tol)
    L.close()


def _calibrate(L, gs, amp, nv):
    im = torch.full((L.n_modes, 2 * nv), float("nan"), device="cuda")
    native.wfs_loop_calibrate(L.lp, L.w.h, gs, amp, im.data_ptr(), L.stream)
    torch.cuda.synchronize()
    native.wfs_sync_status(L.w.h)
    return im.cpu().numpy().astype(np.float64)


def _check_im(im_gpu, im_ref, amp):
    """Rows are slope differences over 2a: the slope bars apply to the rows times 2a."""
    d = (im_gpu - im_ref) * 2 * abs(amp)
    assert np.all(np.sqrt(np.mean(d ** 2, axis=1)) < SLOPE_RMS)
    assert np.abs(d).max() < SLOPE_MAX


@pytest.mark.parametrize("which", ["ngs_small", "config2"])
def test_calibration_matches_oracle(which):
    """Push-pull interaction matrices of every guide star over all modes (two mirrors on
    config 2, one above the ground; modes not a multiple of the 32-mode chunk) against the
    oracle's."""
    if which == "ngs_small":
        cfg, dms = _small_cfg(), [inputs.Dm(11, 0.4, 0.0, 40)]
    else:
        cfg, dms = inputs.config2(), [inputs.Dm(21, 0.4, 0.0, 37), inputs.Dm(15, 0.7, 6000.0, 9)]
    m2a = [inputs.modal_base(d, 21 + i, amplitude_m=2e-8) for i, d in enumerate(dms)]
    n = sum(d.n_modes for d in dms)
    L = _Loop(cfg, dms, m2a, np.zeros((n, 2)), np.zeros(n))
    c = np.random.default_rng(0).standard_normal(n)
    L.set_coeffs(c)
    before = [L.layer(d) for d in range(len(dms))]
    amp = 0.5
    for gs in range(len(cfg.stars)):
        nv = native.wfs_num_valid(L.w.h, gs)
        im = _calibrate(L, gs, amp, nv)
        ref = oracle.interaction_matrix(cfg, gs, dms, m2a, amp)
        _check_im(im, ref, amp)
    # the loop's own state is untouched
    np.testing.assert_array_equal(L.coeffs(), c.astype(np.float32))
    for d in range(len(dms)):
        np.testing.assert_array_equal(L.layer(d), before[d])
    L.close()


@pytest.mark.parametrize("precision", [inputs.PREC_BF16X3, inputs.PREC_FP16S])
def test_calibration_elt_m4_full_size(precision):
    """The paper's calibration workload: the 5000 modes of the 81 x 81 ground mirror with one
    80 x 80 LGS of the ELT frame (tensor-core spots, BF16x3 or scaled FP16x3), all modes on the
    GPU; sampled modes from every chunk position against the oracle."""
    cfg = inputs.config3(precision)
    dm = inputs.elt_dms()[0]
    M = inputs.modal_base(dm, 40)
    L = _Loop(cfg, [dm], [M], np.zeros((dm.n_modes, 2)), np.zeros(dm.n_modes))
    nv = native.wfs_num_valid(L.w.h, 0)
    amp = 1.0
    im = _calibrate(L, 0, amp, nv)
    assert np.all(np.isfinite(im))
    pick = [0, 31, 32, 2500, 4999]
    ref = oracle.interaction_matrix(cfg, 0, [dm], [M.astype(np.float64)], amp, modes=pick)
    _check_im(im[pick], ref, amp)
    L.close()


def test_loop_batch_equals_separate_steps():
    """Five loops of one system (own handles, screens, seeds and coefficients) stepped as a
    batch give, bit for bit, the slopes, coefficients and mirror layers of separate steps (the
    shared reconstruction launch keeps each loop's summation order; four plus one loops)."""
    cfg = inputs.config2()
    dms = [inputs.Dm(21, 0.4, 0.0, 14), inputs.Dm(15, 0.7, 6000.0, 6)]
    m2a = [_dev(inputs.modal_base(d, 60 + i, amplitude_m=2e-8)) for i, d in enumerate(dms)]
    n = sum(d.n_modes for d in dms)
    w = native.Wfs(cfg)
    ns = 2 * w.total
    w.close()
    cm = _dev(inputs.random_control_matrix(n, ns, seed=61, scale=0.5))
    gains = [_dev(np.random.default_rng(70 + i).uniform(0.2, 0.6, n)) for i in range(5)]
    structs = [native.wfs_dm(d.n_act, d.pitch_m, d.alt_m, d.coupling, d.support, d.n_modes, M.data_ptr())
               for d, M in zip(dms, m2a)]
    st = torch.cuda.current_stream().cuda_stream
    scr = [_dev(inputs.make_screens(cfg.layers, 100 + i)) for i in range(5)]
    c0 = [_dev(np.random.default_rng(80 + i).standard_normal(n)) for i in range(5)]

    def make():
        hs, lps = [], []
        for i in range(5):
            h = native.Wfs(cfg, seed=90 + i, noise=True)
            lp = native.wfs_loop_create(h.h, structs, cm.data_ptr(), gains[i].data_ptr())
            native.wfs_loop_set_coeffs(lp, h.h, c0[i].data_ptr(), st)
            hs.append(h)
            lps.append(lp)
        return hs, lps

    ha, la = make()
    hb, lb = make()
    b = native.wfs_loop_batch_create(lb)
    sa = [torch.zeros((ns // 2, 2), device="cuda") for _ in range(5)]
    sb = [torch.zeros((ns // 2, 2), device="cuda") for _ in range(5)]
    for k in range(3):
        ts = [0.003 * k + 0.001 * i for i in range(5)]
        for i in range(5):
            native.wfs_loop_step(la[i], ha[i].h, scr[i].data_ptr(), ts[i], sa[i].data_ptr(), st)
        native.wfs_loop_batch_step(b, [x.data_ptr() for x in scr], ts, [x.data_ptr() for x in sb], st)
        torch.cuda.synchronize()
        for i in range(5):
            assert torch.equal(sa[i], sb[i]), f"step {k} loop {i} slopes"
    ca, cb = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    la_, lb_ = torch.zeros((512, 512), device="cuda"), torch.zeros((512, 512), device="cuda")
    for i in range(5):
        native.wfs_loop_get_coeffs(la[i], ha[i].h, ca.data_ptr(), st)
        native.wfs_loop_get_coeffs(lb[i], hb[i].h, cb.data_ptr(), st)
        torch.cuda.synchronize()
        assert torch.equal(ca, cb), f"loop {i} coefficients"
        for d in range(2):
            native.wfs_loop_get_layer(la[i], ha[i].h, d, la_.data_ptr(), st)
            native.wfs_loop_get_layer(lb[i], hb[i].h, d, lb_.data_ptr(), st)
            torch.cuda.synchronize()
            assert torch.equal(la_, lb_), f"loop {i} mirror {d}"
    # a loop with another control matrix does not join the batch
    other = torch.zeros_like(cm)
    h = native.Wfs(cfg)
    lo = native.wfs_loop_create(h.h, structs, other.data_ptr(), gains[0].data_ptr())
    with pytest.raises(native.WfsError, match="WFS_EINVAL"):
        native.wfs_loop_batch_create([lb[0], lo])
    native.wfs_loop_batch_destroy(b)
    for x in ha + hb + [h]:
        x.close()


def test_loop_step_with_uplink():
    """A loop step of LGS with the uplink tip-tilt on: the launch beam crosses the turbulent
    layers only, not the mirrors' correction layers (the oracle marks them as mirror layers)."""
    import dataclasses
    cfg = inputs.config2()
    cfg = dataclasses.replace(cfg, stars=[dataclasses.replace(s, uplink_diameter_m=0.5, uplink_samples=16)
                                          if s.is_lgs else s for s in cfg.stars])
    scr = inputs.make_screens(cfg.layers, cfg.seed + 3)
    dms = [inputs.Dm(21, 0.4, 0.0, 10), inputs.Dm(15, 0.7, 6000.0, 5)]
    m2a = [inputs.modal_base(d, 40 + i, amplitude_m=3e-8) for i, d in enumerate(dms)]
    n = sum(d.n_modes for d in dms)
    w = native.Wfs(cfg)
    ns = 2 * w.total
    w.close()
    cm = inputs.random_control_matrix(n, ns, seed=41, scale=0.5)
    gain = np.full(n, 0.5)
    c = np.random.default_rng(42).standard_normal(n)
    L = _Loop(cfg, dms, m2a, cm, gain)
    L.set_coeffs(c)
    s_gpu = L.step(_dev(scr), 0.004)
    s_ref, c_ref = oracle.loop_step(cfg, scr, 0.004, dms, m2a, cm, gain, c.astype(np.float32).astype(np.float64))
    assert slope_rms(s_gpu, s_ref) < SLOPE_RMS
    assert np.abs(s_gpu - s_ref).max() < SLOPE_MAX
    assert np.all(np.abs(L.coeffs() - c_ref) <= _coeff_tol(cm, gain, 1) + 1e-5 * np.abs(c_ref))
    L.close()
