"""LGS per-slice model on the GPU (wfs_set_lgs_model(h, 1)) against the FP64 oracle.

Sec. 4: one wavefront per sodium sub-layer (its own cone and its tip-tilt and defocus), one
DFT per sub-layer, the spots weighted by the sodium profile and piled up, then the Gaussian
extent.  The open-loop bars apply: OPD (the first slice's) <= 5e-6 relative, intensities and
expected images <= 1e-4 relative, slopes <= 1e-3 px RMS (noise off).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1408_0698_gb300 import inputs, native

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from _gpu import run_library, slope_rms  # noqa: E402
from test_parity_gpu import SLOPE_RMS, _check_wfs  # noqa: E402


def _per_slice(cfg, **kw):
    stars = [dataclasses.replace(s, per_slice=True, **kw) if s.is_lgs else s for s in cfg.stars]
    return dataclasses.replace(cfg, stars=stars)


def test_per_slice_config2_full_parity():
    cfg = _per_slice(inputs.config2())
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    gpu, w = run_library(cfg, scr, 0.021)
    _check_wfs(cfg, scr, 0.021, gpu)
    w.close()


def test_per_slice_with_uplink_config2():
    cfg = _per_slice(inputs.config2(), uplink_diameter_m=0.5, uplink_samples=16)
    scr = inputs.make_screens(cfg.layers, cfg.seed + 1)
    gpu, w = run_library(cfg, scr, 0.0)
    _check_wfs(cfg, scr, 0.0, gpu)
    w.close()


@pytest.mark.parametrize("precision", [inputs.PREC_BF16X3, inputs.PREC_FP16S, inputs.PREC_FP32])
def test_per_slice_elt_sampled_full_launch(precision):
    """The ELT frame with the per-slice model on the six LGS (8 slices each) at full size, on
    the self-projecting tensor-core kernel (BF16x3) and on the FP32 32-point kernel: sampled
    subapertures of every star against the oracle."""
    cfg = _per_slice(inputs.config3(precision))
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    t = 0.05
    gpu, w = run_library(cfg, scr, t)
    sel = [np.arange(k, len(d["slopes"]), 97, dtype=np.int32) if cfg.stars[k].is_lgs
           else np.arange(len(d["slopes"]), dtype=np.int32) for k, d in enumerate(gpu)]
    _check_wfs(cfg, scr, t, gpu, sel=sel)
    w.close()


def test_per_slice_toggle_and_limits():
    """Back to the elongation-kernel model bit for bit; batches and calibration refuse the
    per-slice model; the two models stay close on the same frame."""
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    plain, w = run_library(cfg, scr, 0.004, stages=False)
    native.wfs_set_lgs_model(w.h, 1)
    sl, _ = run_library(cfg, scr, 0.004, stages=False, handle=w)
    d = np.concatenate([a["slopes"] - b["slopes"] for a, b in zip(sl[:3], plain[:3])])
    assert 1e-6 < np.sqrt(np.mean(d ** 2)) < 0.05
    np.testing.assert_array_equal(sl[3]["slopes"], plain[3]["slopes"])  # the NGS is untouched
    with pytest.raises(native.WfsError, match="WFS_EUNSUPPORTED"):
        native.wfs_batch_create([w.h])
    assert native.lib().wfs_set_lgs_model(w.h, 2) == native.WFS_EINVAL
    native.wfs_set_lgs_model(w.h, 0)
    back, _ = run_library(cfg, scr, 0.004, stages=False, handle=w)
    for a, b in zip(back, plain):
        np.testing.assert_array_equal(a["slopes"], b["slopes"])
    w.close()


def test_per_slice_closed_loop_step():
    """A closed-loop step with the per-slice model: the mirror layers are seen through each
    slice's cone as well."""
    cfg = _per_slice(inputs.config2())
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    dms = [inputs.Dm(21, 0.4, 0.0, 12), inputs.Dm(15, 0.7, 6000.0, 6)]
    m2a = [inputs.modal_base(d, 3 + i, amplitude_m=2e-8) for i, d in enumerate(dms)]
    n = sum(d.n_modes for d in dms)
    w = native.Wfs(cfg)
    ns = 2 * w.total
    Ms = [torch.as_tensor(M).cuda() for M in m2a]
    cm = inputs.random_control_matrix(n, ns, seed=5, scale=0.5)
    gain = np.full(n, 0.4)
    cm_d, g_d = torch.as_tensor(cm).cuda(), torch.as_tensor(gain.astype(np.float32)).cuda()
    lp = native.wfs_loop_create(w.h, [native.wfs_dm(d.n_act, d.pitch_m, d.alt_m, d.coupling, d.support, d.n_modes,
                                                    M.data_ptr()) for d, M in zip(dms, Ms)],
                                cm_d.data_ptr(), g_d.data_ptr())
    c0 = np.random.default_rng(8).standard_normal(n).astype(np.float32)
    c_d = torch.as_tensor(c0).cuda()
    st = torch.cuda.current_stream().cuda_stream
    native.wfs_loop_set_coeffs(lp, w.h, c_d.data_ptr(), st)
    s = torch.zeros((w.total, 2), device="cuda")
    native.wfs_loop_step(lp, w.h, torch.as_tensor(scr).cuda().data_ptr(), 0.01, s.data_ptr(), st)
    torch.cuda.synchronize()
    s_ref, _ = oracle.loop_step(cfg, scr, 0.01, dms, m2a, cm, gain, c0.astype(np.float64))
    assert slope_rms(s.cpu().numpy(), s_ref) < SLOPE_RMS
    out = torch.zeros((n, 2 * native.wfs_num_valid(w.h, 0)), device="cuda")
    with pytest.raises(native.WfsError, match="WFS_EUNSUPPORTED"):
        native.wfs_loop_calibrate(lp, w.h, 0, 1.0, out.data_ptr(), st)
    w.close()


def test_per_slice_then_uplink_elt():
    """The uplink switched on after the per-slice model (the slice projection copies follow the
    work table): sampled ELT subapertures against the oracle with both."""
    base = _per_slice(inputs.config3())
    both = _per_slice(inputs.config3(), uplink_diameter_m=0.4, uplink_samples=16)
    scr = inputs.make_screens(base.layers, base.seed + 2)
    w = native.Wfs(base)
    for k, s in enumerate(base.stars):
        if s.is_lgs:
            native.wfs_set_uplink(w.h, k, 0.4, 16)
    t = 0.02
    gpu, _ = run_library(both, scr, t, handle=w)
    sel = [np.arange(3 * k, len(d["slopes"]), 211, dtype=np.int32) if both.stars[k].is_lgs
           else np.arange(len(d["slopes"]), dtype=np.int32) for k, d in enumerate(gpu)]
    _check_wfs(both, scr, t, gpu, sel=sel)
    w.close()
