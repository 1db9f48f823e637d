"""LGS uplink tip-tilt on the GPU (wfs_set_uplink) against the FP64 oracle.

Sec. 4 "Open Loop generation": the laser's projection on the sodium layer is shifted by the
tip-tilt integrated over the upward path.  The oracle adds the tilt to the pupil OPD, so the
open-loop bars apply unchanged: OPD <= 5e-6 relative per subaperture, intensities and expected
images <= 1e-4 relative, slopes <= 1e-3 px RMS (noise off).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1408_0698_gb300 import inputs, native

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from _gpu import run_library  # noqa: E402
from test_parity_gpu import _check_wfs  # noqa: E402


def _with_uplink(cfg, diameter=0.5, samples=16):
    stars = [dataclasses.replace(s, uplink_diameter_m=diameter, uplink_samples=samples) if s.is_lgs else s
             for s in cfg.stars]
    return dataclasses.replace(cfg, stars=stars)


def test_uplink_config2_full_parity():
    cfg = _with_uplink(inputs.config2())
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    for k in range(3):
        dx, dy = oracle.uplink_tilt(cfg, scr, k, 0.013)
        assert abs(dx) + abs(dy) > 1e-8
    gpu, w = run_library(cfg, scr, 0.013)
    _check_wfs(cfg, scr, 0.013, gpu)
    w.close()


def test_uplink_elt_sampled_full_launch():
    """The ELT frame (BF16x3) with the uplink on for the six LGS at full size: sampled
    subapertures against the oracle."""
    cfg = _with_uplink(inputs.config3(), diameter=0.4, samples=24)
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    t = 0.211
    gpu, w = run_library(cfg, scr, t)
    sel = [np.arange(k, len(d["slopes"]), 37, dtype=np.int32) if cfg.stars[k].is_lgs
           else np.arange(len(d["slopes"]), dtype=np.int32) for k, d in enumerate(gpu)]
    _check_wfs(cfg, scr, t, gpu, sel=sel)
    w.close()


def test_uplink_toggle_and_arguments():
    """Turning the uplink off restores the plain measurement bit for bit; NGS and bad
    arguments are rejected; a handle with the uplink on is not batched."""
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    plain, w = run_library(cfg, scr, 0.004, stages=False)
    native.wfs_set_uplink(w.h, 1, 0.5, 16)
    on, _ = run_library(cfg, scr, 0.004, stages=False, handle=w)
    assert np.abs(on[1]["slopes"] - plain[1]["slopes"]).max() > 1e-3
    np.testing.assert_array_equal(on[0]["slopes"], plain[0]["slopes"])
    with pytest.raises(native.WfsError, match="WFS_EUNSUPPORTED"):
        native.wfs_batch_create([w.h])
    native.wfs_set_uplink(w.h, 1, 0.0)
    off, _ = run_library(cfg, scr, 0.004, stages=False, handle=w)
    for a, b in zip(off, plain):
        np.testing.assert_array_equal(a["slopes"], b["slopes"])
    for args in [(3, 0.5, 16), (1, 0.5, 1), (1, 0.5, 65), (1, -1.0, 16), (7, 0.5, 16), (1, 1e3, 16)]:
        with pytest.raises(native.WfsError, match="WFS_EINVAL"):
            native.wfs_set_uplink(w.h, *args)
    w.close()
