"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Bars: noise-free slopes <= 1e-3 detector-pixel RMS; spot intensities and expected
detector images <= 1e-4 relative (||a - b||_2 / ||b||_2 per subaperture, max over
subaperture); projected OPD <= 5e-6 relative per subaperture (an FP32 sum of up to 10
bilinear layer samples: (L + 3) 2^-24 times a layer-cancellation factor of a few) plus an
absolute floor of (L + 3) 2^-24 times the WFS's largest OPD (a subaperture whose OPD crosses
zero while the summands, e.g. an uplink tilt across the pupil, stay large); valid-subaperture
maps and integer Poisson draws bit-exact (draws up to FP32-vs-FP64 rounding of the
mean).
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1408_0698_gb300 import inputs, native

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from _gpu import rel_per_subap, run_library, slope_rms  # noqa: E402

SLOPE_RMS = 1e-3
INT_REL = 1e-4
OPD_REL = 5e-6


def _check_wfs(cfg, scr, t, gpu, sel=None, noise=False, seed=0):
    for w, d in enumerate(gpu):
        sel_w = sel[w] if sel is not None else None
        ref = oracle.measure_wfs(cfg, scr, w, t, seed=seed, noise=noise, sel=sel_w, stages=True)
        pick = (lambda a: a[sel_w]) if sel_w is not None else (lambda a: a)
        # FP32 sum of the layer samples (and the uplink tilt): per subaperture relative to its
        # OPD, with the absolute floor (L + 3) 2^-24 of the WFS's largest OPD where the
        # subaperture's OPD crosses zero while the summands stay large
        a_opd, r_opd = pick(d["opd"]).astype(np.float64), ref["opd"]
        nb = len(r_opd)
        err = np.sqrt(np.mean(((a_opd - r_opd).reshape(nb, -1)) ** 2, axis=1))
        mag = np.sqrt(np.mean((r_opd.reshape(nb, -1)) ** 2, axis=1))
        floor = (cfg.layers.n_layers + 3) * 2.0 ** -24 * np.abs(r_opd).max()
        assert np.all(err <= OPD_REL * mag + floor), f"wfs {w} opd"
        assert rel_per_subap(pick(d["I"]), ref["I"]) < INT_REL, f"wfs {w} intensity"
        assert rel_per_subap(pick(d["E"]), ref["E"]) < INT_REL, f"wfs {w} expected image"
        if not noise:
            assert slope_rms(pick(d["slopes"]), ref["slopes"]) < SLOPE_RMS, f"wfs {w} slopes"
            assert np.max(np.abs(pick(d["slopes"]) - ref["slopes"])) < 5 * SLOPE_RMS
        # photometry closed form: sum E = photons * fill
        g = cfg.geometries[cfg.stars[w].geometry_index]
        tot = pick(d["E"]).reshape(len(ref["E"]), -1).sum(axis=1)
        assert np.allclose(tot, ref["E"].reshape(len(ref["E"]), -1).sum(axis=1), rtol=1e-5)


def test_valid_maps_bit_exact():
    for cfg in (inputs.config1(), inputs.config2(), inputs.config3(inputs.PREC_FP32)):
        w = native.Wfs(cfg)
        for k, s in enumerate(cfg.stars):
            g = cfg.geometries[s.geometry_index]
            idx, _ = oracle.valid_subaps(cfg.telescope.diameter_m, cfg.telescope.obstruction,
                                         g.n_sub, g.n_pix_sub, g.valid_fill)
            assert np.array_equal(native.wfs_valid_map(w.h, k), idx)
        w.close()


def test_config1_full_parity():
    cfg = inputs.config1()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    for t in (0.0, 0.003, 0.009):
        gpu, w = run_library(cfg, scr, t)
        _check_wfs(cfg, scr, t, gpu)
        w.close()


def test_config2_full_parity():
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    gpu, w = run_library(cfg, scr, 0.05)
    _check_wfs(cfg, scr, 0.05, gpu)
    w.close()


def test_config3_sampled_parity_full_launch():
    """The ELT frame at full size in the benchmark's launch configuration; sampled
    subapertures (every 29th LGS subaperture, all NGS) checked against the oracle."""
    cfg = inputs.config3(inputs.PREC_FP32)
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    t = 0.137
    gpu, w = run_library(cfg, scr, t)
    sel = []
    for k, d in enumerate(gpu):
        nv = len(d["slopes"])
        sel.append(np.arange(k, nv, 29, dtype=np.int32) if cfg.stars[k].is_lgs else np.arange(nv, dtype=np.int32))
    _check_wfs(cfg, scr, t, gpu, sel=sel)
    # every subaperture's expected image sums to photons * fill (property at any size)
    for k, d in enumerate(gpu):
        g = cfg.geometries[cfg.stars[k].geometry_index]
        _, fill = oracle.valid_subaps(cfg.telescope.diameter_m, cfg.telescope.obstruction, g.n_sub, g.n_pix_sub)
        assert np.allclose(d["E"].reshape(len(fill), -1).sum(axis=1), cfg.stars[k].photons_per_subap * fill, rtol=2e-5)
        assert np.all(np.isfinite(d["slopes"]))
    w.close()


def test_noise_stage_bit_exact_poisson():
    E = inputs.random_expected_image(1 << 18, 11, max_mean=80.0)
    dev = torch.device("cuda:0")
    e_d = torch.as_tensor(E).to(dev)
    c_d = torch.empty_like(e_d)
    native.wfs_noise_apply(e_d.data_ptr(), E.size, 0.0, 1234, 5, 0.25, 77, c_d.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    C_gpu = c_d.cpu().numpy()
    C_orc, K = oracle.noise_image(E, 0.0, 1234, 5, 0.25, 77)
    assert np.all(C_gpu == np.round(C_gpu))
    match = np.mean(C_gpu == K)
    assert match >= 0.9999, match
    assert np.all(np.abs(C_gpu - K)[C_gpu != K] <= 1)
    # read noise only: Gaussian values agree to FP32 rounding
    Z = np.zeros(1 << 16, np.float32)
    z_d = torch.as_tensor(Z).to(dev)
    native.wfs_noise_apply(z_d.data_ptr(), Z.size, 3.0, 99, 1, 1.5, 0, c_d.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    Cz, _ = oracle.noise_image(Z, 3.0, 99, 1, 1.5, 0)
    assert np.max(np.abs(c_d.cpu().numpy()[:Z.size] - Cz)) < 1e-4


def test_noisy_frame_matches_oracle():
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    t = 0.02
    gpu, w = run_library(cfg, scr, t, seed=42, noise=True)
    for k in (0, 3):
        ref = oracle.measure_wfs(cfg, scr, k, t, seed=42, noise=True, stages=True)
        same = np.abs(gpu[k]["C"] - ref["C"]) < 1e-3
        assert same.mean() >= 0.999, same.mean()
        ok = np.all(same.reshape(len(same), -1), axis=1)
        assert slope_rms(gpu[k]["slopes"][ok], ref["slopes"][ok]) < SLOPE_RMS
    w.close()


def test_noise_statistics_on_gpu():
    """Counts over many frames of a frozen screen: per-pixel mean E and variance
    E + ron^2 (P10)."""
    cfg = inputs.config1()
    cfg.stars[0].read_noise_e = 2.0
    cfg.layers = dataclasses.replace(cfg.layers, wind_vx_mps=np.zeros(1), wind_vy_mps=np.zeros(1))
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    w = native.Wfs(cfg, seed=7, noise=True)
    dev = torch.device("cuda:0")
    s_d = torch.as_tensor(scr).to(dev)
    nd = cfg.geometries[0].n_det
    slopes = torch.empty((w.total, 2), device=dev)
    E = torch.empty(w.total * nd * nd, device=dev)
    C = torch.empty(w.total * nd * nd, device=dev)
    acc1 = torch.zeros_like(C, dtype=torch.float64)
    acc2 = torch.zeros_like(C, dtype=torch.float64)
    reps = 400
    for r in range(reps):
        native.wfs_measure_stages(w.h, s_d.data_ptr(), 1e-3 * r, slopes.data_ptr(), 0, 0, E.data_ptr(),
                                  C.data_ptr(), torch.cuda.current_stream().cuda_stream)
        acc1 += C.double()
        acc2 += C.double() ** 2
    torch.cuda.synchronize()
    m = (acc1 / reps).cpu().numpy()
    v = (acc2 / reps).cpu().numpy() - m ** 2
    e = E.cpu().numpy().astype(np.float64)
    z_mean = (m - e) / np.sqrt((e + 4.0) / reps)
    assert abs(z_mean.mean()) < 0.05 and 0.9 < z_mean.std() < 1.1
    big = e > 5
    ratio = v[big] / (e[big] + 4.0)
    assert abs(np.mean(ratio) - 1) < 0.02
    w.close()


def test_long_run_offsets_fp64():
    """Frozen-flow offsets are formed in FP64: OPD at t = 2 s and at t = 1e4 s match the
    FP64 oracle (an FP32 offset would be off by ~1e-3 px after 1e4 s at 10 m/s)."""
    cfg = inputs.config1()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    for t in (2.0, 1.0e4 + 0.0123):
        gpu, w = run_library(cfg, scr, t)
        ref = oracle.measure_wfs(cfg, scr, 0, t, stages=True)
        assert rel_per_subap(gpu[0]["opd"], ref["opd"]) < OPD_REL
        w.close()


def test_deterministic_and_time_dependent():
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    a, w = run_library(cfg, scr, 0.01, seed=3, noise=True, stages=False)
    b, _ = run_library(cfg, scr, 0.01, seed=3, noise=True, stages=False, handle=w)
    c, _ = run_library(cfg, scr, 0.011, seed=3, noise=True, stages=False, handle=w)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x["slopes"], y["slopes"])
        assert not np.array_equal(x["slopes"], z["slopes"])
    w.close()


def _small_cfg(n_sub, n, N, nd, lgs, eps=0.0, fill=0.5, photons=500.0, D=4.0):
    dx = D / (n_sub * n)
    S = 1 << int(math.ceil(math.log2(1.5 * n_sub * n + 16)))
    lay = inputs._layers([0.0, 3e3], [0.7, 0.3], 0.1, 20.0, S, dx)
    if lgs:
        star = inputs._lgs(10 * inputs.ARCSEC, -5 * inputs.ARCSEC, 0.7, 0, photons=photons)
        # keep the sodium slices' shifts small enough to stay inside small grids
        star.spot_fwhm_rad = 1.5 * 589e-9 / (N * dx)
    else:
        star = inputs._ngs(3 * inputs.ARCSEC, 0.0, 700e-9, 0, photons=photons)
    return inputs.Config("small", inputs.Telescope(D, eps), [inputs.Geometry(n_sub, n, N, nd, fill)],
                         [star], lay, seed=9)


@pytest.mark.parametrize("n_sub,n,N,nd,lgs", [
    (7, 5, 12, 4, True),     # ragged: odd n, N not a power of two
    (9, 3, 6, 3, False),     # tiny subapertures, odd detector
    (5, 1, 2, 1, False),     # one pupil pixel per subaperture, one detector pixel
    (2, 32, 64, 32, True),   # largest LGS geometry (multi-warp teams)
    (3, 32, 64, 16, False),  # largest NGS geometry, b = 4
    (33, 4, 8, 2, True),     # more subapertures than one CTA covers, ragged tail
])
def test_edge_geometries(n_sub, n, N, nd, lgs):
    cfg = _small_cfg(n_sub, n, N, nd, lgs)
    scr = inputs.make_screens(cfg.layers, 5)
    gpu, w = run_library(cfg, scr, 0.004)
    _check_wfs(cfg, scr, 0.004, gpu)
    w.close()


def _coarse_cfg():
    """An LGS 8x8 of 10x10-pixel subapertures (the 32-point FP32 kernel, fed by the projection
    launch) on screens of half its pupil pitch: no shared-memory tiles, direct gathers."""
    n_sub, n, D = 8, 10, 4.0
    dx = D / (n_sub * n)
    S = 1 << int(math.ceil(math.log2(3.0 * n_sub * n + 16)))
    lay = inputs._layers([0.0, 3e3], [0.7, 0.3], 0.1, 20.0, S, dx / 2)
    star = inputs._lgs(10 * inputs.ARCSEC, -5 * inputs.ARCSEC, 0.7, 0, photons=500.0)
    star.spot_fwhm_rad = 1.5 * 589e-9 / (32 * dx)
    return inputs.Config("coarse", inputs.Telescope(D, 0.0), [inputs.Geometry(n_sub, n, 32, 16, 0.5)], [star],
                         lay, seed=9)


@pytest.mark.parametrize("case", ["elt", "elt_per_slice", "coarse"])
def test_projection_forms_agree_bit_for_bit(case):
    """The bulk-copy projection (16-byte-aligned device screens) and the cp.async form (the same
    screens one float off that alignment) give the same OPD, expected images and slopes bit for
    bit: the ELT frame with the uplink on at times whose LGS boxes cross the periodic screen's
    edges (and the per-slice model), and a coarsely sampled WFS whose blocks are direct gathers
    inside the bulk kernel's pipeline."""
    import dataclasses
    if case == "coarse":
        cfg = _coarse_cfg()
    else:
        cfg = inputs.config3()
        cfg = dataclasses.replace(cfg, stars=[dataclasses.replace(st, uplink_diameter_m=0.4, uplink_samples=16)
                                              if st.is_lgs else st for st in cfg.stars])
    w = native.Wfs(cfg, seed=4, noise=True)
    if case == "elt_per_slice":
        native.wfs_set_lgs_model(w.h, True)
    dev = torch.device("cuda:0")
    scr = torch.as_tensor(inputs.make_screens(cfg.layers, 77)).to(dev).reshape(-1)
    shifted = torch.empty(scr.numel() + 4, device=dev)
    shifted[1:1 + scr.numel()].copy_(scr)
    ptrs = {"bulk": scr.data_ptr(), "cp.async": shifted.data_ptr() + 4}
    assert ptrs["bulk"] % 16 == 0 and ptrs["cp.async"] % 16 != 0
    n_opd = max(sum(L.n_valid * L.n * L.n for L in w.layouts), 1)
    n_int = max(sum(L.n_valid * L.n_fft * L.n_fft for L in w.layouts), 1)
    n_det = max(sum(L.n_valid * L.n_det * L.n_det for L in w.layouts), 1)
    stream = torch.cuda.current_stream().cuda_stream
    for t in (0.0, 2.7, 6.1, 1.0e4 + 0.37):
        res = {}
        for form, ptr in ptrs.items():
            out = [torch.full(sz, float("nan"), device=dev) for sz in ((w.total, 2), (n_opd,), (n_int,), (n_det,), (n_det,))]
            native.wfs_measure_stages(w.h, ptr, t, *[x.data_ptr() for x in out], stream)
            torch.cuda.synchronize()
            native.wfs_sync_status(w.h)
            res[form] = [out[0].cpu().numpy(), out[1].cpu().numpy(), out[3].cpu().numpy()]
        for name, a, b in zip(("slopes", "OPD", "E"), res["bulk"], res["cp.async"]):
            assert np.all(np.isfinite(a)), f"{case} t={t}: {name}"
            assert np.array_equal(a, b), f"{case} t={t}: {name}"
    w.close()


def test_zero_photons_and_no_valid_subaps():
    cfg = _small_cfg(6, 6, 12, 6, False, photons=0.0)
    scr = inputs.make_screens(cfg.layers, 1)
    gpu, w = run_library(cfg, scr, 0.0)
    assert np.all(gpu[0]["slopes"] == 0) and np.all(gpu[0]["E"] == 0)
    w.close()
    cfg = _small_cfg(2, 8, 16, 8, False, eps=0.95, fill=0.99)
    w = native.Wfs(cfg)
    assert w.total == 0
    dev = torch.device("cuda:0")
    s_d = torch.as_tensor(inputs.make_screens(cfg.layers, 1)).to(dev)
    out = torch.empty(1, device=dev)
    native.wfs_measure(w.h, s_d.data_ptr(), 0.0, out.data_ptr(), 0)
    native.wfs_sync_status(w.h)
    w.close()


def test_flat_screen_zero_slopes_ngs():
    cfg = inputs.config1()
    S = cfg.layers.screen_size
    gpu, w = run_library(cfg, np.zeros((1, S, S), np.float32), 0.0)
    assert np.max(np.abs(gpu[0]["slopes"])) < 1e-5
    w.close()


def test_host_buffer_path_and_batch_match_device_path():
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    ref, w = run_library(cfg, scr, 0.03, stages=False)
    ref_s = np.concatenate([d["slopes"] for d in ref])
    host_scr = torch.as_tensor(scr).pin_memory()
    host_out = torch.empty((w.total, 2)).pin_memory()
    native.wfs_measure_host(w.h, host_scr.data_ptr(), 0.03, host_out.data_ptr(), 0)
    torch.cuda.synchronize()
    assert np.array_equal(host_out.numpy(), ref_s)
    cfg1 = inputs.config1()
    scr1 = inputs.make_screens(cfg1.layers, cfg1.seed)
    w1 = native.Wfs(cfg1)
    b = native.wfs_batch_create([w.h, w1.h])
    dev = torch.device("cuda:0")
    s0, s1 = torch.as_tensor(scr).to(dev), torch.as_tensor(scr1).to(dev)
    o0, o1 = torch.empty((w.total, 2), device=dev), torch.empty((w1.total, 2), device=dev)
    native.wfs_batch_measure(b, [s0.data_ptr(), s1.data_ptr()], [0.03, 0.002], [o0.data_ptr(), o1.data_ptr()], 0)
    torch.cuda.synchronize()
    assert np.array_equal(o0.cpu().numpy(), ref_s)
    r1, _ = run_library(cfg1, scr1, 0.002, stages=False, handle=w1)
    assert np.array_equal(o1.cpu().numpy(), r1[0]["slopes"])
    native.wfs_batch_destroy(b)
    w.close()
    w1.close()


# ---------------------------------------------------------------- tensor-core DFT (split BF16, scaled FP16)

TC_PRECISIONS = [inputs.PREC_BF16X3, inputs.PREC_FP16S]


@pytest.mark.parametrize("precision", TC_PRECISIONS)
@pytest.mark.parametrize("ngs_on_tc", [False, True])
def test_config3_bf16x3_sampled_parity_full_launch(precision, ngs_on_tc):
    """The ELT frame with the LGS DFT on the tensor cores (BF16 x3, or FP16 x3 with power-of-two
    scaling; FP32 accumulation), and the NGS on the FP32 kernel or on the 64-point tensor-core
    kernel (self-projecting on its side stream), full launch, sampled subapertures against the
    FP64 oracle at the same bars as the FP32 path."""
    cfg = inputs.config3(precision, ngs_precision=precision if ngs_on_tc else inputs.PREC_FP32)
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    t = 0.071
    gpu, w = run_library(cfg, scr, t)
    sel = []
    for k, d in enumerate(gpu):
        nv = len(d["slopes"])
        sel.append(np.arange(k + 3, nv, 31, dtype=np.int32) if cfg.stars[k].is_lgs else np.arange(nv, dtype=np.int32))
    _check_wfs(cfg, scr, t, gpu, sel=sel)
    for k, d in enumerate(gpu):
        assert np.all(np.isfinite(d["slopes"])) and np.all(np.isfinite(d["E"]))
    w.close()


@pytest.mark.parametrize("precision", TC_PRECISIONS)
def test_bf16x3_matches_fp32_path_everywhere(precision):
    """Full ELT frame: every subaperture of the tensor-core path against the FP32 path."""
    scr = inputs.make_screens(inputs.config3().layers, 3000)
    a, wa = run_library(inputs.config3(inputs.PREC_FP32), scr, 0.2, stages=True)
    b, wb = run_library(inputs.config3(precision), scr, 0.2, stages=True)
    for x, y in zip(a, b):
        assert slope_rms(y["slopes"], x["slopes"]) < SLOPE_RMS
        assert rel_per_subap(y["E"], x["E"]) < INT_REL
        assert rel_per_subap(y["I"], x["I"]) < INT_REL
    wa.close()
    wb.close()


@pytest.mark.parametrize("precision", TC_PRECISIONS)
@pytest.mark.parametrize("n_sub,n,lgs,noise", [(13, 10, True, False), (11, 8, True, True),
                                               (9, 10, False, False), (7, 8, False, True)])
def test_bf16x3_edge_geometries(n_sub, n, lgs, noise, precision):
    """Ragged groups (valid count not a multiple of 4), NGS spots through the tensor-core
    kernel's binning branch, n = 8 and 10, noise on and off."""
    cfg = _small_cfg(n_sub, n, 32, 16, lgs)
    cfg.geometries[0].precision = precision
    scr = inputs.make_screens(cfg.layers, 8)
    gpu, w = run_library(cfg, scr, 0.003, seed=4, noise=noise)
    assert w.total % 4 != 0 or n_sub == 9
    _check_wfs(cfg, scr, 0.003, gpu, noise=noise, seed=4)
    if noise:
        ref = oracle.measure_wfs(cfg, scr, 0, 0.003, seed=4, noise=True, stages=True)
        same = np.abs(gpu[0]["C"] - ref["C"]) < 1e-3
        assert same.mean() >= 0.999
    w.close()


@pytest.mark.parametrize("precision", TC_PRECISIONS)
@pytest.mark.parametrize("cfg_fn", [inputs.config1, inputs.config2])
def test_tensor_core_configs_1_2_full_parity(cfg_fn, precision):
    """Configs 1 (16-point DFT, 8 x 8 detector) and 2 (24-point DFT, 12 x 12 detector, LGS with
    elongation and an NGS) with the DFT on the tensor cores: every subaperture of every WFS
    against the FP64 oracle at the bars of the FP32 path, at two times."""
    cfg = cfg_fn(precision)
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    for t in (0.0, 0.013):
        gpu, w = run_library(cfg, scr, t)
        _check_wfs(cfg, scr, t, gpu)
        w.close()


@pytest.mark.parametrize("precision", TC_PRECISIONS)
def test_tensor_core_config2_noisy_frame(precision):
    """Config 2 on the tensor cores with noise: counts equal the oracle's on >= 99.9 % of the
    pixels, slopes of the subapertures whose counts all agree within the slope bar."""
    cfg = inputs.config2(precision)
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    gpu, w = run_library(cfg, scr, 0.02, seed=42, noise=True)
    for k in (1, 3):
        ref = oracle.measure_wfs(cfg, scr, k, 0.02, seed=42, noise=True, stages=True)
        same = np.abs(gpu[k]["C"] - ref["C"]) < 1e-3
        assert same.mean() >= 0.999, same.mean()
        ok = np.all(same.reshape(len(same), -1), axis=1)
        assert slope_rms(gpu[k]["slopes"][ok], ref["slopes"][ok]) < SLOPE_RMS
    w.close()


@pytest.mark.parametrize("precision", TC_PRECISIONS)
@pytest.mark.parametrize("n_sub,n,N,nd,lgs,noise", [(9, 8, 16, 8, True, False), (7, 8, 16, 8, False, True),
                                                    (15, 6, 24, 12, True, True), (5, 6, 24, 12, False, False)])
def test_tensor_core_16_24_point_edge_geometries(n_sub, n, N, nd, lgs, noise, precision):
    """16- and 24-point geometries on the tensor cores: ragged groups (valid count not a multiple
    of 4), LGS and NGS, noise on and off, against the oracle."""
    cfg = _small_cfg(n_sub, n, N, nd, lgs)
    cfg.geometries[0].precision = precision
    scr = inputs.make_screens(cfg.layers, 8)
    gpu, w = run_library(cfg, scr, 0.003, seed=4, noise=noise)
    _check_wfs(cfg, scr, 0.003, gpu, noise=noise, seed=4)
    if noise:
        ref = oracle.measure_wfs(cfg, scr, 0, 0.003, seed=4, noise=True, stages=True)
        same = np.abs(gpu[0]["C"] - ref["C"]) < 1e-3
        assert same.mean() >= 0.999
    w.close()


@pytest.mark.parametrize("precision", [inputs.PREC_FP32] + TC_PRECISIONS)
@pytest.mark.parametrize("lgs,noise", [(True, False), (True, True), (False, False)])
def test_32_point_n8_geometry(lgs, noise, precision):
    """The 32-point kernels with 8-pixel subapertures (the lane-DFT tail with 15 autocorrelation
    rows, none folded modulo 16; the paired DFT rows k and k + 16 with the quarter turn
    i^(n-1) = -i): a ragged LGS or NGS sensor in full against the oracle, in FP32 and on the
    tensor cores, noise on and off."""
    cfg = _small_cfg(9, 8, 32, 16, lgs)
    cfg.geometries[0].precision = precision
    scr = inputs.make_screens(cfg.layers, 12)
    gpu, w = run_library(cfg, scr, 0.003, seed=6, noise=noise)
    _check_wfs(cfg, scr, 0.003, gpu, noise=noise, seed=6)
    if noise:
        ref = oracle.measure_wfs(cfg, scr, 0, 0.003, seed=6, noise=True, stages=True)
        same = np.abs(gpu[0]["C"] - ref["C"]) < 1e-3
        assert same.mean() >= 0.999
    w.close()


@pytest.mark.parametrize("precision", TC_PRECISIONS)
@pytest.mark.parametrize("n_sub,noise", [(2, False), (3, True), (4, False)])
def test_tensor_core_64_point_ngs(n_sub, noise, precision):
    """The 64-point NGS geometry (32 x 32 pupil pixels, 32 x 32 detector) on the tensor cores:
    2 x 2 to 4 x 4 subapertures (odd valid counts leave half a step idle), noise on and off,
    every subaperture against the oracle."""
    cfg = _small_cfg(n_sub, 32, 64, 32, False)
    cfg.geometries[0].precision = precision
    scr = inputs.make_screens(cfg.layers, 6)
    gpu, w = run_library(cfg, scr, 0.002, seed=5, noise=noise)
    _check_wfs(cfg, scr, 0.002, gpu, noise=noise, seed=5)
    if noise:
        ref = oracle.measure_wfs(cfg, scr, 0, 0.002, seed=5, noise=True, stages=True)
        same = np.abs(gpu[0]["C"] - ref["C"]) < 1e-3
        assert same.mean() >= 0.999
    w.close()


@pytest.mark.parametrize("precision", TC_PRECISIONS)
def test_tensor_core_64_point_lgs_is_refused(precision):
    """The 64-point tensor-core kernel has no elongation stage: an LGS on it is refused."""
    cfg = _small_cfg(2, 32, 64, 32, True)
    cfg.geometries[0].precision = precision
    with pytest.raises(native.WfsError) as ei:
        native.Wfs(cfg)
    assert ei.value.status == native.WFS_EUNSUPPORTED


@pytest.mark.parametrize("precision", TC_PRECISIONS)
def test_tensor_core_unsupported_geometry_is_refused(precision):
    """A geometry without a tensor-core kernel (odd subaperture size) is refused at creation."""
    cfg = _small_cfg(9, 7, 16, 8, False)
    cfg.geometries[0].precision = precision
    with pytest.raises(native.WfsError) as ei:
        native.Wfs(cfg)
    assert ei.value.status == native.WFS_EUNSUPPORTED


def test_fp16s_error_no_larger_than_bf16x3():
    """FP16 carries 11 significand bits to BF16's 8, so with its operands scaled into the normal
    range its split products are the more accurate: on sampled ELT subapertures its largest
    relative intensity error against the oracle stays within that of BF16 x3 (plus a margin for
    the FP32 rounding both share).  Prints both errors."""
    scr = inputs.make_screens(inputs.config3().layers, 77)
    errs = {}
    for prec in TC_PRECISIONS:
        cfg = inputs.config3(prec)
        gpu, w = run_library(cfg, scr, 0.013)
        w.close()
        sel = np.arange(5, len(gpu[0]["slopes"]), 41, dtype=np.int32)
        ref = oracle.measure_wfs(cfg, scr, 0, 0.013, sel=sel, stages=True)
        errs[prec] = (rel_per_subap(gpu[0]["I"][sel], ref["I"]), slope_rms(gpu[0]["slopes"][sel], ref["slopes"]))
    print("intensity rel / slope RMS vs oracle: BF16x3 %.3g / %.3g, FP16S %.3g / %.3g"
          % (errs[inputs.PREC_BF16X3] + errs[inputs.PREC_FP16S]))
    assert errs[inputs.PREC_FP16S][0] <= errs[inputs.PREC_BF16X3][0] * 1.05 + 1e-7


def test_bounded_wait_reports_timeout_without_fault():
    """A wait that nothing satisfies gives up after its bound and reports WFS_ETIMEOUT through
    the status word; the context stays usable (a measurement right after still works)."""
    cfg = inputs.config1()
    w = native.Wfs(cfg)
    native.wfs_check_bounded_wait(w.h, 2000, 0)
    with pytest.raises(native.WfsError) as ei:
        native.wfs_sync_status(w.h)
    assert ei.value.status == native.WFS_ETIMEOUT
    native.wfs_sync_status(w.h)          # cleared after being read
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    gpu, _ = run_library(cfg, scr, 0.0, handle=w)
    assert np.all(np.isfinite(gpu[0]["slopes"]))
    w.close()


def test_host_path_alternating_buffers():
    """Successive host-buffer calls alternate staging buffers and overlap uploads with the
    previous frame; each result equals the device path at its own time."""
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    w = native.Wfs(cfg, seed=5, noise=True)
    host_scr = torch.as_tensor(scr).pin_memory()
    outs = [torch.empty((w.total, 2)).pin_memory() for _ in range(5)]
    ts = [0.001 * k for k in range(5)]
    for t, o in zip(ts, outs):
        native.wfs_measure_host(w.h, host_scr.data_ptr(), t, o.data_ptr(), 0)
    torch.cuda.synchronize()
    for t, o in zip(ts, outs):
        ref, _ = run_library(cfg, scr, t, seed=5, noise=True, stages=False, handle=w)
        assert np.array_equal(o.numpy(), np.concatenate([d["slopes"] for d in ref]))
    w.close()


def test_host_path_uploads_only_the_read_parts(monkeypatch):
    """The host-buffer path copies only the parts of the screens a frame reads: rectangles through
    the gather kernel (pinned mapped screens, the default) or whole rows (GBWFS_HOST_RECTS=0).
    Its staging screens start as NaN and every frame brings a different screen set, so a read
    outside the copied parts would show as NaN or as another frame's data: on the ELT frame
    (uplink on, then the per-slice model, wind shifts of many pixels) every call equals the device
    path bit for bit in both forms, less than the whole set was copied, and the rectangles move
    fewer bytes than the rows.  The two forms alternate, so each keeps to one staging set."""
    import dataclasses
    monkeypatch.setenv("GBWFS_HOST_ZERO_COPY", "0")
    cfg = inputs.config3()
    cfg = dataclasses.replace(cfg, stars=[dataclasses.replace(st, uplink_diameter_m=0.4, uplink_samples=16)
                                          if st.is_lgs else st for st in cfg.stars])
    w = native.Wfs(cfg, seed=9, noise=True)
    full = 4 * cfg.layers.screen_size ** 2 * len(cfg.layers.alt_m)
    out = torch.empty((w.total, 2)).pin_memory()
    for k, (t, per_slice) in enumerate([(0.0, False), (0.37, False), (1.5, False), (2.2, True), (2.9, True)]):
        if per_slice:
            native.wfs_set_lgs_model(w.h, True)
        scr = inputs.make_screens(cfg.layers, 900 + k)
        host_scr = torch.as_tensor(scr).pin_memory()
        ref, _ = run_library(cfg, scr, t, seed=9, noise=True, stages=False, handle=w)
        ref = np.concatenate([d["slopes"] for d in ref])
        moved = {}
        for rects in ("1", "0"):
            monkeypatch.setenv("GBWFS_HOST_RECTS", rects)
            out.fill_(float("nan"))
            native.wfs_measure_host(w.h, host_scr.data_ptr(), t, out.data_ptr(), 0)
            torch.cuda.synchronize()
            h2d, d2h = native.wfs_host_transfer_bytes(w.h)
            assert 0 < h2d < 0.9 * full and d2h == 8 * w.total
            moved[rects] = h2d
            got = out.numpy().copy()
            assert np.all(np.isfinite(got)), f"call {k}, rectangles {rects}"
            assert np.array_equal(got, ref), f"call {k}, rectangles {rects}"
        assert moved["1"] < moved["0"], f"call {k}: {moved}"
    w.close()


def test_host_path_reads_pinned_screens_in_place(monkeypatch):
    """With GBWFS_HOST_ZERO_COPY=1, pinned host screens (mapped into the device's address space)
    are read in place by the kernels: nothing is copied up, and every frame equals the device path
    bit for bit (ELT frame, uplink on, then the per-slice model); pageable screens fall back to the
    row copies with the same results."""
    import dataclasses
    monkeypatch.setenv("GBWFS_HOST_ZERO_COPY", "1")
    cfg = inputs.config3()
    cfg = dataclasses.replace(cfg, stars=[dataclasses.replace(st, uplink_diameter_m=0.4, uplink_samples=16)
                                          if st.is_lgs else st for st in cfg.stars])
    w = native.Wfs(cfg, seed=9, noise=True)
    out = torch.empty((w.total, 2)).pin_memory()
    for k, (t, per_slice) in enumerate([(0.0, False), (0.41, False), (2.3, True)]):
        if per_slice:
            native.wfs_set_lgs_model(w.h, True)
        scr = inputs.make_screens(cfg.layers, 950 + k)
        ref, _ = run_library(cfg, scr, t, seed=9, noise=True, stages=False, handle=w)
        ref = np.concatenate([d["slopes"] for d in ref])
        host_scr = torch.as_tensor(scr).pin_memory()
        native.wfs_measure_host(w.h, host_scr.data_ptr(), t, out.data_ptr(), 0)
        torch.cuda.synchronize()
        h2d, d2h = native.wfs_host_transfer_bytes(w.h)
        assert h2d == 0 and d2h == 8 * w.total
        assert np.array_equal(out.numpy(), ref), f"call {k} (in place)"
        pageable = np.ascontiguousarray(scr)
        native.wfs_measure_host(w.h, pageable.ctypes.data, t, out.data_ptr(), 0)
        torch.cuda.synchronize()
        h2d, _ = native.wfs_host_transfer_bytes(w.h)
        assert h2d > 0
        assert np.array_equal(out.numpy(), ref), f"call {k} (pageable)"
    w.close()


def test_busy_on_another_stream():
    """One stream at a time: while a measurement is still queued or running on one stream, a
    call on another stream is refused with WFS_EBUSY and launches nothing; once it has finished,
    the other stream may use the handle and gets the same slopes."""
    cfg = inputs.config1()
    scr = torch.as_tensor(inputs.make_screens(cfg.layers, cfg.seed)).cuda()
    w = native.Wfs(cfg, seed=2, noise=False)
    a = torch.full((w.total, 2), float("nan"), device="cuda")
    b = torch.full((w.total, 2), float("nan"), device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s1):
        torch.cuda._sleep(200_000_000)  # a bounded busy wait queued ahead of the measurement
        native.wfs_measure(w.h, scr.data_ptr(), 0.004, a.data_ptr(), s1.cuda_stream)
    with pytest.raises(native.WfsError) as err:
        native.wfs_measure(w.h, scr.data_ptr(), 0.004, b.data_ptr(), s2.cuda_stream)
    assert err.value.status == native.STATUS_NAMES.index("WFS_EBUSY")
    torch.cuda.synchronize()
    assert torch.isnan(b).all()
    native.wfs_measure(w.h, scr.data_ptr(), 0.004, b.data_ptr(), s2.cuda_stream)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    w.close()


@pytest.mark.parametrize("precision", TC_PRECISIONS)
def test_first_dft_stage_as_mma_parity(monkeypatch, precision):
    """The tensor-core kernels' variant with U = F X as a third MMA (GBWFS_TC_MMA_U=1): config 2
    in full and the ELT frame sampled against the oracle at the same bars."""
    monkeypatch.setenv("GBWFS_TC_MMA_U", "1")
    cfg = inputs.config2(precision)
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    gpu, w = run_library(cfg, scr, 0.031)
    _check_wfs(cfg, scr, 0.031, gpu)
    w.close()
    cfg = inputs.config3(precision)
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    gpu, w = run_library(cfg, scr, 0.05)
    sel = [np.arange(k, len(d["slopes"]), 37, dtype=np.int32) if cfg.stars[k].is_lgs
           else np.arange(len(d["slopes"]), dtype=np.int32) for k, d in enumerate(gpu)]
    _check_wfs(cfg, scr, 0.05, gpu, sel=sel)
    w.close()
