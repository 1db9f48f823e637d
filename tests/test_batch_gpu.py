"""Uneven batches (config-4 style): one projection launch plus one persistent spot launch per
kernel class, replayed as a CUDA graph, must give the same slopes as measuring every handle
alone -- bit for bit, with and without the graph, before and after autotuning -- and sampled
subapertures of every instance must match the FP64 oracle."""
import os

import numpy as np
import pytest

from paper_1408_0698_gb300 import inputs, native

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from _gpu import check_against_oracle  # noqa: E402


MIXED = "mixed"  # tensor-core geometries alternate between BF16 x3 and scaled FP16 x3
# (n_pix_sub, n_fft, n_det) with a tensor-core spot kernel
TC_GEOMETRIES = {(10, 32, 16), (8, 32, 16), (8, 16, 8), (6, 24, 12), (32, 64, 32)}


def _instances(k, seed=4000, prec=inputs.PREC_FP32):
    insts = inputs.config4_instances(k, seed, precision=inputs.PREC_BF16X3 if prec == MIXED else prec)
    out = []
    for i, c in enumerate(insts):
        g = c.geometries[0]
        tc_ok = (g.n_pix_sub, g.n_fft, g.n_det) in TC_GEOMETRIES
        if prec == MIXED:
            g.precision = (inputs.PREC_BF16X3 if i % 2 else inputs.PREC_FP16S) if tc_ok else inputs.PREC_FP32
        elif prec in (inputs.PREC_BF16X3, inputs.PREC_FP16S) and not tc_ok:
            g.precision = inputs.PREC_FP32
        out.append(c)
    return out


def _setup(insts, noise):
    dev = torch.device("cuda:0")
    hs, scr, outs = [], [], []
    for i, c in enumerate(insts):
        w = native.Wfs(c, seed=c.seed, noise=noise)
        hs.append(w)
        scr.append(torch.as_tensor(inputs.make_screens(c.layers, c.seed)).to(dev))
        outs.append(torch.zeros((max(w.total, 1), 2), device=dev))
    return hs, scr, outs


def _alone(hs, scr, ts):
    res = []
    for w, s, t in zip(hs, scr, ts):
        o = torch.zeros((max(w.total, 1), 2), device="cuda:0")
        native.wfs_measure(w.h, s.data_ptr(), t, o.data_ptr(), 0)
        res.append(o)
    torch.cuda.synchronize()
    return [r.cpu().numpy() for r in res]


@pytest.mark.parametrize("prec,noise", [(inputs.PREC_FP32, True), (inputs.PREC_BF16X3, False), (MIXED, True)])
def test_uneven_batch_equals_alone(prec, noise):
    insts = _instances(24, 4000, prec)
    hs, scr, outs = _setup(insts, noise)
    b = native.wfs_batch_create([w.h for w in hs])
    info = native.wfs_batch_info(b)
    assert sum(c["n_wfs"] for c in info) == len(hs)
    assert {c["n_fft"] for c in info} >= {16, 24, 32, 64}
    for step in range(3):                       # graph build, then two replays
        ts = [0.003 * step + 1e-4 * i for i in range(len(hs))]
        native.wfs_batch_measure(b, [s.data_ptr() for s in scr], ts, [o.data_ptr() for o in outs], 0)
        torch.cuda.synchronize()
        ref = _alone(hs, scr, ts)
        for i, (o, r) in enumerate(zip(outs, ref)):
            assert np.array_equal(o.cpu().numpy(), r), f"instance {i} step {step}"
        if step == 1:
            # every instance (each geometry, precision and layer count config 4 draws) against
            # the oracle on sampled subapertures of each of its WFSs
            for i, (c, w, o) in enumerate(zip(insts, hs, outs)):
                check_against_oracle(c, scr[i].cpu().numpy(), ts[i], o.cpu().numpy(), w.layouts,
                                     seed=c.seed, noise=noise, per_wfs=12)
    # tuning changes launch shapes only, never results
    ts = [0.05 + 1e-4 * i for i in range(len(hs))]
    native.wfs_batch_tune(b, [s.data_ptr() for s in scr], ts, [o.data_ptr() for o in outs], 0)
    info2 = native.wfs_batch_info(b)
    assert all(c["grid_cap"] > 0 for c in info2)
    native.wfs_batch_measure(b, [s.data_ptr() for s in scr], ts, [o.data_ptr() for o in outs], 0)
    torch.cuda.synchronize()
    ref = _alone(hs, scr, ts)
    for o, r in zip(outs, ref):
        assert np.array_equal(o.cpu().numpy(), r)
    native.wfs_batch_destroy(b)
    for w in hs:
        w.close()


def test_batch_direct_launch_matches_graph(monkeypatch):
    insts = _instances(10, 4100)
    hs, scr, outs = _setup(insts, True)
    ts = [0.01 * i for i in range(len(hs))]
    b = native.wfs_batch_create([w.h for w in hs])
    native.wfs_batch_measure(b, [s.data_ptr() for s in scr], ts, [o.data_ptr() for o in outs], 0)
    torch.cuda.synchronize()
    g = [o.cpu().numpy() for o in outs]
    native.wfs_batch_destroy(b)
    monkeypatch.setenv("GBWFS_BATCH_GRAPH", "0")
    b = native.wfs_batch_create([w.h for w in hs])
    for o in outs:
        o.zero_()
    native.wfs_batch_measure(b, [s.data_ptr() for s in scr], ts, [o.data_ptr() for o in outs], 0)
    torch.cuda.synchronize()
    for o, r in zip(outs, g):
        assert np.array_equal(o.cpu().numpy(), r)
    native.wfs_batch_destroy(b)
    for w in hs:
        w.close()


def test_tune_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("GBWFS_TUNE_CACHE", str(path))
    insts = _instances(6, 4200)
    hs, scr, outs = _setup(insts, False)
    ts = [0.0] * len(hs)
    b = native.wfs_batch_create([w.h for w in hs])
    native.wfs_batch_tune(b, [s.data_ptr() for s in scr], ts, [o.data_ptr() for o in outs], 0)
    tuned = [(c["grid_cap"], c["cta_warps"]) for c in native.wfs_batch_info(b)]
    native.wfs_batch_destroy(b)
    assert path.exists() and len(path.read_text().splitlines()) == len(tuned)
    b = native.wfs_batch_create([w.h for w in hs])
    assert [(c["grid_cap"], c["cta_warps"]) for c in native.wfs_batch_info(b)] == tuned
    native.wfs_batch_destroy(b)
    for w in hs:
        w.close()


def test_batch_rejects_bad_arguments():
    c = inputs.config1()
    w = native.Wfs(c)
    with pytest.raises(native.WfsError):
        native.wfs_batch_create([w.h, w.h])
    w.close()


def test_tensor_core_tile_shapes_give_the_same_results(tmp_path, monkeypatch):
    """Both tile shapes of the tensor-core kernels (two warpgroups per CTA, or one, which the tuner
    chooses between) measure every class bit for bit as the handles alone: the shape is forced
    through the tuning cache."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("GBWFS_TUNE_CACHE", str(path))
    insts = _instances(16, 4300, inputs.PREC_BF16X3)
    hs, scr, outs = _setup(insts, True)
    ts = [0.004 + 1e-4 * i for i in range(len(hs))]
    b = native.wfs_batch_create([w.h for w in hs])
    native.wfs_batch_tune(b, [s.data_ptr() for s in scr], ts, [o.data_ptr() for o in outs], 0)
    native.wfs_batch_destroy(b)
    lines = path.read_text().split("\n")
    for shape in (4, 8):
        forced = []
        for ln in lines:
            if not ln.strip():
                continue
            k, cap, w = ln.split()
            forced.append(f"{k} {cap} {shape if k.startswith('kind2_') or k.startswith('kind3_') else w}")
        path.write_text("\n".join(forced) + "\n")
        b = native.wfs_batch_create([w.h for w in hs])
        info = native.wfs_batch_info(b)
        assert any(c["kind"] in (2, 3) and c["n_fft"] <= 32 and c["cta_warps"] == shape for c in info)
        native.wfs_batch_measure(b, [s.data_ptr() for s in scr], ts, [o.data_ptr() for o in outs], 0)
        torch.cuda.synchronize()
        ref = _alone(hs, scr, ts)
        for i, (o, r) in enumerate(zip(outs, ref)):
            assert np.array_equal(o.cpu().numpy(), r), (shape, i)
        native.wfs_batch_destroy(b)
    for w in hs:
        w.close()
