"""Serving: continuous batching of frame requests from concurrent Monte-Carlo runs.  Each
served result must equal the same (run, step) measured alone; admission must respect the HBM
budget; latency statistics must be produced."""
import numpy as np
import pytest

from paper_1408_0698_gb300 import inputs, native, serving

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from _gpu import check_against_oracle  # noqa: E402


def _small_runs(n=6, seed=77):
    return serving.make_runs(n, seed, mix=(inputs.config1, inputs.config2))


def test_served_results_equal_alone():
    runs = _small_runs(6)
    srv = serving.Server(runs, hbm_budget_bytes=64 << 30, slots=3, keep_results=True)
    srv.preadmit()
    arrivals = serving.poisson_arrivals(runs, rate_per_run=400.0, duration_s=0.25, seed=3)
    st = srv.serve(arrivals)
    s = st.summary()
    assert s["requests"] == len(arrivals) and s["batches"] > 0
    assert s["mean_batch"] > 1.0          # requests really were batched together
    assert 0 < s["p50_ms"] <= s["p99_ms"]
    # the same (run, step) measured alone, on a fresh handle with the same seed
    rng = np.random.default_rng(0)
    keys = list(srv.results)
    pick = [keys[i] for i in rng.choice(len(keys), size=min(12, len(keys)), replace=False)]
    dev = torch.device("cuda:0")
    for rid, step in pick:
        r = runs[rid]
        w = native.Wfs(r.cfg, seed=r.seed, noise=True)
        scr = torch.as_tensor(r.screens_host).to(dev)
        out = torch.zeros((w.total, 2), device=dev)
        native.wfs_measure(w.h, scr.data_ptr(), step * r.cfg.dt_s, out.data_ptr(), 0)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), srv.results[(rid, step)]), (rid, step)
        w.close()
    # a few served results against the FP64 oracle (sampled subapertures of every WFS)
    for rid, step in pick[:4]:
        r = runs[rid]
        w = native.Wfs(r.cfg, seed=r.seed)
        check_against_oracle(r.cfg, r.screens_host, step * r.cfg.dt_s, srv.results[(rid, step)],
                             w.layouts, seed=r.seed, noise=True, per_wfs=10)
        w.close()


def test_admission_respects_budget():
    runs = _small_runs(5, seed=78)
    fp = sorted(serving.footprint_bytes(r.cfg) for r in runs)
    budget = fp[-1] + fp[-2]                  # at most two runs resident at once
    arrivals = serving.poisson_arrivals(runs, rate_per_run=300.0, duration_s=0.05, seed=4,
                                        stagger_s=0.01, max_per_run=6)
    st = serving.Server(runs, budget, slots=2).serve(arrivals)
    assert st.completed == len(arrivals)
    assert 1 <= st.admitted_max <= 2


def test_subset_call_validation():
    runs = _small_runs(2, seed=79)
    ws = [native.Wfs(r.cfg) for r in runs]
    b = native.wfs_batch_create([w.h for w in ws])
    with pytest.raises(native.WfsError):
        native.wfs_batch_measure_subset(b, 9, [0], [1], [0.0], [1])      # bad slot
    with pytest.raises(native.WfsError):
        native.wfs_batch_measure_subset(b, 0, [0, 0], [1, 1], [0.0, 0.0], [1, 1])  # repeated
    native.wfs_batch_destroy(b)
    for w in ws:
        w.close()
