"""Host-side pieces of the serving loop that need no GPU: the seeded run mix, the Poisson
request stream and the device-footprint estimate used for admission."""
import numpy as np

from paper_1408_0698_gb300 import inputs, serving


def test_run_mix_is_seeded_and_runs_differ():
    mix = (inputs.config1, inputs.config2)
    a = serving.make_runs(6, seed=77, mix=mix)
    b = serving.make_runs(6, seed=77, mix=mix)
    assert [r.cfg.name for r in a] == [r.cfg.name for r in b]
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x.cfg.layers.x0_m, y.cfg.layers.x0_m)
        assert x.seed == y.seed
    # runs of one configuration share the screens but not their layer offsets or noise seeds
    names = [r.cfg.name for r in a]
    same = [(i, j) for i in range(6) for j in range(i + 1, 6) if names[i] == names[j]]
    assert same
    for i, j in same:
        assert a[i].screens_host is a[j].screens_host
        assert not np.array_equal(a[i].cfg.layers.x0_m, a[j].cfg.layers.x0_m)
        assert a[i].seed != a[j].seed


def test_poisson_arrivals_rate_order_and_caps():
    runs = serving.make_runs(4, seed=3, mix=(inputs.config1,))
    rate, dur = 200.0, 5.0
    arr = serving.poisson_arrivals(runs, rate, dur, seed=9)
    assert arr == serving.poisson_arrivals(runs, rate, dur, seed=9)
    per_run = {}
    for t, rid, step in arr:
        assert 0.0 < t <= dur
        per_run.setdefault(rid, []).append((t, step))
    for rid, lst in per_run.items():
        times = [t for t, _ in lst]
        assert times == sorted(times)
        assert [s for _, s in lst] == list(range(len(lst)))   # steps in order, none skipped
        # Poisson count over 5 s at 200/s: mean 1000, sd ~32
        assert abs(len(lst) - rate * dur) < 5 * np.sqrt(rate * dur)
    capped = serving.poisson_arrivals(runs, rate, dur, seed=9, max_per_run=7)
    assert all(sum(1 for _, r, _ in capped if r == rid) == 7 for rid in per_run)
    staggered = serving.poisson_arrivals(runs, rate, 1.0, seed=9, stagger_s=0.5)
    assert min(t for t, r, _ in staggered if r == runs[3].run_id) > 1.5


def test_footprint_grows_with_the_workload():
    f1, f2, f3 = (serving.footprint_bytes(c()) for c in (inputs.config1, inputs.config2, inputs.config3))
    assert f1 < f2 < f3
    # the screens dominate: config 3 holds 10 layers of 2048^2 FP32
    assert f3 >= 10 * 2048 * 2048 * 4
