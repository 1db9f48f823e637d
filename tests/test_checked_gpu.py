"""The bounds-checked library (built with -DGBWFS_CHECK) on the measurement, loop, calibration
and batch paths.

In that build every kernel tests the global indices it derives (valid subaperture, screen
taps, staged boxes) before the access, skips an out-of-range one and records WFS_EBOUNDS in
the handle's status word.  The same child script runs once per library; every call must
finish with status WFS_OK, and every output must be bit-identical between the two builds
(the checks only add branches that are never taken).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(tmp_path, checked):
    out = str(tmp_path / ("checked.npz" if checked else "normal.npz"))
    env = dict(os.environ, GBWFS_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_checked_run.py"), out], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return dict(np.load(out))


def test_checked_build_matches_and_reports_ok(tmp_path):
    a = _run(tmp_path, checked=False)
    b = _run(tmp_path, checked=True)
    assert str(a.pop("library")).endswith("libgbwfs.so")
    assert str(b.pop("library")).endswith("libgbwfs_check.so")
    assert sorted(a) == sorted(b)
    for k in a:
        assert np.all(np.isfinite(a[k])), k
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
