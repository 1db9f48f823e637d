"""The plain-C99 example (one frame through the C ABI with cudaMalloc'd buffers) gives the same
slopes as the Python binding on the same description and screen, noise off and on."""
import subprocess

import numpy as np
import pytest

from paper_1408_0698_gb300 import inputs, native

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from _c_example import compile_example  # noqa: E402


@pytest.mark.parametrize("noise", [0, 1])
def test_c_example_matches_binding(tmp_path, noise):
    exe = compile_example(str(tmp_path / "measure_frame"))
    cfg = inputs.config1()  # the example's hard-coded sensor
    scr = inputs.make_screens(cfg.layers, cfg.seed).astype(np.float32)
    scr.tofile(tmp_path / "s.f32")
    t = 0.004
    r = subprocess.run([exe, str(tmp_path / "s.f32"), repr(t), str(tmp_path / "o.f32"), str(noise)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = np.fromfile(tmp_path / "o.f32", dtype=np.float32).reshape(-1, 2)
    w = native.Wfs(cfg, seed=1, noise=bool(noise))
    out = torch.empty((w.total, 2), device="cuda")
    native.wfs_measure(w.h, torch.as_tensor(scr).cuda().data_ptr(), t, out.data_ptr(),
                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    w.close()
    assert got.shape == (316, 2)
    np.testing.assert_array_equal(got, out.cpu().numpy())
