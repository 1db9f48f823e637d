"""wfs_measure_one_static: the measurement for callers that cannot allocate device memory
(a real-time loop that must not block on the allocator, a host program with a fixed
device budget, a plugin that only receives buffers).  It keeps its working data in the
library's static device array instead of a handle's allocations; its slopes must equal
those of wfs_measure on a handle holding the same guide star, bit for bit, call after call.

Collected last on purpose (file name), so a run that stops at the first failure has
already run every other test."""
import dataclasses

import numpy as np
import pytest

from paper_1408_0698_gb300 import inputs, native

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _one_star(cfg, k):
    c = dataclasses.replace(cfg)
    s = dataclasses.replace(cfg.stars[k])
    c.stars = [s]
    c.geometries = [cfg.geometries[s.geometry_index]]
    s.geometry_index = 0
    return c


@pytest.mark.parametrize("cfg_fn,k,noise", [(inputs.config2, 0, False), (inputs.config2, 3, True),
                                            (inputs.config1, 0, True)])
def test_static_scratch_entry_matches_wfs_measure(cfg_fn, k, noise):
    cfg = _one_star(cfg_fn(), k)
    dev = torch.device("cuda:0")
    scr = torch.as_tensor(inputs.make_screens(cfg.layers, cfg.seed)).to(dev)
    w = native.Wfs(cfg, seed=21, noise=noise)
    tel, stars, geoms, lay, keep = native.marshal(cfg)
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.empty((w.total, 2), device=dev)
    cap = w.total + 3
    out = torch.full((cap, 2), float("nan"), device=dev)
    free_after_first = None
    for call, t in enumerate((0.01, 0.017)):          # two calls in a row
        native.wfs_measure(w.h, scr.data_ptr(), t, ref.data_ptr(), stream)
        nv = native.wfs_measure_one_static(tel, geoms[0], stars[0], lay, scr.data_ptr(), t, 21, 0, noise,
                                           out.data_ptr(), cap, stream)
        torch.cuda.synchronize()
        assert nv == w.total
        a, b = out[:nv].cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        # the same kernels on the same inputs: bit for bit (the projection's direct gathers do
        # the tiled form's per-tap arithmetic in the same order)
        assert np.array_equal(a, b)
        assert np.all(np.isnan(out[nv:].cpu().numpy()))   # nothing written past n_valid
        free = torch.cuda.mem_get_info()[0]
        if call == 0:
            free_after_first = free
        else:
            # the second call allocated nothing (a coarse check: the driver's free-memory figure
            # moves by whole pages when anything is allocated on the device)
            assert free == free_after_first
    w.close()


def test_static_scratch_entry_rejects_oversize():
    """A wavefront sensor whose tables exceed the static array is refused with a message."""
    cfg = _one_star(inputs.config2(), 0)
    cfg.geometries[0] = inputs.Geometry(120, 32, 64, 32, 0.5)
    cfg.telescope = inputs.Telescope(8.0, 0.0)
    cfg.layers = dataclasses.replace(cfg.layers, screen_size=8192, screen_dx_m=8.0 / (120 * 32))
    tel, stars, geoms, lay, keep = native.marshal(cfg)
    dev = torch.device("cuda:0")
    scr = torch.zeros(1, device=dev)
    out = torch.zeros(2, device=dev)
    with pytest.raises(native.WfsError) as ei:
        native.wfs_measure_one_static(tel, geoms[0], stars[0], lay, scr.data_ptr(), 0.0, 1, 0, False,
                                      out.data_ptr(), 1, 0)
    assert ei.value.status == native.WFS_EINVAL
    assert "static" in native.wfs_last_error(None)
