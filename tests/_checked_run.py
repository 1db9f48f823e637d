"""Runs a fixed set of measurements through the C ABI and saves every output to an .npz file.

Run as a child process, once with the normal library and once with the bounds-checked one
(environment variable GBWFS_CHECKED=1): the parent test compares the two files.  Covered:
the generic, 32-point and tensor-core spot kernels (BF16 x3 and scaled FP16 x3), the projection
(direct and tiled), the noise and centroid pass, the uplink tip-tilt, the per-slice LGS model,
the host-buffer path, a loop step with mirror layers, a push-pull calibration and a batch of two
handles.  Every result is
followed by wfs_sync_status, which raises on a device status such as WFS_EBOUNDS.
"""
import dataclasses
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path[:0] = [os.path.dirname(HERE), HERE]

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1408_0698_gb300 import inputs, native  # noqa: E402


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _measure(cfg, scr, t, noise=False, seed=3):
    w = native.Wfs(cfg, seed=seed, noise=noise)
    s = torch.full((w.total, 2), float("nan"), device="cuda")
    native.wfs_measure(w.h, scr.data_ptr(), t, s.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    native.wfs_sync_status(w.h)
    w.close()
    return s.cpu().numpy()


def _lgs(cfg, **kw):
    return dataclasses.replace(cfg, stars=[dataclasses.replace(s, **kw) if s.is_lgs else s
                                           for s in cfg.stars])


def main(out):
    res = {}
    c2 = inputs.config2()
    s2 = _dev(inputs.make_screens(c2.layers, c2.seed))
    res["config2"] = _measure(c2, s2, 0.013, noise=True)
    res["config2_uplink"] = _measure(_lgs(c2, uplink_diameter_m=0.5, uplink_samples=16), s2, 0.0)
    res["config2_slices"] = _measure(_lgs(c2, per_slice=True), s2, 0.0)
    for name, prec in (("elt_bf16x3", inputs.PREC_BF16X3), ("elt_fp16s", inputs.PREC_FP16S),
                       ("elt_fp32", inputs.PREC_FP32)):
        c3 = inputs.config3(prec)
        s3 = _dev(inputs.make_screens(c3.layers, c3.seed))
        res[name] = _measure(c3, s3, 0.05, noise=True)
        res[name + "_slices"] = _measure(_lgs(c3, per_slice=True), s3, 0.05)
        del s3

    # the host-buffer path (only the rows a frame reads are uploaded), two frames
    w = native.Wfs(c2, seed=4, noise=True)
    host_scr = torch.as_tensor(inputs.make_screens(c2.layers, c2.seed + 5)).pin_memory()
    for k, t in enumerate((0.0, 0.8)):
        hbuf = torch.empty((w.total, 2)).pin_memory()
        native.wfs_measure_host(w.h, host_scr.data_ptr(), t, hbuf.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        native.wfs_sync_status(w.h)
        res[f"host{k}"] = hbuf.numpy().copy()
    w.close()

    # a loop step and a calibration on config 2 with two mirrors
    dms = [inputs.Dm(21, 0.4, 0.0, 37), inputs.Dm(15, 0.7, 6000.0, 9)]
    m2a = [_dev(inputs.modal_base(d, 21 + i, amplitude_m=2e-8)) for i, d in enumerate(dms)]
    n = sum(d.n_modes for d in dms)
    w = native.Wfs(c2)
    cm = _dev(inputs.random_control_matrix(n, 2 * w.total, seed=5, scale=0.5))
    gain = _dev(np.full(n, 0.4))
    structs = [native.wfs_dm(d.n_act, d.pitch_m, d.alt_m, d.coupling, d.support, d.n_modes, M.data_ptr())
               for d, M in zip(dms, m2a)]
    lp = native.wfs_loop_create(w.h, structs, cm.data_ptr(), gain.data_ptr())
    st = torch.cuda.current_stream().cuda_stream
    native.wfs_loop_set_coeffs(lp, w.h, _dev(np.random.default_rng(1).standard_normal(n)).data_ptr(), st)
    sl = torch.zeros((w.total, 2), device="cuda")
    native.wfs_loop_step(lp, w.h, s2.data_ptr(), 0.004, sl.data_ptr(), st)
    co = torch.zeros(n, device="cuda")
    native.wfs_loop_get_coeffs(lp, w.h, co.data_ptr(), st)
    torch.cuda.synchronize()
    native.wfs_sync_status(w.h)
    res["loop_slopes"], res["loop_coeffs"] = sl.cpu().numpy(), co.cpu().numpy()
    nv = native.wfs_num_valid(w.h, 0)
    im = torch.zeros((n, 2 * nv), device="cuda")
    native.wfs_loop_calibrate(lp, w.h, 0, 0.5, im.data_ptr(), st)
    torch.cuda.synchronize()
    native.wfs_sync_status(w.h)
    res["calibration"] = im.cpu().numpy()
    native.wfs_loop_destroy(lp)
    w.close()

    # a batch of two handles of config 2 (different seeds and times)
    hs = [native.Wfs(c2, seed=k, noise=True) for k in range(2)]
    b = native.wfs_batch_create([x.h for x in hs])
    outs = [torch.zeros((x.total, 2), device="cuda") for x in hs]
    native.wfs_batch_measure(b, [s2.data_ptr()] * 2, [0.0, 0.02], [o.data_ptr() for o in outs], st)
    torch.cuda.synchronize()
    for x in hs:
        native.wfs_sync_status(x.h)
    res["batch0"], res["batch1"] = (o.cpu().numpy() for o in outs)
    native.wfs_batch_destroy(b)
    for x in hs:
        x.close()

    res["library"] = np.array(native.lib()._name)
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
