"""Thin ctypes binding of libgbwfs.so (include/gbwfs.h).

Argument marshalling only: every step of the measurement runs in the library's
CUDA kernels.  Device buffers are passed as integer addresses (for example
``torch.Tensor.data_ptr()``), streams as ``torch.cuda.Stream.cuda_stream``.
The library is loaded from the package's in-tree ``_build`` folder; if it is
missing or fails to load, every call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import re
import threading

import numpy as np

from . import build as _build

WFS_OK, WFS_EINVAL, WFS_ENOMEM, WFS_ECUDA, WFS_EBUSY, WFS_ETIMEOUT, WFS_EUNSUPPORTED, WFS_EBOUNDS = range(8)
STATUS_NAMES = ["WFS_OK", "WFS_EINVAL", "WFS_ENOMEM", "WFS_ECUDA", "WFS_EBUSY", "WFS_ETIMEOUT",
                "WFS_EUNSUPPORTED", "WFS_EBOUNDS"]
WFS_PREC_FP32, WFS_PREC_BF16X3, WFS_PREC_FP16S = 0, 1, 2


class WfsError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class wfs_telescope(C.Structure):
    _fields_ = [("diameter_m", C.c_double), ("obstruction", C.c_double)]


class wfs_geometry(C.Structure):
    _fields_ = [("n_sub", C.c_int), ("n_pix_sub", C.c_int), ("n_fft", C.c_int), ("n_det", C.c_int),
                ("valid_fill", C.c_double), ("precision", C.c_int)]


class wfs_guide_star(C.Structure):
    _fields_ = [("is_lgs", C.c_int), ("theta_x_rad", C.c_double), ("theta_y_rad", C.c_double),
                ("range_m", C.c_double), ("wavelength_m", C.c_double), ("launch_x_m", C.c_double),
                ("launch_y_m", C.c_double), ("spot_fwhm_rad", C.c_double),
                ("photons_per_subap", C.c_double), ("read_noise_e", C.c_double),
                ("geometry_index", C.c_int), ("n_na", C.c_int),
                ("na_alt_m", C.POINTER(C.c_double)), ("na_weight", C.POINTER(C.c_double))]


class wfs_layers(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("screen_size", C.c_int), ("screen_dx_m", C.c_double),
                ("alt_m", C.POINTER(C.c_double)), ("wind_vx_mps", C.POINTER(C.c_double)),
                ("wind_vy_mps", C.POINTER(C.c_double)), ("x0_m", C.POINTER(C.c_double)),
                ("y0_m", C.POINTER(C.c_double))]


class wfs_stage_out(C.Structure):
    _fields_ = [("opd", C.c_void_p), ("intensity", C.c_void_p), ("expected", C.c_void_p),
                ("counts", C.c_void_p)]


class wfs_layout_info(C.Structure):
    _fields_ = [("n_valid", C.c_int), ("n", C.c_int), ("n_fft", C.c_int), ("n_det", C.c_int),
                ("is_lgs", C.c_int), ("slope_offset", C.c_size_t), ("opd_offset", C.c_size_t),
                ("intensity_offset", C.c_size_t), ("det_offset", C.c_size_t)]


class wfs_batch_class(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_pix_sub", C.c_int), ("n_fft", C.c_int), ("n_det", C.c_int),
                ("n_wfs", C.c_int), ("n_subaps", C.c_int), ("grid_cap", C.c_int), ("cta_warps", C.c_int)]


class wfs_dm(C.Structure):
    _fields_ = [("n_act", C.c_int), ("pitch_m", C.c_double), ("alt_m", C.c_double),
                ("coupling", C.c_double), ("support", C.c_int), ("n_modes", C.c_int),
                ("m2a", C.c_void_p)]


class wfs_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int), ("total_ms", C.c_double)]


_H = C.c_void_p
_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); the header is the source of truth for the name list
_SIGS = {
    "wfs_create": (C.c_int, [C.POINTER(wfs_telescope), C.c_int, C.POINTER(wfs_guide_star), C.c_int,
                             C.POINTER(wfs_geometry), C.POINTER(wfs_layers), C.c_uint64, C.c_int,
                             C.POINTER(_H)]),
    "wfs_destroy": (C.c_int, [_H]),
    "wfs_measure": (C.c_int, [_H, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    "wfs_measure_stages": (C.c_int, [_H, C.c_void_p, C.c_double, C.c_void_p,
                                     C.POINTER(wfs_stage_out), C.c_void_p]),
    "wfs_measure_host": (C.c_int, [_H, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    "wfs_host_transfer_bytes": (C.c_int, [_H, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "wfs_set_noise": (C.c_int, [_H, C.c_int]),
    "wfs_num_valid": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int)]),
    "wfs_total_valid": (C.c_int, [_H, C.POINTER(C.c_int)]),
    "wfs_valid_map": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int32)]),
    "wfs_layout": (C.c_int, [_H, C.c_int, C.POINTER(wfs_layout_info)]),
    "wfs_sync_status": (C.c_int, [_H]),
    "wfs_last_error": (C.c_char_p, [_H]),
    "wfs_noise_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_float, C.c_uint64, C.c_uint32, C.c_double,
                                  C.c_uint32, C.c_void_p, C.c_void_p]),
    "wfs_batch_create": (C.c_int, [C.c_int, C.POINTER(_H), C.POINTER(_H)]),
    "wfs_batch_measure": (C.c_int, [_H, C.POINTER(C.c_void_p), C.POINTER(C.c_double),
                                    C.POINTER(C.c_void_p), C.c_void_p]),
    "wfs_batch_destroy": (C.c_int, [_H]),
    "wfs_batch_tune": (C.c_int, [_H, C.POINTER(C.c_void_p), C.POINTER(C.c_double),
                                 C.POINTER(C.c_void_p), C.c_void_p]),
    "wfs_batch_measure_subset": (C.c_int, [_H, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_void_p),
                                           C.POINTER(C.c_double), C.POINTER(C.c_void_p), C.c_void_p]),
    "wfs_batch_info": (C.c_int, [_H, C.c_int, C.POINTER(wfs_batch_class), C.POINTER(C.c_int)]),
    "wfs_version": (C.c_char_p, []),
    "wfs_timing_enable": (C.c_int, [_H, C.c_int]),
    "wfs_check_bounded_wait": (C.c_int, [_H, C.c_int, C.c_void_p]),
    "wfs_measure_one_static": (C.c_int, [C.POINTER(wfs_telescope), C.POINTER(wfs_geometry),
                                         C.POINTER(wfs_guide_star), C.POINTER(wfs_layers), C.c_void_p,
                                         C.c_double, C.c_uint64, C.c_uint32, C.c_int, C.c_void_p, C.c_int,
                                         C.POINTER(C.c_int), C.c_void_p]),
    "wfs_timing_read": (C.c_int, [_H, C.c_int, C.POINTER(wfs_kernel_time), C.POINTER(C.c_int)]),
    "wfs_loop_create": (C.c_int, [_H, C.c_int, C.POINTER(wfs_dm), C.c_void_p, C.c_void_p, C.POINTER(_H)]),
    "wfs_loop_step": (C.c_int, [_H, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    "wfs_loop_set_coeffs": (C.c_int, [_H, C.c_void_p, C.c_void_p]),
    "wfs_loop_get_coeffs": (C.c_int, [_H, C.c_void_p, C.c_void_p]),
    "wfs_loop_get_layer": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_void_p]),
    "wfs_loop_destroy": (C.c_int, [_H]),
    "wfs_loop_calibrate": (C.c_int, [_H, C.c_int, C.c_double, C.c_void_p, C.c_void_p]),
    "wfs_set_uplink": (C.c_int, [_H, C.c_int, C.c_double, C.c_int]),
    "wfs_set_lgs_model": (C.c_int, [_H, C.c_int]),
    "wfs_loop_batch_create": (C.c_int, [C.c_int, C.POINTER(_H), C.POINTER(_H)]),
    "wfs_loop_batch_step": (C.c_int, [_H, C.POINTER(C.c_void_p), C.POINTER(C.c_double), C.POINTER(C.c_void_p),
                                      C.c_void_p]),
    "wfs_loop_batch_destroy": (C.c_int, [_H]),
}


def header_symbols(path=None):
    """Function names declared in include/gbwfs.h."""
    path = path or os.path.join(_build.ROOT, "include", "gbwfs.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wfs_[a-z_0-9]+)\s*\(", text)))


def lib(build_if_missing: bool = True):
    """Load libgbwfs.so (building it first if stale and allowed); with the environment variable
    GBWFS_CHECKED=1, the bounds-checked build instead."""
    global _lib
    with _lock:
        if _lib is None:
            checked = os.environ.get("GBWFS_CHECKED") == "1"
            if build_if_missing:
                path = _build.build(check=checked)
            else:
                path = _build.CHECK_SO if checked else _build.SO
            if not os.path.exists(path):
                raise RuntimeError(f"libgbwfs.so not built ({path}); run __graft_entry__.build()")
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _check(st, h=None):
    if st != WFS_OK:
        msg = lib().wfs_last_error(h)
        raise WfsError(st, msg.decode() if msg else "")


# ------------------------------------------------------------------ same-name wrappers

def wfs_version() -> str:
    return lib().wfs_version().decode()


def wfs_last_error(h=None) -> str:
    m = lib().wfs_last_error(h)
    return m.decode() if m else ""


def wfs_create(tel, stars, geoms, layers, seed, noise_enable):
    """Ctypes structs in, handle out (raises WfsError on failure)."""
    h = _H()
    n_gs = len(stars)
    gs_arr = (wfs_guide_star * n_gs)(*stars)
    g_arr = (wfs_geometry * len(geoms))(*geoms)
    st = lib().wfs_create(C.byref(tel), n_gs, gs_arr, len(geoms), g_arr, C.byref(layers),
                          int(seed) & ((1 << 64) - 1), int(bool(noise_enable)), C.byref(h))
    _check(st)
    return h


def wfs_destroy(h):
    _check(lib().wfs_destroy(h), h)


def wfs_measure(h, screens_ptr, t, slopes_ptr, stream=0):
    _check(lib().wfs_measure(h, screens_ptr, float(t), slopes_ptr, stream), h)


def wfs_measure_stages(h, screens_ptr, t, slopes_ptr, opd=0, intensity=0, expected=0, counts=0,
                       stream=0):
    so = wfs_stage_out(opd or None, intensity or None, expected or None, counts or None)
    _check(lib().wfs_measure_stages(h, screens_ptr, float(t), slopes_ptr, C.byref(so), stream), h)


def wfs_measure_host(h, screens_host_ptr, t, slopes_host_ptr, stream=0):
    _check(lib().wfs_measure_host(h, screens_host_ptr, float(t), slopes_host_ptr, stream), h)


def wfs_host_transfer_bytes(h):
    """(host -> device, device -> host) bytes of the handle's last wfs_measure_host call."""
    a, b = C.c_uint64(), C.c_uint64()
    _check(lib().wfs_host_transfer_bytes(h, C.byref(a), C.byref(b)), h)
    return a.value, b.value


def wfs_set_noise(h, enable):
    _check(lib().wfs_set_noise(h, int(bool(enable))), h)


def wfs_num_valid(h, gs):
    n = C.c_int()
    _check(lib().wfs_num_valid(h, gs, C.byref(n)), h)
    return n.value


def wfs_total_valid(h):
    n = C.c_int()
    _check(lib().wfs_total_valid(h, C.byref(n)), h)
    return n.value


def wfs_valid_map(h, gs):
    n = wfs_num_valid(h, gs)
    out = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().wfs_valid_map(h, gs, out.ctypes.data_as(C.POINTER(C.c_int32))), h)
    return out[:n]


def wfs_layout(h, gs):
    info = wfs_layout_info()
    _check(lib().wfs_layout(h, gs, C.byref(info)), h)
    return info


def wfs_sync_status(h):
    _check(lib().wfs_sync_status(h), h)


def wfs_noise_apply(expected_ptr, n, read_noise, seed, wfs_index, t, pixel0, counts_ptr, stream=0):
    _check(lib().wfs_noise_apply(expected_ptr, int(n), float(read_noise), int(seed), int(wfs_index),
                                 float(t), int(pixel0), counts_ptr, stream))


def wfs_check_bounded_wait(h, polls, stream=0):
    _check(lib().wfs_check_bounded_wait(h, int(polls), stream), h)


def wfs_timing_enable(h, enable):
    _check(lib().wfs_timing_enable(h, int(bool(enable))), h)


def wfs_timing_read(h):
    """{kernel name: (launches, total_ms)} since the last read; resets the totals."""
    arr = (wfs_kernel_time * 64)()
    n = C.c_int()
    _check(lib().wfs_timing_read(h, 64, arr, C.byref(n)), h)
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(min(n.value, 64))}


def wfs_measure_one_static(tel, geom, star, layers, screens_ptr, t, seed, wfs_index, noise,
                           slopes_ptr, slopes_capacity, stream=0):
    """One guide star without device allocation (scratch in the library's static array);
    returns the number of valid subapertures written."""
    nv = C.c_int()
    _check(lib().wfs_measure_one_static(C.byref(tel), C.byref(geom), C.byref(star), C.byref(layers),
                                        screens_ptr, float(t), int(seed), int(wfs_index), int(bool(noise)),
                                        slopes_ptr, int(slopes_capacity), C.byref(nv), stream))
    return nv.value


def wfs_batch_create(handles):
    b = _H()
    arr = (_H * len(handles))(*handles)
    _check(lib().wfs_batch_create(len(handles), arr, C.byref(b)))
    return b


def wfs_batch_measure(b, screens_ptrs, ts, slopes_ptrs, stream=0):
    n = len(ts)
    sp = (C.c_void_p * n)(*screens_ptrs)
    tt = (C.c_double * n)(*[float(t) for t in ts])
    op = (C.c_void_p * n)(*slopes_ptrs)
    _check(lib().wfs_batch_measure(b, sp, tt, op, stream))


def wfs_batch_measure_subset(b, slot, active, screens_ptrs, ts, slopes_ptrs, stream=0):
    n = len(active)
    act = (C.c_int * max(n, 1))(*[int(i) for i in active])
    sp = (C.c_void_p * max(n, 1))(*screens_ptrs)
    tt = (C.c_double * max(n, 1))(*[float(t) for t in ts])
    op = (C.c_void_p * max(n, 1))(*slopes_ptrs)
    _check(lib().wfs_batch_measure_subset(b, int(slot), n, act, sp, tt, op, stream))


def wfs_batch_tune(b, screens_ptrs, ts, slopes_ptrs, stream=0):
    n = len(ts)
    sp = (C.c_void_p * n)(*screens_ptrs)
    tt = (C.c_double * n)(*[float(t) for t in ts])
    op = (C.c_void_p * n)(*slopes_ptrs)
    _check(lib().wfs_batch_tune(b, sp, tt, op, stream))


def wfs_batch_info(b):
    arr = (wfs_batch_class * 64)()
    n = C.c_int()
    _check(lib().wfs_batch_info(b, 64, arr, C.byref(n)))
    return [dict((f, getattr(arr[i], f)) for f, _ in wfs_batch_class._fields_) for i in range(min(n.value, 64))]


def wfs_batch_destroy(b):
    _check(lib().wfs_batch_destroy(b))


def wfs_loop_create(h, dms, cm_ptr, gain_ptr):
    """dms: wfs_dm structs (m2a device addresses set); returns the loop handle."""
    lp = _H()
    arr = (wfs_dm * len(dms))(*dms)
    _check(lib().wfs_loop_create(h, len(dms), arr, cm_ptr, gain_ptr, C.byref(lp)), h)
    return lp


def wfs_loop_step(lp, h, screens_ptr, t, slopes_ptr, stream=0):
    _check(lib().wfs_loop_step(lp, screens_ptr, float(t), slopes_ptr, stream), h)


def wfs_loop_set_coeffs(lp, h, coeffs_ptr, stream=0):
    _check(lib().wfs_loop_set_coeffs(lp, coeffs_ptr or None, stream), h)


def wfs_loop_get_coeffs(lp, h, out_ptr, stream=0):
    _check(lib().wfs_loop_get_coeffs(lp, out_ptr, stream), h)


def wfs_loop_get_layer(lp, h, d, out_ptr, stream=0):
    _check(lib().wfs_loop_get_layer(lp, int(d), out_ptr, stream), h)


def wfs_loop_calibrate(lp, h, gs, amplitude, im_ptr, stream=0):
    _check(lib().wfs_loop_calibrate(lp, int(gs), float(amplitude), im_ptr, stream), h)


def wfs_set_uplink(h, gs, diameter_m, samples=16):
    _check(lib().wfs_set_uplink(h, int(gs), float(diameter_m), int(samples)), h)


def wfs_set_lgs_model(h, per_slice):
    _check(lib().wfs_set_lgs_model(h, int(bool(per_slice))), h)


def wfs_loop_batch_create(loops):
    b = _H()
    arr = (_H * len(loops))(*loops)
    _check(lib().wfs_loop_batch_create(len(loops), arr, C.byref(b)))
    return b


def wfs_loop_batch_step(b, screens_ptrs, ts, slopes_ptrs, stream=0):
    n = len(ts)
    sp = (C.c_void_p * n)(*screens_ptrs)
    tt = (C.c_double * n)(*[float(t) for t in ts])
    op = (C.c_void_p * n)(*slopes_ptrs)
    _check(lib().wfs_loop_batch_step(b, sp, tt, op, stream))


def wfs_loop_batch_destroy(b):
    _check(lib().wfs_loop_batch_destroy(b))


def wfs_loop_destroy(lp):
    _check(lib().wfs_loop_destroy(lp))


# ------------------------------------------------------------------ config marshalling

class _Keep:
    def __init__(self):
        self.refs = []

    def d(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.refs.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_double))


def marshal(cfg):
    """Config (paper_1408_0698_gb300.inputs.Config) -> ctypes structs + keep-alive."""
    keep = _Keep()
    tel = wfs_telescope(cfg.telescope.diameter_m, cfg.telescope.obstruction)
    geoms = [wfs_geometry(g.n_sub, g.n_pix_sub, g.n_fft, g.n_det, g.valid_fill, g.precision)
             for g in cfg.geometries]
    stars = []
    for s in cfg.stars:
        na = len(s.na_alt_m) if s.is_lgs else 0
        stars.append(wfs_guide_star(
            int(bool(s.is_lgs)), s.theta_x_rad, s.theta_y_rad,
            s.range_m if s.is_lgs else math.inf, s.wavelength_m, s.launch_x_m, s.launch_y_m,
            s.spot_fwhm_rad, s.photons_per_subap, s.read_noise_e, s.geometry_index, na,
            keep.d(s.na_alt_m if na else [0.0]), keep.d(s.na_weight if na else [0.0])))
    L = cfg.layers
    lay = wfs_layers(L.n_layers, L.screen_size, L.screen_dx_m, keep.d(L.alt_m), keep.d(L.wind_vx_mps),
                     keep.d(L.wind_vy_mps), keep.d(L.x0_m), keep.d(L.y0_m))
    return tel, stars, geoms, lay, keep


class Wfs:
    """Convenience owner of one handle built from a Config."""

    def __init__(self, cfg, seed=0, noise=False):
        tel, stars, geoms, lay, keep = marshal(cfg)
        self.cfg = cfg
        self.h = wfs_create(tel, stars, geoms, lay, seed, noise)
        self.n_gs = len(cfg.stars)
        for k, st in enumerate(cfg.stars):
            if st.is_lgs and getattr(st, "uplink_diameter_m", 0.0) > 0:
                wfs_set_uplink(self.h, k, st.uplink_diameter_m, st.uplink_samples)
        per_slice = {bool(getattr(st, "per_slice", False)) for st in cfg.stars if st.is_lgs}
        if len(per_slice) > 1:
            raise ValueError("the LGS model is per handle: set per_slice on all laser guide stars or none")
        if per_slice == {True}:
            wfs_set_lgs_model(self.h, True)
        self.total = wfs_total_valid(self.h)
        self.layouts = [wfs_layout(self.h, w) for w in range(self.n_gs)]

    def close(self):
        if self.h:
            wfs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
