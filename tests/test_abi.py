"""Host-side checks of the C ABI: the library loads, exports every declared symbol, and
rejects bad descriptions synchronously, before any device work."""
import ctypes as C
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1408_0698_gb300 import inputs, native


def test_library_exports_every_header_symbol():
    L = native.lib()
    names = native.header_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(native._SIGS), "binding and header disagree"
    assert "sm_103a" in native.wfs_version()


def test_binding_argument_counts_match_the_header():
    """Every prototype in include/gbwfs.h has as many parameters as its ctypes signature, and
    pointer parameters sit where the binding passes pointers."""
    import re
    text = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                             "gbwfs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = dict(re.findall(r"\b(wfs_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", text))
    assert set(protos) == set(native._SIGS)
    for name, params in protos.items():
        params = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        argtypes = native._SIGS[name][1]
        assert len(params) == len(argtypes), (name, params, argtypes)
        for p, a in zip(params, argtypes):
            is_ptr = "*" in p or p.startswith("wfs_handle") or p.startswith("wfs_loop") or p.startswith("wfs_batch")
            a_ptr = issubclass(a, (C._Pointer, C.Array, C.c_void_p, C.c_char_p))
            assert is_ptr == a_ptr, (name, p, a)


def test_checked_library_exports_the_same_symbols():
    """The bounds-checked build (-DGBWFS_CHECK) compiles from the same sources and exports the
    same entry points; it names itself in the version string."""
    code = ("from paper_1408_0698_gb300 import native; L = native.lib(); "
            "names = native.header_symbols(); "
            "assert all(hasattr(L, n) for n in names); "
            "assert L._name.endswith('libgbwfs_check.so'); print(native.wfs_version())")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900,
                       env=dict(os.environ, GBWFS_CHECKED="1"),
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0, r.stderr[-2000:]
    assert "bounds-checked" in r.stdout


def _create(cfg, **kw):
    tel, stars, geoms, lay, keep = native.marshal(cfg)
    for k, v in kw.items():
        obj, field, val = v
        setattr({"tel": tel, "lay": lay, "g0": geoms[0], "s0": stars[0]}[obj], field, val)
    h = native._H()
    st = native.lib().wfs_create(C.byref(tel), len(stars), (native.wfs_guide_star * len(stars))(*stars),
                                 len(geoms), (native.wfs_geometry * len(geoms))(*geoms), C.byref(lay),
                                 0, 0, C.byref(h))
    return st, h


@pytest.mark.parametrize("edit,expect", [
    (("tel", "diameter_m", -1.0), native.WFS_EINVAL),
    (("tel", "obstruction", 1.0), native.WFS_EINVAL),
    (("g0", "n_pix_sub", 40), native.WFS_EINVAL),
    (("g0", "n_fft", 4), native.WFS_EINVAL),
    (("g0", "n_det", 7), native.WFS_EINVAL),
    (("g0", "n_fft", 128), native.WFS_EINVAL),
    (("g0", "valid_fill", 0.0), native.WFS_EINVAL),
    (("g0", "precision", 9), native.WFS_EINVAL),
    (("s0", "wavelength_m", 0.0), native.WFS_EINVAL),
    (("s0", "geometry_index", 3), native.WFS_EINVAL),
    (("s0", "spot_fwhm_rad", 0.0), native.WFS_EINVAL),
    (("s0", "range_m", math.inf), native.WFS_EINVAL),
    (("s0", "n_na", 0), native.WFS_EINVAL),
    (("lay", "n_layers", 0), native.WFS_EINVAL),
    (("lay", "screen_size", 64), native.WFS_EINVAL),   # footprint larger than the screen
    (("lay", "screen_dx_m", math.nan), native.WFS_EINVAL),
])
def test_bad_descriptions_rejected(edit, expect):
    cfg = inputs.config2()
    st, h = _create(cfg, e=edit)
    assert st == expect
    assert not h.value
    assert native.wfs_last_error(None)


def test_lgs_needs_band_limited_dft():
    cfg = inputs.config2()
    st, _ = _create(cfg, e1=("g0", "n_fft", 10), e2=("g0", "n_det", 5))   # 10 < 2*6-1
    assert st == native.WFS_EUNSUPPORTED


def test_null_arguments():
    L = native.lib()
    assert L.wfs_measure(None, None, 0.0, None, None) == native.WFS_EINVAL
    assert L.wfs_destroy(None) == native.WFS_EINVAL
    assert L.wfs_create(None, 1, None, 1, None, None, 0, 0, None) == native.WFS_EINVAL
    assert L.wfs_noise_apply(None, 10, 1.0, 0, 0, 0.0, 0, None, None) == native.WFS_EINVAL
    n = C.c_int()
    assert L.wfs_num_valid(None, 0, C.byref(n)) == native.WFS_EINVAL
    lp = native._H()
    assert L.wfs_loop_create(None, 1, None, None, None, C.byref(lp)) == native.WFS_EINVAL
    assert L.wfs_loop_create(None, 1, None, None, None, None) == native.WFS_EINVAL
    assert L.wfs_loop_step(None, None, 0.0, None, None) == native.WFS_EINVAL
    assert L.wfs_loop_set_coeffs(None, None, None) == native.WFS_EINVAL
    assert L.wfs_loop_get_coeffs(None, None, None) == native.WFS_EINVAL
    assert L.wfs_loop_get_layer(None, 0, None, None) == native.WFS_EINVAL
    assert L.wfs_loop_destroy(None) == native.WFS_EINVAL
    assert L.wfs_loop_calibrate(None, 0, 1.0, None, None) == native.WFS_EINVAL
    b = native._H()
    assert L.wfs_loop_batch_create(0, None, C.byref(b)) == native.WFS_EINVAL
    assert L.wfs_loop_batch_create(1, None, None) == native.WFS_EINVAL
    assert L.wfs_loop_batch_step(None, None, None, None, None) == native.WFS_EINVAL
    assert L.wfs_loop_batch_destroy(None) == native.WFS_EINVAL
    assert L.wfs_set_uplink(None, 0, 0.5, 16) == native.WFS_EINVAL
    assert L.wfs_set_lgs_model(None, 1) == native.WFS_EINVAL
    u = C.c_uint64()
    assert L.wfs_host_transfer_bytes(None, C.byref(u), C.byref(u)) == native.WFS_EINVAL


def test_no_silent_cpu_path_without_gpu():
    """On a machine without a GPU a valid description fails with a CUDA error: the library
    has no host fallback."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    st, h = _create(inputs.config1())
    assert st in (native.WFS_ECUDA, native.WFS_ENOMEM)
    assert not h.value


def test_c_example_builds_and_reports_errors(tmp_path):
    """The plain-C99 example compiles with gcc -Wall -Werror against the header and the library;
    without a GPU it stops at wfs_create with the library's CUDA error status and message."""
    torch = pytest.importorskip("torch")
    from _c_example import compile_example
    exe = compile_example(str(tmp_path / "measure_frame"))
    if torch.cuda.is_available():
        pytest.skip("GPU present: tests/test_c_example_gpu.py runs it")
    np.zeros(256 * 256, np.float32).tofile(tmp_path / "s.f32")
    r = subprocess.run([exe, str(tmp_path / "s.f32"), "0.0", str(tmp_path / "o.f32")], capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 1
    assert "wfs_create: status %d" % native.WFS_ECUDA in r.stderr



def test_product_and_oracle_share_no_code():
    """The library's sources include nothing from oracle/ and the oracle nothing from the
    package; the package's Python modules do not import the oracle (only tests/, the smoke entry
    point and bench.py's CPU legs may)."""
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_1408_0698_gb300")
    csrc = os.path.join(pkg, "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in " ".join(re.findall(r'#include\s*[<"]([^>"]+)[>"]', text)), f
    for f in os.listdir(os.path.join(root, "oracle")):
        if f.endswith((".c", ".h")):
            incs = re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(os.path.join(root, "oracle", f)).read())
            assert not any("gbwfs" in i or "csrc" in i or "paper_1408" in i for i in incs), (f, incs)
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            text = open(os.path.join(pkg, f)).read()
            assert not re.search(r"^\s*(import oracle|from oracle)", text, flags=re.M), f


@pytest.mark.parametrize("edit", ["alt_nan", "weights_zero", "n_sub_huge", "launch_inf", "theta_nan"])
def test_static_entry_checks_descriptions_like_create(edit):
    """wfs_measure_one_static applies wfs_create's checks before any device work: descriptions
    that wfs_create rejects are rejected here too (no GPU is needed to see it)."""
    cfg = inputs.config2()
    tel, stars, geoms, lay, keep = native.marshal(cfg)
    s0, g0 = stars[0], geoms[stars[0].geometry_index]
    if edit == "alt_nan":
        lay.alt_m[1] = float("nan")
    elif edit == "weights_zero":
        for k in range(s0.n_na):
            s0.na_weight[k] = 0.0
    elif edit == "n_sub_huge":
        g0.n_sub = 5000
    elif edit == "launch_inf":
        s0.launch_x_m = float("inf")
    else:
        s0.theta_x_rad = float("nan")
    nv = C.c_int(-1)
    st = native.lib().wfs_measure_one_static(C.byref(tel), C.byref(g0), C.byref(s0), C.byref(lay), C.c_void_p(16),
                                             0.0, 1, 0, 0, C.c_void_p(16), 10, C.byref(nv), None)
    assert st == native.WFS_EINVAL
    assert nv.value == 0
