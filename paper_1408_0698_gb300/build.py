"""Builds libgbwfs.so in-tree with nvcc for sm_103a (one -gencode, parallel TUs)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libgbwfs.so")
# The bounds-checked build (-DGBWFS_CHECK): kernels test their global indices, record WFS_EBOUNDS
# and skip an out-of-range access; a debugging stand-in for a memory checker.
CHECK_BUILD = os.path.join(BUILD, "check")
CHECK_SO = os.path.join(CHECK_BUILD, "libgbwfs_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    out = [os.path.join(ROOT, "include", "gbwfs.h")]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC)
            if f.endswith((".cu", ".cuh", ".h"))]
    return out


def up_to_date(so: str = SO) -> bool:
    if not os.path.exists(so):
        return False
    t = os.path.getmtime(so)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra: list | None = None, check: bool = False) -> str:
    """Compiles the library (check=True: the bounds-checked build, in its own folder)."""
    out_dir, so = (CHECK_BUILD, CHECK_SO) if check else (BUILD, SO)
    if not force and up_to_date(so):
        return so
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I", os.path.join(ROOT, "include")] + (["-DGBWFS_CHECK"] if check else []) + (extra or [])
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        cmd = [cc, "-c", src, "-o", obj] + common
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(compile_one, sources()))
    if verbose:
        for _, log in results:
            print(log)
    tmp = so + f".{os.getpid()}.tmp"
    cmd = [cc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + [
        "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
