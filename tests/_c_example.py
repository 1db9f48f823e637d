"""Builds the plain-C example (paper_1408_0698_gb300/examples/measure_frame.c) with gcc against
include/gbwfs.h, libgbwfs.so and the CUDA runtime."""
import os
import subprocess

from paper_1408_0698_gb300 import build, native

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "paper_1408_0698_gb300", "examples", "measure_frame.c")


def compile_example(out_path):
    native.lib()  # builds libgbwfs.so when stale
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(build.nvcc())))
    libdir = os.path.dirname(build.SO)
    cuda_lib = next((os.path.join(cuda, d) for d in ("lib64", "lib", "targets/sbsa-linux/lib",
                                                     "targets/x86_64-linux/lib")
                     if os.path.exists(os.path.join(cuda, d, "libcudart.so"))), os.path.join(cuda, "lib64"))
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), SRC, "-o", out_path, "-L", libdir, "-lgbwfs", "-L", cuda_lib,
           "-lcudart", "-lm", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out_path
