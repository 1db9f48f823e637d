"""Writes the oracle regression fixtures in this folder.

Calls only the oracle and the seeded input generator; run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1408_0698_gb300 import inputs  # noqa: E402


def main():
    cfg = inputs.config1()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    s = oracle.measure_wfs(cfg, scr, 0, 0.003)["slopes"]
    np.savetxt(os.path.join(HERE, "config1_t0.003_slopes.txt"), s, fmt="%.15e",
               header="oracle slopes (det px), config 1, screens seed 1000, t = 0.003 s, noise-free")
    cfg = inputs.config2()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    sel = np.arange(0, 1264, 97)
    s = oracle.measure_wfs(cfg, scr, 1, 0.01, sel=sel)["slopes"]
    np.savetxt(os.path.join(HERE, "config2_lgs1_t0.01_slopes.txt"), np.c_[sel, s], fmt="%.15e",
               header="valid-subap index, oracle slopes (det px), config 2 LGS 1, screens seed 2000, t = 0.01 s")


if __name__ == "__main__":
    main()
