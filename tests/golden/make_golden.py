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
    # the per-slice LGS model with the uplink tip-tilt, config 2 LGS 0 (0.5 m beam, 16 samples)
    import dataclasses
    st = dataclasses.replace(cfg.stars[0], per_slice=True, uplink_diameter_m=0.5, uplink_samples=16)
    cfg_sl = dataclasses.replace(cfg, stars=[st] + cfg.stars[1:])
    s = oracle.measure_wfs(cfg_sl, scr, 0, 0.01, sel=sel)["slopes"]
    np.savetxt(os.path.join(HERE, "config2_lgs0_slices_uplink_t0.01_slopes.txt"), np.c_[sel, s], fmt="%.15e",
               header="valid-subap index, oracle slopes (det px), config 2 LGS 0, per-slice model, uplink 0.5 m / 16, "
                      "screens seed 2000, t = 0.01 s")
    # one closed-loop step on config 1 through a 21 x 21 ground mirror with 12 modes
    cfg = inputs.config1()
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    dm = inputs.Dm(21, 0.4, 0.0, 12)
    M = inputs.modal_base(dm, 5, amplitude_m=2e-8).astype(np.float64)
    ns = 2 * len(oracle.measure(cfg, scr, 0.0))
    cm = inputs.random_control_matrix(12, ns, seed=6, scale=0.5).astype(np.float64)
    c0 = np.random.default_rng(7).standard_normal(12)
    _, c1 = oracle.loop_step(cfg, scr, 0.002, [dm], [M], cm, np.full(12, 0.4), c0)
    np.savetxt(os.path.join(HERE, "config1_loop_step_coeffs.txt"), np.c_[c0, c1], fmt="%.15e",
               header="modal coefficients before and after one integrator step (gain 0.4), config 1, mirror 21 x 21 "
                      "at 0.4 m with 12 modes (modal base seed 5), control matrix seed 6, t = 0.002 s")
    im = oracle.interaction_matrix(cfg, 0, [dm], [M], 0.5, modes=[0, 5, 11])
    np.savetxt(os.path.join(HERE, "config1_interaction_rows.txt"), im.T, fmt="%.15e",
               header="push-pull interaction-matrix rows (columns: modes 0, 5, 11; amplitude 0.5), config 1, same mirror")


if __name__ == "__main__":
    main()
