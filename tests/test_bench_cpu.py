"""The benchmark's own arithmetic, on the CPU: the algorithmic flop count behind the roofline,
the FP32 peak it divides by, and the traffic table keyed by kernel source hashes."""
import math
import os

import bench


def test_spot_flop_model():
    # 32-point LGS subaperture (n = 10, N = 32, 16 x 16 detector pixels), term by term
    n, N, nd = 10, 32, 16
    # Q = G^T M as a folded 16-point DFT: 3 folded rows x 10 columns (2 flops each), then per
    # column 8 butterflies of 4 flops (first stage) and 3 x 8 of 10 flops
    q = 2 * 3 * n + n * (8 * 4 + 3 * 8 * 10)
    assert q == bench.q_dft_flops(n, nd) == 2780
    terms = (8 * N * n * (n + N), 3 * N * N, 4 * N * N * n, 10 * int(math.log2(N)) * N * n,
             12 * (2 * n - 1) * n, q, 4 * nd * nd * n, 2 * nd * nd)
    assert sum(terms) == 183364 == bench.spot_flops(n, N, nd, True)
    # the dense form of Q (8 (2n-1) n nd flops) is 8.7 times the DFT's count
    assert 8 * (2 * n - 1) * n * nd == 24320
    # n = 8 on the 32-point grid: 15 rows, none folded
    assert bench.q_dft_flops(8, 16) == 8 * (8 * 4 + 3 * 8 * 10)
    # the DFT term alone is the useful DFT work of a subaperture, 8 N n (n + N)
    assert terms[0] == 107520
    # NGS (no elongation): DFT, |.|^2, binning, photometry and centroid
    n, N, nd = 32, 64, 32
    assert bench.spot_flops(n, N, nd, False) == 8 * N * n * (n + N) + 3 * N * N + N * N + 6 * nd * nd


def test_fp32_peak_from_unit_counts():
    assert abs(bench.FP32_PEAK_TFLOPS - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert 80.0 < bench.FP32_PEAK_TFLOPS < 81.0


def test_traffic_table_entries():
    """The traffic table parses; an entry whose kernel sources changed since the capture reads as
    None (the bench then reports null).  Where the spot kernel's entry is current, its DRAM bytes
    are its algorithmic reads (elongation tables + OPD) plus the expected images it writes."""
    lines = [l.split() for l in open(os.path.join(bench.ROOT, "profiles", "traffic.txt"))
             if l.strip() and not l.startswith("#")]
    assert lines and all(len(l) == 3 and l[0] in bench.KERNEL_SOURCES and int(l[1]) > 0 for l in lines)
    v = bench.ncu_traffic("spot_tc")
    if v is not None:
        lgs = 6 * 4632
        alg = lgs * (19 * 10 * 8 + 100 * 4)
        assert 0.95 < (v - 2.3e6) / alg < 1.05


def test_cuda_core_and_tensor_split():
    """The roofline's split of a 32-point LGS subaperture.  The tensor-core kernel computes U = F X
    with the rows k and k + 16 paired (4 N n^2 + 2 N n = 13,440 flops for the dense 25,600) and
    Y = U F^T and Ta = I Ga^T as MMAs, so the CUDA cores keep 171,204 - 81,920 - 40,960 = 48,324
    flops; with U = F X as an MMA too (dense), 34,884.  The FP32 kernel pairs U and takes Y and Ta
    by column quadruples: 89,796 flops on the CUDA cores.  The tensor figure divides the useful DFT
    flops, 8 N n (n + N) = 107,520, the dense definition."""
    n, N, nd = 10, 32, 16
    assert bench.dft_forms("spot_tc_bf16x3_N32", N) == {"U": "r2", "Y": "dense", "Ta": "dense"}
    assert bench.dft_forms("spot_tc_bf16x3_N64", 64) == {"U": "dense", "Y": "dense", "Ta": "dense"}
    assert bench.dft_forms("spot_n32_fp32_N32", N) == {"U": "r2", "Y": "r4", "Ta": "r4"}
    dense = bench.spot_flops(n, N, nd, True)
    u2 = 4 * N * n * n + 2 * N * n
    assert u2 == 13440
    on_tc = lambda name: sum(bench.TC_STAGES[s][0](n, N, nd) for s in bench.tc_stages(name))
    tc = bench.spot_flops(n, N, nd, True, "spot_tc_bf16x3_N32")
    assert tc == dense - 8 * N * n * n + u2 == 171204
    assert tc - on_tc("spot_tc_bf16x3_N32") == 48324
    assert bench.spot_flops(n, N, nd, True, "spot_tcu_bf16x3_N32") - on_tc("spot_tcu_bf16x3_N32") == 34884
    # Y by quadruples: per lane 8 column groups x (10 complex MACs + a 4-point DFT of 8 complex adds)
    y4 = 32 * 8 * (10 * 8 + 8 * 2)
    assert y4 == 2 * N * N * n + 4 * N * N == 24576
    # Ta by quadruples: per lane 8 groups x (6 adds + 5 even d x 4 flops + 5 odd d x 8 flops)
    ta4 = 32 * 8 * (6 + 5 * 4 + 5 * 8)
    assert ta4 == 16896
    fp = bench.spot_flops(n, N, nd, True, "spot_n32_fp32_N32")
    assert fp == dense - (8 * N * n * n - u2) - (8 * N * N * n - y4) - (4 * N * N * n - ta4) == 89796
    assert on_tc("spot_n32_fp32_N32") == 0
    assert bench.dft_useful_flops(n, N) == 107520
    # issued BF16 flops per subaperture of the two original MMA chains: 32 rows x (64 x 64 + 2 x 32 x 64)
    iss = sum(bench.TC_STAGES[s][1](n, N, nd) for s in bench.tc_stages("spot_tc_bf16x3_N32"))
    assert iss == 2 * 32 * (64 * 64 + 2 * 32 * 64)


def test_projection_footprint_bytes():
    """Algorithmic bytes of the projection: one on-axis NGS through one ground layer at integer
    offsets touches the pupil's pixels plus one more row and column (the bilinear taps), once;
    two stars through the same ground layer at the same position count the screen once."""
    import dataclasses

    import numpy as np

    import oracle
    from paper_1408_0698_gb300 import inputs

    cfg = inputs.config1()
    g = cfg.geometries[0]
    idx, _ = oracle.valid_subaps(cfg.telescope.diameter_m, cfg.telescope.obstruction, g.n_sub, g.n_pix_sub)
    # 16-point geometry: make it the 32-point group the function measures
    cfg.geometries[0] = dataclasses.replace(g, n_fft=32, n_det=16)
    cfg.layers = dataclasses.replace(cfg.layers, wind_vx_mps=np.zeros(1), wind_vy_mps=np.zeros(1),
                                     x0_m=np.zeros(1), y0_m=np.zeros(1))
    tot, scr, opd = bench.projection_footprint_bytes(cfg, [idx], 0.0)
    n_pix = len(idx) * g.n_pix_sub ** 2
    assert opd == 4 * n_pix
    # pupil pixel centres sit at half-pixel screen coordinates: each touches a 2 x 2 block, and the
    # union over a subaperture of n x n pixels is (n + 1)^2 screen pixels less the shared edges
    assert n_pix < scr / 4 < 1.5 * n_pix
    cfg.stars = [cfg.stars[0], dataclasses.replace(cfg.stars[0])]
    tot2, scr2, opd2 = bench.projection_footprint_bytes(cfg, [idx, idx], 0.0)
    assert scr2 == scr and opd2 == 2 * opd
