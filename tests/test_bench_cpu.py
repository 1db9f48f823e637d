"""The benchmark's own arithmetic, on the CPU: the algorithmic flop count behind the roofline,
the FP32 peak it divides by, and the traffic table keyed by kernel source hashes."""
import math
import os

import bench


def test_spot_flop_model():
    # 32-point LGS subaperture (n = 10, N = 32, 16 x 16 detector pixels), term by term
    n, N, nd = 10, 32, 16
    terms = (8 * N * n * (n + N), 3 * N * N, 4 * N * N * n, 10 * int(math.log2(N)) * N * n,
             12 * (2 * n - 1) * n, 8 * (2 * n - 1) * n * nd, 4 * nd * nd * n, 2 * nd * nd)
    assert sum(terms) == 204904 == bench.spot_flops(n, N, nd, True)
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
