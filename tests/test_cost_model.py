"""The flop count the bench's roofline rests on, pinned to the figures the paper prints for its
paper-scale problem (tests/golden/paper_flop_count.txt, Section 4 and Eq. (tb))."""
import os

import bench

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_flop_count.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].split()
        if len(line) == 2:
            vals[line[0]] = float(line[1])
    return vals


def test_paper_scale_flop_count():
    g = _golden()
    n, p, m, t = int(g["n"]), int(g["p"]), int(g["m"]), int(g["t"])
    flops = bench.algorithmic_flops(n, p, m * t, form="paper")
    # "approximately 1.1 petaflops" (printed to two digits)
    assert abs(flops / 1e15 - g["petaflops"]) < 0.05
    # "at a rate of 25 GFlops/sec ... about 12 hours"
    hours = flops / (g["rate_gflops"] * 1e9) / 3600
    assert abs(hours - g["hours"]) < 0.5


def test_gemm_form_count():
    # 2(p+1)n per pair: num (2n), the p-1 values of z (2n each) and s (2n, squares precomputed);
    # the paper's count adds the n squares and n products of S_BR per pair: (5 + 2(p-1))n
    for n, p in ((1000, 4), (256, 1), (10_000, 20)):
        assert bench.algorithmic_flops(n, p, 1) == 2 * (p + 1) * n
        assert bench.algorithmic_flops(n, p, 1, "paper") - bench.algorithmic_flops(n, p, 1) == n
