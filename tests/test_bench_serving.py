"""Host side of the benchmark (CPU): the served workload's request trace is
reproducible, the same request index carries the same instance and solve
seed at every arrival rate (so targets computed once serve every rate), the
instances come from a bounded catalog, and the large request lands
mid-trace; the roofline's choice of the memory the rows come from."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_trace_is_reproducible_and_sorted():
    a = bench.serve_requests(50.0, 3.0, 4)
    b = bench.serve_requests(50.0, 3.0, 4)
    assert a == b
    t = [q[0] for q in a]
    assert t == sorted(t) and all(0 <= x < 3.0 for x in t)
    assert 100 <= len(a) <= 200  # Poisson(150)


def test_request_keys_agree_across_rates():
    lo = bench.serve_requests(10.0, 5.0, 4)
    hi = bench.serve_requests(50.0, 5.0, 4)
    # request i: same size, instance and solve seed at every rate
    for (_, n1, i1, s1), (_, n2, i2, s2) in zip(lo, hi):
        assert (n1, i1, s1) == (n2, i2, s2)
    seeds = [q[3] for q in hi]
    assert len(set(seeds)) == len(seeds)


def test_catalog_is_bounded_per_size():
    reqs = bench.serve_requests(50.0, 20.0, 4)
    sizes = bench.SERVE_SIZES
    per = {}
    for _, n, inst, _ in reqs:
        assert n in sizes
        k = sizes.index(n)
        assert 5000 + 16 * k <= inst < 5000 + 16 * k + bench.SERVE_CATALOG
        per.setdefault(n, set()).add(inst)
    assert all(len(v) <= bench.SERVE_CATALOG for v in per.values())
    counts = np.array([sum(1 for q in reqs if q[1] == n) for n in sizes])
    assert counts.min() > 0.5 * counts.mean()  # sizes drawn uniformly


def test_large_request_mid_trace():
    reqs = bench.serve_requests(50.0, 4.0, 4, big=16384)
    big = [q for q in reqs if q[1] == 16384]
    assert len(big) == 1 and big[0][0] == 2.0
    assert [q[0] for q in reqs] == sorted(q[0] for q in reqs)


def test_rows_from_l2():
    L2 = 135_528_448
    assert bench.rows_from_l2(4 * 800 * 800, L2, None, 13e9)          # W fits the L2
    assert not bench.rows_from_l2(673_181_040, L2, None, 96e9)       # too big, no capture
    assert bench.rows_from_l2(673_181_040, L2, 1.5e9, 96e9)          # captured: DRAM 1.6% of rows
    assert not bench.rows_from_l2(673_181_040, L2, 40e9, 96e9)       # rows streamed from HBM
