"""Pins for the oracle's hash family, degrees and count-min sketch
(Algorithm 2; Section 3.3; Section 4.2.1).  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import graphgen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
P31 = 2**31 - 1


def test_splitmix64_published_value():
    g = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    _, out = oracle.splitmix64(g["state"])
    assert out == int(g["first_output_hex"], 16)


def test_hash_coefficients_in_range_and_distinct_rows():
    a, b = oracle.hash_coeffs(12345, 8)
    assert np.all((a >= 1) & (a <= P31 - 1))
    assert np.all(b <= P31 - 1)
    assert len(set(a.tolist())) == 8


def test_hash_values_match_big_integer_arithmetic():
    # 64-bit overflow would show up for large a, x; Python ints are exact.
    a, b = oracle.hash_coeffs(7, 4)
    rng = np.random.default_rng(0)
    for x in list(rng.integers(0, 2**31 - 1, 200)) + [0, 1, 2**31 - 2]:
        for i in range(4):
            for w in (1, 7, 4096, 65536, 100003):
                assert oracle.hash_value(a[i], b[i], int(x), w) == ((int(a[i]) * int(x) + int(b[i])) % P31) % w


def test_exact_degrees_match_bincount():
    e = graphgen.random_graph(50, 300, seed=3, self_loops=5)
    d = oracle.exact_degrees(e, 50)
    ref = np.bincount(e.ravel(), minlength=50)
    assert np.array_equal(d, ref)


@pytest.mark.parametrize("rows,width", [(1, 16), (4, 64), (4, 4096), (3, 1000)])
def test_rows_sum_to_twice_m_and_estimate_never_low(rows, width):
    e = graphgen.random_graph(300, 2000, seed=rows * 1000 + width, self_loops=7)
    S, dh = oracle.sketch_degrees(e, 300, rows, width, seed=11)
    m = e.shape[0]
    assert np.all(S.sum(axis=1, dtype=np.int64) == 2 * m)
    deg = np.bincount(e.ravel(), minlength=300)
    assert np.all(dh >= deg)


def test_collision_free_sketch_is_exact():
    # Find a seed whose rows map the 40 node ids injectively into 4096
    # columns; then every row holds the exact degree and the minimum equals it.
    n = 40
    e = graphgen.random_graph(n, 150, seed=5)
    for seed in range(1, 200):
        a, b = oracle.hash_coeffs(seed, 4)
        ok = all(len({oracle.hash_value(a[i], b[i], v, 4096) for v in range(n)}) == n for i in range(4))
        if ok:
            break
    else:
        pytest.skip("no collision-free seed found")
    S, dh = oracle.sketch_degrees(e, n, 4, 4096, seed)
    assert np.array_equal(dh, np.bincount(e.ravel(), minlength=n))


def test_sketch_equals_node_weighted_construction():
    # Integer addition commutes: adding deg(v) once per node and row gives the
    # same matrix as one increment per edge endpoint (what a GPU may do).
    n = 500
    e = graphgen.random_graph(n, 3000, seed=9, self_loops=3)
    rows, width = 4, 97
    S, dh = oracle.sketch_degrees(e, n, rows, width, seed=21)
    a, b = oracle.hash_coeffs(21, rows)
    deg = np.bincount(e.ravel(), minlength=n)
    ref = np.zeros((rows, width), np.int64)
    for i in range(rows):
        h = np.array([oracle.hash_value(a[i], b[i], v, width) for v in range(n)])
        np.add.at(ref[i], h, deg)
        assert np.array_equal(dh <= ref[i][h], np.ones(n, bool))
    assert np.array_equal(S, ref)
    est = np.min(np.stack([ref[i][[oracle.hash_value(a[i], b[i], v, width) for v in range(n)]]
                           for i in range(rows)]), axis=0)
    assert np.array_equal(dh, est)


def test_cormode_muthukrishnan_bound():
    # Count-min guarantee (Section 4.2.1): P[dhat - deg > e * N / w] <= e^-r,
    # N = 2m events.  Checked empirically on 20k nodes, with slack for sampling.
    n, rows, width = 20000, 3, 512
    e = graphgen.random_graph(n, 60000, seed=4)
    S, dh = oracle.sketch_degrees(e, n, rows, width, seed=99)
    deg = np.bincount(e.ravel(), minlength=n)
    N = 2 * e.shape[0]
    frac = np.mean((dh.astype(np.int64) - deg) > math.e * N / width)
    assert frac <= math.exp(-rows) * 1.5 + 0.005


def test_sketch_rejects_bad_endpoint():
    e = np.array([[0, 1], [1, 5]], np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.sketch_degrees(e, 5, 2, 8, 1)
