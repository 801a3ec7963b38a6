"""Pins for the oracle's community passes (Algorithm 3 rounds; Section 3.2.1;
Section 4.2.2).  CPU only."""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _worked():
    return json.load(open(os.path.join(GOLD, "worked_example.json")))


def test_worked_example_by_hand():
    g = _worked()
    e = np.array(g["edges"], np.int32)
    d = np.array(g["degrees"], np.uint32)
    assert np.array_equal(oracle.exact_degrees(e, g["n"]), d)
    for case in g["communities"]:
        for p, want in enumerate(case["labels_after_pass"], start=1):
            lab, deg = oracle.communities(e, g["n"], d, p, case["threshold"], case["growth"], case["tie_mode"])
            assert lab.tolist() == want, (case, p)
            if p == 1:
                assert deg.tolist() == case["degrees_after_pass1"]


def test_zero_passes_is_identity():
    e = graphgen.random_graph(30, 80, seed=1)
    d = oracle.exact_degrees(e, 30)
    lab, deg = oracle.communities(e, 30, d, 0, 100)
    assert np.array_equal(lab, np.arange(30))
    assert np.array_equal(deg, d)


def test_threshold_below_min_degree_is_identity():
    e = graphgen.random_graph(30, 120, seed=2)
    d = oracle.exact_degrees(e, 30)
    lo = int(d.min())
    assert lo >= 1
    lab, _ = oracle.communities(e, 30, d, 1, lo - 1, growth=1)
    assert np.array_equal(lab, np.arange(30))


@pytest.mark.parametrize("k", [2, 5, 40])
def test_star_collapses_in_one_pass(k):
    e = np.array([[0, j] for j in range(1, k + 1)], np.int32)
    d = oracle.exact_degrees(e, k + 1)
    lab, deg = oracle.communities(e, k + 1, d, 1, k)
    assert np.all(lab == 0)
    assert deg[0] == k and np.all(deg[1:] == 2)


def _naive(edges, n, dhat, passes, D, growth, tie_mode):
    """Independent restatement, node-centric: in each round every node looks
    for the first edge (in index order) that would move it, using only the
    labels and degrees from the start of the round."""
    c = list(range(n))
    d = [int(x) for x in dhat]
    for _ in range(passes):
        new_c, new_d = list(c), list(d)
        for w in range(n):
            for (u, v) in edges:
                if u == v or w not in (u, v):
                    continue
                if d[u] > D or d[v] > D or c[u] == c[v]:
                    continue
                other = v if w == u else u
                if d[other] > d[w] or (tie_mode == 1 and d[other] == d[w] and w < other):
                    new_c[w] = c[other]
                    new_d[w] = min(d[w] + 1, 2**32 - 1)
                    break
        c, d = new_c, new_d
        D = min(D * growth, 2**32 - 1)
    return c, d


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 13))
    m = int(rng.integers(1, n * (n - 1) // 2 + 1))
    e = graphgen.random_graph(n, m, seed=seed, self_loops=int(seed % 3))
    tie = seed % 2
    if seed % 3 == 0:
        dh = oracle.exact_degrees(e, n)
    else:
        _, dh = oracle.sketch_degrees(e, n, 2, 5, seed)
    D = int(rng.integers(1, 8))
    P = int(rng.integers(1, 4))
    lab, deg = oracle.communities(e, n, dh, P, D, 2, tie)
    c, d = _naive([tuple(x) for x in e.tolist()], n, dh, P, D, 2, tie)
    assert lab.tolist() == c
    assert deg.tolist() == d


def test_labels_come_from_neighbours_with_higher_rank():
    # After one round every node holds its own label or the start-of-round
    # label of a neighbour whose degree was >= its own.
    e = graphgen.random_graph(200, 900, seed=8)
    d = oracle.exact_degrees(e, 200)
    lab, _ = oracle.communities(e, 200, d, 1, 64, 2, 1)
    nb = [set() for _ in range(200)]
    for u, v in e.tolist():
        nb[u].add(v)
        nb[v].add(u)
    for v in range(200):
        if lab[v] != v:
            assert lab[v] in nb[v]
            assert d[lab[v]] >= d[v]


def _purity(lab, memb):
    tot = 0
    for c in np.unique(lab):
        tot += np.bincount(memb[lab == c]).max()
    return tot / lab.shape[0]


def test_planted_partition_quality_config_graph():
    # Quality floors, not identities: the streamed communities of the
    # 16-community planted partition beat a size-matched random relabelling.
    n, e, memb = graphgen.load("sbm16")
    _, dh = oracle.sketch_degrees(e, n, 4, 4096, 1)
    lab, _ = oracle.communities(e, n, dh, 3, 64, 2, 0)
    rng = np.random.default_rng(0)
    null_p, null_q = [], []
    for _ in range(5):
        r = rng.permutation(lab)
        null_p.append(_purity(r, memb))
        null_q.append(oracle.modularity(e, n, r))
    assert _purity(lab, memb) > 2 * np.mean(null_p)
    q = oracle.modularity(e, n, lab)
    assert q > np.mean(null_q) + 5 * max(np.std(null_q), 1e-3)


def test_strongly_separated_partition():
    e, memb = graphgen.planted_partition([200] * 8, 0.2, 0.001, seed=5)
    d = oracle.exact_degrees(e, 1600)
    lab, _ = oracle.communities(e, 1600, d, 3, 60, 2, 0)
    assert _purity(lab, memb) >= 0.9
    assert len(np.unique(lab)) < 1600 // 2


# ------------------------------------------------------------- variants
# Section 4.2.2: the mode degree as threshold, the delta^i schedule; pointer
# jumping between rounds; the sequential SCoDA of Section 3.2 for comparison.

def test_mode_degree_small_cases():
    assert oracle.mode_degree(np.array([0, 3, 3, 2, 2, 5, 0], np.uint32)) == 2  # tie -> smaller
    assert oracle.mode_degree(np.array([0, 0, 0], np.uint32)) == 0
    assert oracle.mode_degree(np.array([7], np.uint32)) == 7
    assert oracle.mode_degree(np.array([4, 9, 9, 0, 0, 0, 4, 9], np.uint32)) == 9  # zeros do not count


@pytest.mark.parametrize("seed", range(4))
def test_mode_degree_matches_bincount(seed):
    rng = np.random.default_rng(seed)
    d = rng.integers(0, 40, 5000).astype(np.uint32)
    counts = np.bincount(d[d >= 1])
    assert oracle.mode_degree(d) == int(np.argmax(counts))  # argmax takes the first, i.e. smallest, maximum


def test_pointer_jumping_chain_by_hand():
    # Path 0-1-2-3 with degrees 1, 2, 3, 4 and a large threshold: in one
    # round 0 takes 1's label, 1 takes 2's, 2 takes 3's (labels 1, 2, 3, 3).
    # One jump: every label becomes its label's label (2, 3, 3, 3); two: all 3.
    e = np.array([[0, 1], [1, 2], [2, 3]], np.int32)
    dh = np.array([1, 2, 3, 4], np.uint32)
    for jumps, want in [(0, [1, 2, 3, 3]), (1, [2, 3, 3, 3]), (2, [3, 3, 3, 3]), (5, [3, 3, 3, 3])]:
        lab, deg = oracle.communities_ex(e, 4, dh, 1, 100, 2, 0, jumps)
        assert lab.tolist() == want
        assert deg.tolist() == [2, 3, 4, 4]


def _naive_ex(edges, n, dhat, passes, D, growth, tie_mode, jumps):
    factor = growth if growth else D
    c = list(range(n))
    d = [int(x) for x in dhat]
    for _ in range(passes):
        new_c, new_d = list(c), list(d)
        for w in range(n):
            for (u, v) in edges:
                if u == v or w not in (u, v):
                    continue
                if d[u] > D or d[v] > D or c[u] == c[v]:
                    continue
                other = v if w == u else u
                if d[other] > d[w] or (tie_mode == 1 and d[other] == d[w] and w < other):
                    new_c[w] = c[other]
                    new_d[w] = min(d[w] + 1, 2**32 - 1)
                    break
        c, d = new_c, new_d
        for _ in range(jumps):
            c = [c[c[v]] for v in range(n)]
        D = min(D * factor, 2**32 - 1)
    return c, d


@pytest.mark.parametrize("seed", range(10))
def test_variants_brute_force_tiny_graphs(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 13))
    m = int(rng.integers(1, n * (n - 1) // 2 + 1))
    e = graphgen.random_graph(n, m, seed=seed, self_loops=int(seed % 2))
    dh = oracle.exact_degrees(e, n) if seed % 2 else oracle.sketch_degrees(e, n, 2, 5, seed)[1]
    D = int(rng.integers(1, 6))
    growth = int(seed % 3)  # 0 = delta^i
    jumps = int(seed % 4)
    lab, deg = oracle.communities_ex(e, n, dh, 3, D, growth, seed % 2, jumps)
    c, d = _naive_ex([tuple(x) for x in e.tolist()], n, dh, 3, D, growth, seed % 2, jumps)
    assert lab.tolist() == c
    assert deg.tolist() == d


def test_power_schedule_is_growth_by_first_threshold():
    n, e, _ = graphgen.load("sbm16")
    _, dh = oracle.sketch_degrees(e, n, 4, 4096, 1)
    a = oracle.communities_ex(e, n, dh, 3, 9, 0, 0, 0)
    b = oracle.communities_ex(e, n, dh, 3, 9, 9, 0, 0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = oracle.communities(e, n, dh, 3, 9, 9, 0)
    assert np.array_equal(a[0], c[0])


def test_sequential_scoda_by_hand():
    # Two triangles and a bridge, edges in this order, D = 2:
    # (0,1): d=1,1 -> 0 joins 1; (0,2): d0=2,d2=1 -> 2 joins 0 (label 1);
    # (1,2): d=2,2 -> 1 joins 2 (label 1); (3,4): 3 joins 4; (3,5): 5 joins 3
    # (label 4); (4,5): 4 joins 5 (label 4); (2,3): d=3,3 > D, skipped.
    e = np.array([[0, 1], [0, 2], [1, 2], [3, 4], [3, 5], [4, 5], [2, 3]], np.int32)
    assert oracle.scoda_sequential(e, 6, 2).tolist() == [1, 1, 1, 4, 4, 4]


def test_sequential_scoda_finds_disjoint_cliques():
    # Two disjoint 6-cliques in random edge order: one community each.
    rng = np.random.default_rng(3)
    e = np.array([(a, b) for a in range(6) for b in range(a + 1, 6)] +
                 [(a, b) for a in range(6, 12) for b in range(a + 1, 12)], np.int32)
    e = e[rng.permutation(e.shape[0])]
    lab = oracle.scoda_sequential(e, 12, 5)
    assert len(set(lab[:6].tolist())) == 1 and len(set(lab[6:].tolist())) == 1 and lab[0] != lab[6]


def test_rounds_against_sequential_scoda_quality():
    # Quality, not identity (the methods differ): on the 16-community planted
    # partition both find structure; pointer jumping merges chains and
    # raises the modularity of the synchronous rounds.
    n, e, _ = graphgen.load("sbm16")
    _, dh = oracle.sketch_degrees(e, n, 4, 4096, 1)
    q_rounds = oracle.modularity(e, n, oracle.communities(e, n, dh, 3, 64, 2, 0)[0])
    q_jumps = oracle.modularity(e, n, oracle.communities_ex(e, n, dh, 3, 64, 2, 0, 4)[0])
    q_seq = oracle.modularity(e, n, oracle.scoda_sequential(e, n, oracle.mode_degree(oracle.exact_degrees(e, n))))
    assert 0.05 < q_rounds < q_jumps < q_seq < 0.7
