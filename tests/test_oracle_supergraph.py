"""Pins for the oracle's supergraph build (Section 4.1; Algorithm 3) and
modularity (equation of the "Quantity measure" section).  CPU only."""
import collections
import json
import os

import numpy as np
import pytest

import graphgen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_worked_example_supergraph():
    g = json.load(open(os.path.join(GOLD, "worked_example.json")))
    e = np.array(g["edges"], np.int32)
    d = np.array(g["degrees"], np.uint32)
    for case in g["supergraph"]:
        lab, _ = oracle.communities(e, g["n"], d, case["passes"], 64, 2, case["tie_mode"])
        sg = oracle.supergraph(e, g["n"], lab, d, 4, 4096, 1)
        assert sg["K"] == case["K"]
        assert sg["node_map"].tolist() == case["node_map"]
        got = [[int(a), int(b), int(w)] for a, b, w in zip(sg["src"], sg["dst"], sg["w"])]
        assert got == case["superedges"]
        assert sg["vol"].tolist() == case["vol"]


def _brute(e, n, lab, dh, rows, width, seed):
    labels = sorted(set(lab.tolist()))
    rank = {l: i for i, l in enumerate(labels)}
    cnt = collections.Counter()
    for u, v in e.tolist():
        if lab[u] != lab[v]:
            a, b = rank[lab[u]], rank[lab[v]]
            cnt[(min(a, b), max(a, b))] += 1
    sup = sorted(cnt.items())
    a, b = oracle.hash_coeffs(seed, rows)
    M = np.zeros((rows, width), np.int64)
    for v in range(n):
        for i in range(rows):
            M[i, oracle.hash_value(a[i], b[i], int(lab[v]), width)] += int(dh[v])
    mass = [1 + min(M[i, oracle.hash_value(a[i], b[i], l, width)] for i in range(rows)) for l in labels]
    vol = [int(sum(int(dh[v]) for v in range(n) if lab[v] == l)) for l in labels]
    return labels, [rank[l] for l in lab.tolist()], sup, mass, vol


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_random_labels(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 60))
    e = graphgen.random_graph(n, int(rng.integers(1, 3 * n)), seed=seed, self_loops=seed % 2)
    lab = rng.integers(0, n, n).astype(np.int32)
    lab = lab[lab] if seed % 2 else lab  # some labels not used by themselves
    dh = oracle.exact_degrees(e, n) + rng.integers(0, 3, n).astype(np.uint32)
    rows, width = 3, int(rng.integers(2, 20))
    sg = oracle.supergraph(e, n, lab, dh, rows, width, seed)
    labels, nmap, sup, mass, vol = _brute(e, n, lab, dh, rows, width, seed)
    assert sg["K"] == len(labels)
    assert sg["comm_label"].tolist() == labels
    assert sg["node_map"].tolist() == nmap
    assert [(int(a), int(b)) for a, b in zip(sg["src"], sg["dst"])] == [k for k, _ in sup]
    assert sg["w"].tolist() == [c for _, c in sup]
    assert sg["mass"].tolist() == mass
    assert sg["vol"].tolist() == vol
    assert sg["count"].tolist() == [int(np.sum(lab == l)) for l in labels]


def test_cut_edge_sum_volume_and_csr():
    n, e, _ = graphgen.load("sbm16")
    _, dh = oracle.sketch_degrees(e, n, 4, 4096, 1)
    lab, _ = oracle.communities(e, n, dh, 3, 64, 2, 0)
    sg = oracle.supergraph(e, n, lab, dh, 4, 4096, 1)
    m_cut = int(np.sum(lab[e[:, 0]] != lab[e[:, 1]]))
    assert int(sg["w"].sum()) == m_cut
    assert int(sg["vol"].sum()) == int(dh.astype(np.int64).sum())
    assert np.all(sg["mass"].astype(np.int64) - 1 >= sg["vol"].astype(np.int64))
    assert np.all(sg["src"] < sg["dst"])
    keys = sg["src"].astype(np.int64) * sg["K"] + sg["dst"]
    assert np.all(np.diff(keys) > 0)
    # CSR: both directions of each superedge, rows sorted ascending
    off, adj, cw = sg["csr_off"], sg["csr_adj"], sg["csr_w"]
    assert off[-1] == 2 * sg["Es"]
    wmap = {(int(a), int(b)): int(w) for a, b, w in zip(sg["src"], sg["dst"], sg["w"])}
    for r in range(0, sg["K"], 37):
        row = adj[off[r]:off[r + 1]]
        assert np.all(np.diff(row) > 0)
        for c, w in zip(row.tolist(), cw[off[r]:off[r + 1]].tolist()):
            assert wmap[(min(r, c), max(r, c))] == w


def test_mass_equals_volume_without_collisions():
    e = graphgen.random_graph(30, 100, seed=3)
    dh = oracle.exact_degrees(e, 30)
    lab = (np.arange(30) // 5 * 5).astype(np.int32)
    for seed in range(1, 100):
        a, b = oracle.hash_coeffs(seed, 4)
        if all(len({oracle.hash_value(a[i], b[i], l, 64) for l in range(0, 30, 5)}) == 6 for i in range(4)):
            break
    sg = oracle.supergraph(e, 30, lab, dh, 4, 64, seed)
    assert np.array_equal(sg["mass"].astype(np.int64) - 1, sg["vol"].astype(np.int64))


def test_modularity_two_triangles_closed_form():
    # two disjoint triangles, one community each: Q = 2 * (3/6 - (6/12)^2) = 0.5
    e = np.array([[0, 1], [1, 2], [0, 2], [3, 4], [4, 5], [3, 5]], np.int32)
    assert oracle.modularity(e, 6, np.array([0, 0, 0, 3, 3, 3], np.int32)) == pytest.approx(0.5, abs=1e-15)
    # everything in one community: Q = 1 - 1 = 0
    assert oracle.modularity(e, 6, np.zeros(6, np.int32)) == pytest.approx(0.0, abs=1e-15)
    # every node alone: no edge inside, Q = -sum (d_i / 2m)^2 = -6 * (2/12)^2 = -1/6
    assert oracle.modularity(e, 6, np.arange(6, dtype=np.int32)) == pytest.approx(-1.0 / 6.0, abs=1e-15)


def test_modularity_matches_double_sum():
    e = graphgen.random_graph(25, 60, seed=6)
    lab = np.random.default_rng(1).integers(0, 4, 25).astype(np.int32)
    A = np.zeros((25, 25))
    for u, v in e.tolist():
        A[u, v] += 1
        A[v, u] += 1
    k = A.sum(axis=1)
    m2 = A.sum()
    same = lab[:, None] == lab[None, :]
    q = ((A - np.outer(k, k) / m2) * same).sum() / m2
    assert oracle.modularity(e, 25, lab) == pytest.approx(q, abs=1e-12)


def test_colour_groups_small_example():
    # Section 4.3 by hand: sizes 1,1,2,3,5,8,13 (alpha = 33, half 16.5).
    # Ascending prefix sums 1,2,4,7,12,20 -> the first five (sum 12 <= 16.5)
    # are brown; the rest (8, 13) are split into ten groups: ranks 0 and 1 of
    # R = 2 -> groups 1 + 0 and 1 + 5.
    sizes = np.array([13, 1, 8, 2, 1, 5, 3], np.uint32)
    g = oracle.colour_groups(sizes)
    assert g.tolist() == [6, 0, 1, 0, 0, 0, 0]


def test_colour_groups_properties():
    rng = np.random.default_rng(3)
    sizes = rng.lognormal(3, 1.5, 5000).astype(np.uint32) + 1
    g = oracle.colour_groups(sizes)
    total = int(sizes.astype(np.int64).sum())
    brown = int(sizes[g == 0].astype(np.int64).sum())
    assert 2 * brown <= total
    # adding the smallest non-brown community would pass half of alpha
    assert 2 * (brown + int(sizes[g > 0].min())) > total
    # groups are monotone in size and the ten upper groups have near-equal counts
    for a in range(0, 10):
        if np.any(g == a) and np.any(g == a + 1):
            assert sizes[g == a].max() <= sizes[g == a + 1].min()
    counts = np.bincount(g, minlength=11)[1:]
    assert counts.max() - counts.min() <= 1


# ------------------------------------------------------------------ drawing
# Section 4.1 (radius ~ sqrt of the size) and Section 4.3 (colours).

PALETTE = {0: (177, 89, 40), 1: (202, 178, 214), 2: (106, 61, 154), 3: (253, 191, 111), 4: (255, 127, 0),
           5: (251, 154, 153), 6: (227, 26, 28), 7: (178, 223, 138), 8: (51, 160, 44), 9: (166, 206, 227),
           10: (31, 120, 180)}  # ColorBrewer "Paired": brown, then light/dark purple, orange, red, green, blue


def test_render_single_disc_fills_the_square():
    # One disc: its bounding box is the whole image, so the scaled radius is
    # W/2 and the covered pixels are those whose centres lie in the inscribed
    # circle -- counted here independently in integers: (2px+1-W)^2 +
    # (2py+1-W)^2 <= W^2.
    W = 40
    img = oracle.render([[3.0, -7.0]], [2.5], [4], W, W)
    px, py = np.meshgrid(np.arange(W), np.arange(W))
    inside = (2 * px + 1 - W) ** 2 + (2 * py + 1 - W) ** 2 <= W * W
    assert np.array_equal(np.all(img[..., :3] == PALETTE[4], axis=-1), inside)
    assert np.all(img[~inside][:, :3] == 255) and np.all(img[..., 3] == 255)


def test_render_smaller_disc_on_top_and_palette():
    # A big disc with a small one inside it: the small one wins where they
    # overlap; every group maps to its colour.
    for g in range(11):
        img = oracle.render([[0.0, 0.0], [0.0, 0.0]], [10.0, 2.0], [0, g], 50, 50)
        centre = tuple(img[25, 25, :3])
        assert centre == PALETTE[g]
        assert tuple(img[25, 3, :3]) == PALETTE[0]
        assert tuple(img[0, 0, :3]) == (255, 255, 255)  # corner outside the inscribed circle


def test_render_equal_radii_smaller_index_wins():
    img = oracle.render([[0.0, 0.0], [0.0, 0.0], [5.0, 0.0]], [3.0, 3.0, 1.0], [2, 6, 8], 30, 30)
    assert tuple(img[15, 8, :3]) == PALETTE[2]  # discs 0 and 1 coincide: disc 0 is drawn


def test_render_wide_aspect_uses_one_scale():
    # Discs spread along x: one scale for both axes, set by the wider extent.
    img = oracle.render([[0.0, 0.0], [30.0, 0.0]], [1.0, 1.0], [1, 2], 64, 64)
    # the box is 32 wide and 2 high: scale 2; each disc covers ~pi * 2^2 pixels near y in [0, 4)
    for g in (1, 2):
        cnt = int(np.all(img[..., :3] == PALETTE[g], axis=-1).sum())
        assert 8 <= cnt <= 16
    assert np.all(img[8:, :, :3] == 255)
