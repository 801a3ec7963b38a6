"""GPU parity of the integer stages against the oracle, element by element,
bit-exact: degree sketch (Algorithm 2), community rounds (Algorithm 3),
supergraph (Section 4.1).  Calls go through the C ABI."""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle
from oracle import FA2Params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import gpu_pipeline as G  # noqa: E402

B = G.B

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _graphs():
    # (name, edges, n): tiny, ragged, odd m, self-loops, several sort tiles
    yield "single-node", np.zeros((0, 2), np.int32), 1
    yield "one-edge", np.array([[0, 1]], np.int32), 2
    yield "self-loops-only", np.array([[0, 0], [1, 1], [1, 1]], np.int32), 3
    yield "random-odd", graphgen.random_graph(97, 333, seed=1, self_loops=4), 97
    yield "random-mid", graphgen.random_graph(5000, 20001, seed=2, self_loops=9), 5000
    yield "random-tiles", graphgen.random_graph(30000, 150003, seed=3), 30000
    n, e, _ = graphgen.load("sbm16")
    yield "sbm16", e, n


GRAPHS = list(_graphs())


@pytest.mark.parametrize("name,e,n", GRAPHS, ids=[g[0] for g in GRAPHS])
@pytest.mark.parametrize("rows,width", [(4, 4096), (1, 7), (3, 1000), (16, 64)])
def test_sketch_bit_exact(name, e, n, rows, width):
    S, d, st = G.sketch(e, n, rows, width, seed=11)
    S0, d0 = oracle.sketch_degrees(e, n, rows, width, 11)
    assert st == 0
    assert np.array_equal(S, S0)
    assert np.array_equal(d, d0)


def test_sketch_flags_bad_edges():
    e = np.array([[0, 1], [2, 9], [1, 2]], np.int32)
    _, _, st = G.sketch(e, 5, 2, 8, 1)
    assert st & G.B.BGV_DEV_BADEDGE
    _, _, st = G.sketch(np.array([[0, -3], [1, 2]], np.int32), 5, 2, 8, 1)
    assert st & G.B.BGV_DEV_BADEDGE


def test_communities_worked_example():
    g = json.load(open(os.path.join(GOLD, "worked_example.json")))
    e = np.array(g["edges"], np.int32)
    d = np.array(g["degrees"], np.uint32)
    for case in g["communities"]:
        for p, want in enumerate(case["labels_after_pass"], start=1):
            lab, deg, st = G.communities(e, g["n"], d, p, case["threshold"], case["growth"], case["tie_mode"])
            assert st == 0 and lab.tolist() == want


@pytest.mark.parametrize("name,e,n", GRAPHS, ids=[g[0] for g in GRAPHS])
@pytest.mark.parametrize("passes,threshold,growth,tie", [(3, 64, 2, 0), (1, 4, 2, 1), (4, 0, 3, 0), (0, 5, 2, 0),
                                                         (2, 1 << 31, 2, 1)])
def test_communities_bit_exact(name, e, n, passes, threshold, growth, tie):
    _, dh = oracle.sketch_degrees(e, n, 4, 256, 3)
    lab, deg, st = G.communities(e, n, dh, passes, threshold, growth, tie)
    D = threshold if threshold else (2 * e.shape[0]) // n
    lab0, deg0 = oracle.communities(e, n, dh, passes, D, growth, tie)
    assert st == 0
    assert np.array_equal(lab, lab0)
    assert np.array_equal(deg, deg0)


def _check_super(sg, sg0):
    assert sg["status"] == 0
    assert sg["K"] == sg0["K"] and sg["Es"] == sg0["Es"]
    for k in ("node_map", "src", "dst", "w", "mass", "vol", "count", "comm_label", "csr_off", "csr_adj", "csr_w"):
        assert np.array_equal(np.asarray(sg[k]).astype(np.int64), np.asarray(sg0[k]).astype(np.int64)), k


@pytest.mark.parametrize("name,e,n", GRAPHS, ids=[g[0] for g in GRAPHS])
def test_supergraph_from_communities_bit_exact(name, e, n):
    _, dh = oracle.sketch_degrees(e, n, 4, 512, 5)
    lab, _ = oracle.communities(e, n, dh, 3, 32, 2, 1)
    sg = G.supergraph(e, n, lab, dh, 4, 512, 5)
    _check_super(sg, oracle.supergraph(e, n, lab, dh, 4, 512, 5))


@pytest.mark.parametrize("seed", range(4))
def test_supergraph_random_labels_bit_exact(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(50, 40000))
    e = graphgen.random_graph(n, int(rng.integers(1, 6 * n)), seed=seed, self_loops=seed)
    k = int(rng.integers(1, n + 1))
    lab = rng.choice(n, size=k, replace=False)[rng.integers(0, k, n)].astype(np.int32)
    dh = oracle.exact_degrees(e, n) + rng.integers(0, 100, n).astype(np.uint32)
    sg = G.supergraph(e, n, lab, dh, 3, 97, seed)
    _check_super(sg, oracle.supergraph(e, n, lab, dh, 3, 97, seed))


def _shape_cases():
    # Supergraph shapes beyond the random graphs: one row of 20,000 distinct
    # columns, three supernodes joined by runs of tens of thousands of one
    # repeated pair, a dense cluster whose row holds few cut pairs among many
    # intra-community edges, 200,000 mostly empty rows, and ids that need 24
    # bits (keys of 48 bits).
    n = 30000
    star = np.stack([np.zeros(20000, np.int32), np.arange(1, 20001, dtype=np.int32)], 1)
    e = np.concatenate([star, graphgen.random_graph(n, 40000, seed=12)]).astype(np.int32)
    yield "star-20k", e, n, np.arange(n, dtype=np.int32)
    e = graphgen.random_graph(n, 150000, seed=13)
    lab = (np.random.default_rng(13).integers(0, 3, n) * 7).astype(np.int32)
    yield "three-communities", e, n, lab
    iu = np.triu_indices(200, 1)
    clique = np.stack([iu[0], iu[1]], 1).astype(np.int32)
    e = np.concatenate([clique, graphgen.random_graph(n, 60000, seed=14)]).astype(np.int32)
    lab = np.arange(n, dtype=np.int32)
    lab[:200] = 0
    yield "dense-cluster", e, n, lab
    n = 200000
    yield "sparse-rows", graphgen.random_graph(n, 30000, seed=15), n, np.arange(n, dtype=np.int32)
    n = (1 << 23) + 5
    e = graphgen.random_graph(n, 100000, seed=16)
    yield "24-bit-ids", e, n, (np.arange(n, dtype=np.int64) // 3 * 3).astype(np.int32)


SHAPE_CASES = list(_shape_cases())


@pytest.mark.parametrize("name,e,n,lab", SHAPE_CASES, ids=[c[0] for c in SHAPE_CASES])
def test_supergraph_shapes_bit_exact(name, e, n, lab):
    dh = oracle.exact_degrees(e, n)
    sg = G.supergraph(e, n, lab, dh, 2, 256, 3)
    _check_super(sg, oracle.supergraph(e, n, lab, dh, 2, 256, 3))


def test_supergraph_identity_labels_is_the_graph():
    e = graphgen.random_graph(3000, 12000, seed=9)
    n = 3000
    lab = np.arange(n, dtype=np.int32)
    dh = oracle.exact_degrees(e, n)
    sg = G.supergraph(e, n, lab, dh, 4, 64, 1)
    _check_super(sg, oracle.supergraph(e, n, lab, dh, 4, 64, 1))
    assert sg["K"] == n and sg["Es"] == e.shape[0] and np.all(sg["w"] == 1)


def test_supergraph_single_community_and_optional_outputs():
    e = graphgen.random_graph(100, 300, seed=4)
    lab = np.full(100, 7, np.int32)
    dh = oracle.exact_degrees(e, 100)
    sg = G.supergraph(e, 100, lab, dh, 2, 16, 1, optional=False)
    assert sg["K"] == 1 and sg["Es"] == 0 and sg["csr_off"].tolist() == [0, 0]
    assert sg["mass"][0] >= 1 + int(dh.astype(np.int64).sum())


def test_supergraph_flags_bad_labels():
    e = graphgen.random_graph(10, 20, seed=4)
    lab = np.arange(10, dtype=np.int32)
    lab[3] = 10
    sg = G.supergraph(e, 10, lab, oracle.exact_degrees(e, 10), 2, 16, 1)
    assert sg["status"] & G.B.BGV_DEV_BADLABEL


@pytest.mark.parametrize("cutoff", [1 << 40, 1 << 12])
def test_sort_methods_give_the_same_order(cutoff):
    # The radix sort behind the supergraph and the FA2 tree runs as one
    # cooperative kernel or as onesweep passes (8 or 16 keys per thread by
    # the cutoff); every form is the same stable sort, so every output is
    # identical, and equal to the oracle.
    e = graphgen.random_graph(30000, 200000, seed=17)
    n = 30000
    _, dh = oracle.sketch_degrees(e, n, 4, 2048, 1)
    lab, _ = oracle.communities(e, n, dh, 3, 8, 2, 0)
    pos = oracle.fa2_init(n, 5)
    out = {}
    prev_m, prev_c = B.bgv_set_sort_method(1), B.bgv_set_sort_cutoff(cutoff)
    try:
        for method in (0, 1):
            B.bgv_set_sort_method(method)
            sg = G.supergraph(e, n, lab, dh, 4, 2048, 1)
            f = G.fa2_forces(pos, np.ones(n, np.uint32), np.zeros(n + 1, np.int32), np.zeros(0, np.int32),
                             np.zeros(0, np.uint32), FA2Params(leaf_cap=2))
            out[method] = (sg, f)
    finally:
        B.bgv_set_sort_method(prev_m)
        B.bgv_set_sort_cutoff(prev_c)
    sg0 = oracle.supergraph(e, n, lab, dh, 4, 2048, 1)
    for method, (sg, f) in out.items():
        for k in ("node_map", "src", "dst", "w", "mass", "csr_off", "csr_adj", "csr_w"):
            assert np.array_equal(sg[k], sg0[k]), (method, k)
    assert out[0][1]["interactions"] == out[1][1]["interactions"]
    assert np.array_equal(out[0][1]["Fr"], out[1][1]["Fr"])
