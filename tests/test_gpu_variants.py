"""Variants of the community step on the GPU (Section 4.2.2: the mode degree
as the first threshold and the delta^i schedule; pointer jumping between
rounds) against the oracle, bit for bit, through the C ABI."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import gpu_pipeline as G  # noqa: E402

B = G.B


@pytest.mark.parametrize("case", ["random", "ties", "zeros", "single", "big"])
def test_mode_degree_matches_oracle(case):
    rng = np.random.default_rng(3)
    d = {"random": rng.integers(0, 50, 20011), "ties": np.repeat(np.arange(1, 30), 7),
         "zeros": np.zeros(100), "single": np.array([5]),
         "big": rng.zipf(2.0, 1_000_003).clip(0, 2**31)}[case].astype(np.uint32)
    ws = B.alloc_ws(B.bgv_mode_degree_ws_size(d.shape[0]))
    assert B.bgv_mode_degree(G.dev(d), d.shape[0], ws) == oracle.mode_degree(d)


def _graphs():
    n, e, _ = graphgen.load("sbm16")
    yield "sbm16", n, e
    yield "rmat", 1 << 14, graphgen.rmat(14, 120_000, 0.57, 0.19, 0.19, seed=9)
    yield "random", 3000, graphgen.random_graph(3000, 20_000, seed=4, self_loops=10)


@pytest.mark.parametrize("growth,jumps,tmode,tie", [(2, 0, 1, 0), (0, 0, 0, 0), (2, 1, 0, 1), (0, 3, 1, 0),
                                                    (3, 2, 1, 1)])
def test_community_variants_match_oracle(growth, jumps, tmode, tie):
    for name, n, e in _graphs():
        _, dh, _ = G.sketch(e, n, 4, 1024, 1)
        E, m = G.edges_dev(e)
        lab = G.empty(n, np.int32)
        deg = G.empty(n, np.uint32)
        ws = B.alloc_ws(B.bgv_communities_ex_ws_size(m, n))
        D = B.bgv_communities_ex(E, m, n, G.dev(dh), 3, 0, growth, tie, tmode, jumps, lab, deg, ws)
        D0 = oracle.mode_degree(dh) if tmode else (2 * m) // n
        assert D == D0, name
        lab0, deg0 = oracle.communities_ex(e, n, dh, 3, D0, growth, tie, jumps)
        assert np.array_equal(G.host(lab, None, n), lab0), name
        assert np.array_equal(G.host(deg, np.uint32, n), deg0), name
        assert B.bgv_status(ws) == 0


def test_layout_with_variants_matches_oracle_stages():
    n, e, _ = graphgen.load("sbm16")
    p = B.bgv_layout_default_params()
    p.width, p.threshold, p.threshold_mode, p.growth, p.jumps, p.iterations = 1024, 0, 1, 0, 2, 3
    E, m = G.edges_dev(e)
    node_map = G.empty(n, np.int32)
    xy = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    ws = B.alloc_ws(B.bgv_layout_ws_size(m, n, p))
    K, Es = B.bgv_layout(E, m, n, p, node_map, xy, None, ws)
    _, dh = oracle.sketch_degrees(e, n, 4, 1024, 1)
    # the layout takes the most common exact degree of the graph
    lab, _ = oracle.communities_ex(e, n, dh, 3, oracle.mode_degree(oracle.exact_degrees(e, n)), 0, 0, 2)
    sg = oracle.supergraph(e, n, lab, dh, 4, 1024, 1)
    assert (K, Es) == (sg["K"], sg["Es"])
    assert np.array_equal(G.host(node_map), sg["node_map"])


def test_batched_mode_degree_per_graph():
    graphs = [(e, int(mem.shape[0])) for e, mem in graphgen.batch_set(6, 50, 4000, 2, 9, avg_degree=8, seed0=21)]
    p = B.bgv_layout_default_params()
    p.width, p.threshold, p.threshold_mode, p.jumps, p.iterations = 512, 0, 1, 1, 0
    edges = np.concatenate([e for e, _ in graphs]).astype(np.int32)
    eo = np.concatenate([[0], np.cumsum([e.shape[0] for e, _ in graphs])]).astype(np.int64)
    no = np.concatenate([[0], np.cumsum([n for _, n in graphs])]).astype(np.int32)
    N = int(no[-1])
    E, _ = G.edges_dev(edges)
    nm = G.empty(N, np.int32)
    xy = torch.zeros((N, 2), dtype=torch.float32, device="cuda")
    ws = B.alloc_ws(B.bgv_layout_batched_ws_size(len(graphs), eo, no, p))
    K_off, Es_off = B.bgv_layout_batched(E, len(graphs), eo, no, p, nm, xy, None, ws)
    nm = G.host(nm)
    for g, (e, n) in enumerate(graphs):
        _, dh = oracle.sketch_degrees(e, n, 4, 512, 1)
        lab, _ = oracle.communities_ex(e, n, dh, 3, oracle.mode_degree(oracle.exact_degrees(e, n)), 2, 0, 1)
        sg = oracle.supergraph(e, n, lab, dh, 4, 512, 1)
        assert (K_off[g + 1] - K_off[g], Es_off[g + 1] - Es_off[g]) == (sg["K"], sg["Es"]), g
        assert np.array_equal(nm[no[g]:no[g + 1]], sg["node_map"]), g


@pytest.mark.parametrize("which", ["planted", "rounds", "singletons", "one", "bad-rmat"])
def test_modularity_matches_oracle(which):
    n, e, memb = graphgen.load("sbm16")
    if which == "bad-rmat":
        n, e = 1 << 12, graphgen.rmat(12, 30_000, 0.57, 0.19, 0.19, seed=2)
        lab = np.random.default_rng(1).integers(0, 50, n).astype(np.int32)
    elif which == "planted":
        lab = memb.astype(np.int32)
    elif which == "rounds":
        _, dh = oracle.sketch_degrees(e, n, 4, 4096, 1)
        lab = oracle.communities(e, n, dh, 3, 64, 2, 0)[0]
    elif which == "singletons":
        lab = np.arange(n, dtype=np.int32)
    else:
        lab = np.zeros(n, np.int32)
    E, m = G.edges_dev(e)
    ws = B.alloc_ws(B.bgv_modularity_ws_size(n))
    q = B.bgv_modularity(E, m, n, G.dev(lab), ws)
    assert q == pytest.approx(oracle.modularity(e, n, lab), abs=1e-12)


@pytest.mark.parametrize("K,W,H,seed", [(1, 33, 17, 0), (40, 64, 64, 1), (500, 97, 61, 2), (3000, 128, 128, 3)])
def test_render_matches_oracle(K, W, H, seed):
    rng = np.random.default_rng(seed)
    xy = (rng.random((K, 2)) * 100).astype(np.float32)
    xy[K // 2:] = xy[: K - K // 2] if K > 3 else xy[K // 2:]  # coincident discs
    radius = np.sqrt(rng.integers(1, 60, K)).astype(np.float32)
    group = rng.integers(0, 11, K).astype(np.uint8)
    img = torch.zeros((H, W, 4), dtype=torch.uint8, device="cuda")
    ws = B.alloc_ws(B.bgv_render_ws_size(W, H))
    B.bgv_render(K, G.dev(xy), G.dev(radius), torch.from_numpy(group).cuda(), W, H, img, ws)
    assert np.array_equal(img.cpu().numpy(), oracle.render(xy, radius, group, W, H))


def test_render_layout_of_sbm16():
    # The whole styling path: layout, colour groups, drawing.
    n, e, _ = graphgen.load("sbm16")
    p = B.bgv_layout_default_params()
    p.threshold, p.iterations = 64, 30
    E, m = G.edges_dev(e)
    node_map = G.empty(n, np.int32)
    xy = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    rad = torch.zeros(n, dtype=torch.float32, device="cuda")
    ws = B.alloc_ws(B.bgv_layout_ws_size(m, n, p))
    K, _ = B.bgv_layout(E, m, n, p, node_map, xy, rad, ws)
    sizes = (G.host(rad)[:K].astype(np.float64) ** 2).round().astype(np.uint32)
    grp = torch.zeros(K, dtype=torch.uint8, device="cuda")
    wsg = B.alloc_ws(B.bgv_colour_groups_ws_size(K))
    B.bgv_colour_groups(K, G.dev(sizes), grp, wsg)
    W = H = 256
    img = torch.zeros((H, W, 4), dtype=torch.uint8, device="cuda")
    wsr = B.alloc_ws(B.bgv_render_ws_size(W, H))
    B.bgv_render(K, xy, rad, grp, W, H, img, wsr)
    ref = oracle.render(G.host(xy)[:K], G.host(rad)[:K], grp.cpu().numpy(), W, H)
    assert np.array_equal(img.cpu().numpy(), ref)


def test_sort_autotuner_sets_a_consistent_cutoff():
    ws = B.alloc_ws(B.bgv_autotune_sort_ws_size(1 << 20))
    r = B.bgv_autotune_sort(1 << 20, ws)
    assert r.count == 4 and list(r.sizes_log2[:4]) == [14, 16, 18, 20]
    assert all(r.ms8[k] > 0 and r.ms16[k] > 0 for k in range(4))
    wins = [1 << r.sizes_log2[k] for k in range(4) if r.ms8[k] <= r.ms16[k]]
    assert r.cutoff == (max(wins) if wins else 0) == B.bgv_sort_cutoff()
    # whatever the cutoff, the stages that sort stay exact
    n, e, _ = graphgen.load("sbm16")
    for cutoff_case in range(2):
        _, dh, _ = G.sketch(e, n, 4, 4096, 1)
        lab = oracle.communities(e, n, dh, 3, 64, 2, 0)[0]
        sg = G.supergraph(e, n, lab, dh, 4, 4096, 1, optional=False)
        ref = oracle.supergraph(e, n, lab, dh, 4, 4096, 1)
        assert np.array_equal(sg["csr_adj"], ref["csr_adj"]) and np.array_equal(sg["node_map"], ref["node_map"])
