"""Batched form: G independent graphs through bgv_layout_batched and the
batched FA2 entry points, against G separate single-graph calls and the
oracle's stages per graph (Algorithm 3 applied to each graph)."""
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


def _params(width=256, passes=3, threshold=0, iterations=0):
    p = B.bgv_layout_default_params()
    p.width, p.passes, p.threshold, p.iterations = width, passes, threshold, iterations
    return p


def _mixed_batch():
    """Graphs of uneven size and density, plus the degenerate ones: a single
    node without edges, a graph of self loops and isolated nodes."""
    graphs = [(e, int(mem.shape[0])) for e, mem in graphgen.batch_set(5, 40, 3000, 2, 9, avg_degree=6, seed0=7)]
    graphs.insert(1, (np.zeros((0, 2), np.int32), 1))
    graphs.append((np.array([[0, 0], [1, 1], [2, 3], [3, 2], [0, 3]], np.int32), 7))
    dense = graphgen.random_graph(400, 12_000, seed=3)  # 2m/n = 60: a higher threshold
    graphs.append((dense, 400))
    return graphs


def _concat(graphs):
    edges = np.concatenate([np.asarray(e, np.int32).reshape(-1, 2) for e, _ in graphs]) if graphs else None
    edge_off = np.concatenate([[0], np.cumsum([np.asarray(e).reshape(-1, 2).shape[0] for e, _ in graphs])])
    node_off = np.concatenate([[0], np.cumsum([n for _, n in graphs])])
    return edges, edge_off.astype(np.int64), node_off.astype(np.int32)


def _batched(graphs, p):
    edges, eo, no = _concat(graphs)
    N = int(no[-1])
    E, _ = G.edges_dev(edges)
    node_map = G.empty(N, np.int32)
    xy = torch.zeros((N, 2), dtype=torch.float32, device="cuda")
    rad = torch.zeros(N, dtype=torch.float32, device="cuda")
    ws = B.alloc_ws(B.bgv_layout_batched_ws_size(len(graphs), eo, no, p))
    K_off, Es_off = B.bgv_layout_batched(E, len(graphs), eo, no, p, node_map, xy, rad, ws)
    return G.host(node_map), G.host(xy), G.host(rad), K_off, Es_off, no


def _single(e, n, p):
    E, m = G.edges_dev(e)
    node_map = G.empty(n, np.int32)
    xy = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    rad = torch.zeros(n, dtype=torch.float32, device="cuda")
    ws = B.alloc_ws(B.bgv_layout_ws_size(m, n, p))
    K, Es = B.bgv_layout(E, m, n, p, node_map, xy, rad, ws)
    return G.host(node_map), G.host(xy)[:K], G.host(rad)[:K], K, Es


@pytest.mark.parametrize("threshold", [0, 5])
def test_batched_layout_equals_separate_calls_at_start(threshold):
    # Zero FA2 steps: every output is integer or exact, so the batch must
    # reproduce each graph's own call bit for bit.
    graphs = _mixed_batch()
    p = _params(threshold=threshold)
    nm, xy, rad, K_off, Es_off, no = _batched(graphs, p)
    assert K_off[0] == 0 and Es_off[0] == 0
    for g, (e, n) in enumerate(graphs):
        nm1, xy1, rad1, K, Es = _single(e, n, p)
        assert (K_off[g + 1] - K_off[g], Es_off[g + 1] - Es_off[g]) == (K, Es), g
        assert np.array_equal(nm[no[g]:no[g + 1]], nm1), g
        assert np.array_equal(xy[K_off[g]:K_off[g + 1]], xy1), g
        assert np.array_equal(rad[K_off[g]:K_off[g + 1]], rad1), g


def test_batched_integer_stages_match_oracle():
    graphs = _mixed_batch()
    p = _params()
    nm, _, rad, K_off, Es_off, no = _batched(graphs, p)
    for g, (e, n) in enumerate(graphs):
        e = np.asarray(e, np.int32).reshape(-1, 2)
        _, dh = oracle.sketch_degrees(e, n, 4, 256, 1)
        lab, _ = oracle.communities(e, n, dh, 3, (2 * e.shape[0]) // n, 2, 0)
        sg = oracle.supergraph(e, n, lab, dh, 4, 256, 1)
        assert (K_off[g + 1] - K_off[g], Es_off[g + 1] - Es_off[g]) == (sg["K"], sg["Es"]), g
        assert np.array_equal(nm[no[g]:no[g + 1]], sg["node_map"]), g
        r = rad[K_off[g]:K_off[g + 1]].astype(np.float64)
        assert np.allclose(r, np.sqrt(sg["mass"].astype(np.float64)), rtol=1e-6), g


def _oracle_batch(graphs):
    """Per-graph oracle supergraphs joined into one block-diagonal CSR."""
    sgs = []
    for e, n in graphs:
        e = np.asarray(e, np.int32).reshape(-1, 2)
        _, dh = oracle.sketch_degrees(e, n, 4, 256, 1)
        lab, _ = oracle.communities(e, n, dh, 3, (2 * e.shape[0]) // n, 2, 0)
        sgs.append(oracle.supergraph(e, n, lab, dh, 4, 256, 1))
    koff = np.concatenate([[0], np.cumsum([s["K"] for s in sgs])]).astype(np.int64)
    off = [np.zeros(1, np.int64)]
    for s in sgs:
        off.append(s["csr_off"][1:].astype(np.int64) + off[-1][-1])
    off = np.concatenate(off).astype(np.int32)
    adj = np.concatenate([s["csr_adj"] + koff[g] for g, s in enumerate(sgs)]).astype(np.int32)
    w = np.concatenate([s["csr_w"] for s in sgs]).astype(np.uint32)
    mass = np.concatenate([s["mass"] for s in sgs]).astype(np.uint32)
    return sgs, koff, off, adj, w, mass


def test_batched_forces_equal_separate_calls():
    # Same positions, same tree per graph: every force is bit identical to
    # the single-graph call (each row's attraction is summed in an order set
    # by the row's own entries alone).
    graphs = _mixed_batch()
    sgs, koff, off, adj, w, mass = _oracle_batch(graphs)
    Gn, K = len(graphs), int(koff[-1])
    rng = np.random.default_rng(5)
    pos = np.concatenate([rng.normal(0, np.sqrt(s["K"]), (s["K"], 2)) for s in sgs]).astype(np.float32)
    pos[int(koff[2]) + 1] = pos[int(koff[2])]  # coincident bodies
    p = G.fa2_params(FA2Params())
    Fr, Fa, Fg = (torch.zeros((K, 2), dtype=torch.float32, device="cuda") for _ in range(3))
    ws = B.alloc_ws(B.bgv_fa2_ws_size_batched(Gn, K, int(off[-1])))
    O, A, W = G._csr_dev(off, adj, w)
    B.bgv_fa2_forces_batched(Gn, koff, int(off[-1]), O, A, W, G.dev(mass), p, G.dev(pos), Fr, Fa, Fg, ws)
    Fr, Fa, Fg = G.host(Fr), G.host(Fa), G.host(Fg)
    for g, s in enumerate(sgs):
        a, b = int(koff[g]), int(koff[g + 1])
        r = G.fa2_forces(pos[a:b], s["mass"], s["csr_off"], s["csr_adj"], s["csr_w"], FA2Params())
        assert np.array_equal(Fr[a:b].astype(np.float64), r["Fr"]), g
        assert np.array_equal(Fg[a:b].astype(np.float64), r["Fg"]), g
        assert np.array_equal(Fa[a:b].astype(np.float64), r["Fa"]), g


def test_batched_run_tracks_separate_runs():
    graphs = _mixed_batch()
    sgs, koff, off, adj, w, mass = _oracle_batch(graphs)
    Gn, K, nnz = len(graphs), int(koff[-1]), int(off[-1])
    p = G.fa2_params(FA2Params())
    pos = torch.zeros((K, 2), dtype=torch.float32, device="cuda")
    F, Fprev = torch.zeros_like(pos), torch.zeros_like(pos)
    speed = torch.zeros(Gn, dtype=torch.float64, device="cuda")
    ws = B.alloc_ws(B.bgv_fa2_ws_size_batched(Gn, K, nnz))
    B.bgv_fa2_init_batched(Gn, koff, p, pos, Fprev, speed, ws)
    # the batched start is each graph's own start
    start = G.host(pos)
    for g, s in enumerate(sgs):
        assert np.array_equal(start[koff[g]:koff[g + 1]], oracle.fa2_init(s["K"], 1).astype(np.float32)), g
    O, A, W = G._csr_dev(off, adj, w)
    steps = 4
    B.bgv_fa2_run_batched(Gn, koff, nnz, O, A, W, G.dev(mass), p, steps, 1, pos, F, Fprev, speed, ws)
    out, sp = G.host(pos).astype(np.float64), G.host(speed)
    for g, s in enumerate(sgs):
        dv = G.Fa2Device(oracle.fa2_init(s["K"], 1), s["mass"], s["csr_off"], s["csr_adj"], s["csr_w"], FA2Params())
        dv.run(steps, 0)
        ref, _, _, ref_speed = dv.state()
        # the same forces and exact swing/traction sums: the same trajectory
        assert np.array_equal(out[koff[g]:koff[g + 1]], ref), g
        assert sp[g] == ref_speed, g


def test_batched_reports_edges_outside_their_graph():
    graphs = [(np.array([[0, 1], [1, 2]], np.int32), 3), (np.array([[0, 3]], np.int32), 3)]  # 3 is not in graph 1
    with pytest.raises(B.BgvError) as ei:
        _batched(graphs, _params())
    assert ei.value.code == B.BGV_EDEVICE


@pytest.mark.slow
def test_batch_set_integer_stages_equal_separate_calls():
    # The 512-graph batch: supernode maps and counts of every graph equal its
    # own bgv_layout call.
    graphs = [(e, int(mem.shape[0])) for e, mem in graphgen.batch_set()]
    p = _params(width=4096)
    nm, _, _, K_off, Es_off, no = _batched(graphs, p)
    for g, (e, n) in enumerate(graphs):
        nm1, _, _, K, Es = _single(e, n, p)
        assert (K_off[g + 1] - K_off[g], Es_off[g + 1] - Es_off[g]) == (K, Es), g
        assert np.array_equal(nm[no[g]:no[g + 1]], nm1), g


@pytest.mark.slow
def test_batched_forces_match_oracle_above_the_sort_cutoff():
    # Batched forces against the oracle directly, graph by graph: a batch of
    # uneven graphs whose 4.3 M bodies exceed a 2^22-key cutoff of the sort
    # (set here, so it runs 16 keys per thread).  The interaction total equals the sum of the
    # oracle's per-graph totals (same trees and theta) and every force is
    # within 1e-3 of the FP64 oracle.
    rng = np.random.default_rng(9)
    sizes = [4_200_000, 1, 2, 1000, 37_000, 90_001]
    parts = []
    for g, K in enumerate(sizes):
        side = 2.0 * np.sqrt(K)
        pos = (rng.random((K, 2)) * side - side / 2).astype(np.float32)
        e = graphgen.random_graph(K, 2 * K, seed=100 + g) if K > 1 else np.zeros((0, 2), np.int32)
        off, adj, w = G.csr_from_edges(e, K)
        w = rng.integers(1, 4, w.shape[0]).astype(np.uint32)
        src = np.repeat(np.arange(K), np.diff(off))
        key = np.minimum(src, adj).astype(np.int64) * K + np.maximum(src, adj)
        _, inv = np.unique(key, return_inverse=True)
        w = (inv % 3 + 1).astype(np.uint32)  # symmetric weights
        mass = rng.integers(1, 6, K).astype(np.uint32)
        parts.append((pos, mass, off, adj, w))
    Gn = len(sizes)
    koff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    offs = [np.zeros(1, np.int64)]
    for _, _, off, _, _ in parts:
        offs.append(off[1:].astype(np.int64) + offs[-1][-1])
    off = np.concatenate(offs).astype(np.int32)
    adj = np.concatenate([pt[3] + koff[g] for g, pt in enumerate(parts)]).astype(np.int32)
    w = np.concatenate([pt[4] for pt in parts])
    mass = np.concatenate([pt[1] for pt in parts])
    pos = np.concatenate([pt[0] for pt in parts])
    K, nnz = int(koff[-1]), int(off[-1])
    p = FA2Params()
    Fr, Fa, Fg = (torch.zeros((K, 2), dtype=torch.float32, device="cuda") for _ in range(3))
    ws = B.alloc_ws(B.bgv_fa2_ws_size_batched(Gn, K, nnz))
    O, A, W = G._csr_dev(off, adj, w)
    prev = B.bgv_set_sort_cutoff(1 << 22)
    try:
        assert K > B.bgv_sort_cutoff()
        B.bgv_fa2_forces_batched(Gn, koff, nnz, O, A, W, G.dev(mass), G.fa2_params(p), G.dev(pos), Fr, Fa, Fg, ws)
    finally:
        B.bgv_set_sort_cutoff(prev)
    st = B.bgv_fa2_read_stats(ws)
    assert st.status == 0
    Fr, Fa, Fg = G.host(Fr), G.host(Fa), G.host(Fg)
    total = 0
    for g, (pg, mg, og, ag, wg) in enumerate(parts):
        a, b = int(koff[g]), int(koff[g + 1])
        Fr0, inter0 = oracle.bh_repulsion(pg, mg, p)
        total += inter0
        assert G.rel_err(Fr[a:b], Fr0) <= 1e-3, g
        assert G.rel_err(Fa[a:b], oracle.attraction(og, ag, wg, pg)) <= 1e-3, g
        assert G.rel_err(Fg[a:b], oracle.gravity(mg, pg, 1.0, 0)) <= 1e-3, g
    assert st.interactions == total
