"""Precision form: ForceAtlas2 on a whole graph (mass = degree + 1, unit edge
weights), coloured by its streamed communities, with the per-step force
error of the FP32 GPU path measured against the FP64 oracle on a sample of
nodes (Section 4.1 whole-graph layout; Section 4.3 colours)."""
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


def graph_csr(e, n):
    E, m = G.edges_dev(e)
    off, adj, w = G.empty(n + 1, np.int32), G.empty(2 * max(m, 1), np.int32), G.empty(2 * max(m, 1), np.uint32)
    mass, nnz = G.empty(n, np.uint32), G.empty(1, np.int64)
    ws = B.alloc_ws(B.bgv_graph_csr_ws_size(m, n))
    B.bgv_graph_csr(E, m, n, off, adj, w, mass, nnz, ws)
    k = int(nnz.item())
    assert B.bgv_status(ws) == 0
    return (G.host(off, None, n + 1), G.host(adj, None, k), G.host(w, np.uint32, k), G.host(mass, np.uint32, n))


def test_graph_csr_matches_independent_construction():
    rng = np.random.default_rng(0)
    n = 3000
    e = graphgen.random_graph(n, 15000, seed=1, self_loops=20)
    e = np.concatenate([e, e[rng.integers(0, e.shape[0], 500)][:, ::-1]])  # repeated pairs, reversed
    off, adj, w, mass = graph_csr(e, n)
    keep = e[:, 0] != e[:, 1]
    lo, hi = np.minimum(e[keep, 0], e[keep, 1]), np.maximum(e[keep, 0], e[keep, 1])
    pairs, counts = np.unique(lo.astype(np.int64) * n + hi, return_counts=True)
    a, b = pairs // n, pairs % n
    rows = np.concatenate([a, b])
    cols = np.concatenate([b, a])
    cw = np.concatenate([counts, counts])
    order = np.lexsort((cols, rows))
    ref_off = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))])
    assert np.array_equal(off, ref_off)
    assert np.array_equal(adj, cols[order])
    assert np.array_equal(w, cw[order])
    assert np.array_equal(mass, np.diff(ref_off) + 1)


@pytest.mark.parametrize("K,seed", [(1, 0), (7, 1), (5000, 2), (300001, 3)])
def test_colour_groups_match_oracle(K, seed):
    rng = np.random.default_rng(seed)
    sizes = (rng.lognormal(2, 2, K) + 1).astype(np.uint32)
    sizes[: K // 3] = sizes[0]  # many ties
    S = G.dev(sizes)
    g = torch.zeros(max(K, 1), dtype=torch.uint8, device="cuda")
    ws = B.alloc_ws(B.bgv_colour_groups_ws_size(K))
    n = 2 * K + 3
    node_map = rng.integers(0, K, n).astype(np.int32)
    nc = torch.zeros(n, dtype=torch.uint8, device="cuda")
    B.bgv_colour_groups(K, S, g, ws, n=n, node_map=G.dev(node_map), node_colour=nc)
    ref = oracle.colour_groups(sizes)
    assert np.array_equal(g.cpu().numpy()[:K], ref)
    assert np.array_equal(nc.cpu().numpy(), ref[node_map])


def _precision_run(e, n, steps, log_at, sample, seed=4):
    off, adj, w, mass = graph_csr(e, n)
    p = FA2Params()
    dv = G.Fa2Device(oracle.fa2_init(n, seed), mass, off, adj, w, p)
    which = np.random.default_rng(seed).choice(n, size=min(sample, n), replace=False)
    errs = {}
    for t in range(steps + 1):
        if t in log_at:
            pos = G.host(dv.pos).astype(np.float32)
            r = G.fa2_forces(pos, mass, off, adj, w, p)
            Fr0, _ = oracle.bh_repulsion(pos, mass, p, which=which)
            pw = pos.astype(np.float64)
            Fa0 = oracle.attraction(off, adj, w, pos)[which]
            Fg0 = oracle.gravity(mass, pos, p.kg, p.strong_gravity)[which]
            F = r["Fr"][which] + r["Fa"][which] + r["Fg"][which]
            errs[t] = dict(Fr=G.rel_err(r["Fr"][which], Fr0), F=G.rel_err(F, Fr0 + Fa0 + Fg0))
            assert np.all(np.isfinite(pw))
        if t < steps:
            dv.step()
    return errs


def test_precision_form_small_graph():
    # A 40,000-node lognormal planted partition (same recipe as the 1M-node
    # workload): per-step force error on a 2,000-node sample stays <= 1e-3.
    sizes = graphgen._largest_remainder(np.random.default_rng(1).lognormal(5, 1, 64), 40_000, 2)
    e, _ = graphgen.uneven_planted(sizes, 320_000, 0.8, seed=5)
    errs = _precision_run(e, 40_000, steps=30, log_at={0, 10, 30}, sample=2000)
    for t, er in errs.items():
        assert er["Fr"] <= 1e-3, (t, er)
        assert er["F"] <= 1e-3, (t, er)


@pytest.mark.slow
def test_precision_form_full_size():
    # The 1M-node, 8M-edge workload: error on a 20,000-node sample at
    # several steps of the run.
    n, e, _ = graphgen.load("lnpp1m")
    errs = _precision_run(e, n, steps=40, log_at={0, 20, 40}, sample=20_000)
    for t, er in errs.items():
        assert er["Fr"] <= 1e-3, (t, er)
        assert er["F"] <= 1e-3, (t, er)
