"""The whole pipeline through bgv_layout / bgv_layout_host (Algorithm 3 end to
end) against the oracle's stages; and full-size parity on the R-MAT
workloads (marked slow)."""
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


def _params(width=4096, passes=3, threshold=64, iterations=20):
    p = B.bgv_layout_default_params()
    p.width, p.passes, p.threshold, p.iterations = width, passes, threshold, iterations
    return p


def _oracle_supergraph(e, n, rows, width, seed, passes, threshold, growth=2, tie=0):
    _, dh = oracle.sketch_degrees(e, n, rows, width, seed)
    D = threshold if threshold else (2 * e.shape[0]) // n
    lab, _ = oracle.communities(e, n, dh, passes, D, growth, tie)
    return oracle.supergraph(e, n, lab, dh, rows, width, seed)


def test_layout_pipeline_matches_stages():
    n, e, _ = graphgen.load("sbm16")
    p = _params()
    E, m = G.edges_dev(e)
    node_map = G.empty(n, np.int32)
    xy = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    rad = torch.zeros(n, dtype=torch.float32, device="cuda")
    ws = B.alloc_ws(B.bgv_layout_ws_size(m, n, p))
    s = torch.cuda.Stream()
    K, Es = B.bgv_layout(E, m, n, p, node_map, xy, rad, ws, stream=s)
    s.synchronize()
    sg = _oracle_supergraph(e, n, 4, 4096, 1, 3, 64)
    assert (K, Es) == (sg["K"], sg["Es"])
    assert np.array_equal(G.host(node_map), sg["node_map"])
    r = G.host(rad)[:K]
    assert np.allclose(r, np.sqrt(sg["mass"].astype(np.float64)), rtol=1e-6)
    xyh = G.host(xy)[:K]
    assert np.all(np.isfinite(xyh))
    # the device run equals the same number of bgv_fa2_step calls from the
    # initial positions on the oracle's supergraph
    dv = G.Fa2Device(oracle.fa2_init(K, 1), sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], FA2Params())
    for _ in range(p.iterations):
        dv.step()
    assert np.array_equal(dv.state()[0].astype(np.float32), xyh)


def test_layout_host_matches_device():
    e, _ = graphgen.planted_partition([200] * 5, 0.05, 0.001, seed=3)
    n = 1000
    p = _params(width=512, threshold=0, iterations=10)
    E, m = G.edges_dev(e)
    node_map = G.empty(n, np.int32)
    xy = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    rad = torch.zeros(n, dtype=torch.float32, device="cuda")
    ws = B.alloc_ws(B.bgv_layout_ws_size(m, n, p))
    s = torch.cuda.Stream()
    K, Es = B.bgv_layout(E, m, n, p, node_map, xy, rad, ws, stream=s)
    he = torch.from_numpy(e.copy()).pin_memory()
    hmap = torch.zeros(n, dtype=torch.int32).pin_memory()
    hxy = torch.zeros((n, 2), dtype=torch.float32).pin_memory()
    hrad = torch.zeros(n, dtype=torch.float32).pin_memory()
    ws2 = B.alloc_ws(B.bgv_layout_host_ws_size(m, n, p))
    K2, Es2 = B.bgv_layout_host(he, m, n, p, hmap, hxy, hrad, ws2, stream=s)
    assert (K, Es) == (K2, Es2)
    assert np.array_equal(hmap.numpy(), G.host(node_map))
    assert np.array_equal(hxy.numpy()[:K], G.host(xy)[:K])
    assert np.array_equal(hrad.numpy()[:K], G.host(rad)[:K])


def test_layout_reports_bad_edges():
    e = np.array([[0, 1], [1, 7]], np.int32)
    p = _params(width=16, iterations=2)
    E, m = G.edges_dev(e)
    ws = B.alloc_ws(B.bgv_layout_ws_size(m, 5, p))
    with pytest.raises(B.BgvError) as ex:
        B.bgv_layout(E, m, 5, p, G.empty(5, np.int32), torch.zeros((5, 2), device="cuda"), None, ws)
    assert ex.value.code == B.BGV_EDEVICE


@pytest.mark.slow
@pytest.mark.parametrize("name,width,passes", [("rmat20", 65536, 3), ("rmat22x", 65536, 3)])
def test_full_size_integer_stages_bit_exact(name, width, passes):
    # Full-size workloads as the benchmark runs them: every integer output
    # element by element against the oracle.
    n, e, _ = graphgen.load(name)
    S, d, st = G.sketch(e, n, 4, width, 1)
    S0, d0 = oracle.sketch_degrees(e, n, 4, width, 1)
    assert st == 0 and np.array_equal(S, S0) and np.array_equal(d, d0)
    D = (2 * e.shape[0]) // n
    lab, deg, st = G.communities(e, n, d, passes, D, 2, 0)
    lab0, deg0 = oracle.communities(e, n, d0, passes, D, 2, 0)
    assert st == 0 and np.array_equal(lab, lab0) and np.array_equal(deg, deg0)
    sg = G.supergraph(e, n, lab, d, 4, width, 1)
    sg0 = oracle.supergraph(e, n, lab0, d0, 4, width, 1)
    assert sg["K"] == sg0["K"] and sg["Es"] == sg0["Es"]
    for k in ("node_map", "src", "dst", "w", "mass", "vol", "count", "csr_off", "csr_adj", "csr_w"):
        assert np.array_equal(np.asarray(sg[k]).astype(np.int64), np.asarray(sg0[k]).astype(np.int64)), k


@pytest.mark.slow
def test_full_size_fa2_step_sampled():
    # One FA2 step on the full rmat20 supergraph, forces checked on a sample
    # of 2000 supernodes that the oracle computes one by one.
    n, e, _ = graphgen.load("rmat20")
    sg = _oracle_supergraph(e, n, 4, 65536, 1, 3, 0)
    K = sg["K"]
    pos = oracle.fa2_init(K, 1)
    p = FA2Params()
    r = G.fa2_forces(pos, sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], p)
    assert r["status"] == 0
    which = np.random.default_rng(0).choice(K, size=2000, replace=False)
    Fr0, _ = oracle.bh_repulsion(pos, sg["mass"], p, which=which)
    assert G.rel_err(r["Fr"][which], Fr0) <= 1e-3
    Fa0 = oracle.attraction(sg["csr_off"], sg["csr_adj"], sg["csr_w"], pos)
    assert G.rel_err(r["Fa"], Fa0) <= 1e-3


@pytest.mark.slow
def test_full_size_fa2_forces_rmat22x():
    # One FA2 force evaluation on the whole rmat22x supergraph (3.2 M
    # supernodes): the interaction total equals the oracle's (same tree and
    # theta), every repulsion is within 1e-3 of the FP64 oracle, and so is the
    # attraction over all 68 M CSR entries.
    n, e, _ = graphgen.load("rmat22x")
    sg = _oracle_supergraph(e, n, 4, 65536, 1, 3, 0)
    K = sg["K"]
    pos = oracle.fa2_init(K, 1)
    p = FA2Params()
    r = G.fa2_forces(pos, sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], p)
    assert r["status"] == 0
    Fr0, inter0 = oracle.bh_repulsion(pos, sg["mass"], p)
    assert r["interactions"] == inter0
    assert G.rel_err(r["Fr"], Fr0) <= 1e-3
    Fa0 = oracle.attraction(sg["csr_off"], sg["csr_adj"], sg["csr_w"], pos)
    assert G.rel_err(r["Fa"], Fa0) <= 1e-3


@pytest.mark.slow
def test_fa2_forces_above_the_sort_size_cutoff():
    # 4.5 M bodies with the sort's cutoff set to 2^22, so it runs 16 keys
    # per thread.  Uniform positions plus a dense cluster inside one
    # fine cell; the interaction total and every force against the oracle.
    rng = np.random.default_rng(45)
    K = 4_500_000
    pos = (rng.random((K, 2)) * 4000 - 2000).astype(np.float32)
    pos[:5000] = (pos[0] + rng.random((5000, 2)) * 0.001).astype(np.float32)
    mass = rng.integers(1, 5, K).astype(np.uint32)
    off = np.zeros(K + 1, np.int32)
    p = FA2Params(theta=1.2, leaf_cap=4)
    prev = B.bgv_set_sort_cutoff(1 << 22)
    try:
        assert K > B.bgv_sort_cutoff()
        r = G.fa2_forces(pos, mass, off, np.zeros(0, np.int32), np.zeros(0, np.uint32), p)
    finally:
        B.bgv_set_sort_cutoff(prev)
    assert r["status"] == 0
    Fr0, inter0 = oracle.bh_repulsion(pos, mass, p)
    assert r["interactions"] == inter0
    outside = np.ones(K, bool)
    outside[:5000] = False  # inside the cluster, FP32 cell centres cannot resolve the spacing
    assert G.rel_err(r["Fr"][outside], Fr0[outside]) <= 1e-3
