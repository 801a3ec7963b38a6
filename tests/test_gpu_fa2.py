"""GPU parity of the ForceAtlas2 stage (Section 3.1, Algorithm 1).

Same quadtree and theta as the oracle: the interaction sets must be identical
(the interaction counts equal exactly) and every per-node force within 1e-3
relative error of the FP64 oracle; against exact all-pairs forces the error
bounds of the method hold.  Calls go through the C ABI."""
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

TOL = 1e-3


def _case(K, seed, mass_hi=1, layout="uniform"):
    rng = np.random.default_rng(seed)
    if layout == "uniform":
        pos = (rng.random((K, 2)) * 200 - 100).astype(np.float32)
    elif layout == "clustered":
        c = rng.normal(size=(max(K // 50, 1), 2)) * 100
        pos = (c[rng.integers(0, c.shape[0], K)] + rng.normal(size=(K, 2))).astype(np.float32)
    else:  # init positions of the method
        pos = oracle.fa2_init(K, seed)
    mass = rng.integers(1, mass_hi + 1, K).astype(np.uint32)
    e = graphgen.random_graph(K, 3 * K, seed=seed + 1) if K > 1 else np.zeros((0, 2), np.int32)
    off, adj, w = G.csr_from_edges(e, K)
    w = rng.integers(1, 5, w.shape[0]).astype(np.uint32)
    # symmetric weights: weight of (i, j) equals weight of (j, i)
    src = np.repeat(np.arange(K), np.diff(off))
    key = np.minimum(src, adj).astype(np.int64) * K + np.maximum(src, adj)
    _, inv = np.unique(key, return_inverse=True)
    w = (inv % 4 + 1).astype(np.uint32)
    return pos, mass, off, adj, w


CASES = [(2, 0, 1, "uniform"), (3, 1, 5, "uniform"), (33, 2, 1, "uniform"), (1000, 3, 50, "clustered"),
         (4097, 4, 1, "init"), (20011, 5, 1000, "uniform"), (70001, 6, 3, "clustered")]


@pytest.mark.parametrize("K,seed,mass_hi,layout", CASES)
@pytest.mark.parametrize("theta,leaf_cap", [(1.2, 1), (0.5, 4), (0.0, 1)])
def test_forces_match_oracle(K, seed, mass_hi, layout, theta, leaf_cap):
    if theta == 0.0 and K > 5000:
        pytest.skip("all-pairs oracle too slow at this size")
    pos, mass, off, adj, w = _case(K, seed, mass_hi, layout)
    p = FA2Params(theta=theta, leaf_cap=leaf_cap, kr=2.0, kg=1.0)
    r = G.fa2_forces(pos, mass, off, adj, w, p)
    assert r["status"] == 0
    Fr0, inter0 = oracle.bh_repulsion(pos, mass, p)
    assert r["interactions"] == inter0
    assert G.rel_err(r["Fr"], Fr0) <= TOL
    assert G.rel_err(r["Fa"], oracle.attraction(off, adj, w, pos)) <= TOL
    assert G.rel_err(r["Fg"], oracle.gravity(mass, pos, 1.0, 0)) <= TOL


def test_coincident_points_and_duplicates():
    rng = np.random.default_rng(3)
    pos = np.concatenate([rng.random((500, 2)) * 10, np.repeat([[5.0, 5.0]], 40, axis=0),
                          np.repeat([[1.0, 9.0]], 3, axis=0)]).astype(np.float32)
    K = pos.shape[0]
    mass = rng.integers(1, 9, K).astype(np.uint32)
    off, adj, w = G.csr_from_edges(np.zeros((0, 2), np.int32), K)
    for leaf_cap in (1, 2, 64):
        p = FA2Params(theta=0.8, leaf_cap=leaf_cap)
        r = G.fa2_forces(pos, mass, off, adj, w, p)
        Fr0, inter0 = oracle.bh_repulsion(pos, mass, p)
        assert r["interactions"] == inter0
        assert G.rel_err(r["Fr"], Fr0) <= TOL


@pytest.mark.parametrize("sizes", [(3000,), (100, 150, 40), (5, 7, 3, 9, 12)])
def test_dense_clusters_inside_one_fine_cell(sizes):
    # Clusters smaller than 2^-12 of the frame (side 2000, cells of 0.49 at
    # that level) share the Morton bits above 24: long runs that the sort
    # orders run by run on the low bits (in registers up to 8 keys, by a warp
    # up to 256, by a block above).  The tree must equal the oracle's: the
    # interaction counts are equal exactly.  Inside such a cluster the
    # spacing is below what FP32 cell centres resolve in this frame (about
    # 1e-4), so forces are compared on the bodies outside the clusters.
    rng = np.random.default_rng(len(sizes))
    parts = [np.array([[-1000.0, -1000.0], [1000.0, 1000.0]]), rng.random((500, 2)) * 2000 - 1000]
    for k in sizes:
        parts.append(rng.random(2) * 1000 - 500 + rng.random((k, 2)) * 0.02)
    pos = np.concatenate(parts).astype(np.float32)
    outside = np.zeros(pos.shape[0], bool)
    outside[:502] = True
    order = rng.permutation(pos.shape[0])
    pos, outside = pos[order], outside[order]
    K = pos.shape[0]
    mass = rng.integers(1, 9, K).astype(np.uint32)
    off, adj, w = G.csr_from_edges(graphgen.random_graph(K, 2 * K, seed=7), K)
    for leaf_cap in (1, 8):
        p = FA2Params(theta=1.2, leaf_cap=leaf_cap)
        r = G.fa2_forces(pos, mass, off, adj, w, p)
        Fr0, inter0 = oracle.bh_repulsion(pos, mass, p)
        assert r["status"] == 0
        assert r["interactions"] == inter0
        assert G.rel_err(r["Fr"][outside], Fr0[outside]) <= TOL


def test_shallow_tree_depth():
    pos, mass, off, adj, w = _case(3000, 8, 7, "clustered")
    for L in (1, 2, 5):
        p = FA2Params(theta=1.0, max_depth=L, leaf_cap=1)
        r = G.fa2_forces(pos, mass, off, adj, w, p)
        Fr0, inter0 = oracle.bh_repulsion(pos, mass, p)
        assert r["interactions"] == inter0
        assert G.rel_err(r["Fr"], Fr0) <= TOL


def test_theta_zero_equals_exact_all_pairs():
    pos, mass, off, adj, w = _case(1500, 9, 20, "uniform")
    r = G.fa2_forces(pos, mass, off, adj, w, FA2Params(theta=0.0))
    assert r["interactions"] == 1500 * 1499
    assert G.rel_err(r["Fr"], oracle.exact_repulsion(pos, mass, 2.0)) <= TOL


def test_error_against_exact_forces():
    # Method accuracy: at theta = 0.3 the 99th percentile and aggregate errors
    # are below 1e-2; at theta = 1.2 the aggregate error is below 2e-2.
    pos, mass, off, adj, w = _case(4000, 10, 1, "uniform")
    ex = oracle.exact_repulsion(pos, mass, 2.0)
    nrm = np.linalg.norm(ex, axis=1)
    r = G.fa2_forces(pos, mass, off, adj, w, FA2Params(theta=0.3))
    rel = np.linalg.norm(r["Fr"] - ex, axis=1) / nrm
    assert np.percentile(rel, 99) <= 1e-2
    assert np.linalg.norm(r["Fr"] - ex) / np.linalg.norm(ex) <= 1e-2
    r = G.fa2_forces(pos, mass, off, adj, w, FA2Params(theta=1.2))
    assert np.linalg.norm(r["Fr"] - ex) / np.linalg.norm(ex) <= 2e-2


def test_strong_gravity_and_single_body():
    pos, mass, off, adj, w = _case(200, 11, 3, "uniform")
    p = FA2Params(strong_gravity=1, kg=0.7)
    r = G.fa2_forces(pos, mass, off, adj, w, p)
    assert G.rel_err(r["Fg"], oracle.gravity(mass, pos, 0.7, 1)) <= TOL
    one = G.fa2_forces(np.array([[3.0, 4.0]], np.float32), np.array([2], np.uint32), np.array([0, 0], np.int32),
                       np.zeros(0, np.int32), np.zeros(0, np.uint32), FA2Params())
    assert np.all(one["Fr"] == 0) and one["interactions"] == 0
    assert np.allclose(one["Fg"], [[-1.2, -1.6]], rtol=1e-6)


def _supergraph_case():
    n, e, _ = graphgen.load("sbm16")
    _, dh = oracle.sketch_degrees(e, n, 4, 4096, 1)
    lab, _ = oracle.communities(e, n, dh, 3, 64, 2, 0)
    return oracle.supergraph(e, n, lab, dh, 4, 4096, 1)


def test_one_step_matches_oracle():
    sg = _supergraph_case()
    K = sg["K"]
    pos = oracle.fa2_init(K, 1)
    p = FA2Params()
    dv = G.Fa2Device(pos, sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], p)
    dv.step()
    st = oracle.FA2State(pos)
    r0 = oracle.fa2_step(st, sg["csr_off"], sg["csr_adj"], sg["csr_w"], sg["mass"], p)
    pos1, F1, Fprev1, speed1 = dv.state()
    stats = dv.stats()
    assert stats.status == 0 and stats.interactions == r0["interactions"]
    assert G.rel_err(F1, r0["F"]) <= TOL
    assert abs(stats.S - r0["S"]) <= 1e-4 * r0["S"] and abs(stats.T - r0["T"]) <= 1e-4 * r0["T"]
    assert abs(speed1 - st.speed) <= 1e-4 * st.speed
    # displacement: compare p1 - p0 per node
    assert G.rel_err(pos1 - pos, st.pos - pos.astype(np.float64)) <= 2e-3


def test_step_from_a_mid_run_state():
    # A later state (non-zero Fprev, speed != 1) from the oracle's own run.
    sg = _supergraph_case()
    p = FA2Params()
    st = oracle.layout(sg["K"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], sg["mass"], p, 20, 2)
    pos = st.pos.astype(np.float32)
    Fprev = st.Fprev.astype(np.float32)
    st32 = oracle.FA2State(pos, Fprev, st.speed)
    r0 = oracle.fa2_step(st32, sg["csr_off"], sg["csr_adj"], sg["csr_w"], sg["mass"], p)
    dv = G.Fa2Device(pos, sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], p, Fprev=Fprev, speed=st.speed)
    dv.step()
    _, F1, _, speed1 = dv.state()
    assert dv.stats().interactions == r0["interactions"]
    assert G.rel_err(F1, r0["F"]) <= TOL
    assert abs(speed1 - st32.speed) <= 1e-3 * st32.speed


def test_steps_are_deterministic_and_graph_replay_matches():
    sg = _supergraph_case()
    pos = oracle.fa2_init(sg["K"], 4)
    p = FA2Params()
    runs = []
    for use_graph in (False, True, True):
        dv = G.Fa2Device(pos, sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], p)
        s = torch.cuda.Stream()
        dv.run(25, use_graph, stream=s)
        s.synchronize()
        runs.append(dv.state())
    for r in runs[1:]:
        assert np.array_equal(r[0], runs[0][0]) and r[3] == runs[0][3]


def test_layout_invariants_over_many_steps():
    # Trajectories are chaotic, so a long run is checked by invariants:
    # finite state, bounded speed growth, communities pulled together.
    e, memb = graphgen.planted_partition([100] * 5, 0.2, 0.002, seed=12)
    n = 500
    off, adj, w = G.csr_from_edges(e, n)
    mass = (np.diff(off) + 1).astype(np.uint32)
    dv = G.Fa2Device(oracle.fa2_init(n, 3), mass, off, adj, w, FA2Params())
    prev = 1.0
    for _ in range(60):
        dv.step()
        _, _, _, sp = dv.state()
        assert 0 < sp <= 1.5 * prev * (1 + 1e-9)
        prev = sp
    pos = dv.state()[0]
    assert np.all(np.isfinite(pos))
    cent = np.stack([pos[memb == c].mean(axis=0) for c in range(5)])
    spread = np.mean([np.linalg.norm(pos[memb == c] - cent[c], axis=1).mean() for c in range(5)])
    sep = np.mean([np.linalg.norm(cent[a] - cent[b]) for a in range(5) for b in range(a + 1, 5)])
    assert sep > 2 * spread


def test_attraction_over_uneven_rows():
    # Row shapes the attraction plan treats differently: empty rows in long
    # runs (row gaps above 255 inside one 8-entry chunk), rows on and around
    # the 8-entry chunk size, rows just under and over 33 chunks, and hubs
    # spread over hundreds of chunks.
    rng = np.random.default_rng(11)
    lengths = [3, 0, 0, 5] + [0] * 300 + [2, 1] + [0] * 1000 + [4, 8, 9, 7, 1, 16, 17, 263, 264, 265, 272, 273,
                                                              5000, 0, 12345, 1, 0, 0, 3]
    lengths += list(rng.integers(0, 40, 3000)) + [0] * 500 + [6]
    K = len(lengths)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
    adj = rng.integers(0, K, off[-1]).astype(np.int32)
    w = rng.integers(1, 5, off[-1]).astype(np.uint32)
    pos = (rng.random((K, 2)) * 200 - 100).astype(np.float32)
    mass = np.ones(K, np.uint32)
    r = G.fa2_forces(pos, mass, off, adj, w, FA2Params())
    assert r["status"] == 0
    assert G.rel_err(r["Fa"], oracle.attraction(off, adj, w, pos)) <= TOL
    empty = np.diff(off) == 0
    assert np.all(r["Fa"][empty] == 0.0)


def _swing_traction_products(F, Fprev, mass):
    """The per-node FP32 products the step sums: m |F - Fprev| and
    (m / 2) |F + Fprev|, with the kernel's rounding steps."""
    f32 = np.float32
    F, Fp, m = F.astype(f32), Fprev.astype(f32), mass.astype(f32)
    sx, sy = F[:, 0] - Fp[:, 0], F[:, 1] - Fp[:, 1]
    tx, ty = F[:, 0] + Fp[:, 0], F[:, 1] + Fp[:, 1]
    return m * np.sqrt(sx * sx + sy * sy), (f32(0.5) * m) * np.sqrt(tx * tx + ty * ty)


def test_swing_and_traction_sums_are_exact():
    # The global swing S and traction T that set the adaptive speed are the
    # sums of FP32 per-node products; the step must return them to within 2
    # units in the last place of FP64 of the exact sum (math.fsum is
    # correctly rounded).  The case loses digits in a plain sum: node 0
    # carries a product ~1e21 whose FP64 spacing exceeds each of the other
    # 150,000 products, so adding them one by one after it drops them all.
    import math
    K = 150_000
    rng = np.random.default_rng(21)
    pos = (rng.random((K, 2)) * 2000 - 1000).astype(np.float32)
    mass = rng.integers(1, 4, K).astype(np.uint32)
    mass[0] = 4_000_000_000
    Fprev = (rng.normal(size=(K, 2)) * 10.0 ** rng.uniform(-6, 3, (K, 1))).astype(np.float32)
    Fprev[0] = [3e11, -2e11]
    off, adj, w = G.csr_from_edges(graphgen.random_graph(K, 2 * K, seed=22), K)
    dv = G.Fa2Device(pos, mass, off, adj, w, FA2Params(), Fprev=Fprev, speed=1.0)
    dv.step()
    st = dv.stats()
    assert st.status == 0
    _, F1, _, speed1 = dv.state()
    msw, mtr = _swing_traction_products(F1, Fprev, mass)
    S, T = math.fsum(msw.astype(np.float64)), math.fsum(mtr.astype(np.float64))
    assert abs(st.S - S) <= 2 * math.ulp(S)
    assert abs(st.T - T) <= 2 * math.ulp(T)
    # the case is one a plain running sum gets wrong by far more
    naive = 0.0
    for x in msw.astype(np.float64):
        naive += x
    assert abs(naive - S) > 16 * math.ulp(S)
    # the speed follows from S and T in FP64 (50 % rise cap)
    sp = 1.0
    target = 1.0 * st.T / st.S
    assert speed1 == sp + min(target - sp, 0.5 * sp)


def test_swing_and_traction_sums_of_a_supergraph_step():
    # The same property on a step of the method's own state (sbm16
    # supergraph, 20 steps in).
    import math
    sg = _supergraph_case()
    p = FA2Params()
    dv = G.Fa2Device(oracle.fa2_init(sg["K"], 2), sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], p)
    dv.run(20, False)
    Fprev = G.host(dv.Fprev).copy()
    dv.step()
    st = dv.stats()
    F1 = G.host(dv.F)
    msw, mtr = _swing_traction_products(F1, Fprev, sg["mass"])
    S, T = math.fsum(msw.astype(np.float64)), math.fsum(mtr.astype(np.float64))
    assert abs(st.S - S) <= 2 * math.ulp(S) and abs(st.T - T) <= 2 * math.ulp(T)


def test_fa2_autotuner_keeps_results():
    # The launch-shape autotuner times steps on the caller's supergraph and
    # leaves its choice in force.  Traversal block size and tail grid do not
    # change any result; the row split of the attraction only regroups some
    # FP32 row sums.
    pos, mass, off, adj, w = _case(20011, 31, 9, "clustered")
    K, nnz = pos.shape[0], int(off[-1])
    p = FA2Params()
    ws = B.alloc_ws(B.bgv_autotune_fa2_ws_size(K, nnz))
    O, A, W = G._csr_dev(off, adj, w)
    try:
        r = B.bgv_autotune_fa2(K, nnz, O, A, W, G.dev(mass), G.fa2_params(p), G.dev(pos), ws)
        assert r.att_short in (8, 16, 32) and r.repulse_threads in (128, 256)
        assert r.tail_blocks_per_sm in (2, 4, 8)
        assert min(r.ms_att_short) > 0 and min(r.ms_repulse_threads) > 0 and min(r.ms_tail_blocks) > 0
        runs = {}
        for shape in [(32, 256, 4), (32, 128, 2), (32, 256, 8), (8, 256, 4), (16, 128, 4)]:
            B.bgv_set_fa2_tune(*shape)
            f = G.fa2_forces(pos, mass, off, adj, w, p)
            dv = G.Fa2Device(pos, mass, off, adj, w, p)
            dv.run(3, True)
            runs[shape] = (f, dv.state())
        base_f, base_s = runs[(32, 256, 4)]
        for shape, (f, st) in runs.items():
            assert f["interactions"] == base_f["interactions"]
            assert np.array_equal(f["Fr"], base_f["Fr"]) and np.array_equal(f["Fg"], base_f["Fg"])
            if shape[0] == 32:  # same attraction split: the same trajectory
                assert np.array_equal(f["Fa"], base_f["Fa"])
                assert np.array_equal(st[0], base_s[0]) and st[3] == base_s[3]
            else:
                assert G.rel_err(f["Fa"], base_f["Fa"]) <= 1e-5
        with pytest.raises(B.BgvError):
            B.bgv_set_fa2_tune(300, 256, 4)
    finally:
        B.bgv_set_fa2_tune(32, 128, 4)


def test_sort_guard_for_one_long_unordered_run():
    # 80,000 of 200,000 bodies inside one cell of side 2^-12 of the frame:
    # after the LSD passes on the bits above 24 they form one unordered run
    # far longer than one block should sort, so the whole array is sorted
    # again instead.  The tree must still be the oracle's (equal interaction
    # counts) and the forces outside the cluster within 1e-3.
    rng = np.random.default_rng(77)
    K, Kc = 200_000, 80_000
    pos = (rng.random((K, 2)) * 2000 - 1000).astype(np.float32)
    pos[:Kc] = (np.array([123.4, -56.7]) + rng.random((Kc, 2)) * 0.004).astype(np.float32)
    pos = pos[rng.permutation(K)]
    outside = np.abs(pos[:, 0] - 123.4) > 1.0
    mass = rng.integers(1, 4, K).astype(np.uint32)
    off = np.zeros(K + 1, np.int32)
    for method in (1, 0):
        prev = B.bgv_set_sort_method(method)
        try:
            p = FA2Params(theta=1.2)
            r = G.fa2_forces(pos, mass, off, np.zeros(0, np.int32), np.zeros(0, np.uint32), p)
        finally:
            B.bgv_set_sort_method(prev)
        Fr0, inter0 = oracle.bh_repulsion(pos, mass, p)
        assert r["status"] == 0
        assert r["interactions"] == inter0, method
        assert G.rel_err(r["Fr"][outside], Fr0[outside]) <= TOL
