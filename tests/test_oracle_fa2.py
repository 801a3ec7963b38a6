"""Pins for the oracle's ForceAtlas2 stage (Section 3.1, Algorithm 1; FA2
model of Jacomy et al. 2014; Barnes-Hut per Section 3.1).  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import FA2Params


def _uniform(K, seed, scale=100.0):
    return np.random.default_rng(seed).random((K, 2)) * scale


def test_two_bodies_closed_form():
    pos = np.array([[0.0, 0.0], [3.0, 4.0]])
    mass = np.array([2, 5], np.uint32)
    F, inter = oracle.bh_repulsion(pos, mass, FA2Params(kr=1.5))
    # |F| = kr m1 m2 / d, directed away from the other body
    mag = 1.5 * 2 * 5 / 5.0
    assert np.allclose(F[0], -mag * np.array([3.0, 4.0]) / 5.0, rtol=1e-14)
    assert np.allclose(F[1], mag * np.array([3.0, 4.0]) / 5.0, rtol=1e-14)
    assert inter == 2


@pytest.mark.parametrize("leaf_cap", [1, 3, 8])
def test_theta_zero_is_exact_all_pairs(leaf_cap):
    pos = _uniform(700, 1)
    mass = np.random.default_rng(2).integers(1, 100, 700).astype(np.uint32)
    ex = oracle.exact_repulsion(pos, mass, 2.0)
    F, inter = oracle.bh_repulsion(pos, mass, FA2Params(theta=0.0, leaf_cap=leaf_cap))
    assert inter == 700 * 699
    assert np.max(np.abs(F - ex)) <= 1e-10 * np.max(np.abs(ex))


def test_exact_repulsion_newtons_third_law():
    pos = _uniform(500, 3)
    mass = np.random.default_rng(4).integers(1, 10, 500).astype(np.uint32)
    ex = oracle.exact_repulsion(pos, mass, 2.0)
    scale = np.abs(ex).sum()
    assert np.all(np.abs(ex.sum(axis=0)) <= 1e-12 * scale)
    # direction: repulsion pushes the leftmost body further left
    assert ex[np.argmin(pos[:, 0]), 0] < 0


def test_attraction_one_edge_and_third_law():
    pos = np.array([[1.0, 2.0], [4.0, -2.0], [0.0, 0.0]])
    off = np.array([0, 1, 2, 2], np.int32)
    adj = np.array([1, 0], np.int32)
    w = np.array([3, 3], np.uint32)
    Fa = oracle.attraction(off, adj, w, pos)
    assert np.allclose(Fa[0], -3 * (pos[0] - pos[1]), rtol=1e-15)
    assert np.allclose(Fa[1], -3 * (pos[1] - pos[0]), rtol=1e-15)
    assert np.all(Fa[2] == 0)
    assert np.allclose(Fa.sum(axis=0), 0, atol=1e-12)


def test_gravity_closed_forms():
    pos = np.array([[3.0, 4.0], [0.0, 0.0], [-1.0, 0.0]])
    mass = np.array([2, 7, 1], np.uint32)
    g = oracle.gravity(mass, pos, 1.5, 0)
    assert np.allclose(g[0], -1.5 * 2 * np.array([0.6, 0.8]))
    assert np.all(g[1] == 0)
    assert np.allclose(g[2], [1.5, 0.0])
    gs = oracle.gravity(mass, pos, 1.5, 1)
    assert np.allclose(gs, -1.5 * mass[:, None] * pos)


def test_bh_accuracy_against_exact():
    # theta = 0.3: 99th percentile per-node relative error and aggregate
    # relative L2 error at most 1e-2; theta = 1.2: aggregate at most 2e-2.
    for seed, mass in [(0, None), (1, "random")]:
        pos = _uniform(3000, seed)
        m = np.ones(3000, np.uint32) if mass is None else \
            np.random.default_rng(seed).integers(1, 50, 3000).astype(np.uint32)
        ex = oracle.exact_repulsion(pos, m, 2.0)
        nrm = np.linalg.norm(ex, axis=1)
        F, _ = oracle.bh_repulsion(pos, m, FA2Params(theta=0.3))
        rel = np.linalg.norm(F - ex, axis=1) / nrm
        assert np.percentile(rel, 99) <= 1e-2
        assert np.linalg.norm(F - ex) / np.linalg.norm(ex) <= 1e-2
        F, _ = oracle.bh_repulsion(pos, m, FA2Params(theta=1.2))
        assert np.linalg.norm(F - ex) / np.linalg.norm(ex) <= 2e-2


def test_sampled_bodies_match_full_run():
    pos = _uniform(400, 5)
    mass = np.ones(400, np.uint32)
    F, _ = oracle.bh_repulsion(pos, mass, FA2Params())
    which = np.array([0, 17, 399, 5], np.int64)
    Fs, _ = oracle.bh_repulsion(pos, mass, FA2Params(), which=which)
    assert np.array_equal(Fs, F[which])


@pytest.mark.parametrize("leaf_cap,L", [(1, 24), (4, 24), (1, 3)])
def test_quadtree_structure(leaf_cap, L):
    rng = np.random.default_rng(7)
    pos = np.concatenate([rng.random((300, 2)) * 50, np.repeat([[10.0, 10.0]], 5, axis=0)])
    mass = rng.integers(1, 20, pos.shape[0]).astype(np.uint32)
    t = oracle.quadtree_export(pos, mass, leaf_cap, L)
    K = pos.shape[0]
    # every body in exactly one leaf
    cover = np.zeros(K, np.int64)
    for c in range(t["n"]):
        if t["is_leaf"][c]:
            cover[t["start"][c]:t["end"][c]] += 1
            assert t["end"][c] - t["start"][c] <= leaf_cap or t["level"][c] == L
        else:
            kids = [k for k in t["child"][c] if k >= 0]
            assert kids, "internal cell without children"
            # children partition the parent's range in order, one level down
            s = t["start"][c]
            for k in kids:
                assert t["start"][k] == s and t["level"][k] == t["level"][c] + 1
                s = t["end"][k]
            assert s == t["end"][c]
    assert np.all(cover == 1)
    assert sorted(t["order"].tolist()) == list(range(K))
    # root: total mass and the mass-weighted mean
    assert t["mass"][0] == int(mass.astype(np.int64).sum())
    assert np.allclose(t["com"][0], np.average(pos, axis=0, weights=mass.astype(np.float64)), rtol=1e-12)
    # each cell's FP64 centre equals the weighted mean of its bodies; the FP32
    # decision centre is within 2^-20 of the frame side of it
    side = float(t["frame"][2])
    for c in range(0, t["n"], 7):
        idx = t["order"][t["start"][c]:t["end"][c]]
        assert np.allclose(t["com"][c], np.average(pos[idx], axis=0, weights=mass[idx].astype(np.float64)),
                           rtol=1e-12, atol=1e-12)
        assert np.all(np.abs(t["dcom"][c] - t["com"][c]) <= side * 2.0**-20 + np.abs(t["com"][c]) * 2.0**-22)
    # bodies in a cell lie inside the cell's square
    lo = t["frame"][:2].astype(np.float64)
    for c in range(0, t["n"], 5):
        idx = t["order"][t["start"][c]:t["end"][c]]
        cs = side * 2.0**-t["level"][c]
        cell = np.floor((pos[idx] - lo) / cs)
        assert np.all(cell == cell[0])


def test_coincident_bodies_do_not_interact():
    pos = np.array([[1.0, 1.0], [1.0, 1.0], [5.0, 1.0]])
    mass = np.ones(3, np.uint32)
    F, _ = oracle.bh_repulsion(pos, mass, FA2Params(theta=0.0))
    ex = oracle.exact_repulsion(pos, mass, 2.0)
    assert np.allclose(F, ex)
    assert np.allclose(F[0], [-2.0 / 4.0, 0.0])


def test_init_positions():
    p = oracle.fa2_init(10000, 42)
    R = np.sqrt(10000.0)
    assert p.dtype == np.float32 and p.shape == (10000, 2)
    assert np.all(p >= -R) and np.all(p < R)
    assert abs(p.mean()) < 2.0 and abs(p.std() - 2 * R / np.sqrt(12)) < 1.0
    assert np.array_equal(p, oracle.fa2_init(10000, 42))
    assert not np.array_equal(p, oracle.fa2_init(10000, 43))
    # a prefix of the nodes draws the same uniforms; only the square scales
    q = oracle.fa2_init(100, 42)
    assert np.allclose((q + 10.0) / 20.0, (p[:100] + R) / (2 * R), atol=1e-6)


def _two_cliques(k):
    e = [(i, j) for i in range(k) for j in range(i + 1, k)]
    e += [(k + i, k + j) for i in range(k) for j in range(i + 1, k)]
    e += [(0, k)]
    e = np.array(e, np.int32)
    n = 2 * k
    dirs = np.concatenate([e, e[:, ::-1]])
    dirs = dirs[np.lexsort((dirs[:, 1], dirs[:, 0]))]
    off = np.concatenate([[0], np.cumsum(np.bincount(dirs[:, 0], minlength=n))]).astype(np.int32)
    return n, off, dirs[:, 1].astype(np.int32), np.ones(dirs.shape[0], np.uint32)


def test_first_step_speed_and_sums():
    n, off, adj, w = _two_cliques(6)
    mass = (np.diff(off) + 1).astype(np.uint32)
    st = oracle.FA2State(oracle.fa2_init(n, 3))
    r = oracle.fa2_step(st, off, adj, w, mass, FA2Params())
    # Fprev = 0: swing = |F|, traction = |F| / 2, so T = S / 2, target = 1/2
    S = float(np.sum(mass * np.linalg.norm(r["F"], axis=1)))
    assert r["S"] == pytest.approx(S, rel=1e-13)
    assert r["T"] == pytest.approx(S / 2, rel=1e-13)
    assert st.speed == pytest.approx(0.5, rel=1e-15)
    assert np.array_equal(st.Fprev, r["F"])


def test_speed_rise_is_capped_and_layout_separates_cliques():
    n, off, adj, w = _two_cliques(8)
    mass = (np.diff(off) + 1).astype(np.uint32)
    st = oracle.FA2State(oracle.fa2_init(n, 9))
    prev = st.speed
    for _ in range(150):
        oracle.fa2_step(st, off, adj, w, mass, FA2Params())
        assert 0 < st.speed <= 1.5 * prev * (1 + 1e-15)
        prev = st.speed
    p = st.pos
    a, b = p[:8], p[8:]
    intra = np.mean([np.linalg.norm(x - y) for x in a for y in a] + [np.linalg.norm(x - y) for x in b for y in b])
    inter = np.mean([np.linalg.norm(x - y) for x in a for y in b])
    assert inter > 1.5 * intra


def test_no_swing_keeps_speed_and_moves_by_the_cap_rule():
    # Fprev equal to this step's force: every swing is 0, so S = 0 and the
    # global speed stays as it was; traction is |F|; every node moves along F
    # by ks * speed, or by ksmax / |F| where that is smaller.
    n, off, adj, w = _two_cliques(6)
    mass = (np.diff(off) + 1).astype(np.uint32)
    p0 = oracle.fa2_init(n, 5)
    F = oracle.fa2_step(oracle.FA2State(p0), off, adj, w, mass, FA2Params())["F"]
    for ksmax in (10.0, 0.05):  # the cap binds for no node, then for some
        params = FA2Params(ks=0.1, ksmax=ksmax)
        st = oracle.FA2State(p0, Fprev=F, speed=0.7)
        r = oracle.fa2_step(st, off, adj, w, mass, params)
        assert np.array_equal(r["F"], F)
        assert r["S"] == 0.0
        nrm = np.linalg.norm(F, axis=1)
        assert r["T"] == pytest.approx(float(np.sum(mass * nrm)), rel=1e-13)
        assert st.speed == 0.7
        s = np.minimum(params.ks * 0.7, params.ksmax / nrm)
        if ksmax < 1.0:
            assert np.any(s < params.ks * 0.7)
        expected = p0.astype(np.float64) + s[:, None] * F
        assert np.allclose(st.pos, expected, rtol=1e-12, atol=1e-12 * float(np.max(np.abs(expected))))
        assert np.array_equal(st.Fprev, F)


def test_half_previous_force_gives_closed_form_speed_and_steps():
    # Fprev = F / 2: swing_i = |F_i| / 2 and traction_i = 3 |F_i| / 4, so
    # T / S = 3 / 2.  With tau = 1 and speed 0.7 the target 1.5 is more than
    # half above the speed: the rise is capped at 0.35 (new speed 1.05).
    # Each node then moves along F by ks * speed / (1 + speed * sqrt(swing))
    # at the new speed, capped at ksmax / |F|.
    n, off, adj, w = _two_cliques(6)
    mass = (np.diff(off) + 1).astype(np.uint32)
    p0 = oracle.fa2_init(n, 6)
    F = oracle.fa2_step(oracle.FA2State(p0), off, adj, w, mass, FA2Params())["F"]
    params = FA2Params(ks=0.1, ksmax=10.0, tau=1.0)
    st = oracle.FA2State(p0, Fprev=F / 2, speed=0.7)
    r = oracle.fa2_step(st, off, adj, w, mass, params)
    nrm = np.linalg.norm(F, axis=1)
    assert r["S"] == pytest.approx(float(np.sum(mass * nrm / 2)), rel=1e-13)
    assert r["T"] == pytest.approx(float(np.sum(mass * 3 * nrm / 4)), rel=1e-13)
    assert st.speed == pytest.approx(1.05, rel=1e-14)
    s = params.ks * 1.05 / (1 + 1.05 * np.sqrt(nrm / 2))
    s = np.minimum(s, params.ksmax / nrm)
    expected = p0.astype(np.float64) + s[:, None] * F
    assert np.allclose(st.pos, expected, rtol=1e-12, atol=1e-12 * float(np.max(np.abs(expected))))
