"""The hinted sort (the Morton order of the ForceAtlas2 bodies from the
previous step's order) through the C ABI.

The order it must produce is the plain definition: the pairs (key, id)
sorted by key, then id, which NumPy's lexsort gives directly.  The hint only
guides the work, so every hint (perfect, reversed, random, adversarial for
the bucket choice) must give that same order, bit for bit; in the
ForceAtlas2 runs the hinted order must leave every trajectory bit for bit
equal to the full radix sort's (whose steps the oracle tests pin)."""
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


def _expected(keys):
    ids = np.arange(keys.shape[0], dtype=np.uint32)
    o = np.lexsort((ids, keys))
    return keys[o], ids[o]


def _sort(keys, hint):
    K = keys.shape[0]
    ok, oi = G.empty(K, np.uint64), G.empty(K, np.uint32)
    ws = B.alloc_ws(B.bgv_sort_hinted_ws_size(K))
    B.bgv_sort_hinted(G.dev(keys), G.dev(hint.astype(np.uint32)), K, ok, oi, ws)
    return G.host(ok, np.uint64, K), G.host(oi, np.uint32, K)


def _shape(K):
    """Buckets, samples per bucket and sample count the library uses."""
    nb = max(1, -(-K // 1024))
    s = min(8, max(1, 4096 // nb))
    return nb, s, (nb * s if nb > 1 else 0)


def _hints(keys, rng):
    K = keys.shape[0]
    exact = np.lexsort((np.arange(K), keys)).astype(np.uint32)
    near = exact.copy()
    if K > 1:  # local disorder and a few long moves, as between two steps
        for _ in range(K // 8):
            i = rng.integers(0, K)
            j = min(K - 1, max(0, i + int(rng.integers(-300, 301))))
            near[i], near[j] = near[j], near[i]
        for _ in range(max(1, K // 1000)):
            i, j = rng.integers(0, K, 2)
            near[i], near[j] = near[j], near[i]
    hints = {"identity": np.arange(K, dtype=np.uint32), "exact": exact, "reversed": exact[::-1].copy(),
             "random": rng.permutation(K).astype(np.uint32), "near": near}
    nb, s, ns = _shape(K)
    if ns:
        # every sampled place holds one of the smallest pairs: all splitters
        # fall at the bottom and the last bucket takes nearly everything
        p = ((2 * np.arange(ns, dtype=np.int64) + 1) * K) // (2 * ns)
        adv = np.empty(K, np.uint32)
        rest = np.ones(K, bool)
        rest[p] = False
        adv[p] = exact[:ns]
        adv[rest] = rng.permutation(exact[ns:])
        hints["adversarial"] = adv
    return hints


KEY_KINDS = ["wide", "huge", "dups", "equal"]


def _keys(K, kind, rng):
    if kind == "wide":
        return rng.integers(0, 1 << 48, K, dtype=np.uint64)
    if kind == "huge":  # spans too wide for one sort word: buckets sorted as (key, id) pairs
        return rng.integers(0, np.iinfo(np.uint64).max, K, dtype=np.uint64, endpoint=True)
    if kind == "dups":
        return rng.integers(0, max(1, K // 7), K, dtype=np.uint64) << np.uint64(20)
    return np.full(K, 12345, np.uint64)


@pytest.mark.parametrize("K", [1, 2, 7, 1023, 1024, 1025, 2049, 5000, 65537, 200003])
@pytest.mark.parametrize("kind", KEY_KINDS)
def test_hinted_sort_equals_key_id_order(K, kind):
    rng = np.random.default_rng(K * 7 + KEY_KINDS.index(kind))
    keys = _keys(K, kind, rng)
    ek, ei = _expected(keys)
    for name, hint in _hints(keys, rng).items():
        k, i = _sort(keys, hint)
        assert np.array_equal(k, ek) and np.array_equal(i, ei), (K, kind, name)


def test_hinted_sort_at_the_size_limit_and_above():
    K = B.bgv_sort_hinted_max_keys()
    assert K == 4096 * 1024
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 1 << 48, K, dtype=np.uint64)
    ek, ei = _expected(keys)
    exact = np.lexsort((np.arange(K), keys)).astype(np.uint32)
    # local disorder of a few hundred places, then a few long moves
    hint = exact[np.argsort(np.arange(K) + rng.integers(-300, 301, K), kind="stable")]
    for i, j in rng.integers(0, K, (K // 1000, 2)):
        hint[i], hint[j] = hint[j], hint[i]
    assert np.array_equal(np.sort(hint), np.arange(K, dtype=np.uint32))
    k, i = _sort(keys, hint)
    assert np.array_equal(k, ek) and np.array_equal(i, ei)
    assert B.bgv_sort_hinted_ws_size(K + 1) == 0
    with pytest.raises(B.BgvError):
        _sort(np.zeros(K + 1, np.uint64), np.arange(K + 1, dtype=np.uint32))


def test_bad_arguments_are_refused_on_the_host():
    K = 3000
    keys = G.dev(np.arange(K, dtype=np.uint64))
    hint = G.dev(np.arange(K, dtype=np.uint32))
    ok, oi = G.empty(K + 1, np.uint64), G.empty(K, np.uint32)
    ws = B.alloc_ws(B.bgv_sort_hinted_ws_size(K))
    lib, P = B._lib, B._p
    n = B.bgv_sort_hinted_ws_size(K)
    # misaligned output, output aliasing the keys, a short workspace, a null hint
    assert lib.bgv_sort_hinted(P(keys), P(hint), K, ok.data_ptr() + 4, P(oi), P(ws), n, None) == B.BGV_EINVAL
    assert lib.bgv_sort_hinted(P(keys), P(hint), K, P(keys), P(oi), P(ws), n, None) == B.BGV_EINVAL
    assert lib.bgv_sort_hinted(P(keys), P(hint), K, P(ok), P(oi), P(ws), n - 256, None) == B.BGV_ENOSPC
    assert lib.bgv_sort_hinted(P(keys), None, K, P(ok), P(oi), P(ws), n, None) == B.BGV_EINVAL
    assert B.bgv_status(ws) == 0


def test_hint_entry_out_of_range_is_reported():
    K = 5000
    keys = np.random.default_rng(1).integers(0, 1 << 40, K, dtype=np.uint64)
    hint = np.arange(K, dtype=np.uint32)
    hint[17] = K + 3
    ws = B.alloc_ws(B.bgv_sort_hinted_ws_size(K))
    ok, oi = G.empty(K, np.uint64), G.empty(K, np.uint32)
    with pytest.raises(B.BgvError):
        B.bgv_sort_hinted(G.dev(keys), G.dev(hint), K, ok, oi, ws)
    assert B.bgv_status(ws) & B.BGV_DEV_BADHINT
    # the context is still usable
    k, i = _sort(keys, np.arange(K, dtype=np.uint32))
    ek, ei = _expected(keys)
    assert np.array_equal(k, ek) and np.array_equal(i, ei)


def _run(sg, pos, iterations, use_graph, order):
    prev = B.bgv_set_fa2_order(order)
    try:
        dv = G.Fa2Device(pos, sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], FA2Params())
        s = torch.cuda.Stream()
        dv.run(iterations, use_graph, stream=s)
        s.synchronize()
        return dv.state(), dv.stats()
    finally:
        assert B.bgv_set_fa2_order(prev) == order


def _sg(n_blocks, seed):
    e, _ = graphgen.planted_partition([400] * n_blocks, 0.02, 0.0005, seed=seed)
    n = 400 * n_blocks
    _, dh = oracle.sketch_degrees(e, n, 4, 4096, 1)
    lab, _ = oracle.communities(e, n, dh, 1, 2, 2, 0)
    return oracle.supergraph(e, n, lab, dh, 4, 4096, 1)


@pytest.mark.parametrize("use_graph", [False, True])
def test_fa2_runs_equal_with_either_sort(use_graph):
    sg = _sg(50, 3)
    K = sg["K"]
    assert K > 4 * 1024  # several buckets
    pos = oracle.fa2_init(K, 2)
    a, sa = _run(sg, pos, 30, use_graph, 1)
    b, sb = _run(sg, pos, 30, use_graph, 0)
    assert sa.status == 0 and sb.status == 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2]) and a[3] == b[3]
    assert sa.interactions_total == sb.interactions_total and sa.tree_nodes == sb.tree_nodes


@pytest.mark.parametrize("blocks", [12, 50])
def test_a_hinted_step_matches_the_oracle(blocks):
    # A run's second step sorts with the hinted sort.  Its input state is the
    # state after the run's first step, which a one-step run reproduces (the
    # steps are deterministic); the oracle takes the same step from there.
    sg = _sg(blocks, 6)
    K = sg["K"]
    args = (sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], FA2Params())
    warm = G.Fa2Device(oracle.fa2_init(K, 8), *args)
    warm.run(6, False)
    pos0, _, Fprev0, speed0 = warm.state()
    start = dict(Fprev=Fprev0.astype(np.float32), speed=speed0)
    one = G.Fa2Device(pos0.astype(np.float32), *args, **start)
    one.run(1, False)
    pos1, _, Fprev1, speed1 = one.state()
    two = G.Fa2Device(pos0.astype(np.float32), *args, **start)
    two.run(2, False)
    st = oracle.FA2State(pos1.astype(np.float32), Fprev1.astype(np.float32), speed1)
    r0 = oracle.fa2_step(st, sg["csr_off"], sg["csr_adj"], sg["csr_w"], sg["mass"], FA2Params())
    _, F2, _, speed2 = two.state()
    stats = two.stats()
    assert stats.status == 0 and stats.interactions == r0["interactions"]
    assert G.rel_err(F2, r0["F"]) <= 1e-3
    assert abs(speed2 - st.speed) <= 1e-3 * st.speed


def test_fa2_run_with_coincident_bodies_equal_with_either_sort():
    # many bodies on one point: long runs of equal keys, split across buckets
    sg = _sg(12, 4)
    K = sg["K"]
    pos = oracle.fa2_init(K, 5).copy()
    pos[: K // 3] = pos[0]
    a, _ = _run(sg, pos, 8, True, 1)
    b, _ = _run(sg, pos, 8, True, 0)
    assert np.array_equal(a[0], b[0]) and a[3] == b[3]


def test_batched_fa2_runs_equal_with_either_sort():
    rng = np.random.default_rng(9)
    sizes = [int(k) for k in rng.integers(500, 6000, 6)]
    koff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    K = int(koff[-1])
    offs, adjs = [np.zeros(1, np.int64)], []
    for i, (k, base) in enumerate(zip(sizes, koff[:-1])):
        off, adj, _ = G.csr_from_edges(graphgen.random_graph(k, 3 * k, seed=i), k)
        offs.append(off[1:].astype(np.int64) + offs[-1][-1])
        adjs.append(adj.astype(np.int64) + base)
    off = np.concatenate(offs).astype(np.int32)
    adj = np.concatenate(adjs).astype(np.int32)
    w = np.ones(adj.shape[0], np.uint32)
    mass = (np.diff(off) + 1).astype(np.uint32)
    p = G.fa2_params(FA2Params())
    Gn, nnz = len(sizes), int(off[-1])
    out = []
    for order in (1, 0):
        prev = B.bgv_set_fa2_order(order)
        try:
            pos = torch.zeros((K, 2), dtype=torch.float32, device="cuda")
            Fprev, F = torch.zeros_like(pos), torch.zeros_like(pos)
            speed = torch.zeros(Gn, dtype=torch.float64, device="cuda")
            ws = B.alloc_ws(B.bgv_fa2_ws_size_batched(Gn, K, nnz))
            B.bgv_fa2_init_batched(Gn, koff, p, pos, Fprev, speed, ws)
            O, A, W = G._csr_dev(off, adj, w)
            B.bgv_fa2_run_batched(Gn, koff, nnz, O, A, W, G.dev(mass), p, 12, 1, pos, F, Fprev, speed, ws)
            out.append((G.host(pos).copy(), G.host(speed).copy()))
        finally:
            assert B.bgv_set_fa2_order(prev) == order
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
