"""Seeded synthetic graph generators.

These stand in for the paper's real-world inputs (SNAP / NetworkRepository
graphs, Section "Data"), which are not available here.  The module only
*constructs inputs*: it holds none of the BigGraphVis arithmetic (no hashing,
no sketch, no community rule, no force), so both the CPU oracle tests and the
CUDA path can consume the same graphs without sharing method code.

Every generator is deterministic in its ``seed`` (NumPy PCG64).  Edge lists are
returned as C-contiguous ``int32`` arrays of shape ``[m, 2]``: one undirected
edge per row, no self-loops, no duplicate pairs, rows in random order.

Workloads (named by what they are):

* ``sbm16``  -- planted partition, 10,000 nodes in 16 communities of 625,
  independent Bernoulli per pair, p_in = 0.01, p_out = 0.0002, seed 1.
* ``rmat20`` -- R-MAT scale 20 (1,048,576 node ids), exactly 10,000,000 unique
  edges, (a, b, c, d) = (.57, .19, .19, .05), seed 2.
* ``rmat22x`` -- R-MAT scale 22 restricted to ids < 3,200,000, exactly
  34,000,000 unique edges, (a, b, c, d) = (.45, .22, .22, .11), seed 3.
* ``lnpp1m`` -- 1,000,000 nodes in 256 communities with lognormal(8, 1)
  sizes, exactly 8,000,000 unique edges, 80 % inside communities, seed 4.
"""
from __future__ import annotations

import os
import pathlib

import numpy as np

__all__ = [
    "planted_partition",
    "rmat",
    "lognormal_planted",
    "uneven_planted",
    "batch_set",
    "random_graph",
    "load",
    "WORKLOADS",
]


def _finish(u: np.ndarray, v: np.ndarray, rng: np.random.Generator, orient: bool) -> np.ndarray:
    """Stack endpoints into an [m, 2] int32 array in random row order."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if orient:
        flip = rng.random(u.shape[0]) < 0.5
        u, v = np.where(flip, v, u), np.where(flip, u, v)
    perm = rng.permutation(u.shape[0])
    e = np.empty((u.shape[0], 2), dtype=np.int32)
    e[:, 0] = u[perm]
    e[:, 1] = v[perm]
    return np.ascontiguousarray(e)


def planted_partition(sizes, p_in: float, p_out: float, seed: int):
    """Stochastic block model: every unordered pair of distinct nodes is an
    edge independently, with probability ``p_in`` inside a community and
    ``p_out`` across communities.

    Sampled block by block: the number of edges in a block is Binomial(pairs, p)
    and that many distinct pairs are drawn uniformly, which is the same
    distribution as one Bernoulli trial per pair.

    Returns ``(edges, membership)``.  Community ``c`` holds the contiguous node
    ids ``[offset_c, offset_c + sizes[c])``.
    """
    rng = np.random.default_rng(seed)
    sizes = [int(s) for s in sizes]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    us, vs = [], []
    for a, sa in enumerate(sizes):
        # inside community a: pairs i < j
        npairs = sa * (sa - 1) // 2
        cnt = rng.binomial(npairs, p_in) if npairs else 0
        if cnt:
            t = rng.choice(npairs, size=cnt, replace=False).astype(np.int64)
            i_ar = np.arange(sa, dtype=np.int64)
            row_start = i_ar * sa - i_ar * (i_ar + 1) // 2
            i = np.searchsorted(row_start, t, side="right") - 1
            j = i + 1 + (t - row_start[i])
            us.append(off[a] + i)
            vs.append(off[a] + j)
        for b in range(a + 1, len(sizes)):
            sb = sizes[b]
            npairs = sa * sb
            cnt = rng.binomial(npairs, p_out)
            if cnt:
                t = rng.choice(npairs, size=cnt, replace=False).astype(np.int64)
                us.append(off[a] + t // sb)
                vs.append(off[b] + t % sb)
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    membership = np.repeat(np.arange(len(sizes), dtype=np.int32), sizes)
    return _finish(u, v, rng, orient=True), membership


def _dedupe_first(keys_in_order: np.ndarray) -> np.ndarray:
    """Distinct values of ``keys_in_order`` kept in order of first occurrence."""
    _, first = np.unique(keys_in_order, return_index=True)
    return keys_in_order[np.sort(first)]


def rmat(scale: int, m: int, a: float, b: float, c: float, seed: int, n_limit: int | None = None):
    """R-MAT edge generator (Chakrabarti, Zhan, Faloutsos 2004).

    Each edge picks one of four quadrants per level with probabilities
    (a, b, c, d = 1 - a - b - c) for ``scale`` levels.  Self-loops and edges
    with an endpoint >= ``n_limit`` are rejected, pairs are canonicalised to
    (min, max), duplicates are dropped keeping first occurrences, and batches
    are generated until exactly ``m`` unique edges exist.  Node ids are not
    permuted; row order is shuffled.
    """
    rng = np.random.default_rng(seed)
    n = (1 << scale) if n_limit is None else int(n_limit)
    ab, abc = a + b, a + b + c
    have = np.zeros(0, dtype=np.int64)
    while have.shape[0] < m:
        need = m - have.shape[0]
        batch = int(need * 1.25) + 1024
        src = np.zeros(batch, dtype=np.int64)
        dst = np.zeros(batch, dtype=np.int64)
        for _ in range(scale):
            r = rng.random(batch)
            bs = r >= ab
            bd = ((r >= a) & (r < ab)) | (r >= abc)
            src = (src << 1) | bs
            dst = (dst << 1) | bd
        keep = (src != dst) & (src < n) & (dst < n)
        src, dst = src[keep], dst[keep]
        lo = np.minimum(src, dst)
        hi = np.maximum(src, dst)
        have = _dedupe_first(np.concatenate([have, lo * n + hi]))
    have = have[:m]
    return _finish(have // n, have % n, rng, orient=False)


def _largest_remainder(weights: np.ndarray, total: int, minimum: int) -> np.ndarray:
    """Integer sizes proportional to ``weights`` summing exactly to ``total``."""
    w = np.asarray(weights, dtype=np.float64)
    rest = total - minimum * w.shape[0]
    exact = w / w.sum() * rest
    base = np.floor(exact).astype(np.int64)
    short = rest - int(base.sum())
    order = np.argsort(-(exact - base), kind="stable")
    base[order[:short]] += 1
    return base + minimum


def uneven_planted(sizes, m: int, intra: float, seed: int, permute: bool = True):
    """Planted partition with given community ``sizes`` and exactly ``m``
    unique edges, a fraction ``intra`` of them inside communities.

    Intra edges pick a community with probability proportional to its size and
    a uniform pair of distinct nodes in it; inter edges pick a uniform pair of
    nodes in different communities.  Node ids are randomly permuted when
    ``permute`` (so ids carry no community locality).  Returns
    ``(edges, membership)``.
    """
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    n = int(sizes.sum())
    off = np.concatenate([[0], np.cumsum(sizes)])
    comm_of = np.repeat(np.arange(sizes.shape[0]), sizes)
    m_in = int(round(m * intra))
    m_out = m - m_in
    prob = sizes / sizes.sum()

    def draw_intra(k):
        cc = rng.choice(sizes.shape[0], size=k, p=prob)
        s = sizes[cc]
        i = (rng.random(k) * s).astype(np.int64)
        j = (rng.random(k) * (s - 1)).astype(np.int64)
        j = j + (j >= i)
        return off[cc] + i, off[cc] + j

    def draw_inter(k):
        i = rng.integers(0, n, size=k)
        j = rng.integers(0, n, size=k)
        ok = comm_of[i] != comm_of[j]
        return i[ok], j[ok]

    def collect(draw, target):
        have = np.zeros(0, dtype=np.int64)
        while have.shape[0] < target:
            need = target - have.shape[0]
            i, j = draw(int(need * 1.2) + 64)
            lo, hi = np.minimum(i, j), np.maximum(i, j)
            have = _dedupe_first(np.concatenate([have, lo * n + hi]))
        return have[:target]

    k_in = collect(draw_intra, m_in)
    k_out = collect(draw_inter, m_out)
    keys = np.concatenate([k_in, k_out])
    u, v = keys // n, keys % n
    membership = comm_of.astype(np.int32)
    if permute:
        perm = rng.permutation(n)
        u, v = perm[u], perm[v]
        inv = np.empty(n, dtype=np.int32)
        inv[perm] = membership
        membership = inv
    return _finish(u, v, rng, orient=True), membership


def lognormal_planted(n: int = 1_000_000, k: int = 256, m: int = 8_000_000, mu: float = 8.0,
                      sigma: float = 1.0, intra: float = 0.8, seed: int = 4):
    """``k`` communities with lognormal(mu, sigma) sizes rescaled to sum to
    exactly ``n`` (largest remainder, at least 2 nodes each), then
    :func:`uneven_planted` with ``m`` edges."""
    rng = np.random.default_rng(seed)
    raw = rng.lognormal(mu, sigma, size=k)
    sizes = _largest_remainder(raw, n, 2)
    return uneven_planted(sizes, m, intra, seed + 7919)


def batch_set(count: int = 512, n_lo: int = 1000, n_hi: int = 200_000, k_lo: int = 4, k_hi: int = 64,
              avg_degree: float = 10.0, intra: float = 0.8, seed0: int = 1000):
    """``count`` independent planted-partition graphs of uneven size: graph g
    uses seed ``seed0 + g``, n log-uniform in [n_lo, n_hi], k uniform in
    [k_lo, k_hi], m = n * avg_degree / 2 edges, lognormal(0, 0.5) community
    sizes.  Returns a list of ``(edges, membership)``."""
    out = []
    for g in range(count):
        rng = np.random.default_rng(seed0 + g)
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        k = int(rng.integers(k_lo, k_hi + 1))
        sizes = _largest_remainder(rng.lognormal(0.0, 0.5, size=k), n, 2)
        m = int(n * avg_degree / 2)
        out.append(uneven_planted(sizes, m, intra, seed0 + g + 100_000))
    return out


def random_graph(n: int, m: int, seed: int, self_loops: int = 0) -> np.ndarray:
    """Uniform random simple graph with ``n`` nodes and ``m`` distinct edges
    (``m`` capped at n(n-1)/2), plus ``self_loops`` loop rows (u, u) appended
    before shuffling.  For small parity and edge-case tests."""
    rng = np.random.default_rng(seed)
    m = min(m, n * (n - 1) // 2)
    have = np.zeros(0, dtype=np.int64)
    while have.shape[0] < m:
        i = rng.integers(0, n, size=2 * (m - have.shape[0]) + 8)
        j = rng.integers(0, n, size=i.shape[0])
        ok = i != j
        lo, hi = np.minimum(i[ok], j[ok]), np.maximum(i[ok], j[ok])
        have = _dedupe_first(np.concatenate([have, lo * n + hi]))
    have = have[:m]
    u, v = have // max(n, 1), have % max(n, 1)
    if self_loops:
        w = rng.integers(0, n, size=self_loops)
        u = np.concatenate([u, w])
        v = np.concatenate([v, w])
    return _finish(u, v, rng, orient=True)


def _sbm16():
    return planted_partition([625] * 16, 0.01, 0.0002, seed=1)


def _rmat20():
    return rmat(20, 10_000_000, 0.57, 0.19, 0.19, seed=2), None


def _rmat22x():
    return rmat(22, 34_000_000, 0.45, 0.22, 0.22, seed=3, n_limit=3_200_000), None


def _lnpp1m():
    return lognormal_planted()


#: name -> (node count, generator returning (edges, membership or None))
WORKLOADS = {
    "sbm16": (10_000, _sbm16),
    "rmat20": (1 << 20, _rmat20),
    "rmat22x": (3_200_000, _rmat22x),
    "lnpp1m": (1_000_000, _lnpp1m),
}


def _cache_dir() -> pathlib.Path:
    d = os.environ.get("BGV_CACHE_DIR")
    if d:
        p = pathlib.Path(d)
    else:
        p = pathlib.Path(__file__).resolve().parent.parent / "_cache"
    p.mkdir(parents=True, exist_ok=True)
    return p


def load(name: str):
    """Return ``(n, edges, membership)`` for a named workload, generating it
    once and caching it as ``.npy`` files."""
    n, fn = WORKLOADS[name]
    d = _cache_dir()
    fe, fm = d / f"{name}.edges.npy", d / f"{name}.membership.npy"
    if fe.exists():
        edges = np.load(fe)
        memb = np.load(fm) if fm.exists() else None
        return n, edges, memb
    edges, memb = fn()
    tmp = d / f"{name}.edges.tmp.npy"
    np.save(tmp, edges)
    if memb is not None:
        np.save(fm, memb)
    os.replace(tmp, fe)
    return n, edges, memb


def load_batch(name: str = "batch512"):
    """The 512-graph batching workload (``batch_set()`` with its defaults),
    joined for the batched entry point: returns ``(edges, edge_off,
    node_off)`` -- the concatenated int32 edge lists in LOCAL node ids, int64
    edge offsets and int32 node offsets, each offset array of length G + 1.
    Cached as one ``.npz`` file."""
    if name != "batch512":
        raise KeyError(name)
    f = _cache_dir() / f"{name}.npz"
    if f.exists():
        z = np.load(f)
        return z["edges"], z["edge_off"], z["node_off"]
    graphs = batch_set()
    edges = np.concatenate([e for e, _ in graphs]).astype(np.int32)
    edge_off = np.concatenate([[0], np.cumsum([e.shape[0] for e, _ in graphs])]).astype(np.int64)
    node_off = np.concatenate([[0], np.cumsum([mem.shape[0] for _, mem in graphs])]).astype(np.int32)
    tmp = _cache_dir() / f"{name}.tmp.npz"
    np.savez(tmp, edges=edges, edge_off=edge_off, node_off=node_off)
    os.replace(tmp, f)
    return edges, edge_off, node_off
