"""Test helpers: run each stage of the CUDA library through the C ABI
(``paper_2108_00529_gb300.bgv``) on NumPy inputs and return NumPy outputs.

Unsigned arrays travel as same-width signed torch tensors (bit views).
"""
from __future__ import annotations

import numpy as np
import torch

from paper_2108_00529_gb300 import bgv as B

_SIGNED = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype in _SIGNED:
        a = a.view(_SIGNED[a.dtype])
    if a.size == 0:
        a = np.zeros(max(1, a.shape[-1] if a.ndim else 1), a.dtype)
    return torch.from_numpy(a.copy()).cuda()


def host(t, dtype=None, count=None):
    a = t.detach().cpu().numpy()
    if dtype is not None:
        a = a.view(dtype)
    return a if count is None else a[:count]


def empty(count, dtype):
    tdt = {np.uint32: torch.int32, np.int32: torch.int32, np.uint64: torch.int64, np.int64: torch.int64,
           np.float32: torch.float32, np.float64: torch.float64}[dtype]
    return torch.zeros(max(int(count), 1), dtype=tdt, device="cuda")


def edges_dev(e):
    e = np.ascontiguousarray(e, dtype=np.int32).reshape(-1, 2)
    t = dev(e if e.shape[0] else np.zeros((1, 2), np.int32))
    assert t.data_ptr() % 16 == 0
    return t, e.shape[0]


def sketch(e, n, rows, width, seed, stream=None):
    E, m = edges_dev(e)
    S = empty(rows * width, np.uint32)
    d = empty(n, np.uint32)
    ws = B.alloc_ws(B.bgv_sketch_degrees_ws_size(m, n, rows, width))
    B.bgv_sketch_degrees(E, m, n, rows, width, seed, S, d, ws, stream=stream)
    st = B.bgv_status(ws, stream)
    return host(S, np.uint32).reshape(rows, width), host(d, np.uint32, n), st


def communities(e, n, dhat, passes, threshold, growth=2, tie_mode=0, with_deg=True):
    E, m = edges_dev(e)
    D = dev(np.asarray(dhat, np.uint32))
    lab = empty(n, np.int32)
    deg = empty(n, np.uint32) if with_deg else None
    ws = B.alloc_ws(B.bgv_communities_ws_size(m, n))
    B.bgv_communities(E, m, n, D, passes, threshold, growth, tie_mode, lab, deg, ws)
    st = B.bgv_status(ws)
    return host(lab, None, n), (host(deg, np.uint32, n) if with_deg else None), st


def supergraph(e, n, labels, dhat, rows, width, seed, optional=True):
    E, m = edges_dev(e)
    L = dev(np.asarray(labels, np.int32))
    D = dev(np.asarray(dhat, np.uint32))
    mm = max(m, 1)
    node_map = empty(n, np.int32)
    K = empty(1, np.int64)
    Es = empty(1, np.int64)
    src, dst, w = empty(mm, np.int32), empty(mm, np.int32), empty(mm, np.uint32)
    mass = empty(n, np.uint32)
    off = empty(n + 1, np.int32)
    adj, cw = empty(2 * mm, np.int32), empty(2 * mm, np.uint32)
    vol = empty(n, np.uint64) if optional else None
    cnt = empty(n, np.uint32) if optional else None
    cl = empty(n, np.int32) if optional else None
    ws = B.alloc_ws(B.bgv_supergraph_ws_size(m, n, rows, width))
    B.bgv_supergraph(E, m, n, L, D, rows, width, seed, node_map, K, src, dst, w, Es, mass, off, adj, cw, vol, cnt,
                     cl, ws)
    st = B.bgv_status(ws)
    k = int(K.item())
    es = int(Es.item())
    out = dict(K=k, Es=es, status=st, node_map=host(node_map, None, n), src=host(src, None, es),
               dst=host(dst, None, es), w=host(w, np.uint32, es), mass=host(mass, np.uint32, k),
               csr_off=host(off, None, k + 1), csr_adj=host(adj, None, 2 * es), csr_w=host(cw, np.uint32, 2 * es))
    if optional:
        out.update(vol=host(vol, np.uint64, k), count=host(cnt, np.uint32, k), comm_label=host(cl, None, k))
    return out


def fa2_params(p):
    """C parameter struct from an ``oracle.FA2Params``-like object."""
    c = B.bgv_fa2_default_params()
    for f in ("theta", "kr", "kg", "tau", "ks", "ksmax", "strong_gravity", "leaf_cap", "max_depth"):
        if hasattr(p, f):
            setattr(c, f, getattr(p, f))
    if hasattr(p, "seed"):
        c.seed = p.seed
    return c


def _csr_dev(off, adj, w):
    return dev(np.asarray(off, np.int32)), dev(np.asarray(adj, np.int32)), dev(np.asarray(w, np.uint32))


def fa2_forces(pos, mass, off, adj, w, params):
    pos = np.ascontiguousarray(np.asarray(pos, np.float32).reshape(-1, 2))
    K = pos.shape[0]
    P = dev(pos)
    M = dev(np.asarray(mass, np.uint32))
    O, A, W = _csr_dev(off, adj, w)
    Fr, Fa, Fg = (torch.zeros((max(K, 1), 2), dtype=torch.float32, device="cuda") for _ in range(3))
    ws = B.alloc_ws(B.bgv_fa2_ws_size(K, int(np.asarray(off)[-1]) if K else 0))
    B.bgv_fa2_forces(K, int(np.asarray(off)[-1]) if K else 0, O, A, W, M, fa2_params(params), P, Fr, Fa, Fg, ws)
    st = B.bgv_fa2_read_stats(ws)
    return dict(Fr=host(Fr)[:K].astype(np.float64), Fa=host(Fa)[:K].astype(np.float64),
                Fg=host(Fg)[:K].astype(np.float64), interactions=int(st.interactions), status=int(st.status),
                tree_nodes=int(st.tree_nodes))


class Fa2Device:
    """Device FA2 state for step tests."""

    def __init__(self, pos, mass, off, adj, w, params, Fprev=None, speed=1.0):
        pos = np.ascontiguousarray(np.asarray(pos, np.float32).reshape(-1, 2))
        self.K = pos.shape[0]
        self.pos = dev(pos)
        self.F = torch.zeros_like(self.pos)
        self.Fprev = dev(np.zeros_like(pos) if Fprev is None else np.asarray(Fprev, np.float32))
        self.speed = torch.tensor([speed], dtype=torch.float64, device="cuda")
        self.mass = dev(np.asarray(mass, np.uint32))
        self.off, self.adj, self.w = _csr_dev(off, adj, w)
        self.params = fa2_params(params)
        self.nnz = int(np.asarray(off)[-1])
        self.ws = B.alloc_ws(B.bgv_fa2_ws_size(self.K, self.nnz))

    def step(self):
        B.bgv_fa2_step(self.K, self.nnz, self.off, self.adj, self.w, self.mass, self.params, self.pos, self.F, self.Fprev,
                       self.speed, self.ws)

    def run(self, iterations, use_graph, stream=None):
        B.bgv_fa2_run(self.K, self.nnz, self.off, self.adj, self.w, self.mass, self.params, iterations, use_graph, self.pos,
                      self.F, self.Fprev, self.speed, self.ws, stream=stream)

    def stats(self):
        return B.bgv_fa2_read_stats(self.ws)

    def state(self):
        return (host(self.pos).astype(np.float64), host(self.F).astype(np.float64),
                host(self.Fprev).astype(np.float64), float(self.speed.item()))


def rel_err(F, F0, floor=1e-3):
    """max over nodes of |F - F0| / max(|F0|, floor * rms |F0|)."""
    F = np.asarray(F, np.float64)
    F0 = np.asarray(F0, np.float64)
    if F0.shape[0] == 0:
        return 0.0
    nrm = np.linalg.norm(F0, axis=1)
    rms = np.sqrt(np.mean(nrm ** 2))
    den = np.maximum(nrm, floor * rms)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.linalg.norm(F - F0, axis=1) / den))


def csr_from_edges(e, n):
    """Symmetric CSR (ascending neighbours, unit weights) of a simple graph,
    built with NumPy for FA2 tests on raw graphs."""
    e = np.asarray(e, np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    d = np.concatenate([e, e[:, ::-1]])
    d = d[np.lexsort((d[:, 1], d[:, 0]))]
    off = np.concatenate([[0], np.cumsum(np.bincount(d[:, 0], minlength=n))]).astype(np.int32)
    return off, d[:, 1].astype(np.int32), np.ones(d.shape[0], np.uint32)
