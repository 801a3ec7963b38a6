"""CPU oracle for the BigGraphVis hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded restatement (``bgv_oracle.c``) of what the
method computes, used to check the CUDA library.  Only the test suite, the
smoke check and the CPU-baseline leg of the benchmark may import it; the
product path never does, and this module imports nothing from the product
package.

Functions take and return NumPy arrays.  The shared library is compiled with
gcc on first use (or by :func:`build`).

Parity status per function (see the tests under ``tests/`` for the pins):

* ``sketch_degrees`` / ``exact_degrees`` -- pinned (brute force, row sums,
  collision-free instances, Cormode-Muthukrishnan bound).
* ``communities`` -- pinned (hand-computed worked example, identity cases,
  star, independent brute force, planted partition quality).
* ``supergraph`` -- pinned (brute force, cut-edge sum, worked example).
* ``bh_repulsion`` / ``fa2_step`` -- pinned (two-body closed form, theta=0
  equals exact all-pairs, Newton's third law, first-step speed, tree
  structure invariants, exact-force error bounds).
* ``modularity`` -- pinned against the double-sum definition.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import pathlib
import subprocess

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_SRC = _HERE / "bgv_oracle.c"
_LIB = _HERE / "liboracle.so"

CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]


def build(force: bool = False) -> pathlib.Path:
    """Compile ``liboracle.so`` next to the source (gcc, a second or two)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp.so")
        subprocess.run(["gcc", *CFLAGS, "-o", str(tmp), str(_SRC), "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(_LIB))
        P = C.c_void_p
        i32, i64, u32, u64, f64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
        L.orc_splitmix64.restype = u64
        L.orc_splitmix64.argtypes = [P]
        L.orc_hash_coeffs.restype = None
        L.orc_hash_coeffs.argtypes = [u64, i32, P, P]
        L.orc_hash.restype = u32
        L.orc_hash.argtypes = [u64, u64, u32, u32]
        L.orc_exact_degrees.restype = C.c_int
        L.orc_exact_degrees.argtypes = [P, i64, i32, P]
        L.orc_sketch_degrees.restype = C.c_int
        L.orc_sketch_degrees.argtypes = [P, i64, i32, i32, i32, u64, P, P]
        L.orc_communities.restype = C.c_int
        L.orc_communities.argtypes = [P, i64, i32, P, i32, u32, u32, i32, P, P]
        L.orc_communities_ex.restype = C.c_int
        L.orc_communities_ex.argtypes = [P, i64, i32, P, i32, u32, u32, i32, i32, P, P]
        L.orc_mode_degree.restype = C.c_int
        L.orc_mode_degree.argtypes = [P, i32, C.POINTER(u32)]
        L.orc_render.restype = C.c_int
        L.orc_render.argtypes = [i64, P, P, P, i32, i32, P]
        L.orc_scoda_sequential.restype = C.c_int
        L.orc_scoda_sequential.argtypes = [P, i64, i32, u32, P]
        L.orc_supergraph.restype = C.c_int
        L.orc_supergraph.argtypes = [P, i64, i32, P, P, i32, i32, u64, P, P, P, P, P, P, P, P, P, P, P, P, P]
        L.orc_modularity.restype = f64
        L.orc_modularity.argtypes = [P, i64, i32, P]
        L.orc_fa2_init.restype = None
        L.orc_fa2_init.argtypes = [i64, u64, P]
        L.orc_bh_repulsion.restype = C.c_int
        L.orc_bh_repulsion.argtypes = [i64, P, P, P, P, i64, P, P]
        L.orc_quadtree_export.restype = i64
        L.orc_quadtree_export.argtypes = [i64, P, P, i32, i32, i64, P, P, P, P, P, P, P, P, P, P]
        L.orc_exact_repulsion.restype = C.c_int
        L.orc_exact_repulsion.argtypes = [i64, P, P, f64, P]
        L.orc_attraction.restype = C.c_int
        L.orc_attraction.argtypes = [i64, P, P, P, P, P]
        L.orc_gravity.restype = C.c_int
        L.orc_gravity.argtypes = [i64, P, P, f64, i32, P]
        L.orc_colour_groups.restype = C.c_int
        L.orc_colour_groups.argtypes = [i64, P, P]
        L.orc_fa2_step.restype = C.c_int
        L.orc_fa2_step.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P]
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _chk(rc):
    if rc != 0:
        raise OracleError(f"oracle returned {rc}")


def _edges(edges):
    e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    return e, e.shape[0]


# --------------------------------------------------------------------------
# hash family, sketch, degrees
# --------------------------------------------------------------------------

def splitmix64(state: int):
    """Return ``(next_state, output)`` of one SplitMix64 step."""
    st = C.c_uint64(state)
    out = lib().orc_splitmix64(C.byref(st))
    return st.value, out


def hash_coeffs(seed: int, rows: int):
    a = np.zeros(rows, np.uint64)
    b = np.zeros(rows, np.uint64)
    lib().orc_hash_coeffs(seed, rows, _p(a), _p(b))
    return a, b


def hash_value(a: int, b: int, x: int, width: int) -> int:
    return int(lib().orc_hash(int(a), int(b), int(x), int(width)))


def exact_degrees(edges, n: int) -> np.ndarray:
    e, m = _edges(edges)
    d = np.zeros(max(n, 1), np.uint32)
    _chk(lib().orc_exact_degrees(_p(e), m, n, _p(d)))
    return d[:n]


def sketch_degrees(edges, n: int, rows: int, width: int, seed: int):
    """Degree count-min sketch: returns ``(S[rows, width], dhat[n])``."""
    e, m = _edges(edges)
    S = np.zeros((rows, width), np.uint32)
    d = np.zeros(max(n, 1), np.uint32)
    _chk(lib().orc_sketch_degrees(_p(e), m, n, rows, width, seed, _p(S), _p(d)))
    return S, d[:n]


def communities(edges, n: int, dhat, passes: int, threshold: int, growth: int = 2, tie_mode: int = 0):
    """Community labels after ``passes`` synchronous rounds; returns
    ``(labels[n] int32, degrees[n] uint32)``."""
    e, m = _edges(edges)
    dh = np.ascontiguousarray(dhat, dtype=np.uint32)
    lab = np.zeros(max(n, 1), np.int32)
    deg = np.zeros(max(n, 1), np.uint32)
    _chk(lib().orc_communities(_p(e), m, n, _p(dh), passes, threshold, growth, tie_mode, _p(lab), _p(deg)))
    return lab[:n], deg[:n]


def communities_ex(edges, n: int, dhat, passes: int, threshold: int, growth: int, tie_mode: int, jumps: int):
    """Community rounds with the variants: ``growth`` 0 multiplies the
    threshold by its first value each round (the delta^i schedule), and
    ``jumps`` pointer-jumping steps follow every round.  Returns
    ``(labels, degrees)``."""
    e, m = _edges(edges)
    dh = np.ascontiguousarray(dhat, dtype=np.uint32)
    lab = np.zeros(max(n, 1), np.int32)
    deg = np.zeros(max(n, 1), np.uint32)
    _chk(lib().orc_communities_ex(_p(e), m, n, _p(dh), passes, threshold, growth, tie_mode, jumps, _p(lab),
                                  _p(deg)))
    return lab[:n], deg[:n]


def mode_degree(dhat) -> int:
    """Most frequent value of dhat among nodes with dhat >= 1 (ties: the
    smaller value; 0 if there is none)."""
    dh = np.ascontiguousarray(dhat, dtype=np.uint32)
    out = C.c_uint32(0)
    _chk(lib().orc_mode_degree(_p(dh), dh.shape[0], C.byref(out)))
    return int(out.value)


def scoda_sequential(edges, n: int, D: int):
    """Sequential SCoDA (one ordered pass, degrees from 0); returns labels."""
    e, m = _edges(edges)
    lab = np.zeros(max(n, 1), np.int32)
    _chk(lib().orc_scoda_sequential(_p(e), m, n, D, _p(lab)))
    return lab[:n]


def supergraph(edges, n: int, labels, dhat, rows: int, width: int, seed: int):
    """Supergraph of the labelled graph; returns a dict with ``node_map, K,
    src, dst, w, Es, mass, vol, count, comm_label, csr_off, csr_adj, csr_w``."""
    e, m = _edges(edges)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    dh = np.ascontiguousarray(dhat, dtype=np.uint32)
    nn = max(n, 1)
    mm = max(m, 1)
    node_map = np.zeros(nn, np.int32)
    K = C.c_int64(0)
    Es = C.c_int64(0)
    src = np.zeros(mm, np.int32)
    dst = np.zeros(mm, np.int32)
    w = np.zeros(mm, np.uint32)
    mass = np.zeros(nn, np.uint32)
    vol = np.zeros(nn, np.uint64)
    cnt = np.zeros(nn, np.uint32)
    cl = np.zeros(nn, np.int32)
    off = np.zeros(nn + 1, np.int32)
    adj = np.zeros(2 * mm, np.int32)
    cw = np.zeros(2 * mm, np.uint32)
    _chk(lib().orc_supergraph(_p(e), m, n, _p(lab), _p(dh), rows, width, seed, _p(node_map), C.byref(K),
                              _p(src), _p(dst), _p(w), C.byref(Es), _p(mass), _p(vol), _p(cnt), _p(cl),
                              _p(off), _p(adj), _p(cw)))
    k, es = K.value, Es.value
    return dict(node_map=node_map[:n], K=k, src=src[:es], dst=dst[:es], w=w[:es], Es=es, mass=mass[:k],
                vol=vol[:k], count=cnt[:k], comm_label=cl[:k], csr_off=off[:k + 1], csr_adj=adj[:2 * es],
                csr_w=cw[:2 * es])


def colour_groups(sizes) -> np.ndarray:
    """Section 4.3 colour group (0 = the small half, 1..10 by size) per community."""
    sz = np.ascontiguousarray(sizes, dtype=np.uint32)
    g = np.zeros(max(sz.shape[0], 1), np.uint8)
    _chk(lib().orc_colour_groups(sz.shape[0], _p(sz), _p(g)))
    return g[:sz.shape[0]]


def modularity(edges, n: int, labels) -> float:
    e, m = _edges(edges)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    return float(lib().orc_modularity(_p(e), m, n, _p(lab)))


# --------------------------------------------------------------------------
# ForceAtlas2
# --------------------------------------------------------------------------

class _CParams(C.Structure):
    _fields_ = [("theta", C.c_double), ("kr", C.c_double), ("kg", C.c_double), ("tau", C.c_double),
                ("ks", C.c_double), ("ksmax", C.c_double), ("strong_gravity", C.c_int32),
                ("leaf_cap", C.c_int32), ("max_depth", C.c_int32), ("reserved", C.c_int32)]


@dataclasses.dataclass
class FA2Params:
    theta: float = 1.2
    kr: float = 2.0
    kg: float = 1.0
    tau: float = 1.0
    ks: float = 0.1
    ksmax: float = 10.0
    strong_gravity: int = 0
    leaf_cap: int = 1
    max_depth: int = 24

    def c(self):
        return _CParams(self.theta, self.kr, self.kg, self.tau, self.ks, self.ksmax, self.strong_gravity,
                        self.leaf_cap, self.max_depth, 0)


def fa2_init(K: int, seed: int) -> np.ndarray:
    """Initial FP32 positions, shape [K, 2]."""
    pos = np.zeros((max(K, 1), 2), np.float32)
    lib().orc_fa2_init(K, seed, _p(pos))
    return pos[:K]


def _pos64(pos):
    return np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 2))


def bh_repulsion(pos, mass, params: FA2Params, which=None):
    """Barnes-Hut repulsion; returns ``(Fr[k, 2] float64, interactions)``."""
    P = _pos64(pos)
    K = P.shape[0]
    ms = np.ascontiguousarray(mass, dtype=np.uint32)
    cp = params.c()
    inter = C.c_int64(0)
    if which is None:
        out = np.zeros((max(K, 1), 2), np.float64)
        _chk(lib().orc_bh_repulsion(K, _p(P), _p(ms), C.byref(cp), None, 0, _p(out), C.byref(inter)))
        return out[:K], inter.value
    wh = np.ascontiguousarray(which, dtype=np.int64)
    out = np.zeros((max(wh.shape[0], 1), 2), np.float64)
    _chk(lib().orc_bh_repulsion(K, _p(P), _p(ms), C.byref(cp), _p(wh), wh.shape[0], _p(out), C.byref(inter)))
    return out[:wh.shape[0]], inter.value


def quadtree_export(pos, mass, leaf_cap: int = 1, max_depth: int = 24):
    """The literal quadtree as a dict of per-cell arrays plus ``order`` and
    ``frame = (lo_x, lo_y, side)``."""
    P = _pos64(pos)
    K = P.shape[0]
    ms = np.ascontiguousarray(mass, dtype=np.uint32)
    cap = max(4 * K * max_depth + 8, 64)
    level = np.zeros(cap, np.int32)
    leaf = np.zeros(cap, np.int32)
    st = np.zeros(cap, np.int64)
    en = np.zeros(cap, np.int64)
    ch = np.zeros(4 * cap, np.int32)
    cm = np.zeros(cap, np.uint64)
    com = np.zeros(2 * cap, np.float64)
    dcom = np.zeros(2 * cap, np.float32)
    order = np.zeros(max(K, 1), np.int64)
    frame = np.zeros(3, np.float32)
    nc = lib().orc_quadtree_export(K, _p(P), _p(ms), leaf_cap, max_depth, cap, _p(level), _p(leaf), _p(st),
                                   _p(en), _p(ch), _p(cm), _p(com), _p(dcom), _p(order), _p(frame))
    if nc < 0:
        raise OracleError(f"quadtree_export failed ({nc})")
    return dict(n=nc, level=level[:nc], is_leaf=leaf[:nc], start=st[:nc], end=en[:nc],
                child=ch[:4 * nc].reshape(nc, 4), mass=cm[:nc], com=com[:2 * nc].reshape(nc, 2),
                dcom=dcom[:2 * nc].reshape(nc, 2), order=order[:K], frame=frame)


def exact_repulsion(pos, mass, kr: float) -> np.ndarray:
    P = _pos64(pos)
    K = P.shape[0]
    ms = np.ascontiguousarray(mass, dtype=np.uint32)
    out = np.zeros((max(K, 1), 2), np.float64)
    _chk(lib().orc_exact_repulsion(K, _p(P), _p(ms), kr, _p(out)))
    return out[:K]


def attraction(csr_off, csr_adj, csr_w, pos) -> np.ndarray:
    P = _pos64(pos)
    K = P.shape[0]
    off = np.ascontiguousarray(csr_off, dtype=np.int32)
    adj = np.ascontiguousarray(csr_adj, dtype=np.int32)
    w = np.ascontiguousarray(csr_w, dtype=np.uint32)
    out = np.zeros((max(K, 1), 2), np.float64)
    _chk(lib().orc_attraction(K, _p(off), _p(adj), _p(w), _p(P), _p(out)))
    return out[:K]


def gravity(mass, pos, kg: float, strong: int = 0) -> np.ndarray:
    P = _pos64(pos)
    K = P.shape[0]
    ms = np.ascontiguousarray(mass, dtype=np.uint32)
    out = np.zeros((max(K, 1), 2), np.float64)
    _chk(lib().orc_gravity(K, _p(ms), _p(P), kg, strong, _p(out)))
    return out[:K]


class FA2State:
    """FP64 ForceAtlas2 state: positions, previous forces, global speed."""

    def __init__(self, pos, Fprev=None, speed: float = 1.0):
        self.pos = _pos64(pos).copy()
        K = self.pos.shape[0]
        self.Fprev = np.zeros((K, 2), np.float64) if Fprev is None else _pos64(Fprev).copy()
        self.speed = float(speed)


def fa2_step(state: FA2State, csr_off, csr_adj, csr_w, mass, params: FA2Params):
    """One FA2 iteration in place; returns ``dict(F, S, T, interactions)``."""
    K = state.pos.shape[0]
    off = np.ascontiguousarray(csr_off, dtype=np.int32)
    adj = np.ascontiguousarray(csr_adj, dtype=np.int32)
    w = np.ascontiguousarray(csr_w, dtype=np.uint32)
    ms = np.ascontiguousarray(mass, dtype=np.uint32)
    cp = params.c()
    sp = C.c_double(state.speed)
    F = np.zeros((max(K, 1), 2), np.float64)
    ST = np.zeros(2, np.float64)
    inter = C.c_int64(0)
    _chk(lib().orc_fa2_step(K, _p(off), _p(adj), _p(w), _p(ms), C.byref(cp), _p(state.pos), _p(state.Fprev),
                            C.byref(sp), _p(F), _p(ST), C.byref(inter)))
    state.speed = sp.value
    return dict(F=F[:K], S=float(ST[0]), T=float(ST[1]), interactions=inter.value)


def layout(K: int, csr_off, csr_adj, csr_w, mass, params: FA2Params, iterations: int, seed: int):
    """Initial positions then ``iterations`` FA2 steps; returns the state."""
    st = FA2State(fa2_init(K, seed))
    for _ in range(iterations):
        fa2_step(st, csr_off, csr_adj, csr_w, mass, params)
    return st


def render(xy, radius, group, W: int, H: int):
    """RGBA image [H][W][4] uint8 of the discs (Section 4.1 radii, Section 4.3
    colour groups), pixel by pixel over all discs."""
    xy = np.ascontiguousarray(np.asarray(xy, np.float32).reshape(-1, 2))
    r = np.ascontiguousarray(radius, dtype=np.float32)
    g = np.ascontiguousarray(group, dtype=np.uint8)
    out = np.zeros((H, W, 4), np.uint8)
    _chk(lib().orc_render(xy.shape[0], _p(xy), _p(r), _p(g), W, H, _p(out)))
    return out
