"""Thin ctypes binding of libbgv.so (the C ABI declared in include/bgv.h).

Argument marshalling only: every function has the C name, converts torch
tensors to their device pointers (``None`` -> NULL), passes the current CUDA
stream when none is given, and raises :class:`BgvError` on a non-zero return
code.  All work happens in the CUDA kernels of the library.  Importing this
module raises if the library has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import pathlib

import numpy as np
import torch

_LIB_PATH = pathlib.Path(__file__).resolve().parent / "libbgv.so"
if not _LIB_PATH.exists():
    raise ImportError(f"libbgv.so not found at {_LIB_PATH}; build it with paper_2108_00529_gb300.build.build()")
_lib = C.CDLL(str(_LIB_PATH))

BGV_OK, BGV_EINVAL, BGV_ENOSPC, BGV_EDEVICE, BGV_ECUDA, BGV_ELIMIT = 0, 1, 2, 3, 4, 5
BGV_DEV_BADEDGE, BGV_DEV_BADLABEL, BGV_DEV_TIMEOUT, BGV_DEV_BADHINT = 1, 2, 8, 16

P = C.c_void_p
i32, i64, u32, u64, sz = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_size_t


class bgv_fa2_params(C.Structure):
    _fields_ = [("theta", C.c_float), ("kr", C.c_float), ("kg", C.c_float), ("tau", C.c_float),
                ("ks", C.c_float), ("ksmax", C.c_float), ("strong_gravity", i32), ("leaf_cap", i32),
                ("max_depth", i32), ("reserved", i32), ("seed", u64)]


class bgv_fa2_stats(C.Structure):
    _fields_ = [("S", C.c_double), ("T", C.c_double), ("interactions", u64), ("tree_nodes", u64),
                ("interactions_total", u64), ("steps_total", u64), ("status", u32), ("reserved", u32)]


class bgv_tune_report(C.Structure):
    _fields_ = [("count", i32), ("sizes_log2", i32 * 9), ("ms8", C.c_float * 9), ("ms16", C.c_float * 9),
                ("ms_coop", C.c_float * 9), ("method", i32), ("cutoff", i64), ("coop_lo", i64), ("coop_hi", i64)]


class bgv_layout_params(C.Structure):
    _fields_ = [("rows", i32), ("width", i32), ("seed", u64), ("passes", i32), ("threshold", u32),
                ("growth", u32), ("tie_mode", i32), ("threshold_mode", i32), ("jumps", i32), ("iterations", i32),
                ("use_graph", i32), ("fa2", bgv_fa2_params)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("bgv_version", C.c_int, [])
_sig("bgv_strerror", C.c_char_p, [C.c_int])
_sig("bgv_ws_init", C.c_int, [P, P])
_sig("bgv_status", C.c_int, [P, P, C.POINTER(u32), C.c_int])
_sig("bgv_sketch_degrees_ws_size", sz, [i64, i32, i32, i32])
_sig("bgv_sketch_degrees", C.c_int, [P, i64, i32, i32, i32, u64, P, P, P, sz, P])
_sig("bgv_sketch_degrees_noalloc", C.c_int, [P, i64, i32, i32, i32, u64, P, P, P, P])
_sig("bgv_communities_ws_size", sz, [i64, i32])
_sig("bgv_communities", C.c_int, [P, i64, i32, P, i32, u32, u32, i32, P, P, P, sz, P])
_sig("bgv_communities_ex_ws_size", sz, [i64, i32])
_sig("bgv_communities_ex", C.c_int, [P, i64, i32, P, i32, u32, u32, i32, i32, i32, P, P, C.POINTER(u32), P, sz, P])
_sig("bgv_mode_degree_ws_size", sz, [i32])
_sig("bgv_mode_degree", C.c_int, [P, i32, C.POINTER(u32), P, sz, P])
_sig("bgv_modularity_ws_size", sz, [i32])
_sig("bgv_modularity", C.c_int, [P, i64, i32, P, C.POINTER(C.c_double), P, sz, P])
_sig("bgv_supergraph_ws_size", sz, [i64, i32, i32, i32])
_sig("bgv_supergraph", C.c_int, [P, i64, i32, P, P, i32, i32, u64, P, P, P, P, P, P, P, P, P, P, P, P, P, P, sz, P])
_sig("bgv_graph_csr_ws_size", sz, [i64, i32])
_sig("bgv_graph_csr", C.c_int, [P, i64, i32, P, P, P, P, P, P, sz, P])
_sig("bgv_colour_groups_ws_size", sz, [i64])
_sig("bgv_colour_groups", C.c_int, [i64, P, P, i32, P, P, P, sz, P])
_sig("bgv_render_ws_size", sz, [i32, i32])
_sig("bgv_render", C.c_int, [i64, P, P, P, i32, i32, P, P, sz, P])
_sig("bgv_fa2_default_params", None, [C.POINTER(bgv_fa2_params)])
_sig("bgv_fa2_init", C.c_int, [i64, C.POINTER(bgv_fa2_params), P, P, P, P])
_sig("bgv_fa2_ws_size", sz, [i64, i64])
_sig("bgv_fa2_forces", C.c_int, [i64, i64, P, P, P, P, C.POINTER(bgv_fa2_params), P, P, P, P, P, sz, P])
_sig("bgv_fa2_step", C.c_int, [i64, i64, P, P, P, P, C.POINTER(bgv_fa2_params), P, P, P, P, P, sz, P])
_sig("bgv_fa2_run", C.c_int, [i64, i64, P, P, P, P, C.POINTER(bgv_fa2_params), i32, i32, P, P, P, P, P, sz, P])
_sig("bgv_fa2_run_timed", C.c_int, [i64, i64, P, P, P, P, C.POINTER(bgv_fa2_params), i32, P, P, P, P, P, sz, P,
                                    C.POINTER(C.c_float)])
_sig("bgv_launch_count", u64, [])
_sig("bgv_fa2_read_stats", C.c_int, [P, P, C.POINTER(bgv_fa2_stats)])
_sig("bgv_layout_default_params", None, [C.POINTER(bgv_layout_params)])
_sig("bgv_layout_ws_size", sz, [i64, i32, C.POINTER(bgv_layout_params)])
_sig("bgv_layout", C.c_int, [P, i64, i32, C.POINTER(bgv_layout_params), P, P, P, C.POINTER(i64), C.POINTER(i64),
                             P, sz, P])
_sig("bgv_layout_host_ws_size", sz, [i64, i32, C.POINTER(bgv_layout_params)])
_sig("bgv_layout_host", C.c_int, [P, i64, i32, C.POINTER(bgv_layout_params), P, P, P, C.POINTER(i64),
                                  C.POINTER(i64), P, sz, P])
_sig("bgv_layout_batched_ws_size", sz, [i32, P, P, C.POINTER(bgv_layout_params)])
_sig("bgv_layout_batched", C.c_int, [P, i32, P, P, C.POINTER(bgv_layout_params), P, P, P, P, P, P, sz, P])
_sig("bgv_fa2_ws_size_batched", sz, [i32, i64, i64])
_sig("bgv_fa2_init_batched", C.c_int, [i32, P, C.POINTER(bgv_fa2_params), P, P, P, P, sz, P])
_sig("bgv_fa2_forces_batched", C.c_int, [i32, P, i64, P, P, P, P, C.POINTER(bgv_fa2_params), P, P, P, P, P, sz,
                                         P])
_sig("bgv_fa2_run_batched", C.c_int, [i32, P, i64, P, P, P, P, C.POINTER(bgv_fa2_params), i32, i32, P, P, P, P, P,
                                      sz, P])

class bgv_fa2_tune_report(C.Structure):
    _fields_ = [("att_short", i32), ("repulse_threads", i32), ("tail_blocks_per_sm", i32), ("reserved", i32),
                ("ms_att_short", C.c_float * 3), ("ms_repulse_threads", C.c_float * 2),
                ("ms_tail_blocks", C.c_float * 3)]


_sig("bgv_autotune_fa2_ws_size", sz, [i64, i64])
_sig("bgv_autotune_fa2", C.c_int, [i64, i64, P, P, P, P, C.POINTER(bgv_fa2_params), P,
                                   C.POINTER(bgv_fa2_tune_report), P, sz, P])
_sig("bgv_set_fa2_tune", C.c_int, [i32, i32, i32])
_sig("bgv_autotune_sort_ws_size", sz, [i64])
_sig("bgv_autotune_sort", C.c_int, [i64, C.POINTER(bgv_tune_report), P, sz, P])
_sig("bgv_sort_cutoff", i64, [])
_sig("bgv_set_sort_cutoff", i64, [i64])
_sig("bgv_set_sort_method", i32, [i32])
_sig("bgv_sort_hinted_max_keys", i64, [])
_sig("bgv_sort_hinted_ws_size", sz, [i64])
_sig("bgv_sort_hinted", C.c_int, [P, P, i64, P, P, P, sz, P])
_sig("bgv_set_fa2_order", i32, [i32])
_sig("bgv_set_spin_limit", i32, [i32])
_sig("bgv_check_wait_timeout_ws_size", sz, [])
_sig("bgv_check_wait_timeout", C.c_int, [i32, P, sz, P])

#: every symbol this binding resolves from the library
EXPORTS = ["bgv_version", "bgv_strerror", "bgv_ws_init", "bgv_status", "bgv_sketch_degrees_ws_size", "bgv_sketch_degrees", "bgv_sketch_degrees_noalloc",
           "bgv_communities_ws_size", "bgv_communities", "bgv_communities_ex_ws_size", "bgv_communities_ex",
           "bgv_mode_degree_ws_size", "bgv_mode_degree", "bgv_modularity_ws_size", "bgv_modularity",
           "bgv_supergraph_ws_size", "bgv_supergraph",
           "bgv_graph_csr_ws_size", "bgv_graph_csr", "bgv_colour_groups_ws_size", "bgv_colour_groups",
           "bgv_render_ws_size", "bgv_render",
           "bgv_fa2_default_params", "bgv_fa2_init", "bgv_fa2_ws_size", "bgv_fa2_forces", "bgv_fa2_step",
           "bgv_fa2_run", "bgv_fa2_run_timed", "bgv_launch_count", "bgv_fa2_read_stats", "bgv_layout_default_params", "bgv_layout_ws_size", "bgv_layout",
           "bgv_layout_host_ws_size", "bgv_layout_host", "bgv_layout_batched_ws_size", "bgv_layout_batched",
           "bgv_fa2_ws_size_batched", "bgv_fa2_init_batched", "bgv_fa2_forces_batched", "bgv_fa2_run_batched",
           "bgv_autotune_fa2_ws_size", "bgv_autotune_fa2", "bgv_set_fa2_tune",
           "bgv_autotune_sort_ws_size", "bgv_autotune_sort", "bgv_sort_cutoff", "bgv_set_sort_cutoff", "bgv_set_sort_method",
           "bgv_sort_hinted_max_keys", "bgv_sort_hinted_ws_size", "bgv_sort_hinted", "bgv_set_fa2_order",
           "bgv_set_spin_limit", "bgv_check_wait_timeout_ws_size", "bgv_check_wait_timeout"]


class BgvError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {_lib.bgv_strerror(code).decode()} ({code})")
        self.code = code


def _chk(code: int, where: str):
    if code != BGV_OK:
        raise BgvError(code, where)


def _p(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return x.data_ptr()
    return int(x)


def _s(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _nbytes(ws, ws_bytes):
    if ws_bytes is not None:
        return int(ws_bytes)
    return ws.numel() * ws.element_size()


def alloc_ws(nbytes: int, device="cuda") -> torch.Tensor:
    """A caller-owned workspace tensor (uint8, 256-byte aligned) whose
    header has been zeroed with bgv_ws_init."""
    t = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    assert t.data_ptr() % 256 == 0
    bgv_ws_init(t)
    return t


# ----------------------------------------------------------------- C names
def bgv_version() -> int:
    return _lib.bgv_version()


def bgv_strerror(code: int) -> str:
    return _lib.bgv_strerror(code).decode()


def bgv_ws_init(ws, stream=None):
    _chk(_lib.bgv_ws_init(_p(ws), _s(stream)), "bgv_ws_init")


def bgv_status(ws, stream=None, clear: bool = False) -> int:
    out = u32(0)
    _chk(_lib.bgv_status(_p(ws), _s(stream), C.byref(out), 1 if clear else 0), "bgv_status")
    return out.value


def bgv_sketch_degrees_ws_size(m: int, n: int, rows: int, width: int) -> int:
    return _lib.bgv_sketch_degrees_ws_size(m, n, rows, width)


def bgv_sketch_degrees(edges, m, n, rows, width, seed, sketch, deg_est, ws, ws_bytes=None, stream=None):
    _chk(_lib.bgv_sketch_degrees(_p(edges), m, n, rows, width, seed, _p(sketch), _p(deg_est), _p(ws),
                                 _nbytes(ws, ws_bytes), _s(stream)), "bgv_sketch_degrees")


def bgv_sketch_degrees_noalloc(edges, m, n, rows, width, seed, sketch, deg_est, status=None, stream=None):
    """Degree sketch without a workspace, for callers that cannot allocate
    device memory (scratch in a fixed device array, n <= 4,194,304)."""
    _chk(_lib.bgv_sketch_degrees_noalloc(_p(edges), m, n, rows, width, seed, _p(sketch), _p(deg_est), _p(status),
                                         _s(stream)), "bgv_sketch_degrees_noalloc")


def bgv_communities_ws_size(m: int, n: int) -> int:
    return _lib.bgv_communities_ws_size(m, n)


def bgv_communities(edges, m, n, deg_est, passes, threshold, growth, tie_mode, labels, deg_out, ws,
                    ws_bytes=None, stream=None):
    _chk(_lib.bgv_communities(_p(edges), m, n, _p(deg_est), passes, threshold, growth, tie_mode, _p(labels),
                              _p(deg_out), _p(ws), _nbytes(ws, ws_bytes), _s(stream)), "bgv_communities")


def bgv_communities_ex_ws_size(m: int, n: int) -> int:
    return _lib.bgv_communities_ex_ws_size(m, n)


def bgv_communities_ex(edges, m, n, deg_est, passes, threshold, growth, tie_mode, threshold_mode, jumps, labels,
                       deg_out, ws, ws_bytes=None, stream=None) -> int:
    """Returns the first round's threshold."""
    D = u32(0)
    _chk(_lib.bgv_communities_ex(_p(edges), m, n, _p(deg_est), passes, threshold, growth, tie_mode, threshold_mode,
                                 jumps, _p(labels), _p(deg_out), C.byref(D), _p(ws), _nbytes(ws, ws_bytes),
                                 _s(stream)), "bgv_communities_ex")
    return D.value


def bgv_mode_degree_ws_size(n: int) -> int:
    return _lib.bgv_mode_degree_ws_size(n)


def bgv_mode_degree(deg, n, ws, ws_bytes=None, stream=None) -> int:
    out = u32(0)
    _chk(_lib.bgv_mode_degree(_p(deg), n, C.byref(out), _p(ws), _nbytes(ws, ws_bytes), _s(stream)),
         "bgv_mode_degree")
    return out.value


def bgv_modularity_ws_size(n: int) -> int:
    return _lib.bgv_modularity_ws_size(n)


def bgv_modularity(edges, m, n, labels, ws, ws_bytes=None, stream=None) -> float:
    q = C.c_double(0.0)
    _chk(_lib.bgv_modularity(_p(edges), m, n, _p(labels), C.byref(q), _p(ws), _nbytes(ws, ws_bytes), _s(stream)),
         "bgv_modularity")
    return q.value


def bgv_supergraph_ws_size(m: int, n: int, rows: int, width: int) -> int:
    return _lib.bgv_supergraph_ws_size(m, n, rows, width)


def bgv_supergraph(edges, m, n, labels, deg_est, rows, width, seed, node_map, K_dev, ssrc, sdst, sw, Es_dev, mass,
                   csr_off, csr_adj, csr_w, vol, count, comm_label, ws, ws_bytes=None, stream=None):
    _chk(_lib.bgv_supergraph(_p(edges), m, n, _p(labels), _p(deg_est), rows, width, seed, _p(node_map), _p(K_dev),
                             _p(ssrc), _p(sdst), _p(sw), _p(Es_dev), _p(mass), _p(csr_off), _p(csr_adj), _p(csr_w),
                             _p(vol), _p(count), _p(comm_label), _p(ws), _nbytes(ws, ws_bytes), _s(stream)),
         "bgv_supergraph")


def bgv_graph_csr_ws_size(m: int, n: int) -> int:
    return _lib.bgv_graph_csr_ws_size(m, n)


def bgv_graph_csr(edges, m, n, csr_off, csr_adj, csr_w, mass, nnz_dev, ws, ws_bytes=None, stream=None):
    _chk(_lib.bgv_graph_csr(_p(edges), m, n, _p(csr_off), _p(csr_adj), _p(csr_w), _p(mass), _p(nnz_dev), _p(ws),
                            _nbytes(ws, ws_bytes), _s(stream)), "bgv_graph_csr")


def bgv_colour_groups_ws_size(K: int) -> int:
    return _lib.bgv_colour_groups_ws_size(K)


def bgv_colour_groups(K, sizes, group, ws, n=0, node_map=None, node_colour=None, ws_bytes=None, stream=None):
    _chk(_lib.bgv_colour_groups(K, _p(sizes), _p(group), n, _p(node_map), _p(node_colour), _p(ws),
                                _nbytes(ws, ws_bytes), _s(stream)), "bgv_colour_groups")


def bgv_render_ws_size(W: int, H: int) -> int:
    return _lib.bgv_render_ws_size(W, H)


def bgv_render(K, xy, radius, group, W, H, rgba, ws, ws_bytes=None, stream=None):
    _chk(_lib.bgv_render(K, _p(xy), _p(radius), _p(group), W, H, _p(rgba), _p(ws), _nbytes(ws, ws_bytes), _s(stream)),
         "bgv_render")


def bgv_fa2_default_params() -> bgv_fa2_params:
    p = bgv_fa2_params()
    _lib.bgv_fa2_default_params(C.byref(p))
    return p


def bgv_fa2_init(K, params, pos, Fprev, speed, stream=None):
    _chk(_lib.bgv_fa2_init(K, C.byref(params), _p(pos), _p(Fprev), _p(speed), _s(stream)), "bgv_fa2_init")


def bgv_fa2_ws_size(K: int, nnz: int) -> int:
    return _lib.bgv_fa2_ws_size(K, nnz)


def bgv_fa2_forces(K, nnz, csr_off, csr_adj, csr_w, mass, params, pos, Fr, Fa, Fg, ws, ws_bytes=None, stream=None):
    _chk(_lib.bgv_fa2_forces(K, nnz, _p(csr_off), _p(csr_adj), _p(csr_w), _p(mass), C.byref(params), _p(pos), _p(Fr),
                             _p(Fa), _p(Fg), _p(ws), _nbytes(ws, ws_bytes), _s(stream)), "bgv_fa2_forces")


def bgv_fa2_step(K, nnz, csr_off, csr_adj, csr_w, mass, params, pos, F, Fprev, speed, ws, ws_bytes=None, stream=None):
    _chk(_lib.bgv_fa2_step(K, nnz, _p(csr_off), _p(csr_adj), _p(csr_w), _p(mass), C.byref(params), _p(pos), _p(F),
                           _p(Fprev), _p(speed), _p(ws), _nbytes(ws, ws_bytes), _s(stream)), "bgv_fa2_step")


def bgv_fa2_run(K, nnz, csr_off, csr_adj, csr_w, mass, params, iterations, use_graph, pos, F, Fprev, speed, ws,
                ws_bytes=None, stream=None):
    _chk(_lib.bgv_fa2_run(K, nnz, _p(csr_off), _p(csr_adj), _p(csr_w), _p(mass), C.byref(params), iterations,
                          1 if use_graph else 0, _p(pos), _p(F), _p(Fprev), _p(speed), _p(ws),
                          _nbytes(ws, ws_bytes), _s(stream)), "bgv_fa2_run")


BGV_FA2_STAGES = 8
FA2_STAGE_NAMES = ["frame_keys", "sort", "gather", "tree", "preorder", "repulsion", "attraction_wait", "node_speed_update"]


def bgv_fa2_run_timed(K, nnz, csr_off, csr_adj, csr_w, mass, params, iterations, pos, F, Fprev, speed, ws,
                      ws_bytes=None, stream=None):
    """Returns the summed milliseconds per stage (list of BGV_FA2_STAGES)."""
    out = (C.c_float * BGV_FA2_STAGES)()
    _chk(_lib.bgv_fa2_run_timed(K, nnz, _p(csr_off), _p(csr_adj), _p(csr_w), _p(mass), C.byref(params), iterations,
                                _p(pos), _p(F), _p(Fprev), _p(speed), _p(ws), _nbytes(ws, ws_bytes), _s(stream), out),
         "bgv_fa2_run_timed")
    return list(out)


def bgv_launch_count() -> int:
    return int(_lib.bgv_launch_count())


def bgv_fa2_read_stats(ws, stream=None) -> bgv_fa2_stats:
    st = bgv_fa2_stats()
    _chk(_lib.bgv_fa2_read_stats(_p(ws), _s(stream), C.byref(st)), "bgv_fa2_read_stats")
    return st


def bgv_layout_default_params() -> bgv_layout_params:
    p = bgv_layout_params()
    _lib.bgv_layout_default_params(C.byref(p))
    return p


def bgv_layout_ws_size(m: int, n: int, params) -> int:
    return _lib.bgv_layout_ws_size(m, n, C.byref(params))


def bgv_layout(edges, m, n, params, node_map, xy, radius, ws, ws_bytes=None, stream=None):
    """Returns ``(K, Es)``."""
    K, Es = i64(0), i64(0)
    _chk(_lib.bgv_layout(_p(edges), m, n, C.byref(params), _p(node_map), _p(xy), _p(radius), C.byref(K),
                         C.byref(Es), _p(ws), _nbytes(ws, ws_bytes), _s(stream)), "bgv_layout")
    return K.value, Es.value


def bgv_layout_host_ws_size(m: int, n: int, params) -> int:
    return _lib.bgv_layout_host_ws_size(m, n, C.byref(params))


def bgv_layout_host(h_edges, m, n, params, h_node_map, h_xy, h_radius, ws, ws_bytes=None, stream=None):
    """Host buffers (CPU tensors, ideally pinned); returns ``(K, Es)``."""
    K, Es = i64(0), i64(0)
    _chk(_lib.bgv_layout_host(_p(h_edges), m, n, C.byref(params), _p(h_node_map), _p(h_xy), _p(h_radius),
                              C.byref(K), C.byref(Es), _p(ws), _nbytes(ws, ws_bytes), _s(stream)), "bgv_layout_host")
    return K.value, Es.value


def _host(a, dtype):
    """A contiguous host array of ``dtype`` and its address."""
    a = np.ascontiguousarray(np.asarray(a), dtype=dtype)
    return a, a.ctypes.data


def bgv_layout_batched_ws_size(G: int, edge_off, node_off, params) -> int:
    eo, pe = _host(edge_off, np.int64)
    no, pn = _host(node_off, np.int32)
    return _lib.bgv_layout_batched_ws_size(G, pe, pn, C.byref(params))


def bgv_layout_batched(edges, G, edge_off, node_off, params, node_map, xy, radius, ws, ws_bytes=None, stream=None):
    """``edge_off`` [G+1] int64 and ``node_off`` [G+1] int32 on the host;
    returns the host offsets ``(K_off, Es_off)``, each int64 [G+1]."""
    eo, pe = _host(edge_off, np.int64)
    no, pn = _host(node_off, np.int32)
    K_off = np.zeros(G + 1, np.int64)
    Es_off = np.zeros(G + 1, np.int64)
    _chk(_lib.bgv_layout_batched(_p(edges), G, pe, pn, C.byref(params), _p(node_map), _p(xy), _p(radius),
                                 K_off.ctypes.data, Es_off.ctypes.data, _p(ws), _nbytes(ws, ws_bytes), _s(stream)),
         "bgv_layout_batched")
    return K_off, Es_off


def bgv_fa2_ws_size_batched(G: int, K: int, nnz: int) -> int:
    return _lib.bgv_fa2_ws_size_batched(G, K, nnz)


def bgv_fa2_init_batched(G, koff, params, pos, Fprev, speed, ws, ws_bytes=None, stream=None):
    ko, pk = _host(koff, np.int64)
    _chk(_lib.bgv_fa2_init_batched(G, pk, C.byref(params), _p(pos), _p(Fprev), _p(speed), _p(ws),
                                   _nbytes(ws, ws_bytes), _s(stream)), "bgv_fa2_init_batched")


def bgv_fa2_forces_batched(G, koff, nnz, csr_off, csr_adj, csr_w, mass, params, pos, Fr, Fa, Fg, ws, ws_bytes=None,
                           stream=None):
    ko, pk = _host(koff, np.int64)
    _chk(_lib.bgv_fa2_forces_batched(G, pk, nnz, _p(csr_off), _p(csr_adj), _p(csr_w), _p(mass), C.byref(params),
                                     _p(pos), _p(Fr), _p(Fa), _p(Fg), _p(ws), _nbytes(ws, ws_bytes), _s(stream)),
         "bgv_fa2_forces_batched")


def bgv_fa2_run_batched(G, koff, nnz, csr_off, csr_adj, csr_w, mass, params, iterations, use_graph, pos, F, Fprev,
                        speed, ws, ws_bytes=None, stream=None):
    ko, pk = _host(koff, np.int64)
    _chk(_lib.bgv_fa2_run_batched(G, pk, nnz, _p(csr_off), _p(csr_adj), _p(csr_w), _p(mass), C.byref(params),
                                  iterations, use_graph, _p(pos), _p(F), _p(Fprev), _p(speed), _p(ws),
                                  _nbytes(ws, ws_bytes), _s(stream)), "bgv_fa2_run_batched")


def bgv_autotune_sort_ws_size(max_keys: int) -> int:
    return _lib.bgv_autotune_sort_ws_size(max_keys)


def bgv_autotune_sort(max_keys, ws, ws_bytes=None, stream=None) -> bgv_tune_report:
    r = bgv_tune_report()
    _chk(_lib.bgv_autotune_sort(max_keys, C.byref(r), _p(ws), _nbytes(ws, ws_bytes), _s(stream)),
         "bgv_autotune_sort")
    return r


def bgv_sort_cutoff() -> int:
    return _lib.bgv_sort_cutoff()


def bgv_set_sort_cutoff(cutoff: int) -> int:
    """Keys per thread of the radix sort: 8 up to `cutoff` keys, 16 above;
    returns the previous cutoff."""
    return int(_lib.bgv_set_sort_cutoff(cutoff))


def bgv_set_spin_limit(limit: int) -> int:
    """Bound of every look-back wait (polling rounds); returns the previous."""
    return int(_lib.bgv_set_spin_limit(limit))


def bgv_check_wait_timeout_ws_size() -> int:
    return _lib.bgv_check_wait_timeout_ws_size()


def bgv_check_wait_timeout(which, ws, ws_bytes=None, stream=None):
    """Run look-back kernel `which` (0 sort pass, 1 moment pass, 2 CSR pass)
    on an input whose predecessor tile never publishes; its wait must give
    up at the spin limit (BGV_DEV_TIMEOUT in the workspace status word)."""
    _chk(_lib.bgv_check_wait_timeout(which, _p(ws), _nbytes(ws, ws_bytes), _s(stream)), "bgv_check_wait_timeout")


def bgv_autotune_fa2_ws_size(K: int, nnz: int) -> int:
    return _lib.bgv_autotune_fa2_ws_size(K, nnz)


def bgv_autotune_fa2(K, nnz, csr_off, csr_adj, csr_w, mass, params, pos, ws, ws_bytes=None,
                     stream=None) -> bgv_fa2_tune_report:
    """Time FA2 steps on this supergraph for each launch shape and keep the
    fastest (process wide); returns the report."""
    r = bgv_fa2_tune_report()
    _chk(_lib.bgv_autotune_fa2(K, nnz, _p(csr_off), _p(csr_adj), _p(csr_w), _p(mass), C.byref(params), _p(pos),
                               C.byref(r), _p(ws), _nbytes(ws, ws_bytes), _s(stream)), "bgv_autotune_fa2")
    return r


def bgv_set_fa2_tune(att_short: int, repulse_threads: int, tail_blocks_per_sm: int):
    _chk(_lib.bgv_set_fa2_tune(att_short, repulse_threads, tail_blocks_per_sm), "bgv_set_fa2_tune")


def bgv_sort_hinted_max_keys() -> int:
    return int(_lib.bgv_sort_hinted_max_keys())


def bgv_sort_hinted_ws_size(K: int) -> int:
    return _lib.bgv_sort_hinted_ws_size(K)


def bgv_sort_hinted(keys, hint, K, out_keys, out_ids, ws, ws_bytes=None, stream=None):
    _chk(_lib.bgv_sort_hinted(_p(keys), _p(hint), K, _p(out_keys), _p(out_ids), _p(ws), _nbytes(ws, ws_bytes),
                              _s(stream)), "bgv_sort_hinted")


def bgv_set_fa2_order(method: int) -> int:
    """1: ForceAtlas2 runs sort with the previous step's order as the hint
    from their second step on, 0: the full radix sort every step; returns
    the previous value."""
    return int(_lib.bgv_set_fa2_order(method))


def bgv_set_sort_method(method: int) -> int:
    """0: onesweep passes with decoupled look-back, 1: all radix passes in one
    cooperative kernel, 2: cooperative for key counts in the tuned range;
    returns the previous method."""
    return int(_lib.bgv_set_sort_method(method))
