"""The C-ABI library builds, loads and exports every entry point declared in
include/bgv.h; host-side validation and workspace queries work without a GPU
(no compute call is made here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bgv.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2108_00529_gb300 import build
    path = build.build()
    return C.CDLL(str(path))


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(bgv_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_pipeline_calls():
    names = declared_functions()
    for required in ("bgv_sketch_degrees", "bgv_communities", "bgv_supergraph", "bgv_fa2_step", "bgv_layout"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_2108_00529_gb300 import bgv
    assert sorted(bgv.EXPORTS) == declared_functions()


def test_struct_layouts(lib):
    from paper_2108_00529_gb300 import bgv
    assert C.sizeof(bgv.bgv_fa2_params) == 48
    assert C.sizeof(bgv.bgv_layout_params) == 96
    assert C.sizeof(bgv.bgv_fa2_stats) == 56
    assert C.sizeof(bgv.bgv_fa2_tune_report) == 48
    assert C.sizeof(bgv.bgv_tune_report) == 176
    p = bgv.bgv_layout_default_params()
    assert (p.rows, p.width, p.passes, p.growth, p.iterations) == (4, 4096, 3, 2, 200)
    assert (p.threshold_mode, p.jumps, p.use_graph) == (0, 0, 1)
    assert abs(p.fa2.theta - 1.2) < 1e-6 and p.fa2.max_depth == 24 and p.fa2.leaf_cap == 1


def test_workspace_queries_are_monotone(lib):
    from paper_2108_00529_gb300 import bgv
    a = bgv.bgv_sketch_degrees_ws_size(1000, 100, 4, 64)
    b = bgv.bgv_sketch_degrees_ws_size(1000, 100000, 4, 64)
    assert 256 <= a < b and a % 256 == 0
    assert bgv.bgv_supergraph_ws_size(10, 10, 4, 16) < bgv.bgv_supergraph_ws_size(10**6, 10, 4, 16)
    assert bgv.bgv_fa2_ws_size(10, 0) < bgv.bgv_fa2_ws_size(10**5, 0)
    p = bgv.bgv_layout_default_params()
    assert bgv.bgv_layout_ws_size(100, 50, p) < bgv.bgv_layout_host_ws_size(100, 50, p)


def test_host_validation_rejects_bad_arguments(lib):
    # Rejected on the host before any CUDA call: no GPU needed.
    from paper_2108_00529_gb300 import bgv
    L = bgv._lib
    fake_ws = C.c_void_p(256 * 1024)  # never dereferenced: validation fails first
    assert L.bgv_sketch_degrees(None, 0, 0, 4, 16, 1, None, None, fake_ws, 1 << 20, None) == bgv.BGV_EINVAL
    assert L.bgv_sketch_degrees(C.c_void_p(16), 1, 10, 0, 16, 1, C.c_void_p(16), C.c_void_p(16), fake_ws, 1 << 20,
                                None) == bgv.BGV_EINVAL
    assert L.bgv_sketch_degrees(C.c_void_p(8), 1, 10, 4, 16, 1, C.c_void_p(16), C.c_void_p(16), fake_ws, 1 << 20,
                                None) == bgv.BGV_EINVAL  # edges not 16-byte aligned
    assert L.bgv_sketch_degrees(C.c_void_p(16), 1, 10, 4, 16, 1, C.c_void_p(16), C.c_void_p(16), fake_ws, 64,
                                None) == bgv.BGV_ENOSPC
    assert L.bgv_communities(C.c_void_p(16), 1, 10, C.c_void_p(16), 1, 5, 2, 2, C.c_void_p(16), None, fake_ws,
                             1 << 20, None) == bgv.BGV_EINVAL  # tie_mode 2
    assert L.bgv_communities_ex(C.c_void_p(16), 1, 10, C.c_void_p(16), 1, 0, 2, 0, 2, 0, C.c_void_p(16), None, None,
                                fake_ws, 1 << 20, None) == bgv.BGV_EINVAL  # threshold_mode 2
    assert L.bgv_communities_ex(C.c_void_p(16), 1, 10, C.c_void_p(16), 1, 0, 2, 0, 0, 65, C.c_void_p(16), None, None,
                                fake_ws, 1 << 20, None) == bgv.BGV_EINVAL  # jumps above 64
    p = bgv.bgv_fa2_default_params()
    p.max_depth = 25
    assert L.bgv_fa2_step(10, 20, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), C.byref(p),
                          C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), fake_ws, 1 << 30,
                          None) == bgv.BGV_EINVAL
    assert bgv.bgv_strerror(bgv.BGV_ENOSPC) == "workspace too small"


def test_batched_host_validation(lib):
    # Offsets are checked on the host before any CUDA call.
    import numpy as np
    from paper_2108_00529_gb300 import bgv
    L = bgv._lib
    p = bgv.bgv_layout_default_params()
    eo = np.array([0, 10, 25], np.int64)
    no = np.array([0, 5, 9], np.int32)
    assert bgv.bgv_layout_batched_ws_size(2, eo, no, p) > bgv.bgv_layout_ws_size(25, 9, p)
    for bad_e, bad_n in [([1, 10, 25], [0, 5, 9]),      # offsets must start at 0
                         ([0, 10, 25], [0, 5, 5]),      # empty graph
                         ([0, 30, 25], [0, 5, 9])]:     # edge offsets decrease
        assert bgv.bgv_layout_batched_ws_size(2, bad_e, bad_n, p) == 0
        e, pe = bgv._host(bad_e, np.int64)
        n, pn = bgv._host(bad_n, np.int32)
        K = np.zeros(3, np.int64)
        assert L.bgv_layout_batched(C.c_void_p(16), 2, pe, pn, C.byref(p), C.c_void_p(16), C.c_void_p(16), None,
                                    K.ctypes.data, K.ctypes.data, C.c_void_p(256), 1 << 30, None) == bgv.BGV_EINVAL
    fp = bgv.bgv_fa2_default_params()
    ko, pk = bgv._host([0, 3, 3, 7], np.int64)  # graph 1 has no bodies
    assert L.bgv_fa2_run_batched(3, pk, 0, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), C.c_void_p(16),
                                 C.byref(fp), 1, 0, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), C.c_void_p(16),
                                 C.c_void_p(256), 1 << 30, None) == bgv.BGV_EINVAL
    # more graphs need more workspace (frames, speeds, per-body graph ids)
    assert bgv.bgv_fa2_ws_size_batched(1, 1000, 10) <= bgv.bgv_fa2_ws_size_batched(100, 1000, 10)


def test_hinted_sort_queries_and_host_validation(lib):
    # Workspace queries, the order setting and every refusal happen on the
    # host, before any CUDA call.
    from paper_2108_00529_gb300 import bgv
    L = bgv._lib
    kmax = bgv.bgv_sort_hinted_max_keys()
    assert kmax == 4096 * 1024
    a, b = bgv.bgv_sort_hinted_ws_size(0), bgv.bgv_sort_hinted_ws_size(kmax)
    assert 256 <= a < b and b % 256 == 0
    assert bgv.bgv_sort_hinted_ws_size(kmax + 1) == 0 and bgv.bgv_sort_hinted_ws_size(-1) == 0
    K = 1000
    n = bgv.bgv_sort_hinted_ws_size(K)
    ws = C.c_void_p(1 << 20)  # never dereferenced: validation fails first
    keys, hint, ok, oi = (C.c_void_p(v) for v in (1 << 24, 1 << 25, 1 << 26, 1 << 27))
    assert L.bgv_sort_hinted(keys, hint, 0, ok, oi, ws, n, None) == bgv.BGV_OK  # nothing to sort
    assert L.bgv_sort_hinted(keys, hint, K, ok, oi, C.c_void_p((1 << 20) + 8), n, None) == bgv.BGV_EINVAL
    assert L.bgv_sort_hinted(keys, hint, kmax + 1, ok, oi, ws, 1 << 40, None) == bgv.BGV_EINVAL
    assert L.bgv_sort_hinted(keys, hint, K, ok, oi, ws, n - 256, None) == bgv.BGV_ENOSPC
    assert L.bgv_sort_hinted(keys, None, K, ok, oi, ws, n, None) == bgv.BGV_EINVAL
    assert L.bgv_sort_hinted(C.c_void_p((1 << 24) + 4), hint, K, ok, oi, ws, n, None) == bgv.BGV_EINVAL
    assert L.bgv_sort_hinted(keys, hint, K, C.c_void_p((1 << 24) + 8), oi, ws, n, None) == bgv.BGV_EINVAL  # overlap
    prev = bgv.bgv_set_fa2_order(0)
    assert prev in (0, 1)
    assert bgv.bgv_set_fa2_order(2) == -1
    assert bgv.bgv_set_fa2_order(prev) == 0
