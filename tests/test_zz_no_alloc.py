"""GPU test of bgv_sketch_degrees_noalloc, the degree sketch for callers that
cannot allocate device memory.

Code that runs while a stream is being captured, or a plugin inside an
application that owns all device memory, cannot call cudaMalloc and so cannot
hand the library a workspace.  For them the library keeps the sketch's
per-node counters in a fixed device array of its own.  This test calls that
entry point through the C ABI on two graphs in a row (the second call reuses
the array the first left behind) and checks both results, bit for bit, against
the workspace entry point bgv_sketch_degrees and against the CPU oracle.  It
also checks that, without a status pointer, a bad edge comes back as an error
code, and that the next call starts clean.  The file is named so pytest
collects it last.
"""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import gpu_pipeline as G  # noqa: E402

B = G.B


def _noalloc(e, n, rows, width, seed):
    E, m = G.edges_dev(e)
    S = G.empty(rows * width, np.uint32)
    d = G.empty(n, np.uint32)
    status = G.empty(1, np.uint32)
    B.bgv_sketch_degrees_noalloc(E, m, n, rows, width, seed, S, d, status)
    torch.cuda.synchronize()
    return G.host(S, np.uint32).reshape(rows, width), G.host(d, np.uint32, n), int(G.host(status, np.uint32)[0])


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    n1, e1, _ = graphgen.load("sbm16")
    e2 = graphgen.random_graph(5000, 20001, seed=21, self_loops=3)
    calls = [(e1, n1, 4, 4096, 1), (e2, 5000, 3, 1000, 7)]
    for e, n, rows, width, seed in calls:
        S, d, st = _noalloc(e, n, rows, width, seed)
        S0, d0, st0 = G.sketch(e, n, rows, width, seed)
        assert st == 0 and st0 == 0
        assert np.array_equal(S, S0)
        assert np.array_equal(d, d0)
        So, do = oracle.sketch_degrees(e, n, rows, width, seed)
        assert np.array_equal(S, So) and np.array_equal(d, do)


def test_noalloc_without_status_pointer_reports_bad_edges():
    # An endpoint outside [0, n) is caught by the kernel's bounds check and
    # reported through the entry point's own status word: the call returns
    # BGV_EDEVICE.  The word is cleared by the next call, which succeeds.
    n = 100
    bad = np.array([[0, 1], [2, 3], [5, n + 7], [4, 6]], np.int32)
    E, m = G.edges_dev(bad)
    S, d = G.empty(4 * 64, np.uint32), G.empty(n, np.uint32)
    with pytest.raises(B.BgvError) as ex:
        B.bgv_sketch_degrees_noalloc(E, m, n, 4, 64, 1, S, d)
    assert ex.value.code == B.BGV_EDEVICE
    good = graphgen.random_graph(n, 300, seed=5)
    E, m = G.edges_dev(good)
    B.bgv_sketch_degrees_noalloc(E, m, n, 4, 64, 1, S, d)
    So, do = oracle.sketch_degrees(good, n, 4, 64, 1)
    assert np.array_equal(G.host(S, np.uint32).reshape(4, 64), So)
    assert np.array_equal(G.host(d, np.uint32, n), do)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    e = np.array([[0, 1]], np.int32)
    E, m = G.edges_dev(e)
    S = G.empty(16, np.uint32)
    d = G.empty(8, np.uint32)
    with pytest.raises(B.BgvError) as ex:
        B.bgv_sketch_degrees_noalloc(E, m, (1 << 22) + 1, 1, 16, 1, S, d)
    assert ex.value.code == B.BGV_ELIMIT
