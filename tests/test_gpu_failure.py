"""Failure detection and resume on the GPU, without a fault.

Bounded waits: every decoupled look-back wait in the library gives up after a
set number of polling rounds and reports BGV_DEV_TIMEOUT instead of hanging.
Each look-back kernel (a radix-sort pass, the ForceAtlas2 moment pass, the
CSR pass of the supergraph) is run on an input whose predecessor tile never
publishes, with a small bound: the call must come back, the status word must
hold the timeout bit, and the GPU must still work afterwards.

Resume: the ForceAtlas2 state (positions, previous forces, speed) is the whole
state of a layout, so 10 steps, a copy of that state to the host, a fresh
workspace and 15 more steps equal 25 straight steps bit for bit."""
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


@pytest.mark.parametrize("which", [0, 1, 2])
def test_wait_that_cannot_end_reports_timeout(which):
    ws = B.alloc_ws(B.bgv_check_wait_timeout_ws_size())
    prev = B.bgv_set_spin_limit(64)
    try:
        B.bgv_check_wait_timeout(which, ws)
    finally:
        assert B.bgv_set_spin_limit(prev) == 64
    assert B.bgv_status(ws) & B.BGV_DEV_TIMEOUT
    # the context is still usable: a sketch right after is exact
    e = graphgen.random_graph(500, 2000, seed=which)
    S, d, st = G.sketch(e, 500, 4, 128, 3)
    S0, d0 = oracle.sketch_degrees(e, 500, 4, 128, 3)
    assert st == 0 and np.array_equal(S, S0) and np.array_equal(d, d0)


def test_spin_limit_setter_rejects_negative_bounds():
    prev = B.bgv_set_spin_limit(1000)
    assert B.bgv_set_spin_limit(-5) == -1
    assert B.bgv_set_spin_limit(prev) == 1000


def test_normal_waits_end_well_inside_a_small_bound():
    # A whole supergraph and FA2 step with the bound at 1024 rounds: the
    # waits of a normal run end long before it, so nothing times out.
    n, e, _ = graphgen.load("sbm16")
    _, dh = oracle.sketch_degrees(e, n, 4, 4096, 1)
    lab, _ = oracle.communities(e, n, dh, 3, 64, 2, 0)
    prev = B.bgv_set_spin_limit(1 << 10)
    try:
        sg = G.supergraph(e, n, lab, dh, 4, 4096, 1)
        r = G.fa2_forces(oracle.fa2_init(sg["K"], 1), sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"],
                         FA2Params())
    finally:
        B.bgv_set_spin_limit(prev)
    assert sg["status"] == 0 and r["status"] == 0
    sg0 = oracle.supergraph(e, n, lab, dh, 4, 4096, 1)
    assert np.array_equal(sg["csr_adj"], sg0["csr_adj"])


def test_resume_from_host_state_equals_straight_run():
    n, e, _ = graphgen.load("sbm16")
    _, dh = oracle.sketch_degrees(e, n, 4, 4096, 1)
    lab, _ = oracle.communities(e, n, dh, 3, 64, 2, 0)
    sg = oracle.supergraph(e, n, lab, dh, 4, 4096, 1)
    pos0 = oracle.fa2_init(sg["K"], 3)
    p = FA2Params()
    args = (sg["mass"], sg["csr_off"], sg["csr_adj"], sg["csr_w"], p)
    straight = G.Fa2Device(pos0, *args)
    straight.run(25, False)
    first = G.Fa2Device(pos0, *args)
    first.run(10, False)
    pos, Fprev, speed = G.host(first.pos).copy(), G.host(first.Fprev).copy(), float(first.speed.item())
    del first
    resumed = G.Fa2Device(pos, *args, Fprev=Fprev, speed=speed)
    resumed.run(15, True)  # the rest replayed as a captured step
    a, b = straight.state(), resumed.state()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2]) and a[3] == b[3]
