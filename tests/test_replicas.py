"""Replicas on several processes (the path needs no exchange between GPUs):
two ranks under torchrun with a gloo process group on the CPU, through the
bench's own rank helper.  Checks the barrier, the max over ranks, the
whole-job throughput (units of all ranks / the slowest rank's time) and that
only rank 0 runs the reference arm."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_aggregate_throughput_counts_every_rank_at_the_slowest_time():
    import bench
    assert bench.aggregate_throughput(1000.0, 1, 10.0) == pytest.approx(1e5)
    assert bench.aggregate_throughput(1000.0, 4, 20.0) == pytest.approx(2e5)


def test_two_gloo_ranks_share_barrier_and_max(tmp_path):
    pytest.importorskip("torch.distributed")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.join(ROOT, "tests", "replica_worker.py"),
           str(tmp_path)]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads((tmp_path / f"rank{k}.json").read_text()) for k in range(2)]
    assert sorted(x["rank"] for x in lines) == [0, 1]
    for x in lines:
        assert x["world"] == 2 and x["local"] == x["rank"]
        assert x["ms_max"] == 20.0
        assert x["value"] == pytest.approx(1000.0 * 2 / 0.020)
    assert [x["reference_skipped"] for x in sorted(lines, key=lambda x: x["rank"])] == [None, True]

