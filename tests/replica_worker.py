"""One rank of the replica check in tests/test_replicas.py, launched by
torchrun on the CPU: the bench's rank helper over a gloo process group.
Each rank writes one JSON file, rank<r>.json, into the folder given as the
first argument."""
import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def main():
    d = bench.Dist()
    try:
        d.barrier()
        ms = 10.0 * (d.rank + 1)                 # rank r's step time
        ms_max = d.max(ms)                       # the slowest rank's
        value = bench.aggregate_throughput(1000.0, d.world, ms_max)
        # the reference arm runs on rank 0 only; the others return at once
        skipped = None
        if d.rank != 0:
            skipped = bench.reference_arm(argparse.Namespace(workload="rmat20", steps=1, warmup=0), d) is None
        d.barrier()
        with open(os.path.join(sys.argv[1], f"rank{d.rank}.json"), "w") as f:
            json.dump({"rank": d.rank, "world": d.world, "local": d.local, "ms_max": ms_max, "value": value,
                       "reference_skipped": skipped}, f)
    finally:
        d.close()


if __name__ == "__main__":
    main()
