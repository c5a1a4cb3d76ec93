"""Host logic of bench.py's N > 1 path (replicas, one per rank): the job's
rate takes the slowest rank's time, over a world-size-2 gloo group on CPU."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank = dist.get_rank()
t, v = bench.job_rate(100.0 * (rank + 1), 10, dist.get_world_size(), device="cpu")
print(json.dumps({"rank": rank, "t": t, "v": v}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(250.0, 5, 1) == (250.0, 20.0)


def test_job_rate_takes_the_slowest_of_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=120)
            assert p.returncode == 0, err
            outs.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    # both ranks see the slower rank's 200 ms: 2 ranks x 10 steps / 0.2 s
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["t"] == 200.0
        assert o["v"] == 100.0
