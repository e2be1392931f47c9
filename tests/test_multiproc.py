"""The multi-rank logic of bench.py on the CPU: two gloo ranks (world size 2).

Each rank runs its own independent filter (replicas, no collective on the data path);
the job's time is the maximum over the ranks and rank 0 alone prints. Checked here:
max_over_ranks returns the largest rank value on every rank, barrier returns on both,
dist_env reads the launcher's variables, and the reference arm makes ranks other than
0 exit at once without output.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys, io, contextlib
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
ws, rank, local = bench.dist_env()
assert ws == 2 and rank == int(os.environ["RANK"]) and local == rank
m = bench.max_over_ranks(float(10 + 5 * rank), ws)
bench.barrier(ws)
out = io.StringIO()
with contextlib.redirect_stdout(out):
    class A: steps = 1; warmup = 3; gpus = 2
    rc = bench.run_reference(A) if rank == 1 else 0
print(f"rank {rank} max {m} ref_rc {rc} ref_out {len(out.getvalue())}")
dist.destroy_process_group()
'''


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e[-2000:]
        outs.append(o.strip())
    assert "rank 0 max 15.0 ref_rc 0 ref_out 0" in outs[0], outs
    assert "rank 1 max 15.0 ref_rc 0 ref_out 0" in outs[1], outs
