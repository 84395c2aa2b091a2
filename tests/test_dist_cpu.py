"""The multi-process (replicas) path of bench.py on CPU with gloo, world size 2."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": "2", "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local, pg = bench._dist()
    bench._barrier(pg)
    m = bench._max_over_ranks(pg, 1.5 + r)
    with open(os.path.join(out, f"r{r}"), "w") as f:
        f.write(f"{ws} {r} {m}")
    pg.destroy_process_group()


def test_barrier_and_max_over_ranks(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank, args=(_free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    got = sorted(open(tmp_path / f"r{r}").read().split() for r in range(2))
    assert got == [["2", "0", "2.5"], ["2", "1", "2.5"]]


def test_reference_arm_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
