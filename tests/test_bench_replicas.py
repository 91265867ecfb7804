"""bench.py's multi-GPU harness on CPU: world size 2 over gloo, launched the way the multi-GPU bench
is (torchrun, one process per rank, rendezvous on 127.0.0.1).  The path does not shard (each rank
runs an independent replica), so the harness is the barrier and the max over ranks around the
timed region, and the reference arm's rank-0-only output.

* allmax returns the largest value on every rank, and barrier returns on both;
* the reference arm under torchrun: rank 0 alone prints one JSON line (impl "reference", n_gpus 2,
  the oracle as its cpu_baseline), rank 1 exits 0 without work.
"""
import json
import os
import re
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, tmo=300):
    env = dict(os.environ, BM_BENCH_GLOO="1", MASTER_ADDR="127.0.0.1", OMP_NUM_THREADS="2",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=tmo)


def test_allmax_and_barrier_over_gloo(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(
        "import os, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import bench\n"
        "ws, rank, local = bench.dist_init()\n"
        "bench.barrier(ws)\n"
        "v = bench.allmax(ws, 1.5 + rank)\n"
        "bench.barrier(ws)\n"
        "print(f'RANK {rank} WS {ws} MAX {v}', flush=True)\n"
        "import torch.distributed as dist\n"
        "dist.destroy_process_group()\n")
    r = _torchrun([str(script)], tmo=120)
    assert r.returncode == 0, r.stderr[-2000:]
    # the two ranks share one stdout, so their lines may interleave
    found = sorted(re.findall(r"RANK (\d) WS (\d) MAX ([0-9.]+)", r.stdout))
    assert found == [("0", "2", "2.5"), ("1", "2", "2.5")]


def test_reference_arm_prints_once_on_rank_zero():
    r = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--quick", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    rows = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(rows) == 1
    d = rows[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    assert d["value"] > 0 and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
