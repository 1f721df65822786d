"""The benchmark's multi-rank path on CPU ranks (gloo, world size 2): every rank
advances its own replica, the slowest rank's time sets the whole-job number,
and under torchrun only rank 0 runs and prints the reference arm."""
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


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    env = bench.dist_env()
    ms = 10.0 * (rank + 1)  # rank 1 is the slower one
    ms_max = bench.max_over_ranks(ms, ws, device="cpu")
    value = bench.replicas_value(1000, 4, ws, ms_max)
    dist.barrier()
    dist.destroy_process_group()
    with open(out % rank, "w") as f:
        json.dump({"env": env, "ms_max": ms_max, "value": value}, f)


def test_max_over_ranks_and_replica_throughput_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "rank%d.json")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn")
    for rank in range(2):
        r = json.load(open(out % rank))
        assert r["env"] == [2, rank, rank]
        assert r["ms_max"] == 20.0
        # 2 ranks x 1000 units x 4 steps over the slowest rank's 20 ms
        assert r["value"] == pytest.approx(2 * 1000 * 4 / 0.020)


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % port, os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--workload", "sod512", "--steps", "2",
           "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
