"""The multi-process paths of bench.py on the CPU (gloo, world size 2).

The single-grid step does not shard: with N ranks every rank runs an
independent replica and the benchmark reports all ranks' point-steps over the
slowest rank's time. These tests run that aggregation over a real two-rank gloo
process group, and the reference arm under torchrun (rank 0 measures and
prints, the other ranks exit without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + rank, "cpu")  # rank 1 is the slower replica
    v = bench.replica_value(1000, world, t)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
        json.dump({"t": t, "v": v}, f)


def test_replica_time_is_max_over_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / ("r%d.json" % r))) for r in range(2)]
    for r in res:
        assert r["t"] == 11.0
        assert r["v"] == pytest.approx(2 * 1000 / 11e-3)


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_value(500, 1, 2.0) == pytest.approx(250000.0)


def test_reference_arm_under_torchrun():
    """bench.py --impl reference with two ranks: exactly one JSON line (rank 0),
    both ranks exit 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
