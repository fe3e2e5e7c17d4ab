"""The multi-rank path of bench.py on CPU (gloo, world size 2): each rank
advances its own replica, the job's throughput is the units of all ranks over
the slowest rank's time, and only rank 0 prints."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      LBM_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench

    d = bench.Dist(world)
    # rank r processed (r + 1) M lattice updates in 10 (r + 1) ms
    value, ms = bench.aggregate((rank + 1) * 1e6, 10.0 * (rank + 1), d)
    d.barrier()
    d.close()
    with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
        json.dump({"value": value, "ms": ms}, f)


def _free_port():
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_aggregate_is_all_units_over_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        got = json.load(open(tmp_path / f"rank{r}.json"))
        assert got["ms"] == pytest.approx(20.0)
        assert got["value"] == pytest.approx(3e6 / 20e-3 / 1e6)  # 150 MLUPS


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched as two ranks: rank 0 times the
    oracle and prints one JSON line; rank 1 exits 0 without work."""
    env = dict(os.environ, LBM_BENCH_BACKEND="gloo")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1", "--size", "64"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
