"""bench.py's host logic without a GPU: the max-over-ranks reduction under world size 2
(gloo), and the reference arm under torchrun with two ranks (rank 0 prints one JSON line,
rank 1 exits 0 without output), and the oracle thread scan."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(1.5 + rank, dist, device="cpu")
        if rank == 0:
            with open(out_path, "w") as fh:
                fh.write(repr(got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_world_2(tmp_path):
    import torch.multiprocessing as mp
    import bench
    assert bench.max_over_ranks(3.25) == 3.25          # one rank: no collective
    out = str(tmp_path / "max.txt")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    assert float(open(out).read()) == 2.5


@pytest.mark.parametrize("workload,unit", [("c1", "gene-updates/s"), ("c4", "solves/s")])
def test_reference_arm_under_torchrun_two_ranks(workload, unit):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--workload", workload, "--steps", "2", "--warmup", "1", "--ref-budget-s", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == unit and d["value"] > 0
    assert d["n_gpus"] == 2 and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_oracle_scan_on_host_cores():
    """--oracle-scan: the oracle's serial build and its OpenMP build at 1, 8, 16 and all
    threads (those the host has), one JSON line with a positive rate per run."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-scan", "--workload", "c1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    cores = os.cpu_count() or 1
    assert d["oracle_scan"] == "c1" and d["host_cores"] == cores
    got = [(x["build"], x["threads"]) for x in d["runs"]]
    assert got[0] == ("serial", 1)
    assert got[1:] == [("omp", n) for n in sorted({1, 8, 16, cores}) if n <= cores]
    assert all(x["gene_updates_per_s"] > 0 and x["generations"] >= 1 for x in d["runs"])
