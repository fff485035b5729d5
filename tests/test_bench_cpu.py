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


def test_work_adjusted_roofline_arithmetic():
    """The work-adjusted bound of a generation is the slower of its draws at the integer
    ceiling and its bytes at HBM: 32 B for each vector that drew, 2.125 B (a fixed-vector
    bit and the previous alleles read, the alleles written) for each that did not."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.STABLE_BYTES == 2.125
    nvec, hbm, intc = 1000, 1.0, 8.0e6             # GB/s (1e9 B/s) and gene-updates/s
    # all drew: draws 8000 / 8e6 = 1 ms; bytes 32e3 / 1e9 = 32 us -> 1 ms (integer-bound)
    # none drew: bytes 2.125e3 / 1e9 = 2.125 us (HBM-bound)
    w = bench.work_adjusted([2.0, 0.006], [1000, 0], nvec, hbm, intc)
    assert abs(w["bound_us"] - (1000.0 + 2.125)) < 1e-6
    assert abs(w["measured_us"] - 2006.0) < 1e-6
    assert abs(w["frac"] - 1002.125 / 2006.0) < 1e-12
    assert abs(w["drawn_fraction"] - 0.5) < 1e-12


def test_profile_traffic_needs_the_current_kernel_source(tmp_path, monkeypatch):
    """A committed ncu summary's traffic is used only when its source hash matches."""
    sys.path.insert(0, ROOT)
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_c9.md").write_text("kernel_source_sha256: %s\ntraffic_bytes_per_generation: 123\n"
                                  % bench.kernel_source_hash())
    (prof / "old_c9.md").write_text("kernel_source_sha256: 0000000000000000\ntraffic_bytes_per_generation: 5\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: (prof / "k_c9.md").read_text().split()[1])
    assert bench.profile_traffic("k", "c9") == 123.0
    assert bench.profile_traffic("old", "c9") is None
    assert bench.profile_traffic("missing", "c9") is None
