"""bench.py on the GPU: one short run of the default workload prints one JSON line with
every key the benchmark contract names, and the numbers are consistent with each other."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("workload", ["c3", "c2", "c1"])
def test_bench_line_has_the_contract_keys(workload):
    d = _run("--workload", workload, "--steps", "2", "--warmup", "3", "--e2e-steps", "1",
             "--no-cpu-baseline")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3 and d["value"] > 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["config"]["workload"].startswith(workload)
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] in ("hbm", "alu") and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert r["int_ceiling_gene_updates_per_s"] > 0 and r["frac_hbm_4B_formula"] > 0
    slower = max(r["t_hbm_us"], r["t_int_us"])
    assert (r["bound"] == "hbm") == (r["t_hbm_us"] == slower)
    if workload != "c1":                          # one launch per generation: per-phase times
        ph = r["phases"]
        assert len(ph["per_25"]) >= 1 and ph["sum_of_launches_us"] > 0
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert e["value"] <= d["value"] * 1.05        # host copies inside the timed region
    assert d["gpu_launches"] >= 2 * 3
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]


def test_generation_times_and_integer_ceiling():
    """The per-generation event times cover every generation of the last run, and the
    integer ceiling's two kernels give positive rates, Philox alone being the faster."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30862_gb300 import qieo as Q
    from paper_2609_30862_gb300 import workload as W
    Q.load()
    with Q.Instance(W.knapsack(3000, 2), 200, seed=2, flags=Q.QIEO_FLAG_TIME_GENERATIONS) as I:
        I.run(12)
        ms = I.generation_times(100)
        assert len(ms) == 12 and (ms > 0).all()
        I.run(5)
        assert len(I.generation_times(3)) == 3
    with Q.Instance(W.knapsack(30, 2), 20) as plain:
        with pytest.raises(Q.QieoError):
            plain.generation_times(4)
    c = Q.qieo_measure_integer_ceiling(2)
    assert c.drawn_genes_per_s > 0 and c.philox_genes_per_s > c.drawn_genes_per_s
    assert c.genes_per_launch > 0 and c.grid_ctas > 0 and c.reps == 2
