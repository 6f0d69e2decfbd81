"""bench.py's JSON line: the keys and units the measurement contract fixes.
The reference arm (the oracle on the host cores) runs on CPU; our arm needs a
GPU and runs on a small R-MAT workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                       timeout=timeout, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--workload", "rmat_s14_ef8", "--steps", "2", "--warmup", "1"], 600)
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "updates/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["config"]["workload"] == "rmat_s14_ef8" and d["config"]["r_cliques"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.gpu
def test_our_arm_line():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = _run(["--workload", "rmat_s14_ef8", "--steps", "2", "--warmup", "3", "--no-cpu-baseline", "--no-extras"],
             900)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "roofline", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["gpu_launches"] > 0
    assert d["config"]["workload"] == "rmat_s14_ef8"
    e = d["e2e"]
    assert e["unit"] == d["unit"] and e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert d["parity_vs_oracle_digest"] in (True, None) and d["snd_equals_and"] is True
    if r["kernel"] in ("snd_pass", "and_pass"):
        assert r["frac_survey"] > r["frac"] > 0   # the survey model also counts the gathered tau
    assert r["frac_dram"] is None or r["frac_dram"] > 0
    assert 0 < d["value_launched"] <= d["value"]
    ref = _run(["--impl", "reference", "--workload", "rmat_s14_ef8", "--steps", "1", "--warmup", "0"], 600)
    assert ref["config"] == d["config"]   # both arms decompose the same graph


@pytest.mark.gpu
def test_sweeps_line():
    """--mode sweeps: SND, AND and AND-nn reach the same kappa (the bench
    flags any mismatch), and notification only ever saves evaluations."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = _run(["--mode", "sweeps", "--workload", "rmat_s14_ef8"], 900)
    rec = d["workloads"]["rmat_s14_ef8"]
    assert "error" not in rec, rec.get("error")
    for mode in ("snd", "and", "and_nn"):
        assert rec[mode]["passes"] >= 1 and rec[mode]["ms"] > 0 and rec[mode]["evaluations"] > 0
    assert rec["and"]["evaluations"] <= rec["and_nn"]["evaluations"]
    assert rec["and_nn_over_and_time"] > 0
