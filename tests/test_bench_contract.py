"""The benchmark's reference arm (the CPU oracle timed on a bounded sample of
the 640x480 batch) prints one JSON line with the keys the benchmark contract
asks for. Runs on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "3", "--ref-sample", "24"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert "24-hypothesis sample" in d["config"]["workload"]


def test_cpu_baseline_leg_on_the_small_workload():
    """The bench's cpu_baseline leg: the oracle timed on a bounded sample on
    all host threads and on one, with the fields the JSON line carries; the
    C1 time-to-optimum leg reports an error entry, never an exception, where
    no GPU is present."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1510_05613_gb300 import synth
    wl = synth.workload_c1()
    hyps = synth.all_hypotheses(wl.grid, [0, 1])[::50]
    parents = [wl.gt[:0]]
    hp = __import__("numpy").zeros(len(hyps), "int32")
    for threads in (0, 1):
        b = bench.cpu_baseline(wl, parents, hp, hyps, target_s=0.2, threads=threads)
        assert b["kind"] == "oracle" and b["value"] > 0 and b["unit"] == bench.UNIT
        assert b["cores"] >= 1 and (threads == 0 or b["cores"] == 1)
        assert f"{len(hyps)} hypotheses of the batch" in b["sample"]
    import torch
    if not torch.cuda.is_available():
        r = bench.c1_time_to_optimum(1)
        assert set(r) == {"error"}
