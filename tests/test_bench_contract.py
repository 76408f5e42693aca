"""bench.py's reference arm on the CPU: one JSON line with the keys the measurement contract
names (the GPU arm's line is checked by running it on a GB300)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in j, key
    assert j["impl"] == "reference" and j["value"] > 0 and j["unit"] == "layers/s" and j["higher_is_better"]
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in j["config"]


def test_fill_packing_rule_and_workload_names():
    """fill_packing unpacks exactly the layers whose unpacked layout needs no more input and output
    ciphertexts; the reference arm's config names the same per-layer packing as the GPU arm; every
    profiled-traffic entry is keyed by a workload description the bench can produce."""
    sys.path.insert(0, ROOT)
    import bench

    layers = [dict(name=n, c_n=2) for n in ("full", "half", "equal_in_more_out")] + [dict(name="dw4", c_n=4)]
    counts = {("full", 1): (10, 10), ("full", 2): (10, 10), ("half", 1): (20, 20), ("half", 2): (10, 10),
              ("equal_in_more_out", 1): (10, 12), ("equal_in_more_out", 2): (10, 10)}
    out = bench.fill_packing(layers, lambda s: counts[(s["name"], s["c_n"])])
    assert [s["c_n"] for s in out] == [1, 2, 2, 4]
    for wl in bench.WORKLOADS:
        assert bench.workload_name(wl, "2") == bench.WORKLOADS[wl][1]
        assert "c_n per layer" in bench.workload_name(wl, "fill")
    names = {bench.workload_name(wl, pk) for wl in bench.WORKLOADS for pk in bench.PACKING_DESC}
    for key in bench.PROFILED_TRAFFIC:
        assert key[0] in names, key
