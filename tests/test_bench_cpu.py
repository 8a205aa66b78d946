"""bench.py's reference arm on CPU: the FP64 oracle stepping the benchmark
workload, printing the one JSON line of the benchmark contract."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["config"]["n_sph"] == 120000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_captured_traffic_applies_only_to_its_workload_and_source():
    """The ncu DRAM bytes in profiles/traffic.txt belong to the wheel bin on the
    source they were captured on: no other workload, and no edited source, reports them."""
    sys.path.insert(0, ROOT)
    import bench
    for k in ("pair_stage1", "pair_stage2", "bce"):
        assert bench._traffic(k, captured=False) is None
    v = bench._traffic("pair_stage1")
    assert v is None or v > 1e6          # None once crm_step.cu changed since the capture
    assert bench._traffic("no_such_kernel") is None


def test_dominant_kernel_is_one_kernel():
    """The roofline's kernel: the largest time per launch, not the largest per-step
    total of an id that counts several kernels (the four BCE launches)."""
    sys.path.insert(0, ROOT)
    import bench
    per = {"pair_stage1": 0.061, "pair_stage2": 0.047, "bce": 0.016, "neighbors": 0.003}
    assert bench.dominant_kernel(per, "wheel_bin") == "pair_stage1"
    per_skin0 = dict(per, neighbors=0.11)   # a search at every step dominates
    assert bench.dominant_kernel(per_skin0, "wheel_bin") == "neighbors"
    # the strip: gated search kernels do not compete
    assert bench.dominant_kernel(dict(per, keys=0.5), "strip") == "pair_stage1"
