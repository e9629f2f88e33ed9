"""bench.py's reference arm (the oracle on the host cores) prints one JSON line with the
fields of the benchmark contract; runs without a GPU (~20 s)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, check=True, capture_output=True, text=True, timeout=600).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "MDOF/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "grid2d_K16_p4_m256" and d["config"]["iters"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_combined_roofline_arithmetic():
    """t_roof sums per-class max(bytes / HBM, flops / pipe peak), the interior FD's tensor
    work at the BF16 peak."""
    sys.path.insert(0, ROOT)
    import bench
    pk = {"hbm_gbs": 1000.0, "bf16_tflops": 100.0}
    prof = {"apply": {"ms": 5.0, "launches": 3, "flops": 2e12 * bench.FP64_PEAK_TFLOPS / 1e3, "bytes": 1e9},
            "interior_fd": {"ms": 9.0, "launches": 4, "flops": 7e9, "bytes": 4e9},
            "vector": {"ms": 1.0, "launches": 2, "flops": 0.0, "bytes": 3e9},
            "tensor_exec": {"ms": 0.0, "launches": 0, "flops": 5e11, "bytes": 0.0}}
    r = bench.combined_roofline(prof, 20.0, "fp64", pk)
    # apply: max(1 ms HBM, 2 ms FP64) = 2; FD: max(4 ms HBM, 5 ms tensor) = 5; vector: 3 ms HBM
    assert r["per_class_ms"] == {"apply": 2.0, "interior_fd": 5.0, "vector": 3.0}
    assert r["t_roof_ms"] == 10.0 and r["frac"] == 0.5
    r32 = bench.combined_roofline(prof, 20.0, "bf16", pk)
    assert r32["per_class_ms"]["apply"] < 2.0 and r32["alu_peak_tflops"] > 60
