"""The benchmark's reference arm runs on the host (the CPU oracle) and must print
one JSON line with the contract's keys; the roofline helpers must report the
bound, achieved/peak fraction and units they state."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ["impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"]:
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "RHS/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_roofline_entries():
    import bench
    fused = bench.roofline_entry("k_bf_left_adj", 2.5, 8e8, 3e10, 6484.3, "measured", {"sm_max_mhz": 2032.0}, 148)
    assert fused["bound"] == "hbm" and fused["unit"] == "GB/s"
    assert abs(fused["achieved"] - 8e8 / 2.5e-3 / 1e9) < 1e-9
    assert abs(fused["frac"] - fused["achieved"] / fused["peak"]) < 1e-12
    eq = fused["fp32_equivalent"]
    assert abs(eq["peak_tflops"] - 148 * 128 * 2 * 2032e6 / 1e12) < 1e-9
    assert abs(eq["tflops"] - 2 * 3e10 / 2.5e-3 / 1e12) < 1e-9
    hbm = bench.roofline_entry("k_ulv_up", 1.0, 6.4843e9, None, 6484.3, "measured", {}, 148)
    assert hbm["bound"] == "hbm" and hbm["unit"] == "GB/s" and abs(hbm["frac"] - 1.0) < 1e-6
    assert "fp32_equivalent" not in hbm
    # bytes model: a per-level transfer launch moves the state twice plus its table
    b = bench.kernel_bytes("k_quad_ms", 1 << 16, 16, 64, {"L": 16, "sU": 13, "sV": 3, "h": 8}, {})
    assert b == 2 * (1 << 16) * 16 * 64 * 8 + 2 * (1 << 16) * 16 * 8


def test_operator_ranks_from_the_stored_oracle_run():
    import bench
    ranks = bench.operator_ranks(1 << 16, 128)
    assert ranks is not None and len(ranks) == 10 and ranks[0] == 0
    assert bench.operator_ranks(1 << 14, 128) is None
