"""The JSON line of bench.py's reference arm (the CPU oracle timed on a bounded
sample) carries every key of the measurement contract; CPU only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("config,metric", [("fft8_8bit_toy", "encrypted FFTs/s"),
                                           ("refresh32_noisy", "refreshed ciphertexts/s")])
def test_reference_line_keys(config, metric):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", config,
                        "--steps", "1", "--warmup", "0", "--cpu-seconds", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == metric and d["value"] > 0
    assert d["config"]["workload"] == config and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 0


def test_roofline_arithmetic():
    """The roofline's per-product figures at ell 1056 (Ng 2112, 192 digit
    columns): the scope table's algorithmic flops 2 Ng^2 (n+1) ell / 8 for
    `achieved`, the kernel's own MMA flops for `executed`, and the B
    expansion's algorithmic bytes."""
    sys.path.insert(0, ROOT)
    import bench

    class P:
        n, ell = 1, 1056
    assert bench.expand_bytes_per_product(P) == 2112 * 2112 // 8 + 17 * 192 * 256
    r = bench.roofline(P, 2, gate_ms=1000.0, launches=1, gates_timed=1000, tc_columns=192,
                       expand_ms=500.0)
    flops = 2.0 * 2112 * 2112 * 2 * 1056 / 8
    assert r["flops_per_product"] == flops
    assert abs(r["achieved"] - flops * 1000 / 1.0 / 1e12) < 1e-9
    executed = 2.0 * 2112 * 2112 * 192
    assert r["executed"]["flops_per_product"] == executed
    assert abs(r["executed"]["achieved"] - executed * 1000 / 1e12) < 1e-9
    assert abs(r["frac"] / r["executed"]["frac"] - 264 / 192) < 1e-12
    assert abs(r["expand"]["achieved"] - (2112 * 2112 // 8 + 17 * 192 * 256) * 1000 / 0.5 / 1e9) < 1e-6
    assert r["bound"] == "tensor" and r["expand"]["bound"] == "hbm"


@pytest.mark.parametrize("config", ["fft8_8bit_toy", "fft8_8bit_nand"])
def test_reference_arm_never_loads_the_library(config):
    """The reference arm times the oracle on a workload derived from the
    oracle and the synthetic inputs alone: neither the product package nor its
    native library is imported or loaded (P1 configs take the oracle's own
    smallest ell)."""
    code = (
        "import sys, argparse, bench\n"
        f"a = argparse.Namespace(config={config!r}, steps=1, warmup=0, cpu_seconds=0.5, gpus=1)\n"
        "bench.run_reference(a, 0, 1)\n"
        "assert 'paper_1611_08769_gb300' not in sys.modules, 'product package imported'\n"
        "maps = open('/proc/self/maps').read() if sys.platform.startswith('linux') else ''\n"
        "assert 'libsfft' not in maps, 'native library loaded'\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][0])
    assert d["impl"] == "reference" and d["value"] > 0
    if config == "fft8_8bit_nand":
        assert d["config"]["ell"] == 704   # the NAND circuit's own smallest ell (Sec. 7 variant)
