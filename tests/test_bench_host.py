"""Host-side checks of the benchmark's bookkeeping (no GPU): every DRAM-traffic figure that
bench.py may report is recorded, with its source hash, in a committed profile summary, and
the roofline arithmetic follows its stated units."""
import glob
import os

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_have_profiles():
    texts = [open(p, encoding="utf-8").read() for p in glob.glob(os.path.join(ROOT, "profiles", "*.md"))]
    for key, t in bench.TRAFFIC.items():
        assert any(t["sha"] in txt for txt in texts), (key, "no profile names the source hash of its counters")
        assert os.path.exists(os.path.join(bench.CSRC, t["src"])), key
        assert t["bytes"] > 0


def test_traffic_is_null_for_a_changed_source(monkeypatch):
    key = next(iter(bench.TRAFFIC))
    entry = dict(bench.TRAFFIC[key], sha="0" * 16)
    monkeypatch.setitem(bench.TRAFFIC, key, entry)
    assert bench.measured_traffic(key) is None
    assert bench.measured_traffic(("no-such-kernel",)) is None


class _WL:
    n_modes, n_pol, P, N_t = 45, 2, 90, 1 << 17
    parity = np.array([(mx & 1) | ((my & 1) << 1) for g in range(9) for mx in range(g, -1, -1) for my in [g - mx]])


def test_roofline_units_and_peaks():
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
             "_source": "test"}
    kt = {"kerr_ms": 1.0, "lin_ms": 0.1}
    r = bench.roofline(_WL, "pairs-tcgen05", "bf16x3", kt, peaks, "c2")
    # factored pair count at 45 modes: classes of 285, 250, 250, 250 pairs, three rows
    flop = 2 * 3 * (285 ** 2 + 3 * 250 ** 2) * (1 << 17)
    assert r["kernel"] == "kerr" and abs(r["per_launch"]["flop"] / flop - 1) < 1e-12
    assert abs(r["achieved"] - flop / 1e-3 / 1e12) < 1e-9
    assert abs(r["peak"] - 1900.0 / 3) < 1e-9          # burst peak, a third for BF16x3
    # linear step: 26 B per field-sample averaged over the step's four variants
    assert abs(r["other"]["lin_GBps"] - 90 * (1 << 17) * 26.0 / 1e-4 / 1e9) < 1e-6
    r = bench.roofline(_WL, "pairs-tcgen05", "bf16x3", {"kerr_ms": 0.01, "lin_ms": 0.1}, peaks, "c2")
    assert r["kernel"] == "lin" and r["unit"] == "GB/s" and r["peak"] == 6800.0


class _WL240:
    n_modes, n_pol, P, N_t = 120, 2, 240, 1 << 17
    parity = np.zeros(120, dtype=int)


def test_roofline_kappa_paths():
    """The kappa form: FP32 on the CUDA cores against the FP32 FMA peak (2 P^2 flops per
    sample), the tensor-core GEMM against HBM (its bound: 20 B per field-sample averaged over
    the step's one- and two-input launches)."""
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
             "_source": "test"}
    kt = {"kerr_ms": 0.5, "lin_ms": 0.1}
    r = bench.roofline(_WL240, "kappa", "fp32", kt, peaks, "c3k")
    assert r["kernel"] == "kerr" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["per_launch"]["flop"] - 2.0 * 240 * 240 * (1 << 17)) < 1e-3
    assert abs(r["peak"] - 152 * 128 * 2 * 2070.0 * 1e6 / 1e12) < 1e-9
    r = bench.roofline(_WL240, "kappa-tcgen05", "bf16x3", kt, peaks, "c3k")
    bytes_ = 240 * (1 << 17) * 20.0
    assert r["kernel"] == "kerr" and r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6800.0
    assert abs(r["achieved"] - bytes_ / 0.5e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6800.0) < 1e-12
    assert r["other"]["kerr_bound"] == "hbm"
