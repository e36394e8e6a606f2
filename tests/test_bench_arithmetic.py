"""bench.py's measurement arithmetic, on the CPU:
- the algorithmic bytes of one call;
- the whole-job aggregate over replicas;
- where the roofline peaks come from (the measured file, else the stated fallback);
- the parsing of the nvidia-smi clock samples and their throttle reasons;
- the guard that voids the ncu traffic record once the kernels it was taken on change.
"""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2501_14911_gb300 import synthetic  # noqa: E402


def test_bytes_per_call_of_the_sweep():
    p = synthetic.SWEEP
    assert (p.Nm, p.Nd, p.Nt) == (65536, 128, 256)
    # the spectral blocks once, (N_t + 1) N_d N_m complex FP64 (34.49 GB), plus one m and one d in FP64
    blocks = 257 * 128 * 65536 * 16
    assert blocks == 34_493_956_096
    assert bench.bytes_per_call(p, 8, 16) == blocks + (256 * 65536 + 256 * 128) * 8
    # FP32 vectors with FP32 spectra: half of each
    assert bench.bytes_per_call(p, 4, 8) == blocks // 2 + (256 * 65536 + 256 * 128) * 4


def test_aggregate_is_the_sum_over_replicas():
    assert bench.aggregate_gbs(1, 1e9, 10, 1000.0) == 10.0
    assert bench.aggregate_gbs(4, 1e9, 10, 1000.0) == 40.0  # weak scaling: each rank moves its own bytes
    assert bench.aggregate_gbs(2, 1e9, 10, 2000.0) == 10.0  # the slowest rank's time bounds the job


def test_peaks_come_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == (6800.0, 1900.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6787.2, "bf16_tflops": 1902.0}))
    assert bench.load_peaks() == (6787.2, 1902.0, "measured")


class _Exited:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_are_parsed_per_gpu_with_their_throttle_reasons(tmp_path):
    c = bench.Clocks("GPU-abc")
    c.path = str(tmp_path / "clocks.csv")
    rows = [
        "GPU-abc, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "GPU-abc, 2060, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active",
        "GPU-xyz, 1000, 2070, 100.0, 0x8, Active, Not Active, Not Active, Not Active",  # another GPU
        "GPU-abc, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # unreadable
        "a truncated line",
    ]
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    c.proc = _Exited()
    out = c.stop()
    assert out == {"sm_mhz": 2065.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}
    assert not os.path.exists(c.path)
    with open(c.path, "w") as f:
        f.write("GPU-abc, 1400, 2070, 300.0, 0x40, Not Active, Active, Not Active, Not Active\n")
    assert bench.Clocks.stop(c)["reasons"] == ["hw_thermal_slowdown"]
    assert bench.Clocks("GPU-abc").stop() is None  # no sampler started


def test_traffic_record_is_void_once_its_kernels_change(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic_spectral_products.json")) as f:
        rec = json.load(f)
    key = "df64_bytes_per_launch"
    fresh = rec["source_hash"] == bench.kernel_source_hash(rec["kernels"])
    assert bench.ncu_traffic(key) == (rec[key] if fresh else None)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda names: rec["source_hash"])
    assert bench.ncu_traffic(key) == rec[key]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda names: "0" * 16)
    assert bench.ncu_traffic(key) is None
