"""Host-side helpers of the benchmark: the algorithmic flop count behind the
roofline, the derived FP32 peak, the measured tensor peak and its fallback,
and the rule that DRAM traffic is quoted only from a profile summary taken
on the current kernel source."""
import hashlib
import json
import os

import bench


def test_flops_quadratic_term_counts_the_triangle():
    # ||L^-1 k||^2: one multiply-add per nonzero of the N x N lower triangle
    for N in (1, 2, 3, 17, 500):
        macs = sum(i + 1 for i in range(N))
        base = bench.rollout_flops_per_sample_step(0, 0, 0)
        assert bench.rollout_flops_per_sample_step(N, 0, 0) - base - 16 * N == 2 * macs
    # obstacles and lane segments add linearly
    assert (bench.rollout_flops_per_sample_step(10, 4, 7) - bench.rollout_flops_per_sample_step(10, 0, 0)
            == 15 * 4 + 10 * 7)


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA at 2070 MHz
    assert abs(bench.fp32_peak_tflops(2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert abs(bench.fp32_peak_tflops(1000.0, n_sm=1) - 128 * 2 * 1e9 / 1e12) < 1e-12


def test_measured_tensor_peak_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_tensor_peak()[0] == 1900.0          # no file: the stated fallback
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"bf16_tflops": 1234.5}))
    v, note = bench.measured_tensor_peak()
    assert v == 1234.5 and "measured" in note
    (tmp_path / "MEASURED_PEAKS.json").write_text("{}")
    assert bench.measured_tensor_peak()[0] == 1900.0          # malformed: the fallback


def test_traffic_only_from_a_summary_of_the_current_source(tmp_path, monkeypatch):
    csrc, prof = tmp_path / "csrc", tmp_path / "profiles"
    csrc.mkdir()
    prof.mkdir()
    monkeypatch.setattr(bench, "CSRC", str(csrc))
    monkeypatch.setattr(bench, "PROFILES", str(prof))
    src = csrc / "kern.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    assert bench.committed_traffic("kern", "wl") is None              # no summary
    summary = prof / "kern_wl_ncu.md"
    summary.write_text(f"dram bytes per launch (full workload): 123456\nkern.cu sha256: {sha}\n")
    assert bench.committed_traffic("kern", "wl") == 123456.0
    src.write_bytes(b"__global__ void k() { }\n")                     # source changed since
    assert bench.committed_traffic("kern", "wl") is None
    os.remove(summary)
    summary.write_text(f"kern.cu sha256: {hashlib.sha256(src.read_bytes()).hexdigest()}\n")
    assert bench.committed_traffic("kern", "wl") is None              # no traffic line
