"""Host-side logic of the benchmark, without a GPU: the clock sampler keeps only the
samples inside the timed window (and says when it had to fall back to all of
them), reports the throttle reasons it saw, and the fused surrogate kernel's phase
summary divides the statistics counters per CTA, and the bf16 peak of the network
roofline comes from the measured-peaks file when there is one."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(sm, reason="Not Active", power_cap="Not Active"):
    # clocks.sm, clocks.max.sm, power.draw, active reasons, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    return f"{sm}, 2070, 900.0, 0x0, {reason}, Not Active, Not Active, {power_cap}"


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(samples, t0, t1):
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.lines = samples
    c.t0, c.t1 = t0, t1
    return c


def test_only_samples_inside_the_timed_window():
    samples = [(0.0, _line(1000)), (1.0, _line(2070)), (1.5, _line(2060)), (2.0, _line(2070)),
               (3.0, _line(500, reason="Active"))]
    out = _sampler(samples, 0.9, 2.1).stop()
    assert out["samples"] == 3 and out["samples_in_timed_window"] is True
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []                       # the slowdown came after the window
    assert abs(out["window_s"] - 1.2) < 1e-12


def test_falls_back_to_every_sample_and_says_so():
    samples = [(0.0, _line(2070)), (5.0, _line(1900, power_cap="Active"))]
    out = _sampler(samples, 1.0, 2.0).stop()
    assert out["samples"] == 2 and out["samples_in_timed_window"] is False
    assert out["reasons"] == ["sw_power_cap"]


def test_reasons_inside_the_window_are_reported():
    samples = [(1.0, _line(2070, reason="Active")), (1.2, _line(2070, power_cap="Active"))]
    out = _sampler(samples, 0.5, 1.5).stop()
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_malformed_lines_are_skipped():
    samples = [(1.0, "garbage"), (1.1, "N/A, N/A, N/A, N/A, N/A, N/A, N/A, N/A"), (1.2, _line(2000))]
    out = _sampler(samples, 0.0, 2.0).stop()
    assert out["samples"] == 1 and out["sm_mhz"] == 2000.0


def test_surrogate_phase_summary_is_per_cta():
    st = {"sur_ns_cta": 152 * 140_000, "sur_ns_cta_max": 163_000, "sur_ns_produce": 152 * 60_000,
          "sur_ns_list": 152 * 25_000, "sur_ns_eval": 152 * 70_000}
    ph = bench.sur_phases(st, 152)
    assert ph["cta_mean"] == 140.0 and ph["cta_max"] == 163.0
    assert ph["produce"] == 60.0 and ph["cull_lists"] == 25.0 and ph["evaluate"] == 70.0
    assert abs(ph["other"] - 10.0) < 1e-9 and ph["ctas"] == 152


def test_bf16_peak_comes_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.bf16_peak_tflops() == (bench.BF16_TFLOPS_FALLBACK, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"bf16_tflops": 1945.3, "hbm_gbs": 6681.5}')
    assert bench.bf16_peak_tflops() == (1945.3, "measured (bf16 burst)")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6681.5}')
    assert bench.bf16_peak_tflops()[1] == "fallback"


def test_network_flops_split():
    # the two 128 x 128 layers are the tensor-core part of one query's FLOPs
    assert bench.MLP_TENSOR_FLOPS_PER_QUERY == 65536
    assert bench.MLP_FLOPS_PER_QUERY - bench.MLP_TENSOR_FLOPS_PER_QUERY == 2 * (3 * 128 + 128)
