"""Host logic of bench.py that decides whether a measurement is valid, on CPU:
the clock sampler's parsing of nvidia-smi rows (median SM clock under load,
the maximum clock, and the throttle reasons seen), the relative-error
measure the headline is gated on, the algorithmic FLOP count of the roofline,
and the reference arm's whole oracle solves of the small configurations."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pc="Not Active"):
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, hwt, swt, pc]


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _stop(rows):
    c = bench.ClockSampler(0)
    c.proc = _Done()
    c.rows = rows
    return c.stop()


def test_clock_sampler_median_max_and_no_reason():
    out = _stop([_row(2070, 2070), _row(2055, 2070), _row(2070, 2070)])
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == [] and out["samples"] == 3


def test_clock_sampler_reports_throttle_reasons():
    out = _stop([_row(1800, 2070, hw="Active"), _row(1700, 2070, swt="Active"), _row(1900, 2070, pc="Active")])
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1800.0


def test_clock_sampler_without_nvidia_smi():
    c = bench.ClockSampler(0)
    out = c.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_rel_err_is_max_over_instances_of_normwise_error():
    S = [np.array([[3.0, 4.0], [0.0, 0.0]]), np.array([[1.0, 0.0]])]
    U = [S[0] + np.array([[0.0, 0.0], [0.3, 0.4]]), S[1] + np.array([[0.0, 0.05]])]
    # instance 0: max_n ||dU_n|| / max_n ||S_n|| = 0.5 / 5; instance 1: 0.05 / 1
    assert bench.rel_err(U, S) == 0.1


def test_algorithmic_count_of_the_step_and_of_a_solve():
    # K = 3, Q = 6: 4 Q K + 2 Q (2K+1) + K^3/3 + 2K^2 = 72 + 84 + 9 + 18
    assert bench.alg_flops_step_1d(3, 6) == 183.0
    from paper_2510_11023_gb300 import workloads
    wl = workloads.small_batch(B=2, P=4)   # K = 7 (m = 3), 33 (m = 2)
    # instance 0: 2 iterations -> slices 4 + 3; instance 1: 3 iterations -> 4 + 3 + 2
    tot, launches = bench.fstage_alg_flops(wl, [2, 3])
    ref = 7 * 3 * bench.alg_flops_step_1d(7, 14) + 9 * 2 * bench.alg_flops_step_1d(33, 66)
    assert launches == 3 and abs(tot - ref) <= 1e-9 * ref


def test_reference_arm_context_timings_of_the_small_configurations():
    out = bench.oracle_paper_shapes()
    for r in out.values():
        assert r["serial_uniform_s"] > 0 and r["serial_hybrid_s"] > 0 and r["parareal_iterations"] >= 1
        assert any(k.startswith("parareal_s_threads") for k in r)


def test_roofline_traffic_only_from_a_matching_capture(tmp_path, monkeypatch):
    # the DRAM traffic of a committed ncu capture is reported only while the CUDA
    # sources (their digest) and the benched configuration are the captured ones
    key = "batched1d|B=256|mixed|l1x2|inexact=3e-06"
    f = tmp_path / "capture.md"

    def write(digest, config, nbytes="123456789"):
        f.write_text(f"# capture\n\n- `sources_sha256`: `{digest}`\n- `config`: `{config}`\n"
                     f"- `bytes_per_launch`: `{nbytes}`\n- other: text\n")

    monkeypatch.setattr(bench, "TRAFFIC_SUMMARY", str(f))
    assert bench.captured_traffic(key) is None                      # no file
    write(bench.source_digest(), key)
    assert bench.captured_traffic(key) == 123456789.0
    assert bench.captured_traffic(key.replace("l1x2", "l1x4")) is None
    write("0" * 64, key)
    assert bench.captured_traffic(key) is None
    write(bench.source_digest(), key, "not-a-number")
    assert bench.captured_traffic(key) is None
    assert len(bench.source_digest()) == 64
