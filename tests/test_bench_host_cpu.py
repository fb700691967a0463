"""Host logic of bench.py that decides whether a measurement is valid, on CPU:
the clock sampler's parsing of nvidia-smi rows (median SM clock under load,
the maximum clock, and the throttle reasons seen), and the relative-error
measure the headline is gated on."""
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
