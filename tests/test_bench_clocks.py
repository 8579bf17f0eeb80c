"""The benchmark's clock sampler: parsing of nvidia-smi's CSV samples into the
median SM clock under load, the maximum, and the throttle reasons seen."""
import os
import tempfile

import bench


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _stop_with(lines):
    c = bench.Clocks(0)
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    c.proc = _FakeProc()
    out = c.stop()
    assert not os.path.exists(c.path)
    return out


def _line(sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, 900.5, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_median_under_load_and_reasons():
    lines = [_line(345, 2070)] * 3 + [_line(2070, 2070)] * 5 + [_line(1980, 2070, cap="Active")] * 2
    out = _stop_with(lines)
    assert out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2070.0          # idle samples below half the max are left out
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 10


def test_thermal_reasons_and_bad_lines():
    lines = ["garbage", _line(1500, 2070, hwt="Active"), _line(1400, 2070, hw="Active", swt="Active"),
             "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active"]
    out = _stop_with(lines)
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1450.0 and out["samples"] == 2


def test_no_samples_and_no_tool():
    assert _stop_with([])["reasons"] == ["no samples"]
    c = bench.Clocks(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
