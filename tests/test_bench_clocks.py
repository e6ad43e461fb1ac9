"""bench.py's clock summary: only the nvidia-smi samples taken inside the timed region
count (the one just before it when none came after), and each throttle reason that was
active in one of them is reported."""
import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines, first):
    c = bench.ClockSampler(0)
    c.proc = _Proc()
    c.lines = list(lines)
    c.first = first
    return c


def _line(sm, smax=2070, hw="Not Active", thermal="Not Active", sw_thermal="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, 900.00, 0x0, {hw}, {thermal}, {sw_thermal}, {cap}"


def test_samples_before_the_timed_region_are_left_out():
    lines = [_line(345), _line(345), _line(2070), _line(2070, cap="Active"), _line(2055)]
    out = _sampler(lines, 2).stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_no_sample_inside_falls_back_to_the_last_one_before():
    lines = [_line(300), _line(1995, thermal="Active")]
    out = _sampler(lines, 2).stop()
    assert out["samples"] == 1 and out["sm_mhz"] == 1995.0
    assert out["reasons"] == ["hw_thermal_slowdown"]


def test_unreadable_lines_are_skipped():
    out = _sampler(["garbage", _line(2070), "0, N/A, N/A, N/A, 0x0, a, b, c, d"], 0).stop()
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0
