"""The bench's clock record: only nvidia-smi samples stamped inside the
timed region count; a region shorter than the sampling period falls back
to the samples on either side of it.  Host logic only (no nvidia-smi)."""
import datetime

import bench


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def poll(self):
        return 0


def _line(t, mhz, reason="Not Active"):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{stamp}, 0, {mhz}, 2070, 600.5, 0x0, Not Active, Not Active, Not Active, {reason}"


def _sampler(lines):
    s = bench.ClockSampler(0, period_ms=10)
    s.proc = _Done()
    s.lines = lines
    return s


def test_only_samples_inside_the_region_count():
    t0 = 1.8e9
    s = _sampler([_line(t0 - 1, 1000), _line(t0 + 0.1, 2070), _line(t0 + 0.2, 2060, "Active"),
                  _line(t0 + 0.3, 2070), _line(t0 + 2, 900)])
    c = s.stop(t0, t0 + 0.5)
    assert c["in_region"] == 3 and c["samples"] == 3
    assert c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"]


def test_short_region_uses_the_neighbouring_samples():
    t0 = 1.8e9
    s = _sampler([_line(t0 - 2, 900), _line(t0 - 0.05, 2070), _line(t0 + 0.06, 2050),
                  _line(t0 + 3, 800)])
    c = s.stop(t0, t0 + 0.02)
    assert c["in_region"] == 0 and c["samples"] == 2
    assert c["sm_mhz"] == 2060


def test_without_a_region_every_sample_counts():
    t0 = 1.8e9
    s = _sampler([_line(t0, 2070), _line(t0 + 1, 2070, "Active")])
    c = s.stop()
    assert "in_region" not in c and c["samples"] == 2 and c["reasons"] == ["sw_power_cap"]
    assert s.watts == [600.5, 600.5]
