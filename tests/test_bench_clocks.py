"""Host logic of bench.py's clock record (no GPU, no NVML): the summary of the samples the NVML
sampler took and the decoding of the clock-event reason bits (NVML's documented bit values:
0x4 software power cap, 0x8 hardware slowdown, 0x20 software thermal slowdown, 0x40 hardware
thermal slowdown, 0x80 hardware power brake)."""
import threading

import bench


class _FakeNvml:
    def __init__(self):
        self.shut = False

    def nvmlShutdown(self):
        self.shut = True
        return 0


def _summary(samples, sm_max=2070.0):
    s = bench.NvmlClockSampler("fake-uuid")
    s.nvml = _FakeNvml()
    s.thread = threading.Thread(target=lambda: None)
    s.thread.start()
    s.samples = list(samples)
    s.sm_max = sm_max
    out = s.stop()
    assert s.nvml.shut
    return out


def test_clock_summary_median_and_reasons():
    out = _summary([(2070.0, 0x0), (1987.0, 0x4), (2070.0, 0x1), (1900.0, 0x4 | 0x40)])
    assert out["sm_mhz"] == 2028.5 and out["sm_min_mhz"] == 1900.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]     # idle (0x1) is not a slowdown
    assert out["samples"] == 4 and "NVML" in out["source"]


def test_clock_summary_without_samples_or_library():
    assert _summary([]) is None
    assert bench.NvmlClockSampler("x").stop() is None                   # never started
    out = _summary([(1500.0, 0x8 | 0x20 | 0x80)], sm_max=None)
    assert out["reasons"] == ["hw_power_brake_slowdown", "hw_slowdown", "sw_thermal_slowdown"]
    assert out["sm_max_mhz"] == 1500.0
