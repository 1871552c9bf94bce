"""Host logic of bench.py that needs no GPU: the clock record taken during
the timed region (which samples count, which throttle reasons are read)."""
import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _line(sm, reasons):
    r = ["Active" if x else "Not Active" for x in reasons]
    return "0, %d, 2032, 700.0, Active, %s\n" % (sm, ", ".join(r))


def test_clock_record_window_and_reasons():
    cs = bench.ClockSampler(0)
    cs.p = _Proc()
    cs.lines = [(0.0, _line(1000, (0, 0, 0, 0))),   # last sample before the timed region: kept
                (1.0, _line(2032, (0, 0, 0, 1))),   # power cap inside the region
                (1.5, _line(2000, (0, 0, 0, 0))),
                (1.9, "garbage line\n"),
                (3.0, _line(1200, (1, 0, 0, 0)))]   # after the region: ignored
    cs.t0, cs.t1 = 0.9, 2.0
    r = cs.stop()
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2000.0 and r["sm_max_mhz"] == 2032.0
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_record_flags_slowdowns():
    cs = bench.ClockSampler(0)
    cs.p = _Proc()
    cs.lines = [(1.0, _line(1500, (1, 1, 0, 0))), (1.1, _line(1500, (0, 0, 1, 0)))]
    cs.t0, cs.t1 = 0.5, 2.0
    r = cs.stop()
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_sampler():
    cs = bench.ClockSampler(0)
    assert cs.stop() is None
