"""Host logic of bench.py that needs no GPU: the clock record keeps only the
nvidia-smi samples taken inside the timed window, and reports throttle
reasons seen there."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _line(sm, smax=2070, reasons=("Not Active",) * 4):
    return ", ".join(["0", str(sm), str(smax), "600.0", "0x0", *reasons])


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(lines, t0, t1):
    import bench
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.lines = list(lines)
    s.t0, s.t1 = t0, t1
    return s


def test_only_samples_inside_the_window_count():
    lines = [(0.00, _line(1000)), (0.10, _line(2070)), (0.12, _line(2050)), (0.50, _line(900))]
    rec = _sampler(lines, 0.09, 0.13).stop()
    assert rec["samples"] == 2 and rec["sm_mhz"] == 2060.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == []


def test_short_window_takes_the_first_sample_after_it_opened():
    lines = [(0.00, _line(1000)), (0.30, _line(2070)), (0.60, _line(900))]
    rec = _sampler(lines, 0.10, 0.11).stop()
    assert rec["samples"] == 1 and rec["sm_mhz"] == 2070.0


def test_throttle_reasons_inside_the_window_are_reported():
    hot = ("Not Active", "Active", "Not Active", "Active")  # hw_slowdown .. sw_power_cap
    lines = [(0.00, _line(2070, reasons=("Active",) * 4)), (0.10, _line(1900, reasons=hot))]
    rec = _sampler(lines, 0.05, 0.15).stop()
    assert rec["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_no_samples_is_reported_as_such():
    rec = _sampler([], 0.0, 1.0).stop()
    assert rec["samples"] == 0 and rec["reasons"] == ["no samples"]


def test_cpu_sample_keeps_the_mix_of_sources():
    """The oracle's bounded sample takes each source in proportion to its
    share of the workload: 1,080 Markov and 120 uniform blocks give 14 and 2
    of 16; the mixed workload's three sources give 6, 5 and 5."""
    import bench
    from paper_1109_2348_gb300 import datagen
    s = bench.cpu_sample(datagen.config(5), 16)
    srcs = list(s.sources)
    assert len(srcs) == 16 and srcs.count(datagen.UNIFORM) == 2 and srcs.count(datagen.MARKOV3_Z96) == 14
    s = bench.cpu_sample(datagen.config(2), 16)
    counts = sorted(list(s.sources).count(x) for x in set(s.sources))
    assert counts == [5, 5, 6]
    s = bench.cpu_sample(datagen.config(1), 16)
    assert s.num_blocks == 1
