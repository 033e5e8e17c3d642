"""Host logic of bench.py (no GPU): the refill counts behind its per-launch work units
against the oracle's draw rule, and the clock sampler's selection of the samples that
fall inside the timed region."""
import datetime
import os
import tempfile

import bench
from oracle import ranluxpp as R


class _Counting(R.Stream):
    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.refills = 0

    def _refill(self):
        self.refills += 1
        super()._refill()


def test_refill_counts_match_the_draw_rule():
    """1024 doubles from a freshly seeded block, then 4096 more: the refills bench.py
    counts per stream (its work units per launch) are the oracle's."""
    s = _Counting(2048, seed=1)
    s.draw_f64(bench.HBM_COUNT)
    assert (s.refills, s.pos) == (bench.ADV_HBM, bench.POS_AFTER_HBM) == (85, 8)
    s.refills = 0
    s.draw_f64(bench.FUSED_COUNT)
    assert s.refills == bench.ADV_FUSED == 341
    assert bench.ADV_PER_STREAM == 426
    for count in (0, 1, 11, 12, 13, 100, 1000):
        for pos in (0, 8, 22, 24):
            t = _Counting(24, seed=3, pos=pos)
            t.draw_f64(count)
            assert bench.advances_for(count, pos) == (t.refills, t.pos if t.refills else pos + 2 * count)


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def test_clock_samples_inside_the_timed_region():
    c = bench.ClockSampler(0)
    fd, c.path = tempfile.mkstemp()
    os.close(fd)
    t0 = datetime.datetime.now()
    rows = []
    for k in range(8):
        t = t0 + datetime.timedelta(milliseconds=20 * k)
        reason = "Active" if k == 4 else "Not Active"
        rows.append(f"{t.strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]}, 0, {1800 + 10 * k}, 2070, 900.0, 0x0, "
                    f"Not Active, Not Active, Not Active, {reason}")
    with open(c.path, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    c.proc = _Done()
    c.t_begin = t0 + datetime.timedelta(milliseconds=50)
    c.t_end = t0 + datetime.timedelta(milliseconds=110)
    got = c.stop()
    assert got["samples"] == 8 and got["samples_in_timed_region"] == 3      # samples 3, 4, 5
    assert got["sm_mhz"] == 1840 and got["reasons"] == ["sw_power_cap"] and got["sm_max_mhz"] == 2070
    # a region too short to hold a sample: the median over all samples
    fd, c.path = tempfile.mkstemp()
    os.close(fd)
    with open(c.path, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    c.t_begin = c.t_end = t0 + datetime.timedelta(milliseconds=55)
    got = c.stop()
    assert got["samples_in_timed_region"] == 0 and got["sm_mhz"] == 1835


def test_tensor_roofline_is_algorithmic_work_over_the_measured_peak():
    """The tensor path's roofline counts the 5,184 byte products (10,368 flop) of every
    advance over the kernel's time, against the measured tensor peak; the recorded ncu
    figures (traffic, ALU-pipe view) appear only while the kernel sources are the ones
    they were captured from."""
    adv, ms, peak, n = (1 << 20) * 341, 5.79, 1914.4, 1 << 20
    r = bench.tensor_roofline("fused", adv, ms, peak, "measured", n)
    want = adv * 2 * 72 * 72 / (ms * 1e-3) / 1e12
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - want) < 1e-9 * want and abs(r["frac"] - want / peak) < 1e-12
    saved = dict(bench.TC_FUSED_CAPTURE)
    try:
        bench.TC_FUSED_CAPTURE.update(dram_bytes_per_stream=80.0, alu_instr_per_refill=150, streams=262144,
                                      src_sha="0" * 16)
        r = bench.tensor_roofline("fused", adv, ms, peak, "measured", n)
        assert r["traffic"] is None and "secondary_alu_pipe" not in r      # sources changed since
        bench.TC_FUSED_CAPTURE["src_sha"] = bench.kernel_sources_sha()
        r = bench.tensor_roofline("fused", adv, ms, peak, "measured", n)
        assert r["traffic"] == 80.0 * n and r["secondary_alu_pipe"]["instr_per_refill"] == 150
    finally:
        bench.TC_FUSED_CAPTURE.clear()
        bench.TC_FUSED_CAPTURE.update(saved)
