"""Host-side logic of bench.py that its JSON line depends on (no GPU): the algorithmic bytes per
stage and their rooflines, the workload description both arms report, the tuning option, and the
selection of clock samples inside the timed window."""
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


UNITS = dict(N=1000, T=50, V=4000, K=6000, Htl=3000, H=900, M=20)


def test_stage_bytes_follow_the_per_unit_formulas():
    stages, total, comp = bench.stage_roofline(UNITS, [0.0, 1.0, 1.0, 1.0, 2.0, 1.0, 1.0, 0.0, 0.0], 8.0, 1000.0)
    # worked out by hand from the per-unit figures
    want = {"ingest": 25 * 1000, "neighbours": 32 * 1000, "evolution": 24 * 1000 + 4 * 50,
            "construction": 12 * 4000 + 8 * 6000 + 100 * 50, "selection": 20 * 3000, "output": 4 * 900 + 100 * 20}
    assert {k: v["bytes"] for k, v in stages.items()} == want
    # 1 ms stages: bytes / 1e-3 s / 1e9 GB/s; the construction stage took 2 ms
    assert stages["ingest"]["achieved_gbs"] == pytest.approx(25e3 / 1e-3 / 1e9)
    assert stages["construction"]["achieved_gbs"] == pytest.approx(101e3 / 2e-3 / 1e9)
    assert stages["construction"]["frac"] == pytest.approx(stages["construction"]["achieved_gbs"] / 1000.0)
    assert total["bytes"] == sum(want.values()) and total["ms_stages"] == pytest.approx(7.0)
    assert total["frac_of_call"] == pytest.approx(sum(want.values()) / 8e-3 / 1e9 / 1000.0)
    assert comp["bytes"] == 9 * 1000 + 4 * 900 + 112 * 20


def test_units_of_reads_the_call_counters():
    st = dict(clusters=1, tracklets=2, row_visits=3, candidates=4, tracklet_hits=5, hits=6, tracks=7)
    assert bench.units_of(st) == dict(N=1, T=2, V=3, K=4, Htl=5, H=6, M=7)


def test_both_arms_describe_the_same_workload():
    a = bench.workload_config(12, 3278407.2, 1)
    b = bench.workload_config(12, 3278407.2, 1)
    assert a == b and a["clusters_per_event"] == 3278407 and a["resident_events"] == 12
    assert "launch" not in a and "events_per_call" not in a       # launch choices stay out of the workload


def test_tuning_option_parses_fields():
    class T:
        def set_tuning(self, d):
            self.d = d
    t = T()
    bench.apply_tuning(t, "construct_block=64,bin_occupancy=2.0")
    assert t.d == {"construct_block": 64, "bin_occupancy": 2.0}
    u = T()
    bench.apply_tuning(u, "")
    assert not hasattr(u, "d")


def test_clock_samples_are_taken_inside_the_window(tmp_path):
    cs = bench.ClockSampler(0)
    cs.proc = None
    path = tmp_path / "c.csv"
    now = time.time()

    def row(t, mhz, power_cap="Not Active"):
        stamp = time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(t)) + ".%03d" % int((t % 1) * 1000)
        return "%s, 0, %d, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, %s\n" % (stamp, mhz, power_cap)
    path.write_text(row(now - 5, 1000) + row(now - 0.1, 2070) + row(now, 2070, "Active") + row(now + 5, 900))

    class P:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0
    cs.proc = P()
    cs.path = str(path)
    cs.mark(now - 0.2, now + 0.01)
    out = cs.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == 2070 and out["reasons"] == ["sw_power_cap"]
