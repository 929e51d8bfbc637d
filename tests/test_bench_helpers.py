"""CPU checks of bench.py's host-side helpers: the clock record taken during
the timed region, the traffic records and their source hashes, and the
slicing of batched samples that the CPU baseline times."""
import importlib.util
import json
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_reads_median_max_and_reasons():
    b = load_bench()
    c = b.ClockSampler(0)
    c.lines = ["2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "garbled line", "[N/A], 2070, 0, 0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["1500, 2070, 1000, 0x40, Not Active, Active, Not Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_thermal_slowdown"]
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_traffic_records_are_used_only_while_their_sources_match(monkeypatch):
    b = load_bench()
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    assert rec
    for key, r in rec.items():
        kernel, workload = key.split("@")
        v = b.recorded_traffic(kernel, workload)
        if "dram_bytes_per_launch" not in r:     # a capture whose traffic does not scale to a full launch
            assert v is None, key
        elif r["sources"] == b.sources_hash(r["files"]):
            assert v == float(r["dram_bytes_per_launch"]), key
        else:                     # the kernel changed since its counters were taken
            assert v is None, key
    # a changed source file (a different hash) makes every record unusable
    monkeypatch.setattr(b, "sources_hash", lambda files: "0" * 16)
    for key in rec:
        assert b.recorded_traffic(*key.split("@")) is None
    assert b.recorded_traffic("no_such_kernel", "no_such_workload") is None


def test_batched_sample_slices_cover_the_range():
    b = load_bench()
    Y_off = np.array([0, 5, 5, 12, 20, 31], dtype=np.int64)
    for lo, hi in ((0, 31), (3, 17), (5, 12), (12, 13), (30, 31)):
        t0, t1, yo = b._batched_tables(Y_off, lo, hi)
        # the clipped offsets cover exactly [lo, hi), table by table
        assert yo[0] == 0 and yo[-1] == hi - lo and (np.diff(yo) >= 0).all()
        for k in range(t0, t1):
            a, c = max(Y_off[k], lo), min(Y_off[k + 1], hi)
            assert yo[k - t0 + 1] - yo[k - t0] == max(c - a, 0)
        # and no table whose targets lie outside is included at either end
        assert Y_off[t0 + 1] > lo or Y_off[t0 + 1] == Y_off[t0]
        assert Y_off[t1 - 1] < hi


def test_per_table_sample_reaches_every_table():
    b = load_bench()
    Y_off = np.array([0, 1000, 1000, 1003, 50_000, 50_001], dtype=np.int64)
    starts, q = b._per_table_sample(Y_off, 5000)
    cnt = np.diff(Y_off)
    assert (q <= cnt).all() and ((q >= 1) == (cnt >= 1)).all()
    assert abs(int(q.sum()) - 5000) <= len(cnt)
    np.testing.assert_array_equal(starts, Y_off[:-1])


def test_sample_parity_counts_mismatches_and_value_errors():
    b = load_bench()
    r = b.sample_parity("1d", np.array([0, 1, 2], np.int32), np.array([0, 1, 2, 9], np.int32))
    assert r["ok"] and r["units"] == 3
    r = b.sample_parity("1d_batched", np.array([0, 1, 2], np.int32), np.array([0, 5, 2], np.int32))
    assert not r["ok"] and r["index_mismatches"] == 1
    idx = np.array([[0, 1], [2, 3]], np.int32)
    val = np.array([1.0, 2.0])
    r = b.sample_parity("2d", (idx, val), (idx.copy(), val * (1 + 1e-13)))
    assert r["ok"] and r["max_rel_err"] <= 1e-12
    r = b.sample_parity("2d", (idx, val), (idx.copy(), val * (1 + 1e-11)))
    assert not r["ok"]
    r = b.sample_parity("2d_batched", (idx, np.array([1.0, np.nan])), (idx.copy(), np.array([1.0, np.nan])))
    assert r["ok"]
    assert b.sample_parity("1d", np.zeros(1, np.int32), None) is None


def test_host_link_peak_at_the_steps_split():
    """The end-to-end roofline: a 1D step sends 8 bytes per target and
    returns 4, so the host-to-device direction bounds it (12 bytes per
    8 / 210.5 GB/s); a 2D step moves 16 each way, so the rate of both
    directions together bounds it; a one-way step gets that direction."""
    b = load_bench()
    link = {"h2d": 210.5, "d2h": 192.7, "both": 340.5}
    assert abs(b.link_peak_for(8, 4, link) - 12 / (8 / 210.5)) < 1e-9
    assert abs(b.link_peak_for(16, 16, link) - 340.5) < 1e-9
    assert abs(b.link_peak_for(8, 0, link) - 210.5) < 1e-9
    assert abs(b.link_peak_for(0, 4, link) - 192.7) < 1e-9
    assert abs(b.link_peak_for(1, 100, link) - 101 / (100 / 192.7)) < 1e-9
