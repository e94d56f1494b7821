"""Host-side helpers of bench.py that run without a GPU."""
import bench

SAMPLE = """0, 2017, 2070, 1210.50, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, 2010, 2070, 1300.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, [N/A], 2070, 900.00, 0x0, Not Active, Not Active, Not Active, Not Active
garbage line
0, 1980, 2070, 1350.00, 0x0000000000000008, Active, Not Active, Not Active, Not Active
"""


def test_clock_samples_parse():
    r = bench.Clocks.parse(SAMPLE)
    assert r["samples"] == 3                       # the [N/A] and malformed lines are skipped
    assert r["sm_mhz"] == 2010 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_samples_empty():
    r = bench.Clocks.parse("")
    assert r["sm_mhz"] is None and r["reasons"] == [] and r["samples"] == 0


def test_replica_seeds_differ():
    assert len({bench.replica_seed(r) for r in range(8)}) == 8
