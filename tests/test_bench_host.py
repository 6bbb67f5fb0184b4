"""The benchmark's roofline arithmetic on the host: which steps of a timed
window sort or key the next sort, the algorithmic bytes of the push launches
and the DRAM traffic scaled from the per-particle-step counter figures.  The
step schedule restated here is the library's: step s sorts when
(s + 1) % interval == 0 and keys the next sort when (s + 2) % interval == 0
(past the injection window)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_sort_and_key_steps_follow_the_schedule():
    # steps 203..232 of the headline: 2 + 3k sort, 1 + 3k key
    assert bench.n_sort_steps(203, 30, 3) == 10
    assert bench.n_key_steps(203, 30, 3) == 10
    sorts = [s for s in range(203, 233) if (s + 1) % 3 == 0]
    keys = [s for s in range(203, 233) if (s + 2) % 3 == 0]
    assert not set(sorts) & set(keys)  # a step never both keys and sorts
    assert bench.n_sort_steps(0, 100, 0) == 0 and bench.n_key_steps(0, 100, 1) == 0
    # every step sorts at interval 1, and none keys (the key pass runs instead)
    assert bench.n_sort_steps(7, 11, 1) == 11


def test_algorithmic_bytes_per_particle_step():
    """Over a long window at a sort every third step the push moves
    60 + 12/3 + 8/3 B per particle-step in FP32 (state in and out, key and
    rank read and id written on a sorting step, key and rank written on a
    keying step); the batch, which keys in a separate pass, 60 + 12/3."""
    steps, n = 3000, 1.0e7
    k_ps = steps * n
    b = bench.push_bytes("fp32", k_ps, steps, 200, steps, 3, keyed=True)
    assert b / k_ps == pytest.approx(60 + 12 / 3 + 8 / 3)
    b = bench.push_bytes("fp32", k_ps, steps, 200, steps, 3, keyed=False)
    assert b / k_ps == pytest.approx(60 + 12 / 3)
    assert bench.push_bytes("fp64", k_ps, steps, 200, steps, 0) / k_ps == pytest.approx(116)


def test_traffic_is_the_launch_average_of_the_measured_figures():
    tb = {"fp32": {"plain": 50.0, "key": 60.0, "sort": 80.0}, "fp64": None}
    n, steps = 1.0e6, 30
    per = bench.push_traffic(tb, "fp32", n * steps, steps, 203, steps, 3)
    assert per == pytest.approx((50.0 * 10 + 60.0 * 10 + 80.0 * 10) / 30 * n)
    # no figure for a kind of step the window holds: no traffic
    assert bench.push_traffic({"fp32": {"plain": 50.0}}, "fp32", n * steps, steps, 203,
                              steps, 3) is None
    assert bench.push_traffic(tb, "fp64", n * steps, steps, 203, steps, 3) is None
    # a window of plain steps only
    assert bench.push_traffic(tb, "fp32", n * 4, 4, 0, 4, 0) == pytest.approx(50.0 * n)


def test_measured_traffic_stays_near_the_algorithmic_bytes():
    """The committed counter figures are within a few percent below the
    algorithmic bytes on a plain step (nothing is re-read) and within the
    partial-sector overhead of the scattered stores on a sorting step."""
    f = bench.NCU_DRAM_BYTES_PER_PSTEP["fp32"]
    assert 0.85 * 60 < f["plain"] <= 60
    assert 0.85 * 68 < f["key"] <= 68
    assert 72 <= f["sort"] < 1.25 * 72
    g = bench.NCU_BATCH_DRAM_BYTES_PER_PSTEP["fp32"]
    assert 0.95 * 60 < g["plain"] < 1.05 * 60 and 72 <= g["sort"] < 1.35 * 72
