"""The cell sort changes the order of the electrons and nothing else.

The sort inside the step (every sort_interval steps) is folded into the
push: its keys and ranks come from the start-of-step state and the push
writes each electron's new state to its sorted slot of the other buffer.
A run that sorts must therefore carry every electron -- identified by its
id -- through the same trajectory as a run that never sorts, with the same
survivors and the same tallies and grids; the two differ only in the order
of the floating-point atomic additions (FP64 here, so by rounding).  The
cases cover sorting steps during the injection (new electrons appended to
the sorted buffer; the keys from a key pass) and after it (the keys from
the push of the step before), electrons absorbed or escaping on a sorting
step (their sorted slots left dead), a sort on every step, keys dropped when
the electrons are reloaded between the keying and the sorting step, one
target and an uneven batch.
"""
import numpy as np
import pytest

from paper_2107_01723_gb300 import hpic
from paper_2107_01723_gb300 import workloads as W

from parity import (assert_field_close, assert_particles_close, assert_tallies_close,
                    assert_vector_close)

pytestmark = pytest.mark.gpu

TOL = 1e-9  # up to 60 FP64 steps: rounding-order differences grow slowly through the fields


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_01723_gb300 import build
    build.build()


def assert_same_run(a, b, dx):
    assert_particles_close(a.particles(), b.particles(), TOL, dx)
    for f in ("j", "E", "B"):
        assert_vector_close(a.grid, b.grid, f, TOL)
    assert_field_close(a.grid("heat"), b.grid("heat"), TOL, "heat")
    for k in ("T", "eta"):
        err = np.max(np.abs(a.grid(k) - b.grid(k)) / np.abs(b.grid(k)))
        assert err <= TOL, (k, err)
    bt = b.tallies()
    assert_tallies_close(a.tallies(), bt, TOL, TOL * bt["E_injected"])


@pytest.mark.parametrize("interval", [3, 1])
def test_sorting_run_equals_unsorted_run(interval):
    cfg = W.config_small(n=(12, 10, 14), n_macro=6000, I_Wcm2=1e21, steps=40, spot_r=3e-6,
                         t_inj=20e-15)
    dx = cfg["target"]["dx"]
    runs = {}
    for si in (interval, 0):
        s = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=hpic.HPIC_FP64,
                     sort_interval=si)
        s.step(60)  # injecting for 40 steps, then 20 without; the last step sorts
        runs[si] = s
    a, b = runs[interval], runs[0]
    t = b.tallies()
    assert t["n_cut"] + t["n_escaped"] + t["n_reflux_absorbed"] > 0  # some electrons were lost
    assert_same_run(a, b, dx)
    # the sorting run really reordered its electrons, and holds no more slots
    # than electrons injected
    pa, pb = a.particles(), b.particles()
    assert not np.array_equal(pa["id"], pb["id"])
    assert a.n <= t["n_injected"]
    a.close()
    b.close()


def test_keys_are_dropped_when_the_electrons_change():
    """After a keying step (host step 49 keys the sort of step 50) the electrons
    are read and loaded back, which packs them into new slots: the sorting step
    must key them afresh, not use the stale keys and ranks of the old slots."""
    cfg = W.config_small(n=(12, 10, 14), n_macro=6000, I_Wcm2=1e21, steps=40, spot_r=3e-6,
                         t_inj=20e-15)
    dx = cfg["target"]["dx"]
    runs = {}
    for si in (3, 0):
        s = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=hpic.HPIC_FP64,
                     sort_interval=si)
        s.step(50)
        s.set_particles(s.particles())
        s.step(10)
        runs[si] = s
    assert_same_run(runs[3], runs[0], dx)
    for s in runs.values():
        s.close()


def test_sorting_batch_equals_unsorted_batch():
    specs = [((6, 9, 8), "Au", 1e20, 900), ((13, 8, 10), "Al", 1e21, 1500),
             ((9, 12, 7), "Cu", 3e20, 700)]
    targets = [W.target(n=n, material=m) for n, m, _, _ in specs]
    lasers = [W.laser(t, I_Wcm2=I, n_macro=k, spot_r=2e-6, t_inj=10e-15)
              for t, (_, _, I, k) in zip(targets, specs)]
    run = W.run(seed=5, max_history=30)
    a = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP64, sort_interval=3)
    b = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP64, sort_interval=0)
    a.step(30)
    b.step(30)
    for t in range(len(targets)):
        assert_same_run(a.target(t), b.target(t), targets[t]["dx"])
    a.close()
    b.close()
