"""GPU parity of the batch: many targets stepped by one launch per kernel kind.

Target t of a batch must follow the same trajectory as the oracle (and as a
single context) run with the same target, laser and run parameters and
target_index = t: the same random numbers are drawn, only the order of
floating-point atomic additions differs.  Tolerances as in the single-target
parity tests; multi-step FP64 runs are held to 1e-9 (rounding-order
differences grow slowly through the fields).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_01723_gb300 import hpic
from paper_2107_01723_gb300 import workloads as W

from parity import (assert_field_close, assert_particles_close, assert_tallies_close,
                    assert_vector_close, by_id)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_01723_gb300 import build
    build.build()


def uneven_batch(seed=3, steps=30):
    """Three targets of different shape, element and intensity (several 4x4x4
    tiles each, ragged in every dimension), all injecting for 20 steps."""
    specs = [((6, 9, 8), "Au", 1e20, 900), ((13, 8, 10), "Al", 1e21, 1500),
             ((9, 12, 7), "Cu", 3e20, 700)]
    targets = [W.target(n=n, material=m) for n, m, _, _ in specs]
    lasers = [W.laser(t, I_Wcm2=I, n_macro=k, spot_r=2e-6, t_inj=10e-15)
              for t, (_, _, I, k) in zip(targets, specs)]
    return targets, lasers, W.run(seed=seed, max_history=steps)


def assert_targets_close(a, b, tol, dx, abs_frac):
    assert_particles_close(a.particles(), b.particles(), tol, dx)
    for f in ("j", "E", "B"):
        assert_vector_close(a.grid, b.grid, f, tol)
    assert_field_close(a.grid("heat"), b.grid("heat"), tol, "heat")
    for k in ("T", "eta"):
        err = np.max(np.abs(a.grid(k) - b.grid(k)) / np.abs(b.grid(k)))
        assert err <= tol, (k, err)
    bt = b.tallies()
    assert_tallies_close(a.tallies(), bt, tol, abs_frac * bt["E_injected"])
    ea, na = a.hist()
    eb, nb = b.hist()
    assert_field_close(ea, eb, tol, "hist E")
    assert_field_close(na, nb, tol, "hist N")


@pytest.mark.parametrize("graph", [True, False])
def test_batch_targets_follow_oracle_fp64(graph):
    """Each target of an FP64 batch against its own oracle run, 30 steps, with
    a cell sort every 5 steps, from captured graphs and from direct launches."""
    targets, lasers, run = uneven_batch()
    b = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP64, sort_interval=5)
    b.set_tuning(2, 5, use_graph=graph)
    b.step(30)
    for t in range(len(targets)):
        o = O.OracleSim(targets[t], lasers[t], dict(run, target_index=t))
        o.step(30)
        assert_targets_close(b.target(t), o, 1e-9, targets[t]["dx"], 1e-9)
        assert b.target(t).clock()[0] == 30
    b.close()


def test_batch_matches_single_contexts_fp32():
    """FP32 batch against FP32 single contexts with the same parameters: two
    steps (injection, then the first push) element by element at 1e-5, then
    ten more steps statistically."""
    targets, lasers, run = uneven_batch(seed=11)
    b = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP32_MIXED, sort_interval=5)
    s = [hpic.Sim(targets[t], lasers[t], dict(run, target_index=t),
                  precision=hpic.HPIC_FP32_MIXED, sort_interval=5) for t in range(len(targets))]
    b.step(2)
    for t, g in enumerate(s):
        g.step(2)
        assert_targets_close(b.target(t), g, 1e-5, targets[t]["dx"], 1e-6)
    b.step(10)
    for t, g in enumerate(s):
        g.step(10)
        bt, gt = b.target(t).tallies(), g.tallies()
        for k in ("E_injected", "E_drag", "W_field", "E_live"):
            assert bt[k] == pytest.approx(gt[k], rel=1e-3), (t, k)
        g.close()
    b.close()


def test_autotune_leaves_state_unchanged():
    """The autotuner times candidates from a snapshot and restores it: the
    tallies and the electron population are bit-identical afterwards, and the
    run continues on the untuned trajectory (FP64, compared by id)."""
    targets, lasers, run = uneven_batch(seed=5, steps=60)
    a = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP64, sort_interval=5)
    r = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP64, sort_interval=5)
    a.step(12)
    r.step(12)
    before = [(a.target(t).tallies(), by_id(a.target(t).particles())) for t in range(3)]
    tune = a.autotune(trial_steps=40)
    assert tune["blocks_per_sm"] in (1, 2)
    assert tune["sort_interval"] in (5, 10, 20, 40)
    assert tune["ms_per_step"] > 0
    for t in range(3):
        tal, p = before[t]
        now = a.target(t).tallies()
        # E_live and E_B_field are summed at read time by atomic reductions
        # (their rounding order varies between reads); the rest is stored state
        for k in tal:
            if k in ("E_live", "E_B_field"):
                assert now[k] == pytest.approx(tal[k], rel=1e-12, abs=0.0), (t, k)
            else:
                assert now[k] == tal[k], (t, k)
        q = by_id(a.target(t).particles())
        for k in p:
            assert np.array_equal(p[k], q[k]), (t, k)
        assert a.target(t).clock() == r.target(t).clock()
    a.step(20)
    r.step(20)
    for t in range(3):
        assert_targets_close(a.target(t), r.target(t), 1e-9, targets[t]["dx"], 1e-9)
    a.close()
    r.close()


def test_batch_target_handles():
    targets, lasers, run = uneven_batch()
    b = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP64, spare_slots=64)
    h = b.target(1).h
    with pytest.raises(hpic.HpicError) as e:
        hpic.hpic_step(h, 1)
    assert e.value.code == hpic.HPIC_ESTATE
    with pytest.raises(hpic.HpicError) as e:
        hpic.hpic_destroy(h)
    assert e.value.code == hpic.HPIC_ESTATE
    # loading within the spare slots works; beyond them is refused
    p = {k: np.full(64, 1e-6) for k in ("x", "y", "z")}
    p.update(ux=np.full(64, 2.0), uy=np.zeros(64), uz=np.zeros(64), tau=np.ones(64),
             id=np.arange(64, dtype=np.uint32) + 100000)
    b.target(1).set_particles(p)
    assert b.target(1).n == 64
    big = {k: np.concatenate([v, v]) for k, v in p.items()}
    big["id"] = np.arange(128, dtype=np.uint32) + 200000
    with pytest.raises(hpic.HpicError) as e:
        b.target(1).set_particles(big)
    assert e.value.code == hpic.HPIC_ENOMEM
    assert b.target(0).n == 0 and b.target(2).n == 0
    b.close()


def test_batch_empty_and_laserless_targets():
    """Targets without a laser hold no electrons; the batch steps them (fields
    and heating only) next to injecting ones."""
    targets, lasers, run = uneven_batch()
    lasers[1] = dict(lasers[1], n_macro=0)
    b = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP64, sort_interval=5)
    b.step(12)
    assert b.target(1).n == 0
    assert b.target(1).tallies()["n_injected"] == 0
    o = O.OracleSim(targets[2], lasers[2], dict(run, target_index=2))
    o.step(12)
    assert_targets_close(b.target(2), o, 1e-9, targets[2]["dx"], 1e-9)
    b.close()


def test_batched_scan_full_size():
    """The 64-target batched scan (6e7 electrons, FP32) in the launch
    configuration the benchmark times: two steps of one thin and one thick
    target against the oracle element by element, then energy closure and
    electron bookkeeping for every target after 60 steps."""
    cfg = W.config4()
    targets, lasers, run = cfg["targets"], cfg["lasers"], cfg["run"]
    b = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP32_MIXED, sort_interval=10)
    b.step(2)
    thin = int(np.argmin([t["nx"] for t in targets]))
    thick = int(np.argmax([t["nx"] for t in targets]))
    for t in (thin, thick):
        o = O.OracleSim(targets[t], lasers[t], dict(run, target_index=t))
        o.step(2)
        assert_targets_close(b.target(t), o, 1e-5, targets[t]["dx"], 1e-6)
        del o
    b.step(58)
    for t in range(len(targets)):
        T = b.target(t).tallies()
        rhs = T["E_live"] + T["W_field"] + T["E_drag"] + T["E_xray"] + T["E_escaped"] + T["E_reflux"]
        assert abs(T["E_injected"] - rhs) / T["E_injected"] < 1e-4, t
        live = T["n_injected"] - T["n_cut"] - T["n_escaped"] - T["n_reflux_absorbed"]
        assert b.target(t).n == live, t
        S = lasers[t]["t_inj"] / run["dt"]
        assert T["n_injected"] == (lasers[t]["n_macro"] * 60) // int(round(S)), t
    b.close()


def test_batch_with_background_physics_and_compounds_fp64():
    """A batch mixing a CH-plastic compound, aluminium and gold, then a batch
    with F_sigma and e-i equilibration on single-element targets: every
    target against its own oracle run (20 steps, FP64)."""
    ch = W.compound([("C", None), ("H", None)], n=(7, 9, 8))
    al = W.target(n=(9, 8, 7), material="Al")
    au = W.target(n=(6, 8, 9), material="Au")
    for targets, physics in (([ch, al, au], hpic.HPIC_ALL),
                             ([al, au], hpic.HPIC_ALL | hpic.HPIC_FSIGMA | hpic.HPIC_EI_EQUIL)):
        lasers = [W.laser(t, I_Wcm2=5e20, n_macro=900, spot_r=2e-6, t_inj=10e-15) for t in targets]
        run = W.run(seed=7, physics=physics, max_history=20)
        b = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP64, sort_interval=5)
        b.step(20)
        for t in range(len(targets)):
            o = O.OracleSim(targets[t], lasers[t], dict(run, target_index=t))
            o.step(20)
            assert_targets_close(b.target(t), o, 1e-9, targets[t]["dx"], 1e-9)
            if physics & hpic.HPIC_EI_EQUIL:
                np.testing.assert_allclose(b.target(t).grid("Ti"), o.grid("Ti"), rtol=1e-9, atol=0)
        b.close()


def test_batch_target_index_override():
    """A batch built from targets 1 and 0 of a scan with their global indices
    draws what the whole scan draws for them."""
    targets, lasers, run = uneven_batch(seed=9)
    whole = hpic.Batch(targets, lasers, run, precision=hpic.HPIC_FP64, sort_interval=5)
    part = hpic.Batch([targets[2], targets[0]], [lasers[2], lasers[0]], run,
                      precision=hpic.HPIC_FP64, sort_interval=5, target_index=[2, 0])
    whole.step(15)
    part.step(15)
    for mine, glob in ((0, 2), (1, 0)):
        assert_targets_close(part.target(mine), whole.target(glob), 1e-9, targets[glob]["dx"], 1e-9)
    whole.close()
    part.close()
