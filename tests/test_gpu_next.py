"""GPU parity of the optional background physics: the F_sigma ionised-
screening enhancement of bremsstrahlung (App. B) and the electron-ion
temperature equilibration (App. A), against the FP64 oracle.

Aluminium (Z*/Z = 3/13) makes F_sigma depart from 1 by a few per cent; the
ion temperature is set log-uniform between 0.5 eV and 2 keV so that F_sigma
varies from cell to cell and the equilibration moves both temperatures.
Tolerances as in the single-target parity tests.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_01723_gb300 import hpic
from paper_2107_01723_gb300 import workloads as W

from parity import (assert_field_close, assert_particles_close, assert_tallies_close,
                    assert_vector_close, gpu_from_oracle, tally_delta)

pytestmark = pytest.mark.gpu

PREC = {"fp64": (hpic.HPIC_FP64, 1e-12, 1e-12), "fp32": (hpic.HPIC_FP32_MIXED, 1e-5, 1e-6)}
NEXT1 = hpic.HPIC_ALL | hpic.HPIC_FSIGMA | hpic.HPIC_EI_EQUIL
EV_K = 11604.51812


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_01723_gb300 import build
    build.build()


def next1_cfg(seed=5):
    return W.config_small(n=(12, 10, 14), n_macro=6000, I_Wcm2=1e21, steps=40, spot_r=3e-6,
                          t_inj=20e-15, material="Al", physics=NEXT1, seed=seed)


def ion_temperatures(cfg, seed=2):
    t = cfg["target"]
    n = t["nx"] * t["ny"] * t["nz"]
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(0.5), math.log(2000.0), n)) * EV_K


def assert_cell_scalars_close(g, o, tol):
    for k in ("T", "eta", "Ti"):
        err = np.max(np.abs(g.grid(k) - o.grid(k)) / np.abs(o.grid(k)))
        assert err <= tol, (k, err)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fsigma_and_equilibration_single_step(prec):
    cfg = next1_cfg()
    o = O.OracleSim(cfg["target"], cfg["laser"], cfg["run"])
    o.set_grid("Ti", ion_temperatures(cfg))
    o.step(30)
    prec_id, tol, abs_frac = PREC[prec]
    g = gpu_from_oracle(o, cfg, prec_id)
    ot0 = o.tallies()
    o.step(1)
    g.step(1)
    dx = cfg["target"]["dx"]
    assert_particles_close(g.particles(), o.particles(), tol, dx)
    for f in ("j", "E", "B"):
        assert_vector_close(g.grid, o.grid, f, tol)
    assert_cell_scalars_close(g, o, tol)
    ot = tally_delta(o.tallies(), ot0)
    assert_tallies_close(g.tallies(), ot, tol, abs_frac * ot0["E_live"])
    g.close()


def test_fsigma_and_equilibration_run_tracks_oracle():
    """40 steps from an empty target in FP64: injection, heating, e-i exchange
    and F_sigma-weighted emission stay on the oracle's trajectory."""
    cfg = next1_cfg(seed=9)
    Ti = ion_temperatures(cfg, seed=3)
    o = O.OracleSim(cfg["target"], cfg["laser"], cfg["run"])
    g = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=hpic.HPIC_FP64, sort_interval=10)
    o.set_grid("Ti", Ti)
    g.set_grid("Ti", Ti)
    o.step(40)
    g.step(40)
    dx = cfg["target"]["dx"]
    assert_particles_close(g.particles(), o.particles(), 1e-9, dx)
    assert_cell_scalars_close(g, o, 1e-9)
    ot = o.tallies()
    assert_tallies_close(g.tallies(), ot, 1e-9, 1e-9 * ot["E_injected"])
    # the exchange moved the ion temperatures toward T_e
    assert np.max(np.abs(g.grid("Ti") - Ti) / Ti) > 1e-3
    g.close()


def test_equilibration_alone_conserves_fp64():
    """No electrons: Z* T_e + T_i per cell is conserved by the GPU exchange as
    by the oracle's."""
    cfg = W.config_small(n=(6, 5, 7), n_macro=0, material="Al", physics=hpic.HPIC_EI_EQUIL)
    t = cfg["target"]
    n = t["nx"] * t["ny"] * t["nz"]
    rng = np.random.default_rng(1)
    Te = rng.uniform(1.0, 50.0, n) * EV_K
    Ti = rng.uniform(0.5, 5.0, n) * EV_K
    o = O.OracleSim(cfg["target"], cfg["laser"], cfg["run"])
    g = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=hpic.HPIC_FP64)
    for s in (o, g):
        s.set_grid("T", Te)
        s.set_grid("Ti", Ti)
        s.step(25)
    assert_cell_scalars_close(g, o, 1e-12)
    inv = t["Zstar"] * Te + Ti
    assert np.allclose(t["Zstar"] * g.grid("T") + g.grid("Ti"), inv, rtol=1e-13, atol=0)
    g.close()


# ---------------------------------------------------------------- Gaussian injection envelope
def gauss_cfg(per_cell=60, seed=4, physics=hpic.HPIC_ALL):
    t = W.target(n=(16, 12, 12), dx=0.7e-6)
    las = W.laser_gauss(t, I_Wcm2=1e21, per_cell=per_cell)
    return {"target": t, "laser": las, "run": W.run(seed=seed, physics=physics, max_history=40)}


def assert_weights_close(g, o, tol):
    gp, ow = g.particles(), O.weights(o)
    op = o.particles()
    gi, oi = np.argsort(gp["id"]), np.argsort(op["id"])
    assert np.array_equal(gp["id"][gi], op["id"][oi])
    gw = g.weights()[gi]
    np.testing.assert_allclose(gw, ow[oi], rtol=tol, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gaussian_injection_first_steps(prec):
    """Steps 0 and 1 of the paper's envelope: per-cell electrons with their own
    weights and local mean energies, Moore-capped cones, then the first push."""
    cfg = gauss_cfg()
    prec_id, tol, abs_frac = PREC[prec]
    o = O.OracleSim(cfg["target"], cfg["laser"], cfg["run"])
    g = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=prec_id)
    for _ in range(2):
        o.step(1)
        g.step(1)
        dx = cfg["target"]["dx"]
        assert_particles_close(g.particles(), o.particles(), tol, dx)
        assert_weights_close(g, o, tol)
        ot = o.tallies()
        assert_tallies_close(g.tallies(), ot, tol, abs_frac * ot["E_injected"])
    assert o.tallies()["n_injected"] > 0
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gaussian_single_step_from_state(prec):
    """One full step from the oracle's state 12 steps into the envelope
    (electrons of many weights moving, fields and heating on)."""
    cfg = gauss_cfg(per_cell=40, seed=8)
    o = O.OracleSim(cfg["target"], cfg["laser"], cfg["run"])
    o.step(12)
    prec_id, tol, abs_frac = PREC[prec]
    g = gpu_from_oracle(o, cfg, prec_id)
    ot0 = o.tallies()
    o.step(1)
    g.step(1)
    dx = cfg["target"]["dx"]
    assert_particles_close(g.particles(), o.particles(), tol, dx)
    assert_weights_close(g, o, tol)
    for f in ("j", "E", "B"):
        assert_vector_close(g.grid, o.grid, f, tol)
    assert_cell_scalars_close(g, o, tol)
    ot = tally_delta(o.tallies(), ot0)
    assert_tallies_close(g.tallies(), ot, tol, abs_frac * ot0["E_live"])
    g.close()


def test_gaussian_run_tracks_oracle_fp64():
    cfg = gauss_cfg(per_cell=30, seed=12)
    o = O.OracleSim(cfg["target"], cfg["laser"], cfg["run"])
    g = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=hpic.HPIC_FP64, sort_interval=5)
    o.step(30)
    g.step(30)
    dx = cfg["target"]["dx"]
    assert_particles_close(g.particles(), o.particles(), 1e-9, dx)
    assert_weights_close(g, o, 1e-12)
    ot = o.tallies()
    assert_tallies_close(g.tallies(), ot, 1e-9, 1e-9 * ot["E_injected"])
    g.close()


# ---------------------------------------------------------------- compounds, Lee-More fit
def ch_cfg(seed=6, n=(10, 9, 12), **tkw):
    t = W.compound([("C", None), ("H", None)], n=n, **tkw)
    las = W.laser(t, I_Wcm2=1e21, n_macro=5000, spot_r=3e-6, t_inj=20e-15)
    return {"target": t, "laser": las, "run": W.run(seed=seed, max_history=40)}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_compound_single_step(prec):
    """CH plastic: summed stopping powers, scatter variances and emission
    rates, the n_e-weighted heat capacity and the compound resistivity, one
    step from the oracle's state 20 steps in."""
    cfg = ch_cfg()
    o = O.OracleSim(cfg["target"], cfg["laser"], cfg["run"])
    o.step(20)
    prec_id, tol, abs_frac = PREC[prec]
    g = gpu_from_oracle(o, cfg, prec_id)
    ot0 = o.tallies()
    o.step(1)
    g.step(1)
    dx = cfg["target"]["dx"]
    assert_particles_close(g.particles(), o.particles(), tol, dx)
    for f in ("j", "E", "B"):
        assert_vector_close(g.grid, o.grid, f, tol)
    assert_cell_scalars_close(g, o, tol)
    ot = tally_delta(o.tallies(), ot0)
    assert_tallies_close(g.tallies(), ot, tol, abs_frac * ot0["E_live"])
    g.close()


def test_compound_run_tracks_oracle_fp64():
    cfg = ch_cfg(seed=13)
    o = O.OracleSim(cfg["target"], cfg["laser"], cfg["run"])
    g = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=hpic.HPIC_FP64, sort_interval=10)
    o.step(35)
    g.step(35)
    assert_particles_close(g.particles(), o.particles(), 1e-9, cfg["target"]["dx"])
    assert_cell_scalars_close(g, o, 1e-9)
    ot = o.tallies()
    assert_tallies_close(g.tallies(), ot, 1e-9, 1e-9 * ot["E_injected"])
    g.close()


def test_two_overlapping_golds_equal_one_gold_on_gpu():
    """The paper's compound property on the CUDA path: gold at n_i and gold at
    n_i/2 twice give the same run (FP64, 20 steps)."""
    cfg = W.config_small(n=(8, 7, 9), n_macro=1500, steps=20, I_Wcm2=1e21, spot_r=2e-6)
    half = cfg["target"]["n_i"] / 2
    two_t = W.compound([("Au", half), ("Au", half)], n=(8, 7, 9))
    a = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=hpic.HPIC_FP64)
    b = hpic.Sim(two_t, cfg["laser"], cfg["run"], precision=hpic.HPIC_FP64)
    a.step(20)
    b.step(20)
    assert_particles_close(b.particles(), a.particles(), 1e-11, cfg["target"]["dx"])
    assert_cell_scalars_close(b, a, 1e-11)
    a.close()
    b.close()


def test_lee_more_fit_run_tracks_oracle_fp64():
    """The paper's reduced Lee-More fit (lambda1 = 7, lambda2 = 3.5) with the
    cap lifted, so that eta moves between its cold and hot limits."""
    t = W.target(n=(10, 9, 12), T0_eV=5.0, lambda1=7.0, lambda2=3.5, eta_max=1e-3)
    las = W.laser(t, I_Wcm2=1e21, n_macro=5000, spot_r=3e-6, t_inj=20e-15)
    run = W.run(seed=21, max_history=40)
    o = O.OracleSim(t, las, run)
    g = hpic.Sim(t, las, run, precision=hpic.HPIC_FP64, sort_interval=10)
    o.step(30)
    g.step(30)
    assert_particles_close(g.particles(), o.particles(), 1e-9, t["dx"])
    assert_cell_scalars_close(g, o, 1e-9)
    eta = o.grid("eta")
    assert eta.max() > 1.01 * eta.min()  # eta(T) has moved off its initial value
    g.close()
