"""The synthetic workloads the tests and the benchmark run, checked against
their stated recipes: grid, element, laser, electron count and duration of
each configuration, and the batched scan's draws (thickness, element,
log-uniform intensity, macro-electrons proportional to the laser energy,
clamped and summing to the stated total)."""
import math

import numpy as np
import pytest

from paper_2107_01723_gb300 import workloads as W

GOLD = W.MATERIALS["Au"]


def _common(cfg, n, I_Wcm2, n_macro, steps):
    t, l, r = cfg["target"], cfg["laser"], cfg["run"]
    assert (t["nx"], t["ny"], t["nz"]) == n and t["dx"] == 1e-6
    assert t["Z"] == 79.0 and t["n_i"] == 5.9e28
    assert t["I_ex"] == pytest.approx(11.0 * W.EV * 79.0)  # I_ex = 11 eV Z
    assert t["T0"] == pytest.approx(W.KELVIN_PER_EV)  # 1 eV
    assert l["I0"] == pytest.approx(I_Wcm2 * 1e4) and l["lambda"] == 1e-6
    assert l["n_macro"] == n_macro and l["t_inj"] == pytest.approx(100e-15)
    assert l["spot_r"] == 5e-6 and l["cone_half"] == pytest.approx(math.radians(30.0))
    assert l["spot_y"] == pytest.approx(0.5 * n[1] * 1e-6)
    assert l["spot_z"] == pytest.approx(0.5 * n[2] * 1e-6)
    assert r["dt"] == 0.5e-15 and r["seed"] == 0 and cfg["steps"] == steps
    assert (r["kappa_esc"], r["kappa_tnsa"]) == (2.0, 2.7e-3)
    assert r["sigma_dtheta"] == pytest.approx(math.radians(23.0))
    assert r["k_min"] == pytest.approx(10e3 * W.EV) and r["E_cut"] == pytest.approx(1e3 * W.EV)
    assert r["ce_threshold"] == pytest.approx(W.MEV)


def test_correctness_case():
    cfg = W.config1()
    _common(cfg, (32, 32, 32), 1e20, 100_000, 200)
    r = cfg["run"]
    assert (r["n_E"], r["n_theta"]) == (100, 90)
    assert r["tally_E_min"] == pytest.approx(10e3 * W.EV)
    assert r["tally_E_max"] == pytest.approx(100 * W.MEV)


def test_headline_case():
    cfg = W.config2()
    _common(cfg, (128, 128, 128), 1e21, 10_000_000, 20_000)  # 10 ps at 0.5 fs


def test_thick_target_case():
    cfg = W.config3()
    _common(cfg, (500, 256, 256), 1e22, 100_000_000, 200_000)  # 500 um thick, 100 ps


def test_emission_case():
    cfg = W.config5()
    t, r = cfg["target"], cfg["run"]
    assert cfg["n_electrons"] == 2 ** 27 and cfg["steps"] == 1000
    assert cfg["mean_energy"] == pytest.approx(10 * W.MEV)
    assert t["Z"] == 79.0 and t["T0"] == pytest.approx(100.0 * W.KELVIN_PER_EV)
    assert r["physics"] == 1 | 2 | 4 | 64  # drag, scatter, bremsstrahlung, unbounded
    assert (r["n_E"], r["n_theta"]) == (200, 180)
    assert (r["table_rows"], r["table_cols"]) == (200, 200)


def test_batched_scan_draws():
    cfg = W.config4()
    tg, lz = cfg["targets"], cfg["lasers"]
    assert len(tg) == len(lz) == 64
    L = np.array([t["nx"] for t in tg])
    assert L.min() >= 5 and L.max() <= 200 and len(set(L)) > 30
    assert all((t["ny"], t["nz"], t["dx"]) == (64, 64, 1e-6) for t in tg)
    for t, m in zip(tg, cfg["materials"]):
        assert m in ("Al", "Cu", "Au")
        assert (t["Z"], t["n_i"]) == (W.MATERIALS[m]["Z"], W.MATERIALS[m]["n_i"])
    assert set(cfg["materials"]) == {"Al", "Cu", "Au"}
    I = np.array(cfg["I_Wcm2"])
    assert I.min() >= 1e20 and I.max() <= 1e22
    assert np.array([l["I0"] for l in lz]) == pytest.approx(I * 1e4)
    # log10 I uniform on [20, 22]: a loose KS distance for 64 draws
    u = np.sort((np.log10(I) - 20.0) / 2.0)
    assert np.max(np.abs(u - (np.arange(64) + 0.5) / 64)) < 0.25
    n = np.array([l["n_macro"] for l in lz])
    assert n.sum() == 60_000_000
    assert n.min() >= 100_000 and n.max() <= 4_000_000
    free = (n > 100_000) & (n < 4_000_000)
    ratio = n[free] / I[free]
    assert ratio.max() / ratio.min() == pytest.approx(1.0, rel=1e-4)  # proportional to I
    # clamped targets sit on the side of the bound their intensity puts them
    s = ratio.mean()
    assert np.all(s * I[n == 100_000] <= 100_000 * (1 + 1e-6))
    assert np.all(s * I[n == 4_000_000] >= 4_000_000 * (1 - 1e-6))
    # the same seed draws the same scan
    again = W.config4()
    assert [l["n_macro"] for l in again["lasers"]] == list(n)


def test_macro_split_bounds_and_total():
    n = W.macro_split([1.0, 2.0, 3.0, 1000.0], 1000, 10, 500)
    assert sum(n) == 1000 and min(n) >= 10 and max(n) <= 500 and n[3] == 500
    assert n[1] / n[0] == pytest.approx(2.0, rel=0.02) and n[2] / n[0] == pytest.approx(3.0, rel=0.02)
    with pytest.raises(ValueError):
        W.macro_split([1.0, 1.0], 5000, 10, 100)
