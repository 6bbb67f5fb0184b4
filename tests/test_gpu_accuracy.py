"""The headline workload's accuracy gate, FP32-mixed against the plain FP64
GPU path: 128^3 gold, 1e7 electrons at 1e21 W/cm^2, from t = 0 through the
injection window and 1 ps beyond (2,200 steps, about 2e10 particle-steps).

The X-ray conversion efficiency above 1 MeV (Sec. III.A: E_xray(k >= 1 MeV)
over the laser energy, E_laser = E_injected / eta_l2e) of the two precisions
must agree within 1 %, and each run's energy budget (E_injected = E_live +
W_field + E_drag + E_xray + E_escaped + E_reflux) must close to 1e-3.  Both
runs draw the same random numbers, so they differ only through rounding.
"""
import pytest

from paper_2107_01723_gb300 import hpic
from paper_2107_01723_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 2200


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_01723_gb300 import build
    build.build()


def ce_and_closure(prec):
    cfg = W.config2()
    sim = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=prec, sort_interval=3)
    sim.step(STEPS)
    t = sim.tallies()
    sim.close()
    rhs = t["E_live"] + t["W_field"] + t["E_drag"] + t["E_xray"] + t["E_escaped"] + t["E_reflux"]
    ce = t["E_xray_above"] / (t["E_injected"] / cfg["laser"]["eta_l2e"])
    return ce, (t["E_injected"] - rhs) / t["E_injected"], t


def test_headline_ce_fp32_vs_fp64_and_energy_closure():
    ce32, cl32, t32 = ce_and_closure(hpic.HPIC_FP32_MIXED)
    ce64, cl64, t64 = ce_and_closure(hpic.HPIC_FP64)
    assert t32["n_injected"] == t64["n_injected"] == 10_000_000
    assert t64["particle_steps"] > 1.5e10
    assert ce64 > 0.0
    assert abs(ce32 / ce64 - 1.0) < 0.01, (ce32, ce64)
    assert abs(cl32) < 1e-3, cl32
    assert abs(cl64) < 1e-10, cl64
