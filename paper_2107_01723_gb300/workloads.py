"""Seeded synthetic workloads of the fast-electron step, as plain parameter sets.

This module is shared by the CUDA path, its tests and the oracle: it holds
only the parameters of each workload (SI units) and unit conversions, none of
the method's arithmetic.  Every random number of the method is drawn inside
the step from the counter-based generator keyed on `seed`.

Material and laser parameters follow the paper (arXiv 2107.01723):
  * reflux constants kappa_esc = 2, kappa_tnsa = 2.7e-3, sigma = 23 deg
    (Sec. II.A and Table I);
  * mean excitation energy I_ex = 11 eV * Z (Sec. III.B);
  * laser-to-electron efficiency 0.3 and 1 um wavelength (Sec. II.B);
  * a typical resistivity of 1e-6 Ohm m (Sec. III.B) used as the cap.
"""
from __future__ import annotations

import math

EV = 1.602176634e-19          # J per eV
KELVIN_PER_EV = 11604.51812   # K per eV
MEV = 1e6 * EV

# solid-density elements used by the workloads: Z, ion density, conduction Z*
MATERIALS = {
    "Al": {"Z": 13.0, "n_i": 6.03e28, "Zstar": 3.0},
    "Cu": {"Z": 29.0, "n_i": 8.49e28, "Zstar": 1.0},
    "Au": {"Z": 79.0, "n_i": 5.9e28, "Zstar": 1.0},
}


def target(n=(32, 32, 32), dx=1e-6, material="Au", T0_eV=1.0, eta_max=1e-6,
           lnLambda=2.0, lambda1=0.0, lambda2=1.0) -> dict:
    m = MATERIALS[material]
    return {"nx": int(n[0]), "ny": int(n[1]), "nz": int(n[2]), "dx": float(dx),
            "Z": m["Z"], "n_i": m["n_i"], "I_ex": 11.0 * EV * m["Z"],
            "Zstar": m["Zstar"], "lnLambda": lnLambda, "eta_max": eta_max,
            "lambda1": lambda1, "lambda2": lambda2, "T0": T0_eV * KELVIN_PER_EV}


def laser(tgt: dict, I_Wcm2=1e20, n_macro=100_000, spot_r=5e-6, t_inj=100e-15,
          cone_half_deg=30.0, eta_l2e=0.3, lam=1e-6) -> dict:
    """Flat-top injection disc centred on the x = 0 face."""
    return {"I0": I_Wcm2 * 1e4, "lambda": lam, "eta_l2e": eta_l2e, "spot_r": spot_r,
            "spot_y": 0.5 * tgt["ny"] * tgt["dx"], "spot_z": 0.5 * tgt["nz"] * tgt["dx"],
            "t_inj": t_inj, "cone_half": math.radians(cone_half_deg), "n_macro": int(n_macro)}


def run(dt=0.5e-15, seed=0, n_E=100, n_theta=90, E_min=10e3 * EV, E_max=100 * MEV,
        brem_boost=1.0, physics=63, curlB_term=1, max_history=0, target_index=0) -> dict:
    return {"dt": dt, "seed": int(seed), "target_index": int(target_index),
            "kappa_esc": 2.0, "kappa_tnsa": 2.7e-3, "sigma_dtheta": math.radians(23.0),
            "brem_boost": brem_boost, "k_min": 10e3 * EV, "E_cut": 1e3 * EV,
            "n_E": n_E, "n_theta": n_theta, "tally_E_min": E_min, "tally_E_max": E_max,
            "ce_threshold": 1.0 * MEV, "table_rows": 200, "table_cols": 200,
            "table_E_max": 1000 * MEV, "curlB_term": curlB_term, "physics": physics,
            "max_history": int(max_history)}


def config_small(n=(8, 8, 8), n_macro=2000, I_Wcm2=1e20, steps=40, seed=0, spot_r=2e-6,
                 material="Au", t_inj=10e-15, **run_kw) -> dict:
    """A few-tile case the oracle finishes in well under a second."""
    t = target(n=n, material=material)
    return {"target": t, "laser": laser(t, I_Wcm2=I_Wcm2, n_macro=n_macro, spot_r=spot_r,
                                        t_inj=t_inj),
            "run": run(seed=seed, max_history=steps, **run_kw), "steps": steps}


def config1() -> dict:
    """32^3 cells of 1 um gold, 1e5 electrons over 100 fs at 1e20 W/cm^2, 200 steps."""
    t = target(n=(32, 32, 32))
    return {"target": t, "laser": laser(t, I_Wcm2=1e20, n_macro=100_000),
            "run": run(seed=0, max_history=200), "steps": 200}


def config5(n_electrons=2 ** 27, steps=1000) -> dict:
    """Emission microbenchmark: electrons in unbounded uniform gold (no fields,
    no faces, T fixed at 100 eV), drag + scatter + bremsstrahlung only; energies
    exponential with mean 10 MeV, isotropic; photon tally 200 log bins over
    10 keV-100 MeV x 180 polar bins.  The grid is nominal (unused)."""
    t = target(n=(8, 8, 8), T0_eV=100.0)
    physics = 1 | 2 | 4 | 64  # drag, scatter, bremsstrahlung, unbounded
    return {"target": t, "laser": laser(t, I_Wcm2=1e20, n_macro=0, spot_r=1e-6),
            "run": run(n_E=200, n_theta=180, physics=physics, max_history=steps),
            "n_electrons": int(n_electrons), "mean_energy": 10.0 * MEV, "steps": steps}


def config2() -> dict:
    """128^3 cells of 1 um gold, 1e7 electrons over 100 fs at 1e21 W/cm^2, 10 ps."""
    t = target(n=(128, 128, 128))
    return {"target": t, "laser": laser(t, I_Wcm2=1e21, n_macro=10_000_000),
            "run": run(seed=0, max_history=20_000), "steps": 20_000}
