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

# solid-density elements used by the workloads: Z, ion density, conduction
# Z*, standard atomic weight A (ion mass in u)
MATERIALS = {
    "Al": {"Z": 13.0, "n_i": 6.03e28, "Zstar": 3.0, "A": 26.982},
    "Cu": {"Z": 29.0, "n_i": 8.49e28, "Zstar": 1.0, "A": 63.546},
    "Au": {"Z": 79.0, "n_i": 5.9e28, "Zstar": 1.0, "A": 196.967},
    # the elements of CH plastic (1.05 g/cm^3: 4.86e28 m^-3 of each)
    "C": {"Z": 6.0, "n_i": 4.86e28, "Zstar": 1.0, "A": 12.011},
    "H": {"Z": 1.0, "n_i": 4.86e28, "Zstar": 1.0, "A": 1.008},
}


def target(n=(32, 32, 32), dx=1e-6, material="Au", T0_eV=1.0, eta_max=1e-6,
           lnLambda=2.0, lambda1=0.0, lambda2=1.0) -> dict:
    m = MATERIALS[material]
    return {"nx": int(n[0]), "ny": int(n[1]), "nz": int(n[2]), "dx": float(dx),
            "Z": m["Z"], "n_i": m["n_i"], "I_ex": 11.0 * EV * m["Z"],
            "Zstar": m["Zstar"], "lnLambda": lnLambda, "eta_max": eta_max,
            "lambda1": lambda1, "lambda2": lambda2, "T0": T0_eV * KELVIN_PER_EV,
            "A_ion": m["A"], "n_extra": 0, "pad": 0, "extra": []}


def element(material: str, n_i=None) -> dict:
    """One element of a compound (App. A) at its ion density (m^-3)."""
    m = MATERIALS[material]
    return {"Z": m["Z"], "n_i": float(m["n_i"] if n_i is None else n_i), "I_ex": 11.0 * EV * m["Z"],
            "Zstar": m["Zstar"], "A_ion": m["A"]}


def compound(parts, n=(32, 32, 32), dx=1e-6, T0_eV=1.0, eta_max=1e-6, lnLambda=2.0,
             lambda1=0.0, lambda2=1.0) -> dict:
    """A compound solid filling the box: parts = [(material, n_i or None), ...];
    the first is the target's own element, the rest (up to three) share
    every cell with it."""
    mat0, n0 = parts[0]
    t = target(n=n, dx=dx, material=mat0, T0_eV=T0_eV, eta_max=eta_max, lnLambda=lnLambda,
               lambda1=lambda1, lambda2=lambda2)
    if n0 is not None:
        t["n_i"] = float(n0)
    t["extra"] = [element(m, ni) for m, ni in parts[1:]]
    t["n_extra"] = len(t["extra"])
    return t


ENV_FLAT, ENV_GAUSS = 0, 1


def laser(tgt: dict, I_Wcm2=1e20, n_macro=100_000, spot_r=5e-6, t_inj=100e-15,
          cone_half_deg=30.0, eta_l2e=0.3, lam=1e-6, moore_cap=0) -> dict:
    """Flat-top injection disc centred on the x = 0 face."""
    return {"I0": I_Wcm2 * 1e4, "lambda": lam, "eta_l2e": eta_l2e, "spot_r": spot_r,
            "spot_y": 0.5 * tgt["ny"] * tgt["dx"], "spot_z": 0.5 * tgt["nz"] * tgt["dx"],
            "t_inj": t_inj, "cone_half": math.radians(cone_half_deg), "n_macro": int(n_macro),
            "envelope": ENV_FLAT, "per_cell": 0, "r_fwhm": 0.0, "t_fwhm": 0.0, "f_min": 0.0,
            "g_min": 0.0, "moore_cap": int(moore_cap), "pad": 0}


def laser_gauss(tgt: dict, I_Wcm2=1e21, per_cell=1226, r_fwhm=5e-6, t_fwhm=40e-15,
                f_min=0.5, g_min=0.1, cone_half_deg=20.0, moore_cap=1, eta_l2e=0.3,
                lam=1e-6) -> dict:
    """The paper's injection (Sec. II.B): Gaussian f(r) of radial FWHM r_fwhm on
    the x = 0 face and Gaussian g(t) of FWHM t_fwhm, nothing injected where
    g < 0.1 or into cells with f < 0.5, 1226 macro-electrons per injecting
    cell per step, cone half-angle min(20 deg, atan(sqrt(2/(gamma - 1))))."""
    d = laser(tgt, I_Wcm2=I_Wcm2, n_macro=0, spot_r=0.5 * r_fwhm, cone_half_deg=cone_half_deg,
              eta_l2e=eta_l2e, lam=lam, moore_cap=moore_cap)
    d.update(envelope=ENV_GAUSS, per_cell=int(per_cell), r_fwhm=r_fwhm, t_fwhm=t_fwhm,
             f_min=f_min, g_min=g_min, t_inj=t_fwhm * math.sqrt(math.log(1 / g_min) / math.log(2)))
    return d


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


def config3() -> dict:
    """Thick-target long run: 500 x 256 x 256 cells of 1 um gold (500 um thick
    along x), 1e8 electrons injected over 100 fs at 1e22 W/cm^2 (a0 = 85),
    reflux on all faces, 100 ps (200,000 steps)."""
    t = target(n=(500, 256, 256))
    return {"target": t, "laser": laser(t, I_Wcm2=1e22, n_macro=100_000_000),
            "run": run(seed=0, max_history=200_000), "steps": 200_000}


def config2() -> dict:
    """128^3 cells of 1 um gold, 1e7 electrons over 100 fs at 1e21 W/cm^2, 10 ps."""
    t = target(n=(128, 128, 128))
    return {"target": t, "laser": laser(t, I_Wcm2=1e21, n_macro=10_000_000),
            "run": run(seed=0, max_history=20_000), "steps": 20_000}


def macro_split(weights, total: int, lo: int, hi: int) -> list:
    """Integers proportional to `weights`, each clamped to [lo, hi], summing to
    `total` (the scale is re-solved after clamping, so the unclamped shares
    stay proportional)."""
    w = [float(x) for x in weights]
    if not (lo * len(w) <= total <= hi * len(w)):
        raise ValueError("total outside [lo, hi] x count")

    def filled(s):
        return sum(min(max(s * x, lo), hi) for x in w)

    a, b = 0.0, 1.0
    while filled(b) < total:
        b *= 2.0
    for _ in range(200):
        m = 0.5 * (a + b)
        a, b = (m, b) if filled(m) < total else (a, m)
    n = [int(round(min(max(b * x, lo), hi))) for x in w]
    free = [i for i in range(len(w)) if lo < n[i] < hi] or list(range(len(w)))
    n[max(free, key=lambda i: n[i])] += total - sum(n)
    return n


def config4(n_targets=64, seed=1, total_macro=60_000_000, lo=100_000, hi=4_000_000,
            steps=2000, cross=64, thickness=(5, 200)) -> dict:
    """Batched scan: n_targets independent targets drawn from a Philox stream:
    thickness uniform in [5, 200] cells of 1 um along x on a cross x cross
    section, element uniform over Al, Cu, Au at solid density, log10 I
    uniform in [20, 22] (W/cm^2), macro-electrons proportional to the laser
    energy (I at fixed spot and duration) scaled to total_macro and clamped to
    [lo, hi]; 5 um flat-top spot, 100 fs injection, 1 ps window."""
    import numpy as np

    g = np.random.Generator(np.random.Philox(seed))
    L = g.integers(thickness[0], thickness[1] + 1, size=n_targets)
    mats = g.choice(["Al", "Cu", "Au"], size=n_targets)
    I = 10.0 ** g.uniform(20.0, 22.0, size=n_targets)
    n_macro = macro_split(I, total_macro, lo, hi)
    targets = [target(n=(int(L[i]), cross, cross), material=str(mats[i])) for i in range(n_targets)]
    lasers = [laser(targets[i], I_Wcm2=float(I[i]), n_macro=n_macro[i]) for i in range(n_targets)]
    return {"targets": targets, "lasers": lasers, "run": run(seed=0, max_history=steps),
            "steps": steps, "I_Wcm2": [float(x) for x in I], "materials": [str(m) for m in mats]}


def model_point(Z=79.0, I_Wcm2=1e21, L=(100e-6, 100e-6, 100e-6), n_i=6e28, mechanisms=15) -> dict:
    """One point of the paper's loss-channel estimate (Sec. III.B): its
    constants (theta_c = 20 deg, <eta> = 1e-6 Ohm m, 1 MeV threshold,
    n_i = 6e28 m^-3, I_ex = 11 eV Z) and the injection of Sec. II.B (5 um and
    40 fs fwhm, <fg> = 0.41, <sqrt(fg)> = 0.61, eta_l2e = 0.3, 1 um light)."""
    return {"Z": float(Z), "n_i": float(n_i), "I_ex": 11.0 * EV * Z,
            "Lx": L[0], "Ly": L[1], "Lz": L[2], "I0": I_Wcm2 * 1e4, "lambda": 1e-6,
            "eta_l2e": 0.3, "r_fwhm": 5e-6, "t_fwhm": 40e-15, "mean_fg": 0.41,
            "mean_sqrt_fg": 0.61, "kappa_esc": 2.0, "kappa_tnsa": 2.7e-3,
            "theta_c": math.radians(20.0), "eta_avg": 1e-6, "eps_th": 1.0 * MEV,
            "E_stop": 1e3 * EV, "rel_step": 0.01, "mechanisms": int(mechanisms)}


def model_heatmap(n_I=128, n_Z=92, L=(100e-6, 100e-6, 100e-6)) -> list:
    """The heatmap grid of the estimate: log-uniform intensity over
    1e20-1e22 W/cm^2 x Z = 1..n_Z at n_i = 6e28 m^-3, I_ex = 11 eV Z."""
    pts = []
    for iz in range(n_Z):
        for ii in range(n_I):
            I = 10.0 ** (20.0 + 2.0 * ii / max(n_I - 1, 1))
            pts.append(model_point(Z=1.0 + iz, I_Wcm2=I, L=L))
    return pts
