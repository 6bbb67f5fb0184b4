"""ctypes binding of the FP64 CPU oracle (oracle.h, physics.c, sim.c, model.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg load this module; the CUDA library never does.
`build()` compiles the oracle with gcc into oracle/_build/liboracle.so;
`build(threads=True)` compiles the same sources with OpenMP into
liboracle_omp.so, used only to time the oracle on all host cores (the
serial library is the one the tests check against).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
LIB_OMP_PATH = os.path.join(BUILD_DIR, "liboracle_omp.so")
SOURCES = ["physics.c", "sim.c", "model.c"]

ORC_DRAG, ORC_SCATTER, ORC_BREM, ORC_FIELDS, ORC_FARADAY, ORC_HEATING = 1, 2, 4, 8, 16, 32
ORC_ALL = 63
ORC_UNBOUNDED = 64
ORC_FSIGMA, ORC_EI = 128, 256
GRID = {"T": 0, "eta": 1, "Ex": 2, "Ey": 3, "Ez": 4, "Bx": 5, "By": 6, "Bz": 7,
        "jx": 8, "jy": 9, "jz": 10, "heat": 11, "Ti": 12}


def build(force: bool = False, threads: bool = False) -> str:
    """Compile the oracle (plain C11, no FMA contraction so x86 and Arm agree);
    threads: the OpenMP build for all-core timing."""
    path = LIB_OMP_PATH if threads else LIB_PATH
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    newest = max(os.path.getmtime(p) for p in srcs + [os.path.join(HERE, "oracle.h")])
    if not force and os.path.exists(path) and os.path.getmtime(path) >= newest:
        return path
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           *(["-fopenmp"] if threads else []), "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


class Solid(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("Z", "n_i", "I_ex", "Zstar", "A_ion")]


class Target(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("Z", C.c_double), ("n_i", C.c_double),
                ("I_ex", C.c_double), ("Zstar", C.c_double), ("lnLambda", C.c_double),
                ("eta_max", C.c_double), ("lambda1", C.c_double), ("lambda2", C.c_double),
                ("T0", C.c_double), ("A_ion", C.c_double), ("n_extra", C.c_int32),
                ("pad", C.c_int32), ("extra", Solid * 3)]


class ModelIn(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "Z", "n_i", "I_ex", "Lx", "Ly", "Lz", "I0", "lam", "eta_l2e", "r_fwhm", "t_fwhm",
        "mean_fg", "mean_sqrt_fg", "kappa_esc", "kappa_tnsa", "theta_c", "eta_avg", "eps_th",
        "E_stop", "rel_step")] + [("mechanisms", C.c_int32), ("pad", C.c_int32)]


class ModelOut(C.Structure):
    _fields_ = [("E", C.c_double * 8), ("N_e", C.c_double), ("a0", C.c_double),
                ("N_band", C.c_double * 3), ("eps_band", C.c_double * 3), ("x_end", C.c_double * 3)]


MODEL_E = ("E_injected", "E_brem", "E_ion", "E_tnsa", "E_field", "E_xray_above", "E_escaped")
ORC_MODEL_BREM, ORC_MODEL_ION, ORC_MODEL_TNSA, ORC_MODEL_FIELD, ORC_MODEL_ALL = 1, 2, 4, 8, 15


class Laser(C.Structure):
    _fields_ = [("I0", C.c_double), ("lam", C.c_double), ("eta_l2e", C.c_double),
                ("spot_r", C.c_double), ("spot_y", C.c_double), ("spot_z", C.c_double),
                ("t_inj", C.c_double), ("cone_half", C.c_double), ("n_macro", C.c_int64),
                ("envelope", C.c_int32), ("per_cell", C.c_int32), ("r_fwhm", C.c_double),
                ("t_fwhm", C.c_double), ("f_min", C.c_double), ("g_min", C.c_double),
                ("moore_cap", C.c_int32), ("pad", C.c_int32)]


class Run(C.Structure):
    _fields_ = [("dt", C.c_double), ("seed", C.c_uint64), ("target_index", C.c_uint32),
                ("kappa_esc", C.c_double), ("kappa_tnsa", C.c_double),
                ("sigma_dtheta", C.c_double), ("brem_boost", C.c_double),
                ("k_min", C.c_double), ("E_cut", C.c_double),
                ("n_E", C.c_int32), ("n_theta", C.c_int32),
                ("tally_E_min", C.c_double), ("tally_E_max", C.c_double),
                ("ce_threshold", C.c_double), ("table_rows", C.c_int32),
                ("table_cols", C.c_int32), ("table_E_max", C.c_double),
                ("curlB_term", C.c_int32), ("physics", C.c_int32),
                ("max_history", C.c_int32)]


class Tallies(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "E_injected", "N_injected", "W_field", "E_drag", "E_xray", "E_xray_above",
        "E_escaped", "E_reflux", "E_ohmic_grid", "n_injected", "n_escaped",
        "n_refluxed", "n_reflux_absorbed", "n_cut", "n_emitted", "particle_steps")]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


_libs = {}


def lib(threads: bool = False):
    if threads not in _libs:
        L = C.CDLL(build(threads=threads))
        _libs[threads] = L
        dp = C.POINTER(C.c_double)
        up = C.POINTER(C.c_uint32)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(Target), C.POINTER(Laser), C.POINTER(Run)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.c_int64]
        L.orc_fields.argtypes = [C.c_void_p]
        L.orc_seed.argtypes = [C.c_void_p, C.c_int64, C.c_double]
        L.orc_n_particles.restype = C.c_int64
        L.orc_n_particles.argtypes = [C.c_void_p]
        L.orc_get_particles.argtypes = [C.c_void_p] + [dp] * 7 + [up]
        L.orc_set_particles.argtypes = [C.c_void_p, C.c_int64] + [dp] * 7 + [up]
        L.orc_grid_len.restype = C.c_int64
        L.orc_grid_len.argtypes = [C.c_void_p, C.c_int]
        L.orc_get_grid.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_set_grid.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_get_tallies.argtypes = [C.c_void_p, C.POINTER(Tallies)]
        L.orc_reset_tallies.argtypes = [C.c_void_p]
        L.orc_get_hist.argtypes = [C.c_void_p, dp, dp]
        L.orc_get_history.argtypes = [C.c_void_p, dp]
        L.orc_get_clock.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.orc_set_clock.argtypes = [C.c_void_p, C.c_int64, C.c_int64]
        for f in ("orc_live_energy", "orc_field_energy", "orc_weight", "orc_a0_of"):
            getattr(L, f).restype = C.c_double
            getattr(L, f).argtypes = [C.c_void_p]
        L.orc_philox4x32_10.argtypes = [up, up, up]
        L.orc_uniform.restype = C.c_double
        L.orc_uniform.argtypes = [C.c_uint32]
        L.orc_a0.restype = C.c_double
        L.orc_a0.argtypes = [C.c_double, C.c_double]
        tp = C.POINTER(Target)
        for f in ("orc_stop_ion", "orc_stop_brem"):
            getattr(L, f).restype = C.c_double
            getattr(L, f).argtypes = [tp, C.c_double]
        L.orc_dsigma_dk.restype = C.c_double
        L.orc_dsigma_dk.argtypes = [tp, C.c_double, C.c_double]
        L.orc_sigma_tot.restype = C.c_double
        L.orc_sigma_tot.argtypes = [tp, C.c_double, C.c_double]
        L.orc_brem_table.argtypes = [tp, C.c_double, C.c_double, C.c_int, C.c_int, dp]
        L.orc_brem_sample.restype = C.c_double
        L.orc_brem_sample.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.c_double,
                                      C.c_double, C.c_double]
        L.orc_davies_sigma.restype = C.c_double
        L.orc_davies_sigma.argtypes = [tp, C.c_double, C.c_double]
        L.orc_photon_theta.restype = C.c_double
        L.orc_photon_theta.argtypes = [C.c_double, C.c_double]
        L.orc_heat_capacity.restype = C.c_double
        L.orc_heat_capacity.argtypes = [C.c_double, C.c_double]
        L.orc_temperature_rise.restype = C.c_double
        L.orc_temperature_rise.argtypes = [tp, C.c_double, C.c_double]
        L.orc_resistivity.restype = C.c_double
        L.orc_resistivity.argtypes = [tp, C.c_double]
        L.orc_f_sigma.restype = C.c_double
        L.orc_f_sigma.argtypes = [tp, C.c_double]
        L.orc_ei_rates.argtypes = [tp, C.c_double, C.c_double, C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)]
        L.orc_rotate.argtypes = [dp, C.c_double, C.c_double, dp]
        L.orc_tally_bin.argtypes = [C.POINTER(Run), C.c_double, C.c_double,
                                    C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_model.argtypes = [C.POINTER(ModelIn), C.POINTER(ModelOut)]
        L.orc_get_weights.argtypes = [C.c_void_p, dp]
        L.orc_set_weights.argtypes = [C.c_void_p, C.c_int64, dp]
        L.orc_boris.argtypes = [dp, dp, dp, C.c_double]
    return _libs[threads]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _up(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def make_target(d: dict) -> Target:
    d = dict(d)
    extra = d.pop("extra", [])
    t = Target(**d)
    t.n_extra = len(extra)
    for i, e in enumerate(extra):
        t.extra[i] = Solid(e["Z"], e["n_i"], e["I_ex"], e["Zstar"], e["A_ion"])
    return t


def make_laser(d: dict) -> Laser:
    d = dict(d)
    d["lam"] = d.pop("lambda")
    return Laser(**d)


def weights(sim) -> np.ndarray:
    """Per-electron weights of an OracleSim, in the order of particles()."""
    n = sim.n
    w = np.empty(n)
    if n:
        sim._L.orc_get_weights(sim.h, _dp(w))
    return w


def set_weights(sim, w) -> None:
    w = np.ascontiguousarray(w, dtype=np.float64)
    sim._L.orc_set_weights(sim.h, len(w), _dp(w))


def make_run(d: dict) -> Run:
    return Run(**d)


class OracleSim:
    """One target advanced by the FP64 CPU oracle."""

    def __init__(self, target: dict, laser: dict, run: dict, threads: bool = False):
        """threads: step with the OpenMP build on all host cores (timing only)."""
        self.target, self.laser, self.run = dict(target), dict(laser), dict(run)
        self._L = lib(threads)
        self._t = make_target(target)
        self._l = make_laser(laser)
        self._r = make_run(run)
        self.h = self._L.orc_create(C.byref(self._t), C.byref(self._l), C.byref(self._r))
        if not self.h:
            raise ValueError("oracle rejected the configuration")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._L.orc_destroy(h)
            self.h = None

    def step(self, n: int = 1) -> None:
        self._L.orc_step(self.h, int(n))

    def fields(self) -> None:
        self._L.orc_fields(self.h)

    def seed(self, n: int, mean_eps: float) -> None:
        self._L.orc_seed(self.h, int(n), float(mean_eps))

    @property
    def n(self) -> int:
        return int(self._L.orc_n_particles(self.h))

    def particles(self) -> dict:
        n = self.n
        out = {k: np.empty(n) for k in ("x", "y", "z", "ux", "uy", "uz", "tau")}
        out["id"] = np.empty(n, dtype=np.uint32)
        self._L.orc_get_particles(self.h, *[_dp(out[k]) for k in ("x", "y", "z", "ux", "uy", "uz", "tau")],
                                _up(out["id"]))
        return out

    def set_particles(self, p: dict) -> None:
        n = len(p["id"])
        arrs = [np.ascontiguousarray(p[k], dtype=np.float64) for k in ("x", "y", "z", "ux", "uy", "uz", "tau")]
        ids = np.ascontiguousarray(p["id"], dtype=np.uint32)
        self._L.orc_set_particles(self.h, n, *[_dp(a) for a in arrs], _up(ids))

    def grid(self, which: str) -> np.ndarray:
        w = GRID[which]
        out = np.empty(self._L.orc_grid_len(self.h, w))
        self._L.orc_get_grid(self.h, w, _dp(out))
        return out

    def set_grid(self, which: str, values: np.ndarray) -> None:
        w = GRID[which]
        a = np.ascontiguousarray(values, dtype=np.float64)
        assert a.size == self._L.orc_grid_len(self.h, w)
        self._L.orc_set_grid(self.h, w, _dp(a))

    def tallies(self) -> dict:
        t = Tallies()
        self._L.orc_get_tallies(self.h, C.byref(t))
        d = t.as_dict()
        d["E_live"] = self._L.orc_live_energy(self.h)
        d["E_B_field"] = self._L.orc_field_energy(self.h)
        return d

    def reset_tallies(self) -> None:
        self._L.orc_reset_tallies(self.h)

    def hist(self):
        rows = self.run["n_E"] + 2
        hE = np.empty(rows * self.run["n_theta"])
        hN = np.empty_like(hE)
        self._L.orc_get_hist(self.h, _dp(hE), _dp(hN))
        return hE.reshape(rows, -1), hN.reshape(rows, -1)

    def history(self) -> np.ndarray:
        out = np.empty(max(self.run["max_history"], 0))
        self._L.orc_get_history(self.h, _dp(out))
        return out

    def clock(self):
        a, b = C.c_int64(), C.c_int64()
        self._L.orc_get_clock(self.h, C.byref(a), C.byref(b))
        return a.value, b.value

    def set_clock(self, step: int, n_ids: int) -> None:
        self._L.orc_set_clock(self.h, int(step), int(n_ids))

    @property
    def weight(self) -> float:
        return self._L.orc_weight(self.h)

    @property
    def a0(self) -> float:
        return self._L.orc_a0_of(self.h)


# ---- single formulas ----
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_up(c), _up(k), _up(out))
    return out


def uniform(x: int) -> float:
    return lib().orc_uniform(int(x) & 0xFFFFFFFF)


def a0(I0_Wm2: float, lam: float) -> float:
    return lib().orc_a0(I0_Wm2, lam)


def stop_ion(target: dict, eps: float) -> float:
    return lib().orc_stop_ion(C.byref(make_target(target)), eps)


def stop_brem(target: dict, eps: float) -> float:
    return lib().orc_stop_brem(C.byref(make_target(target)), eps)


def dsigma_dk(target: dict, eps: float, k: float) -> float:
    return lib().orc_dsigma_dk(C.byref(make_target(target)), eps, k)


def sigma_tot(target: dict, k_min: float, eps: float) -> float:
    return lib().orc_sigma_tot(C.byref(make_target(target)), k_min, eps)


def brem_table(target: dict, k_min: float, E_max: float, rows: int, cols: int) -> np.ndarray:
    v = np.empty(rows * cols)
    lib().orc_brem_table(C.byref(make_target(target)), k_min, E_max, rows, cols, _dp(v))
    return v.reshape(rows, cols)


def brem_sample(table: np.ndarray, k_min: float, E_max: float, eps: float, r: float) -> float:
    t = np.ascontiguousarray(table, dtype=np.float64)
    return lib().orc_brem_sample(_dp(t), t.shape[0], t.shape[1], k_min, E_max, eps, r)


def davies_sigma(target: dict, p_SI: float, dt: float) -> float:
    return lib().orc_davies_sigma(C.byref(make_target(target)), p_SI, dt)


def photon_theta(gamma: float, u: float) -> float:
    return lib().orc_photon_theta(gamma, u)


def heat_capacity(T_K: float, Z: float) -> float:
    return lib().orc_heat_capacity(T_K, Z)


def temperature_rise(target: dict, T_K: float, rho: float) -> float:
    return lib().orc_temperature_rise(C.byref(make_target(target)), T_K, rho)


def resistivity(target: dict, T_K: float) -> float:
    return lib().orc_resistivity(C.byref(make_target(target)), T_K)


def f_sigma(target: dict, Ti_K: float) -> float:
    return lib().orc_f_sigma(C.byref(make_target(target)), Ti_K)


def ei_rates(target: dict, Te_K: float, Ti_K: float):
    a, b = C.c_double(), C.c_double()
    lib().orc_ei_rates(C.byref(make_target(target)), Te_K, Ti_K, C.byref(a), C.byref(b))
    return a.value, b.value


def rotate(d, theta: float, phi: float) -> np.ndarray:
    dd = np.ascontiguousarray(d, dtype=np.float64)
    out = np.empty(3)
    lib().orc_rotate(_dp(dd), theta, phi, _dp(out))
    return out


def tally_bin(run: dict, k: float, theta: float):
    """(row, column) of a photon of energy k (J) at polar angle theta (rad,
    from +x) in the photon tallies of the run."""
    r, c = C.c_int(), C.c_int()
    lib().orc_tally_bin(C.byref(make_run(run)), k, theta, C.byref(r), C.byref(c))
    return r.value, c.value


def boris(u, E, B, dt: float) -> np.ndarray:
    uu = np.array(u, dtype=np.float64)
    EE = np.ascontiguousarray(E, dtype=np.float64)
    BB = np.ascontiguousarray(B, dtype=np.float64)
    lib().orc_boris(_dp(uu), _dp(EE), _dp(BB), dt)
    return uu


def model(m: dict) -> dict:
    """The three-macro-electron estimate (Sec. III.B) for one parameter set
    (keys as ModelIn, wavelength as "lambda")."""
    d = dict(m)
    d["lam"] = d.pop("lambda")
    out = ModelOut()
    lib().orc_model(C.byref(ModelIn(**d)), C.byref(out))
    r = {k: out.E[i] for i, k in enumerate(MODEL_E)}
    r.update(N_e=out.N_e, a0=out.a0, N_band=list(out.N_band), eps_band=list(out.eps_band),
             x_end=list(out.x_end))
    return r
