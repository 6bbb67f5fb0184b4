"""ctypes binding of the C-ABI in include/hpic.h (argument marshalling only).

Every step of the method runs in the CUDA library; this module converts
Python dicts and numpy arrays to the ABI's structs and pointers.  The
library is paper_2107_01723_gb300/_build/libhpic.so; if it is missing the
first call raises (build it with `python -m paper_2107_01723_gb300.build`).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libhpic.so")

HPIC_OK, HPIC_EINVAL, HPIC_ENOMEM, HPIC_ECUDA, HPIC_ETIMEOUT, HPIC_ESTATE, HPIC_ENONFINITE = \
    0, -1, -2, -3, -4, -5, -6
HPIC_FP64, HPIC_FP32_MIXED = 0, 1
HPIC_DRAG, HPIC_SCATTER, HPIC_BREM, HPIC_FIELDS, HPIC_FARADAY, HPIC_HEATING = 1, 2, 4, 8, 16, 32
HPIC_ALL = 63
HPIC_UNBOUNDED = 64
HPIC_FSIGMA, HPIC_EI_EQUIL = 128, 256
HPIC_ENV_FLAT, HPIC_ENV_GAUSS = 0, 1
HPIC_BATCH_MAX_TARGETS = 256
GRID = {"T": 0, "eta": 1, "Ex": 2, "Ey": 3, "Ez": 4, "Bx": 5, "By": 6, "Bz": 7,
        "jx": 8, "jy": 9, "jz": 10, "heat": 11, "Ti": 12}


class HpicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hpic error {code}: {msg}")
        self.code = code


class hpic_solid(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("Z", "n_i_m3", "I_ex_J", "Zstar", "A_ion")]


class hpic_target_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dx_m", C.c_double),
                ("Z", C.c_double), ("n_i_m3", C.c_double), ("I_ex_J", C.c_double),
                ("Zstar", C.c_double), ("lnLambda", C.c_double), ("eta_max_ohm_m", C.c_double),
                ("lambda1", C.c_double), ("lambda2", C.c_double), ("T0_K", C.c_double),
                ("A_ion", C.c_double), ("n_extra", C.c_int32), ("pad", C.c_int32),
                ("extra", hpic_solid * 3)]


class hpic_laser_desc(C.Structure):
    _fields_ = [("I0_Wm2", C.c_double), ("lambda_m", C.c_double), ("eta_l2e", C.c_double),
                ("spot_radius_m", C.c_double), ("spot_y_m", C.c_double), ("spot_z_m", C.c_double),
                ("t_inj_s", C.c_double), ("cone_half_angle_rad", C.c_double),
                ("n_macro", C.c_int64), ("envelope", C.c_int32), ("per_cell", C.c_int32),
                ("r_fwhm_m", C.c_double), ("t_fwhm_s", C.c_double), ("f_min", C.c_double),
                ("g_min", C.c_double), ("moore_cap", C.c_int32), ("pad", C.c_int32)]


class hpic_run_params(C.Structure):
    _fields_ = [("dt_s", C.c_double), ("seed", C.c_uint64), ("target_index", C.c_uint32),
                ("precision", C.c_int32), ("kappa_esc", C.c_double), ("kappa_tnsa", C.c_double),
                ("sigma_dtheta_rad", C.c_double), ("brem_boost", C.c_double),
                ("k_min_J", C.c_double), ("E_cut_J", C.c_double), ("n_Ebins", C.c_int32),
                ("n_thbins", C.c_int32), ("tally_Emin_J", C.c_double), ("tally_Emax_J", C.c_double),
                ("ce_threshold_J", C.c_double), ("table_rows", C.c_int32),
                ("table_cols", C.c_int32), ("table_Emax_J", C.c_double),
                ("curlB_term", C.c_int32), ("physics", C.c_int32), ("sort_interval", C.c_int32),
                ("max_history", C.c_int32)]


_TALLY_NAMES = ("E_injected", "N_injected", "W_field", "E_drag", "E_xray", "E_xray_above",
                "E_escaped", "E_reflux", "E_ohmic_grid", "n_injected", "n_escaped", "n_refluxed",
                "n_reflux_absorbed", "n_cut", "n_emitted", "particle_steps", "n_nonfinite",
                "E_live", "E_B_field")


class hpic_batch_tuning(C.Structure):
    _fields_ = [("blocks_per_sm", C.c_int32), ("sort_interval", C.c_int32),
                ("use_graph", C.c_int32), ("reserved", C.c_int32), ("ms_per_step", C.c_double)]


class hpic_model_in(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "Z", "n_i_m3", "I_ex_J", "Lx_m", "Ly_m", "Lz_m", "I0_Wm2", "lambda_m", "eta_l2e",
        "r_fwhm_m", "t_fwhm_s", "mean_fg", "mean_sqrt_fg", "kappa_esc", "kappa_tnsa",
        "theta_c_rad", "eta_avg_ohm_m", "eps_th_J", "E_stop_J", "rel_step")] + [
        ("mechanisms", C.c_int32), ("pad", C.c_int32)]


class hpic_model_out(C.Structure):
    _fields_ = [("E", C.c_double * 8), ("N_e", C.c_double), ("a0", C.c_double),
                ("N_band", C.c_double * 3), ("eps_band", C.c_double * 3),
                ("x_end", C.c_double * 3), ("steps", C.c_int64)]


MODEL_E = ("E_injected", "E_brem", "E_ion", "E_tnsa", "E_field", "E_xray_above", "E_escaped")
HPIC_MODEL_BREM, HPIC_MODEL_ION, HPIC_MODEL_TNSA, HPIC_MODEL_FIELD, HPIC_MODEL_ALL = 1, 2, 4, 8, 15


class hpic_tallies(C.Structure):
    _fields_ = [(n, C.c_double) for n in _TALLY_NAMES]


_lib = None
_DP = C.POINTER(C.c_double)
_UP = C.POINTER(C.c_uint32)
_I64P = C.POINTER(C.c_int64)


def lib() -> C.CDLL:
    """Load libhpic.so; raise if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FileNotFoundError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2107_01723_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        sig = {
            "hpic_init_target": [C.POINTER(vp), C.POINTER(hpic_target_desc),
                                 C.POINTER(hpic_run_params), C.c_int, vp],
            "hpic_inject_electrons": [vp, C.POINTER(hpic_laser_desc)],
            "hpic_step": [vp, C.c_int64],
            "hpic_seed_electrons": [vp, C.c_int64, C.c_double],
            "hpic_sort": [vp],
            "hpic_read_tallies": [vp, C.POINTER(hpic_tallies)],
            "hpic_reset_tallies": [vp],
            "hpic_read_hist": [vp, _DP, _DP],
            "hpic_read_history": [vp, _DP],
            "hpic_grid_len": [vp, C.c_int, _I64P],
            "hpic_read_grid": [vp, C.c_int, _DP],
            "hpic_write_grid": [vp, C.c_int, _DP],
            "hpic_count_particles": [vp, _I64P],
            "hpic_read_particles": [vp] + [_DP] * 7 + [_UP, C.c_int64, _I64P],
            "hpic_load_particles": [vp, C.c_int64] + [_DP] * 7 + [_UP],
            "hpic_read_weights": [vp, _DP, C.c_int64, _I64P],
            "hpic_save": [vp, C.c_char_p],
            "hpic_load": [C.POINTER(vp), C.c_char_p, C.c_int, vp],
            "hpic_load_weights": [vp, C.c_int64, _DP],
            "hpic_get_clock": [vp, _I64P, _I64P],
            "hpic_set_clock": [vp, C.c_int64, C.c_int64],
            "hpic_profile": [vp, C.c_int],
            "hpic_kernel_time": [vp, _DP, _I64P, _DP],
            "hpic_launch_count": [vp, _I64P],
            "hpic_destroy": [vp],
            "hpic_batch_init": [C.POINTER(vp), C.c_int32, C.POINTER(hpic_target_desc),
                                C.POINTER(hpic_laser_desc), C.POINTER(hpic_run_params),
                                C.POINTER(C.c_uint32), C.c_int64, C.c_int, vp],
            "hpic_batch_target": [vp, C.c_int32, C.POINTER(vp)],
            "hpic_batch_step": [vp, C.c_int64],
            "hpic_batch_get_tuning": [vp, C.POINTER(hpic_batch_tuning)],
            "hpic_batch_set_tuning": [vp, C.POINTER(hpic_batch_tuning)],
            "hpic_batch_autotune": [vp, C.c_int32, C.POINTER(hpic_batch_tuning)],
            "hpic_batch_profile": [vp, C.c_int],
            "hpic_batch_kernel_time": [vp, _DP, _I64P, _DP],
            "hpic_batch_launch_count": [vp, _I64P],
            "hpic_batch_destroy": [vp],
        }
        sig["hpic_sort_cells_noalloc"] = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64,
                                          C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                          C.c_void_p, C.c_int, C.c_void_p]
        sig["hpic_model"] = [C.c_int64, C.POINTER(hpic_model_in), C.POINTER(hpic_model_out),
                             C.c_int, vp]
        sig["hpic_model_device"] = [C.c_int64, vp, vp, C.c_int, vp]
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.hpic_last_error.argtypes = [vp]
        L.hpic_last_error.restype = C.c_char_p
        L.hpic_batch_last_error.argtypes = [vp]
        L.hpic_batch_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(code: int, h=None) -> int:
    if code != HPIC_OK:
        msg = lib().hpic_last_error(h)
        raise HpicError(code, msg.decode() if msg else "")
    return code


def _bcheck(code: int, b=None) -> int:
    if code != HPIC_OK:
        msg = lib().hpic_batch_last_error(b)
        raise HpicError(code, msg.decode() if msg else "")
    return code


def _dp(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def _up(a):
    return a.ctypes.data_as(_UP) if a is not None else None


# ---- structs from the workload dicts (SI units) ----
def target_desc(t: dict) -> hpic_target_desc:
    d = hpic_target_desc(t["nx"], t["ny"], t["nz"], t["dx"], t["Z"], t["n_i"], t["I_ex"],
                         t["Zstar"], t["lnLambda"], t["eta_max"], t["lambda1"], t["lambda2"],
                         t["T0"], t["A_ion"])
    extra = t.get("extra", [])
    d.n_extra = len(extra)
    for i, e in enumerate(extra):
        d.extra[i] = hpic_solid(e["Z"], e["n_i"], e["I_ex"], e["Zstar"], e["A_ion"])
    return d


def laser_desc(l: dict) -> hpic_laser_desc:
    return hpic_laser_desc(l["I0"], l["lambda"], l["eta_l2e"], l["spot_r"], l["spot_y"],
                           l["spot_z"], l["t_inj"], l["cone_half"], int(l["n_macro"]),
                           int(l.get("envelope", 0)), int(l.get("per_cell", 0)),
                           l.get("r_fwhm", 0.0), l.get("t_fwhm", 0.0), l.get("f_min", 0.0),
                           l.get("g_min", 0.0), int(l.get("moore_cap", 0)), 0)


def run_params(r: dict, precision: int = HPIC_FP64, sort_interval: int = 0) -> hpic_run_params:
    return hpic_run_params(r["dt"], int(r["seed"]), int(r.get("target_index", 0)), precision,
                           r["kappa_esc"], r["kappa_tnsa"], r["sigma_dtheta"], r["brem_boost"],
                           r["k_min"], r["E_cut"], r["n_E"], r["n_theta"], r["tally_E_min"],
                           r["tally_E_max"], r["ce_threshold"], r["table_rows"], r["table_cols"],
                           r["table_E_max"], r["curlB_term"], r["physics"], sort_interval,
                           r["max_history"])


# ---- the ABI's calls, same names ----
def hpic_init_target(target: dict, run: dict, precision: int = HPIC_FP64, device: int = 0,
                     stream: int = 0, sort_interval: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    t, r = target_desc(target), run_params(run, precision, sort_interval)
    _check(lib().hpic_init_target(C.byref(h), C.byref(t), C.byref(r), device,
                                  C.c_void_p(stream) if stream else None))
    return h


def hpic_inject_electrons(h, laser: dict) -> None:
    l = laser_desc(laser)
    _check(lib().hpic_inject_electrons(h, C.byref(l)), h)


def hpic_seed_electrons(h, n: int, mean_energy_J: float) -> None:
    _check(lib().hpic_seed_electrons(h, int(n), float(mean_energy_J)), h)


def hpic_step(h, n: int = 1) -> None:
    _check(lib().hpic_step(h, int(n)), h)


def hpic_sort(h) -> None:
    _check(lib().hpic_sort(h), h)


def hpic_read_tallies(h, allow_nonfinite: bool = False) -> dict:
    t = hpic_tallies()
    code = lib().hpic_read_tallies(h, C.byref(t))
    if not (allow_nonfinite and code == HPIC_ENONFINITE):
        _check(code, h)
    return {n: getattr(t, n) for n in _TALLY_NAMES}


def hpic_reset_tallies(h) -> None:
    _check(lib().hpic_reset_tallies(h), h)


def hpic_read_hist(h, n_E: int, n_th: int):
    hE = np.empty((n_E + 2) * n_th)
    hN = np.empty_like(hE)
    _check(lib().hpic_read_hist(h, _dp(hE), _dp(hN)), h)
    return hE.reshape(n_E + 2, n_th), hN.reshape(n_E + 2, n_th)


def hpic_read_history(h, length: int) -> np.ndarray:
    out = np.empty(max(length, 1))
    _check(lib().hpic_read_history(h, _dp(out)), h)
    return out[:length]


def hpic_read_grid(h, which: str) -> np.ndarray:
    n = C.c_int64()
    _check(lib().hpic_grid_len(h, GRID[which], C.byref(n)), h)
    out = np.empty(n.value)
    _check(lib().hpic_read_grid(h, GRID[which], _dp(out)), h)
    return out


def hpic_write_grid(h, which: str, values) -> None:
    a = np.ascontiguousarray(values, dtype=np.float64)
    n = C.c_int64()
    _check(lib().hpic_grid_len(h, GRID[which], C.byref(n)), h)
    if a.size != n.value:
        raise ValueError(f"grid {which} needs {n.value} values, got {a.size}")
    _check(lib().hpic_write_grid(h, GRID[which], _dp(a)), h)


def hpic_count_particles(h) -> int:
    n = C.c_int64()
    _check(lib().hpic_count_particles(h, C.byref(n)), h)
    return n.value


def hpic_read_particles(h, out: dict | None = None) -> dict:
    """The live electrons in storage order.  With `out` (float64 arrays x ..
    tau and a uint32 array id, C-contiguous, all of one length: the capacity,
    e.g. page-locked buffers allocated once) they are written there and views
    of the first n entries are returned; otherwise new arrays are made."""
    keys = ("x", "y", "z", "ux", "uy", "uz", "tau")
    if out is None:
        n = hpic_count_particles(h)
        out = {k: np.empty(n) for k in keys}
        out["id"] = np.empty(n, dtype=np.uint32)
    else:
        n = len(out["id"])
        for k in keys:
            if out[k].dtype != np.float64 or not out[k].flags.c_contiguous or len(out[k]) != n:
                raise ValueError(f"out[{k!r}] must be a C-contiguous float64 array of length {n}")
        if out["id"].dtype != np.uint32 or not out["id"].flags.c_contiguous:
            raise ValueError("out['id'] must be a C-contiguous uint32 array")
    got = C.c_int64()
    _check(lib().hpic_read_particles(h, *[_dp(out[k]) for k in keys], _up(out["id"]), n,
                                     C.byref(got)), h)
    m = got.value
    return {k: v[:m] for k, v in out.items()}


def hpic_load_particles(h, p: dict) -> None:
    arrs = [np.ascontiguousarray(p[k], dtype=np.float64) for k in ("x", "y", "z", "ux", "uy", "uz", "tau")]
    ids = np.ascontiguousarray(p["id"], dtype=np.uint32)
    _check(lib().hpic_load_particles(h, len(ids), *[_dp(a) for a in arrs], _up(ids)), h)


def hpic_read_weights(h) -> np.ndarray:
    n = C.c_int64()
    cnt = hpic_count_particles(h)
    out = np.empty(max(cnt, 1))
    _check(lib().hpic_read_weights(h, _dp(out), cnt, C.byref(n)), h)
    return out[:n.value]


def hpic_load_weights(h, w) -> None:
    a = np.ascontiguousarray(w, dtype=np.float64)
    _check(lib().hpic_load_weights(h, len(a), _dp(a)), h)


def hpic_save(h, path: str) -> None:
    _check(lib().hpic_save(h, os.fsencode(path)), h)


def hpic_load(path: str, device: int = 0, stream: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().hpic_load(C.byref(h), os.fsencode(path), device,
                           C.c_void_p(stream) if stream else None))
    return h


def hpic_get_clock(h):
    a, b = C.c_int64(), C.c_int64()
    _check(lib().hpic_get_clock(h, C.byref(a), C.byref(b)), h)
    return a.value, b.value


def hpic_set_clock(h, step: int, next_id: int) -> None:
    _check(lib().hpic_set_clock(h, int(step), int(next_id)), h)


def hpic_profile(h, enable: bool) -> None:
    _check(lib().hpic_profile(h, 1 if enable else 0), h)


def hpic_kernel_time(h):
    ms, n, ps = C.c_double(), C.c_int64(), C.c_double()
    _check(lib().hpic_kernel_time(h, C.byref(ms), C.byref(n), C.byref(ps)), h)
    return ms.value, n.value, ps.value


def hpic_launch_count(h) -> int:
    n = C.c_int64()
    _check(lib().hpic_launch_count(h, C.byref(n)), h)
    return n.value


def hpic_sort_cells_noalloc(nx: int, ny: int, nz: int, precision: int, n: int, in_ptrs,
                            out_ptrs, n_live_dev_ptr: int, device: int = 0,
                            stream: int = 0) -> None:
    """Cell sort without any allocation, for callers that cannot allocate
    (see include/hpic.h).  in_ptrs/out_ptrs: 8 device addresses each
    (x, y, z in cells, ux, uy, uz, tau, id); n_live_dev_ptr: a device int64."""
    ins = (C.c_void_p * 8)(*[int(p) for p in in_ptrs])
    outs = (C.c_void_p * 8)(*[int(p) for p in out_ptrs])
    _check(lib().hpic_sort_cells_noalloc(nx, ny, nz, precision, int(n), ins, outs,
                                         C.c_void_p(int(n_live_dev_ptr)), device,
                                         C.c_void_p(stream) if stream else None))


def hpic_destroy(h) -> None:
    if h:
        _check(lib().hpic_destroy(h))


# ---- the three-macro-electron estimate (Sec. III.B) ----
def model_in(m: dict) -> hpic_model_in:
    return hpic_model_in(m["Z"], m["n_i"], m["I_ex"], m["Lx"], m["Ly"], m["Lz"], m["I0"],
                         m["lambda"], m["eta_l2e"], m["r_fwhm"], m["t_fwhm"], m["mean_fg"],
                         m["mean_sqrt_fg"], m["kappa_esc"], m["kappa_tnsa"], m["theta_c"],
                         m["eta_avg"], m["eps_th"], m["E_stop"], m["rel_step"],
                         int(m["mechanisms"]), 0)


def model_out_dict(o: hpic_model_out) -> dict:
    r = {k: o.E[i] for i, k in enumerate(MODEL_E)}
    r.update(N_e=o.N_e, a0=o.a0, N_band=list(o.N_band), eps_band=list(o.eps_band),
             x_end=list(o.x_end), steps=o.steps)
    return r


def hpic_model(points: list, device: int = 0, stream: int = 0) -> list:
    n = len(points)
    src = (hpic_model_in * max(n, 1))(*[model_in(m) for m in points])
    dst = (hpic_model_out * max(n, 1))()
    _check(lib().hpic_model(n, src, dst, device, C.c_void_p(stream) if stream else None))
    return [model_out_dict(dst[i]) for i in range(n)]


def hpic_model_device(n: int, in_ptr: int, out_ptr: int, device: int = 0, stream: int = 0) -> None:
    _check(lib().hpic_model_device(n, C.c_void_p(in_ptr), C.c_void_p(out_ptr), device,
                                   C.c_void_p(stream) if stream else None))


# ---- batches ----
def hpic_batch_init(targets: list, lasers: list | None, run: dict, precision: int = HPIC_FP64,
                    spare_slots: int = 0, device: int = 0, stream: int = 0,
                    sort_interval: int = 0, target_index=None) -> C.c_void_p:
    n = len(targets)
    T = (hpic_target_desc * n)(*[target_desc(t) for t in targets])
    Lz = (hpic_laser_desc * n)(*[laser_desc(l) for l in lasers]) if lasers is not None else None
    ti = (C.c_uint32 * n)(*[int(v) for v in target_index]) if target_index is not None else None
    r = run_params(run, precision, sort_interval)
    b = C.c_void_p()
    _bcheck(lib().hpic_batch_init(C.byref(b), n, T, Lz, C.byref(r), ti, spare_slots, device,
                                  C.c_void_p(stream) if stream else None))
    return b


def hpic_batch_target(b, t: int) -> C.c_void_p:
    h = C.c_void_p()
    _bcheck(lib().hpic_batch_target(b, t, C.byref(h)), b)
    return h


def hpic_batch_step(b, n: int = 1) -> None:
    _bcheck(lib().hpic_batch_step(b, n), b)


def _tuning_dict(t: hpic_batch_tuning) -> dict:
    return {"blocks_per_sm": t.blocks_per_sm, "sort_interval": t.sort_interval,
            "use_graph": bool(t.use_graph), "ms_per_step": t.ms_per_step}


def hpic_batch_get_tuning(b) -> dict:
    t = hpic_batch_tuning()
    _bcheck(lib().hpic_batch_get_tuning(b, C.byref(t)), b)
    return _tuning_dict(t)


def hpic_batch_set_tuning(b, blocks_per_sm: int, sort_interval: int, use_graph: bool = True) -> None:
    t = hpic_batch_tuning(blocks_per_sm, sort_interval, int(use_graph), 0, 0.0)
    _bcheck(lib().hpic_batch_set_tuning(b, C.byref(t)), b)


def hpic_batch_autotune(b, trial_steps: int) -> dict:
    t = hpic_batch_tuning()
    _bcheck(lib().hpic_batch_autotune(b, trial_steps, C.byref(t)), b)
    return _tuning_dict(t)


def hpic_batch_profile(b, enable: bool) -> None:
    _bcheck(lib().hpic_batch_profile(b, int(enable)), b)


def hpic_batch_kernel_time(b):
    ms, ps = C.c_double(), C.c_double()
    nl = C.c_int64()
    _bcheck(lib().hpic_batch_kernel_time(b, C.byref(ms), C.byref(nl), C.byref(ps)), b)
    return ms.value, nl.value, ps.value


def hpic_batch_launch_count(b) -> int:
    v = C.c_int64()
    _bcheck(lib().hpic_batch_launch_count(b, C.byref(v)), b)
    return v.value


def hpic_batch_destroy(b) -> None:
    if b:
        _bcheck(lib().hpic_batch_destroy(b))


class Target:
    """Reads and writes of one target's state through a context handle."""

    def __init__(self, h, target: dict, run: dict):
        self.h, self.target, self.run = h, dict(target), dict(run)

    def tallies(self) -> dict:
        return hpic_read_tallies(self.h)

    def reset_tallies(self) -> None:
        hpic_reset_tallies(self.h)

    def hist(self):
        return hpic_read_hist(self.h, self.run["n_E"], self.run["n_theta"])

    def history(self) -> np.ndarray:
        return hpic_read_history(self.h, self.run["max_history"])

    def grid(self, which: str) -> np.ndarray:
        return hpic_read_grid(self.h, which)

    def set_grid(self, which: str, values) -> None:
        hpic_write_grid(self.h, which, values)

    @property
    def n(self) -> int:
        return hpic_count_particles(self.h)

    def particles(self, out: dict | None = None) -> dict:
        return hpic_read_particles(self.h, out)

    def set_particles(self, p: dict) -> None:
        hpic_load_particles(self.h, p)

    def weights(self) -> np.ndarray:
        return hpic_read_weights(self.h)

    def set_weights(self, w) -> None:
        hpic_load_weights(self.h, w)

    def clock(self):
        return hpic_get_clock(self.h)

    def set_clock(self, step: int, next_id: int) -> None:
        hpic_set_clock(self.h, step, next_id)


class Sim(Target):
    """One target on the GPU: the C-ABI calls bundled with their workload dicts."""

    def __init__(self, target: dict, laser: dict | None, run: dict, precision: int = HPIC_FP64,
                 device: int = 0, stream: int = 0, sort_interval: int = 0):
        super().__init__(None, target, run)
        self.h = hpic_init_target(target, run, precision, device, stream, sort_interval)
        if laser is not None:
            hpic_inject_electrons(self.h, laser)

    def close(self) -> None:
        if getattr(self, "h", None):
            hpic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> None:
        hpic_step(self.h, n)

    def seed(self, n: int, mean_energy_J: float) -> None:
        hpic_seed_electrons(self.h, n, mean_energy_J)

    def save(self, path: str) -> None:
        hpic_save(self.h, path)

    @classmethod
    def load(cls, path: str, target: dict, run: dict, device: int = 0, stream: int = 0) -> "Sim":
        """A context restored from a checkpoint (target and run: the dicts the
        saved run was made from, kept for the reads' shapes)."""
        s = cls.__new__(cls)
        Target.__init__(s, None, target, run)
        s.h = hpic_load(path, device, stream)
        return s

    def sort(self) -> None:
        hpic_sort(self.h)


class Batch:
    """Many targets stepped together; batch.target(t) reads target t."""

    def __init__(self, targets: list, lasers: list | None, run: dict,
                 precision: int = HPIC_FP64, spare_slots: int = 0, device: int = 0,
                 stream: int = 0, sort_interval: int = 0, target_index=None):
        self.run = dict(run)
        self.b = hpic_batch_init(targets, lasers, run, precision, spare_slots, device, stream,
                                 sort_interval, target_index)
        ti = (list(target_index) if target_index is not None else
              [int(run.get("target_index", 0)) + t for t in range(len(targets))])
        self.targets = [Target(hpic_batch_target(self.b, t), targets[t],
                               dict(run, target_index=ti[t])) for t in range(len(targets))]

    def __len__(self) -> int:
        return len(self.targets)

    def target(self, t: int) -> Target:
        return self.targets[t]

    def step(self, n: int = 1) -> None:
        hpic_batch_step(self.b, n)

    def tuning(self) -> dict:
        return hpic_batch_get_tuning(self.b)

    def set_tuning(self, blocks_per_sm: int, sort_interval: int, use_graph: bool = True) -> None:
        hpic_batch_set_tuning(self.b, blocks_per_sm, sort_interval, use_graph)

    def autotune(self, trial_steps: int = 40) -> dict:
        return hpic_batch_autotune(self.b, trial_steps)

    def close(self) -> None:
        if getattr(self, "b", None):
            for t in self.targets:
                t.h = None
            hpic_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
