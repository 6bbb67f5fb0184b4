"""Helpers for the GPU-vs-oracle parity tests: move a state from the oracle
into a GPU context through the C-ABI, and compare states element by element."""
import numpy as np

from oracle import oracle as O
from paper_2107_01723_gb300 import hpic

PKEYS = ("x", "y", "z", "ux", "uy", "uz", "tau")
GRIDS_STATE = ("T", "eta", "Ti", "Ex", "Ey", "Ez", "Bx", "By", "Bz")
ENERGY_TALLIES = ("E_injected", "W_field", "E_drag", "E_xray", "E_xray_above", "E_escaped",
                  "E_reflux", "E_ohmic_grid")
COUNT_TALLIES = ("n_injected", "n_escaped", "n_refluxed", "n_reflux_absorbed", "n_cut",
                 "n_emitted", "particle_steps")


def gpu_from_oracle(osim: O.OracleSim, cfg: dict, precision: int, sort_interval: int = 0):
    g = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=precision,
                 sort_interval=sort_interval)
    g.set_particles(osim.particles())
    if cfg["laser"].get("envelope", 0) == 1:  # per-electron weights
        g.set_weights(O.weights(osim))
    for k in GRIDS_STATE:
        g.set_grid(k, osim.grid(k))
    step, nid = osim.clock()
    g.set_clock(step, nid)
    g.reset_tallies()
    return g


def by_id(p: dict) -> dict:
    o = np.argsort(p["id"], kind="stable")
    return {k: np.asarray(v)[o] for k, v in p.items()}


def assert_particles_close(gp: dict, op: dict, tol: float, dx: float):
    gp, op = by_id(gp), by_id(op)
    assert np.array_equal(gp["id"], op["id"]), (
        f"surviving ids differ: {len(gp['id'])} vs {len(op['id'])}, "
        f"only GPU {np.setdiff1d(gp['id'], op['id'])[:10]}, only oracle {np.setdiff1d(op['id'], gp['id'])[:10]}")
    for k in PKEYS:
        scale = dx if k in ("x", "y", "z") else 1.0
        err = np.abs(gp[k] - op[k]) / (np.abs(op[k]) + scale)
        assert err.size == 0 or err.max() <= tol, (k, float(err.max()), int(np.argmax(err)))


def assert_field_close(g: np.ndarray, o: np.ndarray, tol: float, name: str, scale=None):
    """Max-norm error relative to `scale` (default: the field's own max-norm)."""
    if scale is None:
        scale = np.abs(o).max()
    err = np.abs(g - o).max() / max(scale, 1e-300)
    assert err <= tol, (name, float(err))


def assert_vector_close(gsim, osim_grid, prefix: str, tol: float):
    """Components of one vector field (E, B or j_h) against the max-norm of the
    whole vector: a transverse component that nearly cancels is judged on the
    field's scale, not on its own small maximum."""
    comps = [prefix + c for c in "xyz"]
    o = {c: osim_grid(c) for c in comps}
    scale = max(np.abs(v).max() for v in o.values())
    for c in comps:
        assert_field_close(gsim(c), o[c], tol, c, scale)


def faraday_tol(o, cfg: dict, tol: float) -> float:
    """Tolerance on B (against its max-norm) one Faraday step after B = 0,
    propagated from the tolerance on E (against E's max-norm): each B
    component is dt times two differences of E components over dx, so an
    element error of tol max|E| in E bounds B's error by 4 tol dt max|E| / dx
    (Eq. (A3); B is not deposited, it follows from E).  Never below tol."""
    E = max(np.abs(o.grid(k)).max() for k in ("Ex", "Ey", "Ez"))
    B = max(np.abs(o.grid(k)).max() for k in ("Bx", "By", "Bz"))
    if B == 0.0:
        return tol
    return max(tol, 4.0 * tol * cfg["run"]["dt"] * E / (cfg["target"]["dx"] * B))


def tally_delta(after: dict, before: dict) -> dict:
    return {k: after[k] - before[k] for k in after}


def assert_tallies_close(gt: dict, ot: dict, tol: float, abs_tol: float, exact_counts: bool = True):
    """Energy tallies within tol relative plus abs_tol (J).  In FP32 a
    per-electron energy difference carries a few ulp of the electron's own
    energy, so abs_tol scales with the kinetic energy held by the electrons."""
    for k in ENERGY_TALLIES:
        assert abs(gt[k] - ot[k]) <= tol * abs(ot[k]) + abs_tol, (k, gt[k], ot[k])
    for k in COUNT_TALLIES:
        if exact_counts:
            assert gt[k] == ot[k], (k, gt[k], ot[k])


def heat_cells(p: dict, dx: float, shape, fp32: bool) -> np.ndarray:
    """Cell of x^n that receives each electron's drag heat (the clamped floor of
    its position in cells), taken in the precision the position is held in."""
    idx = []
    for k, n in zip("xyz", shape):
        X = np.asarray(p[k]) / dx
        if fp32:  # the kernel's own FP32 coordinate, recovered exactly
            X = X.astype(np.float32)
        idx.append(np.clip(np.floor(X), 0, n - 1).astype(np.int64))
    return idx[0] + shape[0] * (idx[1] + shape[1] * idx[2])


def heat_with_cell_swaps(cfg: dict, state: dict, clock, gp: dict, op: dict,
                         o_heat: np.ndarray, fp32: bool, limit: int = 64):
    """The oracle's drag heat of one step, with the heat of every electron whose
    cell the kernel took differently moved to the kernel's cell.

    The drag heat goes to the cell holding x^n, a decision by floor(x/dx): an
    FP32 coordinate within rounding of a cell face can land on the other side
    than the FP64 one.  `gp`, `op` are the kernel's and the oracle's electrons
    at the start of the step, `state` and `clock` the oracle's grids and clock
    there.  The heat of each swapped electron comes from the oracle stepping
    that electron alone in the same fields.  Returns the corrected heat and
    the cells involved (whose T and eta then differ by that electron's heat)."""
    t = cfg["target"]
    shape, dx = (t["nx"], t["ny"], t["nz"]), t["dx"]
    gp, op = by_id(gp), by_id(op)
    assert np.array_equal(gp["id"], op["id"])
    cg, co = heat_cells(gp, dx, shape, fp32), heat_cells(op, dx, shape, False)
    swapped = np.nonzero(cg != co)[0]
    assert swapped.size <= limit, f"{swapped.size} electrons change heat cell"
    heat = o_heat.copy()
    touched = np.unique(np.concatenate([cg[swapped], co[swapped]]))
    todo = list(swapped)
    while todo:  # electrons stepped together must sit in distinct oracle cells
        batch, seen, rest = [], set(), []
        for i in todo:
            (rest if co[i] in seen else batch).append(i)
            seen.add(co[i])
        s = O.OracleSim(t, cfg["laser"], cfg["run"])
        for k in GRIDS_STATE:
            s.set_grid(k, state[k])
        s.set_particles({k: v[batch] for k, v in op.items()})
        s.set_clock(*clock)
        s.reset_tallies()
        s.step(1)
        h = s.grid("heat")[co[batch]]
        del s
        np.add.at(heat, co[batch], -h)
        np.add.at(heat, cg[batch], h)
        todo = rest
    return heat, touched


def smooth_grids(t: dict, seed: int, E0=3e9, B0=200.0) -> dict:
    """Smooth non-zero fields over the whole grid (oracle layout): each E and
    B component a sum of two plane waves of random low wave numbers (E0 V/m,
    B0 T), padding entries past a component's staggered extent left at 0;
    T from 1 to 500 eV as a smooth pattern with eta = eta(T); T_i = T."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = t["nx"], t["ny"], t["nz"]
    i = np.arange(nx + 1, dtype=np.float64)[None, None, :] / nx
    j = np.arange(ny + 1, dtype=np.float64)[None, :, None] / ny
    k = np.arange(nz + 1, dtype=np.float64)[:, None, None] / nz

    def wave(a, b, c):
        p = rng.integers(1, 4, size=(2, 3))
        ph = rng.uniform(0, 2 * np.pi, 2)
        return (0.6 * np.sin(2 * np.pi * (p[0, 0] * a + p[0, 1] * b + p[0, 2] * c) + ph[0])
                + 0.4 * np.cos(2 * np.pi * (p[1, 0] * a + p[1, 1] * b + p[1, 2] * c) + ph[1]))

    out = {}
    # staggering (half cells) of Ex Ey Ez Bx By Bz along x, y, z
    stag = {"Ex": (1, 0, 0), "Ey": (0, 1, 0), "Ez": (0, 0, 1),
            "Bx": (0, 1, 1), "By": (1, 0, 1), "Bz": (1, 1, 0)}
    for name, (sx, sy, sz) in stag.items():
        amp = E0 if name[0] == "E" else B0
        v = amp * wave(i + 0.5 * sx / nx, j + 0.5 * sy / ny, k + 0.5 * sz / nz)
        v = np.broadcast_to(v, (nz + 1, ny + 1, nx + 1)).copy()
        if sx:
            v[:, :, nx] = 0.0
        if sy:
            v[:, ny, :] = 0.0
        if sz:
            v[nz, :, :] = 0.0
        out[name] = v.ravel()
    ci = (np.arange(nx) + 0.5)[None, None, :] / nx
    cj = (np.arange(ny) + 0.5)[None, :, None] / ny
    ck = (np.arange(nz) + 0.5)[:, None, None] / nz
    # T on 64 levels, geometric from 1 to 500 eV, and eta = eta(T) of each
    # level: a stepped state keeps eta equal to eta(T) (a cell without heat or
    # current keeps both), so the input does too
    levels = 11604.5 * np.geomspace(1.0, 500.0, 64)
    eta_lv = np.array([O.resistivity(t, T) for T in levels])
    lv = np.clip(((wave(ci, cj, ck) + 1.0) * 32.0).astype(np.int64), 0, 63)
    lv = np.broadcast_to(lv, (nz, ny, nx)).ravel()
    out["T"] = levels[lv]
    out["eta"] = eta_lv[lv]
    out["Ti"] = out["T"].copy()
    return out


def spread_electrons(t: dict, n: int, seed: int, e_lo=5e4, e_hi=6e7) -> dict:
    """n electrons over the whole box plus electrons at its 8 corners and in
    the first and last cell of each axis, moving in all directions, kinetic
    energies log-uniform over [e_lo, e_hi] eV.  Coordinates (in cells) are
    FP32 numbers whose fractional parts stay 1e-4 away from 0 and 1/2, so
    that the FP32 path holds the same positions exactly and every cell
    decision (the drag heat's cell, a lattice's base node) is the oracle's."""
    rng = np.random.default_rng(seed)
    dims = np.array([t["nx"], t["ny"], t["nz"]], dtype=np.float64)
    X = rng.uniform(0.0, 1.0, size=(n, 3)) * dims
    lo = [0.3, 0.7]
    corners = np.array([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)], float)
    edge = np.vstack([corners * (dims - 0.6) + 0.3,
                      np.column_stack([dims[0] - np.array(lo), np.full(2, dims[1] / 2), np.full(2, dims[2] / 2)]),
                      np.column_stack([np.full(2, dims[0] / 2), dims[1] - np.array(lo), np.full(2, dims[2] / 2)]),
                      np.column_stack([np.full(2, dims[0] / 2), np.full(2, dims[1] / 2), dims[2] - np.array(lo)]),
                      np.column_stack([np.array(lo), np.array(lo), np.array(lo)])])
    X = np.vstack([edge, X]).astype(np.float32).astype(np.float64)
    fr = X - np.floor(X)
    keep = np.all((np.abs(fr - 0.5) > 1e-4) & (fr > 1e-4) & (fr < 1 - 1e-4), axis=1)
    X = X[keep]
    m = len(X)
    eps = 1.602176634e-19 * np.exp(rng.uniform(np.log(e_lo), np.log(e_hi), m))
    mc2 = 9.1093837015e-31 * 299792458.0 ** 2
    e = eps / mc2
    u = np.sqrt(e * (e + 2.0))
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    # the corner and edge electrons head out through their nearest faces
    ne = int(keep[:len(edge)].sum())
    out_dir = np.sign(X[:ne] - dims / 2)
    d[:ne] = out_dir / np.linalg.norm(out_dir, axis=1)[:, None]
    dx = t["dx"]
    return {"x": X[:, 0] * dx, "y": X[:, 1] * dx, "z": X[:, 2] * dx,
            "ux": u * d[:, 0], "uy": u * d[:, 1], "uz": u * d[:, 2],
            "tau": -np.log(1.0 - rng.uniform(0.0, 1.0, m)),
            "id": np.arange(m, dtype=np.uint32)}


def live_state(cfg: dict, n: int, seed: int, step: int, e_hi=6e7) -> "O.OracleSim":
    """An oracle context at clock `step` (after the injection window) holding
    smooth non-zero grids and electrons spread over the whole box (kinetic
    energies up to e_hi eV)."""
    o = O.OracleSim(cfg["target"], cfg["laser"], cfg["run"])
    for k, v in smooth_grids(cfg["target"], seed).items():
        o.set_grid(k, v)
    p = spread_electrons(cfg["target"], n, seed + 1, e_hi=e_hi)
    o.set_particles(p)
    o.set_clock(step, len(p["id"]))
    o.reset_tallies()
    return o
