"""The allocation-free cell sort against the library's own cell sort.

hpic_sort_cells_noalloc serves callers that cannot call cudaMalloc (code
inside a CUDA stream capture, hosts with a fixed device-memory budget,
plug-ins whose framework owns all device memory): it takes its scratch from a
fixed array inside the library.  These tests feed it the same electrons that
a context then sorts with hpic_sort, on two calls in a row (the second call
must not see the first call's scratch), in both precisions, and check that
an oversized request is refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2107_01723_gb300 import build as B
from paper_2107_01723_gb300 import hpic
from paper_2107_01723_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "ux", "uy", "uz", "tau")
DEAD = 0xFFFFFFFF


def tile_key(p, dx, n):
    nx, ny, nz = n
    ci = np.minimum(np.floor(p["x"] / dx), nx - 1).astype(np.int64)
    cj = np.minimum(np.floor(p["y"] / dx), ny - 1).astype(np.int64)
    ck = np.minimum(np.floor(p["z"] / dx), nz - 1).astype(np.int64)
    nti, ntj = (nx + 3) // 4, (ny + 3) // 4
    tile = ((ck >> 2) * ntj + (cj >> 2)) * nti + (ci >> 2)
    return tile * 64 + ((ck & 3) << 4) + ((cj & 3) << 2) + (ci & 3)


def noalloc_sort(p, prec, n, dx, n_dead, rng):
    """Upload p (SI, live electrons) in cell units with n_dead dead slots mixed
    in, sort with the allocation-free entry point, return the kept electrons
    in output order (SI)."""
    import torch
    dt = torch.float32 if prec == hpic.HPIC_FP32_MIXED else torch.float64
    m = len(p["id"]) + n_dead
    slots = rng.permutation(m)
    live_slots, dead_slots = slots[:len(p["id"])], slots[len(p["id"]):]
    host = {}
    for k in KEYS:
        a = np.zeros(m)
        a[live_slots] = p[k] / dx if k in ("x", "y", "z") else p[k]
        a[dead_slots] = 0.5
        host[k] = a
    ids = np.full(m, DEAD, dtype=np.uint32)
    ids[live_slots] = p["id"]
    dev_in = [torch.tensor(host[k], dtype=dt, device="cuda") for k in KEYS]
    dev_in.append(torch.tensor(ids.view(np.int32), dtype=torch.int32, device="cuda"))
    dev_out = [torch.full_like(t, -7) for t in dev_in]
    n_live = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    hpic.hpic_sort_cells_noalloc(n[0], n[1], n[2], prec, m, [t.data_ptr() for t in dev_in],
                                 [t.data_ptr() for t in dev_out], n_live.data_ptr(), 0, stream)
    torch.cuda.synchronize()
    kept = int(n_live.item())
    out = {}
    for i, k in enumerate(KEYS):
        v = dev_out[i][:kept].cpu().numpy().astype(np.float64)
        out[k] = v * dx if k in ("x", "y", "z") else v
    out["id"] = dev_out[7][:kept].cpu().numpy().view(np.uint32)
    return out


def assert_same_sort(got, ref, dx, n):
    """Same electrons, same values, same key sequence; order inside one cell
    is free (the sort places equal keys in any order)."""
    assert len(got["id"]) == len(ref["id"])
    kg, kr = tile_key(got, dx, n), tile_key(ref, dx, n)
    assert np.all(np.diff(kg) >= 0)
    assert np.array_equal(kg, kr)
    og = np.lexsort((got["id"], kg))
    orf = np.lexsort((ref["id"], kr))
    assert np.array_equal(got["id"][og], ref["id"][orf])
    # positions pass through metres and back, so allow the FP64 parity
    # tolerance (1e-12 relative); the sort itself only copies values
    for k in KEYS:
        scale = dx if k in ("x", "y", "z") else 1.0
        err = np.abs(got[k][og] - ref[k][orf]) / (np.abs(ref[k][orf]) + scale)
        assert err.size == 0 or err.max() <= 1e-12, (k, float(err.max()))


@pytest.mark.parametrize("prec", [hpic.HPIC_FP32_MIXED, hpic.HPIC_FP64])
def test_noalloc_sort_matches_context_sort_twice(prec):
    B.build()
    cfg = W.config_small(n=(13, 11, 9), n_macro=5000, I_Wcm2=1e21, steps=60, spot_r=3e-6,
                         t_inj=20e-15)
    dx = cfg["target"]["dx"]
    n = (cfg["target"]["nx"], cfg["target"]["ny"], cfg["target"]["nz"])
    rng = np.random.default_rng(21)
    sim = hpic.Sim(cfg["target"], cfg["laser"], cfg["run"], precision=prec)
    for call, (steps, n_dead) in enumerate(((25, 300), (17, 41))):
        sim.step(steps)
        before = sim.particles()  # storage order, live only
        got = noalloc_sort(before, prec, n, dx, n_dead, rng)
        sim.sort()
        ref = sim.particles()
        assert_same_sort(got, ref, dx, n)
    sim.close()


def test_noalloc_sort_refuses_oversize():
    B.build()
    null8 = [0] * 8
    with pytest.raises(hpic.HpicError) as e:
        hpic.hpic_sort_cells_noalloc(8, 8, 8, hpic.HPIC_FP32_MIXED, (1 << 20) + 1, null8, null8, 0)
    assert e.value.code == hpic.HPIC_EINVAL and "1048576" in str(e.value)
    with pytest.raises(hpic.HpicError) as e:
        hpic.hpic_sort_cells_noalloc(1024, 1024, 8, hpic.HPIC_FP32_MIXED, 10, null8, null8, 0)
    assert e.value.code == hpic.HPIC_EINVAL and "cells" in str(e.value)
    # an output array that aliases an input array is refused before any launch
    import torch
    x = torch.zeros(8 * 64, dtype=torch.float32, device="cuda")
    ins = [x.data_ptr() + 4 * 64 * a for a in range(8)]
    with pytest.raises(hpic.HpicError) as e:
        hpic.hpic_sort_cells_noalloc(8, 8, 8, hpic.HPIC_FP32_MIXED, 64, ins, ins, x.data_ptr())
    assert e.value.code == hpic.HPIC_EINVAL and "overlaps" in str(e.value)
