"""Host-side checks of the C-ABI (no GPU): the library loads, exports every
function include/hpic.h declares, its struct layouts match the binding, and
argument validation fails with the documented codes before any CUDA work."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2107_01723_gb300 import build as B
from paper_2107_01723_gb300 import hpic
from paper_2107_01723_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hpic.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return hpic.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hpic_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "hpic.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(hpic_target_desc), sizeof(hpic_laser_desc), sizeof(hpic_run_params),"
        "sizeof(hpic_tallies), offsetof(hpic_run_params, kappa_esc),"
        "offsetof(hpic_run_params, max_history), offsetof(hpic_laser_desc, n_macro),"
        "sizeof(hpic_batch_tuning), offsetof(hpic_batch_tuning, ms_per_step));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(hpic.hpic_target_desc), C.sizeof(hpic.hpic_laser_desc),
            C.sizeof(hpic.hpic_run_params), C.sizeof(hpic.hpic_tallies),
            hpic.hpic_run_params.kappa_esc.offset, hpic.hpic_run_params.max_history.offset,
            hpic.hpic_laser_desc.n_macro.offset, C.sizeof(hpic.hpic_batch_tuning),
            hpic.hpic_batch_tuning.ms_per_step.offset]
    assert got == want


def _bad(lib, target, run):
    h = C.c_void_p()
    t, r = hpic.target_desc(target), hpic.run_params(run)
    code = lib.hpic_init_target(C.byref(h), C.byref(t), C.byref(r), 0, None)
    assert not h.value
    return code, lib.hpic_last_error(None).decode()


def test_validation_rejects_bad_arguments(lib):
    c = W.config_small()
    t, r = c["target"], c["run"]
    assert _bad(lib, dict(t, nx=1), r)[0] == hpic.HPIC_EINVAL
    assert _bad(lib, dict(t, dx=1e-7), r)[0] == hpic.HPIC_EINVAL  # c dt > dx
    assert _bad(lib, dict(t, Z=0.0), r)[0] == hpic.HPIC_EINVAL
    assert _bad(lib, t, dict(r, n_E=0))[0] == hpic.HPIC_EINVAL
    assert _bad(lib, t, dict(r, table_rows=1))[0] == hpic.HPIC_EINVAL
    assert _bad(lib, t, dict(r, physics=512))[0] == hpic.HPIC_EINVAL  # undefined bit
    assert _bad(lib, dict(t, A_ion=0.0), dict(r, physics=hpic.HPIC_ALL | hpic.HPIC_EI_EQUIL))[0] == hpic.HPIC_EINVAL
    code, msg = _bad(lib, dict(t, nx=1), r)
    assert "dimension" in msg
    assert lib.hpic_init_target(None, None, None, 0, None) == hpic.HPIC_EINVAL
    assert lib.hpic_step(None, 1) == hpic.HPIC_EINVAL
    assert lib.hpic_destroy(None) == hpic.HPIC_EINVAL
    # the electron transfers refuse a missing context before any device call
    n = C.c_int64()
    assert lib.hpic_count_particles(None, C.byref(n)) == hpic.HPIC_EINVAL
    assert lib.hpic_read_particles(None, *([None] * 8), 0, C.byref(n)) == hpic.HPIC_EINVAL
    assert lib.hpic_load_particles(None, 0, *([None] * 8)) == hpic.HPIC_EINVAL


def test_no_device_is_an_error_not_a_fallback(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    c = W.config_small()
    code, msg = _bad(lib, c["target"], c["run"])
    assert code == hpic.HPIC_ECUDA


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(hpic, "_lib", None)
    monkeypatch.setattr(hpic, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(FileNotFoundError):
        hpic.lib()


def _bad_batch(lib, targets, lasers, run, spare=0):
    b = C.c_void_p()
    n = len(targets)
    T = (hpic.hpic_target_desc * max(n, 1))(*[hpic.target_desc(t) for t in targets])
    L = (hpic.hpic_laser_desc * max(n, 1))(*[hpic.laser_desc(l) for l in lasers]) if lasers else None
    r = hpic.run_params(run)
    code = lib.hpic_batch_init(C.byref(b), n, T, L, C.byref(r), None, spare, 0, None)
    assert not b.value
    return code, lib.hpic_batch_last_error(None).decode()


def test_batch_validation_rejects_bad_arguments(lib):
    c = W.config_small()
    t, l, r = c["target"], c["laser"], c["run"]
    assert _bad_batch(lib, [], None, r)[0] == hpic.HPIC_EINVAL
    assert _bad_batch(lib, [t] * (hpic.HPIC_BATCH_MAX_TARGETS + 1), None, r)[0] == hpic.HPIC_EINVAL
    code, msg = _bad_batch(lib, [t, dict(t, nx=1)], None, r)
    assert code == hpic.HPIC_EINVAL and msg.startswith("target 1:")
    code, msg = _bad_batch(lib, [t, t], [l, dict(l, spot_r=1.0)], r)
    assert code == hpic.HPIC_EINVAL and msg.startswith("laser 1:")
    assert _bad_batch(lib, [t], [l], r, spare=-1)[0] == hpic.HPIC_EINVAL
    assert lib.hpic_batch_step(None, 1) == hpic.HPIC_EINVAL
    assert lib.hpic_batch_destroy(None) == hpic.HPIC_EINVAL
    assert lib.hpic_batch_target(None, 0, None) == hpic.HPIC_EINVAL


def test_batch_without_device_is_an_error(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    c = W.config_small()
    code, _ = _bad_batch(lib, [c["target"]] * 2, [c["laser"]] * 2, c["run"])
    assert code == hpic.HPIC_ECUDA


def test_model_validation_and_no_device(lib):
    good = W.model_point()
    with pytest.raises(hpic.HpicError) as e:
        hpic.hpic_model([good, dict(good, rel_step=0.0)])
    assert e.value.code == hpic.HPIC_EINVAL
    with pytest.raises(hpic.HpicError) as e:
        hpic.hpic_model([dict(good, mechanisms=hpic.HPIC_MODEL_FIELD)])  # nothing else slows it
    assert e.value.code == hpic.HPIC_EINVAL
    assert hpic.hpic_model([]) == []
    try:
        import torch
        if torch.cuda.is_available():
            return
    except ImportError:
        pass
    with pytest.raises(hpic.HpicError) as e:
        hpic.hpic_model([good])
    assert e.value.code == hpic.HPIC_ECUDA


def test_checkpoint_load_rejects_bad_files(lib, tmp_path):
    with pytest.raises(hpic.HpicError) as e:
        hpic.hpic_load(str(tmp_path / "missing.ckpt"))
    assert e.value.code == hpic.HPIC_EINVAL
    junk = tmp_path / "junk.ckpt"
    junk.write_bytes(b"not a checkpoint at all" * 10)
    with pytest.raises(hpic.HpicError) as e:
        hpic.hpic_load(str(junk))
    assert e.value.code == hpic.HPIC_EINVAL
    assert "checkpoint" in lib.hpic_last_error(None).decode()


def test_batch_refuses_the_gaussian_envelope(lib):
    c = W.config_small()
    t = c["target"]
    g = W.laser_gauss(t, per_cell=10)
    code, msg = _bad_batch(lib, [t, t], [c["laser"], g], c["run"])
    assert code == hpic.HPIC_EINVAL and "flat-top" in msg


def test_noalloc_sort_refuses_overlapping_arrays(lib):
    """The allocation-free sort reads its input arrays while it writes its
    output arrays, so any output range that overlaps an input range is
    refused with HPIC_EINVAL before any device call (the addresses below are
    never dereferenced).  Disjoint ranges pass this check and, with no GPU
    here, stop at the device call instead."""
    n = 100
    base = 1 << 32
    ins = [base + a * 4096 for a in range(8)]
    outs = [base + (1 << 20) + a * 4096 for a in range(8)]
    for prec, rb in ((hpic.HPIC_FP32_MIXED, 4), (hpic.HPIC_FP64, 8)):
        for a, b, shift in ((3, 3, 0), (0, 5, rb * (n - 1)), (7, 2, -rb * n + 4)):
            bad = list(outs)
            bad[b] = ins[a] + shift
            with pytest.raises(hpic.HpicError) as e:
                hpic.hpic_sort_cells_noalloc(8, 8, 8, prec, n, ins, bad, base - 64)
            assert e.value.code == hpic.HPIC_EINVAL and "overlaps" in str(e.value), (a, b, shift)
        # adjacent but disjoint: the next range starts where the input ends
        ok = list(outs)
        ok[0] = ins[6] + rb * n
        with pytest.raises(hpic.HpicError) as e:
            hpic.hpic_sort_cells_noalloc(8, 8, 8, prec, n, ins, ok, base - 64)
        assert e.value.code != hpic.HPIC_EINVAL


def test_read_into_buffers_checks_them_first():
    """Reading the electrons into caller-owned buffers (page-locked ones, for
    instance) checks each buffer's type, layout and length before any library
    call, so a wrong buffer is an error and never a partial copy."""
    n = 4
    good = {k: np.zeros(n) for k in ("x", "y", "z", "ux", "uy", "uz", "tau")}
    good["id"] = np.zeros(n, dtype=np.uint32)
    for k, bad in (("ux", np.zeros(n, dtype=np.float32)), ("x", np.zeros(2 * n)[::2]),
                   ("tau", np.zeros(n + 1)), ("id", np.zeros(n, dtype=np.int64))):
        with pytest.raises(ValueError):
            hpic.hpic_read_particles(None, dict(good, **{k: bad}))
