"""CPU-side checks of the CUDA library: it builds for sm_103a, loads without a GPU, and exports every
entry point include/hydro.h declares; plus host-only argument validation that needs no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hydro.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:[A-Za-z_][\w ]*?[\s\*]+)?(\w+)\s*\(", src, flags=re.M))
    return {n for n in names if n.startswith("hydro_") or n.startswith("conserved_totals")}


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("hydro_init", "hydro_step", "hydro_adjoint_step", "hydro_batch_step", "conserved_totals",
              "hydro_last_error", "hydro_destroy"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1507_08549_gb300 import build, hydro
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(hydro.EXPORTS) == _declared()


def test_init_rejects_bad_configs_without_touching_the_device():
    """Configuration errors are found on the host before any CUDA call."""
    from paper_1507_08549_gb300 import hydro, workloads
    lib = hydro.load()
    good = workloads.advected_wave(16)
    bad = [
        good.with_(nx=2),
        good.with_(nfields=3),
        good.with_(bc=(hydro.BC_PERIODIC, hydro.BC_TRANSMISSIVE, 0, 0)),
        good.with_(bc=(hydro.BC_AXIS, hydro.BC_TRANSMISSIVE, 0, 0)),
        good.with_(gamma=1.0),
        good.with_(cfl=0.0),
    ]
    for p in bad:
        cfg = hydro.make_config(p, hydro.HYDRO_F32)
        ctx = ctypes.c_void_p()
        assert lib.hydro_init(ctypes.byref(cfg), None, ctypes.byref(ctx)) == hydro.EINVAL
        assert not ctx.value
    cfg = hydro.make_config(good, 7)
    ctx = ctypes.c_void_p()
    assert lib.hydro_init(ctypes.byref(cfg), None, ctypes.byref(ctx)) == hydro.EINVAL
    assert lib.hydro_init(None, None, ctypes.byref(ctx)) == hydro.EINVAL
    assert lib.hydro_step(None, None, 1, None, None) == hydro.EINVAL
    lib.hydro_destroy(None)
    assert lib.hydro_last_error(None) == b"null context"


def test_binding_rejects_bad_arguments_on_the_host():
    """The Python binding refuses a non-CUDA device and mismatched ensemble lists before any CUDA call."""
    from paper_1507_08549_gb300 import hydro, workloads
    with pytest.raises(hydro.HydroError) as e:
        hydro.Hydro(workloads.advected_wave(16), dtype="f64", device="cpu")
    assert e.value.code == hydro.EINVAL
    with pytest.raises(hydro.HydroError):
        hydro.hydro_batch_step([], [], 1)
    with pytest.raises(hydro.HydroError):
        hydro.hydro_batch_step([object(), object()], [None], 1)


def test_every_entry_point_is_documented():
    """Each declaration in include/hydro.h sits under a comment block (one block may describe a pair of
    related calls declared together)."""
    lines = open(os.path.join(ROOT, "include", "hydro.h")).read().split("\n")
    decl = re.compile(r"^\s*(?:[A-Za-z_][\w ]*?[\s\*]+)?((?:hydro_|conserved_totals)\w*)\s*\(")
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m or line.lstrip().startswith(("*", "/*")):
            continue
        j = i - 1
        while j >= 0 and not lines[j].rstrip().endswith("*/"):
            assert i - j <= 3, f"{m.group(1)} has no comment above it"
            j -= 1
        assert j >= 0, m.group(1)


def test_context_manager_destroys_the_context_once():
    from paper_1507_08549_gb300 import hydro

    class Lib:
        destroyed = []

        def hydro_destroy(self, ctx):
            Lib.destroyed.append(ctx.value)

    h = hydro.Hydro.__new__(hydro.Hydro)
    h.lib, h.ctx = Lib(), ctypes.c_void_p(0x1234)
    with h as inside:
        assert inside is h
    assert Lib.destroyed == [0x1234] and not h.ctx.value
    h.close()
    assert Lib.destroyed == [0x1234]


def test_noalloc_wrapper_refuses_bad_tensors_before_any_launch():
    """The allocation-free totals wrapper checks dtype and shape on the host: a half-precision or a
    smaller tensor would otherwise be read past its end by the kernel."""
    import torch
    from paper_1507_08549_gb300 import hydro, workloads
    p = workloads.advected_wave(16)
    for U in (torch.zeros((4, 16, 16), dtype=torch.float16),
              torch.zeros((4, 16, 16), dtype=torch.bfloat16),
              torch.zeros((4, 16, 16), dtype=torch.int32),
              torch.zeros((4, 16, 15), dtype=torch.float32),
              torch.zeros((3, 16, 16), dtype=torch.float64),
              torch.zeros(4 * 16 * 16, dtype=torch.float32)):
        with pytest.raises(hydro.HydroError) as e:
            hydro.conserved_totals_noalloc(p, U)
        assert e.value.code == hydro.EINVAL
    with pytest.raises(hydro.HydroError):  # right dtype and shape, but not on a CUDA device
        hydro.conserved_totals_noalloc(p, torch.zeros((4, 16, 16), dtype=torch.float32))
