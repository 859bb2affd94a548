"""The C ABI without a GPU: the library builds and loads, exports every entry
point that include/pcdf.h declares, and rejects bad arguments on the host
before anything is enqueued."""
import ctypes
import os
import re

import pytest

from paper_2201_05058_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pcdf_\w+)\s*\(", src, re.M))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("pcdf_build_static_sdf", "pcdf_build_predicted_composite", "pcdf_query_cost",
              "pcdf_query_cost_backward", "pcdf_build_from_scratch", "pcdf_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(_lib.EXPORTS) <= set(declared_functions())


def grid(nx=8, ny=8, nz=8, vox=0.05):
    return _lib.PcdfGrid(nx, ny, nz, vox, (ctypes.c_float * 3)(0, 0, 0))


def err():
    return _lib.load().pcdf_last_error().decode()


@pytest.mark.parametrize("dims", [(0, 8, 8), (8, -1, 8), (8, 8, 513)])
def test_bad_grid_is_rejected(dims):
    lib = _lib.load()
    g = grid(*dims)
    n = ctypes.c_size_t(0)
    assert lib.pcdf_static_workspace_bytes(ctypes.byref(g), ctypes.byref(n)) == -1
    assert "outside" in err()
    fake = ctypes.c_void_p(256)  # never dereferenced: the checks fail first
    assert lib.pcdf_build_static_sdf(ctypes.byref(g), fake, fake, None, fake, 1 << 20, None) == -1


def test_bad_voxel_size_is_rejected():
    lib = _lib.load()
    n = ctypes.c_size_t(0)
    for vox in (0.0, -1.0, float("nan"), float("inf")):
        assert lib.pcdf_static_workspace_bytes(ctypes.byref(grid(vox=vox)), ctypes.byref(n)) == -1


def test_workspace_sizes():
    lib = _lib.load()
    n = ctypes.c_size_t(0)
    g = grid(64, 64, 64)
    assert lib.pcdf_static_workspace_bytes(ctypes.byref(g), ctypes.byref(n)) == 0
    assert n.value >= 64 ** 3 * 6
    # composite: slab of one standing capsule (z from 0 to 1.8 m at 5 cm)
    caps = (ctypes.c_int32 * 7)(512, 512, 80, 512, 512, 496, 80)
    assert lib.pcdf_composite_workspace_bytes(ctypes.byref(g), 1, 1, caps, ctypes.byref(n)) == 0
    S = 36  # voxels k with 16 k + 8 in [0, 576]
    assert n.value >= S * 64 * 64 * 4 + 64 * 64 * 4  # int32 partial per slab voxel, column maxima
    # no capsule touches the grid: no workspace needed beyond alignment
    far = (ctypes.c_int32 * 7)(-8000, -8000, -8000, -8000, -8000, -7000, 80)
    assert lib.pcdf_composite_workspace_bytes(ctypes.byref(g), 1, 1, far, ctypes.byref(n)) == 0
    assert n.value == 0


def test_capsule_range_checks():
    lib = _lib.load()
    n = ctypes.c_size_t(0)
    g = grid()
    bad = (ctypes.c_int32 * 7)(0, 0, 0, 0, 0, 20000, 10)
    assert lib.pcdf_composite_workspace_bytes(ctypes.byref(g), 1, 1, bad, ctypes.byref(n)) == -1
    assert "outside" in err()
    bad_r = (ctypes.c_int32 * 7)(0, 0, 0, 0, 0, 0, -1)
    assert lib.pcdf_composite_workspace_bytes(ctypes.byref(g), 1, 1, bad_r, ctypes.byref(n)) == -1
    assert lib.pcdf_composite_workspace_bytes(ctypes.byref(g), 0, 1, bad_r, ctypes.byref(n)) == -1
    assert lib.pcdf_composite_workspace_bytes(ctypes.byref(g), 1, 65, None, ctypes.byref(n)) == -1
    assert lib.pcdf_composite_workspace_bytes(ctypes.byref(g), 1, 1, None, ctypes.byref(n)) == -1


def test_query_rejects_unaligned_spheres():
    lib = _lib.load()
    g = grid()
    fake = ctypes.c_void_p(256)
    rc = lib.pcdf_query_cost(ctypes.byref(g), fake, 1, ctypes.c_void_p(260), fake, 10, 0.2, fake, None, None)
    assert rc == -1 and "aligned" in err()
    assert lib.pcdf_query_cost(ctypes.byref(g), fake, 0, fake, fake, 10, 0.2, fake, None, None) == -1
    assert lib.pcdf_query_cost(ctypes.byref(g), fake, 1, fake, fake, -1, 0.2, fake, None, None) == -1
