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
    # row words and their carries (4 + 8 bytes per 32 voxels of a row), int32 partial field
    assert n.value >= 64 ** 3 * 4 + 64 * 64 * 2 * 12
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


def test_template_box_matches_the_oracle_and_rejects_bad_primitives():
    """The host-side template box of the translated primitive field against the
    oracle's, and its argument checks (no device work)."""
    import numpy as np

    import oracle
    import paper_2201_05058_gb300 as pcdf

    rng = np.random.default_rng(7)
    for n in range(200):
        a = rng.integers(-1500, 4000, 3)
        b = a + rng.integers(-300, 300, 3)
        r = int(rng.integers(0, 200))
        if n % 4 == 3 and not np.array_equal(a, b):
            r |= oracle.CYLINDER
        cap = np.array([*a, *b, r], np.int32)
        R = int(rng.integers(0, 40))
        try:
            want = oracle.template_box(cap, R)
        except ValueError:
            with pytest.raises(RuntimeError):
                pcdf.template_box(cap, R)
            continue
        if max(want[1]) > 512:
            with pytest.raises(RuntimeError):
                pcdf.template_box(cap, R)
            continue
        assert pcdf.template_box(cap, R) == (list(want[0]), list(want[1]))
    lib = _lib.load()
    lo = (ctypes.c_int32 * 3)()
    dims = (ctypes.c_int32 * 3)()
    ok = np.array([40, 40, 40, 40, 40, 200, 30], np.int32)
    p = ok.ctypes.data_as(ctypes.c_void_p)
    assert lib.pcdf_template_box(p, 4, lo, dims) == 0
    assert lib.pcdf_template_box(p, -1, lo, dims) == -1          # R < 0
    assert lib.pcdf_template_box(p, 600, lo, dims) == -1         # side > PCDF_MAX_DIM
    assert lib.pcdf_template_box(None, 4, lo, dims) == -1
    zero_cyl = np.array([40, 40, 40, 40, 40, 40, 30 | oracle.CYLINDER], np.int32)
    assert lib.pcdf_template_box(zero_cyl.ctypes.data_as(ctypes.c_void_p), 4, lo, dims) == -1
    g = grid()
    placements = np.zeros((1, 1, 3), np.int32)
    placements[0, 0, 0] = 900                                    # outside [-512, 512]
    d3 = (ctypes.c_int32 * 3)(8, 8, 8)
    small = (ctypes.c_int32 * 3)(4, 4, 4)   # with R = 2: 2 R >= side
    fake = ctypes.c_void_p(256)                                  # never dereferenced: rejected first
    assert lib.pcdf_composite_translated(ctypes.byref(g), fake, None, 1, 1, fake, d3, 2,
                                         placements.ctypes.data_as(ctypes.c_void_p), fake, None, None) == -1
    assert lib.pcdf_composite_translated(ctypes.byref(g), fake, None, 1, 1, None, d3, 2,
                                         placements.ctypes.data_as(ctypes.c_void_p), fake, None, None) == -1
    placements[0, 0, 0] = 0
    assert lib.pcdf_composite_translated(ctypes.byref(g), fake, None, 1, 1, fake, small, 2,
                                         placements.ctypes.data_as(ctypes.c_void_p), fake, None, None) == -1  # 2 R >= side
    bad_dims = (ctypes.c_int32 * 3)(4, 0, 4)
    assert lib.pcdf_composite_translated(ctypes.byref(g), fake, None, 1, 1, fake, bad_dims, 2,
                                         placements.ctypes.data_as(ctypes.c_void_p), fake, None, None) == -1


def test_lattice_placements_follow_the_moved_boxes():
    """Placements of whole-voxel moves are the moved primitives' own template
    boxes (oracle), and anything that is not such a move is refused."""
    import numpy as np

    import oracle
    import paper_2201_05058_gb300 as pcdf
    import scenes

    rng = np.random.default_rng(21)
    ref = np.array([300, 410, 100, 300, 410, 620, 100], np.int32)
    lo0, _ = oracle.template_box(ref, 7)
    moves = rng.integers(-20, 20, (4, 3, 3))
    caps = np.empty((4, 3, 7), np.int32)
    caps[..., 0:3] = ref[0:3] + 16 * moves
    caps[..., 3:6] = ref[3:6] + 16 * moves
    caps[..., 6] = ref[6]
    lo = pcdf.lattice_placements(caps, ref, lo0)
    for t in range(4):
        for h in range(3):
            assert list(lo[t, h]) == list(oracle.template_box(caps[t, h], 7)[0])
    # the scene helper lays sub-voxel positions on that lattice, keeping the shape
    sc = scenes.scene_composite(seed=1, n=64, n_boxes=4, T=5)
    lat = scenes.lattice_moves(sc["caps"], sc["caps"][0, 0])
    step = lat[..., 0:3].astype(np.int64) - sc["caps"][0, 0, 0:3]
    assert np.all(step % 16 == 0)
    assert np.all(np.abs(lat[..., 0:3].astype(np.int64) - sc["caps"][..., 0:3]) <= 8)
    pcdf.lattice_placements(lat, lat[0, 0], lo0)
    bad = caps.copy()
    bad[1, 2, 0] += 3                       # a sub-voxel move
    bad[1, 2, 3] += 3
    with pytest.raises(ValueError):
        pcdf.lattice_placements(bad, ref, lo0)
    bad = caps.copy()
    bad[0, 1, 6] += 1                       # another radius
    with pytest.raises(ValueError):
        pcdf.lattice_placements(bad, ref, lo0)
    bad = caps.copy()
    bad[2, 0, 5] += 16                      # another length
    with pytest.raises(ValueError):
        pcdf.lattice_placements(bad, ref, lo0)


def test_template_radius_is_the_ceiling_square_root():
    """pcdf_template_radius against the integer square root (rounded up) and
    its argument checks."""
    import math

    lib = _lib.load()
    R = ctypes.c_int32(-1)
    for m in [0, 1, 2, 3, 4, 5, 8, 9, 10, 11880, 11881, 11882, 3 * 511 * 511, 2 ** 31 - 2, 2 ** 31 - 1]:
        assert lib.pcdf_template_radius(m, ctypes.byref(R)) == 0
        r = math.isqrt(m)
        assert R.value == (r if r * r >= m else r + 1), m
    assert lib.pcdf_template_radius(-1, ctypes.byref(R)) == -1
    assert lib.pcdf_template_radius(4, None) == -1


def test_bounds_check_entry_point_in_the_normal_build():
    """pcdf_bounds_check exists in every build; only the debug build
    (PCDF_CHECK_BOUNDS) has index checks to report, so the normal one refuses."""
    lib = _lib.load(checked=False)
    first, count = ctypes.c_uint32(7), ctypes.c_uint32(7)
    assert lib.pcdf_bounds_check(ctypes.byref(first), ctypes.byref(count), 0) == -1
    assert "not a bounds-checked build" in err()
    assert first.value == 0 and count.value == 0


def test_context_calls_check_their_arguments_before_the_device():
    """The context calls refuse a NULL context (and pcdf_create a NULL out,
    pcdf_build_batched a bad use_graph) before touching a device;
    pcdf_destroy(NULL) is a no-op; pcdf_scratch_bytes bounds the scratch of
    every context call (host only)."""
    lib = _lib.load()
    g = grid(64, 48, 32)
    fake = ctypes.c_void_p(256)  # never dereferenced: the checks fail first
    assert lib.pcdf_create(None, 0, None) == -1
    lib.pcdf_destroy(None)
    assert lib.pcdf_ctx_reserve(None, 1024) == -1
    assert lib.pcdf_ctx_build_static_sdf(None, ctypes.byref(g), fake, fake, None) == -1
    assert "ctx is NULL" in err()
    assert lib.pcdf_ctx_build_predicted_composite(None, ctypes.byref(g), fake, None, 1, 0, None, fake, None) == -1
    assert lib.pcdf_ctx_build_from_scratch(None, ctypes.byref(g), fake, 1, 0, None, fake, None) == -1
    assert lib.pcdf_ctx_query_cost(None, ctypes.byref(g), fake, 1, fake, fake, 1, 0.2, fake, None) == -1
    assert lib.pcdf_ctx_query_cost_backward(None, ctypes.byref(g), fake, 1, fake, fake, 1, 0.2, fake, fake,
                                            None) == -1
    assert lib.pcdf_build_batched(None, None, 1, 0) == -1
    n = ctypes.c_size_t(0)
    assert lib.pcdf_scratch_bytes(ctypes.byref(g), 5, 2, ctypes.byref(n)) == 0
    V = 64 * 48 * 32
    # a composite touching every slice: int16 and int32 slab intermediates and the column maxima
    assert n.value >= 5 * V * 6 + 64 * 48 * 4
    static = ctypes.c_size_t(0)
    assert lib.pcdf_static_workspace_bytes(ctypes.byref(g), ctypes.byref(static)) == 0
    assert n.value >= static.value
    assert lib.pcdf_scratch_bytes(ctypes.byref(g), 0, 2, ctypes.byref(n)) == -1
    assert lib.pcdf_scratch_bytes(ctypes.byref(g), 5, -1, ctypes.byref(n)) == -1
    assert lib.pcdf_scratch_bytes(ctypes.byref(g), 5, 2, None) == -1
