"""The bounds-checked debug build (libpcdf_checked.so, compiled with
PCDF_CHECK_BOUNDS; the stand-in for a memory checker, which this pool does
not offer).  Odd-size and edge cases of the static EDT, the composite
(capsules cut by the grid boundary, thin and slanted), the from-scratch
comparator and the cost query with its backward run through it: the results
equal the oracle's, and the device's record of failed index checks stays
empty."""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu

pcdf = pytest.importorskip("paper_2201_05058_gb300")
from paper_2201_05058_gb300 import _lib  # noqa: E402

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2201_05058_gb300", "csrc")


def file_tag(name: str) -> int:
    """The 16-bit tag the checks record for a source file (djb2 of its name)."""
    h = 5381
    for ch in name.encode():
        h = (h * 33 + ch) & 0xFFFFFFFF
    return h & 0xFFFF


def where(code: int) -> str:
    tags = {file_tag(f): f for f in os.listdir(CSRC)}
    return f"{tags.get(code >> 16, hex(code >> 16))}:{code & 0xFFFF}"


@pytest.fixture
def checked():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.use_checked(True)
    lib = _lib.load()
    assert lib.pcdf_bounds_check(None, None, 1) == 0, lib.pcdf_last_error().decode()
    yield lib
    _lib.use_checked(False)


def assert_clean(lib):
    first, count = ctypes.c_uint32(0), ctypes.c_uint32(0)
    assert lib.pcdf_bounds_check(ctypes.byref(first), ctypes.byref(count), 0) == 0
    assert count.value == 0, f"{count.value} failed index checks, first at {where(first.value)}"


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


SHAPES = [(1, 1, 37), (37, 1, 1), (33, 1, 70), (37, 45, 29), (70, 65, 33), (512, 3, 2), (2, 3, 512), (31, 33, 65)]


@pytest.mark.parametrize("shape", SHAPES)
def test_static_edt_checked(checked, shape):
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 7 + ny * 3 + nz)
    for density in (0.0, 0.05, 0.5):
        occ = (rng.random((nz, ny, nx)) < density).astype(np.uint8)
        grid = scenes.Grid(nx, ny, nz, 0.05)
        sq, sdf = pcdf.build_static_sdf(cuda(occ), grid)
        torch.cuda.synchronize()
        want = oracle.edt(occ)
        assert np.array_equal(sq.cpu().numpy(), want), (shape, density)
        assert np.array_equal(sdf.cpu().numpy().view(np.int32), oracle.sdf_from_sq(want, 0.05).view(np.int32))
    assert_clean(checked)


def edge_caps():
    return np.array([[[-40, 100, 0, -40, 100, 480, 90], [300, 300, 8, 300, 300, 16, 60],
                      [320, 300, 100, 420, 340, 300, 70]],
                     [[620, 560, 200, 640, 570, 470, 80], [100, 500, 470, 120, 520, 479, 10],
                      [330, 310, 110, 410, 330, 290, 75]]], np.int32)


def test_composite_scratch_and_query_checked(checked):
    grid = scenes.Grid(41, 37, 31, 0.05)
    rng = np.random.default_rng(5)
    occ, _ = scenes.boxes_occupancy(grid, 8, rng)
    cases = [edge_caps(), scenes.scene_small_walking(seed=3, T=4, H=2)["caps"]]
    for caps in cases:
        T = caps.shape[0]
        static_sq, static_sdf = pcdf.build_static_sdf(cuda(occ), grid)
        comp_sq, comp_sdf = pcdf.build_predicted_composite(static_sq, grid, caps, static_sdf=static_sdf)
        scr_sq, _ = pcdf.build_from_scratch(cuda(occ), grid, caps)
        torch.cuda.synchronize()
        S = oracle.edt(occ)
        assert np.array_equal(comp_sq.cpu().numpy(), oracle.predicted_composite(S, caps))
        for t in range(T):
            occ_t = np.maximum(occ, oracle.capsule_occupancy(grid.shape, caps[t]))
            assert np.array_equal(scr_sq[t].cpu().numpy(), oracle.edt(occ_t)), t
        sph = scenes.spheres_uniform(grid, 3000, rng)
        sph[::5, :3] += np.float32(0.4)  # some centres outside the grid
        tidx = rng.integers(-1, T + 2, 3000).astype(np.int32)
        h = pcdf.query_cost(comp_sdf, grid, cuda(sph), cuda(tidx), 0.2)
        gc, _ = pcdf.query_cost_backward(comp_sdf, grid, cuda(sph), cuda(tidx), 0.2, torch.ones(3000, device="cuda"))
        want, _ = oracle.hinge_cost(comp_sdf.cpu().numpy(), grid.origin, grid.vox, sph, tidx, 0.2)
        assert np.max(np.abs(h.cpu().numpy() - want)) <= 1e-5
        assert torch.isfinite(gc).all()
    assert_clean(checked)
