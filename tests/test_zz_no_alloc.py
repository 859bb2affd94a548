"""The allocation-free static-field entry point.

It is for callers that cannot allocate device memory when they need a field
(real-time loops that forbid allocation after start-up, hosts whose device
memory belongs to another runtime).  Called through the C ABI, it must give
the same fields as pcdf_build_static_sdf (bit for bit, as all integer and
float fields of this library) on two calls in a row, whatever the shared
scratch array holds from the call before, and a call after the first on a
device must leave the device's free memory and PyTorch's allocation count
unchanged.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

pcdf = pytest.importorskip("paper_2201_05058_gb300")
from paper_2201_05058_gb300 import _lib  # noqa: E402


def noalloc_into(occ, grid, sq, sdf):
    lib = _lib.load()
    g = _lib.PcdfGrid(grid.nx, grid.ny, grid.nz, grid.vox, (ctypes.c_float * 3)(*grid.origin))
    return lib.pcdf_build_static_sdf_noalloc(ctypes.byref(g), ctypes.c_void_p(occ.data_ptr()),
                                             ctypes.c_void_p(sq.data_ptr()), ctypes.c_void_p(sdf.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_workspace_build_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda", 0)
    rng = np.random.default_rng(0)
    cases = [scenes.scene_small(seed=1)["grid"], scenes.Grid(37, 45, 29, 0.05)]
    occs = [scenes.boxes_occupancy(cases[0], 10, rng)[0], scenes.random_occupancy(cases[1].shape, 0.05, rng)]
    for grid, occ_np in zip(cases, occs):
        occ = torch.from_numpy(occ_np).to(d)
        want_sq, want_sdf = pcdf.build_static_sdf(occ, grid)
        sq = torch.empty(occ.shape, dtype=torch.int32, device=d)
        sdf = torch.empty(occ.shape, dtype=torch.float32, device=d)
        for k in range(2):  # two calls in a row share the scratch array
            sq.fill_(7)
            sdf.fill_(7.0)
            torch.cuda.synchronize()
            free0, alloc0 = torch.cuda.mem_get_info(d)[0], torch.cuda.memory_allocated(d)
            rc = noalloc_into(occ, grid, sq, sdf)
            assert rc == 0, _lib.load().pcdf_last_error().decode()
            torch.cuda.synchronize()
            if k == 1:  # the first call on the device may load the library's module; later calls allocate nothing
                assert torch.cuda.mem_get_info(d)[0] == free0
                assert torch.cuda.memory_allocated(d) == alloc0
            assert torch.equal(sq, want_sq)
            assert torch.equal(sdf.view(torch.int32), want_sdf.view(torch.int32))


def test_noalloc_rejects_grids_beyond_the_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib.load()
    g = _lib.PcdfGrid(256, 128, 65, 0.05, (ctypes.c_float * 3)(0, 0, 0))  # 2,129,920 voxels
    fake = ctypes.c_void_p(256)  # never used: the size check fails first
    assert lib.pcdf_build_static_sdf_noalloc(ctypes.byref(g), fake, fake, None, None) == -1
    assert "exceeds" in lib.pcdf_last_error().decode()
