"""The static-map utilities of the mapping pipeline (Sec. 8) against the
oracle: the voxel filter bit for bit, the collapsed 2-D map and its EDT."""
import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu

pcdf = pytest.importorskip("paper_2201_05058_gb300")


def cuda(a):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def noisy(shape, seed, density=0.01):
    """Boxes plus isolated noise voxels and small clusters."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    grid = scenes.Grid(nx, ny, nz, 0.05)
    occ, _ = scenes.boxes_occupancy(grid, max(1, nx * ny * nz // 40000), rng)
    occ = occ | (rng.random(shape) < density).astype(np.uint8)
    return grid, occ


@pytest.mark.parametrize("shape", [(64, 64, 64), (30, 17, 33), (40, 1, 1), (5, 9, 70), (1, 1, 1), (20, 260, 37)])
@pytest.mark.parametrize("k", [5, 0, 3, 27])
def test_voxel_filter_matches_oracle(shape, k):
    grid, occ = noisy(shape, seed=sum(shape) + k)
    got = pcdf.filter_voxels(cuda(occ), grid, k).cpu().numpy()
    assert np.array_equal(got, oracle.voxel_filter(occ, k))


def test_voxel_filter_full_size_scene():
    sc = scenes.scene_composite(seed=2, T=1, H=1)
    rng = np.random.default_rng(3)
    occ = sc["occ"] | (rng.random(sc["occ"].shape) < 0.002).astype(np.uint8)
    got = pcdf.filter_voxels(cuda(occ), sc["grid"]).cpu().numpy()
    assert np.array_equal(got, oracle.voxel_filter(occ, 5))


def test_filter_rejects_bad_arguments():
    grid, occ = noisy((8, 8, 8), 1)
    d = cuda(occ)
    with pytest.raises(RuntimeError):
        pcdf.filter_voxels(d, grid, 28)
    with pytest.raises(RuntimeError):
        pcdf.filter_voxels(d, grid, 5, out=d)


@pytest.mark.parametrize("z0,z1", [(0, 64), (0, 36), (10, 11), (-4, 7), (50, 99), (20, 20), (30, 10)])
def test_collapse_and_2d_edt(z0, z1):
    sc = scenes.scene_small(seed=4)
    grid, occ = sc["grid"], sc["occ"]
    c = pcdf.collapse_2d(cuda(occ), grid, z0, z1).cpu().numpy()
    want = oracle.collapse(occ, z0, z1)
    assert np.array_equal(c, want)
    sq, sdf = pcdf.edt_2d(cuda(occ), grid, z0, z1)
    S = oracle.edt(want[None])[0]
    assert np.array_equal(sq.cpu().numpy(), S)
    assert np.array_equal(sdf.cpu().numpy().view(np.uint32), oracle.sdf_from_sq(S, grid.vox).view(np.uint32))
