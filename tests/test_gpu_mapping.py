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


# nx a multiple of 4 takes the kernel that filters four voxels per thread
# (one warp per row of up to 128 voxels: 132 spans two warps, 4 is one word);
# the other widths take the byte kernel
@pytest.mark.parametrize("shape", [(64, 64, 64), (30, 17, 33), (40, 1, 1), (5, 9, 70), (1, 1, 1), (20, 260, 37),
                                   (33, 7, 132), (3, 70, 36), (17, 5, 4), (70, 9, 8)])
@pytest.mark.parametrize("k", [5, 0, 3, 27])
def test_voxel_filter_matches_oracle(shape, k):
    grid, occ = noisy(shape, seed=sum(shape) + k)
    got = pcdf.filter_voxels(cuda(occ), grid, k).cpu().numpy()
    assert np.array_equal(got, oracle.voxel_filter(occ, k))


def test_voxel_filter_any_nonzero_byte_is_occupied():
    """Occupancy bytes other than 0 and 1 (2, 7, 128, 255) count as occupied in
    both kernels; the output is 0/1."""
    for shape in ((21, 13, 48), (21, 13, 47)):
        grid, occ = noisy(shape, seed=77, density=0.05)
        rng = np.random.default_rng(5)
        vals = rng.choice(np.array([1, 2, 7, 128, 255], np.uint8), size=occ.shape)
        occ_v = (occ * vals).astype(np.uint8)
        got = pcdf.filter_voxels(cuda(occ_v), grid, 4).cpu().numpy()
        assert np.array_equal(got, oracle.voxel_filter(occ_v, 4)), shape


def test_voxel_filter_unaligned_map_takes_the_byte_kernel():
    grid, occ = noisy((12, 10, 64), seed=9, density=0.05)
    d = cuda(occ)
    flat = torch.zeros(occ.size + 1, dtype=torch.uint8, device=d.device)
    flat[1:].copy_(d.reshape(-1))
    view = flat[1:].view(occ.shape)  # starts one byte past an aligned address
    got = pcdf.filter_voxels(view, grid, 5).cpu().numpy()
    assert np.array_equal(got, oracle.voxel_filter(occ, 5))


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
