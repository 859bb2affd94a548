"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer fields (signed squared EDT, composite) and the float fields derived
from them must match bit for bit.  The hinge cost must match the fp64 oracle
within 1e-5 m and its gradient within 1e-4, away from the hinge kink and the
cell faces where the derivative jumps.
"""
import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu

pcdf = pytest.importorskip("paper_2201_05058_gb300")

COST_TOL = 1e-5
GRAD_TOL = 1e-4


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def gpu_static(occ, grid):
    sq, sdf = pcdf.build_static_sdf(cuda(occ), grid)
    return sq.cpu().numpy(), sdf.cpu().numpy()


def assert_equal_fields(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        i = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {i}: got {got[i]} want {want[i]}")


def assert_bits_equal(got, want, what):
    assert_equal_fields(got.view(np.int32), want.view(np.int32), what)


# ---------------------------------------------------------------------------
# static signed EDT
# ---------------------------------------------------------------------------

SMALL_SHAPES = [(16, 16, 16), (13, 17, 15), (23, 29, 37), (1, 1, 40), (40, 1, 1), (1, 37, 1), (3, 2, 70),
                (2, 5, 512), (33, 7, 65)]


@pytest.mark.parametrize("shape", SMALL_SHAPES)
@pytest.mark.parametrize("density", [0.0, 0.002, 0.05, 0.3, 0.9, 1.0])
def test_static_edt_matches_definition(shape, density):
    rng = np.random.default_rng(hash((shape, density)) % 2 ** 32)
    occ = scenes.random_occupancy(shape, density, rng)
    grid = scenes.Grid(shape[2], shape[1], shape[0], 0.05)
    sq, sdf = gpu_static(occ, grid)
    want = oracle.edt_brute(occ) if occ.size <= 40000 else oracle.edt(occ)
    assert_equal_fields(sq, want, "static_sq")
    assert_bits_equal(sdf, oracle.sdf_from_sq(want, grid.vox), "static_sdf")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_static_edt_small_scene(seed):
    sc = scenes.scene_small(seed=seed)
    grid = sc["grid"]
    sq, sdf = gpu_static(sc["occ"], grid)
    want = oracle.edt(sc["occ"])
    assert_equal_fields(sq, want, "static_sq")
    assert_bits_equal(sdf, oracle.sdf_from_sq(want, grid.vox), "static_sdf")


def test_static_edt_box_and_wall_structures():
    # walls produce full-depth envelopes; a hollow box produces interior runs
    shape = (48, 50, 66)
    occ = np.zeros(shape, np.uint8)
    occ[:, :, 40] = 1
    occ[10:30, 5:45, 3:20] = 1
    occ[12:28, 7:43, 5:18] = 0
    occ[:, 25, :] |= (np.arange(66) % 3 == 0).astype(np.uint8)
    grid = scenes.Grid(66, 50, 48, 0.04)
    sq, _ = gpu_static(occ, grid)
    assert_equal_fields(sq, oracle.edt(occ), "static_sq")


# ---------------------------------------------------------------------------
# composite fields
# ---------------------------------------------------------------------------

def check_composite(occ, caps, grid):
    """Every output variant against the oracle: the static float field reused
    or recomputed, the int32 field with or without the float field, the
    float field alone."""
    static_sq, static_sdf = pcdf.build_static_sdf(cuda(occ), grid)
    want = oracle.predicted_composite(oracle.edt(occ), caps)
    out = None
    for reuse, want_sq, want_sdf in ((False, True, True), (True, True, True), (True, False, True),
                                     (False, True, False)):
        comp_sq, comp_sdf = pcdf.build_predicted_composite(static_sq, grid, caps, want_sq=want_sq, want_sdf=want_sdf,
                                                           static_sdf=static_sdf if reuse else None)
        for t in range(caps.shape[0]):
            if want_sq:
                assert_equal_fields(comp_sq[t].cpu().numpy(), want[t], f"comp_sq[{t}] reuse={reuse}")
            if want_sdf:
                assert_bits_equal(comp_sdf[t].cpu().numpy(), oracle.sdf_from_sq(want[t], grid.vox),
                                  f"comp_sdf[{t}] reuse={reuse}")
        if want_sq:
            out = comp_sq.cpu().numpy()
    return out


@pytest.mark.parametrize("seed", [0, 5])
def test_composite_small_scene_one_human(seed):
    sc = scenes.scene_small(seed=seed, T=1)
    check_composite(sc["occ"], sc["caps"], sc["grid"])


@pytest.mark.parametrize("H,T", [(1, 5), (2, 7), (4, 3)])
def test_composite_walking_humans(H, T):
    sc = scenes.scene_small_walking(seed=10 + H, T=T, H=H)
    check_composite(sc["occ"], sc["caps"], sc["grid"])


def test_composite_ragged_grid_and_edge_capsules():
    grid = scenes.Grid(45, 70, 37, 0.05)
    rng = np.random.default_rng(3)
    occ, _ = scenes.boxes_occupancy(grid, 8, rng)
    caps = np.array([
        [[0, 0, 80, 0, 0, 400, 100], [700, 1100, -50, 760, 1150, 300, 60]],      # corner, below floor
        [[-300, 500, 100, -100, 500, 500, 120], [400, 400, 580, 400, 400, 590, 30]],  # partly outside; near top
        [[104, 104, 104, 104, 104, 104, 0], [296, 296, 296, 504, 296, 296, 0]],   # r = 0: on-centre points only
    ], np.int32)
    check_composite(occ, caps, grid)


def test_composite_slab_map_dedup_and_its_limits():
    """Slab slices of equal capsule cross-sections are computed once and read
    through a map.  Upright capsules and a cylinder (deduplicated) mixed with
    a slanted capsule (a key of its own in every slice it touches), then the
    two limits where the map falls back to the identity: more than 255 slab
    slices, and more than 4096 (t, slice) entries."""
    grid = scenes.Grid(20, 18, 80, 0.05)
    rng = np.random.default_rng(21)
    occ, _ = scenes.boxes_occupancy(grid, 4, rng)
    T = 3
    caps = np.zeros((T, 3, 7), np.int32)
    for t in range(T):
        caps[t, 0] = [40 + 16 * t, 150, 90, 40 + 16 * t, 150, 900, 60]            # upright capsule
        caps[t, 1] = [200, 60 + 8 * t, 200, 200, 60 + 8 * t, 700, 50 | pcdf.CYLINDER]  # upright cylinder
        caps[t, 2] = [100, 100, 300 + 20 * t, 260, 220, 600, 40]                   # slanted
    check_composite(occ, caps, grid)
    # a slab of more than 255 slices: 8 x 8 x 300 voxels, one capsule over the whole height
    tall = scenes.Grid(8, 8, 300, 0.05)
    occ_t = np.zeros(tall.shape, np.uint8)
    occ_t[10:20, 2:4, 1:3] = 1
    caps_t = np.array([[[56, 56, 40, 56, 56, 4700, 30]], [[72, 56, 40, 72, 56, 4700, 30]]], np.int32)
    check_composite(occ_t, caps_t, tall)
    # more than 4096 (t, slice) entries: T = 24 over a 180-slice slab
    mid = scenes.Grid(8, 8, 200, 0.05)
    occ_m = np.zeros(mid.shape, np.uint8)
    occ_m[5:9, 1:3, 4:6] = 1
    caps_m = np.array([[[40 + (t % 4) * 8, 64, 100, 40 + (t % 4) * 8, 64, 2900, 40]] for t in range(24)], np.int32)
    check_composite(occ_m, caps_m, mid)


def test_composite_tall_slab_narrow_ctas():
    """A slab of more than 400 slices leaves shared memory for 64 columns per
    CTA of the z stage: with 96 columns per slice the second CTA of each t has
    32 live columns, and each CTA prefetches its own part of the static planes
    into L2 (16-byte aligned outputs)."""
    grid = scenes.Grid(12, 8, 512, 0.05)
    occ = np.zeros(grid.shape, np.uint8)
    occ[100:140, 2:5, 1:4] = 1
    occ[300:310, :, 9] = 1
    caps = np.array([[[96, 64, 168, 96, 64, 7048, 24]], [[112, 64, 168, 112, 64, 7048, 24]]], np.int32)
    check_composite(occ, caps, grid)


def test_composite_odd_slice_size():
    # nx * ny not a multiple of 4: all-static column blocks are copied one
    # column per thread instead of with 16-byte accesses
    grid = scenes.Grid(33, 17, 30, 0.05)
    rng = np.random.default_rng(8)
    occ, _ = scenes.boxes_occupancy(grid, 5, rng)
    caps = scenes.walking_capsules(grid, 2, 3, rng)
    check_composite(occ, caps, grid)


def test_composite_unaligned_outputs_and_far_humans():
    """Outputs that start 4 bytes past a 16-byte boundary take the per-column
    copies of the static planes; aligned outputs take the 16-byte block
    copies.  A human in one corner of a wide room leaves most column blocks
    all-static, so the copies carry most of the field."""
    grid = scenes.Grid(96, 80, 40, 0.05)
    rng = np.random.default_rng(21)
    occ, _ = scenes.boxes_occupancy(grid, 6, rng)
    caps = np.array([[[160, 160, 60, 160, 160, 500, 70]],
                     [[240, 200, 60, 250, 220, 500, 70]]], np.int32)
    static_sq, static_sdf = pcdf.build_static_sdf(cuda(occ), grid)
    want = oracle.predicted_composite(oracle.edt(occ), caps)
    T, n = caps.shape[0], grid.nvox
    ws = pcdf.composite_workspace(grid, caps, static_sq.device)
    for reuse in (False, True):
        buf_sq = torch.zeros(T * n + 1, dtype=torch.int32, device=static_sq.device)
        buf_sdf = torch.zeros(T * n + 1, dtype=torch.float32, device=static_sq.device)
        comp_sq = buf_sq[1:].view((T,) + grid.shape)
        comp_sdf = buf_sdf[1:].view((T,) + grid.shape)
        pcdf.composite_prepare(grid, caps, ws)
        pcdf.composite_finish(static_sq, grid, caps, ws, comp_sq, comp_sdf, static_sdf=static_sdf if reuse else None)
        for t in range(T):
            assert_equal_fields(comp_sq[t].cpu().numpy(), want[t], f"comp_sq[{t}] unaligned")
            assert_bits_equal(comp_sdf[t].cpu().numpy(), oracle.sdf_from_sq(want[t], grid.vox),
                              f"comp_sdf[{t}] unaligned")
    # aligned outputs: 16-byte copies of the all-static planes
    comp_sq = torch.empty((T,) + grid.shape, dtype=torch.int32, device=static_sq.device)
    comp_sdf = torch.empty((T,) + grid.shape, dtype=torch.float32, device=static_sq.device)
    pcdf.composite_prepare(grid, caps, ws)
    pcdf.composite_finish(static_sq, grid, caps, ws, comp_sq, comp_sdf, static_sdf=static_sdf)
    for t in range(T):
        assert_equal_fields(comp_sq[t].cpu().numpy(), want[t], f"comp_sq[{t}] aligned")
        assert_bits_equal(comp_sdf[t].cpu().numpy(), oracle.sdf_from_sq(want[t], grid.vox), f"comp_sdf[{t}] aligned")
    check_composite(occ, caps, grid)


def test_composite_no_humans_and_humans_outside():
    sc = scenes.scene_small(seed=1)
    grid = sc["grid"]
    static_sq, _ = pcdf.build_static_sdf(cuda(sc["occ"]), grid)
    want = oracle.edt(sc["occ"])
    sq, sdf = pcdf.build_predicted_composite(static_sq, grid, np.zeros((3, 0, 7), np.int32))
    for t in range(3):
        assert_equal_fields(sq[t].cpu().numpy(), want, "H=0")
    far = np.array([[[-8000, -8000, -8000, -8000, -8000, -7000, 80]]] * 2, np.int32)
    sq, sdf = pcdf.build_predicted_composite(static_sq, grid, far)
    assert_equal_fields(sq[1].cpu().numpy(), want, "outside")
    assert_bits_equal(sdf[1].cpu().numpy(), oracle.sdf_from_sq(want, grid.vox), "outside sdf")


def test_composite_degenerate_maps():
    grid = scenes.Grid(20, 18, 22, 0.05)
    caps = np.array([[[160, 144, 80, 160, 144, 200, 48]]], np.int32)
    # empty static map: composite = dynamic field alone
    check_composite(np.zeros(grid.shape, np.uint8), caps, grid)
    # capsule covering the whole grid: no free voxel anywhere at that t
    big = np.array([[[160, 144, 176, 160, 144, 176, 8000]]], np.int32)
    comp = check_composite(scenes.random_occupancy(grid.shape, 0.1, np.random.default_rng(0)), big, grid)
    assert np.all(comp == -oracle.INF32)
    # static map with no free voxel: every column maximum is -INF, every
    # column a copy of the static field
    comp = check_composite(np.ones(grid.shape, np.uint8), caps, grid)
    assert np.all(comp == -oracle.INF32)


def test_from_scratch_matches_oracle_and_composite_invariant():
    sc = scenes.scene_small_walking(seed=21, T=4, H=2)
    occ, caps, grid = sc["occ"], sc["caps"], sc["grid"]
    sq, sdf = pcdf.build_from_scratch(cuda(occ), grid, caps)
    sq = sq.cpu().numpy()
    want = oracle.from_scratch(occ, caps)
    for t in range(caps.shape[0]):
        assert_equal_fields(sq[t], want[t], f"scratch[{t}]")
        assert_bits_equal(sdf[t].cpu().numpy(), oracle.sdf_from_sq(want[t], grid.vox), f"scratch sdf[{t}]")
    static_sq, _ = pcdf.build_static_sdf(cuda(occ), grid)
    comp, _ = pcdf.build_predicted_composite(static_sq, grid, caps)
    comp = comp.cpu().numpy()
    for t in range(caps.shape[0]):
        free = (occ == 0) & (oracle.capsule_occupancy(occ.shape, caps[t]) == 0)
        assert np.array_equal(comp[t][free], sq[t][free])


# ---------------------------------------------------------------------------
# full-size workload: 256^3, 60 boxes, 3 walking humans, T = 20
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big_scene():
    sc = scenes.scene_composite(seed=0)
    grid = sc["grid"]
    static_sq, static_sdf = pcdf.build_static_sdf(cuda(sc["occ"]), grid)
    comp_sq, comp_sdf = pcdf.build_predicted_composite(static_sq, grid, sc["caps"], static_sdf=static_sdf)
    # the benchmark's one-call update (its static z pass also writes the column maxima of the z stage)
    up = pcdf.predicted_fields(cuda(sc["occ"]), grid, sc["caps"])
    torch.cuda.synchronize()
    return sc, static_sq.cpu().numpy(), static_sdf.cpu().numpy(), comp_sq, comp_sdf, up


def test_full_size_static_matches_oracle(big_scene):
    sc, static_sq, static_sdf, _, _, up = big_scene
    want = oracle.edt(sc["occ"])
    assert_equal_fields(static_sq, want, "static_sq 256^3")
    assert_bits_equal(static_sdf, oracle.sdf_from_sq(want, sc["grid"].vox), "static_sdf 256^3")
    assert_equal_fields(up[0].cpu().numpy(), want, "update static_sq 256^3")
    assert_bits_equal(up[1].cpu().numpy(), oracle.sdf_from_sq(want, sc["grid"].vox), "update static_sdf 256^3")
    # and against the definition at sampled voxels
    rng = np.random.default_rng(0)
    for _ in range(60):
        k, j, i = (int(rng.integers(0, 256)) for _ in range(3))
        assert static_sq[k, j, i] == oracle.edt_at(sc["occ"], i, j, k)


@pytest.mark.parametrize("t", [0, 9, 19])
def test_full_size_composite_matches_oracle(big_scene, t):
    sc, _, _, comp_sq, comp_sdf, up = big_scene
    grid = sc["grid"]
    S_static = oracle.edt(sc["occ"])
    dyn_occ = oracle.capsule_occupancy(grid.shape, sc["caps"][t])
    want = oracle.composite(S_static, oracle.edt(dyn_occ))
    got = comp_sq[t].cpu().numpy()
    want_sdf = oracle.sdf_from_sq(want, grid.vox)
    assert_equal_fields(got, want, f"comp_sq[{t}] 256^3")
    assert_bits_equal(comp_sdf[t].cpu().numpy(), want_sdf, f"comp_sdf[{t}] 256^3")
    assert_equal_fields(up[2][t].cpu().numpy(), want, f"update comp_sq[{t}] 256^3")
    assert_bits_equal(up[3][t].cpu().numpy(), want_sdf, f"update comp_sdf[{t}] 256^3")
    # sampled against the definition, biased towards the humans
    rng = np.random.default_rng(t)
    occ_pts = np.argwhere(dyn_occ)
    for q in range(30):
        if q % 2 == 0 and len(occ_pts):
            k, j, i = occ_pts[rng.integers(0, len(occ_pts))] + rng.integers(-3, 4, 3)
            k, j, i = (int(np.clip(v, 0, 255)) for v in (k, j, i))
        else:
            k, j, i = (int(rng.integers(0, 256)) for _ in range(3))
        w = min(oracle.edt_at(sc["occ"], i, j, k), oracle.edt_at(dyn_occ, i, j, k))
        assert got[k, j, i] == w


# ---------------------------------------------------------------------------
# hinge cost and gradient
# ---------------------------------------------------------------------------

def oracle_distance(sdf, grid, sph, tidx):
    """The oracle's interpolated distance d (from its hinge with a huge eps)."""
    big = 1.0e4
    h, _ = oracle.hinge_cost(sdf, grid.origin, grid.vox, sph, tidx, big)
    return big + sph[:, 3].astype(np.float64) - h


def near_face_or_kink(sph, grid, d_oracle, eps, margin_u=1e-3, margin_h=1e-5):
    """Samples where fp32 and fp64 may legitimately disagree on the derivative:
    within margin_u (voxels) of a cell face, or within margin_h (m) of the kink."""
    u = (sph[:, :3].astype(np.float64) - np.asarray(grid.origin)) / grid.vox - 0.5
    face = np.any(np.abs(u - np.rint(u)) < margin_u, axis=1)
    kink = np.abs(eps + sph[:, 3].astype(np.float64) - d_oracle) < margin_h
    return face | kink


@pytest.mark.parametrize("seed", [0, 1])
def test_query_cost_small_scene(seed):
    sc = scenes.scene_small(seed=seed, T=1)
    grid = sc["grid"]
    static_sq, _ = pcdf.build_static_sdf(cuda(sc["occ"]), grid)
    _, comp_sdf = pcdf.build_predicted_composite(static_sq, grid, sc["caps"], want_sq=False)
    sph = sc["spheres"].copy()
    sph[::7, :3] += np.float32(0.3)   # some centres outside the grid
    sph[1::7, :3] -= np.float32(0.2)
    h, oob = pcdf.query_cost(comp_sdf, grid, cuda(sph), cuda(sc["tidx"]), sc["eps"], count_oob=True)
    want, want_oob = oracle.hinge_cost(comp_sdf.cpu().numpy(), grid.origin, grid.vox, sph, sc["tidx"], sc["eps"])
    assert np.max(np.abs(h.cpu().numpy() - want)) <= COST_TOL
    assert int(oob.item()) == want_oob
    assert want_oob > 0 and (want > 0).sum() > 10


def test_query_cost_and_gradient_trajectories():
    """[256 trajectories, 40 support states, 30 spheres] on T = 20 composite
    fields of a 64^3 scene; tidx = min(state, 19)."""
    sc = scenes.scene_small_walking(seed=4, T=20, H=1)
    grid = sc["grid"]
    static_sq, _ = pcdf.build_static_sdf(cuda(sc["occ"]), grid)
    _, comp_sdf = pcdf.build_predicted_composite(static_sq, grid, sc["caps"], want_sq=False)
    rng = np.random.default_rng(44)
    sph, tidx = scenes.spheres_along_paths(grid, 256, 40, 30, rng, T=20)
    sph_f = sph.reshape(-1, 4)
    tid_f = tidx.reshape(-1)
    h = pcdf.query_cost(comp_sdf, grid, cuda(sph), cuda(tidx), 0.2).cpu().numpy().reshape(-1)
    sdf_np = comp_sdf.cpu().numpy()
    want, _, gc, gr = oracle.hinge_cost(sdf_np, grid.origin, grid.vox, sph_f, tid_f, 0.2, need_grad=True)
    assert np.max(np.abs(h - want)) <= COST_TOL
    g_h = rng.normal(size=tid_f.shape).astype(np.float32)
    got_c, got_r = pcdf.query_cost_backward(comp_sdf, grid, cuda(sph), cuda(tidx), 0.2, cuda(g_h.reshape(tidx.shape)))
    got_c = got_c.cpu().numpy().reshape(-1, 3)
    got_r = got_r.cpu().numpy().reshape(-1)
    skip = near_face_or_kink(sph_f, grid, oracle_distance(sdf_np, grid, sph_f, tid_f), 0.2)
    keep = ~skip
    assert keep.mean() > 0.95
    want_c = gc * g_h[:, None].astype(np.float64)
    want_r = gr * g_h.astype(np.float64)
    assert np.max(np.abs(got_c[keep] - want_c[keep])) <= GRAD_TOL
    assert np.max(np.abs(got_r[keep] - want_r[keep])) <= GRAD_TOL
    assert (gr > 0).sum() > 1000


def test_hinge_autograd_function():
    sc = scenes.scene_small(seed=6, T=1, n_spheres=2048)
    grid = sc["grid"]
    static_sq, _ = pcdf.build_static_sdf(cuda(sc["occ"]), grid)
    _, sdf = pcdf.build_predicted_composite(static_sq, grid, sc["caps"], want_sq=False)
    sph = sc["spheres"].copy()
    sph[:, 3] = 0.5
    centres = cuda(sph[:, :3]).requires_grad_(True)
    radii = cuda(sph[:, 3]).requires_grad_(True)
    tidx = cuda(sc["tidx"])
    h = pcdf.hinge_cost(centres, radii, sdf, tidx, 0.2, grid)
    loss = (h * h).sum()
    loss.backward()
    want, _, gc, gr = oracle.hinge_cost(sdf.detach().cpu().numpy(), grid.origin, grid.vox, sph, sc["tidx"], 0.2,
                                        need_grad=True)
    up = 2.0 * want
    keep = ~near_face_or_kink(sph, grid, oracle_distance(sdf.detach().cpu().numpy(), grid, sph, sc["tidx"]), 0.2)
    gcn = centres.grad.cpu().numpy()
    assert np.max(np.abs(gcn[keep] - (gc * up[:, None])[keep])) <= 10 * GRAD_TOL
    assert np.max(np.abs(radii.grad.cpu().numpy()[keep] - (gr * up)[keep])) <= 10 * GRAD_TOL
    # fp32 central differences on the GPU (reported, loosely bounded: error ~ ulp / step)
    step = 1e-3
    # the difference interval must not cross a cell face (the derivative jumps there)
    u = sph[:, :3].astype(np.float64) / grid.vox - 0.5
    clear = np.all(np.abs(u - np.rint(u)) > 2 * step / grid.vox, axis=1)
    idx = np.nonzero(keep & clear & (want > 0.05))[0][:64]
    for a in range(3):
        cp = centres.detach().clone()
        cm = centres.detach().clone()
        cp[idx, a] += step
        cm[idx, a] -= step
        hp = pcdf.hinge_cost(cp, radii.detach(), sdf, tidx, 0.2, grid)
        hm = pcdf.hinge_cost(cm, radii.detach(), sdf, tidx, 0.2, grid)
        fd = ((hp * hp - hm * hm) / (2 * step)).cpu().numpy()[idx]
        assert np.max(np.abs(fd - gcn[idx, a])) < 0.05


def test_query_edge_cases():
    grid = scenes.Grid(1, 5, 7, 0.1)  # single-voxel x axis
    occ = np.zeros(grid.shape, np.uint8)
    occ[3, 2, 0] = 1
    sq, sdf = pcdf.build_static_sdf(cuda(occ), grid)
    sph = np.array([[0.05, 0.25, 0.35, 0.1], [0.3, 0.21, 0.33, 0.05], [np.nan, 0.2, 0.3, 0.1]], np.float32)
    tid = np.array([0, 3, -1], np.int32)
    h, oob = pcdf.query_cost(sdf, grid, cuda(sph), cuda(tid), 0.2, count_oob=True)
    want, want_oob = oracle.hinge_cost(sdf.cpu().numpy(), grid.origin, grid.vox, sph, tid, 0.2)
    assert np.max(np.abs(h.cpu().numpy() - want)) <= COST_TOL
    assert int(oob.item()) == want_oob
    # N = 0
    h0 = pcdf.query_cost(sdf, grid, cuda(np.zeros((0, 4), np.float32)), cuda(np.zeros(0, np.int32)), 0.2)
    assert h0.numel() == 0
    # infinite fields: empty map -> h = 0; full map -> h = inf
    for fill, expect in ((0, 0.0), (1, np.inf)):
        s2, f2 = pcdf.build_static_sdf(cuda(np.full(grid.shape, fill, np.uint8)), grid)
        hh = pcdf.query_cost(f2, grid, cuda(sph[:2]), cuda(tid[:2]), 0.2).cpu().numpy()
        assert np.all(hh == expect)


def test_predicted_fields_overlapped_and_graph_captured():
    """The one-call update (pcdf_update_fields: capsule x+y pass on a side
    stream beside the static build) equals the oracle, also when captured in a
    CUDA graph and replayed on a new occupancy in the same buffers."""
    sc = scenes.scene_small_walking(seed=31, T=6, H=2)
    grid, caps = sc["grid"], sc["caps"]
    d = torch.device("cuda", 0)
    occ = cuda(sc["occ"])
    st_sq, st_sdf, sq, sdf = pcdf.predicted_fields(occ, grid, caps)
    want = oracle.predicted_composite(oracle.edt(sc["occ"]), caps)
    for t in range(caps.shape[0]):
        assert_equal_fields(sq[t].cpu().numpy(), want[t], f"comp_sq[{t}]")
        assert_bits_equal(sdf[t].cpu().numpy(), oracle.sdf_from_sq(want[t], grid.vox), f"comp_sdf[{t}]")
    assert_equal_fields(st_sq.cpu().numpy(), oracle.edt(sc["occ"]), "static")
    ws = pcdf.update_workspace(grid, caps, d)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(device=d)
    s.wait_stream(torch.cuda.current_stream(d))
    with torch.cuda.stream(s):
        pcdf.predicted_fields(occ, grid, caps, workspace=ws, out_static_sq=st_sq, out_static_sdf=st_sdf,
                              out_sq=sq, out_sdf=sdf)  # warm-up outside the capture
        with torch.cuda.graph(g, stream=s):
            pcdf.predicted_fields(occ, grid, caps, workspace=ws, out_static_sq=st_sq, out_static_sdf=st_sdf,
                                  out_sq=sq, out_sdf=sdf)
    torch.cuda.current_stream(d).wait_stream(s)
    occ2 = scenes.scene_small_walking(seed=32, T=6, H=2)["occ"]
    occ.copy_(cuda(occ2))
    sq.zero_()
    g.replay()
    torch.cuda.synchronize()
    want2 = oracle.predicted_composite(oracle.edt(occ2), caps)
    for t in range(caps.shape[0]):
        assert_equal_fields(sq[t].cpu().numpy(), want2[t], f"replayed comp_sq[{t}]")


def test_update_to_host_chunks_equal_the_oracle():
    """Host buffers in and out, fields copied in chunks while later ones are
    computed; also a chunk size that does not divide T."""
    sc = scenes.scene_small_walking(seed=33, T=7, H=2)
    grid, caps = sc["grid"], sc["caps"]
    d = torch.device("cuda", 0)
    T = caps.shape[0]
    bufs = {"occ": torch.empty(grid.shape, dtype=torch.uint8, device=d),
            "static_sq": torch.empty(grid.shape, dtype=torch.int32, device=d),
            "static_sdf": torch.empty(grid.shape, dtype=torch.float32, device=d),
            "comp_sdf": torch.empty((T,) + grid.shape, dtype=torch.float32, device=d),
            "workspace": pcdf.composite_workspace(grid, caps, d)}
    occ_h = torch.from_numpy(sc["occ"]).pin_memory()
    want = oracle.predicted_composite(oracle.edt(sc["occ"]), caps)
    for chunk in (3, 7):
        out_h = torch.full((T,) + grid.shape, float("nan"), dtype=torch.float32).pin_memory()
        pcdf.update_to_host(occ_h, grid, caps, out_h, bufs, chunk=chunk)
        torch.cuda.synchronize()
        for t in range(T):
            assert_bits_equal(out_h[t].numpy(), oracle.sdf_from_sq(want[t], grid.vox), f"host field {t}")


def test_cylinders_and_growing_radius():
    """The paper's primitive (finite cylinder), mixed with capsules, with a
    radius that grows over the horizon; composite, from-scratch and the
    batched kernel against the oracle."""
    grid = scenes.Grid(48, 44, 40, 0.05)
    rng = np.random.default_rng(17)
    occ, _ = scenes.boxes_occupancy(grid, 6, rng)
    T = 5
    a = np.array([[0.8 + 0.1 * t, 0.9, 0.25] for t in range(T)])
    b = a + np.array([0.0, 0.0, 1.3])
    r = 0.25 + 0.03 * np.arange(T)           # growing over the horizon
    cyl = pcdf.capsule_fixed(a, b, r, grid, cylinder=True)
    slanted = pcdf.capsule_fixed(a + [1.0, 0.7, 0.1], b + [1.3, 0.9, 0.0], r, grid, cylinder=True)
    capsule = pcdf.capsule_fixed(a + [0.2, 1.2, 0.0], b + [0.2, 1.2, 0.0], r, grid)
    caps = np.stack([cyl, slanted, capsule], axis=1)            # [T][3][7]
    assert np.all(caps[:, :2, 6] & pcdf.CYLINDER)
    check_composite(occ, caps, grid)
    sq, _ = pcdf.build_from_scratch(cuda(occ), grid, caps, want_sdf=False)
    want = oracle.from_scratch(occ, caps)
    for t in range(T):
        assert_equal_fields(sq[t].cpu().numpy(), want[t], f"scratch[{t}]")
    b = pcdf.Batch([(grid, cuda(occ), caps)])
    b.run()
    assert b.error() == 0
    comp = oracle.predicted_composite(oracle.edt(occ), caps)
    assert np.array_equal(b.comp_sq[0].cpu().numpy(), comp)
    b.close()
    # the surrogate models capsules only
    d = torch.device("cuda", 0)
    static_sq, static_sdf = pcdf.build_static_sdf(cuda(occ), grid)
    sph = torch.from_numpy(scenes.spheres_uniform(grid, 64, rng)).to(d)
    tidx = torch.zeros(64, dtype=torch.int32, device=d)
    y = torch.zeros(64 * 3, dtype=torch.float32, device=d)
    with pytest.raises(RuntimeError):
        pcdf.surrogate_finish(grid, static_sq, static_sdf, sph, tidx, T, caps, y, 0.2, 0.1)
