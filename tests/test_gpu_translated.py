"""GPU parity of the translated primitive field (Sec. 6: the field of the human
primitive is computed once and composited at each predicted position) through
the C ABI, against the CPU oracle.

The template is an exact signed EDT and the translated composite a per-voxel
min, so both are compared bit for bit (int32 and the fp32 field).  At the
256^3 workload the translated composite is also checked against the exact
composite path on lattice-moved humans, where the two must agree everywhere.
"""
import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu

pcdf = pytest.importorskip("paper_2201_05058_gb300")

CYL = oracle.CYLINDER

PRIMS = [
    np.array([40, 56, 30, 40, 56, 90, 20], np.int32),          # upright capsule
    np.array([10, 30, 20, 70, 50, 60, 17], np.int32),          # slanted capsule
    np.array([40, 40, 10, 40, 40, 70, 18 | CYL], np.int32),    # upright cylinder
    np.array([24, 40, 8, 60, 28, 100, 21 | CYL], np.int32),    # slanted cylinder
    np.array([100, 100, 100, 100, 100, 100, 40], np.int32),    # sphere (a = b)
    np.array([24, 24, 24, 24, 24, 24, 3], np.int32),           # a single voxel centre
]


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def assert_equal_fields(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        i = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {i}: got {got[i]} want {want[i]}")


def assert_bits_equal(got, want, what):
    assert_equal_fields(got.view(np.int32), want.view(np.int32), what)


@pytest.mark.parametrize("ci", range(len(PRIMS)))
@pytest.mark.parametrize("R", [0, 3, 9])
def test_template_matches_oracle(ci, R):
    cap = PRIMS[ci]
    tmpl, lo = pcdf.build_template(cap, R, dev())
    torch.cuda.synchronize()
    want, wlo = oracle.template_field(cap, R)
    assert lo == list(wlo)
    assert_equal_fields(tmpl.cpu().numpy(), want, "template")


def box_static(shape, seed, n_boxes=6):
    rng = np.random.default_rng(seed)
    occ = np.zeros(shape, np.uint8)
    for _ in range(n_boxes):
        lo = [int(rng.integers(0, n)) for n in shape]
        hi = [min(lo[q] + int(rng.integers(1, 5)), shape[q]) for q in range(3)]
        occ[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = 1
    return occ


def random_placements(rng, T, H, dims, shape):
    nz, ny, nx = shape
    lo = np.empty((T, H, 3), np.int32)
    for a, n in enumerate((nx, ny, nz)):
        lo[..., a] = rng.integers(-dims[a] - 2, n + 2, (T, H))   # some boxes partly or wholly outside
    return lo


@pytest.mark.parametrize("shape", [(20, 18, 22), (24, 20, 32), (9, 33, 17), (1, 6, 40)])
@pytest.mark.parametrize("outputs", ["both", "both_no_static_sdf", "sq", "sdf"])
def test_translated_composite_matches_oracle(shape, outputs):
    rng = np.random.default_rng(hash((shape, outputs)) % 2 ** 32)
    occ = box_static(shape, rng.integers(1 << 30))
    grid = scenes.Grid(shape[2], shape[1], shape[0], 0.05)
    S = oracle.edt(occ)
    sq, sdf = pcdf.build_static_sdf(cuda(occ), grid)
    cap = PRIMS[1]
    R = 4
    tmpl, lo0 = pcdf.build_template(cap, R, dev())
    want_t, _ = oracle.template_field(cap, R)
    T, H = 5, 3
    lo = random_placements(rng, T, H, list(tmpl.shape[::-1]), shape)
    lo[0, 0] = lo0                   # the primitive where cap puts it
    got_sq, got_sdf = pcdf.composite_translated(
        sq, grid, tmpl, lo, R, static_sdf=sdf if outputs == "both" or outputs == "sdf" else None,
        want_sq=outputs != "sdf", want_sdf=outputs != "sq")
    torch.cuda.synchronize()
    want = oracle.translated_composite(S, want_t, lo)
    if outputs != "sdf":
        assert_equal_fields(got_sq.cpu().numpy(), want, "comp_sq")
    else:
        assert got_sq is None
    if outputs != "sq":
        assert_bits_equal(got_sdf.cpu().numpy(), oracle.sdf_from_sq(want, grid.vox), "comp_sdf")
    else:
        assert got_sdf is None


def test_translated_composite_without_primitives_is_the_static_field():
    shape = (12, 10, 16)
    occ = box_static(shape, 5)
    grid = scenes.Grid(shape[2], shape[1], shape[0], 0.05)
    sq, sdf = pcdf.build_static_sdf(cuda(occ), grid)
    tmpl = torch.zeros((1, 1, 1), dtype=torch.int32, device=dev())
    got_sq, got_sdf = pcdf.composite_translated(sq, grid, tmpl, np.zeros((3, 0, 3), np.int32), 0,
                                                static_sdf=sdf)
    torch.cuda.synchronize()
    for t in range(3):
        assert torch.equal(got_sq[t], sq)
        assert torch.equal(got_sdf[t].view(torch.int32), sdf.view(torch.int32))


def test_translated_composite_many_time_steps_over_several_launches():
    """T * H above one launch's placement table (1536 entries): the time steps
    are split over launches and every output is still written."""
    shape = (6, 8, 12)
    rng = np.random.default_rng(9)
    occ = box_static(shape, 9, n_boxes=3)
    grid = scenes.Grid(shape[2], shape[1], shape[0], 0.05)
    S = oracle.edt(occ)
    sq, _ = pcdf.build_static_sdf(cuda(occ), grid)
    cap = PRIMS[0]
    tmpl, _ = pcdf.build_template(cap, 2, dev())
    want_t, _ = oracle.template_field(cap, 2)
    T, H = 700, 3
    lo = random_placements(rng, T, H, list(tmpl.shape[::-1]), shape)
    got, _ = pcdf.composite_translated(sq, grid, tmpl, lo, 2, want_sdf=False)
    torch.cuda.synchronize()
    assert_equal_fields(got.cpu().numpy(), oracle.translated_composite(S, want_t, lo), "comp_sq")


def test_translated_composite_replays_from_a_graph():
    """The placements travel as kernel parameters, so a captured call replays
    the captured placements."""
    shape = (16, 16, 32)
    occ = box_static(shape, 11)
    grid = scenes.Grid(shape[2], shape[1], shape[0], 0.05)
    sq, sdf = pcdf.build_static_sdf(cuda(occ), grid)
    tmpl, lo0 = pcdf.build_template(PRIMS[2], 3, dev())
    rng = np.random.default_rng(12)
    lo = random_placements(rng, 4, 2, list(tmpl.shape[::-1]), shape)
    want_sq, want_sdf = pcdf.composite_translated(sq, grid, tmpl, lo, 3, static_sdf=sdf)
    out_sq = torch.empty_like(want_sq)
    out_sdf = torch.empty_like(want_sdf)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            pcdf.composite_translated(sq, grid, tmpl, lo, 3, static_sdf=sdf, comp_sq=out_sq, comp_sdf=out_sdf)
    lo[:] = 0  # the host array changes after capture; the replay keeps the captured placements
    out_sq.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out_sq, want_sq)
    assert torch.equal(out_sdf.view(torch.int32), want_sdf.view(torch.int32))


def test_field_max_matches_numpy():
    rng = np.random.default_rng(13)
    for n in (1, 255, 257, 100003):
        a = rng.integers(-(1 << 30), 1 << 20, n).astype(np.int32)
        a[rng.integers(0, n, max(n // 10, 1))] = oracle.INF32
        t = cuda(a)
        fin = a[(a > 0) & (a < oracle.INF32)]
        want = int(fin.max()) if fin.size else 0
        R = pcdf.template_radius(t)
        assert R * R >= want and (R - 1) * (R - 1) < want or (want == 0 and R == 0)
    assert pcdf.template_radius(cuda(np.full(64, oracle.INF32, np.int32))) == 0
    assert pcdf.template_radius(cuda(np.full(64, -5, np.int32))) == 0


def humans_apart(caps, margin_fp=3 * 28):
    """Upright capsules of one t whose axes are further apart than their radii
    plus a gap of a few voxels (no shared or face-adjacent voxels)."""
    for t in range(caps.shape[0]):
        for h in range(caps.shape[1]):
            for g in range(h + 1, caps.shape[1]):
                a, b = caps[t, h], caps[t, g]
                dist = np.hypot(float(a[0] - b[0]), float(a[1] - b[1]))
                if dist <= (a[6] & ~CYL) + (b[6] & ~CYL) + margin_fp:
                    return False
    return True


def test_translated_equals_the_exact_composite_on_the_256_workload():
    """The bench workload (256^3, 60 boxes, 3 walking humans, T = 20) with every
    human laid on the lattice relative to human 0 at t = 0 and lifted one
    voxel: with R^2 above
    every static value the translated template reproduces the exact composite
    path everywhere, and sampled time steps match the oracle in full."""
    sc = scenes.scene_composite(seed=0)
    grid, occ = sc["grid"], sc["occ"]
    caps = scenes.lattice_moves(sc["caps"], sc["caps"][0, 0])
    # one voxel off the floor, so that the free voxels around every human lie
    # in the grid (on the floor the exact path, counting in-grid voxels only,
    # gives the interior voxels of the feet larger magnitudes)
    caps[..., 2] += 16
    caps[..., 5] += 16
    ref = caps[0, 0]
    assert humans_apart(caps)
    sq, sdf = pcdf.build_static_sdf(cuda(occ), grid)
    R = pcdf.template_radius(sq)
    tmpl, lo0 = pcdf.build_template(ref, R, dev())
    lo = pcdf.lattice_placements(caps, ref, lo0)
    got_sq, got_sdf = pcdf.composite_translated(sq, grid, tmpl, lo, R, static_sdf=sdf)
    want_sq, want_sdf = pcdf.build_predicted_composite(sq, grid, caps, static_sdf=sdf)
    torch.cuda.synchronize()
    assert torch.equal(got_sq, want_sq)
    assert torch.equal(got_sdf.view(torch.int32), want_sdf.view(torch.int32))
    del want_sq, want_sdf
    S = oracle.edt(occ)
    t_oracle, lo_oracle = oracle.template_field(ref, R)
    assert list(lo_oracle) == list(lo0)
    for t in (0, 11, 19):
        want = oracle.translated_composite(S, t_oracle, lo[t:t + 1])[0]
        assert_equal_fields(got_sq[t].cpu().numpy(), want, f"comp_sq[{t}]")
