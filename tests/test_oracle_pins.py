"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks an oracle routine against brute force, a closed form, a
textbook/library routine (scipy's exact EDT) or an invariant, chosen so that a
dropped term, a wrong sign, an off-by-one index or a transposed axis in the
oracle fails at least one of them.  No GPU is needed.
"""
import numpy as np
import pytest

import oracle
import scenes

INF = oracle.INF32


def sq_dist_to_set(shape, pts):
    """Squared index distance from every voxel to the nearest of pts (numpy, O(V*|pts|))."""
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    best = np.full(shape, np.iinfo(np.int64).max, np.int64)
    for (pk, pj, pi) in pts:
        best = np.minimum(best, (k - pk) ** 2 + (j - pj) ** 2 + (i - pi) ** 2)
    return best


# ---------------------------------------------------------------------------
# signed squared EDT: closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("fn", [oracle.edt_brute, oracle.edt])
def test_edt_single_voxel(fn):
    shape = (7, 11, 9)
    occ = np.zeros(shape, np.uint8)
    occ[3, 4, 6] = 1
    S = fn(occ)
    k, j, i = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    want = (k - 3) ** 2 + (j - 4) ** 2 + (i - 6) ** 2
    want[3, 4, 6] = -1  # the occupied voxel: nearest free neighbour at distance 1
    assert np.array_equal(S, want)


@pytest.mark.parametrize("fn", [oracle.edt_brute, oracle.edt])
def test_edt_empty_and_full(fn):
    shape = (5, 6, 7)
    assert np.all(fn(np.zeros(shape, np.uint8)) == INF)
    assert np.all(fn(np.ones(shape, np.uint8)) == -INF)


def box_closed_form(shape, lo, hi):
    """Signed squared EDT of one axis-aligned box [lo, hi] (inclusive indices, zyx)."""
    nz, ny, nx = shape
    idx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside = np.ones(shape, bool)
    ext = np.zeros(shape, np.int64)
    for a in range(3):
        c = idx[a]
        inside &= (c >= lo[a]) & (c <= hi[a])
        gap = np.maximum(np.maximum(lo[a] - c, 0), c - hi[a])
        ext += gap ** 2
    # interior: nearest free voxel is straight out through the nearest face
    # that has an in-grid voxel beyond it
    n = (nz, ny, nx)
    best = np.full(shape, np.iinfo(np.int64).max, np.int64)
    for a in range(3):
        c = idx[a]
        if lo[a] - 1 >= 0:
            best = np.minimum(best, (c - lo[a] + 1) ** 2)
        if hi[a] + 1 <= n[a] - 1:
            best = np.minimum(best, (hi[a] - c + 1) ** 2)
    interior = np.where(best == np.iinfo(np.int64).max, -INF, -best)
    return np.where(inside, interior, ext).astype(np.int64)


@pytest.mark.parametrize("fn", [oracle.edt_brute, oracle.edt])
@pytest.mark.parametrize("lo,hi", [((2, 3, 4), (5, 7, 6)), ((0, 0, 3), (3, 12, 8)), ((1, 2, 0), (4, 4, 10))])
def test_edt_single_box(fn, lo, hi):
    shape = (9, 13, 11)
    occ = np.zeros(shape, np.uint8)
    occ[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] = 1
    assert np.array_equal(fn(occ).astype(np.int64), box_closed_form(shape, lo, hi))


@pytest.mark.parametrize("fn", [oracle.edt_brute, oracle.edt])
def test_edt_halfspace_wall(fn):
    # wall occupying x >= 5: S is the squared 1-D distance along x
    shape = (4, 6, 12)
    occ = np.zeros(shape, np.uint8)
    occ[:, :, 5:] = 1
    x = np.arange(12)
    row = np.where(x < 5, (5 - x) ** 2, -((x - 4) ** 2))
    assert np.array_equal(fn(occ), np.broadcast_to(row, shape))


# ---------------------------------------------------------------------------
# signed squared EDT: brute force and scipy
# ---------------------------------------------------------------------------

def scipy_signed(occ):
    """Signed squared EDT from scipy's exact EDT (distance of non-zero elements
    to the nearest zero element)."""
    ndi = pytest.importorskip("scipy.ndimage")
    occ = occ != 0
    out = np.empty(occ.shape, np.int64)
    if occ.any():
        d = ndi.distance_transform_edt(~occ)  # free voxels: distance to occupied
        out[~occ] = np.rint(d[~occ] ** 2).astype(np.int64)
    else:
        out[:] = INF
    if (~occ).any():
        d = ndi.distance_transform_edt(occ)  # occupied voxels: distance to free
        out[occ] = -np.rint(d[occ] ** 2).astype(np.int64)
    else:
        out[:] = -INF
    return out


@pytest.mark.parametrize("density", [0.01, 0.1, 0.5, 0.9])
@pytest.mark.parametrize("shape", [(13, 17, 15), (16, 16, 16), (1, 1, 23), (23, 1, 1), (3, 29, 2)])
def test_brute_against_numpy_and_scipy(density, shape):
    rng = np.random.default_rng(int(density * 1000) + sum(shape))
    occ = scenes.random_occupancy(shape, density, rng)
    S = oracle.edt_brute(occ).astype(np.int64)
    if 0 < occ.sum() < occ.size:
        assert np.array_equal(S, scipy_signed(occ))
    occ_pts = np.argwhere(occ != 0)
    free_pts = np.argwhere(occ == 0)
    if len(occ_pts) and len(free_pts):
        dO = sq_dist_to_set(shape, occ_pts)
        dF = sq_dist_to_set(shape, free_pts)
        assert np.array_equal(S, np.where(occ != 0, -dF, dO))


@pytest.mark.parametrize("density", [0.0, 0.001, 0.01, 0.1, 0.5, 1.0])
@pytest.mark.parametrize("shape", [(16, 16, 16), (13, 17, 15), (1, 1, 40), (40, 1, 1), (1, 37, 1), (2, 3, 31)])
def test_separable_against_brute(density, shape):
    rng = np.random.default_rng(7 + int(density * 1e4) + shape[0] * 31 + shape[2])
    occ = scenes.random_occupancy(shape, density, rng)
    if density == 0.001:
        occ[:] = 0
        occ[tuple(rng.integers(0, n) for n in shape)] = 1
    assert np.array_equal(oracle.edt(occ), oracle.edt_brute(occ))


def test_separable_against_scipy_small_scene():
    sc = scenes.scene_small(seed=3)
    occ = sc["occ"]
    assert 0 < occ.sum() < occ.size
    assert np.array_equal(oracle.edt(occ).astype(np.int64), scipy_signed(occ))


def test_edt_at_matches_brute_samples():
    rng = np.random.default_rng(11)
    occ = scenes.random_occupancy((9, 10, 11), 0.2, rng)
    S = oracle.edt_brute(occ)
    for _ in range(40):
        k, j, i = (int(rng.integers(0, n)) for n in occ.shape)
        assert oracle.edt_at(occ, i, j, k) == S[k, j, i]


# ---------------------------------------------------------------------------
# capsules
# ---------------------------------------------------------------------------

def test_capsule_predicate_exact_boundaries():
    # sphere (a == b) of radius 80 at the origin: Pythagorean boundary points
    cap = [0, 0, 0, 0, 0, 0, 80]
    assert oracle.capsule_inside((48, 64, 0), cap)
    assert not oracle.capsule_inside((48, 65, 0), cap)
    assert oracle.capsule_inside((0, 0, -80), cap)
    assert not oracle.capsule_inside((0, 1, -80), cap)
    # vertical segment 0..160 on the z axis, radius 80
    cap = [0, 0, 0, 0, 0, 160, 80]
    assert oracle.capsule_inside((48, 64, 80), cap)      # side, distance exactly 80
    assert not oracle.capsule_inside((49, 64, 80), cap)
    assert oracle.capsule_inside((0, 0, 240), cap)       # top cap apex
    assert not oracle.capsule_inside((1, 0, 240), cap)
    assert oracle.capsule_inside((0, 0, -80), cap)       # bottom cap apex
    assert not oracle.capsule_inside((0, 0, -81), cap)
    # a slanted segment: (0,0,0)-(30,40,0), radius 50; the point (-40, 30, 0) is
    # perpendicular to the axis at a, distance exactly 50
    cap = [0, 0, 0, 30, 40, 0, 50]
    assert oracle.capsule_inside((-40, 30, 0), cap)
    assert not oracle.capsule_inside((-40, 31, 0), cap)
    # mid-segment perpendicular point: (15,20,0) + 50*(-0.8, 0.6, 0) = (-25, 50, 0)
    assert oracle.capsule_inside((-25, 50, 0), cap)
    assert not oracle.capsule_inside((-25, 51, 0), cap)


def seg_dist(p, a, b):
    p, a, b = (np.asarray(v, np.float64) for v in (p, a, b))
    d = b - a
    L = d @ d
    s = 0.0 if L == 0 else np.clip((p - a) @ d / L, 0.0, 1.0)
    return np.linalg.norm(p - (a + s * d))


def test_capsule_predicate_vs_float_distance():
    rng = np.random.default_rng(5)
    n_checked = 0
    for _ in range(3000):
        a = rng.integers(-500, 1500, 3)
        b = a + rng.integers(-400, 400, 3) * (rng.uniform() < 0.8)
        r = int(rng.integers(0, 300))
        p = rng.integers(-800, 1800, 3)
        dist = seg_dist(p, a, b)
        if abs(dist - r) < 1e-6 * max(1.0, r):
            continue
        n_checked += 1
        assert oracle.capsule_inside(p, list(a) + list(b) + [r]) == (dist <= r)
    assert n_checked > 2900


def test_capsule_field_sandwich():
    """Exterior voxels: continuous distance to the capsule <= sqrt(S) <= that + sqrt(3)
    (voxel units), since any ball of radius sqrt(3)/2 holds a lattice point."""
    grid = scenes.Grid(40, 36, 48, 0.05)
    cap = scenes.standing_capsule(grid, (1.0, 0.9))
    occ = oracle.capsule_occupancy(grid.shape, cap[None])
    S = oracle.edt(occ)
    nz, ny, nx = grid.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    P = np.stack([16 * i + 8, 16 * j + 8, 16 * k + 8], -1).reshape(-1, 3).astype(np.float64)
    a = cap[:3].astype(np.float64)
    b = cap[3:6].astype(np.float64)
    d = b - a
    s = np.clip((P - a) @ d / (d @ d), 0, 1)
    dc = (np.linalg.norm(P - (a + s[:, None] * d), axis=1) - cap[6]) / 16.0  # voxel units
    Sf = S.reshape(-1)
    ext = Sf > 0
    assert ext.sum() > 0 and (~ext).sum() > 0
    root = np.sqrt(Sf[ext].astype(np.float64))
    assert np.all(dc[ext] <= root + 1e-9)
    assert np.all(root <= dc[ext] + np.sqrt(3.0) + 1e-9)
    # interior voxels are exactly those with dc <= 0
    assert np.array_equal(Sf < 0, dc <= 1e-12)


def test_capsule_field_bounds_of_the_certificate():
    """The two inequalities that the surrogate's certificate rests on, on
    random slanted capsules (radius >= 14/16 voxel, inside the grid, some
    touching the floor) and on unions of two: outside every capsule the exact
    field lies in [min_k d_k, min_k d_k + sqrt(3)] (voxel units, d_k the
    continuous distance to capsule k); inside the union it is at most
    min_k d_k (no lower bound is claimed there)."""
    rng = np.random.default_rng(31)
    grid = scenes.Grid(24, 22, 26, 0.05)
    nz, ny, nx = grid.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    P = np.stack([16 * i + 8, 16 * j + 8, 16 * k + 8], -1).reshape(-1, 3).astype(np.float64)
    checked = 0
    for trial in range(12):
        caps = []
        for h in range(1 + trial % 2):
            r = int(rng.integers(14, 70))
            lo = np.array([r, r, r]) + 1
            hi = 16 * np.array([nx, ny, nz]) - r - 1
            a = rng.integers(lo, hi)
            b = rng.integers(lo, hi)
            if trial % 3 == 0:  # standing on the floor
                a[2] = r
                b[:2] = a[:2]
            caps.append([*a, *b, r])
        caps = np.array(caps, np.int32)
        S = oracle.edt(oracle.capsule_occupancy(grid.shape, caps)).reshape(-1).astype(np.float64)
        dmin = np.min([(np.array([seg_dist(q, c[:3], c[3:6]) for q in P]) - c[6]) / 16.0 for c in caps], axis=0)
        ext = S > 0
        root = np.sqrt(S[ext])
        assert np.all(dmin[ext] <= root + 1e-9)
        assert np.all(root <= dmin[ext] + np.sqrt(3.0) + 1e-9)
        inside = (S < 0) & (S != -oracle.INF32)
        assert np.all(-np.sqrt(-S[inside]) <= dmin[inside] + 1e-9)
        checked += int(ext.sum() + inside.sum())
    assert checked > 50000


def test_capsule_occupancy_matches_predicate_loop():
    grid = scenes.Grid(12, 10, 14, 0.05)
    caps = np.array([[40, 50, 30, 150, 60, 180, 45], [10, 10, 10, 10, 10, 10, 60]], np.int32)
    occ = oracle.capsule_occupancy(grid.shape, caps)
    for k in range(grid.nz):
        for j in range(grid.ny):
            for i in range(grid.nx):
                p = (16 * i + 8, 16 * j + 8, 16 * k + 8)
                want = any(oracle.capsule_inside(p, c) for c in caps)
                assert bool(occ[k, j, i]) == want


# ---------------------------------------------------------------------------
# composite (Sec. 6)
# ---------------------------------------------------------------------------

def test_composite_equals_union_edt_outside_obstacles():
    """min(d^2 to A, d^2 to B) = d^2 to A u B: exact on voxels free in both maps;
    inside obstacles the min's magnitude never exceeds the union's."""
    sc = scenes.scene_small_walking(seed=2, T=3, H=2)
    occ, caps = sc["occ"], sc["caps"]
    S_static = oracle.edt(occ)
    comp = oracle.predicted_composite(S_static, caps)
    scratch = oracle.from_scratch(occ, caps)
    for t in range(caps.shape[0]):
        dyn_occ = oracle.capsule_occupancy(occ.shape, caps[t])
        free_both = (occ == 0) & (dyn_occ == 0)
        assert free_both.sum() > 0
        assert np.array_equal(comp[t][free_both], scratch[t][free_both])
        inside = ~free_both
        assert np.all(comp[t][inside] < 0) and np.all(scratch[t][inside] < 0)
        assert np.all(-comp[t][inside].astype(np.int64) <= -scratch[t][inside].astype(np.int64))
        # composite against the brute-force definition on samples
        rng = np.random.default_rng(t)
        for _ in range(20):
            kk, jj, ii = (int(rng.integers(0, n)) for n in occ.shape)
            want = min(oracle.edt_at(occ, ii, jj, kk), oracle.edt_at(dyn_occ, ii, jj, kk))
            assert comp[t, kk, jj, ii] == want


def test_composite_without_humans_is_static():
    rng = np.random.default_rng(1)
    occ = scenes.random_occupancy((10, 12, 14), 0.1, rng)
    S = oracle.edt(occ)
    caps_far = np.array([[[-3000, -3000, -3000, -3000, -3000, -2000, 50]]], np.int32)
    comp = oracle.predicted_composite(S, caps_far)
    assert np.array_equal(comp[0], S)


# ---------------------------------------------------------------------------
# float field
# ---------------------------------------------------------------------------

def test_sdf_from_sq_values():
    S = np.array([1, 4, 9, -16, 2, 3, INF, -INF, 783363], np.int32)
    vox = np.float32(0.04)
    got = oracle.sdf_from_sq(S, float(vox))
    assert got[0] == vox and got[1] == np.float32(2) * vox and got[2] == np.float32(3) * vox
    assert got[3] == -(np.float32(4) * vox)
    assert got[4] == np.float32(np.sqrt(np.float32(2))) * vox  # numpy float32 sqrt is IEEE
    assert got[6] == np.inf and got[7] == -np.inf
    # every integer magnitude below 2^24 is exact in fp32; compare with numpy's IEEE fp32 chain
    S2 = np.arange(-50000, 50000, 7, dtype=np.int32)
    S2 = S2[S2 != 0]
    want = np.sign(S2).astype(np.float32) * (np.sqrt(np.abs(S2).astype(np.float32)) * vox)
    assert np.array_equal(oracle.sdf_from_sq(S2, float(vox)), want)


# ---------------------------------------------------------------------------
# trilinear sampling, hinge cost, gradient
# ---------------------------------------------------------------------------

def affine_field(shape, coef):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (coef[0] * i + coef[1] * j + coef[2] * k + coef[3]).astype(np.float32)


def test_trilinear_reproduces_voxel_centres():
    rng = np.random.default_rng(0)
    field = rng.normal(size=(6, 7, 8)).astype(np.float32)
    vox = 0.25
    origin = np.array([0.5, -1.0, 2.0], np.float32)
    for _ in range(50):
        i, j, k = rng.integers(0, 8), rng.integers(0, 7), rng.integers(0, 6)
        p = origin + (np.array([i, j, k]) + 0.5) * vox
        d, oob, _ = oracle.trilinear(field, origin, vox, p)
        assert not oob
        assert d == float(field[k, j, i])


def test_trilinear_exact_on_affine_field_and_gradient():
    coef = (2.0, 3.0, -1.0, 5.0)
    shape = (9, 10, 11)
    field = affine_field(shape, coef)
    vox = 0.5
    origin = np.zeros(3, np.float32)
    rng = np.random.default_rng(1)
    for _ in range(200):
        u = rng.uniform(0.0, 1.0, 3) * (np.array([11, 10, 9]) - 1)
        p = ((u + 0.5) * vox).astype(np.float32)
        uu = p.astype(np.float64) / vox - 0.5  # exact for vox = 0.5
        d, oob, g = oracle.trilinear(field, origin, vox, p)
        assert not oob
        assert abs(d - (coef[0] * uu[0] + coef[1] * uu[1] + coef[2] * uu[2] + coef[3])) < 1e-12
        assert np.allclose(g, np.array(coef[:3]) / vox, atol=1e-12)


def test_trilinear_clamps_outside():
    field = affine_field((4, 5, 6), (1.0, 10.0, 100.0, 0.0))
    vox = 1.0
    origin = np.zeros(3, np.float32)
    d, oob, g = oracle.trilinear(field, origin, vox, np.array([-3.0, 2.5, 1.5], np.float32))
    assert oob and d == 0.0 * 1 + 10.0 * 2 + 100.0 * 1 and g[0] == 0.0 and g[1] == 10.0
    d, oob, g = oracle.trilinear(field, origin, vox, np.array([100.0, 2.5, 100.0], np.float32))
    assert oob and d == 5.0 + 20.0 + 300.0 and g[0] == 0.0 and g[2] == 0.0


def test_trilinear_mirror_symmetry():
    rng = np.random.default_rng(2)
    field = rng.normal(size=(5, 6, 7)).astype(np.float32)
    mirrored = field[:, :, ::-1].copy()
    vox = 0.5
    origin = np.zeros(3, np.float32)
    for _ in range(50):
        p = (rng.uniform(0.6, 2.9, 3) * np.array([1, 1, 1])).astype(np.float32)
        q = p.copy()
        q[0] = np.float32(7 * vox) - p[0]
        d1, _, g1 = oracle.trilinear(field, origin, vox, p)
        d2, _, g2 = oracle.trilinear(mirrored, origin, vox, q)
        assert abs(d1 - d2) < 1e-6
        assert abs(g1[0] + g2[0]) < 1e-5 and abs(g1[1] - g2[1]) < 1e-5


def test_trilinear_gradient_finite_differences():
    rng = np.random.default_rng(3)
    field = rng.normal(size=(6, 6, 6)).astype(np.float32)
    vox = 0.5
    origin = np.zeros(3, np.float32)
    h = 1.0 / 1024  # exact in fp32 at these magnitudes; cells are multilinear
    checked = 0
    for _ in range(300):
        p = rng.uniform(0.4, 2.6, 3)
        u = p / vox - 0.5
        if np.any(np.abs(u - np.rint(u)) < 4 * h / vox):
            continue
        p = p.astype(np.float32)
        _, _, g = oracle.trilinear(field, origin, vox, p)
        for a in range(3):
            pp, pm = p.copy(), p.copy()
            pp[a] += np.float32(h)
            pm[a] -= np.float32(h)
            dp, _, _ = oracle.trilinear(field, origin, vox, pp)
            dm, _, _ = oracle.trilinear(field, origin, vox, pm)
            fd = (dp - dm) / (float(pp[a]) - float(pm[a]))
            assert abs(fd - g[a]) < 1e-9
        checked += 1
    assert checked > 100


def test_trilinear_infinite_fields():
    vox = 1.0
    origin = np.zeros(3, np.float32)
    d, _, g = oracle.trilinear(np.full((3, 3, 3), np.inf, np.float32), origin, vox, np.ones(3, np.float32))
    assert d == np.inf and np.all(g == 0)
    d, _, _ = oracle.trilinear(np.full((3, 3, 3), -np.inf, np.float32), origin, vox, np.ones(3, np.float32))
    assert d == -np.inf


def test_hinge_cost_closed_form_and_time_index():
    """h = max(0, eps + r - d) (Sec. 7 hinge, radius added to eps); field index
    clamp(s, 0, T-1) (Sec. 8)."""
    shape = (4, 5, 6)
    T = 3
    sdf = np.stack([np.full(shape, 0.1 * (t + 1), np.float32) for t in range(T)])
    sph = np.array([[1.0, 1.0, 1.0, 0.1]] * 5, np.float32)
    tidx = np.array([0, 1, 2, 7, -2], np.int32)
    h, n_oob, gc, gr = oracle.hinge_cost(sdf, np.zeros(3), 0.5, sph, tidx, 0.2, need_grad=True)
    d = np.array([0.1, 0.2, 0.3, 0.3, 0.1])
    want = np.maximum(0.0, np.float32(0.2) + np.float64(np.float32(0.1)) - d.astype(np.float32).astype(np.float64))
    assert np.allclose(h, want, atol=1e-7)
    assert n_oob == 0
    assert np.all(gc == 0)  # constant field
    assert np.array_equal(gr, (want > 0).astype(np.float64))


def test_hinge_gradient_matches_finite_differences_of_cost():
    """dh/dc against central differences of the cost itself.  The field comes
    from a real scene; the sampling voxel size is 1/16 m and the step 2^-12 m so
    that every fp32 coordinate and continuous index is exact and the
    differences of the multilinear cells are exact up to fp64 rounding."""
    sc = scenes.scene_small(seed=4, n_spheres=400)
    g = sc["grid"]
    S = oracle.edt(sc["occ"])
    sdf = oracle.sdf_from_sq(S, g.vox)
    vox = 1.0 / 16
    rng = np.random.default_rng(9)
    sph = np.concatenate([rng.uniform(0.2, 3.8, (400, 3)), np.full((400, 1), 0.6)], 1).astype(np.float32)
    tidx = np.zeros(400, np.int32)
    h, _, gc, gr = oracle.hinge_cost(sdf, np.zeros(3), vox, sph, tidx, sc["eps"], need_grad=True)
    step = 2.0 ** -12
    checked = 0
    for q in range(sph.shape[0]):
        u = sph[q, :3].astype(np.float64) / vox - 0.5
        if np.any(np.abs(u - np.rint(u)) < 4 * step / vox) or not (0.05 < h[q]):
            continue
        for a in range(3):
            p = np.repeat(sph[q:q + 1], 2, axis=0)
            p[0, a] += np.float32(step)
            p[1, a] -= np.float32(step)
            assert float(p[0, a]) - float(p[1, a]) == 2 * step
            hh, _ = oracle.hinge_cost(sdf, np.zeros(3), vox, p, np.zeros(2, np.int32), sc["eps"])
            fd = (hh[0] - hh[1]) / (2 * step)
            assert abs(fd - gc[q, a]) < 1e-7 * max(1.0, abs(gc[q, a]))
        assert gr[q] == 1.0
        checked += 1
    assert checked > 100


# ---------------------------------------------------------------------------
# Sec. 8 static-map clean-up and the collapsed 2-D map
# ---------------------------------------------------------------------------

def test_voxel_filter_closed_forms():
    g = np.zeros((7, 7, 7), np.uint8)
    g[3, 3, 3] = 1                                   # isolated: 0 neighbours
    assert oracle.voxel_filter(g).sum() == 0
    g[:] = 0
    g[2:5, 2:5, 2:5] = 1                             # 3x3x3 cube: corners have 7 neighbours
    assert np.array_equal(oracle.voxel_filter(g), g)
    g[:] = 0
    g[1:3, 1:3, 1:3] = 1                             # 2x2x2 cube: 7 neighbours each
    assert np.array_equal(oracle.voxel_filter(g), g)
    g[:] = 0
    g[3, 3, :] = 1                                   # a line: at most 2 neighbours
    assert oracle.voxel_filter(g).sum() == 0
    g[:] = 0
    g[3, 1:3, 1:3] = 1                               # 2x2 square: 3 neighbours each
    assert oracle.voxel_filter(g).sum() == 0
    assert np.array_equal(oracle.voxel_filter(g, 3), g)
    assert oracle.voxel_filter(g, 4).sum() == 0
    g[:] = 0
    g[3, 1:4, 1:4] = 1                               # 3x3 square: corners 3, edges 5, centre 8
    want = np.zeros_like(g)
    want[3, 2, 1:4] = 1
    want[3, 1:4, 2] = 1
    assert np.array_equal(oracle.voxel_filter(g), want)
    # the grid boundary is not occupied: a full grid keeps only voxels with >= 5
    # in-grid neighbours (a corner of a 2x2x2 grid has 7)
    assert oracle.voxel_filter(np.ones((2, 2, 2), np.uint8)).sum() == 8
    assert oracle.voxel_filter(np.ones((1, 1, 4), np.uint8)).sum() == 0


@pytest.mark.parametrize("shape,density,k", [((9, 11, 13), 0.3, 5), ((16, 16, 16), 0.1, 5), ((5, 1, 40), 0.6, 2),
                                             ((12, 10, 8), 0.5, 0), ((12, 10, 8), 0.9, 26)])
def test_voxel_filter_matches_a_convolution(shape, density, k):
    from scipy import ndimage
    g = (np.random.default_rng(len(shape) + k).random(shape) < density).astype(np.uint8)
    n = ndimage.convolve(g.astype(np.int32), np.ones((3, 3, 3), np.int32), mode="constant", cval=0) - g
    want = ((g == 1) & (n >= k)).astype(np.uint8)
    assert np.array_equal(oracle.voxel_filter(g, k), want)


def test_collapse_and_2d_edt():
    from scipy import ndimage
    rng = np.random.default_rng(7)
    g = (rng.random((20, 31, 37)) < 0.02).astype(np.uint8)
    for z0, z1 in ((0, 20), (3, 9), (-5, 4), (15, 40), (6, 6)):
        want = g[max(z0, 0):max(min(z1, 20), 0)].any(axis=0).astype(np.uint8)
        assert np.array_equal(oracle.collapse(g, z0, z1), want)
    c = oracle.collapse(g, 2, 12)
    S = oracle.edt(c[None])[0]
    dO = ndimage.distance_transform_edt(c == 0)
    dF = ndimage.distance_transform_edt(c == 1)
    want = np.where(c == 0, np.rint(dO ** 2), -np.rint(dF ** 2)).astype(np.int64)
    assert np.array_equal(S.astype(np.int64), want)


# ---------------------------------------------------------------------------
# cylinder primitive (Sec. 6's human primitive; radius-word flag)
# ---------------------------------------------------------------------------

CYL = 1 << 30


def test_cylinder_predicate_upright_exact():
    a, b, r = (104, 88, 24), (104, 88, 216), 40
    cap = np.array([*a, *b, r | CYL], np.int32)
    for k in range(16):
        for j in range(12):
            for i in range(14):
                p = (16 * i + 8, 16 * j + 8, 16 * k + 8)
                want = (p[0] - a[0]) ** 2 + (p[1] - a[1]) ** 2 <= r * r and a[2] <= p[2] <= b[2]
                assert oracle.capsule_inside(p, cap) == want, (i, j, k)


def test_cylinder_boundaries_and_caps():
    cap = np.array([0, 0, 0, 0, 0, 160, 48 | CYL], np.int32)
    capsule = np.array([0, 0, 0, 0, 0, 160, 48], np.int32)
    assert oracle.capsule_inside((48, 0, 80), cap)          # on the side
    assert not oracle.capsule_inside((48, 1, 80), cap)
    assert oracle.capsule_inside((0, 0, 0), cap)            # on an end face
    assert oracle.capsule_inside((30, 30, 160), cap)
    assert not oracle.capsule_inside((0, 0, -1), cap)       # beyond the end: only the capsule holds it
    assert oracle.capsule_inside((0, 0, -1), capsule)
    assert not oracle.capsule_inside((0, 0, 161), cap)
    zero = np.array([5, 5, 5, 5, 5, 5, 40 | CYL], np.int32)
    assert not oracle.capsule_inside((5, 5, 5), zero)       # a zero-length axis holds nothing


def test_cylinder_slanted_against_geometry_and_inside_capsule():
    rng = np.random.default_rng(12)
    for _ in range(20):
        a = rng.integers(0, 400, 3)
        b = a + rng.integers(-200, 200, 3)
        r = int(rng.integers(8, 90))
        cap = np.array([*a, *b, r | CYL], np.int32)
        capsule = np.array([*a, *b, r], np.int32)
        d = (b - a).astype(np.float64)
        L = d @ d
        for _ in range(300):
            p = rng.integers(-100, 600, 3)
            w = (p - a).astype(np.float64)
            s = w @ d
            dist2 = w @ w - s * s / L
            inside = oracle.capsule_inside(tuple(int(v) for v in p), cap)
            if inside:
                assert oracle.capsule_inside(tuple(int(v) for v in p), capsule)
            if abs(dist2 - r * r) > 1e-6 * r * r and min(abs(s), abs(s - L)) > 1e-9 * L:
                assert inside == (0 <= s <= L and dist2 <= r * r)


def test_cylinder_field_sandwich():
    """EDT of the cylinder's voxels: an exterior voxel's distance is at least
    its continuous distance to the solid (brute force on a small grid)."""
    cap = np.array([[72, 72, 40, 72, 72, 200, 36 | CYL]], np.int32)
    occ = oracle.capsule_occupancy((16, 10, 10), cap)
    S = oracle.edt_brute(occ)
    assert np.array_equal(S, oracle.edt(occ))
    for k, j, i in np.argwhere(occ == 0)[::7]:
        p = np.array([16 * i + 8, 16 * j + 8, 16 * k + 8], np.float64)
        radial = max(np.hypot(p[0] - 72, p[1] - 72) - 36, 0.0)
        axial = max(40 - p[2], p[2] - 200, 0.0)
        cont = np.hypot(radial, axial) / 16.0
        assert np.sqrt(S[k, j, i]) >= cont - 1e-9


# ---------------------------------------------------------------------------
# translated primitive field (Sec. 6: one primitive field, moved to each
# predicted position)
# ---------------------------------------------------------------------------

def inside_voxels_map(cap, lo, dims):
    """occupancy [dz,dy,dx] of the box at map index lo, tested voxel by voxel
    with the primitive in map coordinates (no shift of the primitive)."""
    dx, dy, dz = dims
    occ = np.zeros((dz, dy, dx), np.uint8)
    for k in range(dz):
        for j in range(dy):
            for i in range(dx):
                p = (16 * (lo[0] + i) + 8, 16 * (lo[1] + j) + 8, 16 * (lo[2] + k) + 8)
                occ[k, j, i] = oracle.capsule_inside(p, cap)
    return occ


def test_template_box_is_the_tight_box_of_an_upright_capsule():
    """An upright capsule whose axis passes through voxel centres: the inner box
    (without R) is exactly the bounding box of its voxels."""
    for (i, j, k0, k1, rv) in [(5, 7, 3, 9, 2), (0, 0, 0, 0, 1), (-4, 11, -2, 6, 3)]:
        r = 16 * rv + 5
        cap = np.array([16 * i + 8, 16 * j + 8, 16 * k0 + 8, 16 * i + 8, 16 * j + 8, 16 * k1 + 8, r], np.int32)
        for R in (0, 2):
            lo, dims = oracle.template_box(cap, R)
            assert lo == [i - rv - R, j - rv - R, k0 - rv - R]
            assert dims == [2 * rv + 1 + 2 * R, 2 * rv + 1 + 2 * R, k1 - k0 + 2 * rv + 1 + 2 * R]


def test_template_box_holds_every_voxel_of_the_primitive():
    rng = np.random.default_rng(40)
    for n in range(12):
        a = rng.integers(-200, 300, 3)
        b = a + rng.integers(-120, 120, 3)
        r = int(rng.integers(10, 60))
        if n % 3 == 2 and not np.array_equal(a, b):
            r |= oracle.CYLINDER
        cap = np.array([*a, *b, r], np.int32)
        lo, dims = oracle.template_box(cap, 0)
        # scan a wider box: nothing inside the primitive lies outside the template box
        wide_lo = [lo[q] - 2 for q in range(3)]
        wide = inside_voxels_map(cap, wide_lo, [dims[q] + 4 for q in range(3)])
        inner = np.zeros_like(wide)
        inner[2:-2, 2:-2, 2:-2] = 1
        assert not np.any(wide & (1 - inner))


def test_template_box_rejects_a_primitive_between_centres():
    cap = np.array([20, 20, 20, 20, 20, 20, 3], np.int32)  # radius 3/16 voxel, 4/16 from any centre
    with pytest.raises(ValueError):
        oracle.template_box(cap, 4)


def test_template_field_brute_force():
    """Template values against the squared distance to the primitive's voxels,
    found in map coordinates with no shift, and against the distance to the
    free voxels inside it."""
    for cap in (np.array([40, 56, 30, 40, 56, 90, 20], np.int32),
                np.array([10, 30, 20, 70, 50, 60, 17], np.int32),
                np.array([40, 40, 10, 40, 40, 70, 18 | oracle.CYLINDER], np.int32)):
        R = 2
        tmpl, lo = oracle.template_field(cap, R)
        dz, dy, dx = tmpl.shape
        occ = inside_voxels_map(cap, lo, (dx, dy, dz))
        assert occ.any()
        pts_in = [tuple(p) for p in np.argwhere(occ == 1)]
        pts_out = [tuple(p) for p in np.argwhere(occ == 0)]
        d_in = sq_dist_to_set(tmpl.shape, pts_in)
        d_out = sq_dist_to_set(tmpl.shape, pts_out)
        want = np.where(occ == 1, -d_out, d_in)
        assert np.array_equal(tmpl, want)


def _static_and_R(shape, seed, n_boxes=4):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    occ = np.zeros(shape, np.uint8)
    for _ in range(n_boxes):
        lo = [int(rng.integers(0, n - 3)) for n in shape]
        hi = [min(lo[q] + int(rng.integers(1, 4)), shape[q]) for q in range(3)]
        occ[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = 1
    S = oracle.edt(occ)
    R = int(np.ceil(np.sqrt(float(S.max()))))
    return S, R


def test_translated_composite_equals_the_exact_composite():
    """Integer moves of a primitive well inside the grid, template box widened
    to R with R^2 >= every static value: the translated template gives the
    exact composite of the moved primitives (two humans kept apart)."""
    shape = (20, 18, 22)
    S, R = _static_and_R(shape, 3)
    ref = np.array([16 * 5 + 8, 16 * 5 + 3, 16 * 4 + 8, 16 * 5 + 8, 16 * 5 + 3, 16 * 9 + 8, 26], np.int32)
    tmpl, lo0 = oracle.template_field(ref, R)
    moves = [[(0, 0, 0), (9, 6, 1)], [(1, 2, 0), (10, 8, 2)], [(3, 1, 1), (8, 3, 3)]]
    T, H = len(moves), 2
    caps = np.zeros((T, H, 7), np.int32)
    lo = np.zeros((T, H, 3), np.int64)
    for t in range(T):
        for h in range(H):
            m = np.array(moves[t][h])
            caps[t, h, :3] = ref[:3] + 16 * m
            caps[t, h, 3:6] = ref[3:6] + 16 * m
            caps[t, h, 6] = ref[6]
            lo[t, h] = np.array(lo0) + m
    want = oracle.predicted_composite(S, caps)
    got = oracle.translated_composite(S, tmpl, lo)
    assert np.array_equal(got, want)
    # a box cut too tight (R = 0) misses voxels where the human is nearer than the static field
    tight, lo_t = oracle.template_field(ref, 0)
    lo_tight = lo - np.array(lo0) + np.array(lo_t)
    assert not np.array_equal(oracle.translated_composite(S, tight, lo_tight), want)


def test_translated_composite_clips_boxes_at_the_grid_edges():
    """Boxes partly or wholly outside the grid, by explicit loops over voxels."""
    rng = np.random.default_rng(41)
    S = rng.integers(-30, 60, (5, 6, 7)).astype(np.int32)
    tmpl = rng.integers(-9, 50, (3, 4, 5)).astype(np.int32)
    lo = np.array([[[-2, -1, 3], [4, 3, -1]], [[6, 5, 4], [-7, 0, 0]], [[1, 1, 1], [0, -3, 2]]], np.int64)
    got = oracle.translated_composite(S, tmpl, lo)
    for t in range(3):
        for k in range(5):
            for j in range(6):
                for i in range(7):
                    best = int(S[k, j, i])
                    for h in range(2):
                        u = (i - lo[t, h, 0], j - lo[t, h, 1], k - lo[t, h, 2])
                        if 0 <= u[0] < 5 and 0 <= u[1] < 4 and 0 <= u[2] < 3:
                            best = min(best, int(tmpl[u[2], u[1], u[0]]))
                    assert got[t, k, j, i] == best
