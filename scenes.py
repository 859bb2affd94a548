"""Seeded synthetic scenes for the composite-distance-field workloads.

This module only draws and lays out inputs: box occupancy grids, predicted
human capsules along walking paths and robot body spheres.  It holds none of
the method's arithmetic (no distance transform, composite, interpolation or
cost) and is the one module that both the product tests and the oracle use.

Workloads (all RNG is ``numpy.random.default_rng(seed)``):
  * ``scene_small``: 64^3 grid of 5 cm voxels, 10 boxes with per-axis sizes
    U(0.1, 0.8) m, one standing human capsule (r = 0.25 m, height 1.8 m),
    1024 spheres with radius U(0.05, 0.15) m.
  * ``scene_composite``: 256^3 grid of 4 cm voxels, 60 boxes, 3 humans each
    walking a 4-waypoint polyline at 1.2 m/s, predicted over T = 20 steps of
    0.1 s.
  * ``scene_batch``: ragged environments (per-axis sizes, horizon, humans).
  * ``spheres_along_paths``: robot trajectories as straight lines with body
    spheres scattered about each support state.

Capsules are 7 int32 values (a_xyz, b_xyz, radius) in 1/16-voxel fixed point
measured from the grid corner, so the centre of voxel (i, j, k) is
16*(i, j, k) + 8; metres are converted by round-half-even of
(x - origin) / vox * 16.  A standing human of height h and radius r has its
axis from z = r to z = h - r above the grid floor.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    vox: float
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def extent(self):
        return np.array([self.nx, self.ny, self.nz], np.float64) * self.vox

    @property
    def nvox(self):
        return self.nx * self.ny * self.nz


def to_fixed(x_m, origin_m, vox):
    """Metres -> 1/16-voxel fixed point (round half to even)."""
    return np.rint((np.asarray(x_m, np.float64) - origin_m) / vox * 16.0).astype(np.int64)


def boxes_occupancy(grid: Grid, n_boxes: int, rng, size_range=(0.1, 0.8)):
    """uint8 [nz,ny,nx]: voxel occupied iff its centre lies in a closed box.

    Box centres are uniform over the grid extent, sizes uniform per axis."""
    ext = grid.extent
    org = np.asarray(grid.origin, np.float64)
    centres = org + rng.uniform(0.0, 1.0, size=(n_boxes, 3)) * ext
    sizes = rng.uniform(size_range[0], size_range[1], size=(n_boxes, 3))
    lo = centres - sizes / 2
    hi = centres + sizes / 2
    xs = org[0] + (np.arange(grid.nx) + 0.5) * grid.vox
    ys = org[1] + (np.arange(grid.ny) + 0.5) * grid.vox
    zs = org[2] + (np.arange(grid.nz) + 0.5) * grid.vox
    occ = np.zeros(grid.shape, np.uint8)
    for b in range(n_boxes):
        ix = (xs >= lo[b, 0]) & (xs <= hi[b, 0])
        iy = (ys >= lo[b, 1]) & (ys <= hi[b, 1])
        iz = (zs >= lo[b, 2]) & (zs <= hi[b, 2])
        occ[np.ix_(iz, iy, ix)] = 1
    return occ, np.stack([lo, hi], axis=1)


def standing_capsule(grid: Grid, xy_m, radius=0.25, height=1.8):
    """One upright human capsule standing on the grid floor, fixed point."""
    org = np.asarray(grid.origin, np.float64)
    a = np.array([xy_m[0], xy_m[1], org[2] + radius])
    b = np.array([xy_m[0], xy_m[1], org[2] + height - radius])
    fa = to_fixed(a, org, grid.vox)
    fb = to_fixed(b, org, grid.vox)
    fr = int(np.rint(radius / grid.vox * 16.0))
    return np.array([fa[0], fa[1], fa[2], fb[0], fb[1], fb[2], fr], np.int32)


def walking_capsules(grid: Grid, H: int, T: int, rng, dt=0.1, speed=1.2, n_way=4, radius=0.25,
                     height=1.8):
    """int32 [T][H][7]: each human walks a polyline of n_way waypoints (uniform
    in xy with a margin of radius + 1 voxel); at step k its position is the
    point at arc length speed*dt*k along the polyline (held at the end)."""
    org = np.asarray(grid.origin, np.float64)
    ext = grid.extent
    margin = radius + grid.vox
    caps = np.zeros((T, H, 7), np.int32)
    for h in range(H):
        way = org[:2] + margin + rng.uniform(0.0, 1.0, size=(n_way, 2)) * (ext[:2] - 2 * margin)
        seg = np.diff(way, axis=0)
        seg_len = np.linalg.norm(seg, axis=1)
        cum = np.concatenate([[0.0], np.cumsum(seg_len)])
        for k in range(T):
            s = min(speed * dt * k, cum[-1])
            q = min(int(np.searchsorted(cum, s, side="right")) - 1, n_way - 2)
            frac = 0.0 if seg_len[q] == 0 else (s - cum[q]) / seg_len[q]
            xy = way[q] + frac * seg[q]
            caps[k, h] = standing_capsule(grid, xy, radius, height)
    return caps


def spheres_uniform(grid: Grid, N: int, rng, r_range=(0.05, 0.15)):
    """float32 [N,4]: centres uniform in the grid extent, radius uniform."""
    org = np.asarray(grid.origin, np.float64)
    c = org + rng.uniform(0.0, 1.0, size=(N, 3)) * grid.extent
    r = rng.uniform(r_range[0], r_range[1], size=(N, 1))
    return np.concatenate([c, r], axis=1).astype(np.float32)


def spheres_along_paths(grid: Grid, n_traj: int, n_states: int, n_spheres: int, rng, T: int,
                        sigma=0.1, r_range=(0.05, 0.15)):
    """Robot body spheres about straight-line trajectories.

    Returns (spheres float32 [n_traj, n_states, n_spheres, 4],
             tidx int32 [n_traj, n_states, n_spheres]) with tidx = min(state, T-1)."""
    org = np.asarray(grid.origin, np.float64)
    ext = grid.extent
    p0 = org + rng.uniform(0.1, 0.9, size=(n_traj, 1, 3)) * ext
    p1 = org + rng.uniform(0.1, 0.9, size=(n_traj, 1, 3)) * ext
    s = np.linspace(0.0, 1.0, n_states).reshape(1, n_states, 1)
    states = p0 + s * (p1 - p0)  # [n_traj, n_states, 3]
    offs = rng.normal(0.0, sigma, size=(n_traj, n_states, n_spheres, 3))
    c = states[:, :, None, :] + offs
    r = rng.uniform(r_range[0], r_range[1], size=(n_traj, n_states, n_spheres, 1))
    sph = np.concatenate([c, r], axis=-1).astype(np.float32)
    tidx = np.broadcast_to(np.minimum(np.arange(n_states), T - 1).reshape(1, n_states, 1),
                           (n_traj, n_states, n_spheres)).astype(np.int32).copy()
    return sph, tidx


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------

def scene_small(seed=0, T=1, n_spheres=1024):
    """64^3, 5 cm voxels, 10 boxes, one standing human (held still for T steps),
    n_spheres uniform spheres with tidx = 0."""
    rng = np.random.default_rng(seed)
    grid = Grid(64, 64, 64, 0.05)
    occ, _ = boxes_occupancy(grid, 10, rng)
    margin = 0.25 + grid.vox
    xy = margin + rng.uniform(0.0, 1.0, size=2) * (grid.extent[:2] - 2 * margin)
    cap = standing_capsule(grid, xy)
    caps = np.broadcast_to(cap.reshape(1, 1, 7), (T, 1, 7)).copy()
    spheres = spheres_uniform(grid, n_spheres, rng)
    tidx = np.zeros(n_spheres, np.int32)
    return dict(grid=grid, occ=occ, caps=caps, spheres=spheres, tidx=tidx, eps=0.2)


def scene_small_walking(seed=0, T=20, H=1):
    """64^3 scene as scene_small but with H humans walking over T steps."""
    rng = np.random.default_rng(seed)
    grid = Grid(64, 64, 64, 0.05)
    occ, _ = boxes_occupancy(grid, 10, rng)
    caps = walking_capsules(grid, H, T, rng)
    return dict(grid=grid, occ=occ, caps=caps, eps=0.2)


def scene_room(seed=0, T=20, H=3, nx=256, ny=256, nz=64, vox=0.05, n_boxes=160):
    """A room of 12.8 x 12.8 x 3.2 m in 5 cm voxels (the 64^3 scenes' voxel
    size and box density: 10 boxes per 64^3), H humans walking over T steps."""
    rng = np.random.default_rng(seed)
    grid = Grid(nx, ny, nz, vox)
    occ, _ = boxes_occupancy(grid, n_boxes, rng)
    caps = walking_capsules(grid, H, T, rng)
    return dict(grid=grid, occ=occ, caps=caps, eps=0.2)


def scene_composite(seed=0, n=256, vox=0.04, n_boxes=60, H=3, T=20):
    """256^3 grid of 4 cm voxels, 60 boxes, 3 walking humans over T = 20 steps."""
    rng = np.random.default_rng(seed)
    grid = Grid(n, n, n, vox)
    occ, _ = boxes_occupancy(grid, n_boxes, rng)
    caps = walking_capsules(grid, H, T, rng)
    return dict(grid=grid, occ=occ, caps=caps, eps=0.2)


def scene_batch(seed=0, n_env=64, vox=0.04, dims=((64, 320), (64, 320), (64, 128)), T_range=(5, 30),
                H_range=(1, 4)):
    """Ragged environments: per-axis integer sizes, horizon and human count
    uniform; boxes scale with volume as ceil(60 * V / 256^3)."""
    rng = np.random.default_rng(seed)
    envs = []
    for _ in range(n_env):
        nx = int(rng.integers(dims[0][0], dims[0][1] + 1))
        ny = int(rng.integers(dims[1][0], dims[1][1] + 1))
        nz = int(rng.integers(dims[2][0], dims[2][1] + 1))
        grid = Grid(nx, ny, nz, vox)
        T = int(rng.integers(T_range[0], T_range[1] + 1))
        H = int(rng.integers(H_range[0], H_range[1] + 1))
        nb = int(np.ceil(60 * grid.nvox / 256 ** 3))
        occ, _ = boxes_occupancy(grid, nb, rng)
        caps = walking_capsules(grid, H, T, rng)
        envs.append(dict(grid=grid, occ=occ, caps=caps))
    return envs


def random_occupancy(shape_zyx, density, rng):
    """uint8 occupancy with i.i.d. voxels (density in [0, 1])."""
    return (rng.uniform(0.0, 1.0, size=shape_zyx) < density).astype(np.uint8)


def lattice_moves(caps, ref):
    """caps [T][H][7] laid on the voxel lattice relative to the primitive ref:
    each primitive becomes ref moved by the whole-voxel step nearest to its own
    displacement from ref (same shape and sub-voxel phase as ref).  The input
    of the translated-primitive variant, where a predicted position is an
    integer voxel move of one template."""
    caps = np.asarray(caps, np.int64)
    ref = np.asarray(ref, np.int64).reshape(7)
    move = np.rint((caps[..., 0:3] - ref[0:3]) / 16.0).astype(np.int64)
    out = np.empty(caps.shape, np.int64)
    out[..., 0:3] = ref[0:3] + 16 * move
    out[..., 3:6] = ref[3:6] + 16 * move
    out[..., 6] = ref[6]
    return out.astype(np.int32)
