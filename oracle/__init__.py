"""CPU oracle for predicted composite distance fields (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product (``paper_2201_05058_gb300``) never imports it and shares no code with
it; the two meet only through the seeded inputs of ``scenes.py``.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, see its header
for the definitions it follows); this module compiles it with gcc on first use
and exposes numpy-friendly wrappers.  A few definitions are also written here
in numpy where a plain array expression states them directly.

Paper passages followed (Finean et al., arXiv 2201.05058):
  * Sec. 6: the composite field is a per-voxel ``min`` of the environment field
    and the field of each dynamic obstacle at its predicted position; the
    human primitive is a cylinder (read here as a capsule).
  * Sec. 7, hinge-loss obstacle factor (GPMP2 form): cost ``eps - d`` when the
    distance ``d`` is within ``eps``, else 0; the sphere radius is added to eps.
  * Sec. 8: obstacle factor i reads composite field ``min(i, n)``.
  * Sec. 6, the primitive's field computed once: ``template_field`` is the
    signed EDT of one primitive on a box around it, ``translated_composite``
    places copies of it at integer voxel offsets and takes the same ``min``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF32 = 2147483647


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (plain -O2, no fast-math,
    no FMA contraction, so the fp32 float field is IEEE on every host)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, f32, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
            lib.or_capsule_inside.argtypes = [i64, i64, i64, P]
            lib.or_capsule_inside.restype = ctypes.c_int
            lib.or_capsule_occupancy.argtypes = [ctypes.c_int] * 4 + [P, P]
            lib.or_edt_at.argtypes = [ctypes.c_int] * 3 + [P] + [ctypes.c_int] * 3
            lib.or_edt_at.restype = i32
            lib.or_edt_brute.argtypes = [ctypes.c_int] * 3 + [P, P]
            lib.or_edt_separable.argtypes = [ctypes.c_int] * 3 + [P, P]
            lib.or_composite.argtypes = [sz, P, P, P]
            lib.or_sdf_from_sq.argtypes = [sz, P, f32, P]
            lib.or_trilinear.argtypes = [P] + [ctypes.c_int] * 3 + [P, f32, P, P, P]
            lib.or_trilinear.restype = ctypes.c_double
            lib.or_hinge_cost.argtypes = [P, ctypes.c_int] + [ctypes.c_int] * 3 + [P, f32, P, P, i64, f32, P, P, P]
            lib.or_hinge_cost.restype = i64
            lib.or_voxel_filter.argtypes = [ctypes.c_int] * 3 + [P, ctypes.c_int, P]
            lib.or_collapse.argtypes = [ctypes.c_int] * 3 + [P, ctypes.c_int, ctypes.c_int, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# capsules
# --------------------------------------------------------------------------

def capsule_inside(p, cap) -> bool:
    """Exact int64 test: fixed-point point p inside capsule cap (7 int32)."""
    cap = _c(cap, np.int32)
    return bool(_load().or_capsule_inside(int(p[0]), int(p[1]), int(p[2]), _ptr(cap)))


def capsule_occupancy(shape_zyx, caps) -> np.ndarray:
    """uint8 [nz,ny,nx] occupancy of the voxels whose centres lie inside any capsule."""
    nz, ny, nx = shape_zyx
    caps = _c(np.asarray(caps).reshape(-1, 7), np.int32)
    occ = np.zeros((nz, ny, nx), np.uint8)
    _load().or_capsule_occupancy(nx, ny, nz, caps.shape[0], _ptr(caps), _ptr(occ))
    return occ


# --------------------------------------------------------------------------
# signed squared EDT
# --------------------------------------------------------------------------

def edt_brute(occ) -> np.ndarray:
    """Signed squared EDT by its definition (O(V * |opposite set|))."""
    occ = _c(occ, np.uint8)
    nz, ny, nx = occ.shape
    S = np.empty(occ.shape, np.int32)
    _load().or_edt_brute(nx, ny, nz, _ptr(occ), _ptr(S))
    return S


def edt_at(occ, i, j, k) -> int:
    """Signed squared EDT at voxel (i, j, k) by its definition (O(V))."""
    occ = _c(occ, np.uint8)
    nz, ny, nx = occ.shape
    return int(_load().or_edt_at(nx, ny, nz, _ptr(occ), int(i), int(j), int(k)))


def edt(occ) -> np.ndarray:
    """Signed squared EDT by the separable lower-envelope algorithm."""
    occ = _c(occ, np.uint8)
    nz, ny, nx = occ.shape
    S = np.empty(occ.shape, np.int32)
    _load().or_edt_separable(nx, ny, nz, _ptr(occ), _ptr(S))
    return S


def sdf_from_sq(S, vox: float) -> np.ndarray:
    """float32 field sign(S)*sqrtf(|S|)*vox, +/-INT32_MAX -> +/-inf."""
    S = _c(S, np.int32)
    out = np.empty(S.shape, np.float32)
    _load().or_sdf_from_sq(S.size, _ptr(S), ctypes.c_float(vox), _ptr(out))
    return out


# --------------------------------------------------------------------------
# composite (Sec. 6) and the per-timestep fields
# --------------------------------------------------------------------------

def composite(S_static, S_dyn) -> np.ndarray:
    a = _c(S_static, np.int32)
    b = _c(S_dyn, np.int32)
    assert a.shape == b.shape
    out = np.empty(a.shape, np.int32)
    _load().or_composite(a.size, _ptr(a), _ptr(b), _ptr(out))
    return out


def dynamic_field(shape_zyx, caps_t) -> np.ndarray:
    """Signed squared EDT of the capsule-only occupancy at one time."""
    return edt(capsule_occupancy(shape_zyx, caps_t))


def predicted_composite(S_static, caps) -> np.ndarray:
    """comp[t] = min(S_static, S_dyn[t]) for caps [T][H][7]."""
    caps = np.asarray(caps, np.int32)
    T = caps.shape[0]
    out = np.empty((T,) + S_static.shape, np.int32)
    for t in range(T):
        out[t] = composite(S_static, dynamic_field(S_static.shape, caps[t]))
    return out


def from_scratch(occ, caps) -> np.ndarray:
    """S_t = signed EDT of (occ OR capsules at t), recomputed for every t."""
    caps = np.asarray(caps, np.int32)
    T = caps.shape[0]
    out = np.empty((T,) + occ.shape, np.int32)
    for t in range(T):
        u = capsule_occupancy(occ.shape, caps[t]) | (np.asarray(occ) != 0).astype(np.uint8)
        out[t] = edt(u)
    return out


# --------------------------------------------------------------------------
# translated primitive field (Sec. 6: the field of the human primitive is
# computed once and composited at each predicted position)
# --------------------------------------------------------------------------

CYLINDER = 1 << 30


def template_box(cap, R: int):
    """(lo, dims), both (x, y, z) voxel indices: the box of voxels whose centres
    16*i + 8 can lie in the primitive, i.e. within [min(a, b) - r, max(a, b) + r]
    on each axis, widened by R voxels on every side.  Not clipped to any grid.
    Raises ValueError when no voxel centre lies in that range on some axis."""
    cap = [int(v) for v in np.asarray(cap).reshape(7)]
    r = cap[6] & ~CYLINDER
    lo, dims = [], []
    for a in range(3):
        mn = min(cap[a], cap[3 + a]) - r
        mx = max(cap[a], cap[3 + a]) + r
        first = -((8 - mn) // 16)  # ceil((mn - 8) / 16)
        last = (mx - 8) // 16      # floor((mx - 8) / 16)
        if last < first:
            raise ValueError("no voxel centre within the primitive's range on axis %d" % a)
        lo.append(first - R)
        dims.append(last - first + 1 + 2 * R)
    return lo, dims


def template_field(cap, R: int):
    """(tmpl, lo): the signed squared EDT of the primitive's voxels on its
    template box (int32 [dz][dy][dx]), and the map index of the box's voxel 0.
    Template voxel (i, j, k) is map voxel lo + (i, j, k); the primitive is moved
    into the box's frame by subtracting 16*lo from a and b."""
    lo, dims = template_box(cap, R)
    c = np.asarray(cap, np.int64).reshape(7).copy()
    for a in range(3):
        c[a] -= 16 * lo[a]
        c[3 + a] -= 16 * lo[a]
    occ = capsule_occupancy((dims[2], dims[1], dims[0]), c.astype(np.int32))
    return edt(occ), lo


def translated_composite(S_static, tmpl, lo) -> np.ndarray:
    """comp[t] = min(S_static, min_h P_th) where P_th(v) = tmpl[v - lo[t][h]]
    inside the template box placed at lo[t][h] ((x, y, z) map index of its
    voxel 0) and +INF outside it.  lo: int [T][H][3]."""
    S_static = np.asarray(S_static, np.int32)
    tmpl = np.asarray(tmpl, np.int32)
    lo = np.asarray(lo, np.int64)
    T, H = lo.shape[0], lo.shape[1]
    nz, ny, nx = S_static.shape
    dz, dy, dx = tmpl.shape
    out = np.empty((T, nz, ny, nx), np.int32)
    for t in range(T):
        dyn = np.full(S_static.shape, INF32, np.int32)
        for h in range(H):
            x0, y0, z0 = (int(v) for v in lo[t, h])
            xa, xb = max(x0, 0), min(x0 + dx, nx)
            ya, yb = max(y0, 0), min(y0 + dy, ny)
            za, zb = max(z0, 0), min(z0 + dz, nz)
            if xa >= xb or ya >= yb or za >= zb:
                continue
            sub = tmpl[za - z0:zb - z0, ya - y0:yb - y0, xa - x0:xb - x0]
            dyn[za:zb, ya:yb, xa:xb] = np.minimum(dyn[za:zb, ya:yb, xa:xb], sub)
        out[t] = composite(S_static, dyn)
    return out


# --------------------------------------------------------------------------
# trilinear hinge cost (Sec. 7 / Sec. 8)
# --------------------------------------------------------------------------

def trilinear(field, origin, vox, p):
    """(d, oob, grad) at one point of one [nz,ny,nx] float32 field."""
    field = _c(field, np.float32)
    nz, ny, nx = field.shape
    o = _c(origin, np.float32)
    pp = _c(p, np.float32)
    oob = ctypes.c_int(0)
    g = np.zeros(3, np.float64)
    d = _load().or_trilinear(_ptr(field), nx, ny, nz, _ptr(o), ctypes.c_float(vox), _ptr(pp),
                             ctypes.byref(oob), _ptr(g))
    return d, bool(oob.value), g


def hinge_cost(sdf, origin, vox, spheres, tidx, eps, need_grad=False):
    """h[N] (float64), n_oob and optionally (grad_c [N,3], grad_r [N]).

    sdf is float32 [T,nz,ny,nx] (or [nz,ny,nx] for T = 1); spheres float32 [N,4];
    tidx int32 [N]."""
    sdf = _c(sdf, np.float32)
    if sdf.ndim == 3:
        sdf = sdf[None]
    T, nz, ny, nx = sdf.shape
    sph = _c(spheres, np.float32).reshape(-1, 4)
    N = sph.shape[0]
    ti = _c(tidx, np.int32).reshape(-1)
    assert ti.shape[0] == N
    o = _c(origin, np.float32)
    h = np.empty(N, np.float64)
    gc = np.empty((N, 3), np.float64) if need_grad else None
    gr = np.empty(N, np.float64) if need_grad else None
    n_oob = _load().or_hinge_cost(_ptr(sdf), T, nx, ny, nz, _ptr(o), ctypes.c_float(vox), _ptr(sph), _ptr(ti),
                                  N, ctypes.c_float(eps), _ptr(h),
                                  _ptr(gc) if need_grad else None, _ptr(gr) if need_grad else None)
    if need_grad:
        return h, int(n_oob), gc, gr
    return h, int(n_oob)


def voxel_filter(occ, min_neighbours: int = 5) -> np.ndarray:
    """Sec. 8 clean-up: keep an occupied voxel iff at least min_neighbours of
    its 26 in-grid neighbours are occupied."""
    o = _c(occ, np.uint8)
    nz, ny, nx = o.shape
    out = np.empty_like(o)
    _load().or_voxel_filter(nx, ny, nz, _ptr(o), int(min_neighbours), _ptr(out))
    return out


def collapse(occ, z0: int, z1: int) -> np.ndarray:
    """Sec. 8 2-D map: uint8 [ny, nx], a column occupied iff some voxel of it
    in slices [z0, z1) is."""
    o = _c(occ, np.uint8)
    nz, ny, nx = o.shape
    out = np.empty((ny, nx), np.uint8)
    _load().or_collapse(nx, ny, nz, _ptr(o), int(z0), int(z1), _ptr(out))
    return out
