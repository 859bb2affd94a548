"""Python binding of the C ABI (argument marshalling only).

Every function here checks tensor placement, dtype and shape, takes the
workspace from PyTorch's caching allocator, passes raw pointers and the
current CUDA stream to ``libpcdf.so`` and raises if the library reports an
error.  No step of the computation runs in Python or PyTorch.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


@dataclass(frozen=True)
class Grid:
    """Voxel grid: nx, ny, nz voxels of edge ``vox`` metres, corner at ``origin``."""
    nx: int
    ny: int
    nz: int
    vox: float
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def _cgrid(g) -> _lib.PcdfGrid:
    o = tuple(float(v) for v in getattr(g, "origin", (0.0, 0.0, 0.0)))
    return _lib.PcdfGrid(int(g.nx), int(g.ny), int(g.nz), float(g.vox), (ctypes.c_float * 3)(*o))


def _shape(g):
    return (int(g.nz), int(g.ny), int(g.nx))


def _stream(dev: torch.device) -> int:
    return torch.cuda.current_stream(dev).cuda_stream


def _need(t: torch.Tensor, name: str, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _caps_host(caps):
    """int32 [T][H][7] capsules as a contiguous host array (or None for H = 0)."""
    if isinstance(caps, torch.Tensor):
        caps = caps.detach().cpu().numpy()
    caps = np.ascontiguousarray(np.asarray(caps), dtype=np.int32)
    if caps.ndim != 3 or caps.shape[2] != 7:
        raise ValueError(f"caps must be [T][H][7], got {caps.shape}")
    return caps


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _workspace(nbytes: int, dev) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)


CYLINDER = 1 << 30  # radius-word flag of PCDF_CYLINDER


def capsule_fixed(a_m, b_m, r_m, grid, cylinder: bool = False) -> np.ndarray:
    """Capsule(s) from metres to the library's 1/16-voxel fixed point.

    a_m, b_m: [..., 3] segment end points (world metres); r_m: [...] radius
    (per time step for a radius that grows over the horizon).  cylinder: the
    finite cylinder with flat ends at a and b (the paper's primitive) instead
    of the capsule.  Returns int32 [..., 7] (round half to even of
    (x - origin) / vox * 16)."""
    o = np.asarray(getattr(grid, "origin", (0.0, 0.0, 0.0)), np.float64)
    a = np.rint((np.asarray(a_m, np.float64) - o) / grid.vox * 16.0)
    b = np.rint((np.asarray(b_m, np.float64) - o) / grid.vox * 16.0)
    r = np.rint(np.asarray(r_m, np.float64) / grid.vox * 16.0)[..., None]
    out = np.concatenate([a, b, r], axis=-1).astype(np.int32)
    if cylinder:
        out[..., 6] |= CYLINDER
    return out


# ---------------------------------------------------------------------------
# fields
# ---------------------------------------------------------------------------

def build_static_sdf(occ: torch.Tensor, grid, want_sdf: bool = True, out_sq=None, out_sdf=None):
    """Signed squared EDT (int32) and float field (fp32, metres) of a static map.

    occ: CUDA uint8 [nz, ny, nx], nonzero = occupied."""
    shp = _shape(grid)
    _need(occ, "occ", torch.uint8, shp)
    dev = occ.device
    lib = _lib.load()
    g = _cgrid(grid)
    nbytes = ctypes.c_size_t(0)
    _lib.check(lib.pcdf_static_workspace_bytes(ctypes.byref(g), ctypes.byref(nbytes)), "static workspace")
    sq = out_sq if out_sq is not None else torch.empty(shp, dtype=torch.int32, device=dev)
    _need(sq, "static_sq", torch.int32, shp)
    sdf = None
    if want_sdf:
        sdf = out_sdf if out_sdf is not None else torch.empty(shp, dtype=torch.float32, device=dev)
        _need(sdf, "static_sdf", torch.float32, shp)
    ws = _workspace(nbytes.value, dev)
    _lib.check(lib.pcdf_build_static_sdf(ctypes.byref(g), _ptr(occ), _ptr(sq), _ptr(sdf), _ptr(ws), ws.numel(),
                                         ctypes.c_void_p(_stream(dev))), "pcdf_build_static_sdf")
    return sq, sdf


def filter_voxels(occ: torch.Tensor, grid, min_neighbours: int = 5, out=None) -> torch.Tensor:
    """Sec. 8 static-map clean-up: occupied voxels with fewer than
    min_neighbours occupied voxels among their 26 neighbours are cleared.
    occ: CUDA uint8 [nz, ny, nx]; returns uint8 0/1 of the same shape."""
    shp = _shape(grid)
    _need(occ, "occ", torch.uint8, shp)
    out = out if out is not None else torch.empty_like(occ)
    _need(out, "out", torch.uint8, shp)
    g = _cgrid(grid)
    _lib.check(_lib.load().pcdf_filter_voxels(ctypes.byref(g), _ptr(occ), int(min_neighbours), _ptr(out),
                                              ctypes.c_void_p(_stream(occ.device))), "pcdf_filter_voxels")
    return out


def collapse_2d(occ: torch.Tensor, grid, z0: int, z1: int) -> torch.Tensor:
    """Sec. 8 2-D map: uint8 [ny, nx], a column occupied iff one of its voxels
    in slices [z0, z1) is."""
    _need(occ, "occ", torch.uint8, _shape(grid))
    out = torch.empty((grid.ny, grid.nx), dtype=torch.uint8, device=occ.device)
    g = _cgrid(grid)
    _lib.check(_lib.load().pcdf_collapse_2d(ctypes.byref(g), _ptr(occ), int(z0), int(z1), _ptr(out),
                                            ctypes.c_void_p(_stream(occ.device))), "pcdf_collapse_2d")
    return out


def edt_2d(occ: torch.Tensor, grid, z0: int, z1: int, want_sdf: bool = True):
    """The prediction module's 2-D EDT (Sec. 8): the signed squared EDT (and
    float field) of the grid collapsed over slices [z0, z1).  Returns
    (int32 [ny, nx], fp32 [ny, nx] or None)."""
    c = collapse_2d(occ, grid, z0, z1)
    g2 = Grid(grid.nx, grid.ny, 1, grid.vox, tuple(getattr(grid, "origin", (0.0, 0.0, 0.0))))
    sq, sdf = build_static_sdf(c.view(1, grid.ny, grid.nx), g2, want_sdf=want_sdf)
    return sq.view(grid.ny, grid.nx), (sdf.view(grid.ny, grid.nx) if sdf is not None else None)


def build_predicted_composite(static_sq: torch.Tensor, grid, caps, want_sq: bool = True, want_sdf: bool = True,
                              out_sq=None, out_sdf=None, static_sdf=None):
    """Composite fields comp[t] = min(static, capsules at t) for t < T (Sec. 6, 8).

    static_sq: CUDA int32 [nz, ny, nx]; caps: host int32 [T][H][7] fixed point;
    static_sdf: optional float field built with static_sq (reused where the
    static field wins).  Returns (comp_sq int32 [T, nz, ny, nx] or None,
    comp_sdf fp32 or None)."""
    shp = _shape(grid)
    _need(static_sq, "static_sq", torch.int32, shp)
    if static_sdf is not None:
        _need(static_sdf, "static_sdf", torch.float32, shp)
    caps = _caps_host(caps)
    T, H = int(caps.shape[0]), int(caps.shape[1])
    dev = static_sq.device
    lib = _lib.load()
    g = _cgrid(grid)
    cp = caps.ctypes.data_as(ctypes.c_void_p) if H > 0 else None
    nbytes = ctypes.c_size_t(0)
    _lib.check(lib.pcdf_composite_workspace_bytes(ctypes.byref(g), T, H, cp, ctypes.byref(nbytes)),
               "composite workspace")
    sq = sdf = None
    if want_sq:
        sq = out_sq if out_sq is not None else torch.empty((T,) + shp, dtype=torch.int32, device=dev)
        _need(sq, "comp_sq", torch.int32, (T,) + shp)
    if want_sdf:
        sdf = out_sdf if out_sdf is not None else torch.empty((T,) + shp, dtype=torch.float32, device=dev)
        _need(sdf, "comp_sdf", torch.float32, (T,) + shp)
    ws = _workspace(nbytes.value, dev)
    _lib.check(lib.pcdf_build_predicted_composite(ctypes.byref(g), _ptr(static_sq), _ptr(static_sdf), T, H, cp,
                                                  _ptr(sq), _ptr(sdf),
                                                  _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(dev))),
               "pcdf_build_predicted_composite")
    return sq, sdf


def composite_workspace(grid, caps, device) -> torch.Tensor:
    """A device workspace large enough for build_predicted_composite / the stages."""
    caps = _caps_host(caps)
    T, H = int(caps.shape[0]), int(caps.shape[1])
    g = _cgrid(grid)
    cp = caps.ctypes.data_as(ctypes.c_void_p) if H > 0 else None
    nbytes = ctypes.c_size_t(0)
    _lib.check(_lib.load().pcdf_composite_workspace_bytes(ctypes.byref(g), T, H, cp, ctypes.byref(nbytes)),
               "composite workspace")
    return _workspace(nbytes.value, device)


def composite_slab(grid, caps):
    """(zlo, S): the z-slab of voxel slices that the capsules touch."""
    caps = _caps_host(caps)
    T, H = int(caps.shape[0]), int(caps.shape[1])
    g = _cgrid(grid)
    cp = caps.ctypes.data_as(ctypes.c_void_p) if H > 0 else None
    zlo, S = ctypes.c_int32(0), ctypes.c_int32(0)
    _lib.check(_lib.load().pcdf_composite_slab(ctypes.byref(g), T, H, cp, ctypes.byref(zlo), ctypes.byref(S)),
               "pcdf_composite_slab")
    return zlo.value, S.value


def composite_prepare(grid, caps, workspace: torch.Tensor):
    """First stage of the composite: capsule row pass and y pass into workspace."""
    caps = _caps_host(caps)
    T, H = int(caps.shape[0]), int(caps.shape[1])
    _need(workspace, "workspace", torch.uint8)
    g = _cgrid(grid)
    cp = caps.ctypes.data_as(ctypes.c_void_p) if H > 0 else None
    _lib.check(_lib.load().pcdf_composite_prepare(ctypes.byref(g), T, H, cp, _ptr(workspace), workspace.numel(),
                                                  ctypes.c_void_p(_stream(workspace.device))),
               "pcdf_composite_prepare")


def composite_finish(static_sq, grid, caps, workspace: torch.Tensor, comp_sq=None, comp_sdf=None, static_sdf=None,
                     t_range=None):
    """Second stage: fused z pass + composite min + float epilogue into the
    given outputs ([T, ...] arrays); t_range = (t0, nt) writes only the
    fields t0 .. t0 + nt - 1."""
    shp = _shape(grid)
    caps = _caps_host(caps)
    T, H = int(caps.shape[0]), int(caps.shape[1])
    _need(static_sq, "static_sq", torch.int32, shp)
    if static_sdf is not None:
        _need(static_sdf, "static_sdf", torch.float32, shp)
    _need(workspace, "workspace", torch.uint8)
    if comp_sq is not None:
        _need(comp_sq, "comp_sq", torch.int32, (T,) + shp)
    if comp_sdf is not None:
        _need(comp_sdf, "comp_sdf", torch.float32, (T,) + shp)
    g = _cgrid(grid)
    cp = caps.ctypes.data_as(ctypes.c_void_p) if H > 0 else None
    if t_range is None:
        _lib.check(_lib.load().pcdf_composite_finish(ctypes.byref(g), _ptr(static_sq), _ptr(static_sdf), T, H, cp,
                                                     _ptr(comp_sq), _ptr(comp_sdf), _ptr(workspace),
                                                     workspace.numel(), ctypes.c_void_p(_stream(static_sq.device))),
                   "pcdf_composite_finish")
    else:
        t0, nt = (int(v) for v in t_range)
        _lib.check(_lib.load().pcdf_composite_finish_range(ctypes.byref(g), _ptr(static_sq), _ptr(static_sdf), T, H,
                                                           cp, t0, nt, _ptr(comp_sq), _ptr(comp_sdf),
                                                           _ptr(workspace), workspace.numel(),
                                                           ctypes.c_void_p(_stream(static_sq.device))),
                   "pcdf_composite_finish_range")


_side_streams = {}


def _side_stream(dev):
    st = _side_streams.get(dev.index)
    if st is None:
        st = torch.cuda.Stream(device=dev)
        _side_streams[dev.index] = st
    return st


def update_workspace(grid, caps, device) -> torch.Tensor:
    """Workspace of predicted_fields (pcdf_update_workspace_bytes)."""
    caps = _caps_host(caps)
    T, H = int(caps.shape[0]), int(caps.shape[1])
    g = _cgrid(grid)
    cp = caps.ctypes.data_as(ctypes.c_void_p) if H > 0 else None
    n = ctypes.c_size_t(0)
    _lib.check(_lib.load().pcdf_update_workspace_bytes(ctypes.byref(g), T, H, cp, ctypes.byref(n)),
               "pcdf_update_workspace_bytes")
    return _workspace(n.value, torch.device(device))


def predicted_fields(occ: torch.Tensor, grid, caps, workspace=None, out_static_sq=None, out_static_sdf=None,
                     out_sq=None, out_sdf=None):
    """One map update (Sec. 6, Sec. 8): the static field of `occ` and the T
    composite fields with the capsules `caps` (host int32 [T][H][7]), through
    pcdf_update_fields on the current stream and a side stream (the capsule
    pass beside the static build).  Returns (static_sq, static_sdf, comp_sq,
    comp_sdf); `workspace` (from update_workspace) and the outputs may be
    passed in to reuse them."""
    dev = occ.device
    caps = _caps_host(caps)
    T, H = int(caps.shape[0]), int(caps.shape[1])
    shp = _shape(grid)
    _need(occ, "occ", torch.uint8, shp)
    ws = workspace if workspace is not None else update_workspace(grid, caps, dev)
    st_sq = out_static_sq if out_static_sq is not None else torch.empty(shp, dtype=torch.int32, device=dev)
    st_sdf = out_static_sdf if out_static_sdf is not None else torch.empty(shp, dtype=torch.float32, device=dev)
    sq = out_sq if out_sq is not None else torch.empty((T,) + shp, dtype=torch.int32, device=dev)
    sdf = out_sdf if out_sdf is not None else torch.empty((T,) + shp, dtype=torch.float32, device=dev)
    _need(st_sq, "static_sq", torch.int32, shp)
    _need(st_sdf, "static_sdf", torch.float32, shp)
    _need(sq, "comp_sq", torch.int32, (T,) + shp)
    _need(sdf, "comp_sdf", torch.float32, (T,) + shp)
    main = torch.cuda.current_stream(dev)
    side = _side_stream(dev)
    g = _cgrid(grid)
    cp = caps.ctypes.data_as(ctypes.c_void_p) if H > 0 else None
    _lib.check(_lib.load().pcdf_update_fields(ctypes.byref(g), _ptr(occ), T, H, cp, _ptr(st_sq), _ptr(st_sdf),
                                              _ptr(sq), _ptr(sdf), _ptr(ws), ws.numel(),
                                              ctypes.c_void_p(main.cuda_stream), ctypes.c_void_p(side.cuda_stream)),
               "pcdf_update_fields")
    ws.record_stream(side)
    for t_ in (st_sq, st_sdf, sq, sdf, occ):
        t_.record_stream(side)
    return st_sq, st_sdf, sq, sdf


_copy_streams = {}


def _copy_stream(dev):
    st = _copy_streams.get(dev.index)
    if st is None:
        st = torch.cuda.Stream(device=dev)
        _copy_streams[dev.index] = st
    return st


def update_to_host(occ_host: torch.Tensor, grid, caps, out_host: torch.Tensor, buffers: dict, chunk: int = 4):
    """One map update with host buffers: the occupancy comes from pinned host
    memory (uint8 [nz, ny, nx]) and the T float composite fields go to pinned
    host memory (out_host fp32 [T, nz, ny, nx]).

    `buffers` holds the device tensors, reused between calls: "occ" (uint8),
    "static_sq", "static_sdf", "comp_sq" (optional), "comp_sdf" and
    "workspace" (composite_workspace).  The static build and the capsule pass
    overlap as in predicted_fields; the z pass then runs `chunk` time steps at
    a time, and each finished chunk is copied to the host on a copy stream
    while the next one is computed.  The current stream waits for every copy
    (synchronise it before reading out_host)."""
    caps = _caps_host(caps)
    T = int(caps.shape[0])
    occ_d, ws = buffers["occ"], buffers["workspace"]
    st_sq, st_sdf = buffers["static_sq"], buffers["static_sdf"]
    comp_sq, comp_sdf = buffers.get("comp_sq"), buffers["comp_sdf"]
    dev = occ_d.device
    if (out_host.is_cuda or out_host.dtype != torch.float32 or not out_host.is_contiguous()
            or tuple(out_host.shape) != (T,) + _shape(grid)):
        raise ValueError(f"out_host must be a contiguous host float32 tensor of shape {(T,) + _shape(grid)}")
    main = torch.cuda.current_stream(dev)
    occ_d.copy_(occ_host, non_blocking=True)
    side = _side_stream(dev)
    side.wait_stream(main)
    with torch.cuda.stream(side):
        composite_prepare(grid, caps, ws)
    build_static_sdf(occ_d, grid, out_sq=st_sq, out_sdf=st_sdf)
    main.wait_stream(side)
    cp = _copy_stream(dev)
    for t0 in range(0, T, chunk):
        nt = min(chunk, T - t0)
        composite_finish(st_sq, grid, caps, ws, comp_sq, comp_sdf, static_sdf=st_sdf, t_range=(t0, nt))
        cp.wait_stream(main)
        with torch.cuda.stream(cp):
            out_host[t0:t0 + nt].copy_(comp_sdf[t0:t0 + nt], non_blocking=True)
    main.wait_stream(cp)


def build_from_scratch(occ: torch.Tensor, grid, caps, want_sdf: bool = True, out_sq=None, out_sdf=None):
    """The comparator: full signed EDT of (occ OR capsules at t) for every t."""
    shp = _shape(grid)
    _need(occ, "occ", torch.uint8, shp)
    caps = _caps_host(caps)
    T, H = int(caps.shape[0]), int(caps.shape[1])
    dev = occ.device
    lib = _lib.load()
    g = _cgrid(grid)
    cp = caps.ctypes.data_as(ctypes.c_void_p) if H > 0 else None
    nbytes = ctypes.c_size_t(0)
    _lib.check(lib.pcdf_scratch_workspace_bytes(ctypes.byref(g), T, H, ctypes.byref(nbytes)), "scratch workspace")
    sq = out_sq if out_sq is not None else torch.empty((T,) + shp, dtype=torch.int32, device=dev)
    _need(sq, "sq", torch.int32, (T,) + shp)
    sdf = None
    if want_sdf:
        sdf = out_sdf if out_sdf is not None else torch.empty((T,) + shp, dtype=torch.float32, device=dev)
        _need(sdf, "sdf", torch.float32, (T,) + shp)
    ws = _workspace(nbytes.value, dev)
    _lib.check(lib.pcdf_build_from_scratch(ctypes.byref(g), _ptr(occ), T, H, cp, _ptr(sq), _ptr(sdf), _ptr(ws),
                                           ws.numel(), ctypes.c_void_p(_stream(dev))), "pcdf_build_from_scratch")
    return sq, sdf


# ---------------------------------------------------------------------------
# translated primitive field (Sec. 6: the primitive's field computed once)
# ---------------------------------------------------------------------------

def _cap7(cap) -> np.ndarray:
    c = np.asarray(cap.detach().cpu().numpy() if isinstance(cap, torch.Tensor) else cap, dtype=np.int64)
    if c.size != 7:
        raise ValueError(f"a primitive is 7 int32 values, got {c.shape}")
    return np.ascontiguousarray(c.reshape(7), dtype=np.int32)


def template_box(cap, R: int):
    """(lo, dims), each [x, y, z]: the template box of primitive cap (the voxels
    whose centres can lie in it, widened by R voxels) in map voxel indices."""
    c = _cap7(cap)
    lo = (ctypes.c_int32 * 3)()
    dims = (ctypes.c_int32 * 3)()
    _lib.check(_lib.load().pcdf_template_box(c.ctypes.data_as(ctypes.c_void_p), int(R), lo, dims),
               "pcdf_template_box")
    return list(lo), list(dims)


def build_template(cap, R: int, device):
    """(tmpl, lo): the signed squared EDT of primitive cap on its template box,
    int32 [dz][dy][dx] on `device`, and the box's map index [x, y, z]."""
    c = _cap7(cap)
    lo, dims = template_box(c, R)
    dev = torch.device(device)
    lib = _lib.load()
    nbytes = ctypes.c_size_t(0)
    cp = c.ctypes.data_as(ctypes.c_void_p)
    _lib.check(lib.pcdf_template_workspace_bytes(cp, int(R), ctypes.byref(nbytes)), "template workspace")
    tmpl = torch.empty((dims[2], dims[1], dims[0]), dtype=torch.int32, device=dev)
    ws = _workspace(nbytes.value, dev)
    _lib.check(lib.pcdf_build_template(cp, int(R), _ptr(tmpl), _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(dev))),
               "pcdf_build_template")
    return tmpl, lo


def template_radius(static_sq: torch.Tensor) -> int:
    """Least R with R * R at least every finite positive static value: with a box
    widened by R, the translated composite is exact wherever the static field
    is finite (one device-to-host read)."""
    _need(static_sq, "static_sq", torch.int32)
    out = torch.empty(1, dtype=torch.int32, device=static_sq.device)
    _lib.check(_lib.load().pcdf_field_max(_ptr(static_sq), static_sq.numel(), _ptr(out),
                                          ctypes.c_void_p(_stream(static_sq.device))), "pcdf_field_max")
    R = ctypes.c_int32(0)
    _lib.check(_lib.load().pcdf_template_radius(int(out.item()), ctypes.byref(R)), "pcdf_template_radius")
    return int(R.value)


def lattice_placements(caps, ref_cap, ref_lo) -> np.ndarray:
    """Box placements int32 [T][H][3] for primitives that are ref_cap moved by
    whole voxels (the template built from ref_cap has its box at ref_lo).
    Raises ValueError for a primitive of another shape or a sub-voxel move."""
    c = _caps_host(caps)
    ref = _cap7(ref_cap)
    rlo = np.ascontiguousarray(np.asarray(ref_lo, np.int64), dtype=np.int32)
    T, H = int(c.shape[0]), int(c.shape[1])
    lo = np.empty((T, H, 3), np.int32)
    rc = _lib.load().pcdf_lattice_placements(c.ctypes.data_as(ctypes.c_void_p), T, H,
                                             ref.ctypes.data_as(ctypes.c_void_p),
                                             rlo.ctypes.data_as(ctypes.c_void_p), lo.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError(_lib.load().pcdf_last_error().decode())
    return lo


def composite_translated(static_sq: torch.Tensor, grid, tmpl: torch.Tensor, lo, R: int, static_sdf=None,
                         want_sq: bool = True, want_sdf: bool = True, comp_sq=None, comp_sdf=None):
    """comp[t] = min(static, min_h template placed at lo[t][h]) for lo int [T][H][3];
    R is the widening the template was built with (see
    pcdf_composite_translated for when this equals the exact composite)."""
    shp = _shape(grid)
    _need(static_sq, "static_sq", torch.int32, shp)
    if static_sdf is not None:
        _need(static_sdf, "static_sdf", torch.float32, shp)
    _need(tmpl, "tmpl", torch.int32)
    if tmpl.dim() != 3:
        raise ValueError("tmpl must be [dz][dy][dx]")
    lo = np.ascontiguousarray(np.asarray(lo, dtype=np.int64), dtype=np.int32)
    if lo.ndim != 3 or lo.shape[2] != 3:
        raise ValueError(f"lo must be [T][H][3], got {lo.shape}")
    T, H = int(lo.shape[0]), int(lo.shape[1])
    dev = static_sq.device
    if want_sq and comp_sq is None:
        comp_sq = torch.empty((T,) + shp, dtype=torch.int32, device=dev)
    if want_sdf and comp_sdf is None:
        comp_sdf = torch.empty((T,) + shp, dtype=torch.float32, device=dev)
    if comp_sq is not None:
        _need(comp_sq, "comp_sq", torch.int32, (T,) + shp)
    if comp_sdf is not None:
        _need(comp_sdf, "comp_sdf", torch.float32, (T,) + shp)
    dims = (ctypes.c_int32 * 3)(int(tmpl.shape[2]), int(tmpl.shape[1]), int(tmpl.shape[0]))
    g = _cgrid(grid)
    _lib.check(_lib.load().pcdf_composite_translated(
        ctypes.byref(g), _ptr(static_sq), _ptr(static_sdf), T, H, _ptr(tmpl), dims, int(R),
        lo.ctypes.data_as(ctypes.c_void_p) if H > 0 else None, _ptr(comp_sq), _ptr(comp_sdf),
        ctypes.c_void_p(_stream(dev))), "pcdf_composite_translated")
    return comp_sq, comp_sdf


# ---------------------------------------------------------------------------
# hinge cost (Sec. 7) and its gradient
# ---------------------------------------------------------------------------

def _query_args(sdf, grid, spheres, tidx):
    shp = _shape(grid)
    if sdf.dim() == 3:
        sdf = sdf.unsqueeze(0)
    T = int(sdf.shape[0])
    _need(sdf, "sdf", torch.float32, (T,) + shp)
    _need(spheres, "spheres", torch.float32)
    if spheres.shape[-1] != 4:
        raise ValueError("spheres must be [..., 4] (x, y, z, r)")
    N = spheres.numel() // 4
    _need(tidx, "tidx", torch.int32)
    if tidx.numel() != N:
        raise ValueError(f"tidx has {tidx.numel()} entries for {N} spheres")
    return sdf, T, N


def query_cost(sdf: torch.Tensor, grid, spheres: torch.Tensor, tidx: torch.Tensor, eps: float,
               count_oob: bool = False):
    """h = max(0, eps + r - trilinear(sdf[clamp(tidx)], c)) per sphere.

    sdf: CUDA fp32 [T, nz, ny, nx] (or [nz, ny, nx]); spheres: CUDA fp32
    [..., 4]; tidx: CUDA int32 [...].  Returns h shaped like tidx (and the
    number of clamped spheres if count_oob)."""
    sdf, T, N = _query_args(sdf, grid, spheres, tidx)
    dev = sdf.device
    h = torch.empty(tidx.shape, dtype=torch.float32, device=dev)
    oob = torch.zeros(1, dtype=torch.int32, device=dev) if count_oob else None
    g = _cgrid(grid)
    _lib.check(_lib.load().pcdf_query_cost(ctypes.byref(g), _ptr(sdf), T, _ptr(spheres), _ptr(tidx), N,
                                           float(eps), _ptr(h), _ptr(oob), ctypes.c_void_p(_stream(dev))),
               "pcdf_query_cost")
    if count_oob:
        return h, oob
    return h


def query_cost_backward(sdf: torch.Tensor, grid, spheres: torch.Tensor, tidx: torch.Tensor, eps: float,
                        grad_h: torch.Tensor, want_grad_r: bool = True):
    """(grad_c [..., 3], grad_r [...] or None) of sum(grad_h * h)."""
    sdf, T, N = _query_args(sdf, grid, spheres, tidx)
    dev = sdf.device
    _need(grad_h, "grad_h", torch.float32)
    if grad_h.numel() != N:
        raise ValueError("grad_h must have one entry per sphere")
    gc = torch.empty(tuple(spheres.shape[:-1]) + (3,), dtype=torch.float32, device=dev)
    gr = torch.empty(tidx.shape, dtype=torch.float32, device=dev) if want_grad_r else None
    g = _cgrid(grid)
    _lib.check(_lib.load().pcdf_query_cost_backward(ctypes.byref(g), _ptr(sdf), T, _ptr(spheres), _ptr(tidx), N,
                                                    float(eps), _ptr(grad_h), _ptr(gc), _ptr(gr),
                                                    ctypes.c_void_p(_stream(dev))),
               "pcdf_query_cost_backward")
    return gc, gr


class HingeCost(torch.autograd.Function):
    """Hinge obstacle cost with a hand-written backward to the sphere centres
    (and radii).  Inputs: centres [..., 3] and radii [...] (fp32, CUDA)."""

    @staticmethod
    def forward(ctx, centres, radii, sdf, tidx, eps, grid):
        spheres = torch.cat([centres.detach(), radii.detach().unsqueeze(-1)], dim=-1).contiguous()
        tidx = tidx.contiguous()
        h = query_cost(sdf, grid, spheres, tidx, eps)
        ctx.save_for_backward(spheres, sdf, tidx)
        ctx.eps = eps
        ctx.grid = grid
        return h

    @staticmethod
    def backward(ctx, grad_h):
        spheres, sdf, tidx = ctx.saved_tensors
        gc, gr = query_cost_backward(sdf, ctx.grid, spheres, tidx, ctx.eps, grad_h.contiguous().float(),
                                     want_grad_r=ctx.needs_input_grad[1])
        return gc, gr, None, None, None, None


def hinge_cost(centres, radii, sdf, tidx, eps, grid):
    """Differentiable hinge cost h[...] (autograd through HingeCost)."""
    return HingeCost.apply(centres, radii, sdf, tidx, float(eps), grid)


# ---------------------------------------------------------------------------
# batched environments: one persistent launch
# ---------------------------------------------------------------------------

class Context:
    """The C interface's context (pcdf_create): a device, a stream and scratch
    that the library owns and grows, so its calls take no workspace.  Each
    method marshals its arguments for the pcdf_ctx_* call of the same name;
    the stream is the device's current PyTorch stream at creation unless one
    is given.  close() (or garbage collection) releases the scratch."""

    def __init__(self, device, stream=None):
        self._lib = _lib.load()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        idx = self.device.index if self.device.index is not None else torch.cuda.current_device()
        _lib.check(self._lib.pcdf_create(ctypes.byref(h), int(idx), ctypes.c_void_p(self.stream.cuda_stream)),
                   "pcdf_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pcdf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    @staticmethod
    def scratch_bytes(grid, T: int, H: int) -> int:
        """Upper bound of the scratch of any call for grid with up to T fields and H humans."""
        g = _cgrid(grid)
        n = ctypes.c_size_t(0)
        _lib.check(_lib.load().pcdf_scratch_bytes(ctypes.byref(g), int(T), int(H), ctypes.byref(n)),
                   "pcdf_scratch_bytes")
        return n.value

    def reserve(self, nbytes: int):
        _lib.check(self._lib.pcdf_ctx_reserve(self._h, int(nbytes)), "pcdf_ctx_reserve")

    def build_static_sdf(self, occ: torch.Tensor, grid, want_sdf: bool = True):
        shp = _shape(grid)
        _need(occ, "occ", torch.uint8, shp)
        sq = torch.empty(shp, dtype=torch.int32, device=occ.device)
        sdf = torch.empty(shp, dtype=torch.float32, device=occ.device) if want_sdf else None
        g = _cgrid(grid)
        _lib.check(self._lib.pcdf_ctx_build_static_sdf(self._h, ctypes.byref(g), _ptr(occ), _ptr(sq), _ptr(sdf)),
                   "pcdf_ctx_build_static_sdf")
        return sq, sdf

    def build_predicted_composite(self, static_sq: torch.Tensor, grid, caps, static_sdf=None, want_sq: bool = True,
                                  want_sdf: bool = True):
        shp = _shape(grid)
        _need(static_sq, "static_sq", torch.int32, shp)
        caps = _caps_host(caps)
        T, H = int(caps.shape[0]), int(caps.shape[1])
        dev = static_sq.device
        sq = torch.empty((T,) + shp, dtype=torch.int32, device=dev) if want_sq else None
        sdf = torch.empty((T,) + shp, dtype=torch.float32, device=dev) if want_sdf else None
        g = _cgrid(grid)
        cp = caps.ctypes.data_as(ctypes.c_void_p) if H > 0 else None
        _lib.check(self._lib.pcdf_ctx_build_predicted_composite(self._h, ctypes.byref(g), _ptr(static_sq),
                                                                _ptr(static_sdf), T, H, cp, _ptr(sq), _ptr(sdf)),
                   "pcdf_ctx_build_predicted_composite")
        return sq, sdf

    def build_from_scratch(self, occ: torch.Tensor, grid, caps, want_sdf: bool = True):
        shp = _shape(grid)
        _need(occ, "occ", torch.uint8, shp)
        caps = _caps_host(caps)
        T, H = int(caps.shape[0]), int(caps.shape[1])
        sq = torch.empty((T,) + shp, dtype=torch.int32, device=occ.device)
        sdf = torch.empty((T,) + shp, dtype=torch.float32, device=occ.device) if want_sdf else None
        g = _cgrid(grid)
        cp = caps.ctypes.data_as(ctypes.c_void_p) if H > 0 else None
        _lib.check(self._lib.pcdf_ctx_build_from_scratch(self._h, ctypes.byref(g), _ptr(occ), T, H, cp, _ptr(sq),
                                                         _ptr(sdf)), "pcdf_ctx_build_from_scratch")
        return sq, sdf

    def query_cost(self, sdf: torch.Tensor, grid, spheres: torch.Tensor, tidx: torch.Tensor, eps: float):
        sdf, T, N = _query_args(sdf, grid, spheres, tidx)
        h = torch.empty(tidx.shape, dtype=torch.float32, device=sdf.device)
        g = _cgrid(grid)
        _lib.check(self._lib.pcdf_ctx_query_cost(self._h, ctypes.byref(g), _ptr(sdf), T, _ptr(spheres), _ptr(tidx),
                                                 N, float(eps), _ptr(h), None), "pcdf_ctx_query_cost")
        return h

    def query_cost_backward(self, sdf: torch.Tensor, grid, spheres: torch.Tensor, tidx: torch.Tensor, eps: float,
                            grad_h: torch.Tensor):
        sdf, T, N = _query_args(sdf, grid, spheres, tidx)
        _need(grad_h, "grad_h", torch.float32)
        if grad_h.numel() != N:
            raise ValueError("grad_h must have one entry per sphere")
        gc = torch.empty(tuple(spheres.shape[:-1]) + (3,), dtype=torch.float32, device=sdf.device)
        gr = torch.empty(tidx.shape, dtype=torch.float32, device=sdf.device)
        g = _cgrid(grid)
        _lib.check(self._lib.pcdf_ctx_query_cost_backward(self._h, ctypes.byref(g), _ptr(sdf), T, _ptr(spheres),
                                                          _ptr(tidx), N, float(eps), _ptr(grad_h), _ptr(gc),
                                                          _ptr(gr)), "pcdf_ctx_query_cost_backward")
        return gc, gr

    def build_batched(self, envs, use_graph: bool = True):
        """envs: sequence of (grid, occ CUDA uint8, caps host int32 [T][H][7]);
        returns the int32 composite fields of every environment.  Synchronises
        the context's stream."""
        arr = (_lib.PcdfEnv * len(envs))()
        keep, outs = [], []
        for i, (grid, occ, caps) in enumerate(envs):
            _need(occ, f"occ[{i}]", torch.uint8, _shape(grid))
            c = _caps_host(caps)
            keep.append(c)
            T, H = int(c.shape[0]), int(c.shape[1])
            out = torch.empty((T,) + _shape(grid), dtype=torch.int32, device=occ.device)
            outs.append(out)
            arr[i].grid = _cgrid(grid)
            arr[i].T = T
            arr[i].H = H
            arr[i].caps = c.ctypes.data if H > 0 else None
            arr[i].occ = occ.data_ptr()
            arr[i].comp_sq = out.data_ptr()
        _lib.check(self._lib.pcdf_build_batched(self._h, arr, len(envs), 1 if use_graph else 0),
                   "pcdf_build_batched")
        return outs


class Batch:
    """Many environments updated by one persistent kernel launch.

    envs: sequence of (grid, occ CUDA uint8 [nz,ny,nx], caps host int32
    [T][H][7]).  Allocates the int32 composite outputs ``self.comp_sq[e]``
    ([T_e, nz, ny, nx]) and the workspace from PyTorch, builds and uploads the
    plan.  ``run()`` enqueues the counter reset and the launch on the current
    stream (capturable in a CUDA graph); ``error()`` synchronises and returns
    the kernel's status code (0 = ok)."""

    def __init__(self, envs, tiles=None, device=None):
        self._lib = _lib.load()
        self.device = device if device is not None else envs[0][1].device
        self._caps = []
        self.comp_sq = []
        arr = (_lib.PcdfEnv * len(envs))()
        for i, (grid, occ, caps) in enumerate(envs):
            _need(occ, f"occ[{i}]", torch.uint8, _shape(grid))
            c = _caps_host(caps)
            self._caps.append(c)
            T, H = int(c.shape[0]), int(c.shape[1])
            out = torch.empty((T,) + _shape(grid), dtype=torch.int32, device=self.device)
            self.comp_sq.append(out)
            arr[i].grid = _cgrid(grid)
            arr[i].T = T
            arr[i].H = H
            arr[i].caps = c.ctypes.data if H > 0 else None
            arr[i].occ = occ.data_ptr()
            arr[i].comp_sq = out.data_ptr()
        self._envs = arr
        self._occ = [e[1] for e in envs]
        t = _lib.PcdfBatchTiles(*(tiles or (0, 0, 0)))
        h = ctypes.c_void_p()
        _lib.check(self._lib.pcdf_batch_create(arr, len(envs), ctypes.byref(t), ctypes.byref(h)), "pcdf_batch_create")
        self._h = h
        nbytes = ctypes.c_size_t(0)
        _lib.check(self._lib.pcdf_batch_workspace_bytes(h, ctypes.byref(nbytes)), "pcdf_batch_workspace_bytes")
        self.workspace = _workspace(nbytes.value, self.device)
        _lib.check(self._lib.pcdf_batch_upload(h, _ptr(self.workspace), self.workspace.numel(),
                                               ctypes.c_void_p(_stream(self.device))), "pcdf_batch_upload")

    @property
    def tiles(self):
        t = _lib.PcdfBatchTiles()
        _lib.check(self._lib.pcdf_batch_tiles_used(self._h, ctypes.byref(t)), "pcdf_batch_tiles_used")
        return (t.row_rows, t.dyn_slices, t.comp_t)

    def run(self):
        _lib.check(self._lib.pcdf_batch_run(self._h, _ptr(self.workspace), ctypes.c_void_p(_stream(self.device))),
                   "pcdf_batch_run")

    def error(self) -> int:
        code = ctypes.c_int32(0)
        _lib.check(self._lib.pcdf_batch_error(self._h, _ptr(self.workspace), ctypes.c_void_p(_stream(self.device)),
                                              ctypes.byref(code)), "pcdf_batch_error")
        return code.value

    def block_stage(self, env: int, stage: int):
        """Testing aid for the failure path (pcdf_batch_block_stage): the
        items waiting on stage `stage` of environment `env` can only time out;
        the next run() then reports PCDF_ETIMEOUT through error()."""
        _lib.check(self._lib.pcdf_batch_block_stage(self._h, int(env), int(stage)), "pcdf_batch_block_stage")
        _lib.check(self._lib.pcdf_batch_upload(self._h, _ptr(self.workspace), self.workspace.numel(),
                                               ctypes.c_void_p(_stream(self.device))), "pcdf_batch_upload")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pcdf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_autotune(envs, reps: int = 3, device=None):
    """Time every candidate tile shape of the batched kernel on these
    environments; returns ((row_rows, dyn_slices, comp_t), ms)."""
    lib = _lib.load()
    device = device if device is not None else envs[0][1].device
    arr = (_lib.PcdfEnv * len(envs))()
    keep = []
    for i, (grid, occ, caps) in enumerate(envs):
        c = _caps_host(caps)
        keep.append(c)
        T, H = int(c.shape[0]), int(c.shape[1])
        out = torch.empty((T,) + _shape(grid), dtype=torch.int32, device=device)
        keep.append(out)
        arr[i].grid = _cgrid(grid)
        arr[i].T = T
        arr[i].H = H
        arr[i].caps = c.ctypes.data if H > 0 else None
        arr[i].occ = occ.data_ptr()
        arr[i].comp_sq = out.data_ptr()
    nbytes = ctypes.c_size_t(0)
    _lib.check(lib.pcdf_batch_autotune_workspace_bytes(arr, len(envs), ctypes.byref(nbytes)), "autotune workspace")
    ws = _workspace(nbytes.value, device)
    best = _lib.PcdfBatchTiles()
    ms = ctypes.c_float(0)
    _lib.check(lib.pcdf_batch_autotune(arr, len(envs), _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(device)),
                                       int(reps), ctypes.byref(best), ctypes.byref(ms)), "pcdf_batch_autotune")
    return (best.row_rows, best.dyn_slices, best.comp_t), ms.value


# ---------------------------------------------------------------------------
# learned surrogate of the dynamic field (BF16 MLP, FP32 accumulation)
# ---------------------------------------------------------------------------

MLP_IN, MLP_IN_PAD, MLP_WIDTH = 13, 16, 256
MLP_PARAMS, MLP_PARAMS_PAD, MLP_BF16 = 136193, 136196, 135424
# element offsets in the FP32 parameter vector and in the BF16 weight copies
_P_OFF = {"W1": (0, (256, 16)), "b1": (4096, (256,)), "W2": (4352, (256, 256)), "b2": (69888, (256,)),
          "W3": (70144, (256, 256)), "b3": (135680, (256,)), "w4": (135936, (256,)), "b4": (136192, ())}
_H_OFF = {"W1": (0, (256, 16)), "W2": (4096, (256, 256)), "W3": (69632, (256, 256)), "w4": (135168, (256,))}


class SurrogateMLP:
    """State of the surrogate network in one device buffer (FP32 parameters,
    Adam moments, gradient, BF16 weight copies; layout in include/pcdf.h)."""

    def __init__(self, device, seed: int = 0):
        self._lib = _lib.load()
        self.device = torch.device(device)
        n = ctypes.c_size_t(0)
        _lib.check(self._lib.pcdf_mlp_state_bytes(ctypes.byref(n)), "pcdf_mlp_state_bytes")
        self.state = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        self.step = 0
        self._ws = None
        self.reset(seed)

    def reset(self, seed: int):
        _lib.check(self._lib.pcdf_mlp_init(_ptr(self.state), int(seed), ctypes.c_void_p(_stream(self.device))),
                   "pcdf_mlp_init")
        self.step = 0

    def _workspace(self, M):
        n = ctypes.c_size_t(0)
        _lib.check(self._lib.pcdf_mlp_workspace_bytes(int(M), ctypes.byref(n)), "pcdf_mlp_workspace_bytes")
        if self._ws is None or self._ws.numel() < n.value:
            self._ws = _workspace(n.value, self.device)
        return self._ws

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """x: CUDA bfloat16 [M, 16] -> y float32 [M]."""
        _need(x, "x", torch.bfloat16)
        M = x.shape[0]
        y = torch.empty(M, dtype=torch.float32, device=self.device)
        ws = self._workspace(M)
        _lib.check(self._lib.pcdf_mlp_forward(_ptr(self.state), _ptr(x), M, _ptr(y), _ptr(ws), ws.numel(),
                                              ctypes.c_void_p(_stream(self.device))), "pcdf_mlp_forward")
        return y

    def infer(self, x: torch.Tensor) -> torch.Tensor:
        """The same y as forward, from one fused launch with the activations on
        chip (no workspace).  x: CUDA bfloat16 [M, 16] -> y float32 [M]."""
        _need(x, "x", torch.bfloat16)
        M = x.shape[0]
        y = torch.empty(M, dtype=torch.float32, device=self.device)
        _lib.check(self._lib.pcdf_mlp_infer(_ptr(self.state), _ptr(x), M, _ptr(y),
                                            ctypes.c_void_p(_stream(self.device))), "pcdf_mlp_infer")
        return y

    def infer_tc(self, x: torch.Tensor, count: torch.Tensor = None) -> torch.Tensor:
        """forward on the tcgen05 tensor cores (FP32 accumulator in tensor
        memory): y within FP32 rounding of forward.  x: CUDA bfloat16 [M, 16].
        count: optional CUDA int32 [1]; then only the first count rows are
        computed (read on the device, no host synchronisation) and y past
        them is left unwritten."""
        _need(x, "x", torch.bfloat16)
        M = x.shape[0]
        y = torch.empty(M, dtype=torch.float32, device=self.device)
        st = ctypes.c_void_p(_stream(self.device))
        if count is None:
            _lib.check(self._lib.pcdf_mlp_infer_tc(_ptr(self.state), _ptr(x), M, _ptr(y), st), "pcdf_mlp_infer_tc")
        else:
            _need(count, "count", torch.int32)
            _lib.check(self._lib.pcdf_mlp_infer_tc_count(_ptr(self.state), _ptr(x), M, _ptr(count), _ptr(y), st),
                       "pcdf_mlp_infer_tc_count")
        return y

    def backward(self, x: torch.Tensor, target: torch.Tensor):
        """Forward + loss + gradient (into the state).  Returns (y, loss[1])."""
        _need(x, "x", torch.bfloat16)
        _need(target, "target", torch.float32)
        M = x.shape[0]
        y = torch.empty(M, dtype=torch.float32, device=self.device)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        ws = self._workspace(M)
        _lib.check(self._lib.pcdf_mlp_backward(_ptr(self.state), _ptr(x), _ptr(target), M, _ptr(y), _ptr(loss),
                                               _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(self.device))),
                   "pcdf_mlp_backward")
        return y, loss

    def stored(self, M: int):
        """What the last forward or backward pass of M rows stored in the
        workspace (layout in include/pcdf.h), unpacked from the tensor-core
        tile layout (copies): H1, H2, H3, D2, D1 as bfloat16 [M, 256] and dy
        as float32 [M].  A forward pass stores H1, H2, H3; a backward pass H1,
        H2, D2, D1 and dy (D3 = dy w4 where H3 > 0 is not stored)."""
        T = -(-M // 128)
        tile = 128 * 256 * 2
        ws = self._ws
        out = {}
        for i, k in enumerate(("H1", "H2", "H3", "D2", "D1")):
            raw = ws[i * T * tile:(i + 1) * T * tile].view(torch.bfloat16)
            # element (m, c) at tile m // 128, 8-row group, 8-column group, row in group, column in group
            t = raw.view(T, 16, 32, 8, 8).permute(0, 1, 3, 2, 4).reshape(T * 128, 256)
            out[k] = t[:M].clone()
        o = 5 * T * tile + T * 4096 + 3 * T * 4096
        out["dy"] = ws[o:o + 4 * M].view(torch.float32).clone()
        return out

    def adam(self, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        _lib.check(self._lib.pcdf_mlp_adam(_ptr(self.state), float(lr), float(beta1), float(beta2), float(eps),
                                           self.step, ctypes.c_void_p(_stream(self.device))), "pcdf_mlp_adam")

    def train_step(self, x, target, lr):
        _, loss = self.backward(x, target)
        self.adam(lr)
        return loss

    def _f32(self, region):
        off = {"master": 0, "m": 4, "v": 8, "grad": 12}[region] * MLP_PARAMS_PAD
        return self.state[off:off + 4 * MLP_PARAMS_PAD].view(torch.float32)

    def _bf16(self):
        off = 16 * MLP_PARAMS_PAD
        return self.state[off:off + 2 * MLP_BF16].view(torch.bfloat16)

    def params(self):
        """dict of float64 numpy arrays as the network computes with them: the
        BF16 weight copies and the FP32 biases."""
        master = self._f32("master").detach().cpu().double().numpy()
        half = self._bf16().detach().cpu().float().double().numpy()
        out = {}
        for k, (o, shp) in _P_OFF.items():
            if k in _H_OFF:
                ho, _ = _H_OFF[k]
                out[k] = half[ho:ho + int(np.prod(shp))].reshape(shp)
            else:
                out[k] = master[o:o + max(1, int(np.prod(shp)))].reshape(shp)
        return out

    def grads(self):
        g = self._f32("grad").detach().cpu().double().numpy()
        return {k: g[o:o + max(1, int(np.prod(shp)))].reshape(shp) for k, (o, shp) in _P_OFF.items()}

    def save(self, path):
        torch.save({"state": self.state.cpu(), "step": self.step}, path)

    def load(self, path):
        d = torch.load(path, map_location="cpu")
        if d["state"].numel() != self.state.numel():
            raise ValueError("checkpoint size does not match the network state")
        self.state.copy_(d["state"].to(self.device))
        self.step = int(d["step"])


def surrogate_samples(grid, fields, caps, tf, T, M, seed, near=0.5):
    """Training rows from exact dynamic fields (see pcdf_surrogate_samples)."""
    _need(fields, "fields", torch.float32)
    _need(caps, "caps", torch.int32)
    _need(tf, "tf", torch.int32)
    dev = fields.device
    x = torch.empty((M, MLP_IN_PAD), dtype=torch.bfloat16, device=dev)
    t = torch.empty(M, dtype=torch.float32, device=dev)
    g = _cgrid(grid)
    _lib.check(_lib.load().pcdf_surrogate_samples(ctypes.byref(g), _ptr(fields), _ptr(caps), _ptr(tf),
                                                  int(fields.shape[0]), int(T), int(M), int(seed), float(near),
                                                  _ptr(x), _ptr(t), ctypes.c_void_p(_stream(dev))),
               "pcdf_surrogate_samples")
    return x, t


def surrogate_features(grid, spheres, tidx, T, caps_dev):
    """Network rows (sphere q, human h) -> CUDA bfloat16 [N * H, 16]."""
    _need(spheres, "spheres", torch.float32)
    _need(tidx, "tidx", torch.int32)
    _need(caps_dev, "caps", torch.int32)
    H = int(caps_dev.shape[1])
    N = spheres.numel() // 4
    dev = spheres.device
    x = torch.empty((N * H, MLP_IN_PAD), dtype=torch.bfloat16, device=dev)
    g = _cgrid(grid)
    _lib.check(_lib.load().pcdf_surrogate_features(ctypes.byref(g), _ptr(spheres), _ptr(tidx), N, int(T), H,
                                                   _ptr(caps_dev), _ptr(x), ctypes.c_void_p(_stream(dev))),
               "pcdf_surrogate_features")
    return x


def surrogate_select(grid, static_sdf, spheres, tidx, T, caps_dev, eps, certified=True, sync=True):
    """The certificate of every query (bounds float32 [N, 2]: d_lo <= d <= d_hi
    for the exact path's distance d) and the rows the network must answer:
    with certified=True only rows of queries that are certainly in collision
    (the only ones whose cost uses the network), else every row whose human
    can matter in the query's cell (to measure the network).  Returns (x BF16
    [kept rows][16], y_index int32 [N * H], bounds); with sync=False no host
    synchronisation: (x BF16 [N * H][16] whose first count rows are the kept
    ones, y_index, count int32 [1] on the device, bounds)."""
    N = spheres.numel() // 4
    H = int(caps_dev.shape[1])
    dev = spheres.device
    x = torch.empty((max(N * H, 1), MLP_IN_PAD), dtype=torch.bfloat16, device=dev)
    yi = torch.empty(max(N * H, 1), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    bounds = torch.empty((max(N, 1), 2), dtype=torch.float32, device=dev)
    g = _cgrid(grid)
    _lib.check(_lib.load().pcdf_surrogate_select(ctypes.byref(g), _ptr(static_sdf), _ptr(spheres), _ptr(tidx), N,
                                                 int(T), H, _ptr(caps_dev), float(eps), 0 if certified else 1,
                                                 _ptr(x), _ptr(yi), _ptr(cnt), _ptr(bounds),
                                                 ctypes.c_void_p(_stream(dev))), "pcdf_surrogate_select")
    if not sync:
        return x, yi, cnt, bounds
    return x[: int(cnt.item())], yi, bounds


def surrogate_finish(grid, static_sq, static_sdf, spheres, tidx, T, caps, y, eps, band, comp_workspace=None,
                     y_index=None, bounds=None):
    """Hinge cost from the network outputs.  With bounds (the certificate of
    surrogate_select) every collision decision is the exact path's: the
    prediction is clamped to the certified interval, and queries whose
    decision is not certain, or whose prediction lies within `band` of the
    threshold, are answered exactly.  Without bounds the band alone decides.
    With comp_workspace (after composite_prepare on the same grid and caps)
    the exact answers come from its capsule-slab partials, else from a local
    search over the capsules' voxels.  Returns (h, d, n_fallback[1])."""
    caps = _caps_host(caps)
    H = int(caps.shape[1])
    N = spheres.numel() // 4
    dev = spheres.device
    h = torch.empty(tidx.shape, dtype=torch.float32, device=dev)
    d = torch.empty(tidx.shape, dtype=torch.float32, device=dev)
    nfb = torch.zeros(1, dtype=torch.int32, device=dev)
    n = ctypes.c_size_t(0)
    lib = _lib.load()
    _lib.check(lib.pcdf_surrogate_finish_workspace_bytes(int(T), H, N, ctypes.byref(n)), "surrogate workspace")
    ws = _workspace(n.value, dev)
    g = _cgrid(grid)
    cp = caps.ctypes.data_as(ctypes.c_void_p)
    tail = (float(eps), float(band), _ptr(h), _ptr(d), _ptr(nfb), _ptr(ws), ws.numel(), ctypes.c_void_p(_stream(dev)))
    if comp_workspace is None:
        _lib.check(lib.pcdf_surrogate_finish(ctypes.byref(g), _ptr(static_sq), _ptr(static_sdf), _ptr(spheres),
                                             _ptr(tidx), N, int(T), H, cp, _ptr(y), _ptr(y_index), _ptr(bounds),
                                             *tail), "pcdf_surrogate_finish")
    else:
        _need(comp_workspace, "comp_workspace", torch.uint8)
        _lib.check(lib.pcdf_surrogate_finish_slab(ctypes.byref(g), _ptr(static_sq), _ptr(static_sdf), _ptr(spheres),
                                                  _ptr(tidx), N, int(T), H, cp, _ptr(comp_workspace),
                                                  comp_workspace.numel(), _ptr(y), _ptr(y_index), _ptr(bounds),
                                                  *tail), "pcdf_surrogate_finish_slab")
    return h, d, nfb


def surrogate_step(model, grid, static_sq, static_sdf, spheres, tidx, caps, eps, band, comp_workspace,
                   caps_dev=None):
    """One certified plan step of the surrogate: the capsule-slab partials of
    the composite's first stage (composite_prepare into comp_workspace) run on
    a side stream while the certificate and the rows are computed on the
    current stream; the network waits for both (its persistent grid wants
    every SM), then the exact answers read the partials.  Every collision
    decision is the exact path's.  No host synchronisation: capturable in a
    CUDA graph.  Returns (h, d, n_fallback[1]) as surrogate_query."""
    caps = _caps_host(caps)
    dev = spheres.device
    if caps_dev is None:
        caps_dev = torch.from_numpy(caps).to(dev)
    T = int(caps.shape[0])
    main = torch.cuda.current_stream(dev)
    side = _side_stream(dev)
    side.wait_stream(main)
    with torch.cuda.stream(side):
        composite_prepare(grid, caps, comp_workspace)
    comp_workspace.record_stream(side)
    x, yi, cnt, bounds = surrogate_select(grid, static_sdf, spheres, tidx, T, caps_dev, eps, sync=False)
    main.wait_stream(side)
    y = model.infer_tc(x, count=cnt) if x.shape[0] else torch.empty(1, dtype=torch.float32, device=dev)
    return surrogate_finish(grid, static_sq, static_sdf, spheres, tidx, T, caps, y, eps, band, comp_workspace,
                            y_index=yi, bounds=bounds)


def surrogate_query(model, grid, static_sq, static_sdf, spheres, tidx, caps, eps, band, caps_dev=None,
                    comp_workspace=None, certified=True):
    """Hinge cost of every sphere through the network, exact where needed (from
    the capsule-slab partials in comp_workspace when given, after
    composite_prepare).  certified=True: every collision decision is the
    exact path's (see surrogate_finish); certified=False: the network's own
    prediction for every query where the humans can matter, exact only within
    `band` of the threshold (band 0: the network alone).
    Returns (h, d, n_fallback[1])."""
    caps = _caps_host(caps)
    if caps_dev is None:
        caps_dev = torch.from_numpy(caps).to(spheres.device)
    T = int(caps.shape[0])
    # select -> network -> finish with the kept-row count on the device
    x, yi, cnt, bounds = surrogate_select(grid, static_sdf, spheres, tidx, T, caps_dev, eps, certified=certified,
                                          sync=False)
    y = model.infer_tc(x, count=cnt) if x.shape[0] else torch.empty(1, dtype=torch.float32, device=spheres.device)
    return surrogate_finish(grid, static_sq, static_sdf, spheres, tidx, T, caps, y, eps, band, comp_workspace,
                            y_index=yi, bounds=bounds if certified else None)
