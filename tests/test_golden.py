"""Golden fixtures (tests/golden/, written by make_golden.py from the oracle).

CPU: the stored fields equal the signed squared EDT and the composite by
their definitions (Sec. 6), computed here by brute force with an exact
rational capsule test that shares nothing with the oracle's; the stored
hinge values follow the hinge's closed form (Sec. 7.2) at voxel centres with
the paper's eps = 0.4 m (Sec. 7.3); the oracle still reproduces them.
GPU: the CUDA path reproduces the stored fields bit for bit and the costs
within 1e-5 m.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def fixture_inputs():
    d = load("composite_12x10x8.json")
    nx, ny, nz = d["grid"]
    occ = np.zeros((nz, ny, nx), np.uint8)
    for z0, z1, y0, y1, x0, x1 in d["occupied_boxes_zyx"]:
        occ[z0:z1, y0:y1, x0:x1] = 1
    caps = np.array(d["caps"], np.int32)
    static = np.array(d["static_sq"], np.int64).reshape(nz, ny, nx)
    comp = np.array(d["comp_sq"], np.int64).reshape(len(caps), nz, ny, nx)
    return d, occ, caps, static, comp


def inside_exact(p, cap):
    """Centre p (1/16 voxel) in the closed capsule, by exact rationals."""
    a = [Fraction(v) for v in cap[0:3]]
    b = [Fraction(v) for v in cap[3:6]]
    r = Fraction(int(cap[6]))
    w = [Fraction(p[i]) - a[i] for i in range(3)]
    ab = [b[i] - a[i] for i in range(3)]
    L = sum(x * x for x in ab)
    t = Fraction(0) if L == 0 else min(max(sum(w[i] * ab[i] for i in range(3)) / L, Fraction(0)), Fraction(1))
    d2 = sum((w[i] - t * ab[i]) ** 2 for i in range(3))
    return d2 <= r * r


def edt_by_definition(occ):
    idx = np.argwhere(np.ones_like(occ, dtype=bool))
    o = occ.reshape(-1).astype(bool)
    out = np.empty(o.size, np.int64)
    for n, v in enumerate(idx):
        other = idx[~o] if o[n] else idx[o]
        if len(other) == 0:
            out[n] = (-1 if o[n] else 1) * oracle.INF32
            continue
        d2 = int(np.min(np.sum((other - v) ** 2, axis=1)))
        out[n] = -d2 if o[n] else d2
    return out.reshape(occ.shape)


def test_golden_static_field_is_the_definition():
    _, occ, _, static, _ = fixture_inputs()
    assert np.array_equal(edt_by_definition(occ), static)


def test_golden_composite_is_the_definition():
    _, occ, caps, static, comp = fixture_inputs()
    nz, ny, nx = occ.shape
    for t in range(len(caps)):
        dyn = np.zeros_like(occ)
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    p = (16 * i + 8, 16 * j + 8, 16 * k + 8)
                    dyn[k, j, i] = any(inside_exact(p, c) for c in caps[t])
        assert dyn.sum() > 0
        want = np.minimum(static, edt_by_definition(dyn))
        assert np.array_equal(want, comp[t]), t


def test_golden_fixtures_are_reproduced_by_the_oracle():
    d, occ, caps, static, comp = fixture_inputs()
    assert np.array_equal(oracle.edt(occ), static)
    assert np.array_equal(oracle.predicted_composite(oracle.edt(occ), caps), comp)
    h = load("hinge_eps04.json")
    sdf = np.stack([oracle.sdf_from_sq(comp[t], d["vox"]) for t in range(len(caps))])
    got, _ = oracle.hinge_cost(sdf, d["origin"], d["vox"], np.array(h["spheres"], np.float32),
                               np.array(h["tidx"], np.int32), h["eps"])
    assert np.array_equal(got, np.array(h["h"]))


def test_golden_hinge_closed_form_at_voxel_centres():
    """At a voxel centre the interpolated distance is the field's value, so
    h = max(0, eps - d) with d = sign(S) sqrt(|S|) vox (radius 0)."""
    d, _, caps, _, comp = fixture_inputs()
    h = load("hinge_eps04.json")
    assert h["eps"] == 0.4
    vox = d["vox"]
    checked = 0
    for (x, y, z, r), t, hv in zip(h["spheres"], h["tidx"], h["h"]):
        u = np.array([x, y, z]) / vox - 0.5
        if not np.allclose(u, np.rint(u), atol=1e-4) or np.any(u < 0):
            continue
        i, j, k = (int(v) for v in np.rint(u))
        S = int(comp[t, k, j, i])
        dist = np.sign(S) * np.sqrt(abs(S)) * vox
        assert abs(hv - max(0.0, 0.4 + r - dist)) <= 1e-5
        checked += 1
    assert checked >= 12


@pytest.mark.gpu
def test_golden_cuda_path():
    pcdf = pytest.importorskip("paper_2201_05058_gb300")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    d, occ, caps, static, comp = fixture_inputs()
    nx, ny, nz = d["grid"]
    grid = pcdf.Grid(nx, ny, nz, d["vox"], tuple(d["origin"]))
    st_sq, st_sdf = pcdf.build_static_sdf(torch.from_numpy(occ).to(dev), grid)
    assert np.array_equal(st_sq.cpu().numpy(), static)
    sq, sdf = pcdf.build_predicted_composite(st_sq, grid, caps, static_sdf=st_sdf)
    assert np.array_equal(sq.cpu().numpy(), comp)
    h = load("hinge_eps04.json")
    got = pcdf.query_cost(sdf, grid, torch.tensor(h["spheres"], dtype=torch.float32, device=dev),
                          torch.tensor(h["tidx"], dtype=torch.int32, device=dev), h["eps"])
    assert np.max(np.abs(got.cpu().numpy() - np.array(h["h"]))) <= 1e-5
