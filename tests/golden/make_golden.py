"""Writes the golden fixtures of this folder from the oracle alone.

    python tests/golden/make_golden.py

Inputs are written out by hand below; every expected value comes from
`oracle/` (plain C, fp64 where it is floating point).  The fixtures are
pinned independently of the oracle in tests/test_golden.py (brute force
from the definitions, the hinge's closed form), and the CUDA path is
checked against them there too.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

# 12 x 10 x 8 voxels of 0.1 m, corner at the origin
NX, NY, NZ, VOX = 12, 10, 8, 0.1


def occupancy():
    occ = np.zeros((NZ, NY, NX), np.uint8)
    occ[0:3, 6:9, 2:5] = 1      # a box on the floor
    occ[:, :, 11] = 1           # a wall: the last x plane
    occ[5, 2, 7] = 1            # a single occupied voxel
    return occ


# capsules in 1/16 voxel from the grid corner (voxel centre 16 i + 8):
# t = 0 a vertical capsule, t = 1 a slanted one; radius 1.5 voxels
CAPS = np.array([[[104, 72, 16, 104, 72, 96, 24]],
                 [[136, 72, 16, 120, 88, 96, 24]]], np.int32)

# hinge cost with the obstacle safety distance of the paper's experiments
# (Sec. 7.3: Sigma_obs = 0.1, eps = 0.4 m, eps counting the person's radius,
# so the query points carry radius 0)
EPS = 0.4


def query_points():
    pts = []
    # voxel centres (trilinear value = the field's value there)
    for (i, j, k) in [(0, 0, 0), (6, 4, 3), (8, 4, 1), (5, 5, 5), (10, 9, 7), (3, 7, 3), (7, 2, 4)]:
        pts.append([(i + 0.5) * VOX, (j + 0.5) * VOX, (k + 0.5) * VOX, 0.0])
    # points between centres, and one outside the grid (clamped)
    pts += [[0.6125, 0.4375, 0.3125, 0.0], [0.9, 0.55, 0.25, 0.0], [0.33, 0.71, 0.42, 0.0],
            [-0.2, 0.5, 0.4, 0.0]]
    return np.array(pts, np.float32)


def main():
    occ = occupancy()
    static = oracle.edt(occ)
    comp = oracle.predicted_composite(static, CAPS)
    sdf = np.stack([oracle.sdf_from_sq(comp[t], VOX) for t in range(CAPS.shape[0])])
    pts = query_points()
    out = {"grid": [NX, NY, NZ], "vox": VOX, "origin": [0.0, 0.0, 0.0], "caps": CAPS.tolist(),
           "occupied_boxes_zyx": [[0, 3, 6, 9, 2, 5], [0, 8, 0, 10, 11, 12], [5, 6, 2, 3, 7, 8]],
           "static_sq": static.reshape(-1).tolist(),
           "comp_sq": [comp[t].reshape(-1).tolist() for t in range(CAPS.shape[0])]}
    with open(os.path.join(HERE, "composite_12x10x8.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    hin = {"eps": EPS, "citation": "Sec. 7.2 hinge on the environment field (after GPMP2); "
                                   "Sec. 7.3 Sigma_obs = 0.1, eps = 0.4",
           "spheres": pts.tolist(), "tidx": [], "h": []}
    for t in range(CAPS.shape[0]):
        tidx = np.full(len(pts), t, np.int32)
        h, _ = oracle.hinge_cost(sdf, out["origin"], VOX, pts, tidx, EPS)
        hin["tidx"] += tidx.tolist()
        hin["h"] += [float(v) for v in h]
    hin["spheres"] = pts.tolist() * CAPS.shape[0]
    with open(os.path.join(HERE, "hinge_eps04.json"), "w") as f:
        json.dump(hin, f, indent=1)


if __name__ == "__main__":
    main()
