"""Training and evaluation helpers of the learned surrogate (host orchestration).

Every numeric step runs in the library's kernels: the exact dynamic fields
come from the composite path with an empty static map, the training rows from
pcdf_surrogate_samples, the network passes and the Adam update from the MLP
kernels, the queries from pcdf_surrogate_features / _finish.  This module only
sequences those calls.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import api


def exact_dynamic_fields(grid, caps_list, device):
    """Float fields of the humans alone: for each capsule array caps [T][1][7]
    in caps_list, the T fields of that one capsule (composite with an empty
    static map).  Returns (fields fp32 [n, nz, ny, nx], caps int32 [n, 7],
    tf int32 [n]) on the device, n = sum of the T's."""
    empty = torch.zeros(api._shape(grid), dtype=torch.uint8, device=device)
    static_sq, _ = api.build_static_sdf(empty, grid, want_sdf=False)
    fields, caps, tf = [], [], []
    for c in caps_list:
        c = np.ascontiguousarray(c, np.int32)
        if c.ndim != 3 or c.shape[1] != 1:
            raise ValueError("each capsule array must be [T][1][7]")
        _, sdf = api.build_predicted_composite(static_sq, grid, c, want_sq=False)
        fields.append(sdf)
        caps.append(torch.from_numpy(c[:, 0, :].copy()))
        tf.append(torch.arange(c.shape[0], dtype=torch.int32))
    return (torch.cat(fields).contiguous(), torch.cat(caps).to(device).contiguous(),
            torch.cat(tf).to(device).contiguous())


def train(model, grid, fields, caps, tf, T, steps, batch, lr=2e-3, lr_min=5e-5, seed=0, near=0.6,
          log_every=0, draw=4):
    """Adam with cosine learning-rate decay on fresh samples every step, drawn
    `draw` steps at a time (one sampling launch for several steps: the draw is
    bound by the latency of its random reads, not by its size).  Returns the
    list of (step, loss) at the logged steps (device sync there)."""
    hist = []
    xs = ts = None
    for k in range(steps):
        if k % draw == 0:
            n = min(draw, steps - k)
            xs, ts = api.surrogate_samples(grid, fields, caps, tf, T, n * batch, seed * 1_000_003 + k, near)
        i = k % draw
        x, t = xs[i * batch:(i + 1) * batch], ts[i * batch:(i + 1) * batch]
        rate = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * k / max(steps - 1, 1)))
        loss = model.train_step(x, t, rate)
        if log_every and (k % log_every == 0 or k == steps - 1):
            hist.append((k, float(loss.item())))
    return hist
