"""Runs the oracle on independent composite fields in parallel processes.

TEST INFRASTRUCTURE ONLY (the CPU-baseline and reference legs of bench.py).
Nothing here changes the oracle's arithmetic: each worker process calls the
unmodified single-threaded ``oracle.dynamic_field`` and ``oracle.composite``
(Sec. 6: each field is the per-voxel min of the environment field and the
field of the dynamic obstacles at one time index) on one field, and the
fields of a plan horizon do not depend on one another.

The pool is started with ``spawn`` (never ``fork``, which is unsafe in a
process that has used CUDA), and every map is bounded by a timeout so that a
pool whose workers cannot start raises instead of waiting forever.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile
import time

import numpy as np


def field_seconds(job):
    """Pool worker: one composite field from the environment field saved at
    ``path`` and the capsules ``caps_t`` of one time index.  Returns seconds."""
    path, caps_t = job
    import oracle
    S = np.ascontiguousarray(np.load(path))
    t0 = time.perf_counter()
    oracle.composite(S, oracle.dynamic_field(S.shape, caps_t))
    return time.perf_counter() - t0


class FieldPool:
    """One process per host core, at most ``cap``."""

    def __init__(self, cap: int, timeout_s: float = 900.0):
        self.workers = max(1, min(os.cpu_count() or 1, cap))
        self.timeout_s = timeout_s
        self.pool = mp.get_context("spawn").Pool(self.workers)
        # start every worker before anything is timed
        self.pool.map_async(time.sleep, [0] * self.workers).get(timeout=self.timeout_s)

    def fields(self, S_static: np.ndarray, caps_list) -> float:
        """Wall seconds for the composite fields of ``caps_list`` (one
        [H][7] capsule array per field) over ``S_static``."""
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "static.npy")
            np.save(path, S_static)
            t0 = time.perf_counter()
            self.pool.map_async(field_seconds, [(path, c) for c in caps_list], chunksize=1).get(
                timeout=self.timeout_s)
            return time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()
