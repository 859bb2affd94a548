"""The process pool that times the oracle on independent fields (bench.py's
CPU baseline and reference legs) starts, runs every field and shuts down."""
import numpy as np

import oracle
from oracle.pool import FieldPool


def test_field_pool_runs_the_oracle_on_independent_fields():
    occ = np.zeros((16, 16, 16), np.uint8)
    occ[2:5, 3:9, 4:6] = 1
    S = oracle.edt(occ)
    caps = [np.array([[8 + 16 * (4 + t), 72, 24, 8 + 16 * (4 + t), 72, 120, 24]], np.int32) for t in range(3)]
    pool = FieldPool(2, timeout_s=120.0)
    try:
        assert pool.workers >= 1
        assert pool.fields(S, caps) > 0.0
    finally:
        pool.close()
