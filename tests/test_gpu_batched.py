"""Batched persistent launch: ragged environments, bit-identical to the oracle
and to the per-environment calls, for every autotuner tile shape, and when
replayed from a captured CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu

pcdf = pytest.importorskip("paper_2201_05058_gb300")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def ragged_envs(seed=0):
    """Uneven sizes (ragged tails), horizons and human counts, one environment
    whose humans are all outside the grid and one without humans."""
    rng = np.random.default_rng(seed)
    dims = [(37, 45, 29), (64, 20, 33), (20, 70, 41), (50, 50, 50), (33, 17, 64), (40, 40, 12)]
    Ts = [1, 3, 6, 2, 4, 3]
    Hs = [2, 1, 3, 0, 1, 2]
    envs = []
    for i, ((nx, ny, nz), T, H) in enumerate(zip(dims, Ts, Hs)):
        grid = scenes.Grid(nx, ny, nz, 0.05)
        occ, _ = scenes.boxes_occupancy(grid, 4 + i, rng)
        if H > 0:
            caps = scenes.walking_capsules(grid, H, T, rng)
        else:
            caps = np.zeros((T, 0, 7), np.int32)
        if i == 5:  # humans entirely outside the grid
            caps[..., 0] = -6000
            caps[..., 3] = -6000
        envs.append((grid, occ, caps))
    return envs


def oracle_fields(envs):
    return [oracle.predicted_composite(oracle.edt(occ), caps) for grid, occ, caps in envs]


@pytest.fixture(scope="module")
def batch_case():
    envs = ragged_envs()
    d = dev()
    dev_envs = [(g, torch.from_numpy(o).to(d), c) for g, o, c in envs]
    return envs, dev_envs, oracle_fields(envs)


def test_batched_matches_oracle_and_single_calls(batch_case):
    envs, dev_envs, want = batch_case
    b = pcdf.Batch(dev_envs)
    b.run()
    assert b.error() == 0
    for e, (grid, occ_d, caps) in enumerate(dev_envs):
        got = b.comp_sq[e].cpu().numpy()
        assert np.array_equal(got, want[e]), f"environment {e} differs from the oracle"
        static_sq, _ = pcdf.build_static_sdf(occ_d, grid)
        single, _ = pcdf.build_predicted_composite(static_sq, grid, caps, want_sdf=False)
        assert np.array_equal(got, single.cpu().numpy()), f"environment {e} differs from the single call"
    b.close()


def test_an_expired_wait_reports_timeout_and_the_context_stays_usable(batch_case):
    """The failure path without a GPU fault: environment 0's row stage is
    given a target no run reaches, so its y items wait until their bound
    (about a second) expires; every later wait then gives up at once, so
    nothing reads unfinished inputs, and error() reports PCDF_ETIMEOUT.  The
    capsule stage, which nothing waits on, is refused.  A fresh batch on the
    same context is then exact again."""
    envs, dev_envs, want = batch_case
    b = pcdf.Batch(dev_envs)
    with pytest.raises(RuntimeError):
        b.block_stage(0, 3)
    b.block_stage(0, 0)
    b.run()
    assert b.error() == -4  # PCDF_ETIMEOUT
    b.close()
    b2 = pcdf.Batch(dev_envs)
    b2.run()
    assert b2.error() == 0
    for e in range(len(dev_envs)):
        assert np.array_equal(b2.comp_sq[e].cpu().numpy(), want[e]), e
    b2.close()


@pytest.mark.parametrize("tiles", [(8, 1, 1), (32, 4, 1), (128, 1, 4), (8, 4, 4), (128, 4, 1), (32, 1, 4)])
def test_every_tile_shape_gives_identical_bits(batch_case, tiles):
    envs, dev_envs, want = batch_case
    b = pcdf.Batch(dev_envs, tiles=tiles)
    assert b.tiles == tiles
    b.run()
    assert b.error() == 0
    for e in range(len(envs)):
        assert np.array_equal(b.comp_sq[e].cpu().numpy(), want[e]), f"tiles {tiles}, environment {e}"
    b.close()


def test_graph_capture_replay(batch_case):
    envs, dev_envs, want = batch_case
    b = pcdf.Batch(dev_envs, tiles=(32, 1, 1))
    b.run()  # first run outside the graph
    torch.cuda.synchronize()
    for out in b.comp_sq:
        out.fill_(7)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run()
    for _ in range(2):
        for out in b.comp_sq:
            out.fill_(-3)
        g.replay()
        torch.cuda.synchronize()
        assert b.error() == 0
        for e in range(len(envs)):
            assert np.array_equal(b.comp_sq[e].cpu().numpy(), want[e])
    b.close()


def test_autotune_picks_a_candidate(batch_case):
    envs, dev_envs, want = batch_case
    tiles, ms = pcdf.batch_autotune(dev_envs, reps=2)
    assert tiles[0] in (8, 32, 128) and tiles[1] in (1, 4) and tiles[2] in (1, 4)
    assert ms > 0
    b = pcdf.Batch(dev_envs, tiles=tiles)
    b.run()
    assert b.error() == 0
    for e in range(len(envs)):
        assert np.array_equal(b.comp_sq[e].cpu().numpy(), want[e])
    b.close()


def test_full_size_batch_matches_oracle_on_samples():
    """The 64-environment batch at its full sizes (64-320 x 64-320 x 64-128,
    T 5-30, 1-4 humans), in the launch configuration the benchmark times
    (autotuned tiles, graph-captured run): whole fields of sampled
    environments and time steps against the oracle, and voxels against the
    definition."""
    d = dev()
    envs = scenes.scene_batch(seed=0)
    dev_envs = [(e["grid"], torch.from_numpy(e["occ"]).to(d), e["caps"]) for e in envs]
    tiles, _ = pcdf.batch_autotune(dev_envs, reps=1)
    b = pcdf.Batch(dev_envs, tiles=tiles)
    b.run()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run()
    for f in b.comp_sq:
        f.fill_(7)
    g.replay()
    torch.cuda.synchronize()
    assert b.error() == 0
    rng = np.random.default_rng(5)
    largest = max(range(64), key=lambda e: envs[e]["grid"].nvox)
    for e in sorted({largest, 0, 37}):
        grid, occ, caps = envs[e]["grid"], envs[e]["occ"], envs[e]["caps"]
        S = oracle.edt(occ)
        T = caps.shape[0]
        got = b.comp_sq[e].cpu().numpy()
        for t in sorted({0, T - 1, int(rng.integers(0, T))}):
            dyn_occ = oracle.capsule_occupancy(grid.shape, caps[t])
            want = oracle.composite(S, oracle.edt(dyn_occ))
            assert np.array_equal(got[t], want), f"environment {e}, t = {t}"
            for _ in range(8):
                k, j, i = (int(rng.integers(0, n)) for n in grid.shape)
                assert got[t, k, j, i] == min(oracle.edt_at(occ, i, j, k), oracle.edt_at(dyn_occ, i, j, k))
    b.close()
