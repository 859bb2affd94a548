"""The context calls (pcdf_create ... pcdf_build_batched): every result
bit-identical to the workspace call of the same name, the scratch growing
across calls of growing size, and the batched call with and without a graph
equal to the pcdf_batch_* path."""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

pcdf = pytest.importorskip("paper_2201_05058_gb300")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def test_context_calls_equal_the_workspace_calls():
    d = dev()
    ctx = pcdf.Context(d)
    # a small scene first, then a larger one: the scratch grows in between
    for n, T, H, seed in [(32, 3, 1, 4), (96, 7, 3, 5)]:
        sc = scenes.scene_composite(seed=seed, n=n, n_boxes=6, T=T, H=H)
        grid, caps = sc["grid"], sc["caps"]
        occ = torch.from_numpy(sc["occ"]).to(d)
        sq, sdf = pcdf.build_static_sdf(occ, grid)
        csq, csdf = ctx.build_static_sdf(occ, grid)
        assert torch.equal(sq, csq) and torch.equal(sdf, csdf)
        comp_sq, comp_sdf = pcdf.build_predicted_composite(sq, grid, caps, static_sdf=sdf)
        c_sq, c_sdf = ctx.build_predicted_composite(csq, grid, caps, static_sdf=csdf)
        assert torch.equal(comp_sq, c_sq) and torch.equal(comp_sdf, c_sdf)
        # no human: no scratch needed, every field the static one
        e_sq, _ = ctx.build_predicted_composite(csq, grid, np.zeros((T, 0, 7), np.int32), want_sdf=False)
        assert torch.equal(e_sq, sq.expand(T, *sq.shape))
        fs_sq, fs_sdf = pcdf.build_from_scratch(occ, grid, caps)
        cf_sq, cf_sdf = ctx.build_from_scratch(occ, grid, caps)
        assert torch.equal(fs_sq, cf_sq) and torch.equal(fs_sdf, cf_sdf)
        rng = np.random.default_rng(seed)
        sph, tidx = scenes.spheres_along_paths(grid, 16, 10, 6, rng, T=T)
        sph, tidx = torch.from_numpy(sph).to(d), torch.from_numpy(tidx).to(d)
        h = pcdf.query_cost(comp_sdf, grid, sph, tidx, 0.2)
        assert torch.equal(h, ctx.query_cost(c_sdf, grid, sph, tidx, 0.2))
        gh = torch.ones_like(h)
        gc, gr = pcdf.query_cost_backward(comp_sdf, grid, sph, tidx, 0.2, gh)
        cgc, cgr = ctx.query_cost_backward(c_sdf, grid, sph, tidx, 0.2, gh)
        assert torch.equal(gc, cgc) and torch.equal(gr, cgr)
    ctx.close()
    ctx.close()  # idempotent


def test_context_reserve_and_scratch_bound():
    d = dev()
    sc = scenes.scene_composite(seed=2, n=64, n_boxes=5, T=4, H=2)
    grid, caps = sc["grid"], sc["caps"]
    bound = pcdf.Context.scratch_bytes(grid, 4, 2)
    ctx = pcdf.Context(d)
    ctx.reserve(bound)
    occ = torch.from_numpy(sc["occ"]).to(d)
    before = torch.cuda.memory_allocated(d)
    sq, sdf = ctx.build_static_sdf(occ, grid)
    comp, _ = ctx.build_predicted_composite(sq, grid, caps, static_sdf=sdf, want_sdf=False)
    ref, _ = pcdf.build_predicted_composite(sq, grid, caps, static_sdf=sdf, want_sdf=False)
    assert torch.equal(comp, ref)
    # PyTorch's allocator holds only the outputs (the context's scratch is the
    # library's; the workspace call's own workspace was released)
    assert torch.cuda.memory_allocated(d) - before <= sq.numel() * 8 + 2 * comp.numel() * 4 + 4 * 2 ** 20


@pytest.mark.parametrize("use_graph", [False, True])
def test_build_batched_equals_the_batch_path(use_graph):
    d = dev()
    envs = scenes.scene_batch(seed=3, n_env=6)
    dev_envs = [(e["grid"], torch.from_numpy(e["occ"]).to(d), e["caps"]) for e in envs]
    b = pcdf.Batch(dev_envs)
    b.run()
    assert b.error() == 0
    ctx = pcdf.Context(d)
    outs = ctx.build_batched(dev_envs, use_graph=use_graph)
    for i, out in enumerate(outs):
        assert torch.equal(out, b.comp_sq[i]), i
