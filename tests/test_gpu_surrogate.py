"""The learned surrogate: its tensor-core forward and backward against the
fp64 oracle, the exactness of the fallback, and what training buys."""
import numpy as np
import pytest
import torch

import oracle
import scenes
from oracle import mlp as omlp
from tests import mlp_parity

pytestmark = pytest.mark.gpu

pcdf = pytest.importorskip("paper_2201_05058_gb300")
from paper_2201_05058_gb300 import surrogate as sg  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def rand_x(M, rng, d):
    x = np.zeros((M, 16), np.float32)
    x[:, :13] = rng.normal(0.0, 0.7, size=(M, 13))
    return torch.from_numpy(x).to(d).to(torch.bfloat16)


@pytest.mark.parametrize("M", [300, 4096])
def test_mlp_forward_and_gradients_match_oracle(M):
    """Every stored value of a training step, element by element, against the
    network's definition evaluated on the GPU's own inputs to that step
    (tests/mlp_parity.py): each BF16 activation and pre-activation gradient
    equals the rounding of its exact value unless that value lies within the
    FP32 accumulation bound of a rounding midpoint (then either neighbour);
    the layer-3 gradient matches the head's FP32 arithmetic bit for bit; every
    weight and bias gradient entry, the outputs and the loss lie within the
    FP32 accumulation bound of their exact sums."""
    d = dev()
    rng = np.random.default_rng(M)
    net = pcdf.SurrogateMLP(d, seed=3)
    x = rand_x(M, rng, d)
    t = torch.from_numpy(rng.normal(size=M).astype(np.float32)).to(d)
    y, loss = net.backward(x, t)
    torch.cuda.synchronize()
    stb = net.stored(M)
    # the forward pass: the same y and activations, and H3 (which the
    # training step uses on chip without storing it)
    y2 = net.forward(x)
    torch.cuda.synchronize()
    assert torch.equal(y2, y)
    stf = net.stored(M)
    assert torch.equal(stf["H1"], stb["H1"]) and torch.equal(stf["H2"], stb["H2"])
    P = net.params()
    st = {k: v.float().cpu().double().numpy() for k, v in stf.items()}
    st["y"] = y.cpu().double().numpy()
    xo = x.float().cpu().double().numpy()
    amb = mlp_parity.check_passes(P, xo, t.cpu().double().numpy(), st, net.grads(), float(loss.item()))
    assert all(v < 0.5 for v in amb.values()), amb
    # and the FP64 oracle with its own activations agrees on the loss
    want_loss, _, _ = omlp.loss_and_grad(P, xo, t.cpu().double().numpy(), rounding=True)
    assert abs(float(loss.item()) - want_loss) <= 1e-3 * want_loss
    # inference without a workspace: the same kernel, bit-identical (tail
    # tiles included); the legacy mma.sync kernel within FP32 rounding
    assert torch.equal(net.infer_tc(x), y)
    assert torch.equal(net.infer_tc(x[: M - 7]), y[: M - 7])
    scale = max(1.0, float(y.abs().max()))
    assert torch.allclose(net.infer(x), y, rtol=0, atol=1e-5 * scale)
    y_tc = net.infer_tc(x)
    # a row count on the device: the first count rows, the rest untouched
    for c in (M - 7, 0, M + 5, -3):
        cnt = torch.tensor([c], dtype=torch.int32, device=d)
        y_c = net.infer_tc(x, count=cnt)
        k = max(0, min(c, M))
        assert torch.equal(y_c[:k], y_tc[:k])


def test_training_step_over_many_tiles_per_cta():
    """A training step at several 128-row tiles per CTA and a ragged last tile
    (the A buffers, accumulators and barrier phases of the persistent kernels
    wrap; every weight-gradient job sums several tiles): stored values on
    sampled rows (all of the last tile) element by element, and every
    gradient entry, against the definition on the GPU's own inputs."""
    d = dev()
    sms = torch.cuda.get_device_properties(d).multi_processor_count
    M = sms * 128 * 3 + 77
    rng = np.random.default_rng(5)
    net = pcdf.SurrogateMLP(d, seed=11)
    x = rand_x(M, rng, d)
    t = torch.from_numpy(rng.normal(size=M).astype(np.float32)).to(d)
    y, loss = net.backward(x, t)
    stb = net.stored(M)
    y2 = net.forward(x)
    torch.cuda.synchronize()
    assert torch.equal(y2, y) and not torch.isnan(y).any()
    stf = net.stored(M)
    P = net.params()
    full = {k: v.float().cpu().double().numpy() for k, v in stf.items()}
    full["y"] = y.cpu().double().numpy()
    xo = x.float().cpu().double().numpy()
    to = t.cpu().double().numpy()
    g = net.grads()
    rows = np.unique(np.concatenate([rng.choice(M, 600, replace=False), np.arange(M - 77, M)]))
    # the row-wise values on the sampled rows; the head's dy needs the true M
    sub = {k: v[rows] for k, v in full.items()}
    amb = {}
    E, S = mlp_parity.dense(xo[rows], P["W1"], P["b1"])
    amb["H1"] = mlp_parity.check_stored("H1", sub["H1"], E, S, 16, True)
    E, S = mlp_parity.dense(sub["H1"], P["W2"], P["b2"])
    amb["H2"] = mlp_parity.check_stored("H2", sub["H2"], E, S, 256, True)
    E, S = mlp_parity.dense(sub["H2"], P["W3"], P["b3"])
    amb["H3"] = mlp_parity.check_stored("H3", sub["H3"], E, S, 256, True)
    f32 = np.float32
    # the head's arithmetic needs the true M: emulate it on all rows, compare the stored dy
    dyf, d3f = mlp_parity.head_gradient(P, full["y"], to, full["H3"], full["dy"])
    d3 = d3f[rows]
    E, S = d3 @ P["W3"], np.abs(d3) @ np.abs(P["W3"])
    amb["D2"] = mlp_parity.check_stored("D2", sub["D2"], E, S, 256, False, mask=sub["H2"] > 0)
    E, S = sub["D2"] @ P["W2"], np.abs(sub["D2"]) @ np.abs(P["W2"])
    amb["D1"] = mlp_parity.check_stored("D1", sub["D1"], E, S, 256, False, mask=sub["H1"] > 0)
    assert all(v < 0.5 for v in amb.values()), amb
    # every gradient entry over all M rows
    dyf = dyf.astype(np.float64)
    H3 = full["H3"]
    mlp_parity.check_sum("grad w4", g["w4"], H3.T @ dyf, np.abs(H3).T @ np.abs(dyf), M)
    mlp_parity.check_sum("grad b4", g["b4"], dyf.sum(), np.abs(dyf).sum(), M)
    for l, (D, Hp) in {3: (d3f, full["H2"]), 2: (full["D2"], full["H1"]), 1: (full["D1"], xo)}.items():
        mlp_parity.check_sum(f"grad W{l}", g[f"W{l}"], D.T @ Hp, np.abs(D).T @ np.abs(Hp), M)
        mlp_parity.check_sum(f"grad b{l}", g[f"b{l}"], D.sum(0), np.abs(D).sum(0), M)
    e = (full["y"].astype(f32) - to.astype(f32)).astype(np.float64)
    mlp_parity.check_sum("loss", float(loss.item()), float(np.sum(e * e) / M), float(np.sum(e * e) / M), 2 * M)


def test_tensor_core_inference_over_many_tiles_per_cta():
    """The persistent kernel at several 128-row tiles per CTA (every SM busy,
    a ragged last tile): accumulators alternate across tiles, barrier phases
    wrap, and each tile's head sums are added one tile later.  All rows
    against the bit-exact mma.sync kernel, sampled rows against the oracle."""
    d = dev()
    sms = torch.cuda.get_device_properties(d).multi_processor_count
    M = sms * 128 * 5 + 77
    rng = np.random.default_rng(12)
    net = pcdf.SurrogateMLP(d, seed=9)
    x = rand_x(M, rng, d)
    y_ref = net.infer(x)
    y_tc = net.infer_tc(x)
    torch.cuda.synchronize()
    assert not torch.isnan(y_tc).any()
    scale = max(1.0, float(y_ref.abs().max()))
    assert float((y_tc - y_ref).abs().max()) <= 1e-5 * scale
    rows = np.concatenate([rng.choice(M, 500, replace=False), np.arange(M - 77, M)])
    want, _ = omlp.forward(net.params(), x[rows].float().cpu().double().numpy(), rounding=True)
    got = y_tc[rows].cpu().double().numpy()
    assert np.max(np.abs(got - want)) <= 2e-2 * max(1.0, np.max(np.abs(want)))
    # the same rows through a device row count
    cnt = torch.tensor([M - 77], dtype=torch.int32, device=d)
    assert torch.equal(net.infer_tc(x, count=cnt)[: M - 77], y_tc[: M - 77])


def test_adam_step():
    d = dev()
    rng = np.random.default_rng(1)
    net = pcdf.SurrogateMLP(d, seed=4)
    x = rand_x(1024, rng, d)
    t = torch.from_numpy(rng.normal(size=1024).astype(np.float32)).to(d)
    net.backward(x, t)
    p0 = net._f32("master").clone()
    g = net._f32("grad").clone()
    net.adam(1e-3)
    p1 = net._f32("master")
    # first Adam step: m = 0.1 g, v = 0.001 g^2, bias-corrected -> p - lr g / (|g| + eps)
    want = p0 - 1e-3 * g / (g.abs() + 1e-8)
    live = torch.ones_like(g, dtype=torch.bool)
    live[:4096] = (torch.arange(4096, device=d) % 16) < 13  # zero input columns stay
    live[136193:] = False
    assert torch.allclose(p1[live], want[live], atol=1e-6, rtol=1e-4)
    # the BF16 copy follows the master copy
    half = net._bf16()
    assert torch.equal(half[4096:4096 + 65536], p1[4352:4352 + 65536].to(torch.bfloat16))
    # the tensor-core kernels read packed copies of W2 and W3, which the step
    # refreshed: after more steps a forward pass still follows the network's
    # definition with the current weights, layer by layer
    for _ in range(3):
        net.backward(x, t)
        net.adam(1e-2)
    y = net.forward(x)
    torch.cuda.synchronize()
    st = {k: v.float().cpu().double().numpy() for k, v in net.stored(1024).items()}
    st["y"] = y.cpu().double().numpy()
    amb = mlp_parity.check_forward(net.params(), x.float().cpu().double().numpy(), st)
    assert all(v < 0.5 for v in amb.values()), amb
    assert torch.equal(net.infer_tc(x), y)


def scene_set(seeds, grid_only=False):
    out = [scenes.scene_small_walking(seed=s, T=20, H=1) for s in seeds]
    return out


def exact_query(sc, d, sph, tidx, eps):
    grid = sc["grid"]
    static_sq, static_sdf = pcdf.build_static_sdf(torch.from_numpy(sc["occ"]).to(d), grid)
    _, comp_sdf = pcdf.build_predicted_composite(static_sq, grid, sc["caps"], want_sq=False, static_sdf=static_sdf)
    h = pcdf.query_cost(comp_sdf, grid, sph, tidx, eps)
    # exact distance from the same kernel (an eps above every distance in the
    # grid keeps the hinge linear; 16 m keeps the fp32 resolution near 2e-6 m)
    big = 16.0
    hb = pcdf.query_cost(comp_sdf, grid, sph, tidx, big)
    dd = (big + sph[..., 3]) - hb
    return static_sq, static_sdf, h, dd


def test_fallback_everywhere_is_bit_exact():
    d = dev()
    sc = scenes.scene_small_walking(seed=77, T=20, H=1)
    grid = sc["grid"]
    rng = np.random.default_rng(2)
    sph_np, tidx_np = scenes.spheres_along_paths(grid, 16, 40, 8, rng, T=20)
    sph = torch.from_numpy(sph_np).to(d)
    tidx = torch.from_numpy(tidx_np).to(d)
    static_sq, static_sdf, h_ex, _ = exact_query(sc, d, sph, tidx, 0.2)
    net = pcdf.SurrogateMLP(d, seed=5)
    # untrained, band and error bound huge: every answer comes from the
    # fallback, except where the static field provably wins the whole cell
    # (the rows the selection skips), which is exact too
    h, _, nfb = pcdf.surrogate_query(net, grid, static_sq, static_sdf, sph, tidx, sc["caps"], 0.2, band=1.0e9)
    assert 0 < int(nfb.item()) <= sph_np.size // 4
    assert torch.equal(h, h_ex)
    # the same answers from the capsule-slab partials of the composite's first stage
    ws = pcdf.composite_workspace(grid, sc["caps"], d)
    pcdf.composite_prepare(grid, sc["caps"], ws)
    h2, _, nfb2 = pcdf.surrogate_query(net, grid, static_sq, static_sdf, sph, tidx, sc["caps"], 0.2, band=1.0e9,
                                       comp_workspace=ws)
    assert int(nfb2.item()) == int(nfb.item())
    assert torch.equal(h2, h_ex)


def test_full_size_plan_step_exact_path_is_bit_exact():
    """The bench's plan step at full size: 1,024,000 spheres (1024
    trajectories x 40 states x 25 spheres) on 20 fields of 64^3, through
    surrogate_step (capsule slab on a side stream, device row count, slab
    fallback).  Untrained network and an unbounded band: every answer comes
    from the exact path or from a cell the static field provably wins, so h
    equals the exact composite query bit for bit."""
    d = dev()
    sc = scenes.scene_small_walking(seed=6001, T=20, H=1)
    grid = sc["grid"]
    rng = np.random.default_rng(6001)
    sph_np, tidx_np = scenes.spheres_along_paths(grid, 1024, 40, 25, rng, T=20)
    sph = torch.from_numpy(sph_np).to(d)
    tidx = torch.from_numpy(tidx_np).to(d)
    assert sph.numel() // 4 == 1024000
    static_sq, static_sdf, h_ex, _ = exact_query(sc, d, sph, tidx, 0.2)
    net = pcdf.SurrogateMLP(d, seed=21)
    ws = pcdf.composite_workspace(grid, sc["caps"], d)
    h, _, nfb = pcdf.surrogate_step(net, grid, static_sq, static_sdf, sph, tidx, sc["caps"], 0.2, 1.0e9, ws)
    torch.cuda.synchronize()
    assert 0 < int(nfb.item()) <= 1024000
    assert torch.equal(h, h_ex)


def test_fallback_exact_with_several_humans():
    d = dev()
    sc = scenes.scene_small_walking(seed=78, T=6, H=3)
    grid = sc["grid"]
    rng = np.random.default_rng(3)
    sph_np = scenes.spheres_uniform(grid, 3000, rng)
    tidx_np = rng.integers(0, 6, 3000).astype(np.int32)
    sph = torch.from_numpy(sph_np).to(d)
    tidx = torch.from_numpy(tidx_np).to(d)
    static_sq, static_sdf, h_ex, _ = exact_query(sc, d, sph, tidx, 0.2)
    net = pcdf.SurrogateMLP(d, seed=6)
    h, _, nfb = pcdf.surrogate_query(net, grid, static_sq, static_sdf, sph, tidx, sc["caps"], 0.2, band=1.0e9)
    assert 0 < int(nfb.item()) <= 3000
    assert torch.equal(h, h_ex)
    ws = pcdf.composite_workspace(grid, sc["caps"], d)
    pcdf.composite_prepare(grid, sc["caps"], ws)
    h2, _, _ = pcdf.surrogate_query(net, grid, static_sq, static_sdf, sph, tidx, sc["caps"], 0.2, band=1.0e9,
                                    comp_workspace=ws)
    assert torch.equal(h2, h_ex)
    # and the oracle agrees with both (within the cost tolerance)
    comp = oracle.predicted_composite(oracle.edt(sc["occ"]), sc["caps"])
    sdf_o = np.stack([oracle.sdf_from_sq(comp[t], grid.vox) for t in range(6)])
    want, _ = oracle.hinge_cost(sdf_o, grid.origin, grid.vox, sph_np, tidx_np, 0.2)
    assert np.max(np.abs(h.cpu().numpy() - want)) <= 1e-5


def test_surrogate_step_replays_from_a_cuda_graph():
    """The plan step (capsule-slab partials, selection, network, exact
    fallback) has no host round trip, so it captures into a CUDA graph; a
    replay on new query contents gives the eager answers bit for bit."""
    d = dev()
    sc = scenes.scene_small_walking(seed=81, T=20, H=1)
    grid = sc["grid"]
    rng = np.random.default_rng(9)
    sph_np, tidx_np = scenes.spheres_along_paths(grid, 64, 40, 8, rng, T=20)
    sph = torch.from_numpy(sph_np).to(d)
    tidx = torch.from_numpy(tidx_np).to(d)
    occ = torch.from_numpy(sc["occ"]).to(d)
    static_sq, static_sdf = pcdf.build_static_sdf(occ, grid)
    caps_dev = torch.from_numpy(np.ascontiguousarray(sc["caps"])).to(d)
    net = pcdf.SurrogateMLP(d, seed=8)
    ws = pcdf.composite_workspace(grid, sc["caps"], d)

    def step():
        pcdf.composite_prepare(grid, sc["caps"], ws)
        return pcdf.surrogate_query(net, grid, static_sq, static_sdf, sph, tidx, sc["caps"], 0.2, band=0.3,
                                    caps_dev=caps_dev, comp_workspace=ws)

    def step_overlapped():
        return pcdf.surrogate_step(net, grid, static_sq, static_sdf, sph, tidx, sc["caps"], 0.2, 0.3, ws,
                                   caps_dev=caps_dev)

    side = torch.cuda.Stream(d)
    side.wait_stream(torch.cuda.current_stream(d))
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream(d).wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        h_g, d_g, n_g = step()
    # new query contents in the captured buffers
    sph2_np, tidx2_np = scenes.spheres_along_paths(grid, 64, 40, 8, np.random.default_rng(10), T=20)
    sph.copy_(torch.from_numpy(sph2_np).to(d))
    tidx.copy_(torch.from_numpy(tidx2_np).to(d))
    graph.replay()
    torch.cuda.synchronize()
    h_e, d_e, n_e = step()
    assert torch.equal(h_g, h_e) and torch.equal(d_g, d_e)
    assert int(n_g.item()) == int(n_e.item()) > 0
    # the overlapped plan step (capsule slab on a side stream), eager and as a graph
    h_o, d_o, n_o = step_overlapped()
    assert torch.equal(h_o, h_e) and torch.equal(d_o, d_e) and int(n_o.item()) == int(n_e.item())
    side = torch.cuda.Stream(d)
    side.wait_stream(torch.cuda.current_stream(d))
    with torch.cuda.stream(side):
        step_overlapped()
    torch.cuda.current_stream(d).wait_stream(side)
    graph2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph2):
        h_g2, d_g2, _ = step_overlapped()
    graph2.replay()
    torch.cuda.synchronize()
    assert torch.equal(h_g2, h_e) and torch.equal(d_g2, d_e)


def test_row_selection_skips_only_static_cells():
    """The selection keeps a row wherever the exact capsule field beats the
    static field at some corner of the query's cell (the skip rule is a
    proof, checked here against the exact fields)."""
    d = dev()
    sc = scenes.scene_small_walking(seed=79, T=8, H=2)
    grid, caps = sc["grid"], sc["caps"]
    rng = np.random.default_rng(4)
    sph_np = scenes.spheres_uniform(grid, 4000, rng)
    tidx_np = rng.integers(0, 8, 4000).astype(np.int32)
    sph = torch.from_numpy(sph_np).to(d)
    tidx = torch.from_numpy(tidx_np).to(d)
    static_sq, static_sdf = pcdf.build_static_sdf(torch.from_numpy(sc["occ"]).to(d), grid)
    x, yi, _ = pcdf.surrogate_select(grid, static_sdf, sph, tidx, 8, torch.from_numpy(caps).to(d), 0.2,
                                     certified=False)
    yi = yi.cpu().numpy().reshape(4000, 2)
    kept = yi >= 0
    assert 0 < kept.sum() < kept.size
    assert np.array_equal(np.sort(yi[kept]), np.arange(kept.sum()))  # slots 0 .. kept - 1, each once
    S = oracle.edt(sc["occ"])
    dyns = [oracle.dynamic_field(grid.shape, caps[t]) for t in range(8)]
    for q in np.nonzero(~kept.any(axis=1))[0][:300]:
        dyn = dyns[tidx_np[q]]
        u = (sph_np[q, :3].astype(np.float64) - np.asarray(grid.origin)) / grid.vox - 0.5
        lo = [int(min(max(np.floor(u[a]), 0), grid.shape[2 - a] - 2)) for a in range(3)]
        for k in range(8):
            i, j, kk = lo[0] + (k & 1), lo[1] + ((k >> 1) & 1), lo[2] + ((k >> 2) & 1)
            assert S[kk, j, i] <= dyn[kk, j, i], (q, k)


CERT_SCENES = {
    # walking humans standing on the floor, one and three of them
    "walking_1": lambda: scenes.scene_small_walking(seed=91, T=8, H=1),
    "walking_3": lambda: scenes.scene_small_walking(seed=92, T=6, H=3),
}


def cert_cases():
    """(name, grid, occ, caps): the walking scenes plus capsules cut by the
    grid boundary, overlapping, below sqrt(3)/2 voxel in radius, and slanted."""
    out = [(k, *(lambda sc: (sc["grid"], sc["occ"], sc["caps"]))(f())) for k, f in CERT_SCENES.items()]
    grid = scenes.Grid(48, 40, 36, 0.05)
    occ, _ = scenes.boxes_occupancy(grid, 8, np.random.default_rng(5))
    caps = np.array([[[-40, 100, 0, -40, 100, 480, 90], [300, 300, 8, 300, 300, 16, 60],
                      [320, 300, 100, 420, 340, 300, 70]],
                     [[620, 560, 200, 640, 570, 470, 80], [100, 500, 470, 120, 520, 479, 10],
                      [330, 310, 110, 410, 330, 290, 75]]], np.int32)
    out.append(("boundary_overlap_thin", grid, occ, caps))
    return out


@pytest.mark.parametrize("case", range(3))
def test_certificate_brackets_the_exact_distance(case):
    """Every query's certified interval [d_lo, d_hi] holds the exact
    composite path's interpolated distance, whatever the network (both
    selection modes give the same bounds), and a query's decision is certain
    exactly when the threshold lies outside the interval."""
    d = dev()
    name, grid, occ, caps = cert_cases()[case]
    T = caps.shape[0]
    rng = np.random.default_rng(100 + case)
    sph_np = scenes.spheres_uniform(grid, 20000, rng)
    tidx_np = rng.integers(0, T, 20000).astype(np.int32)
    sph = torch.from_numpy(sph_np).to(d)
    tidx = torch.from_numpy(tidx_np).to(d)
    static_sq, static_sdf = pcdf.build_static_sdf(torch.from_numpy(occ).to(d), grid)
    _, comp = pcdf.build_predicted_composite(static_sq, grid, caps, want_sq=False, static_sdf=static_sdf)
    big = 16.0
    d_ex = ((big + sph[..., 3]) - pcdf.query_cost(comp, grid, sph, tidx, big)).cpu().numpy()
    caps_dev = torch.from_numpy(np.ascontiguousarray(caps)).to(d)
    _, _, b0 = pcdf.surrogate_select(grid, static_sdf, sph, tidx, T, caps_dev, 0.2, certified=True)
    _, _, b1 = pcdf.surrogate_select(grid, static_sdf, sph, tidx, T, caps_dev, 0.2, certified=False)
    assert torch.equal(b0, b1)
    b = b0.cpu().numpy()
    finite = np.isfinite(d_ex)
    assert np.all(b[finite, 0] <= d_ex[finite]) and np.all(d_ex[finite] <= b[finite, 1]), name
    # infinite exact distances (empty maps) sit at the matching end
    assert np.all((d_ex[~finite] > 0) <= (b[~finite, 1] == np.inf))
    # the intervals are tight where the static field decides the cell
    width = b[:, 1] - b[:, 0]
    assert np.mean(width[np.isfinite(width)] <= 1e-3) > 0.3, name


def test_certified_decisions_are_the_exact_ones_for_any_network():
    """At the stated band of 0.05 m, and with no band at all, every collision
    decision of the certified query equals the exact path's, for networks
    whose outputs are anything (untrained, and forced far off)."""
    d = dev()
    for name, grid, occ, caps in cert_cases():
        T = caps.shape[0]
        rng = np.random.default_rng(7)
        sph_np = scenes.spheres_uniform(grid, 20000, rng)
        tidx_np = rng.integers(0, T, 20000).astype(np.int32)
        sph = torch.from_numpy(sph_np).to(d)
        tidx = torch.from_numpy(tidx_np).to(d)
        static_sq, static_sdf = pcdf.build_static_sdf(torch.from_numpy(occ).to(d), grid)
        _, comp = pcdf.build_predicted_composite(static_sq, grid, caps, want_sq=False, static_sdf=static_sdf)
        h_ex = pcdf.query_cost(comp, grid, sph, tidx, 0.2)
        caps_dev = torch.from_numpy(np.ascontiguousarray(caps)).to(d)
        ws = pcdf.composite_workspace(grid, caps, d)
        pcdf.composite_prepare(grid, caps, ws)
        x, yi, cnt, bounds = pcdf.surrogate_select(grid, static_sdf, sph, tidx, T, caps_dev, 0.2, sync=False)
        for y in (torch.zeros(x.shape[0], device=d), torch.full((x.shape[0],), 5.0, device=d),
                  torch.full((x.shape[0],), -5.0, device=d), pcdf.SurrogateMLP(d, seed=13).infer_tc(x, count=cnt)):
            for band in (0.05, 0.0):
                h, _, _ = pcdf.surrogate_finish(grid, static_sq, static_sdf, sph, tidx, T, caps, y, 0.2, band,
                                                comp_workspace=ws, y_index=yi, bounds=bounds)
                assert torch.equal(h > 0, h_ex > 0), (name, band)


def test_slab_fallback_edge_cases():
    """Slab fallback with capsules cut by the grid boundary, touching the
    floor and ceiling, a capsule covering the whole grid, and none at all."""
    d = dev()
    grid = scenes.Grid(40, 36, 30, 0.05)
    rng = np.random.default_rng(9)
    occ, _ = scenes.boxes_occupancy(grid, 6, rng)
    caps_sets = [
        np.array([[[-40, 100, 0, -40, 100, 480, 90], [300, 300, 8, 300, 300, 16, 60]],
                  [[620, 560, 200, 640, 570, 470, 80], [100, 500, 470, 120, 520, 479, 40]]], np.int32),
        np.array([[[320, 288, 240, 320, 288, 240, 8000]]], np.int32),
        np.array([[[-8000, -8000, -8000, -8000, -8000, -7000, 80]]], np.int32),
    ]
    sph_np = scenes.spheres_uniform(grid, 2000, rng)
    sph = torch.from_numpy(sph_np).to(d)
    for caps in caps_sets:
        T = caps.shape[0]
        tidx = torch.from_numpy(rng.integers(0, T, 2000).astype(np.int32)).to(d)
        static_sq, static_sdf = pcdf.build_static_sdf(torch.from_numpy(occ).to(d), grid)
        _, comp_sdf = pcdf.build_predicted_composite(static_sq, grid, caps, want_sq=False, static_sdf=static_sdf)
        h_ex = pcdf.query_cost(comp_sdf, grid, sph, tidx, 0.2)
        net = pcdf.SurrogateMLP(d, seed=7)
        ws = pcdf.composite_workspace(grid, caps, d)
        pcdf.composite_prepare(grid, caps, ws)
        h, _, _ = pcdf.surrogate_query(net, grid, static_sq, static_sdf, sph, tidx, caps, 0.2, band=1.0e9,
                                       comp_workspace=ws)
        assert torch.equal(h, h_ex)


def test_training_gains_and_decisions_stay_identical():
    """Train on 40 scenes x 20 steps.  On held-out scenes, at the stated
    fallback band of 0.05 m, the certified query makes every collision
    decision of the exact path with the trained network and with an
    untrained one; what training gains is the accuracy of the costs it
    answers without the exact path (and of the network's own distances)."""
    d = dev()
    train_sc = scene_set(range(2000, 2040))
    grid = train_sc[0]["grid"]
    fields, caps, tf = sg.exact_dynamic_fields(grid, [s["caps"] for s in train_sc], d)
    net = pcdf.SurrogateMLP(d, seed=11)
    hist = sg.train(net, grid, fields, caps, tf, 20, steps=1500, batch=32768, lr=2e-3, log_every=100)
    assert hist[-1][1] < 0.1 * hist[0][1]
    untrained = pcdf.SurrogateMLP(d, seed=12)

    def evaluate(model, certified, band):
        res = []
        for s in range(3100, 3104):
            sc = scenes.scene_small_walking(seed=s, T=20, H=1)
            rng = np.random.default_rng(s)
            sph_np, tidx_np = scenes.spheres_along_paths(grid, 64, 40, 8, rng, T=20)
            sph = torch.from_numpy(sph_np).to(d)
            tidx = torch.from_numpy(tidx_np).to(d)
            static_sq, static_sdf, h_ex, d_ex = exact_query(sc, d, sph, tidx, 0.2)
            ws = pcdf.composite_workspace(grid, sc["caps"], d)
            pcdf.composite_prepare(grid, sc["caps"], ws)
            h, dp, nfb = pcdf.surrogate_query(model, grid, static_sq, static_sdf, sph, tidx, sc["caps"], 0.2,
                                              band=band, comp_workspace=ws, certified=certified)
            res.append((h, dp, nfb, h_ex, d_ex))
        return res

    for model in (net, untrained):
        for h, _, nfb, h_ex, _ in evaluate(model, True, 0.05):
            assert torch.equal(h > 0, h_ex > 0)
            assert int(nfb.item()) > 0

    def h_error(model):
        res = evaluate(model, True, 0.05)
        return float(torch.cat([(r[0] - r[3]).abs().reshape(-1) for r in res]).mean())

    def d_error(model):
        res = evaluate(model, False, 0.0)
        e = torch.cat([(r[1] - r[4]).abs().reshape(-1) for r in res])
        return float(e[torch.isfinite(e)].mean())

    assert h_error(net) < 0.5 * h_error(untrained)
    assert d_error(net) < 0.2 * d_error(untrained)
