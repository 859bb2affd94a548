#!/usr/bin/env python
"""Throughput of the predicted composite distance field update on GB300.

Workload: a 256^3 grid of 4 cm voxels with a static map of 60 seeded boxes and
3 humans walking seeded 4-waypoint paths at 1.2 m/s, predicted over T = 20
steps of 0.1 s as capsules (r = 0.25 m, h = 1.8 m).  One step = the static
signed EDT of the map plus the T composite fields (int32 squared distances and
fp32 metres), i.e. the field update of one perception cycle.  The metric is
T * 256^3 voxels per step / step time, in Gvox/s.

Printed as one JSON line (rank 0).  Beside the main number it carries the
from-scratch comparator (full EDT per t), the hinge-cost query rate on the
trajectory-sphere workload, the roofline of the dominant kernel, the
end-to-end rate through the public API with host buffers, the CPU oracle
baseline and the SM clocks seen while timing.

``--impl reference`` times the CPU oracle (the plain C implementation under
oracle/) on the host cores instead, on bounded samples of the same workload.

Multi-GPU (torchrun): every rank updates its own independent environment
(seed + rank); there is no data-path collective; the timing is the max over
ranks and the value counts the voxels of all ranks ("weak" scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "Composite SDF Gvox/s at 256^3 x T=20 (static EDT + T composite fields per step)"
WORKLOAD = "predicted composite: 256^3 grid, 4 cm voxels, 60 boxes, 3 walking humans, T=20 x 0.1 s"
N_VOX, T_STEPS, H_HUMANS = 256, 20, 3
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-environment measurement")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-surrogate measurement")
    ap.add_argument("--profile-case", choices=["composite", "update", "static", "scratch", "query", "mlp", "train",
                                               "surrogate", "translated"],
                    default=None,
                    help="run one small untimed case of the named stage (for ncu captures) and exit")
    ap.add_argument("--profile-T", type=int, default=4, help="horizon of the --profile-case composite")
    return ap.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def rank_seed(seed: int, rank: int) -> int:
    """Each rank owns an independent environment (weak scaling, no exchange)."""
    return seed + 1000 * rank


def slowest_rank_ms(ms: float, world: int, device) -> float:
    """The job's time for a timed region: the largest of the ranks' times (one
    all-reduce MAX over the default process group; the local time at world 1)."""
    if world == 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gvox_s(world: int, steps: int, T: int, V: int, total_ms: float) -> float:
    """Whole-job throughput: every rank updates its own T fields of V voxels
    per step (weak scaling), over the slowest rank's time."""
    return world * steps * T * V / (total_ms * 1e-3) / 1e9


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def measured_bf16_peak():
    """Dense BF16 TF/s (cuBLAS burst) of MEASURED_PEAKS.json, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def sources_sha(names):
    """sha256 (16 hex digits) of the named csrc files, concatenated in order."""
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2201_05058_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.txt: one line per kernel or stage, `name sources=a,b
    sha=<hex> bytes=<n>`), if none of the sources it is compiled from changed
    since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        for line in f:
            parts = line.split()
            if not parts or parts[0] != kernel:
                continue
            kv = dict(x.split("=", 1) for x in parts[1:] if "=" in x)
            try:
                if sources_sha(kv["sources"].split(",")) != kv["sha"]:
                    return None
            except (OSError, KeyError):
                return None
            return float(kv["bytes"])
    return None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", self.gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline of the native arm; the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(sc, n_fields: int, z_depth: int):
    """Time the oracle on the static field plus n_fields composite fields of the
    scene cropped to its first z_depth slices.  Returns (seconds_static,
    seconds_per_field, voxels_per_field)."""
    import oracle
    occ = np.ascontiguousarray(sc["occ"][:z_depth])
    caps = sc["caps"]
    t0 = time.perf_counter()
    S_static = oracle.edt(occ)
    t1 = time.perf_counter()
    for t in range(n_fields):
        oracle.composite(S_static, oracle.dynamic_field(occ.shape, caps[t % caps.shape[0]]))
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / max(n_fields, 1), occ.size


def cpu_baseline(sc):
    """The oracle on one full update of the 256^3 scene (static field + T
    fields): the static field single-threaded (the oracle's own code), the T
    independent fields on a process pool over the host cores; plus a
    single-threaded sample of the same update."""
    import oracle
    from oracle.pool import FieldPool
    n_fields = 6
    ts1, tf1, vpf = oracle_sample(sc, n_fields, sc["grid"].nz)
    single = T_STEPS * vpf / (ts1 + T_STEPS * tf1) / 1e9
    pool = FieldPool(T_STEPS)
    try:
        t0 = time.perf_counter()
        S_static = oracle.edt(np.ascontiguousarray(sc["occ"]))
        ts = time.perf_counter() - t0
        tw = pool.fields(S_static, [sc["caps"][t] for t in range(T_STEPS)])
    finally:
        pool.close()
    step_s = ts + tw
    return {"value": T_STEPS * vpf / step_s / 1e9, "unit": "Gvox/s", "cores": pool.workers, "kind": "oracle",
            "sample": f"C oracle (separable EDT) on one full update of the 256^3 scene: static field "
                      f"single-threaded ({ts:.2f} s), the {T_STEPS} composite fields on a spawn pool of "
                      f"{pool.workers} processes ({tw:.2f} s wall)",
            "single_core": {"value": single, "cores": 1,
                            "sample": f"static field + {n_fields} of {T_STEPS} fields single-threaded, scaled "
                                      f"to the update ({ts1:.2f} s static, {tf1:.2f} s per field)"}}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import oracle
    from oracle.pool import FieldPool
    sc = scenes.scene_composite(seed=rank_seed(args.seed, 0), T=T_STEPS, H=H_HUMANS)
    pool = FieldPool(T_STEPS)
    W = pool.workers
    rounds = -(-T_STEPS // W)  # the T fields in rounds of W processes
    try:
        # one step is one full update of the scene cropped to `depth` z-slices:
        # the static field (single-threaded, as the oracle computes it) and the
        # T composite fields on the pool, all timed; `depth` keeps warmup +
        # steps within about two and a half minutes
        probe_s, probe_f, _ = oracle_sample(sc, 1, 64)
        per_slice = (probe_s + rounds * probe_f) / 64
        budget = 150.0 / max(args.steps + args.warmup, 1)
        depth = int(max(8, min(N_VOX, budget / per_slice)))
        occ = np.ascontiguousarray(sc["occ"][:depth])
        caps_all = [sc["caps"][t] for t in range(T_STEPS)]

        def step():
            t0 = time.perf_counter()
            S_static = oracle.edt(occ)
            pool.fields(S_static, caps_all)
            return time.perf_counter() - t0

        for _ in range(args.warmup):
            step()
        total = sum(step() for _ in range(args.steps))
        vox = args.steps * T_STEPS * occ.size
    finally:
        pool.close()
    value = vox / total / 1e9
    sample = (f"per step: one full update of the 256^3 scene cropped to {depth} z-slices, every part timed: the "
              f"static field single-threaded, then the {T_STEPS} composite fields on a spawn pool of {W} processes "
              f"({rounds} rounds); C oracle (separable EDT)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gvox/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [N_VOX] * 3, "T": T_STEPS,
                                            "H": H_HUMANS, "sample_depth": depth},
            "cpu_baseline": {"value": value, "unit": "Gvox/s", "cores": W, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gvox/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------

def bench_batched(dev, seed, steps):
    """64 ragged environments (per-axis sizes 64-320 x 64-320 x 64-128, T 5-30,
    1-4 humans, 4 cm voxels), int32 composite fields: one graph-captured
    persistent launch with autotuned tiles, against 64 separate per-environment
    calls on the same stream."""
    import torch

    import paper_2201_05058_gb300 as pcdf
    envs = scenes.scene_batch(seed=seed)
    dev_envs = [(e["grid"], torch.from_numpy(e["occ"]).to(dev), e["caps"]) for e in envs]
    vox_t = sum(e["grid"].nvox * e["caps"].shape[0] for e in envs)
    tiles, tune_ms = pcdf.batch_autotune(dev_envs, reps=2)
    b = pcdf.Batch(dev_envs, tiles=tiles)
    b.run()
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run()
    g.replay()
    torch.cuda.synchronize(dev)
    k = max(3, min(steps, 10))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for a, z in ev:
        a.record()
        g.replay()
        z.record()
    torch.cuda.synchronize(dev)
    graph_ms = float(np.mean([a.elapsed_time(z) for a, z in ev]))
    status = b.error()
    # the same work as separate calls (static + composite per environment)
    statics = [torch.empty(gr.shape, dtype=torch.int32, device=dev) for gr, _, _ in dev_envs]

    def separate():
        for (gr, occ, caps), st, out in zip(dev_envs, statics, b.comp_sq):
            pcdf.build_static_sdf(occ, gr, want_sdf=False, out_sq=st)
            pcdf.build_predicted_composite(st, gr, caps, want_sdf=False, out_sq=out)

    separate()
    torch.cuda.synchronize(dev)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for a, z in ev2:
        a.record()
        separate()
        z.record()
    torch.cuda.synchronize(dev)
    sep_ms = float(np.mean([a.elapsed_time(z) for a, z in ev2]))
    b.close()
    return {"workload": "64 ragged environments, 64-320 x 64-320 x 64-128 voxels, T 5-30, 1-4 humans, int32 fields",
            "voxel_fields": int(vox_t), "graph_ms": graph_ms, "gvox_s": vox_t / (graph_ms * 1e-3) / 1e9,
            "separate_calls_ms": sep_ms, "separate_gvox_s": vox_t / (sep_ms * 1e-3) / 1e9,
            "tiles": {"row_rows": tiles[0], "dyn_slices": tiles[1], "comp_t": tiles[2]},
            "autotune_best_ms": tune_ms, "status": status}


def bench_surrogate(dev, seed, n_train_scenes=500, n_samples=50_000_000, batch=262144, lr=6e-3):
    """Learned surrogate: trained on the exact fields of n_train_scenes 64^3
    scenes (5 cm voxels, one human walking over T = 20 steps) with n_samples
    samples, then 1M trajectory-sphere queries per plan step on held-out scenes:
    error against the exact composite field, fallback fraction, decision
    identity, and the time of the surrogate path against the exact paths."""
    import torch

    import paper_2201_05058_gb300 as pcdf
    from paper_2201_05058_gb300 import surrogate as sg

    def ev_time(fn, k=5):
        fn()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for a, z in ev:
            a.record()
            fn()
            z.record()
        torch.cuda.synchronize(dev)
        return float(np.median([a.elapsed_time(z) for a, z in ev]))

    T = 20
    train_sc = [scenes.scene_small_walking(seed=seed + 1000 + i, T=T, H=1) for i in range(n_train_scenes)]
    grid = train_sc[0]["grid"]
    t0 = time.perf_counter()
    fields, caps, tf = sg.exact_dynamic_fields(grid, [s["caps"] for s in train_sc], dev)
    torch.cuda.synchronize(dev)
    t_fields = time.perf_counter() - t0
    net = pcdf.SurrogateMLP(dev, seed=seed + 17)
    steps = max(1, n_samples // batch)
    t0 = time.perf_counter()
    hist = sg.train(net, grid, fields, caps, tf, T, steps=steps, batch=batch, lr=lr, log_every=max(1, steps // 8))
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    # one training step at the training batch: the network's products alone
    # (backward = forward + input and weight gradients), with the Adam update,
    # and the sample generation that feeds it
    xb, tb = pcdf.surrogate_samples(grid, fields, caps, tf, T, batch, 12345, 0.6)
    t_bwd = ev_time(lambda: net.backward(xb, tb), k=20)
    t_fwd_train = ev_time(lambda: net.forward(xb), k=20)

    def step():
        net.backward(xb, tb)
        net.adam(1e-5)
    t_step = ev_time(step, k=20)
    t_samples = ev_time(lambda: pcdf.surrogate_samples(grid, fields, caps, tf, T, batch, 777, 0.6), k=20)
    # the same step at a quarter of the batch (fixed costs per step weigh more)
    q = batch // 4
    xq, tq = xb[:q], tb[:q]
    t_bwd_q = ev_time(lambda: net.backward(xq, tq), k=20)
    # tensor-core products per row: forward 2 (16 256 + 2 256^2), input
    # gradients 2 (2 256^2), weight gradients 2 (2 256^2 + 256 16)
    train_flops = 802816 * batch
    peak, peak_src = measured_bf16_peak()
    del fields

    def queries(s):
        sc = scenes.scene_small_walking(seed=s, T=T, H=1)
        rng = np.random.default_rng(s)
        sph, tidx = scenes.spheres_along_paths(grid, 1024, 40, 25, rng, T=T)  # 1,024,000 spheres
        return sc, torch.from_numpy(sph).to(dev), torch.from_numpy(tidx).to(dev)

    def exact(sc, sph, tidx):
        sgrid = sc["grid"]
        occ = torch.from_numpy(sc["occ"]).to(dev)
        st_sq, st_sdf = pcdf.build_static_sdf(occ, sgrid)
        _, comp = pcdf.build_predicted_composite(st_sq, sgrid, sc["caps"], want_sq=False, static_sdf=st_sdf)
        big = 16.0
        d = (big + sph[..., 3]) - pcdf.query_cost(comp, sgrid, sph, tidx, big)
        return occ, st_sq, st_sdf, comp, d

    # The stated fallback band: |d - (eps + r)| < 0.05 m.  Certified: the
    # certificate of every query sends the uncertain ones to the exact path
    # too, so decisions are the exact path's by construction.
    BAND = 0.05

    def graph_ms(fn):
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            fn()
        torch.cuda.current_stream(dev).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return ev_time(g.replay)

    def evaluate(sc, sph, tidx, timing):
        sgrid = sc["grid"]
        occ, st_sq, st_sdf, comp, d_ex = exact(sc, sph, tidx)
        h_ex = pcdf.query_cost(comp, sgrid, sph, tidx, 0.2)
        cws = pcdf.composite_workspace(sgrid, sc["caps"], dev)
        pcdf.composite_prepare(sgrid, sc["caps"], cws)
        caps_dev = torch.from_numpy(np.ascontiguousarray(sc["caps"])).to(dev)
        # the network's own distances (every row where the humans can matter, no exact answers)
        _, d_pr, _ = pcdf.surrogate_query(net, sgrid, st_sq, st_sdf, sph, tidx, sc["caps"], 0.2, band=0.0,
                                          certified=False)
        # the plain band rule without the certificate
        h_u, _, nfb_u = pcdf.surrogate_query(net, sgrid, st_sq, st_sdf, sph, tidx, sc["caps"], 0.2, band=BAND,
                                             comp_workspace=cws, certified=False)
        # the certified plan step, and the same step without the network (zero residual: the
        # continuous capsule distance clamped to the certified interval)
        x, yi, cnt, bnd = pcdf.surrogate_select(sgrid, st_sdf, sph, tidx, T, caps_dev, 0.2, sync=False)
        y = net.infer_tc(x, count=cnt)
        h, _, nfb = pcdf.surrogate_finish(sgrid, st_sq, st_sdf, sph, tidx, T, sc["caps"], y, 0.2, BAND,
                                          comp_workspace=cws, y_index=yi, bounds=bnd)
        h0, _, nfb0 = pcdf.surrogate_finish(sgrid, st_sq, st_sdf, sph, tidx, T, sc["caps"], torch.zeros_like(y),
                                            0.2, BAND, comp_workspace=cws, y_index=yi, bounds=bnd)
        e = (d_pr - d_ex).abs()
        e = e[torch.isfinite(e)]
        nq = sph.numel() // 4
        r = {"max_err": float(e.max()), "mean_err": float(e.mean()),
             "fallback": int(nfb.item()) / nq, "wrong": int(((h > 0) != (h_ex > 0)).sum()),
             "rows": int(cnt.item()) / nq, "active": int((h_ex > 0).sum()) / nq,
             "h_err": float((h - h_ex).abs().mean()), "h_err0": float((h0 - h_ex).abs().mean()),
             "h_err_max": float((h - h_ex).abs().max()), "h_err0_max": float((h0 - h_ex).abs().max()),
             "wrong0": int(((h0 > 0) != (h_ex > 0)).sum()), "fallback0": int(nfb0.item()) / nq,
             "u_fallback": int(nfb_u.item()) / nq, "u_wrong": int(((h_u > 0) != (h_ex > 0)).sum()), "nq": nq}
        if not timing:
            return r

        def surrogate_path():
            # exact answers from the capsule-slab partials (the composite's
            # first stage, run for this plan step's capsules), one stream
            pcdf.composite_prepare(sgrid, sc["caps"], cws)
            pcdf.surrogate_query(net, sgrid, st_sq, st_sdf, sph, tidx, sc["caps"], 0.2, band=BAND,
                                 caps_dev=caps_dev, comp_workspace=cws)

        def surrogate_path_overlapped():
            # the capsule slab on a side stream while the certificate and the rows are computed
            pcdf.surrogate_step(net, sgrid, st_sq, st_sdf, sph, tidx, sc["caps"], 0.2, BAND, cws,
                                caps_dev=caps_dev)

        comp_out = torch.empty((T,) + sgrid.shape, dtype=torch.float32, device=dev)

        def exact_composite():
            # the T composite fields (kept on the device) and the query on them
            pcdf.composite_prepare(sgrid, sc["caps"], cws)
            pcdf.composite_finish(st_sq, sgrid, sc["caps"], cws, None, comp_out, static_sdf=st_sdf)
            pcdf.query_cost(comp_out, sgrid, sph, tidx, 0.2)

        def exact_scratch():
            _, fs = pcdf.build_from_scratch(occ, sgrid, sc["caps"])
            pcdf.query_cost(fs, sgrid, sph, tidx, 0.2)

        r["surrogate_ms"] = ev_time(surrogate_path)
        r["exact_composite_ms"] = ev_time(exact_composite)
        r["exact_scratch_ms"] = ev_time(exact_scratch)
        try:
            r["surrogate_graph_ms"] = graph_ms(surrogate_path_overlapped)
            r["exact_composite_graph_ms"] = graph_ms(exact_composite)
        except RuntimeError as exc:  # capture unsupported here: eager numbers only
            print(f"graph capture failed: {exc}", file=sys.stderr)
            r["surrogate_graph_ms"] = r["exact_composite_graph_ms"] = None
        return r, (sc, sph, tidx, st_sq, st_sdf, caps_dev, cws)

    stats = []
    for s in range(seed + 6000, seed + 6002):
        sc, sph, tidx = queries(s)
        res = evaluate(sc, sph, tidx, timing=(s == seed + 6001))
        if isinstance(res, tuple):
            res, keep = res
        stats.append(res)
    timing = stats[-1]
    sc, sph, tidx, st_sq, st_sdf, caps_dev, cws = keep
    # a larger workload of the same voxel size: the 12.8 x 12.8 x 3.2 m room
    # (256 x 256 x 64 voxels of 5 cm, 160 boxes, 3 walking humans), where
    # keeping all T fields costs 16 times as much and the queries do not grow
    room = scenes.scene_room(seed=seed + 7000, T=T, H=3)
    rsph, rtidx = scenes.spheres_along_paths(room["grid"], 1024, 40, 25, np.random.default_rng(seed + 7000), T=T)
    room_r, _ = evaluate(room, torch.from_numpy(rsph).to(dev), torch.from_numpy(rtidx).to(dev), timing=True)
    t_sur_local = ev_time(lambda: pcdf.surrogate_query(net, grid, st_sq, st_sdf, sph, tidx, sc["caps"], 0.2,
                                                       band=BAND, caps_dev=caps_dev))
    x_q = pcdf.surrogate_features(grid, sph, tidx, T, caps_dev)
    t_feat = ev_time(lambda: pcdf.surrogate_features(grid, sph, tidx, T, caps_dev))
    t_mlp = ev_time(lambda: net.forward(x_q))
    x_sel, _, _ = pcdf.surrogate_select(grid, st_sdf, sph, tidx, T, caps_dev, 0.2, certified=False)
    t_mlp_sel = ev_time(lambda: net.forward(x_sel))
    t_inf = ev_time(lambda: net.infer(x_q))
    t_inf_sel = ev_time(lambda: net.infer(x_sel))
    t_tc = ev_time(lambda: net.infer_tc(x_q))
    t_tc_sel = ev_time(lambda: net.infer_tc(x_sel))

    def speeds(r):
        out = {"surrogate_ms": r["surrogate_ms"], "surrogate_graph_ms": r["surrogate_graph_ms"],
               "exact_composite_ms": r["exact_composite_ms"], "exact_composite_graph_ms": r["exact_composite_graph_ms"],
               "exact_scratch_ms": r["exact_scratch_ms"],
               "speedup_vs_composite": r["exact_composite_ms"] / r["surrogate_ms"],
               "speedup_vs_scratch": r["exact_scratch_ms"] / r["surrogate_ms"]}
        if r["surrogate_graph_ms"] and r["exact_composite_graph_ms"]:
            out["graph_speedup_vs_composite"] = r["exact_composite_graph_ms"] / r["surrogate_graph_ms"]
            out["graph_speedup_vs_scratch"] = r["exact_scratch_ms"] / r["surrogate_graph_ms"]
        return out

    return {"workload": f"MLP 16-256-256-256-1 bf16/fp32, trained on {n_train_scenes} 64^3 scenes x T=20 "
                        f"({steps * batch} samples); 1,024,000 sphere queries per plan step on held-out scenes",
            "train_s": t_train, "fields_s": t_fields, "loss_first": hist[0][1], "loss_last": hist[-1][1],
            "train_lr": lr, "train_batch": batch, "train_steps": steps,
            "train_tflops": 802816 * steps * batch / t_train / 1e12,
            "train_frac_of_bf16_peak": 802816 * steps * batch / t_train / 1e12 / peak,
            "bf16_peak_tflops": peak, "bf16_peak_source": peak_src,
            "train_step": {"batch": batch, "backward_ms": t_bwd, "backward_tflops": train_flops / (t_bwd * 1e-3) / 1e12,
                           "forward_stored_ms": t_fwd_train, "step_with_adam_ms": t_step,
                           "step_tflops": train_flops / (t_step * 1e-3) / 1e12, "samples_ms": t_samples,
                           "flops_per_row": 802816, "quarter_batch": q, "quarter_backward_ms": t_bwd_q,
                           "quarter_backward_tflops": 802816 * q / (t_bwd_q * 1e-3) / 1e12},
            "band_m": BAND, "certified": True,
            "max_err_m": max(x["max_err"] for x in stats), "mean_err_m": float(np.mean([x["mean_err"] for x in stats])),
            "fallback_frac": float(np.mean([x["fallback"] for x in stats])),
            "wrong_decisions": int(sum(x["wrong"] for x in stats)), "queries": int(sum(x["nq"] for x in stats)),
            "decisions_identical": all(x["wrong"] == 0 for x in stats),
            "network_rows_frac": float(np.mean([x["rows"] for x in stats])),
            "active_frac": float(np.mean([x["active"] for x in stats])),
            "h_mean_abs_err_m": float(np.mean([x["h_err"] for x in stats])),
            "h_max_abs_err_m": max(x["h_err_max"] for x in stats),
            "without_network": {"h_mean_abs_err_m": float(np.mean([x["h_err0"] for x in stats])),
                                "h_max_abs_err_m": max(x["h_err0_max"] for x in stats),
                                "wrong_decisions": int(sum(x["wrong0"] for x in stats)),
                                "fallback_frac": float(np.mean([x["fallback0"] for x in stats])),
                                "what": "zero residual: the continuous capsule distance clamped to the certified "
                                        "interval, same certificate and band"},
            "uncertified_at_band_0_05_m": {"fallback_frac": float(np.mean([x["u_fallback"] for x in stats])),
                                           "wrong_decisions": int(sum(x["u_wrong"] for x in stats))},
            **speeds(timing),
            "room": {"workload": "12.8 x 12.8 x 3.2 m room, 256 x 256 x 64 voxels of 5 cm, 160 boxes, 3 walking "
                                 "humans, T = 20; 1,024,000 sphere queries; the same network",
                     "max_err_m": room_r["max_err"], "mean_err_m": room_r["mean_err"],
                     "fallback_frac": room_r["fallback"], "wrong_decisions": room_r["wrong"],
                     "queries": room_r["nq"], "network_rows_frac": room_r["rows"],
                     "h_mean_abs_err_m": room_r["h_err"], "without_network_h_mean_abs_err_m": room_r["h_err0"],
                     **speeds(room_r)},
            "surrogate_local_search_ms": t_sur_local, "features_ms": t_feat,
            "rows_to_network_frac": x_sel.shape[0] / (sph.numel() // 4), "mlp_forward_selected_ms": t_mlp_sel,
            "mlp_infer_ms": t_inf, "mlp_infer_selected_ms": t_inf_sel,
            "mlp_infer_tflops": 2 * 136193 * sph.numel() / 4 / (t_inf * 1e-3) / 1e12,
            "mlp_infer_tcgen05_ms": t_tc, "mlp_infer_tcgen05_selected_ms": t_tc_sel,
            "mlp_infer_tcgen05_tflops": 2 * 136193 * sph.numel() / 4 / (t_tc * 1e-3) / 1e12,
            "mlp_forward_ms": t_mlp,
            "mlp_tflops": 2 * 136193 * sph.numel() / 4 / (t_mlp * 1e-3) / 1e12}


def bench_translated(pcdf, dev, grid, caps, static_sq, static_sdf, comp_sq, comp_sdf, timed, k):
    """The paper's own primitive handling (Sec. 6): one field of the human
    primitive computed once and moved to each predicted position.  It is exact
    on lattice moves only, so every human is laid on the lattice relative to
    human 0 at t = 0; the exact composite path runs on the same lattice
    capsules for comparison."""
    import torch

    T = caps.shape[0]
    V = grid.nvox
    tr_caps = scenes.lattice_moves(caps, caps[0, 0])
    ref = tr_caps[0, 0]
    R = pcdf.template_radius(static_sq)
    tmpl, lo0 = pcdf.build_template(ref, R, dev)
    stream = torch.cuda.current_stream(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    tmpl, lo0 = pcdf.build_template(ref, R, dev)
    b.record(stream)
    torch.cuda.synchronize(dev)
    tmpl_ms = a.elapsed_time(b)
    lo = pcdf.lattice_placements(tr_caps, ref, lo0)
    ws_tr = pcdf.composite_workspace(grid, tr_caps, dev)

    def tr_step(_=None):
        pcdf.composite_translated(static_sq, grid, tmpl, lo, R, static_sdf=static_sdf, comp_sq=comp_sq,
                                  comp_sdf=comp_sdf)

    def exact_step(_=None):
        pcdf.composite_prepare(grid, tr_caps, ws_tr)
        pcdf.composite_finish(static_sq, grid, tr_caps, ws_tr, comp_sq, comp_sdf, static_sdf=static_sdf)

    tr_step()
    tr_ms, _ = timed(tr_step, k)
    exact_step()
    ex_ms, _ = timed(exact_step, k)
    tr_avg, ex_avg = float(np.mean(tr_ms)), float(np.mean(ex_ms))
    # bytes: the static pair read once, T int32 + fp32 fields written, the template read once
    tr_bytes = 8 * V + 8 * T * V + 4 * tmpl.numel()
    peak, peak_kind = measured_peaks()
    gbs = tr_bytes / (tr_avg * 1e-3) / 1e9
    return {"ms": tr_avg, "gvox_s": T * V / (tr_avg * 1e-3) / 1e9, "template_build_ms": tmpl_ms, "R": R,
            "template_box": list(tmpl.shape[::-1]), "exact_composite_same_caps_ms": ex_avg,
            "speedup_vs_exact_composite": ex_avg / tr_avg, "algorithmic_bytes": tr_bytes, "achieved_gbs": gbs,
            "frac_of_hbm": gbs / peak, "peak_source": peak_kind,
            "what": "k_composite_translated: T fields from one template moved by whole voxels (humans on the "
                    "lattice relative to human 0 at t = 0); exact composite path timed on the same capsules"}


def run_native(args):
    import torch

    import paper_2201_05058_gb300 as pcdf

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    sc = scenes.scene_composite(seed=rank_seed(args.seed, rank), T=T_STEPS, H=H_HUMANS)
    grid, caps = sc["grid"], sc["caps"]
    V = grid.nvox
    T = caps.shape[0]
    occ = torch.from_numpy(sc["occ"]).to(dev)
    static_sq = torch.empty(grid.shape, dtype=torch.int32, device=dev)
    static_sdf = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    comp_sq = torch.empty((T,) + grid.shape, dtype=torch.int32, device=dev)
    comp_sdf = torch.empty((T,) + grid.shape, dtype=torch.float32, device=dev)
    ws = pcdf.composite_workspace(grid, caps, dev)
    ws_upd = pcdf.update_workspace(grid, caps, dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(_=None):
        # one map update (pcdf_update_fields): the capsules' x+y pass on a side
        # stream beside the static build, then the composite's z stage
        pcdf.predicted_fields(occ, grid, caps, workspace=ws_upd, out_static_sq=static_sq, out_static_sdf=static_sdf,
                              out_sq=comp_sq, out_sdf=comp_sdf)

    def z_stage(z_events=None):
        # the composite's z stage alone (k_colmax + k_composite_z, all columns)
        if z_events:
            z_events[0].record(stream)
        pcdf.composite_finish(static_sq, grid, caps, ws, comp_sq, comp_sdf, static_sdf=static_sdf)
        if z_events:
            z_events[1].record(stream)

    def timed(fn, k, extra_events=False):
        """k steps, L2 flushed before each; per-step CUDA events on the launch stream."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        zev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)] \
            if extra_events else None
        for i in range(k):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            fn(zev[i] if zev else None)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        ms = [a.elapsed_time(b) for a, b in ev]
        zms = [a.elapsed_time(b) for a, b in zev] if zev else None
        return ms, zms

    # warm-up
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)

    gpu_uuid = None
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_uuid = str(local_rank)
    sampler = ClockSampler(gpu_uuid)
    sampler.start()
    time.sleep(0.2)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms, _ = timed(step, args.steps)
    torch.cuda.synchronize(dev)
    # the z stage's own time for its roofline, on the step's inputs (the slab
    # intermediate from one prepare), L2 flushed before each
    pcdf.composite_prepare(grid, caps, ws)
    _, z_ms = timed(z_stage, args.steps, extra_events=True)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    total_ms = slowest_rank_ms(float(sum(step_ms)), world, dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = job_gvox_s(world, args.steps, T, V, total_ms)

    # composite stage alone and the from-scratch comparator (same inputs)
    def comp_only(_=None):
        pcdf.composite_prepare(grid, caps, ws)
        pcdf.composite_finish(static_sq, grid, caps, ws, comp_sq, comp_sdf, static_sdf=static_sdf)

    ws_scr = None

    def scratch(_=None):
        pcdf.build_from_scratch(occ, grid, caps, out_sq=comp_sq, out_sdf=comp_sdf)

    k_side = max(3, min(args.steps, 10))
    comp_ms, _ = timed(comp_only, k_side)
    scratch(None)
    scr_ms, _ = timed(scratch, k_side)
    comp_avg = float(np.mean(comp_ms))
    scr_avg = float(np.mean(scr_ms))
    try:
        translated = bench_translated(pcdf, dev, grid, caps, static_sq, static_sdf, comp_sq, comp_sdf, timed,
                                      k_side)
    except (RuntimeError, ValueError) as exc:  # e.g. a template box beyond 512 voxels on a sparse map
        translated = {"skipped": str(exc)}

    # roofline of the dominant stage, timed by the events around
    # composite_finish (k_colmax, then k_composite_z). Algorithmic bytes of
    # the composite's second stage per the method: the T int32 + T fp32
    # fields out, the dynamic slab intermediate in, the static field (int32)
    # in once. The implementation also reads static_sq a second time for the
    # column maxima (writing one int32 per column) and reads static_sdf so as
    # to copy instead of taking square roots: implementation_bytes.
    _, S = pcdf.composite_slab(grid, caps)
    V2 = grid.nx * grid.ny
    z_bytes = 8 * T * V + 4 * T * S * V2 + 4 * V
    z_impl_bytes = (4 * V + 4 * V2) + (8 * V + 4 * T * S * V2 + 8 * T * V)
    z_avg_ms = float(np.mean(z_ms))
    peak, peak_kind = measured_peaks()
    achieved = z_bytes / (z_avg_ms * 1e-3) / 1e9
    traffic = recorded_traffic("z_stage")
    roofline = {"bound": "hbm", "kernel": "k_colmax + k_composite_z (composite_finish)", "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
                "algorithmic_bytes": z_bytes, "implementation_bytes": z_impl_bytes,
                "implementation_frac": z_impl_bytes / (z_avg_ms * 1e-3) / 1e9 / peak, "kernel_ms": z_avg_ms,
                "kernel_share_of_step": z_avg_ms / ms_per_step}

    # hinge-cost queries: 256 trajectories x 40 states x 30 spheres on T = 20
    # composite fields of a 64^3 scene
    qs = scenes.scene_small_walking(seed=rank_seed(args.seed, rank) + 4, T=20, H=1)
    qgrid = qs["grid"]
    q_static, _ = pcdf.build_static_sdf(torch.from_numpy(qs["occ"]).to(dev), qgrid)
    _, q_sdf = pcdf.build_predicted_composite(q_static, qgrid, qs["caps"], want_sq=False)
    sph, tidx = scenes.spheres_along_paths(qgrid, 256, 40, 30, np.random.default_rng(44), T=20)
    sph_d = torch.from_numpy(sph).to(dev)
    tid_d = torch.from_numpy(tidx).to(dev)
    g_h = torch.ones(tidx.shape, dtype=torch.float32, device=dev)
    nq = tidx.size
    for _ in range(3):
        pcdf.query_cost(q_sdf, qgrid, sph_d, tid_d, 0.2)
        pcdf.query_cost_backward(q_sdf, qgrid, sph_d, tid_d, 0.2, g_h)
    fwd_ms, _ = timed(lambda _=None: pcdf.query_cost(q_sdf, qgrid, sph_d, tid_d, 0.2), 20)
    bwd_ms, _ = timed(lambda _=None: pcdf.query_cost_backward(q_sdf, qgrid, sph_d, tid_d, 0.2, g_h), 20)
    query = {"workload": "256 trajectories x 40 states x 30 spheres on T=20 composite fields of 64^3 (5 cm)",
             "spheres": nq, "fwd_queries_per_s": nq / (np.mean(fwd_ms) * 1e-3),
             "bwd_queries_per_s": nq / (np.mean(bwd_ms) * 1e-3), "fields_l2_resident": True}

    # static-map utilities of the mapping pipeline (Sec. 8) on the 256^3 map:
    # the voxel clean-up filter and the collapsed 2-D map with its EDT
    filt = torch.empty_like(occ)
    f_ms, _ = timed(lambda _=None: pcdf.filter_voxels(occ, grid, 5, out=filt), k_side)
    z_top = int(round(1.8 / grid.vox))
    e2_ms, _ = timed(lambda _=None: pcdf.edt_2d(occ, grid, 0, z_top), k_side)
    mapping = {"voxel_filter": {"ms": float(np.mean(f_ms)), "gvox_s": V / (np.mean(f_ms) * 1e-3) / 1e9,
                                "hbm_gbs_min_bytes": 2 * V / (np.mean(f_ms) * 1e-3) / 1e9},
               "edt_2d": {"ms": float(np.mean(e2_ms)), "slices": z_top,
                          "what": "collapse of slices [0, 1.8 m) + signed EDT of the 256^2 map"}}

    # end to end through the public API with host buffers: pinned occupancy in,
    # capsules from host memory, composite float fields back to pinned memory
    occ_h = torch.from_numpy(sc["occ"]).pin_memory()
    out_h = torch.empty((T,) + grid.shape, dtype=torch.float32).pin_memory()
    occ_d = torch.empty_like(occ)

    bufs = {"occ": occ_d, "static_sq": static_sq, "static_sdf": static_sdf, "comp_sq": comp_sq,
            "comp_sdf": comp_sdf, "workspace": ws}

    def e2e_step(_=None):
        # fields copied to the host in chunks of 4 time steps while the next
        # chunk is computed
        pcdf.update_to_host(occ_h, grid, caps, out_h, bufs, chunk=4)

    e2e_step()
    k_e2e = max(3, min(args.steps, 10))
    e2e_ms, _ = timed(e2e_step, k_e2e)
    e2e_total = slowest_rank_ms(float(sum(e2e_ms)), world, dev)
    e2e = {"value": job_gvox_s(world, k_e2e, T, V, e2e_total), "unit": "Gvox/s",
           "h2d_bytes_per_step": int(occ_h.numel() + caps.nbytes), "d2h_bytes_per_step": int(out_h.numel() * 4),
           "ms_per_step": e2e_total / k_e2e,
           "what": "H2D occupancy (pinned) + capsules, static + composite, D2H of the T float fields (pinned), "
                   "copies of finished 4-step chunks overlapping the next chunk's z pass"}

    # a planner update: occupancy in from pinned host memory, the fields kept
    # on the device, the hinge costs of a trajectory set (256 x 40 x 30
    # spheres through the 256^3 room) computed there and read back
    sph_p, tidx_p = scenes.spheres_along_paths(grid, 256, 40, 30, np.random.default_rng(45), T=T)
    sph_pd = torch.from_numpy(sph_p).to(dev)
    tid_pd = torch.from_numpy(tidx_p).to(dev)
    h_host = torch.empty(tidx_p.shape, dtype=torch.float32).pin_memory()

    def planner_step(_=None):
        occ_d.copy_(occ_h, non_blocking=True)
        pcdf.predicted_fields(occ_d, grid, caps, workspace=ws_upd, out_static_sq=static_sq,
                              out_static_sdf=static_sdf, out_sq=comp_sq, out_sdf=comp_sdf)
        h_host.copy_(pcdf.query_cost(comp_sdf, grid, sph_pd, tid_pd, 0.2), non_blocking=True)

    planner_step()
    pl_ms, _ = timed(planner_step, k_e2e)
    pl_total = slowest_rank_ms(float(sum(pl_ms)), world, dev)
    e2e_planner = {"value": job_gvox_s(world, k_e2e, T, V, pl_total), "unit": "Gvox/s",
                   "h2d_bytes_per_step": int(occ_h.numel() + caps.nbytes),
                   "d2h_bytes_per_step": int(h_host.numel() * 4), "ms_per_step": pl_total / k_e2e,
                   "what": "H2D occupancy (pinned) + capsules, static + composite kept on the device, hinge costs "
                           "of 307,200 trajectory spheres on the 20 fields, D2H of the costs (pinned)"}

    batched = bench_batched(dev, rank_seed(args.seed, rank), args.steps) if not args.no_batched else None
    surrogate = bench_surrogate(dev, rank_seed(args.seed, rank)) if not args.no_surrogate else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc)

    launches_per_step = 6  # static: row, y, z; composite: capsule x+y, column maxima, fused z
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gvox/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [grid.nx, grid.ny, grid.nz], "vox_m": grid.vox, "T": T,
                       "H": H_HUMANS, "boxes": 60, "slab_slices": S,
                       "outputs": "int32 squared + fp32 metres, all T fields",
                       "l2": "flushed before every timed step (512 MB write)", "parallelism": f"replicas{world}"},
            "composite_only": {"ms": comp_avg, "gvox_s": T * V / (comp_avg * 1e-3) / 1e9},
            "from_scratch": {"ms": scr_avg, "gvox_s": T * V / (scr_avg * 1e-3) / 1e9,
                             "composite_speedup": scr_avg / comp_avg},
            "translated": translated, "query": query, "mapping": mapping, "batched": batched, "surrogate": surrogate, "roofline": roofline,
            "cpu_baseline": cpu, "e2e": e2e, "e2e_planner": e2e_planner,
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_profile_surrogate(dev):
    """The surrogate plan step (1,024,000 queries, 20 fields of 64^3) with a
    network trained briefly (200 scenes, 300 steps), twice inside the NVTX
    range "plan_step" after three warm-up steps."""
    import torch

    import paper_2201_05058_gb300 as pcdf
    from paper_2201_05058_gb300 import surrogate as sg
    T = 20
    train_sc = [scenes.scene_small_walking(seed=1000 + i, T=T, H=1) for i in range(200)]
    grid = train_sc[0]["grid"]
    fields, caps, tf = sg.exact_dynamic_fields(grid, [sc["caps"] for sc in train_sc], dev)
    net = pcdf.SurrogateMLP(dev, seed=17)
    sg.train(net, grid, fields, caps, tf, T, steps=300, batch=65536, lr=2e-3, log_every=100)
    del fields
    sc = scenes.scene_small_walking(seed=6001, T=T, H=1)
    sph, tidx = scenes.spheres_along_paths(grid, 1024, 40, 25, np.random.default_rng(6001), T=T)
    sph, tidx = torch.from_numpy(sph).to(dev), torch.from_numpy(tidx).to(dev)
    st_sq, st_sdf = pcdf.build_static_sdf(torch.from_numpy(sc["occ"]).to(dev), grid)
    caps_dev = torch.from_numpy(np.ascontiguousarray(sc["caps"])).to(dev)
    cws = pcdf.composite_workspace(grid, sc["caps"], dev)

    def step():
        pcdf.composite_prepare(grid, sc["caps"], cws)
        return pcdf.surrogate_query(net, grid, st_sq, st_sdf, sph, tidx, sc["caps"], 0.2, band=0.05,
                                    caps_dev=caps_dev, comp_workspace=cws)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("plan_step")
    for _ in range(2):
        _, _, nfb = step()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(f"profile case surrogate done: {int(nfb.item())} fallback queries")
    return 0


def run_profile_case(args):
    """One small untimed case for an ncu capture: the 256^3 scene with a short
    horizon (outputs still far larger than L2), run twice so a capture can skip
    the first (cold) launch."""
    import torch

    import paper_2201_05058_gb300 as pcdf
    dev = torch.device("cuda", 0)
    if args.profile_case == "mlp":
        # tcgen05 inference on 362,000 rows (the kept rows of a 1,024,000-query plan step)
        net = pcdf.SurrogateMLP(dev, seed=3)
        g = torch.Generator(device="cpu").manual_seed(1)
        x = torch.randn(362000, 16, generator=g).to(torch.bfloat16)
        x[:, 13:] = 0
        x = x.to(dev)
        for _ in range(2):
            net.infer_tc(x)
        torch.cuda.synchronize()
        print("profile case mlp done")
        return 0
    if args.profile_case == "train":
        # two training steps at 65,536 rows inside the NVTX range train_step
        # (forward with the head's backward, input and weight gradients, Adam)
        net = pcdf.SurrogateMLP(dev, seed=3)
        g = torch.Generator(device="cpu").manual_seed(1)
        x = torch.randn(65536, 16, generator=g).to(torch.bfloat16)
        x[:, 13:] = 0
        x, t = x.to(dev), torch.randn(65536, generator=g).to(dev)
        net.train_step(x, t, 1e-4)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("train_step")
        for _ in range(2):
            net.train_step(x, t, 1e-4)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        print("profile case train done")
        return 0
    if args.profile_case == "surrogate":
        return run_profile_surrogate(dev)
    sc = scenes.scene_composite(seed=args.seed, T=args.profile_T, H=H_HUMANS)
    grid, caps = sc["grid"], sc["caps"]
    occ = torch.from_numpy(sc["occ"]).to(dev)
    if args.profile_case == "translated":
        static_sq, static_sdf = pcdf.build_static_sdf(occ, grid)
        tr_caps = scenes.lattice_moves(caps, caps[0, 0])
        R = pcdf.template_radius(static_sq)
        tmpl, lo0 = pcdf.build_template(tr_caps[0, 0], R, dev)
        lo = pcdf.lattice_placements(tr_caps, tr_caps[0, 0], lo0)
        for _ in range(2):
            pcdf.composite_translated(static_sq, grid, tmpl, lo, R, static_sdf=static_sdf)
        torch.cuda.synchronize()
        print("profile case translated done")
        return 0
    if args.profile_case == "update":
        # the headline step: one-call update (capsule pass on a side stream)
        ws = pcdf.update_workspace(grid, caps, dev)
        for _ in range(2):
            pcdf.predicted_fields(occ, grid, caps, workspace=ws)
        torch.cuda.synchronize()
        print("profile case update done")
        return 0
    for _ in range(2):
        if args.profile_case in ("static", "composite"):
            static_sq, static_sdf = pcdf.build_static_sdf(occ, grid)
        if args.profile_case == "composite":
            pcdf.build_predicted_composite(static_sq, grid, caps, static_sdf=static_sdf)
        if args.profile_case == "scratch":
            pcdf.build_from_scratch(occ, grid, caps)
        if args.profile_case == "query":
            qs = scenes.scene_small_walking(seed=4, T=20, H=1)
            q_static, _ = pcdf.build_static_sdf(torch.from_numpy(qs["occ"]).to(dev), qs["grid"])
            _, q_sdf = pcdf.build_predicted_composite(q_static, qs["grid"], qs["caps"], want_sq=False)
            sph, tidx = scenes.spheres_along_paths(qs["grid"], 256, 40, 30, np.random.default_rng(44), T=20)
            pcdf.query_cost(q_sdf, qs["grid"], torch.from_numpy(sph).to(dev), torch.from_numpy(tidx).to(dev), 0.2)
    torch.cuda.synchronize()
    print(f"profile case {args.profile_case} done")
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
