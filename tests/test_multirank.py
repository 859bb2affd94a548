"""The multi-rank logic of bench.py on CPU ranks (gloo, world size 2): each
rank owns its own environment (distinct seeds), the job's time is the
slowest rank's, the throughput counts every rank's voxels, and the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = bench.dist_env()
    ms = 10.0 + 5.0 * rank          # rank 1 is the slower one
    job = bench.slowest_rank_ms(ms, w, torch.device("cpu"))
    seeds = [None] * w
    dist.all_gather_object(seeds, bench.rank_seed(7, r))
    out.put((r, lr, w, job, bench.job_gvox_s(w, 4, 20, 256 ** 3, job), seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, lrank, world, job, gv, seeds) in enumerate(res):
        assert (rank, lrank, world) == (r, r, 2)
        assert job == 15.0                      # the max over ranks, seen by both
        assert gv == pytest.approx(2 * 4 * 20 * 256 ** 3 / 15e-3 / 1e9)
        assert len(set(seeds)) == 2             # independent environments


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.slowest_rank_ms(3.5, 1, torch.device("cpu")) == 3.5


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == ""
