"""The N > 1 host path on CPU: world-size-2 process groups on the gloo backend.

Queries are independent problems, so ranks share no data: each solves its own slice of one
seeded draw (weak scaling) and the job time is the maximum over the ranks. These tests check
that host logic of bench.py with two processes, and that the reference arm prints exactly one
line under torchrun.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import bench
    import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        wl = synth.WORKLOADS["uneven_n120"]
        q = bench.rank_queries(wl, 37, rank, world)
        mu = torch.from_numpy(q.mu)
        n = torch.from_numpy(q.n.astype(np.int64))
        mus = [torch.empty_like(mu) for _ in range(world)]
        ns = [torch.empty_like(n) for _ in range(world)]
        dist.all_gather(mus, mu)
        dist.all_gather(ns, n)
        t_max = bench.max_over_ranks(1.5 + rank, "cpu")
        if rank == 0:
            np.save(os.path.join(out_dir, "mu.npy"), torch.cat(mus).numpy())
            np.save(os.path.join(out_dir, "n.npy"), torch.cat(ns).numpy())
        np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t_max]))
    finally:
        dist.destroy_process_group()


def test_ranks_split_the_batch_and_take_the_max_time(tmp_path):
    import torch.multiprocessing as mp

    import synth
    world = 2
    mp.spawn(_worker, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    wl = synth.WORKLOADS["uneven_n120"]
    full = synth.make_queries(wl, batch=37 * world)
    # the ranks' slices, gathered in rank order, are the whole draw: disjoint and complete
    np.testing.assert_array_equal(np.load(tmp_path / "mu.npy"), full.mu)
    np.testing.assert_array_equal(np.load(tmp_path / "n.npy"), full.n)
    for r in range(world):
        assert np.load(tmp_path / f"t{r}.npy")[0] == 2.5


@pytest.mark.timeout(300)
def test_reference_arm_under_torchrun():
    """Two ranks under torchrun: rank 0 times the oracle and prints one JSON line, rank 1 exits
    without work; the job exits 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node",
           "2", "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--workload", "single_n20", "--steps", "2", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=280, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
