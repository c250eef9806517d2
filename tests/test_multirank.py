"""The multi-process path of bench.py, on CPU with the gloo backend.

The path partitions work by system: each rank builds and times its own
independent system (different seed), and the only collective is one
all-reduce of the timing (max over ranks).  World size 2, loopback
rendezvous.  On the CPU the per-rank system is built and walked by the FP64
oracle (test infrastructure), through the same per-rank loop (bench.rank_run)
that times the library on a GPU.
"""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import og_inputs as gi
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = 10.0 + 5.0 * rank
        worst = bench.max_over_ranks(local_ms, ws, "cpu")
        pos, mass, _ = gi.config("uniform-32k", n=1000, seed=bench.seed_for_rank(rank))
        q.put((rank, worst, float(pos.sum()), bench.job_value(len(mass), ws, worst)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _physics_rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import time

    import torch.distributed as dist

    import bench
    import og_inputs as gi
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        pos, mass, prm = gi.config("uniform-32k", n=3000, seed=bench.seed_for_rank(rank))

        def step():
            t0 = time.perf_counter()
            acc, npp, npn = oracle.Tree(pos, mass, prm).force(nthreads=1)
            if rank == 1:
                time.sleep(0.05)                  # rank 1 is the slow one
            return (time.perf_counter() - t0) * 1e3, (acc, npp, npn)

        ms, (acc, npp, npn) = bench.rank_run(step, 2, ws, "cpu")
        q.put((rank, ms, acc, npp, npn))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_walk_their_own_systems_like_one_process():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    import og_inputs as gi
    import oracle
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_physics_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0][1] == got[1][1] >= 50.0        # both report the slower rank's time
    for rank, _, acc, npp, npn in got:
        pos, mass, prm = gi.config("uniform-32k", n=3000, seed=bench.seed_for_rank(rank))
        ref, rpp, rpn = oracle.Tree(pos, mass, prm).force(nthreads=1)
        assert np.array_equal(acc, ref) and np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
    assert not np.array_equal(got[0][2], got[1][2])   # each rank its own system


def test_two_ranks_take_the_slowest_time_and_their_own_systems():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, s0, v0), (r1, w1, s1, v1) = got
    assert (r0, r1) == (0, 1)
    assert w0 == w1 == 15.0                       # both see the slower rank
    assert s0 != s1                               # each rank its own system
    assert v0 == v1 == pytest.approx(2 * 1000 / 15e-3)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.seed_for_rank(0) == 12346       # rank 0 runs the single-GPU workload
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    calls = iter([(2.0, "a"), (4.0, "b")])
    assert bench.rank_run(lambda: next(calls), 2, 1, "cpu") == (3.0, "b")
    assert bench.job_value(2_097_152, 1, 10.0) == pytest.approx(2.097152e8)
    assert np.isfinite(bench.job_value(1, 8, 0.5))
