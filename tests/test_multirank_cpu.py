"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): independent
systems sharded over ranks with no data-path exchange, and the whole-job
aggregation (slowest rank's time, sum of every rank's work)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import ics

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        wl = bench.workload("batch32")
        # each rank derives its own share from the seeded sizes alone
        p, off, mine = bench.rank_batch(wl, rank, world)
        shares = [None] * world
        dist.all_gather_object(shares, (mine, int(off[-1]), p.n))
        # the particles of a shard are exactly its systems' particles
        systems, sizes, _ = ics.batch(wl["n_systems"], wl["seed"])
        first = systems[mine[0]]
        same = bool((p.x[:first.n] == first.x).all())
        # aggregation: max of the times, sum of the counts
        t, c = bench.aggregate(dist, torch.device("cpu"), 1.0 + rank, 10.0 * (rank + 1))
        q.put((rank, shares, same, t, c, [int(s) for s in sizes]))
    finally:
        dist.destroy_process_group()


def test_sharded_systems_and_aggregation_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    out.sort()
    shares = out[0][1]
    assert shares == out[1][1]  # both ranks agree on the assignment
    sizes = out[0][5]
    all_sys = sorted(s for mine, _, _ in shares for s in mine)
    assert all_sys == list(range(len(sizes)))  # every system exactly once
    loads = [sum(sizes[s] for s in mine) for mine, _, _ in shares]
    assert [n for _, n, _ in shares] == loads and [n for _, _, n in shares] == loads
    assert max(loads) - min(loads) <= max(sizes)  # greedy balance bound
    assert all(o[2] for o in out)
    for _, _, _, t, c, _ in out:
        assert t == 2.0 and c == 30.0


def test_shard_assignment_edge_cases():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.shard_systems([5, 3, 3], 1) == [[0, 1, 2]]
    assert bench.shard_systems([5, 3, 3], 2) == [[0], [1, 2]]
    assert bench.shard_systems([1, 1], 4) == [[0], [1], [], []]
    assert bench.aggregate(None, None, 3.5, 7) == (3.5, 7)


def _combine_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        gen = np.random.default_rng(11)
        full = torch.tensor(gen.normal(size=(1000, 4)).astype(np.float32))
        owner = torch.tensor(gen.integers(0, world, 1000))  # disjoint rows per rank
        acc = full.clone()
        acc[owner != rank] = 0.0
        bench.combine_forces(dist, acc)
        q.put((rank, bool(torch.equal(acc, full))))
    finally:
        dist.destroy_process_group()


def test_group_slices_combine_to_the_whole_system():
    """The N > 1 group-slice mode: each rank holds the forces of its own
    groups and zeros elsewhere; the all-reduce gives every rank the whole
    system's forces bit for bit."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_combine_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=300) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert [ok for _, ok in out] == [True, True]


def test_reference_arm_under_torchrun_prints_once():
    """bench.py --impl reference launched as the driver launches N > 1 runs
    (torchrun, two ranks, rendezvous on 127.0.0.1): rank 0 alone times the
    oracle and prints one line with n_gpus = 2 and the GPU arm's config for
    two ranks; every rank exits 0."""
    import json
    import subprocess

    sys.path.insert(0, ROOT)
    import bench

    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    out = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["config"] == bench.bench_config(bench.workload("plummer_1m"), 2)
    assert d["config"]["parallelism"] == "replicas"
