"""CPU, two ranks over gloo: the host logic of bench.py's multi-GPU path.
Instances are independent, so N > 1 splits one batch into contiguous
instance ranges, one per rank, with no data-path collective; each rank's
handle starts its noise streams at its range's first instance, so the ranks
compute exactly the one-GPU batch (strong scaling).  The cross-rank steps are
the barrier around the timed region, the reduction of its result (the job's
time is the slowest rank's, its work the instances solved on all ranks) and
the final gather of every instance's U and cost.  The reference arm runs on
rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        # rank r timed 10 + 5 r ms and solved 250 + r of its replica's instances
        ms, solved = bench.reduce_over_ranks(10.0 + 5.0 * rank, 250 + rank, w, "cpu")
        dist.barrier()
        q.put((r, w, lr, ms, solved))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_the_sum_of_solved_instances():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    # every rank agrees on the job's time (max) and work (sum)
    assert all(o[3] == 15.0 and o[4] == 501 for o in out)
    # value = whole-job instances solved per second over the slowest rank's time
    steps = 1
    value = out[0][4] / (out[0][3] / steps / 1e3)
    assert value == pytest.approx(501 / 0.015)


def test_one_rank_reduction_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(12.5, 255, 1, "cpu") == (12.5, 255)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def _gather_worker(rank, world, port, batch, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = bench.partition(batch, rank, world)
        # this rank's per-instance results: U rows and costs that name their instance
        U = torch.stack([torch.arange(6, dtype=torch.float64) + 100.0 * i for i in range(lo, hi)])
        C = torch.tensor([[0.5 * i] for i in range(lo, hi)], dtype=torch.float64)
        Ug = bench.gather_rows(U, batch, world, "cpu")
        Cg = bench.gather_rows(C, batch, world, "cpu")
        q.put((rank, lo, hi, Ug.numpy(), Cg.view(-1).numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("batch", [256, 255, 3])
def test_two_ranks_split_one_batch_and_gather_it_in_instance_order(batch):
    import numpy as np
    import torch.multiprocessing as mp

    sys.path.insert(0, ROOT)
    import bench

    ranges = [bench.partition(batch, r, 2) for r in range(2)]
    assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == batch
    assert abs((ranges[0][1] - ranges[0][0]) - (ranges[1][1] - ranges[1][0])) <= 1
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, 2, port, batch, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the single-rank concatenation: every instance's row, in instance order
    U1 = np.stack([np.arange(6, dtype=float) + 100.0 * i for i in range(batch)])
    C1 = 0.5 * np.arange(batch, dtype=float)
    for rank, lo, hi, Ug, Cg in out:
        assert (lo, hi) == ranges[rank]
        assert np.array_equal(Ug, U1) and np.array_equal(Cg, C1)


def test_one_rank_partition_is_the_whole_batch():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.partition(256, 0, 1) == (0, 256)
    assert [bench.partition(10, r, 4) for r in range(4)] == [(0, 3), (3, 6), (6, 8), (8, 10)]
