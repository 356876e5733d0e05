"""The replica path for several GPUs, exercised on the CPU with the gloo
backend and two ranks: each rank evaluates its own independent system (its
own seed), the bench line's whole-job value is the sum of the ranks' units
over the slowest rank's time, and the reference arm runs on rank 0 alone."""
import os
import socket

import torch.multiprocessing as mp

import bench
import workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_env()
        # units and times differ per rank: the whole job sums the units and takes the slowest time
        count, ms = 1000.0 * (rank + 1), 10.0 + 5.0 * rank
        tot, slowest = bench.whole_job(count, ms, w, torch.device("cpu"))
        # each rank's system is its own seed: replicas never share particles
        pos = workloads.make("plummer", 64, 2 + r)
        # the reference arm is rank 0's job only: the other ranks return at once
        ref_rc = bench.run_reference(None, None) if r != 0 else None
        dist.barrier()
        q.put((r, lr, w, tot, slowest, float(pos[:, :3].sum()), ref_rc))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, (rank, lr, w, tot, slowest, psum, ref_rc) in enumerate(out):
        assert (rank, lr, w) == (r, r, world)
        assert tot == 3000.0 and slowest == 15.0
    # different seeds: different systems
    assert out[0][5] != out[1][5]
    # rank 1 skipped the reference arm
    assert out[1][6] == 0


def test_single_process_whole_job_is_local():
    assert bench.whole_job(123.0, 4.5, 1, None) == (123.0, 4.5)
