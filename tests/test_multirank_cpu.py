"""The multi-process path of bench.py (one process per GPU, launched by torchrun) on CPU with the
gloo backend and two ranks: the job's time is the slowest rank's, the rate counts every rank's
rays, each rank draws its own samples, and the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        m = bench.max_over_ranks(ms, world, device="cpu")
        rate = bench.whole_job_rate(1000.0, world, m)
        seed = bench.rank_seed(7, rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        buf = io.StringIO()
        ref_ran = None
        if rank != 0:
            # the reference arm returns at once on every rank but 0, printing nothing
            class A:
                gpus, steps, warmup = world, 1, 0
            with redirect_stdout(buf):
                ref_ran = bench.run_reference(A())
        out.put((rank, m, rate, seeds, buf.getvalue(), ref_ran))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_sum_rays():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, m, rate, seeds, printed, ref_ran in res:
        assert m == 15.0  # the slowest rank's time, on every rank
        assert rate == pytest.approx(2 * 1000.0 / 0.015)
        assert seeds == [7, 1007] and len(set(seeds)) == 2
        if rank == 1:
            assert printed == "" and ref_ran is None
