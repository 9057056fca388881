"""Replica layout of bench.py on world_size-2 gloo ranks (CPU).

Every rank analyses its own clip; the only collective is the timing: each
step time is the maximum over ranks and the whole-job throughput counts the
frames of all ranks.  The reference arm runs on rank 0 alone.
"""
import multiprocessing as mp
import os
import socket
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import io
    import contextlib
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 + r ms on the device and 5 - r ms end to end
        ms, ms_e2e = bench.reduce_max_over_ranks([10.0 + rank, 5.0 - rank], world)
        value = bench.job_throughput(world, 1500, ms)
        out = io.StringIO()
        with contextlib.redirect_stdout(out):
            rc = bench.run_reference(types.SimpleNamespace(gpus=world, steps=1, warmup=0, ref_frames=2)) \
                if rank != 0 else 0
        dist.barrier()
        q.put((rank, ms, ms_e2e, value, rc, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_replica_timing_and_throughput_on_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, ms, ms_e2e, value, rc, out = q.get(timeout=120)
        got[rank] = (ms, ms_e2e, value, rc, out)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        ms, ms_e2e, value, rc, out = got[rank]
        assert (ms, ms_e2e) == (11.0, 5.0)          # the slowest rank decides each time
        assert abs(value - 2 * 1500 / 0.011) < 1e-6   # frames of both ranks / slowest step
    ms, ms_e2e, value, rc, out = got[1]
    assert rc == 0 and out == ""                       # reference arm: rank 1 exits without work


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_over_ranks([3.5, 7], 1) == [3.5, 7.0]
    assert bench.job_throughput(1, 1500, 500.0) == 3000.0
