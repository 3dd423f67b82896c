"""The multi-rank host logic of bench.py, on CPU with the gloo backend and
two ranks: a run's time is its slowest rank's, every rank builds its own
seeded particle bed, the whole-job throughput counts every rank's cells, and
only rank 0 of the reference arm does any work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench._dist()
        slowest = bench._max_over_ranks(1.5 + rank, "cpu")
        bed = bench._workload("tiny", rank)
        again = bench._workload("tiny", rank)
        dist.barrier()
        q.put((r, w, slowest, int(bed.seed), bed.xyz.tobytes() == again.xyz.tobytes(),
               float(bed.xyz.sum()), int(len(bed.radius))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    (r0, w0, t0, s0, same0, sum0, n0), (r1, w1, t1, s1, same1, sum1, n1) = got
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert t0 == t1 == 2.5                      # both ranks report the slower rank's time
    assert s1 - s0 == 1000                      # one seed per rank
    assert same0 and same1                      # a rank's bed is reproducible
    assert sum0 != sum1 and n0 > 0 and n1 > 0   # and the ranks' beds differ


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.25, "cpu") == 3.25          # no process group: the value itself
    assert bench._throughput(2, 1000, 10, 0.5) == pytest.approx(2 * 1000 * 10 / 0.5 / 1e6)

    class Args:
        pass
    assert bench.run_reference(Args(), 2, 1) is None           # ranks other than 0 do no work
