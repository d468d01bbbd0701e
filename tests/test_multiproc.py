"""Host logic of the multi-process benchmark (one independent replica per
rank, no collective on the data path): ranks rendezvous, the job time is the
slowest rank's, throughput counts every rank's units.  Two gloo ranks on the
CPU; the GPU runs use the same functions with NCCL."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, _ = bench.setup_dist("gloo")
    local_ms = 100.0 + 50.0 * r                 # rank 1 is the slow one
    ms = bench.allmax(w, local_ms, device="cpu")
    rate = bench.job_rate(w, 1.0e6, ms)
    bench.barrier(w)
    out.put((r, w, ms, rate))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms, rate in res:
        assert w == 2
        assert ms == pytest.approx(150.0)
        assert rate == pytest.approx(2 * 1.0e6 / 0.150 / 1e6)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.allmax(1, 3.0) == 3.0
    assert bench.job_rate(1, 5.0e6, 1000.0) == pytest.approx(5.0)
