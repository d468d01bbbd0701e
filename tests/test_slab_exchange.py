"""Host logic of the slab exchange (paper_2607_15362_b300.slab) on CPU ranks
(gloo): each rank's slab is a stand-in whose pack writes its rank and side
into the message and whose unpack records what arrived, so the test checks
who talks to whom with which tags -- two and three ranks, walls and a
periodic axis (where with two ranks both neighbours are the same rank).  On
the GPU the same Halo.exchange moves the device messages over NCCL."""
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


class _FakeSlab:
    """Messages of 8 bytes: (rank, side) as two int32 values."""

    halo_bytes = 8

    def __init__(self, rank):
        self.rank = rank
        self.got = {}
        self._bufs = {}

    def pack(self, lo, hi):
        import numpy as np
        for side, t in (("lo", lo), ("hi", hi)):
            if t is not None:
                self._bufs[side + "_send"].view(-1).numpy().view(np.int32)[:] = (self.rank, 0 if side == "lo" else 1)

    def unpack(self, lo, hi):
        import numpy as np
        for side, t in (("lo", lo), ("hi", hi)):
            if t is not None:
                self.got[side] = tuple(int(x) for x in self._bufs[side + "_recv"].numpy().view(np.int32))


def _rank_main(rank, world, periodic, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2607_15362_b300.slab import Halo
    fake = _FakeSlab(rank)
    h = Halo(fake, rank, world, periodic, "cpu")
    fake._bufs = {"lo_send": h.send_lo, "hi_send": h.send_hi, "lo_recv": h.recv_lo, "hi_recv": h.recv_hi}
    # the fake slab sees buffer addresses; map them back to the tensors
    addr = {t.data_ptr(): t for t in (h.send_lo, h.send_hi, h.recv_lo, h.recv_hi)}
    fake.pack = (lambda f: (lambda lo, hi: f(addr.get(lo), addr.get(hi))))(fake.pack)
    fake.unpack = (lambda f: (lambda lo, hi: f(addr.get(lo), addr.get(hi))))(fake.unpack)
    h.exchange(dist)
    out.put((rank, h.lower, h.upper, dict(fake.got)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, False), (3, False), (2, True), (3, True)])
def test_ghost_rows_come_from_the_right_neighbour(world, periodic):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, periodic, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, lower, upper, got in res:
        want_lower = rank - 1 if rank > 0 else (world - 1 if periodic else None)
        want_upper = rank + 1 if rank < world - 1 else (0 if periodic else None)
        assert (lower, upper) == (want_lower, want_upper)
        # the lower ghost rows hold the lower neighbour's top rows, the upper ones the upper neighbour's bottom rows
        assert got.get("lo") == ((lower, 1) if lower is not None else None)
        assert got.get("hi") == ((upper, 0) if upper is not None else None)


def test_rows_are_split_as_the_oracle_splits_them():
    sys.path.insert(0, ROOT)
    from oracle.slab import rows_of as oracle_rows
    from paper_2607_15362_b300.slab import rows_of
    for ny in (7, 64, 1000, 4096):
        for size in (1, 2, 3, 5, 8):
            assert [rows_of(r, size, ny) for r in range(size)] == [oracle_rows(r, size, ny) for r in range(size)]
