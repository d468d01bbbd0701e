"""Ghost-row exchange of a lattice cut into slabs along xi2, one slab per
rank and GPU (goc_create_slab).

Rank r owns the rows rows_of(r, size, ny); after creation and after every
step each slab packs the two owned rows nearest each cut into device
buffers, sends them to the neighbouring ranks and unpacks what it receives
into its ghost rows.  The rows sent down go into the lower neighbour's upper
ghost rows (tag 1), the rows sent up into the upper neighbour's lower ghost
rows (tag 0): with two ranks on a periodic axis both neighbours are the same
rank and the tags keep the messages apart.  The messages are plain device
buffers, so the transport is torch.distributed point-to-point (NCCL between
GPUs) -- into local staging buffers that the unpack kernel reads.
"""
from __future__ import annotations


def rows_of(rank: int, size: int, ny: int) -> tuple[int, int]:
    """Global rows [r0, r1) of `rank`: ny rows split as evenly as possible
    (every row holds nx nodes, so this balances the node count)."""
    base, extra = divmod(ny, size)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def neighbours(rank: int, size: int, periodic: bool):
    """(lower, upper) ranks, None where the slab meets a wall."""
    lower = rank - 1 if rank > 0 else (size - 1 if periodic else None)
    upper = rank + 1 if rank < size - 1 else (0 if periodic else None)
    return lower, upper


class Halo:
    """The four message buffers of one slab on its device and the exchange."""

    def __init__(self, slab, rank: int, size: int, periodic: bool, device):
        import torch
        self.slab = slab
        self.lower, self.upper = neighbours(rank, size, periodic)
        n = max(1, slab.halo_bytes)
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = (
            torch.empty(n, dtype=torch.uint8, device=device) for _ in range(4))

    def pack(self):
        self.slab.pack(self.send_lo.data_ptr() if self.lower is not None else None,
                       self.send_hi.data_ptr() if self.upper is not None else None)

    def unpack(self):
        self.slab.unpack(self.recv_lo.data_ptr() if self.lower is not None else None,
                         self.recv_hi.data_ptr() if self.upper is not None else None)

    def exchange(self, dist):
        """pack, point-to-point messages with the neighbours, unpack."""
        self.pack()
        ops = []
        if self.lower is not None:
            ops.append(dist.P2POp(dist.isend, self.send_lo, self.lower, tag=1))
            ops.append(dist.P2POp(dist.irecv, self.recv_lo, self.lower, tag=0))
        if self.upper is not None:
            ops.append(dist.P2POp(dist.isend, self.send_hi, self.upper, tag=0))
            ops.append(dist.P2POp(dist.irecv, self.recv_hi, self.upper, tag=1))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        self.unpack()
