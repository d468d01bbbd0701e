"""Slab decomposition of one lattice along xi2, run by the FP64 oracle (test
infrastructure: it checks that the decomposition reproduces the single
lattice exactly).

Rank r of `size` owns the global rows [r0, r1), the rows split as evenly as
possible (balanced by node count: every row has nx nodes).  Its local lattice
adds two ghost rows on each side that has a neighbouring rank (both sides
when xi2 is periodic).  The local lattice treats its xi2 edges as walls: the
ghost rows are then updated wrongly, but no owned row depends on that
update -- an owned row's new populations are streamed from rows one away,
collided with the normal derivatives of the fields one row further (Appendix
E: fields, second-order differences, collision, streaming), so the rows two
away must hold the right populations before the step and nothing beyond them
is read.  After every step each rank overwrites its ghost rows with the state
(populations, stored force, MIE populations) of the two rows of its
neighbour nearest the cut: one exchange per step and side.  The metric is
the global lattice's, sliced, and c_s^2 is the global one (q is the minimum
over all nodes, Eq. GOC-LBE_CFL).

The exchange uses torch.distributed point-to-point messages (gloo on the
CPU).  Its protocol: the rows a rank sends to its lower neighbour go into
that neighbour's upper ghost rows (tag 1), the rows it sends to its upper
neighbour into the lower ghost rows (tag 0); with two ranks on a periodic
axis both neighbours are the same rank and the tags keep the messages apart.
"""
from __future__ import annotations

import numpy as np

from .metric import Metric
from .oracle import Oracle, build_metric

GHOST = 2   # ghost rows per internal side


def rows_of(rank: int, size: int, ny: int) -> tuple[int, int]:
    """Global rows [r0, r1) owned by `rank`: ny split as evenly as possible."""
    base, extra = divmod(ny, size)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


class _SlabMetric(Metric):
    """Rows of a global metric; c_s^2 stays the global lattice's."""

    def cs2(self) -> float:
        return self._cs2


class SlabOracle:
    """The oracle on the slab of `rank` (local rows: ghosts, owned, ghosts)."""

    def __init__(self, spec: dict, rank: int, size: int, threads: int = 1):
        ny = int(spec["ny"])
        walls = spec["walls"]
        self.periodic = walls.get("S") is None
        self.rank, self.size = rank, size
        self.r0, self.r1 = rows_of(rank, size, ny)
        if self.r1 - self.r0 < GHOST:
            raise ValueError("each slab needs at least two rows")
        self.glo = GHOST if (self.periodic or self.r0 > 0) else 0
        self.ghi = GHOST if (self.periodic or self.r1 < ny) else 0
        self.rows = np.array([(self.r0 - self.glo + k) % ny for k in range(self.r1 - self.r0 + self.glo + self.ghi)])
        g = build_metric(spec)
        m = _SlabMetric.__new__(_SlabMetric)
        m.nx, m.ny = g.nx, len(self.rows)
        m._cs2 = g.cs2()
        for k in ("h1", "h2", "t11", "t12", "t21", "t22"):
            setattr(m, k, np.ascontiguousarray(getattr(g, k)[self.rows]))
        m.h1_axis, m.h2_axis = m.h1[0].copy(), m.h2[:, 0].copy()
        inner = {"u": 0.0, "B": (0.0, 0.0)}   # an internal cut: a wall for the local lattice
        lw = dict(walls)
        lw["S"] = walls["S"] if self.glo == 0 else inner
        lw["N"] = walls["N"] if self.ghi == 0 else inner
        m.wall = {"W": (g.wall["W"][0][self.rows], g.wall["W"][1][self.rows]),
                  "E": (g.wall["E"][0][self.rows], g.wall["E"][1][self.rows]),
                  "S": g.wall["S"] if self.glo == 0 else (m.h1[0].copy(), m.h2[0].copy()),
                  "N": g.wall["N"] if self.ghi == 0 else (m.h1[-1].copy(), m.h2[-1].copy())}
        local = dict(spec, ny=len(self.rows), walls=lw)
        if spec.get("init"):
            local["init"] = {k: np.asarray(v)[self.rows] for k, v in spec["init"].items()}
        self.oracle = Oracle(local, threads=threads, metric=m)

    @property
    def own(self) -> slice:
        """Local rows owned by this rank."""
        return slice(self.glo, self.glo + self.r1 - self.r0)

    def step(self, n: int = 1):
        self.oracle.step(n)

    def fields(self):
        """(rho, U1, U2, B1, B2) of the owned rows."""
        return tuple(a[self.own] for a in self.oracle.fields())

    def _planes(self):
        f, F1, F2, g = self.oracle.state()
        planes = [f[a] for a in range(9)] + [F1, F2]
        if self.oracle.spec.get("mhd"):
            planes += [g[c, a] for c in range(2) for a in range(5)]
        return f, F1, F2, g, planes

    def exchange(self, dist):
        """One ghost-row exchange with the neighbouring ranks (torch.distributed)."""
        import torch
        f, F1, F2, g, planes = self._planes()
        o0, o1 = self.own.start, self.own.stop
        lower = self.rank - 1 if self.rank > 0 else (self.size - 1 if self.periodic else None)
        upper = self.rank + 1 if self.rank < self.size - 1 else (0 if self.periodic else None)
        reqs, recv = [], {}
        if lower is not None:
            send = torch.from_numpy(np.stack([p[o0:o0 + GHOST] for p in planes]).copy())
            reqs.append(dist.isend(send, dst=lower, tag=1))
            recv["lo"] = torch.empty_like(send)
            reqs.append(dist.irecv(recv["lo"], src=lower, tag=0))
        if upper is not None:
            send = torch.from_numpy(np.stack([p[o1 - GHOST:o1] for p in planes]).copy())
            reqs.append(dist.isend(send, dst=upper, tag=0))
            recv["hi"] = torch.empty_like(send)
            reqs.append(dist.irecv(recv["hi"], src=upper, tag=1))
        for r in reqs:
            r.wait()
        for side, rows in (("lo", slice(0, self.glo)), ("hi", slice(o1, o1 + self.ghi))):
            if side in recv:
                data = recv[side].numpy()
                for p, d in zip(planes, data):
                    p[rows] = d
        self.oracle.set_state(f, F1, F2, g if self.oracle.spec.get("mhd") else None)

    def mass(self) -> float:
        """sum f over the owned rows (this rank's share of the total mass)."""
        f = self.oracle.state()[0]
        return float(f[:, self.own].sum())
