"""Slab decomposition of one lattice along xi2 (one ghost-row exchange per
step), checked with the FP64 oracle on CPU ranks (gloo): two or three ranks
give, row for row, bitwise the state of the single lattice, and the ranks'
shares of the mass add up to its total.  Cases: a clustered lid-driven cavity
(walls on every side, a moving lid at the top rank), a Taylor-Green vortex on
a sine-stretched doubly periodic grid (every rank has neighbours on both
sides, the last rank wraps to the first) and a Hartmann strip with the MIE
(the ghost rows carry the vector populations too)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 60


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spec(case):
    sys.path.insert(0, ROOT)
    import goc_inputs as gi
    import oracle
    if case == "cavity":
        prob = gi.Problem("cavity", 20, 26, {"kind": "tanh2", "beta": 1.3}, {"kind": "tanh2", "beta": 1.6},
                          {"Re": 100.0, "u_lid": 0.05, "mach_matched": True})
    elif case == "taylor_green":
        prob = gi.taylor_green(n=24, a=0.3, u0=0.01, tau=0.8)
        prob = gi.Problem(prob.kind, 16, 24, {"kind": "sine", "a": 0.2}, prob.map2, prob.params)
    else:
        prob = gi.Problem("hartmann", 4, 40, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                          {"Ha": 10.0, "Re": 10.0, "tau": 1.0, "tau_m": 1.0})
    return prob.lattice_spec(oracle.build_metric(prob.lattice_spec(1.0)).cs2())


def _rank_main(rank, world, port, case, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle.slab import SlabOracle
    s = SlabOracle(_spec(case), rank, world)
    for _ in range(STEPS):
        s.step(1)
        s.exchange(dist)
    import torch
    m = torch.tensor([s.mass()], dtype=torch.float64)
    dist.all_reduce(m)
    out.put((rank, s.r0, s.r1, [a.copy() for a in s.fields()], float(m.item())))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("cavity", 2), ("cavity", 3), ("taylor_green", 2), ("hartmann", 2)])
def test_slab_ranks_reproduce_the_single_lattice_bitwise(case, world):
    sys.path.insert(0, ROOT)
    import oracle
    spec = _spec(case)
    ref = oracle.Oracle(spec, threads=1)
    ref.step(STEPS)
    want = ref.fields()
    mass = float(ref.state()[0].sum())
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    covered = 0
    for rank, r0, r1, fields, total in res:
        assert r0 == covered
        covered = r1
        for k, (a, b) in enumerate(zip(fields, want)):
            np.testing.assert_array_equal(a, b[r0:r1], err_msg=f"{case}: rank {rank}, field {k}")
        assert total == pytest.approx(mass, rel=1e-13)
    assert covered == spec["ny"]


def test_rows_are_split_as_evenly_as_possible():
    sys.path.insert(0, ROOT)
    from oracle.slab import rows_of
    for ny in (7, 26, 1024):
        for size in (1, 2, 3, 8):
            if ny < 2 * size:
                continue
            parts = [rows_of(r, size, ny) for r in range(size)]
            assert parts[0][0] == 0 and parts[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
