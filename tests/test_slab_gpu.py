"""A lattice cut into slabs along xi2 (goc_create_slab), all on one GPU: the
ghost rows are exchanged after creation and after every step by device
copies between the slabs' message buffers, in place of the messages the
ranks of a multi-GPU run send each other.  The owned rows of the slabs are
bitwise the rows of the single lattice -- FP32, FP16 and BF16 storage (the
per-row storage reference of the 16-bit storage, refreshed every 16 steps
here, travels with the ghost rows), walls and moving lid, a doubly periodic
grid, the MIE -- and the slabs' mass shares add up to its mass."""
import numpy as np
import pytest
import torch

import goc_inputs as gi
import oracle
import paper_2607_15362_b300 as goc
from paper_2607_15362_b300.slab import Halo, rows_of

pytestmark = pytest.mark.gpu
STEPS = 200


def spec_of(prob):
    return prob.lattice_spec(oracle.build_metric(prob.lattice_spec(1.0)).cs2())


CASES = {
    "cavity": gi.Problem("cavity", 37, 53, {"kind": "tanh2", "beta": 1.3}, {"kind": "tanh2", "beta": 1.7},
                         {"Re": 100.0, "u_lid": 0.05, "mach_matched": True}),
    "taylor_green": gi.Problem("taylor_green", 32, 40, {"kind": "sine", "a": 0.2}, {"kind": "sine", "a": 0.3},
                               {"u0": 0.01, "tau": 0.8}),
    "hartmann": gi.Problem("hartmann", 4, 64, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                           {"Ha": 10.0, "Re": 10.0, "tau": 1.0, "tau_m": 1.0}),
}


def exchange(halos):
    for h in halos:
        h.pack()
    for h in halos:
        if h.lower is not None:
            h.recv_lo.copy_(halos[h.lower].send_hi)
        if h.upper is not None:
            h.recv_hi.copy_(halos[h.upper].send_lo)
    for h in halos:
        h.unpack()


def run_slabs(spec, size, storage, reference_every=0):
    stream = torch.cuda.current_stream().cuda_stream
    periodic = spec["walls"].get("S") is None
    slabs = [goc.Slab(spec, *rows_of(r, size, spec["ny"]), storage=storage, stream=stream,
                      reference_every=reference_every) for r in range(size)]
    halos = [Halo(s, r, size, periodic, "cuda") for r, s in enumerate(slabs)]
    exchange(halos)
    for _ in range(STEPS):
        for s in slabs:
            s.step(1)
        exchange(halos)
    torch.cuda.synchronize()
    return slabs


@pytest.mark.parametrize("case,size,storage", [("cavity", 2, "fp32"), ("cavity", 3, "fp32"),
                                               ("taylor_green", 2, "fp32"), ("hartmann", 2, "fp32"),
                                               ("cavity", 2, "fp16"), ("hartmann", 3, "bf16"),
                                               ("taylor_green", 3, "fp16")])
def test_slabs_reproduce_the_single_lattice_bitwise(gpu, case, size, storage):
    spec = spec_of(CASES[case])
    ref_every = 16 if storage != "fp32" else 0
    stream = torch.cuda.current_stream().cuda_stream
    whole = goc.Lattice(spec, storage=storage, stream=stream, fixed_launch=True, reference_every=ref_every)
    whole.step(STEPS)
    want = whole.moments()
    slabs = run_slabs(spec, size, storage, ref_every)
    covered = 0
    for s in slabs:
        assert s.row_begin == covered
        got = s.owned_moments()
        for k, (a, b) in enumerate(zip(got, want)):
            np.testing.assert_array_equal(a, b[s.row_begin:s.row_end], err_msg=f"{case} field {k}")
        covered = s.row_end
    assert covered == spec["ny"]
    assert sum(s.mass() for s in slabs) == pytest.approx(whole.mass(), rel=1e-12)
    for s in slabs:
        s.close()
    whole.close()


def test_slabs_match_the_oracle(gpu):
    """The slab run against the FP64 oracle of the whole lattice (FP32
    velocity relative L2 <= 1e-5)."""
    spec = spec_of(CASES["cavity"])
    o = oracle.Oracle(spec, threads=8)
    o.step(STEPS)
    fo = o.fields()
    slabs = run_slabs(spec, 2, "fp32")
    u = np.concatenate([np.stack(s.owned_moments()[1:3]) for s in slabs], axis=1)
    err = np.linalg.norm(u - np.stack(fo[1:3])) / np.linalg.norm(np.stack(fo[1:3]))
    assert err <= 1e-5


def test_slab_arguments_are_checked(gpu):
    spec = spec_of(CASES["cavity"])
    with pytest.raises(goc.GocError):
        goc.Slab(spec, 10, 11)            # fewer than two rows
    with pytest.raises(goc.GocError):
        goc.Slab(spec, 40, 60)            # beyond the lattice
    s = goc.Slab(spec, 0, 26)
    with pytest.raises(goc.GocError):
        s.step(2)                         # one step between exchanges
    with pytest.raises(goc.GocError):
        s.run_until(1e-6, 100)            # the residual is global
    s.close()
