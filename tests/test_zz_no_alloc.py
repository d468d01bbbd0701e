"""goc_mass_noalloc: the total-mass diagnostic for callers that cannot
allocate device memory when they call it (real-time loops that must not stall
on the allocator, applications whose device memory is all owned by their own
pool).  Its scratch is a fixed array inside the library; this test checks,
through the C ABI, that it returns what goc_diagnostics returns, on two calls
in a row, on every grid kind (per-axis maps, the annular sector with the MIE,
a node-table grid) and storage format, that it leaves the caller's current
device as it was, and that it rejects lattices above its stated size limit."""
import ctypes

import pytest

import goc_inputs as gi
import paper_2607_15362_b300 as goc
from paper_2607_15362_b300 import _abi

pytestmark = pytest.mark.gpu


def _mass_noalloc(lat):
    out = ctypes.c_double()
    st = goc.lib().goc_mass_noalloc(lat._h, ctypes.byref(out))
    return st, out.value


def _spec(case):
    if case == "channel":
        prob = gi.poiseuille_channel()
    elif case == "cavity":
        prob = gi.Problem("cavity", 300, 211, {"kind": "tanh2", "beta": 1.5}, {"kind": "tanh2", "beta": 1.5},
                          {"Re": 400.0, "u_lid": 0.05, "mach_matched": True})
    elif case == "annulus_mhd":
        prob = gi.taylor_couette(n1=45, n2=11, r_in=6.0, sectors=9.0, Re=20.0, u_in=1.0, u_out=1.5)
    else:
        prob = gi.spiral_cavity(40, 37, phi=0.6)
    _, cs2 = goc.metric_info(prob.lattice_spec(1.0))
    spec = prob.lattice_spec(cs2)
    if case == "annulus_mhd":
        spec["walls"]["W"] = dict(spec["walls"]["W"], B=(0.02, 0.005))
        spec["mhd"] = {"tau_m": 0.9, "mu_m": 2.0, "B_init": (0.01, 0.004)}
    return spec


def _current_device():
    import torch
    return torch.cuda.current_device()


@pytest.mark.parametrize("case,storage", [("channel", "fp32"), ("channel", "fp16"), ("cavity", "fp32"),
                                          ("cavity", "bf16"), ("annulus_mhd", "fp32"), ("annulus_mhd", "fp16"),
                                          ("spiral", "fp32"), ("spiral", "bf16")])
def test_noalloc_mass_matches_diagnostics_twice(gpu, case, storage):
    lat = goc.Lattice(_spec(case), storage=storage)
    dev = _current_device()
    for steps in (70, 131):          # two calls in a row, the state changing in between
        lat.step(steps)
        st, m_noalloc = _mass_noalloc(lat)
        assert st == _abi.GOC_OK, goc.lib().goc_last_error()
        assert _current_device() == dev
        m_ref = lat.mass()
        assert m_noalloc == pytest.approx(m_ref, rel=1e-12)
    lat.close()


def test_noalloc_mass_rejects_lattices_above_the_limit(gpu):
    big = gi.Problem("poiseuille", 4096, 2049, {"kind": "uniform"}, {"kind": "tanh2", "beta": 1.0},
                     {"Re": 10.0, "tau": 0.8})
    assert big.nodes > 8388608
    _, cs2 = goc.metric_info(big.lattice_spec(1.0))
    lat = goc.Lattice(big.lattice_spec(cs2))
    st, _ = _mass_noalloc(lat)
    assert st == _abi.GOC_EINVAL
    assert b"at most 8388608" in goc.lib().goc_last_error()
    lat.close()
