"""goc_mass_noalloc: the total-mass diagnostic for callers that cannot
allocate device memory when they call it (inside a stream capture, in a
real-time loop, or with all device memory owned by their own pool).  Its
scratch is a fixed array inside the library; this test checks, through the
C ABI, that it returns what goc_diagnostics returns, on two calls in a row,
and that it rejects lattices above its stated size limit."""
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


def _lattice(prob, storage="fp32"):
    _, cs2 = goc.metric_info(prob.lattice_spec(1.0))
    return goc.Lattice(prob.lattice_spec(cs2), storage=storage)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_noalloc_mass_matches_diagnostics_twice(gpu, storage):
    for prob in (gi.poiseuille_channel(),
                 gi.Problem("cavity", 300, 211, {"kind": "tanh2", "beta": 1.5}, {"kind": "tanh2", "beta": 1.5},
                            {"Re": 400.0, "u_lid": 0.05, "mach_matched": True})):
        lat = _lattice(prob, storage)
        for steps in (70, 131):          # two calls in a row, the state changing in between
            lat.step(steps)
            st, m_noalloc = _mass_noalloc(lat)
            assert st == _abi.GOC_OK, goc.lib().goc_last_error()
            m_ref = lat.mass()
            assert m_noalloc == pytest.approx(m_ref, rel=1e-12)
        lat.close()


def test_noalloc_mass_rejects_lattices_above_the_limit(gpu):
    big = gi.Problem("poiseuille", 4096, 2049, {"kind": "uniform"}, {"kind": "tanh2", "beta": 1.0},
                     {"Re": 10.0, "tau": 0.8})
    assert big.nodes > 8388608
    lat = _lattice(big)
    st, _ = _mass_noalloc(lat)
    assert st == _abi.GOC_EINVAL
    assert b"at most 8388608" in goc.lib().goc_last_error()
    lat.close()
