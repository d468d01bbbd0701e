"""The standard uniform-grid central-moment LBM (goc_exec.scheme = 1, the
matched-accuracy comparator) against the FP64 oracle run at h1 = h2 = 1 with
the cubic correction terms dropped, where the GOC scheme reduces to it (the
oracle's reduction is pinned bitwise in tests/test_oracle_pins.py)."""
import numpy as np
import pytest

import goc_inputs as gi
import oracle
import paper_2607_15362_b300 as goc

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def uniform_spec(prob):
    spec = prob.lattice_spec(1.0 / 3.0)
    spec["gi"] = 0
    return spec


@pytest.mark.parametrize("nx,ny", [(64, 48), (131, 7), (9, 130)])
def test_standard_cavity_matches_the_oracle(gpu, nx, ny):
    """Walls on all sides and a moving lid; sizes with ragged blocks in x and
    y and interior blocks (131 x 7)."""
    prob = gi.Problem("cavity", nx, ny, {"kind": "uniform"}, {"kind": "uniform"}, {"Re": 100.0, "u_lid": 0.05})
    spec = uniform_spec(prob)
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec, scheme="standard")
    for n in (1, 999):
        o.step(n)
        L.step(n)
        fo, fg = o.fields(), L.moments()
        assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
        assert np.abs(fg[0] - fo[0]).max() <= 1e-6
    L.close()


def test_standard_poiseuille_matches_the_oracle(gpu):
    """Periodic x, walls in y, constant body force (the force of the first
    step's velocity is zero, as in the GOC scheme)."""
    prob = gi.Problem("poiseuille", 16, 40, {"kind": "uniform"}, {"kind": "uniform"}, {"Re": 10.0, "tau": 0.8})
    spec = uniform_spec(prob)
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec, scheme="standard")
    o.step(2000)
    L.step(2000)
    assert relerr(L.moments()[1], o.fields()[1]) <= 1e-5
    L.close()


def test_standard_periodic_vortex_matches_the_oracle(gpu):
    """Doubly periodic Taylor-Green initial field (wrap on both axes, init
    from host fields)."""
    prob = gi.taylor_green(n=40, a=0.0, u0=0.02, tau=0.7)
    spec = uniform_spec(prob)
    o = oracle.Oracle(spec, threads=8)          # initialised from spec["init"]
    L = goc.Lattice(spec, scheme="standard")    # likewise, through goc_init_fields
    o.step(500)
    L.step(500)
    assert relerr(np.stack(L.moments()[1:3]), np.stack(o.fields()[1:3])) <= 1e-5
    L.close()


def test_standard_equals_the_goc_kernel_at_unit_metric(gpu):
    """Both library kernels on the same uniform problem with gi = 0: the
    fused GOC step and the standard step agree to FP32 rounding."""
    prob = gi.Problem("cavity", 48, 40, {"kind": "uniform"}, {"kind": "uniform"}, {"Re": 100.0, "u_lid": 0.05})
    spec = uniform_spec(prob)
    A = goc.Lattice(spec, scheme="standard")
    B = goc.Lattice(spec)
    A.step(1000)
    B.step(1000)
    fa, fb = A.moments(), B.moments()
    assert relerr(np.stack(fa[1:3]), np.stack(fb[1:3])) <= 1e-6
    A.close()
    B.close()


def test_standard_scheme_moves_fewer_bytes(gpu):
    prob = gi.uniform_cavity(n=64)
    spec = uniform_spec(prob)
    A = goc.Lattice(spec, scheme="standard")
    assert A.bytes_per_node == 72.0
    A.close()
