"""Lattices updated in place (goc_exec.streaming = 1: one population buffer,
two alternating access patterns, a fields pass and a collision pass per
step) against the two-buffer step, which the oracle checks, and against the
oracle itself."""
import numpy as np
import pytest

import goc_inputs as gi
import oracle
import paper_2607_15362_b300 as goc

pytestmark = pytest.mark.gpu


def cs2_of(problem):
    return oracle.build_metric(problem.lattice_spec(1.0)).cs2()


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


PROBLEMS = {
    # moving lid (the moving-wall term reads the population sum of the wall nodes), ragged tiles
    "cavity": gi.Problem("cavity", 200, 90, {"kind": "tanh2", "beta": 1.2}, {"kind": "tanh2", "beta": 1.4},
                         {"Re": 100.0, "u_lid": 0.05}),
    # periodic along xi1, body force
    "channel": gi.poiseuille_channel(),
    # the benchmark's grid
    "cavity512": gi.lid_cavity(512),
    # the MIE (Appendix G): periodic along xi1, Hartmann walls with their fields
    "hartmann": gi.Problem("hartmann", 4, 96, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                           {"Ha": 20.0, "Re": 20.0, "tau": 1.0, "tau_m": 1.0}),
}


def _spec(name):
    prob = PROBLEMS[name]
    spec = prob.lattice_spec(cs2_of(prob))
    if name == "cavity_mie":
        spec["mhd"] = {"tau_m": 0.9, "mu_m": 2.0, "B_init": (0.01, 0.004)}
    return spec


# the MIE with walls all round and a moving lid (ragged tiles)
PROBLEMS["cavity_mie"] = PROBLEMS["cavity"]


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_in_place_steps_give_the_two_buffer_populations_bitwise(gpu, name):
    """After 1, 2, 3, 70 (a captured graph and a remainder) and 131 more
    steps the fields of the in-place lattice equal those of the two-buffer
    lattice bitwise, and the mass agrees to rounding of the FP64 sum.  With
    the MIE the wall nodes' updates are separate compilations of the same
    source in the two paths, whose multiply-adds the compiler may fuse
    differently (measured: one node of the lid row one FP32 unit apart in
    B1 of the 200 x 90 cavity); there the fields agree to 1e-6 of their
    largest value."""
    spec = _spec(name)
    mie = "mhd" in spec or PROBLEMS[name].mhd
    A = goc.Lattice(spec)
    B = goc.Lattice(spec, streaming="in_place")
    for n in (1, 1, 1, 70, 131):
        A.step(n)
        B.step(n)
        for x, y in zip(A.moments(), B.moments()):
            if mie:
                assert np.abs(x - y).max() <= 1e-6 * max(np.abs(x).max(), 1e-30)
            else:
                np.testing.assert_array_equal(x, y)
        assert B.mass() == pytest.approx(A.mass(), rel=1e-13)
    assert B.steps_done == A.steps_done == 204
    A.close()
    B.close()


@pytest.mark.parametrize("name", ["cavity", "hartmann"])
def test_in_place_lattice_matches_the_oracle(gpu, name):
    """The ragged cavity with a moving lid and the Hartmann strip with the
    MIE, in place, against the FP64 oracle: velocity (and induced field)
    relative L2 <= 1e-5 after 1000 steps."""
    spec = _spec(name)
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec, streaming="in_place")
    o.step(1000)
    L.step(1000)
    ro, uo, vo, bo1, bo2 = o.fields()
    rg, ug, vg, bg1, bg2 = L.moments()
    assert relerr(np.stack([ug, vg]), np.stack([uo, vo])) <= 1e-5
    assert np.abs(rg - ro).max() <= 1e-6
    if name == "hartmann":
        assert relerr(bg1, bo1) <= 1e-5
    L.close()


def test_in_place_state_round_trip(gpu):
    """A state saved after an odd and after an even number of steps (the two
    layouts) and restored into a new in-place lattice continues bitwise; it
    does not fit a two-buffer lattice."""
    prob = PROBLEMS["cavity"]
    spec = prob.lattice_spec(cs2_of(prob))
    for first in (7, 8):
        A = goc.Lattice(spec, streaming="in_place")
        A.step(first)
        st = A.get_state()
        A.step(25)
        B = goc.Lattice(spec, streaming="in_place")
        B.set_state(st)
        assert B.steps_done == first
        B.step(25)
        for x, y in zip(A.moments(), B.moments()):
            np.testing.assert_array_equal(x, y)
        C = goc.Lattice(spec)
        with pytest.raises(goc.GocError):
            C.set_state(st)
        for L in (A, B, C):
            L.close()


def test_in_place_lattice_holds_less_memory(gpu):
    """56 B of populations, force and fields per node instead of 88 B (FP32),
    34 B instead of 44 B (FP16)."""
    prob = gi.lid_cavity(512)
    spec = prob.lattice_spec(cs2_of(prob))
    A = goc.Lattice(spec)
    B = goc.Lattice(spec, streaming="in_place")
    _, ba = A.footprint()
    _, bb = B.footprint()
    nodes = 512 * 512
    assert bb < 0.67 * ba
    assert 56 * nodes <= bb < 60 * nodes
    assert B.bytes_per_node == pytest.approx(156.0, abs=0.5)
    A.close()
    B.close()
    # 16-bit storage: 18 B of populations, 4 B of force and the 12 B FP32 fields
    A = goc.Lattice(spec, storage="fp16")
    B = goc.Lattice(spec, storage="fp16", streaming="in_place")
    _, ba = A.footprint()
    _, bb = B.footprint()
    assert 34 * nodes <= bb < 0.8 * ba
    assert B.bytes_per_node == pytest.approx(90.0, abs=0.5)
    A.close()
    B.close()


def test_in_place_run_until_matches_the_two_buffer_run(gpu):
    """The residual checks (snapshots written by the collision pass) stop
    both lattices at the same step with the same residual (to the rounding
    of its FP64 sum, whose atomics add in any order)."""
    prob = gi.poiseuille_channel()
    spec = prob.lattice_spec(cs2_of(prob))
    A = goc.Lattice(spec, check_every=50)
    B = goc.Lattice(spec, check_every=50, streaming="in_place")
    ra = A.run_until(1e-6, 4000)
    rb = B.run_until(1e-6, 4000)
    assert ra[0] == rb[0]
    assert rb[1] == pytest.approx(ra[1], rel=1e-12)
    A.close()
    B.close()


def test_in_place_reinitialisation_between_graph_runs(gpu):
    """Steps replayed from a captured graph, a new initial state mid-run (the
    layout starts again from f^0), and more graph steps: the fields still
    equal the two-buffer lattice's bitwise."""
    spec = _spec("cavity")
    rng = np.random.default_rng(5)
    u1 = 0.01 * rng.standard_normal((spec["ny"], spec["nx"]))
    A = goc.Lattice(spec)
    B = goc.Lattice(spec, streaming="in_place")
    for L in (A, B):
        L.step(131)
        L.init_fields(u1=u1)
        L.step(133)
    for x, y in zip(A.moments(), B.moments()):
        np.testing.assert_array_equal(x, y)
    A.close()
    B.close()


@pytest.mark.parametrize("storage, tol", [("fp16", 2e-3), ("bf16", 2e-2)])
@pytest.mark.parametrize("name", ["cavity", "channel"])
def test_in_place_16bit_matches_the_oracle(gpu, name, storage, tol):
    """16-bit storage in place, the per-row storage reference refreshed every
    16 steps in both layouts (its row means read the populations where the
    layout keeps them), against the FP64 oracle after 2000 steps: FP16
    within the stated 2e-3, BF16 within 2e-2 (its 8 significant bits); and
    within the same bound of the two-buffer lattice.  (Not bitwise: the
    two-buffer lattice's interior tiles run the straight-grid kernel, whose
    products fuse differently in the last bit, and stochastic rounding turns
    a last-bit difference into the other rounding of a stored value.)"""
    spec = _spec(name)
    o = oracle.Oracle(spec, threads=8)
    A = goc.Lattice(spec, storage=storage, reference_every=16)
    B = goc.Lattice(spec, storage=storage, reference_every=16, streaming="in_place")
    o.step(2000)
    A.step(2000)
    B.step(2000)
    fo, fa, fb = o.fields(), A.moments(), B.moments()
    assert relerr(np.stack(fb[1:3]), np.stack(fo[1:3])) <= tol
    assert relerr(np.stack(fb[1:3]), np.stack(fa[1:3])) <= tol
    assert np.abs(fb[0] - fo[0]).max() <= tol / 2   # density (about 1)
    A.close()
    B.close()


def test_in_place_16bit_with_the_mie_matches_the_oracle(gpu):
    """The Hartmann strip in FP16 with stochastic rounding, in place, against
    the FP64 oracle after 2000 steps: velocity and induced field within the
    stated 2e-3; and within 1e-3 of the two-buffer FP16 lattice (the wall
    nodes' separate compilations may round a stored value the other way)."""
    spec = _spec("hartmann")
    o = oracle.Oracle(spec, threads=8)
    A = goc.Lattice(spec, storage="fp16")
    B = goc.Lattice(spec, storage="fp16", streaming="in_place")
    o.step(2000)
    A.step(2000)
    B.step(2000)
    fo, fa, fb = o.fields(), A.moments(), B.moments()
    assert relerr(np.stack(fb[1:3]), np.stack(fo[1:3])) <= 2e-3
    assert relerr(fb[3], fo[3]) <= 2e-3
    assert relerr(np.stack(fb[1:3]), np.stack(fa[1:3])) <= 1e-3
    A.close()
    B.close()
