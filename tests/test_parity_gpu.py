"""CUDA path vs the FP64 oracle, element by element, through the C ABI."""
import math
import os

import numpy as np
import pytest

import goc_inputs as gi
import oracle
import paper_2607_15362_b300 as goc

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_pair(spec, steps, storage="fp32", threads=8):
    o = oracle.Oracle(spec, threads=threads)
    L = goc.Lattice(spec, storage=storage)
    o.step(steps)
    L.step(steps)
    return o, L, o.fields(), L.moments()


def cs2_of(problem):
    return oracle.build_metric(problem.lattice_spec(1.0)).cs2()


def test_library_cs_rule_matches_the_oracle(gpu):
    for p in (gi.poiseuille_channel(), gi.lid_cavity(), gi.hartmann_channel()):
        spec = p.lattice_spec(1.0)
        q, cs2 = goc.metric_info(spec)
        m = oracle.build_metric(spec)
        assert q == pytest.approx(m.q(), rel=1e-14)
        assert cs2 == pytest.approx(m.cs2(), rel=1e-14)


def test_poiseuille_channel_fp32_matches_the_oracle(gpu):
    """Poiseuille channel (32 x 64, tanh beta = 1.5, Re = 10): FP32 velocity relative L2
    <= 1e-5 after 1000 and after 2000 steps."""
    p = gi.poiseuille_channel()
    spec = p.lattice_spec(cs2_of(p))
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec)
    for n in (1000, 1000):
        o.step(n)
        L.step(n)
        ro, uo, vo, *_ = o.fields()
        rg, ug, vg, *_ = L.moments()
        assert relerr(np.stack([ug, vg]), np.stack([uo, vo])) <= 1e-5
        assert np.abs(rg - ro).max() <= 1e-6


def test_library_metric_of_every_wall_map_matches_the_oracle(gpu):
    """q and c_s^2 from the library's FP64 metric kernel for the one-wall
    tanh map (Sec. 6.3), the interior-point map (Sec. 6.4) and the Roberts
    map on either axis, against the oracle's numpy metric."""
    maps = [{"kind": "tanh1", "beta": 2.0}, {"kind": "sinh", "mu": 4.0, "yc": 0.3},
            {"kind": "roberts", "gamma": 1.05, "alpha": 0.5}, {"kind": "roberts", "gamma": 1.2, "alpha": 0.0}]
    for m in maps:
        for prob in (gi.Problem("poiseuille", 8, 77, {"kind": "uniform"}, m, {"Re": 10.0, "tau": 0.8}),
                     gi.Problem("cavity", 77, 40, m, {"kind": "tanh2", "beta": 0.5}, {"Re": 10.0, "u_lid": 0.01})):
            spec = prob.lattice_spec(1.0)
            q, cs2 = goc.metric_info(spec)
            mo = oracle.build_metric(spec)
            assert q == pytest.approx(mo.q(), rel=1e-13)
            assert cs2 == pytest.approx(mo.cs2(), rel=1e-13)


@pytest.mark.parametrize("map2", [{"kind": "tanh1", "beta": 1.5}, {"kind": "sinh", "mu": 4.0, "yc": 0.3}])
def test_one_wall_and_interior_maps_fp32_match_the_oracle(gpu, map2):
    """Body-force channel (37 x 70) on the one-wall tanh map and on the
    interior-point map: FP32 velocity relative L2 <= 1e-5 after 1000 steps."""
    prob = gi.Problem("poiseuille", 37, 70, {"kind": "uniform"}, map2, {"Re": 10.0, "tau": 0.8})
    spec = prob.lattice_spec(cs2_of(prob))
    o, L, fo, fg = run_pair(spec, 1000)
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    assert np.abs(fg[0] - fo[0]).max() <= 1e-6


def test_transient_couette_fp32_matches_the_oracle(gpu):
    """Shear-driven channel of Sec. 7.2 on its 6 x 50 grid (Roberts gamma =
    1.06, tau = 1, top wall at U = 0.02, from rest): FP32 velocity relative
    L2 <= 1e-5 against the oracle after 3125 and 15625 steps (t = 0.01 and
    0.05 H^2/nu)."""
    prob = gi.Problem("couette", 6, 50, {"kind": "uniform"}, {"kind": "roberts", "gamma": 1.06, "alpha": 0.5},
                      {"tau": 1.0, "u_wall": 0.02})
    spec = prob.lattice_spec(cs2_of(prob))
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec)
    for n in (3125, 12500):
        o.step(n)
        L.step(n)
        fo, fg = o.fields(), L.moments()
        assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
        assert np.abs(fg[0] - fo[0]).max() <= 1e-6


@pytest.mark.parametrize("nx,ny", [(16, 12), (37, 29), (64, 48)])
def test_cavity_fp32_matches_the_oracle_on_ragged_tiles(gpu, nx, ny):
    """Walls on all sides, moving lid, tanh clustering on both axes; sizes that
    leave ragged tiles in x and y."""
    prob = gi.Problem("cavity", nx, ny, {"kind": "tanh2", "beta": 1.2}, {"kind": "tanh2", "beta": 1.4},
                      {"Re": 100.0, "u_lid": 0.05})
    spec = prob.lattice_spec(cs2_of(prob))
    o, L, fo, fg = run_pair(spec, 1000)
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    assert np.abs(fg[0] - fo[0]).max() <= 1e-6


def test_stretched_periodic_vortex_fp32_matches_the_oracle(gpu):
    """Sine-stretched periodic grid with a random smooth initial field: every
    correction term (Eqs. 82-85) and both geometric forces are active."""
    u1, u2 = gi.random_periodic_fields(40, 24, seed=3, amp=0.03)
    spec = dict(nx=40, ny=24, map1={"kind": "sine", "a": 0.3}, map2={"kind": "sine", "a": -0.25},
                walls={"W": None, "E": None, "S": None, "N": None}, tau=0.7, tau_zeta=0.8,
                fext=(1e-6, -2e-6), init={"u1": u1, "u2": u2})
    o, L, fo, fg = run_pair(spec, 500)
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    assert np.abs(fg[0] - fo[0]).max() <= 1e-6


def test_periodic_node_table_matches_the_per_axis_grid(gpu):
    """The sine-stretched periodic vortex with its metric given node by node
    (both axes periodic: the node-table corrections wrap across both seams)
    against the oracle, and against the same problem on the per-axis maps
    stepped by the library (the same scheme; FP32 rounding apart)."""
    u1, u2 = gi.random_periodic_fields(40, 24, seed=3, amp=0.03)
    spec = dict(nx=40, ny=24, map1={"kind": "sine", "a": 0.3}, map2={"kind": "sine", "a": -0.25},
                walls={"W": None, "E": None, "S": None, "N": None}, tau=0.7, tau_zeta=0.8,
                fext=(1e-6, -2e-6), init={"u1": u1, "u2": u2})
    m = oracle.build_metric(spec)
    one = np.ones(1)
    tab = dict(spec, map1={"kind": "table"}, map2={"kind": "uniform"},
               metric={"h1": m.h1, "h2": m.h2, "t11": m.t11, "t12": m.t12, "t21": m.t21, "t22": m.t22,
                       "wall": {w: (one.repeat(24 if w in "WE" else 40), one.repeat(24 if w in "WE" else 40))
                                for w in "WESN"}})
    o, L, fo, fg = run_pair(tab, 500)
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    assert np.abs(fg[0] - fo[0]).max() <= 1e-6
    L2 = goc.Lattice(spec)
    L2.step(500)
    fa = L2.moments()
    assert relerr(np.stack(fg[1:3]), np.stack(fa[1:3])) <= 1e-5
    L.close()
    L2.close()


def test_hartmann_strip_fp32_matches_the_oracle(gpu):
    """Coupled NSE + MIE (Appendix G) on a wall-normal tanh grid: FP32 velocity
    and induced field within 1e-5 relative L2 after 1000 and 3000 steps (the
    field does not drift: measured 6.8e-7 and 7.1e-7)."""
    prob = gi.Problem("hartmann", 4, 96, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                      {"Ha": 20.0, "Re": 20.0, "tau": 1.0, "tau_m": 1.0})
    spec = prob.lattice_spec(cs2_of(prob))
    B0 = spec["derived"]["B0"]
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec)
    for n, tol_b in ((1000, 1e-5), (3000, 1e-5)):
        o.step(n - o.steps_done)
        L.step(n - L.steps_done)
        fo, fg = o.fields(), L.moments()
        assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
        assert relerr(fg[3], fo[3]) <= tol_b
        assert np.abs(fg[4] - fo[4]).max() <= 1e-6 * B0


def test_mass_is_conserved_on_the_gpu(gpu):
    prob = gi.Problem("cavity", 48, 40, {"kind": "tanh2", "beta": 1.5}, {"kind": "tanh2", "beta": 1.5},
                      {"Re": 200.0, "u_lid": 0.05})
    spec = prob.lattice_spec(cs2_of(prob))
    L = goc.Lattice(spec)
    m0 = L.mass()
    L.step(2000)
    assert abs(L.mass() - m0) / m0 < 1e-6


@pytest.mark.parametrize("case", ["channel", "annulus_mhd", "spiral_fp16"])
def test_checkpoint_restore_is_bitwise(gpu, case):
    """Save after 150 steps, restore into a fresh lattice, run 130 more: the
    fields equal those of the uninterrupted run bit for bit (straight grid;
    annulus with the MIE; node table with FP16 storage and its stochastic
    rounding stream)."""
    storage = "fp16" if case == "spiral_fp16" else "fp32"
    if case == "channel":
        p = gi.poiseuille_channel()
        spec = p.lattice_spec(cs2_of(p))
    elif case == "annulus_mhd":
        p = gi.taylor_couette(n1=45, n2=11, r_in=6.0, sectors=9.0, Re=20.0, u_in=1.0, u_out=1.5)
        spec = p.lattice_spec(cs2_of(p))
        spec["walls"]["W"] = dict(spec["walls"]["W"], B=(0.02, 0.005))
        spec["mhd"] = {"tau_m": 0.9, "mu_m": 2.0, "B_init": (0.01, 0.004)}
    else:
        p = gi.spiral_cavity(40, 37)
        spec = p.lattice_spec(cs2_of(p))
    a = goc.Lattice(spec, storage=storage)
    a.step(150)
    st = a.get_state()
    a.step(130)
    b = goc.Lattice(spec, storage=storage)
    b.set_state(st)
    b.step(130)
    for x, y in zip(a.moments(), b.moments()):
        np.testing.assert_array_equal(x, y)
    assert b.steps_done == 280
    a.close()
    b.close()


def _mixed_specs():
    out = []
    for prob in (gi.poiseuille_channel(),
                 gi.Problem("cavity", 37, 29, {"kind": "tanh2", "beta": 1.2}, {"kind": "tanh2", "beta": 1.4},
                            {"Re": 100.0, "u_lid": 0.05}),
                 gi.Problem("hartmann", 4, 96, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                            {"Ha": 20.0, "Re": 20.0, "tau": 1.0, "tau_m": 1.0})):
        out.append(prob.lattice_spec(cs2_of(prob)))
    return out


def test_batched_lattices_match_individual_runs_bitwise(gpu):
    """One persistent launch per step over uneven lattices (NSE and NSE+MIE
    mixed) gives bitwise the same FP32 result as each lattice alone."""
    specs = _mixed_specs()
    batch = goc.Batch(hbm_budget_bytes=1 << 30, max_lattices=8)
    slots = [batch.add(s) for s in specs]
    batch.step(1)
    batch.step(150)      # graph part (32-step graphs) plus remainder, odd phase start
    batch.step(49)
    for spec, slot in zip(specs, slots):
        alone = goc.Lattice(spec)
        alone.step(200)
        for x, y in zip(batch.lattice(slot).moments(), alone.moments()):
            np.testing.assert_array_equal(x, y)
    # a late admission joins the running batch and still matches its own run
    late = batch.add(specs[1])
    batch.step(70)
    alone = goc.Lattice(specs[1])
    alone.step(70)
    for x, y in zip(batch.lattice(late).moments(), alone.moments()):
        np.testing.assert_array_equal(x, y)
    used, budget, count = batch.usage()
    assert count == 4 and 0 < used <= budget
    batch.close()


def test_batch_admission_respects_the_hbm_budget(gpu):
    specs = _mixed_specs()
    batch = goc.Batch(hbm_budget_bytes=200_000, max_lattices=8)
    assert batch.try_add(specs[0]) is not None      # 32 x 64 fits
    assert batch.try_add(gi.lid_cavity().lattice_spec(0.007)) is None   # 512^2 does not
    batch.close()


def test_run_until_reaches_the_residual_and_reports_it(gpu):
    prob = gi.Problem("poiseuille", 2, 24, {"kind": "uniform"}, {"kind": "tanh2", "beta": 1.0},
                      {"Re": 5.0, "tau": 1.0})
    spec = prob.lattice_spec(cs2_of(prob))
    L = goc.Lattice(spec, check_every=200)
    done, res = L.run_until(1e-7, 400000)
    assert res < 1e-7 and 0 < done < 400000
    assert L.residuals()[0] == pytest.approx(res)


@pytest.mark.parametrize("kind", ["cavity", "channel", "hartmann"])
def test_interior_tiles_match_the_oracle(gpu, kind):
    """Lattices wide enough to contain interior tiles (the check-free path) as
    well as wall tiles and periodic-wrap tiles."""
    if kind == "cavity":
        prob = gi.Problem("cavity", 130, 90, {"kind": "tanh2", "beta": 1.5}, {"kind": "tanh2", "beta": 1.3},
                          {"Re": 300.0, "u_lid": 0.05})
        steps = 600
    elif kind == "channel":
        prob = gi.Problem("poiseuille", 100, 72, {"kind": "uniform"}, {"kind": "tanh2", "beta": 1.8},
                          {"Re": 10.0, "tau": 0.8})
        steps = 600
    else:
        prob = gi.Problem("hartmann", 100, 64, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                          {"Ha": 15.0, "Re": 15.0, "tau": 1.0, "tau_m": 1.0})
        steps = 600
    spec = prob.lattice_spec(cs2_of(prob))
    if kind == "channel":   # add a transverse perturbation so that every term is exercised
        u1, u2 = gi.random_periodic_fields(prob.nx, prob.ny, seed=8, amp=0.002)
        spec["init"] = {"u1": u1, "u2": u2}
    o, L, fo, fg = run_pair(spec, steps)
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    assert np.abs(fg[0] - fo[0]).max() <= 1e-6
    if prob.mhd:
        assert relerr(fg[3], fo[3]) <= 1e-5


@pytest.mark.parametrize("kind,storage", [("channel", "fp32"), ("channel", "fp16"), ("hartmann", "fp32")])
def test_tiles_across_the_periodic_seam_match_the_oracle(gpu, kind, storage):
    """Lattices whose width is a multiple of the tile width, periodic along
    xi1: the tiles whose staged box crosses the seam are staged like interior
    tiles and get the columns beyond the seam copied from the other side (the
    straight-grid kernel's seam path), with the MIE pulls wrapping.  A channel
    64 x 72 (every tile column at the seam; FP32 with a transverse
    perturbation, 600 steps; FP16 from rest, 2000 steps as the FP16
    Poiseuille test) and a Hartmann strip 96 x 64 (600 steps); velocity (and
    field) relative L2 <= 1e-5 (FP16 storage: 2e-3)."""
    steps = 600
    if kind == "channel":
        prob = gi.Problem("poiseuille", 64, 72, {"kind": "uniform"}, {"kind": "tanh2", "beta": 1.8},
                          {"Re": 10.0, "tau": 0.8})
    else:
        prob = gi.Problem("hartmann", 96, 64, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                          {"Ha": 15.0, "Re": 15.0, "tau": 1.0, "tau_m": 1.0})
    spec = prob.lattice_spec(cs2_of(prob))
    if kind == "channel" and storage == "fp32":
        u1, u2 = gi.random_periodic_fields(prob.nx, prob.ny, seed=9, amp=0.002)
        spec["init"] = {"u1": u1, "u2": u2}
    if storage == "fp16":
        steps = 2000
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec, storage=storage)
    o.step(steps)
    L.step(steps)
    fo, fg = o.fields(), L.moments()
    tol = 1e-5 if storage == "fp32" else 2e-3
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= tol
    if prob.mhd:
        assert relerr(fg[3], fo[3]) <= tol
    L.close()


def test_launch_configurations_give_bitwise_identical_populations(gpu):
    """Tile queue vs static tile order, dependent launch on or off, the
    balanced grid and the tile height (32 x 8 or 32 x 16 nodes) change only
    which block computes which node and when: the populations agree bitwise
    (on a cavity with interior, wall and ragged tiles, and on a periodic
    channel with the MIE whose seam tiles read global memory)."""
    for prob in (gi.Problem("cavity", 200, 90, {"kind": "tanh2", "beta": 1.2}, {"kind": "tanh2", "beta": 1.4},
                            {"Re": 100.0, "u_lid": 0.05}),
                 gi.Problem("hartmann", 70, 96, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                            {"Ha": 20.0, "Re": 20.0, "tau": 1.0, "tau_m": 1.0})):
        spec = prob.lattice_spec(cs2_of(prob))
        states = []
        for dyn, pdl, bal, rows in ((True, True, False, 8), (False, True, False, 8), (True, False, False, 8),
                                    (False, False, False, 8), (True, True, True, 8), (False, True, True, 8),
                                    (True, True, False, 16), (False, True, True, 16), (True, False, False, 16)):
            L = goc.Lattice(spec)
            L.set_launch_config(dyn, pdl, bal, tile_rows=rows)
            L.step(150)
            assert L.launch_config == {"dynamic_tiles": dyn, "pdl": pdl, "balanced_grid": bal, "tile_rows": rows,
                                       "tuned": True}
            states.append(L.get_state())
            L.close()
        assert all(s == states[0] for s in states[1:])
        A = goc.Lattice(spec)            # autotuned on its first long call
        A.step(150)
        assert A.launch_config["tuned"]
        assert A.get_state() == states[0]
        A.close()


def test_tile_queues_survive_changes_of_launch_configuration(gpu):
    """The tile queues of the two buffer parities stay consistent when the
    tile order or the tile height changes between steps, each setting for an
    odd number of steps: the populations equal those of one configuration
    throughout, bitwise."""
    prob = gi.Problem("cavity", 200, 90, {"kind": "tanh2", "beta": 1.2}, {"kind": "tanh2", "beta": 1.4},
                      {"Re": 100.0, "u_lid": 0.05})
    spec = prob.lattice_spec(cs2_of(prob))
    ref = goc.Lattice(spec)
    ref.set_launch_config(True, True)
    ref.step(1 + 7 + 5 + 3 + 9 + 7 + 11)
    want = ref.get_state()
    ref.close()
    L = goc.Lattice(spec)
    L.step(1)
    for dyn, rows, n in ((True, 8, 7), (False, 8, 5), (True, 16, 3), (False, 16, 9), (True, 8, 7), (False, 8, 11)):
        L.set_launch_config(dyn, True, tile_rows=rows)
        L.step(n)
    assert L.get_state() == want
    L.close()


def test_tall_tiles_are_for_straight_grids_only(gpu):
    """The 32 x 16 tiles run the straight-grid central-moment kernel; a curved
    grid reports 8-row tiles and refuses 16."""
    prob = gi.taylor_couette(n1=45, n2=11, r_in=6.0, sectors=9.0, Re=20.0, u_in=1.0, u_out=1.5)
    L = goc.Lattice(prob.lattice_spec(cs2_of(prob)))
    assert L.launch_config["tile_rows"] == 8
    with pytest.raises(goc.GocError) as e:
        L.set_launch_config(True, True, False, tile_rows=16)
    assert "straight grids" in str(e.value)
    L.close()


# ---- collisions on raw moments: SRT of Appendix F (goc_exec.scheme = 2) and
# raw-moment MRT of Appendix D (scheme 3) --------------------------------------
def _srt_pair(prob, steps_list, collision="srt"):
    spec = prob.lattice_spec(cs2_of(prob))
    spec["collision"] = collision
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec, scheme={"srt": "goc_srt", "raw": "goc_raw"}[collision])
    out = []
    for n in steps_list:
        o.step(n)
        L.step(n)
        out.append((o.fields(), L.moments()))
    L.close()
    return out


@pytest.mark.parametrize("collision", ["srt", "raw"])
@pytest.mark.parametrize("name", ["poiseuille_roberts", "couette", "cavity", "hartmann"])
def test_srt_fp32_matches_the_oracle(gpu, name, collision):
    """The SRT GOC-LBM (Appendix F) and the raw-moment MRT (Appendix D) in the
    library against the oracle's:
    body-force channel on the paper's Roberts grid (gamma = 1.06, tau = 1),
    the shear-driven channel of Sec. 7.2 (6 x 50), a cavity with ragged tiles,
    and a Hartmann strip with the MIE; FP32 velocity (and induced field)
    relative L2 <= 1e-5."""
    probs = {
        "poiseuille_roberts": gi.Problem("poiseuille", 8, 48, {"kind": "uniform"},
                                         {"kind": "roberts", "gamma": 1.06, "alpha": 0.5}, {"Re": 20.0, "tau": 1.0}),
        "couette": gi.Problem("couette", 6, 50, {"kind": "uniform"}, {"kind": "roberts", "gamma": 1.06, "alpha": 0.5},
                              {"tau": 1.0, "u_wall": 0.02}),
        "cavity": gi.Problem("cavity", 37, 29, {"kind": "tanh2", "beta": 1.2}, {"kind": "tanh2", "beta": 1.4},
                             {"Re": 30.0, "u_lid": 0.05}),   # tau = 1.84 (at Re = 10, tau = 4.5, the raw MRT diverges)
        "hartmann": gi.Problem("hartmann", 4, 96, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                               {"Ha": 20.0, "Re": 20.0, "tau": 1.0, "tau_m": 1.0}),
    }
    for fo, fg in _srt_pair(probs[name], (1000, 1000), collision):
        assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
        assert np.abs(fg[0] - fo[0]).max() <= 1e-6
        if name == "hartmann":
            assert relerr(fg[3], fo[3]) <= 1e-5


@pytest.mark.parametrize("collision", ["srt", "raw"])
@pytest.mark.parametrize("name", ["annulus", "spiral", "annulus_mhd"])
def test_raw_moment_collisions_on_curved_grids_match_the_oracle(gpu, name, collision):
    """The SRT (Appendix F) and raw-moment MRT (Appendix D) collisions on the
    curved grids: Taylor-Couette flow in the annular sector (45 x 11, ragged
    tiles; and with the MIE), and the spiral cavity given as a node table
    (every theta_ij non-zero).  FP32 velocity and field relative L2 <= 1e-5
    after 500 and 1500 steps."""
    if name == "spiral":
        prob = gi.spiral_cavity(40, 37, phi=0.6)
    else:
        prob = gi.taylor_couette(n1=45, n2=11, r_in=6.0, sectors=9.0, Re=20.0, u_in=1.0, u_out=1.5)
    spec = prob.lattice_spec(cs2_of(prob))
    if name == "annulus_mhd":
        spec["walls"]["W"] = dict(spec["walls"]["W"], B=(0.02, 0.005))
        spec["walls"]["E"] = dict(spec["walls"]["E"], B=(0.01, -0.004))
        spec["mhd"] = {"tau_m": 0.9, "mu_m": 2.0, "B_init": (0.01, 0.004)}
    spec["collision"] = collision
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec, scheme={"srt": "goc_srt", "raw": "goc_raw"}[collision])
    for n in (500, 1000):
        o.step(n)
        L.step(n)
        fo, fg = o.fields(), L.moments()
        assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5, (name, n)
        assert np.abs(fg[0] - fo[0]).max() <= 1e-6
        if "mhd" in spec:
            assert relerr(np.stack(fg[3:5]), np.stack(fo[3:5])) <= 1e-5
    L.close()


# ---- curvilinear grid: annular sector of Sec. 8 (goc_map kind ANNULUS) --------
@pytest.mark.parametrize("n1,n2,r_in,sectors,storage", [(256, 6, 32.0, 60.0, "fp32"), (45, 11, 6.0, 9.0, "fp32"),
                                                       (40, 6, 5.0, 10.0, "fp16")])
def test_taylor_couette_on_the_annulus_matches_the_oracle(gpu, n1, n2, r_in, sectors, storage):
    """Taylor-Couette flow in an annular sector (inner wall U0, outer 1.5 U0,
    from rest): the paper's 256 x 6 grid with 60 sectors and inner radius 32,
    and ragged tiles on both axes.  FP32 velocity relative L2 <= 1e-5 after
    500 and 1500 steps (FP16 storage: 2e-3)."""
    prob = gi.taylor_couette(n1=n1, n2=n2, r_in=r_in, sectors=sectors, Re=20.0, u_in=1.0, u_out=1.5)
    spec = prob.lattice_spec(cs2_of(prob))
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec, storage=storage)
    tol = 1e-5 if storage == "fp32" else 2e-3
    for n in (500, 1000):
        o.step(n)
        L.step(n)
        fo, fg = o.fields(), L.moments()
        assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= tol
        assert np.abs(fg[0] - fo[0]).max() <= (1e-6 if storage == "fp32" else 1e-3)
    L.close()


def test_taylor_couette_on_the_annulus_reaches_the_analytic_profile(gpu):
    """The library alone on the paper's grid (256 x 6, 60 sectors, R1 = 32,
    R2 = 288), started from the analytic u_theta(r) of Sec. 8.2 and run for
    two viscous times: it stays on the analytic profile (relative L2 below
    1e-3; 2e-3 is the oracle's error on this grid at tau ~ 2.3) and mass is
    conserved."""
    prob = gi.taylor_couette(n1=256, n2=6, r_in=32.0, sectors=60.0, Re=20.0, u_in=1.0, u_out=1.5)
    m = oracle.build_metric(prob.lattice_spec(1.0))
    spec = prob.lattice_spec(m.cs2())
    ua = gi.taylor_couette_profile(m.radius, 32.0, 288.0, 0.01, 0.015)
    spec["init"] = {"u1": 0.0, "u2": np.broadcast_to(ua[None, :], (6, 256)).copy()}
    L = goc.Lattice(spec)
    mass0 = L.mass()
    L.step(int(2.0 * 256 ** 2 / spec["nu"]))
    rho, u1, u2, *_ = L.moments()
    assert relerr(u2[0], ua) < 1e-3
    assert np.abs(u1).max() < 1e-3 * ua.max()
    assert abs(L.mass() - mass0) / mass0 < 1e-5
    L.close()


# ---- general orthogonal grid given node by node (goc_map kind TABLE) ----------
def _table_of(m):
    return {"h1": m.h1, "h2": m.h2, "t11": m.t11, "t12": m.t12, "t21": m.t21, "t22": m.t22, "wall": m.wall}


def _transposed_table_of(m):
    """The metric of the same grid with xi1 and xi2 exchanged."""
    return {"h1": m.h2.T, "h2": m.h1.T, "t11": m.t22.T, "t12": m.t21.T, "t21": m.t12.T, "t22": m.t11.T,
            "wall": {"W": (m.wall["S"][1], m.wall["S"][0]), "E": (m.wall["N"][1], m.wall["N"][0]),
                     "S": (m.wall["W"][1], m.wall["W"][0]), "N": (m.wall["E"][1], m.wall["E"][0])}}


@pytest.mark.parametrize("case,storage", [("annulus", "fp32"), ("transposed", "fp32"), ("spiral", "fp32"),
                                          ("spiral", "fp16"), ("spiral", "bf16")])
def test_node_table_metric_matches_the_oracle(gpu, case, storage):
    """The node-table step kernel (h1, h2, theta_ij and the link corrections
    read per node) against the oracle: the annular sector of Sec. 8 given as a
    table (45 x 11, ragged tiles, moving W/E walls), the same sector with the
    radial direction along xi2 (theta12, theta22 in place of theta21,
    theta11; moving S/N walls) and the lid-driven cavity on the
    logarithmic-spiral grid (40 x 37, every theta_ij non-zero).  Velocity
    relative L2 <= 1e-5 (FP16 storage: 2e-3; BF16, 8 significant bits: 2e-2)
    after 500 and 1500 steps."""
    if case == "spiral":
        prob = gi.spiral_cavity(40, 37, phi=0.6)
        m = oracle.build_metric(prob.lattice_spec(1.0))
        spec_o = spec_g = prob.lattice_spec(m.cs2())
        transpose = False
    else:
        prob = gi.taylor_couette(n1=45, n2=11, r_in=6.0, sectors=9.0, Re=20.0, u_in=1.0, u_out=1.5)
        m = oracle.build_metric(prob.lattice_spec(1.0))
        spec_o = prob.lattice_spec(m.cs2())
        spec_g = dict(spec_o, map1={"kind": "table"}, map2={"kind": "uniform"})
        transpose = case == "transposed"
        if transpose:
            w = spec_o["walls"]
            spec_g.update(nx=spec_o["ny"], ny=spec_o["nx"], metric=_transposed_table_of(m),
                          walls={"S": w["W"], "N": w["E"], "W": None, "E": None})
            spec_o = spec_g   # the oracle runs the table too
        else:
            spec_g["metric"] = _table_of(m)
    q, cs2 = goc.metric_info(spec_g)
    assert cs2 == pytest.approx(m.cs2(), rel=1e-14)
    o = oracle.Oracle(spec_o, threads=8)
    L = goc.Lattice(spec_g, storage=storage)
    tol = {"fp32": 1e-5, "fp16": 2e-3, "bf16": 2e-2}[storage]
    for n in (500, 1000):
        o.step(n)
        L.step(n)
        fo, fg = o.fields(), L.moments()
        assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= tol, (case, n)
        assert np.abs(fg[0] - fo[0]).max() <= {"fp32": 1e-6, "fp16": 1e-3, "bf16": 1e-2}[storage]
    if storage == "fp32":
        mo = (fo[0] * m.h1 * m.h2).sum() if not transpose else (fo[0] * m.h1.T * m.h2.T).sum()
        assert L.mass() == pytest.approx(mo, rel=1e-6)
    L.close()


@pytest.mark.parametrize("case,storage", [("annulus", "fp32"), ("transposed", "fp32"), ("spiral", "fp32"),
                                          ("annulus", "fp16")])
def test_mie_on_curvilinear_grids_matches_the_oracle(gpu, case, storage):
    """The MIE of Appendix G on curvilinear grids (the gradient formula,
    g^corr and J3 with theta21 / theta12, the source Y of Eq. 6ab_C and the
    2 x 2 solve for B) coupled to the flow (mu_m = 2): the annular sector
    (45 x 11, ragged tiles, rotating walls imposing both field components,
    an initial uniform field), the same sector transposed into a node table,
    and the spiral cavity with every theta_ij non-zero.  Velocity and field
    relative L2 <= 1e-5 (FP16 storage: 2e-3) after 500 and 1500 steps
    (measured: at most 1.8e-6 and 4.6e-6 in FP32, 1.1e-3 in FP16)."""
    mhd = {"tau_m": 0.9, "mu_m": 2.0, "B_init": (0.01, 0.004)}
    if case == "spiral":
        prob = gi.spiral_cavity(40, 37, phi=0.6)
        m = oracle.build_metric(prob.lattice_spec(1.0))
        spec_o = prob.lattice_spec(m.cs2())
        for w, bw in zip("WESN", ((0.02, 0.0), (0.01, 0.005), (0.0, 0.015), (-0.005, 0.01))):
            spec_o["walls"][w] = dict(spec_o["walls"][w], B=bw)
        spec_o["mhd"] = mhd
        spec_g = spec_o
    else:
        prob = gi.taylor_couette(n1=45, n2=11, r_in=6.0, sectors=9.0, Re=20.0, u_in=1.0, u_out=1.5)
        m = oracle.build_metric(prob.lattice_spec(1.0))
        spec_o = prob.lattice_spec(m.cs2())
        spec_o["walls"]["W"] = dict(spec_o["walls"]["W"], B=(0.02, 0.005))
        spec_o["walls"]["E"] = dict(spec_o["walls"]["E"], B=(0.01, -0.004))
        spec_o["mhd"] = mhd
        spec_g = spec_o
        if case == "transposed":
            w = spec_o["walls"]
            spec_g = dict(spec_o, nx=spec_o["ny"], ny=spec_o["nx"], map1={"kind": "table"}, map2={"kind": "uniform"},
                          metric=_transposed_table_of(m), mhd=dict(mhd, B_init=(0.004, 0.01)),
                          walls={"S": dict(w["W"], B=(0.005, 0.02)), "N": dict(w["E"], B=(-0.004, 0.01)),
                                 "W": None, "E": None})
            spec_o = spec_g
    o = oracle.Oracle(spec_o, threads=8)
    L = goc.Lattice(spec_g, storage=storage)
    tol = 1e-5 if storage == "fp32" else 2e-3
    for n in (500, 1000):
        o.step(n)
        L.step(n)
        fo, fg = o.fields(), L.moments()
        assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= tol, (case, n)
        assert relerr(np.stack(fg[3:5]), np.stack(fo[3:5])) <= tol, (case, n)
    L.close()


def test_cartesian_components_on_the_annulus(gpu):
    """goc_moments(cartesian=1) on the annular sector (Eq. vectormapping)
    against the oracle's radial and azimuthal components rotated by the
    azimuth of each node position of the map (Sec. 8.1); a node table, which
    carries no coordinates, refuses."""
    from oracle.metric import annulus_position
    prob = gi.taylor_couette(n1=45, n2=11, r_in=6.0, sectors=9.0, Re=20.0, u_in=1.0, u_out=1.5)
    m = oracle.build_metric(prob.lattice_spec(1.0))
    spec = prob.lattice_spec(m.cs2())
    spec["walls"]["W"] = dict(spec["walls"]["W"], B=(0.02, 0.005))
    spec["mhd"] = {"tau_m": 0.9, "mu_m": 2.0, "B_init": (0.01, 0.004)}
    o = oracle.Oracle(spec, threads=8)
    L = goc.Lattice(spec)
    o.step(300)
    L.step(300)
    x, y = annulus_position(np.arange(45)[None, :] + 0.5, np.arange(11)[:, None], 45, 11, 6.0, 51.0, 9.0)
    phi = np.arctan2(y, x)
    c, s_ = np.cos(phi), np.sin(phi)
    rho, ur, up, br, bp = o.fields()
    want = [c * ur - s_ * up, s_ * ur + c * up, c * br - s_ * bp, s_ * br + c * bp]
    got = L.moments(cartesian=True)
    assert relerr(np.stack(got[1:3]), np.stack(want[:2])) <= 1e-5
    assert relerr(np.stack(got[3:5]), np.stack(want[2:])) <= 1e-4
    L.close()
    t = dict(spec, map1={"kind": "table"}, map2={"kind": "uniform"},
             metric={"h1": m.h1, "h2": m.h2, "t11": m.t11, "t12": m.t12, "t21": m.t21, "t22": m.t22, "wall": m.wall})
    L = goc.Lattice(t)
    with pytest.raises(Exception, match="no coordinates"):
        L.moments(cartesian=True)
    L.close()


def test_degenerate_single_column_and_zero_steps(gpu):
    """A channel one node wide (every x pull wraps to the node itself) matches
    the oracle; goc_step(0) changes nothing; a negative count is refused."""
    prob = gi.Problem("poiseuille", 1, 40, {"kind": "uniform"}, {"kind": "roberts", "gamma": 1.06, "alpha": 0.5},
                      {"Re": 20.0, "tau": 0.8})
    spec = prob.lattice_spec(cs2_of(prob))
    o, L, fo, fg = run_pair(spec, 3000)
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    before = L.get_state()
    L.step(0)
    assert L.get_state() == before
    with pytest.raises(goc.GocError):
        L.step(-1)
    L.close()


# ---- full-size workloads in the launch configuration the benchmark times -------
def test_full_size_cavity_in_the_benchmark_configuration_matches_the_oracle(gpu):
    """The 512 x 512 clustered cavity of the benchmark, stepped as bench.py
    steps it (autotuned launch configuration, captured graph chunks), against
    the oracle on the whole lattice after 300 steps: FP32 velocity relative
    L2 <= 1e-5."""
    prob = gi.lid_cavity()
    spec = prob.lattice_spec(cs2_of(prob))
    o = oracle.Oracle(spec, threads=os.cpu_count() or 1)
    L = goc.Lattice(spec)
    L.step(300)
    assert L.launch_config["tuned"]
    o.step(300)
    fo, fg = o.fields(), L.moments()
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    assert np.abs(fg[0] - fo[0]).max() <= 1e-6
    L.close()


def test_full_size_spiral_cavity_in_the_benchmark_configuration_matches_the_oracle(gpu):
    """The 512 x 512 cavity on the logarithmic-spiral node table, as
    `bench.py --grid spiral` steps it (autotuned launch, graph chunks),
    against the oracle on the whole lattice after 300 steps: FP32 velocity
    relative L2 <= 1e-5."""
    prob = gi.spiral_cavity(512, 512, Re=1000.0, u_lid=0.05, mach_matched=True)
    spec = prob.lattice_spec(cs2_of(prob))
    o = oracle.Oracle(spec, threads=os.cpu_count() or 1)
    L = goc.Lattice(spec)
    L.step(300)
    assert L.launch_config["tuned"]
    o.step(300)
    fo, fg = o.fields(), L.moments()
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    assert np.abs(fg[0] - fo[0]).max() <= 1e-6
    L.close()


def test_full_size_hartmann_channel_matches_the_oracle(gpu):
    """The 256 x 1024 Hartmann channel (tanh beta = 3, Ha = 100) with the MIE,
    started from the analytic u_x, B_x of Sec. 7.4 (from rest the flow is
    still near the FP32 floor after any affordable number of steps: the
    time step is tied to the smallest cell), 200 steps, against the oracle
    on the whole lattice: velocity and induced field relative L2 <= 1e-5, B2
    within 1e-6 B0."""
    from oracle.metric import map_position
    prob = gi.hartmann_channel()
    spec = prob.lattice_spec(cs2_of(prob))
    d = spec["derived"]
    Ha, H, B0 = 100.0, d["H"], d["B0"]
    ys = map_position("tanh2", prob.ny, np.arange(prob.ny) + 0.5, beta=3.0) / H - 1.0
    Ur, Br = H * H * d["Fx"] / d["nu"], H * H * d["Fx"] / math.sqrt(d["nu"] * d["eta"])
    ua = Ur / (Ha * math.tanh(Ha)) * (1 - np.cosh(Ha * ys) / math.cosh(Ha))
    ba = Br * (-ys / Ha + np.sinh(Ha * ys) / (Ha * math.tanh(Ha) * math.cosh(Ha)))
    u1 = np.repeat(ua[:, None], prob.nx, axis=1)
    b1 = np.repeat(ba[:, None], prob.nx, axis=1)
    o = oracle.Oracle(spec, threads=os.cpu_count() or 1)
    o.initialize(u1=u1, b1=b1)
    L = goc.Lattice(spec)
    L.init_fields(u1=u1, b1=b1)
    L.step(200)
    o.step(200)
    fo, fg = o.fields(), L.moments()
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    eb = relerr(fg[3], fo[3])
    assert eb <= 1e-5, (eb, np.abs(fg[3] - fo[3]).max() / B0, np.abs(ba).max() / B0)
    assert np.abs(fg[4] - fo[4]).max() <= 1e-6 * B0
    L.close()


def test_full_size_batch_matches_individual_lattices_on_a_sample(gpu):
    """The 64-lattice batch of seed 7 (19.8 M nodes) stepped together for 40
    steps gives bitwise the fields of each lattice stepped alone, checked
    on 6 lattices spread over the size range (both kinds, with and without
    the MIE)."""
    probs = gi.batch_lattices()
    specs = [p.lattice_spec(cs2_of(p)) for p in probs]
    batch = goc.Batch(hbm_budget_bytes=8 << 30, max_lattices=64)
    slots = [batch.add(s) for s in specs]
    batch.step(40)
    order = sorted(range(len(probs)), key=lambda k: probs[k].nodes)
    for k in [order[0], order[12], order[25], order[38], order[51], order[-1]]:
        alone = goc.Lattice(specs[k])
        alone.step(40)
        for x, y in zip(batch.lattice(slots[k]).moments(), alone.moments()):
            np.testing.assert_array_equal(x, y)
        alone.close()
    batch.close()


def test_divergence_is_reported_and_cleared_by_reinitialisation(gpu):
    """A lattice driven far past its stability limit (Mach 0.87 lid, tau =
    0.50007: NaN within 50 steps in the oracle) raises GOC_EDIVERGED from the
    next synchronising call, from later goc_step calls (sticky), and from
    goc_moments (which still fills the arrays); re-initialising clears it."""
    from paper_2607_15362_b300 import _abi
    p = gi.Problem("cavity", 48, 48, {"kind": "uniform"}, {"kind": "uniform"}, {"Re": 1e6, "u_lid": 0.5})
    L = goc.Lattice(p.lattice_spec(1.0 / 3.0))
    L.step(400)
    with pytest.raises(goc.GocError) as e:
        L.sync()
    assert e.value.status == _abi.GOC_EDIVERGED and "diverged" in str(e.value)
    with pytest.raises(goc.GocError) as e:
        L.step(10)
    assert e.value.status == _abi.GOC_EDIVERGED
    with pytest.raises(goc.GocError):
        L.moments()
    L.init_fields()
    L.step(5)
    L.sync()
    rho = L.moments()[0]
    assert np.isfinite(rho).all()
    L.close()


def test_bounded_device_wait_times_out_and_leaves_the_device_usable(gpu):
    """The failure-detection self-test: a wait on a device barrier that
    nothing completes gives up after its poll budget and reports
    GOC_ETIMEOUT (the bounded-wait status of the step kernels); a lattice
    then steps normally on the same device."""
    from paper_2607_15362_b300 import _abi
    lib = goc.lib()
    assert lib.goc_selftest_bounded_wait(0) == _abi.GOC_EINVAL
    assert lib.goc_selftest_bounded_wait(1 << 16) == _abi.GOC_ETIMEOUT
    assert b"ran out" in lib.goc_last_error()
    prob = gi.poiseuille_channel()
    o, L, fo, fg = run_pair(prob.lattice_spec(cs2_of(prob)), 200)
    L.sync()
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    L.close()


@pytest.mark.parametrize("case", ["cavity", "hartmann_fp16", "annulus_mhd", "spiral"])
def test_no_stray_writes_into_guard_bands(gpu, case, monkeypatch):
    """With GOC_GUARD_BANDS set, the padding columns of every plane and a
    64 KB tail after every population, force and MIE buffer hold a canary;
    after stepping (ragged tiles, periodic seams, walls, the MIE, 16-bit
    storage, node tables) and re-initialising, no guard byte has changed."""
    import ctypes
    from paper_2607_15362_b300 import _abi
    monkeypatch.setenv("GOC_GUARD_BANDS", "1")
    storage = "fp16" if case.endswith("fp16") else "fp32"
    if case == "cavity":
        prob = gi.Problem("cavity", 100, 90, {"kind": "tanh2", "beta": 1.2}, {"kind": "tanh2", "beta": 1.4},
                          {"Re": 30.0, "u_lid": 0.05})
        spec = prob.lattice_spec(cs2_of(prob))
    elif case == "hartmann_fp16":
        prob = gi.Problem("hartmann", 4, 48, {"kind": "uniform"}, {"kind": "tanh2", "beta": 1.5},
                          {"Ha": 10.0, "Re": 10.0, "tau": 1.0, "tau_m": 1.0})
        spec = prob.lattice_spec(cs2_of(prob))
    elif case == "annulus_mhd":
        prob = gi.taylor_couette(n1=45, n2=11, r_in=6.0, sectors=9.0, Re=20.0, u_in=1.0, u_out=1.5)
        spec = prob.lattice_spec(cs2_of(prob))
        spec["walls"]["W"] = dict(spec["walls"]["W"], B=(0.02, 0.005))
        spec["mhd"] = {"tau_m": 0.9, "mu_m": 2.0, "B_init": (0.01, 0.004)}
    else:
        prob = gi.spiral_cavity(40, 37)
        spec = prob.lattice_spec(cs2_of(prob))
    L = goc.Lattice(spec, storage=storage)
    bad = ctypes.c_longlong(-1)
    _abi.check(goc.lib().goc_check_guards(L._h, ctypes.byref(bad)))
    assert bad.value == 0
    L.step(300)
    L.moments()
    L.init_fields()
    L.step(101)
    _abi.check(goc.lib().goc_check_guards(L._h, ctypes.byref(bad)))
    assert bad.value == 0
    if case == "cavity":   # the check sees a changed guard byte: one written through goc_set_state
        st = bytearray(L.get_state())
        st[64 + 100 * 4] ^= 0xFF            # first padding byte of row 0 of population plane 0
        L.set_state(bytes(st))
        _abi.check(goc.lib().goc_check_guards(L._h, ctypes.byref(bad)))
        assert bad.value >= 1
    L.close()


def test_single_column_node_table_matches_the_oracle_and_the_per_axis_grid(gpu):
    """A one-node-wide periodic channel (every xi1 pull wraps onto the node
    itself) whose wall-normal tanh metric is given as a node table: against
    the oracle and against the same channel on the per-axis map."""
    prob = gi.Problem("poiseuille", 1, 48, {"kind": "uniform"}, {"kind": "tanh2", "beta": 1.5},
                      {"Re": 10.0, "tau": 0.8})
    spec = prob.lattice_spec(cs2_of(prob))
    m = oracle.build_metric(spec)
    tab = dict(spec, map1={"kind": "table"}, map2={"kind": "uniform"},
               metric={"h1": m.h1, "h2": m.h2, "t11": m.t11, "t12": m.t12, "t21": m.t21, "t22": m.t22,
                       "wall": m.wall})
    o, L, fo, fg = run_pair(tab, 1000)
    assert relerr(np.stack(fg[1:3]), np.stack(fo[1:3])) <= 1e-5
    A = goc.Lattice(spec)
    A.step(1000)
    fa = A.moments()
    assert relerr(np.stack(fg[1:3]), np.stack(fa[1:3])) <= 1e-5
    L.close()
    A.close()
