"""Host-side helpers of bench.py (no GPU)."""
import numpy as np

import bench
import goc_inputs as gi


def _tanh_positions(beta, n):
    eta = (np.arange(n) + 0.5) / n
    return 0.5 * (1.0 + np.tanh(beta * (2.0 * eta - 1.0)) / np.tanh(beta))


def test_vortex_centres_are_found_at_a_known_extremum():
    """A stream function psi = (x - x0)^2 y + (y - y0)^2 - y0^2 (zero on the
    bottom wall, minimum at (x0, y0)) sampled on the clustered nodes through
    u = dpsi/dy: the primary centre comes back to 1e-3; a lone local maximum
    of psi in the bottom-right corner region is found there."""
    prob = gi.lid_cavity(n=96, beta=1.2)
    x = _tanh_positions(1.2, 96)
    X, Y = np.meshgrid(x, x)
    x0, y0 = 0.5314, 0.5646
    u = (X - x0) ** 2 + 2 * (Y - y0)
    c = bench._vortex_centres(prob, [None, u, None])
    assert abs(c["primary"][0] - x0) < 1e-3 and abs(c["primary"][1] - y0) < 1e-3
    # a secondary vortex alone: psi a bump (local maximum) centred at (0.86, 0.11)
    xb, yb, w = 0.86, 0.11, 0.03
    bump = 1e-3 * np.exp(-((X - xb) ** 2 + (Y - yb) ** 2) / w ** 2)
    u2 = bump * (-2 * (Y - yb) / w ** 2)
    c2 = bench._vortex_centres(prob, [None, u2, None])
    assert abs(c2["bottom_right"][0] - xb) < 0.01 and abs(c2["bottom_right"][1] - yb) < 0.01


def test_job_rate_counts_every_rank():
    """value = node updates of all ranks / the slowest rank's time."""
    assert bench.job_rate(4, 1e6, 2000.0) == 4 * 1e6 / 2.0 / 1e6


def test_bench_wall_positions_match_the_maps():
    """The node positions bench.py scores profiles against are the uniform,
    tanh and Roberts maps at cell-centred nodes (checked against the
    oracle's map positions)."""
    from oracle.metric import map_position
    for m, n in (({"kind": "uniform"}, 40), ({"kind": "tanh2", "beta": 1.2}, 64), ({"kind": "tanh2", "beta": 3.0}, 50),
                 ({"kind": "roberts", "gamma": 1.05, "alpha": 0.5}, 270)):
        kw = {k: v for k, v in m.items() if k != "kind"}
        want = map_position(m["kind"], n, np.arange(n) + 0.5, **kw) / n
        np.testing.assert_allclose(bench._wall_positions(m, n), want, rtol=0, atol=1e-13)
