"""Continuous batching on the GPU: requests admitted while others run give,
each, the same result as when run alone (bitwise in FP32: the batched step
is the same arithmetic and a budget request runs exactly its budget)."""
import numpy as np
import pytest

import goc_inputs as gi
import paper_2607_15362_b300 as goc
from paper_2607_15362_b300.serve import Request, Server, lattice_spec, run_sequential

pytestmark = pytest.mark.gpu


def _mix():
    probs = [
        gi.Problem("cavity", 48, 40, {"kind": "tanh2", "beta": 1.5}, {"kind": "tanh2", "beta": 1.5},
                   {"Re": 200.0, "u_lid": 0.05, "mach_matched": True}),
        gi.Problem("poiseuille", 24, 64, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0}, {"Re": 50.0, "tau": 0.8}),
        gi.Problem("hartmann", 8, 64, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                   {"Ha": 20.0, "Re": 20.0, "tau": 1.0, "tau_m": 1.0}),
        gi.Problem("cavity", 96, 80, {"kind": "tanh2", "beta": 2.0}, {"kind": "tanh2", "beta": 2.0},
                   {"Re": 500.0, "u_lid": 0.05, "mach_matched": True}),
        gi.Problem("poiseuille", 40, 40, {"kind": "uniform"}, {"kind": "tanh2", "beta": 1.0}, {"Re": 20.0, "tau": 1.0}),
        gi.Problem("hartmann", 33, 50, {"kind": "uniform"}, {"kind": "tanh2", "beta": 1.5},
                   {"Ha": 8.0, "Re": 10.0, "tau": 1.0, "tau_m": 1.0}),
    ]
    budgets = [900, 1300, 700, 1100, 20000, 500]
    tols = [None, None, None, None, 1e-5, None]
    arrivals = [0.0, 0.0, 0.02, 0.05, 0.05, 0.08]
    return [Request(k, a, p, b, t) for k, (p, b, t, a) in enumerate(zip(probs, budgets, tols, arrivals))]


def test_each_result_is_the_same_alone_and_in_the_mix(gpu):
    reqs = _mix()
    srv = Server(hbm_budget_bytes=1 << 30, max_slots=16, chunk=250, keep_fields=True)
    results, summary = srv.run(reqs)
    srv.close()
    assert summary["done"] == len(reqs)
    for res in results:
        rq = reqs[res.rid]
        alone = goc.Lattice(lattice_spec(rq.problem))
        alone.step(res.steps)           # the residual request: same number of steps
        for x, y in zip(res.fields, alone.moments()):
            np.testing.assert_array_equal(x, y)
        if rq.tol is None:
            assert res.steps == rq.budget
        else:
            assert res.residual < rq.tol and res.steps < rq.budget
        alone.close()


def test_admission_waits_for_memory_and_sequential_baseline_agrees(gpu):
    reqs = _mix()[:4]
    # budget for about two of these lattices at a time: later ones wait for retirements
    srv = Server(hbm_budget_bytes=900_000, max_slots=16, chunk=200, keep_fields=True)
    results, summary = srv.run(reqs)
    srv.close()
    assert summary["done"] == 4
    seq, seq_summary = run_sequential(reqs, keep_fields=True)
    by = {r.rid: r for r in seq}
    for res in results:
        for x, y in zip(res.fields, by[res.rid].fields):
            np.testing.assert_array_equal(x, y)
    assert summary["p50_latency_s"] is not None and summary["p99_latency_s"] >= summary["p50_latency_s"]
