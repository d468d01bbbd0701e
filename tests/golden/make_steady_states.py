"""Write the oracle's states of the x-invariant channel strips of
goc_inputs.steady_strips() to tests/golden/steady_<name>.txt.

Calls only the FP64 oracle (oracle/) and the problem definitions
(goc_inputs).  Each strip is run one column wide (the problems are invariant
along xi1, so every column of the wider lattice has the same solution) from
the start its GPU test uses (rest, or the analytic Hartmann profiles of Sec.
7.4) for the same number of steps, i.e. to the steady state of the flow: the
file records the largest relative change of U1 (and B1) over the last block
of steps as the evidence (the clustered Hartmann channel's own discrete
steady state differs from the analytic profiles by about 2e-5 and its slowest
mode decays over ~1e7 steps, so it is scored at a fixed step count).

Usage: python tests/golden/make_steady_states.py [name ...]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import goc_inputs as gi  # noqa: E402
import oracle  # noqa: E402

BLOCK = 20_000


def steady(name: str, prob: gi.Problem, start: str, steps: int) -> str:
    strip = gi.Problem(prob.kind, 1, prob.ny, prob.map1, prob.map2, prob.params)
    cs2 = oracle.build_metric(strip.lattice_spec(1.0)).cs2()
    spec = strip.lattice_spec(cs2)
    o = oracle.Oracle(spec, threads=1)
    if start == "analytic":
        y = strip.ny * gi.wall_positions(strip.map2, strip.ny)
        ua, ba = gi.hartmann_profiles(spec, float(strip.params["Ha"]), y)
        o.initialize(u1=ua.reshape(strip.ny, 1), b1=ba.reshape(strip.ny, 1))
    t0 = time.time()
    o.step(steps - BLOCK)
    prev = o.fields()
    o.step(BLOCK)
    f = o.fields()
    change = float(np.abs(f[1] - prev[1]).max() / np.abs(f[1]).max())
    if strip.mhd:
        change = max(change, float(np.abs(f[3] - prev[3]).max() / np.abs(f[3]).max()))
    prev = f
    rho, u1, u2, b1, b2 = (a[:, 0] for a in prev)
    path = os.path.join(HERE, f"steady_{name}.txt")
    with open(path, "w") as fh:
        fh.write(f"# State of the FP64 oracle at the steady flow: {name}, {strip.ny} rows, one column (x-invariant).\n")
        fh.write(f"# Written by tests/golden/make_steady_states.py: {steps} steps from {start};\n")
        fh.write(f"# largest relative change of U1{' and B1' if strip.mhd else ''} over the last {BLOCK} steps: "
                 f"{change:.3e}.  c_s^2 = {cs2:.17g}.\n")
        fh.write("# columns: row j, rho, U1, U2, B1, B2\n")
        for j in range(strip.ny):
            fh.write(f"{j} {rho[j]:.17g} {u1[j]:.17g} {u2[j]:.17g} {b1[j]:.17g} {b2[j]:.17g}\n")
    return f"{name}: {steps} steps from {start}, change {change:.2e}, {time.time() - t0:.0f} s -> {path}"


def load(name: str) -> dict:
    """The stored profile of strip `name`: arrays rho, U1, U2, B1, B2 over the rows."""
    a = np.loadtxt(os.path.join(HERE, f"steady_{name}.txt"))
    return {"rho": a[:, 1], "U1": a[:, 2], "U2": a[:, 3], "B1": a[:, 4], "B2": a[:, 5]}


if __name__ == "__main__":
    strips = gi.steady_strips()
    for name in (sys.argv[1:] or list(strips)):
        print(steady(name, *strips[name]), flush=True)
