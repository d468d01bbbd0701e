"""Seeded synthetic problem generators shared by the tests and the benchmark.

This module holds problem definitions only (sizes, stretching maps, boundary
conditions, Reynolds/Hartmann numbers, seeds).  It contains none of the
GOC-LBM arithmetic: the speed of sound c_s^2 = q^2/3 comes from whichever
implementation is being driven (the oracle's metric or the library's own
query), and is passed in to ``Problem.lattice_spec``.

Conversions from the physical definitions to lattice parameters follow the
problem statements of the paper:
  * Poiseuille channel (Sec. 7.1): U = F_ext (H/2)^2 / (2 nu), Re = U (H/2)/nu.
  * Lid-driven cavity (Sec. 7.3): Re = U_lid H / nu.
  * Hartmann channel (Sec. 7.4): Ha = B0 H sqrt(sigma/(rho nu)), eta = 1/(sigma mu_m),
    U_r = H^2 F_x / (rho nu), centreline u(0) = U_r (1 - 1/cosh Ha)/(Ha tanh Ha),
    Re = u(0) H / nu (H = half-width).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    kind: str                     # "poiseuille" | "cavity" | "hartmann" | "taylor_green" | "couette" | "taylor_couette"
    nx: int
    ny: int
    map1: dict
    map2: dict
    params: dict = field(default_factory=dict)
    steps: int = 0
    name: str = ""
    metric: dict | None = None    # node table of a general orthogonal grid (map1 kind "table")

    # ---- geometry ------------------------------------------------------
    def walls(self) -> dict:
        k = self.kind
        if k in ("poiseuille", "hartmann"):
            w = {"W": None, "E": None, "S": {"u": 0.0}, "N": {"u": 0.0}}
        elif k == "couette":
            w = {"W": None, "E": None, "S": {"u": 0.0}, "N": {"u": self.params["u_wall"]}}
        elif k == "cavity":
            w = {"W": {"u": 0.0}, "E": {"u": 0.0}, "S": {"u": 0.0}, "N": {"u": self.params["u_lid"]}}
        elif k == "taylor_green":
            w = {"W": None, "E": None, "S": None, "N": None}
        elif k == "taylor_couette":   # radial walls (xi1) move along xi2; azimuth periodic
            w = {"W": {"u": self.params["u_in"]}, "E": {"u": self.params["u_out"]}, "S": None, "N": None}
        else:
            raise ValueError(k)
        if k == "hartmann":
            b = (0.0, 0.0)  # filled by lattice_spec once B0 is known
            w["S"]["B"] = b
            w["N"]["B"] = b
        return w

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    @property
    def mhd(self) -> bool:
        return self.kind == "hartmann"

    # ---- lattice parameters -----------------------------------------------
    def lattice_spec(self, cs2: float) -> dict:
        """Spec in lattice units for a given c_s^2 (taken from the metric of
        the implementation that will run it)."""
        p = self.params
        spec = {"nx": self.nx, "ny": self.ny, "map1": dict(self.map1), "map2": dict(self.map2),
                "walls": self.walls(), "rho0": 1.0, "gi": int(p.get("gi", 1)),
                "tau_zeta": float(p.get("tau_zeta", 1.0))}
        if self.metric is not None:
            spec["metric"] = self.metric
        k = self.kind
        if k == "poiseuille":
            tau = float(p["tau"])
            nu = cs2 * (tau - 0.5)
            H = float(self.ny)
            U = p["Re"] * nu / (0.5 * H)
            if "mach_max" in p:   # keep the centreline speed subsonic on this lattice
                U = min(U, float(p["mach_max"]) * math.sqrt(cs2))
            spec.update(tau=tau, fext=(2.0 * nu * U / (0.5 * H) ** 2, 0.0))
            spec["derived"] = {"U": U, "nu": nu, "H": H}
        elif k == "couette":
            spec.update(tau=float(p["tau"]), fext=(0.0, 0.0))
        elif k == "cavity":
            u = float(p["u_lid"])
            if p.get("mach_matched"):       # same Mach number as u_lid on a lattice with cs^2 = 1/3
                u = u * math.sqrt(3.0 * cs2)
            if "lid_cs_fraction" in p:     # keep the lid Mach number moderate
                u = min(u, float(p["lid_cs_fraction"]) * math.sqrt(cs2))
            spec["walls"]["N"]["u"] = u
            nu = u * self.nx / p["Re"]
            if "tau_max" in p:   # keep tau = 1/2 + nu/cs^2 inside the step's stability range
                nu = min(nu, cs2 * (float(p["tau_max"]) - 0.5))
            spec.update(nu=nu, fext=(0.0, 0.0))
            spec["derived"] = {"nu": nu, "u_lid": u}
        elif k == "taylor_green":
            spec.update(tau=float(p["tau"]), fext=(0.0, 0.0))
            spec["init"] = taylor_green_init(self, float(p["u0"]))
        elif k == "taylor_couette":   # Re = U0 (R2 - R1)/nu, R2 - R1 = nx lattice units (Sec. 8.2)
            nu = float(p["U0"]) * self.nx / float(p["Re"])
            spec.update(nu=nu, fext=(0.0, 0.0))
            spec["derived"] = {"nu": nu}
        elif k == "hartmann":
            tau = float(p.get("tau", 1.0))
            taum = float(p.get("tau_m", 1.0))
            nu = cs2 * (tau - 0.5)
            eta = cs2 * (taum - 0.5)       # c_sm = c_s
            H = 0.5 * self.ny
            Ha, Re = float(p["Ha"]), float(p["Re"])
            B0 = Ha * math.sqrt(nu * eta) / H          # rho = mu_m = 1
            u0 = Re * nu / H
            if "mach_max" in p:   # keep the centreline speed subsonic on this lattice
                u0 = min(u0, float(p["mach_max"]) * math.sqrt(cs2))
            Fx = u0 * nu / (H * H) / ((1.0 - 1.0 / math.cosh(Ha)) / (Ha * math.tanh(Ha)))
            spec.update(tau=tau, fext=(Fx, 0.0), mhd={"tau_m": taum, "mu_m": 1.0, "B_init": (0.0, B0)})
            spec["walls"]["S"]["B"] = (0.0, B0)
            spec["walls"]["N"]["B"] = (0.0, B0)
            spec["derived"] = {"nu": nu, "eta": eta, "B0": B0, "u0": u0, "Fx": Fx, "H": H}
        return spec


def taylor_green_init(prob: Problem, u0: float) -> dict:
    """u = -U0 cos(k x) sin(k y), v = U0 sin(k x) cos(k y) at the physical node
    positions of the periodic maps, k = 2 pi / N (Cartesian components equal
    the GOC ones for straight grids)."""
    from_axis = _node_positions
    x = from_axis(prob.map1, prob.nx)
    y = from_axis(prob.map2, prob.ny)
    kx, ky = 2 * math.pi / prob.nx, 2 * math.pi / prob.ny
    X, Y = np.meshgrid(x, y)
    return {"u1": -u0 * np.cos(kx * X) * np.sin(ky * Y), "u2": u0 * np.sin(kx * X) * np.cos(ky * Y)}


def _node_positions(m: dict, n: int) -> np.ndarray:
    """Physical positions of periodic-axis nodes xi = 0..n-1 (problem geometry)."""
    xi = np.arange(n, dtype=np.float64)
    if m.get("kind", "uniform") == "uniform":
        return xi
    if m["kind"] == "sine":
        return xi + m["a"] * n / (2 * math.pi) * np.sin(2 * math.pi * xi / n)
    raise ValueError(m)


def wall_positions(m: dict, n: int) -> np.ndarray:
    """Physical node positions, as a fraction of the side, of a wall axis
    with cell-centred nodes (eta = (j + 1/2)/n, walls at 0 and 1) under the
    uniform map, the two-wall tanh map (Sec. 6.1) or the two-wall Roberts map
    (Sec. 6.2, alpha = 1/2, lambda = (gamma + 1)/(gamma - 1)): problem
    geometry for scoring against analytic profiles."""
    eta = (np.arange(n) + 0.5) / n
    kind = m.get("kind", "uniform")
    if kind == "uniform":
        return eta
    if kind == "tanh2":
        b = float(m["beta"])
        return 0.5 * (1.0 + np.tanh(b * (2.0 * eta - 1.0)) / np.tanh(b))
    if kind == "roberts" and float(m.get("alpha", 0.5)) == 0.5:
        g = float(m["gamma"])
        ls = ((g + 1.0) / (g - 1.0)) ** (2.0 * eta - 1.0)
        return ((g + 1.0) * ls + 1.0 - g) / (2.0 * (1.0 + ls))
    raise ValueError(m)


def hartmann_profiles(spec: dict, Ha: float, y: np.ndarray):
    """Analytic u_x and B_x of the Hartmann flow (Sec. 7.4) at physical
    positions y in [0, 2H] of a channel of half-width H (spec["derived"] of a
    "hartmann" Problem): u = U_r (1 - cosh(Ha y*)/cosh Ha)/(Ha tanh Ha),
    B_x = B_r (-y*/Ha + sinh(Ha y*)/(Ha tanh(Ha) cosh Ha)), y* = y/H - 1,
    U_r = H^2 F_x/nu, B_r = H^2 F_x/sqrt(nu eta) (rho = mu_m = 1)."""
    d = spec["derived"]
    ys = np.asarray(y, dtype=np.float64) / d["H"] - 1.0
    Ur = d["H"] ** 2 * d["Fx"] / d["nu"]
    Br = d["H"] ** 2 * d["Fx"] / math.sqrt(d["nu"] * d["eta"])
    ua = Ur / (Ha * math.tanh(Ha)) * (1 - np.cosh(Ha * ys) / math.cosh(Ha))
    ba = Br * (-ys / Ha + np.sinh(Ha * ys) / (Ha * math.tanh(Ha) * math.cosh(Ha)))
    return ua, ba


def steady_strips() -> dict:
    """x-invariant channel strips whose steady states the 16-bit storage
    tests score against (oracle profiles in tests/golden/): the Poiseuille
    channel of the benchmark (32 x 64), a Hartmann strip (4 x 96, tanh beta =
    2, Ha = 20, Re = 20) and a strip of the 256 x 1024 Hartmann channel with
    its clustering (tanh beta = 3, Ha = 100, Re = 100).  name -> (Problem,
    start, steps on the GPU); start "analytic" begins from the profiles of
    Sec. 7.4 (the clustered channel needs ~1e8 steps from rest)."""
    return {
        "poiseuille_64": (poiseuille_channel(), "rest", 800_000),
        "hartmann_ha20_96": (Problem("hartmann", 4, 96, {"kind": "uniform"}, {"kind": "tanh2", "beta": 2.0},
                                     {"Ha": 20.0, "Re": 20.0, "tau": 1.0, "tau_m": 1.0}), "rest", 800_000),
        "hartmann_ha100_1024": (hartmann_channel(nx=4), "analytic", 500_000),
    }


# ---- the benchmark configurations -------------------------------------------

def poiseuille_channel(nx: int = 32, ny: int = 64, beta: float = 1.5) -> Problem:
    """Plain GOC-LBM Poiseuille channel: 32 x 64, wall-normal tanh map
    beta = 1.5, Re = 10, tau = 0.8, body-force driven, 2000 steps from rest."""
    return Problem("poiseuille", nx, ny, {"kind": "uniform"}, {"kind": "tanh2", "beta": beta},
                   {"Re": 10.0, "tau": 0.8}, steps=2000, name="poiseuille_channel_32x64")


def lid_cavity(n: int = 512, beta: float = 2.0, Re: float = 1000.0, u_lid: float = 0.05,
                steps: int = 20000, mach_matched: bool = True) -> Problem:
    """Lid-driven cavity 512 x 512, tanh clustering to all four walls (beta = 2),
    Re = 1000, 20000 steps.  The lid speed 0.05 is taken at the Mach number it
    has on a standard lattice (Ma = 0.05 sqrt 3 = 0.087), i.e. 0.05 q in the
    GOC lattice units where c_s = q/sqrt 3; taken literally (mach_matched=False)
    it is Mach 0.58 on this grid and the FP64 oracle diverges near step 850."""
    return Problem("cavity", n, n, {"kind": "tanh2", "beta": beta}, {"kind": "tanh2", "beta": beta},
                   {"Re": Re, "u_lid": u_lid, "mach_matched": mach_matched}, steps=steps,
                   name=f"lid_cavity_{n}x{n}")


def uniform_cavity(n: int = 1024, Re: float = 1000.0, u_lid: float = 0.05,
                            steps: int = 20000) -> Problem:
    """The matched-accuracy baseline: the same cavity on a uniform 1024^2 grid
    (c_s^2 = 1/3, lid 0.05 = Mach 0.087), run by the standard uniform-grid
    central-moment LBM, i.e. without the cubic correction terms (gi = 0)."""
    return Problem("cavity", n, n, {"kind": "uniform"}, {"kind": "uniform"},
                   {"Re": Re, "u_lid": u_lid, "gi": 0}, steps=steps, name=f"uniform_cavity_{n}x{n}")


def hartmann_channel(nx: int = 256, ny: int = 1024, beta: float = 3.0, Ha: float = 100.0,
                  Re: float = 100.0) -> Problem:
    """Coupled MHD Hartmann channel 256 x 1024, wall-normal tanh beta = 3,
    Ha = 100, Re = 100, magnetic Prandtl number 1 (tau = tau_m)."""
    return Problem("hartmann", nx, ny, {"kind": "uniform"}, {"kind": "tanh2", "beta": beta},
                   {"Ha": Ha, "Re": Re, "tau": 1.0, "tau_m": 1.0}, steps=0,
                   name=f"hartmann_channel_{nx}x{ny}")


def batch_lattices(seed: int = 7, count: int = 64, steps: int = 5000) -> list[Problem]:
    """64 independent stretched-grid lattices: long side log-uniform in
    [128, 2048], aspect uniform in [1, 4], beta uniform in [0.5, 3], Re
    log-uniform in [100, 2000]; half cavities, half channels (Poiseuille or
    Hartmann with probability 1/2, Ha uniform in [10, 200]).  A cavity's
    viscosity is capped at tau = 1 (over long runs the clustered-grid step
    diverged at tau = 1.5), which raises its Reynolds number where n/Re is
    large; channel speeds are capped at Mach 0.1 on the lattice, which lowers
    the Reynolds number of small, fast channels."""
    rng = np.random.default_rng(seed)
    kinds = np.array(["cavity"] * (count // 2) + ["channel"] * (count - count // 2))
    rng.shuffle(kinds)
    out = []
    for k, kind in enumerate(kinds):
        L = int(round(math.exp(rng.uniform(math.log(128), math.log(2048)))))
        a = rng.uniform(1.0, 4.0)
        short = max(128, int(round(L / a)))
        beta = float(rng.uniform(0.5, 3.0))
        Re = float(math.exp(rng.uniform(math.log(100), math.log(2000))))
        if kind == "cavity":
            out.append(Problem("cavity", L, short, {"kind": "tanh2", "beta": beta},
                               {"kind": "tanh2", "beta": beta},
                               {"Re": Re, "u_lid": 0.05, "lid_cs_fraction": 0.1, "tau_max": 1.0},
                               steps=steps, name=f"b{k}_cavity_{L}x{short}"))
        else:
            hart = rng.uniform() < 0.5
            Ha = float(rng.uniform(10, 200))
            if hart:
                out.append(Problem("hartmann", short, L, {"kind": "uniform"},
                                   {"kind": "tanh2", "beta": beta},
                                   {"Ha": Ha, "Re": Re, "tau": 1.0, "tau_m": 1.0, "mach_max": 0.1},
                                   steps=steps, name=f"b{k}_hartmann_{short}x{L}"))
            else:
                out.append(Problem("poiseuille", short, L, {"kind": "uniform"},
                                   {"kind": "tanh2", "beta": beta}, {"Re": Re, "tau": 0.8, "mach_max": 0.1},
                                   steps=steps, name=f"b{k}_poiseuille_{short}x{L}"))
    return out


def serving_trace(seed: int = 11, count: int = 2000, rate_hz: float = 200.0,
                side_range=(64, 2048)) -> list[dict]:
    """Serving trace: Poisson arrivals (rate 200/s), NSE : NSE+MIE = 1 : 1,
    cavity : channel = 1 : 1 among NSE, square sides log-uniform in [64, 2048],
    beta uniform in [0.5, 3], Re log-uniform in [100, 2000], Ha uniform in
    [10, 200]; stop at a step budget log-uniform in [1k, 50k] (p = 1/2) or at
    residual 1e-8 capped at 50k steps.  Cavity viscosities and channel speeds
    are capped as in batch_lattices."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate_hz)
        mhd = rng.uniform() < 0.5
        side = int(round(math.exp(rng.uniform(math.log(side_range[0]), math.log(side_range[1])))))
        beta = float(rng.uniform(0.5, 3.0))
        Re = float(math.exp(rng.uniform(math.log(100), math.log(2000))))
        Ha = float(rng.uniform(10, 200))
        if rng.uniform() < 0.5:
            budget = int(round(math.exp(rng.uniform(math.log(1000), math.log(50000)))))
            tol = None
        else:
            budget, tol = 50000, 1e-8
        if mhd:
            prob = Problem("hartmann", side, side, {"kind": "uniform"}, {"kind": "tanh2", "beta": beta},
                           {"Ha": Ha, "Re": Re, "tau": 1.0, "tau_m": 1.0, "mach_max": 0.1},
                           name=f"r{k}_hartmann_{side}")
        elif rng.uniform() < 0.5:
            prob = Problem("cavity", side, side, {"kind": "tanh2", "beta": beta},
                           {"kind": "tanh2", "beta": beta},
                           {"Re": Re, "u_lid": 0.05, "lid_cs_fraction": 0.1, "tau_max": 1.0},
                           name=f"r{k}_cavity_{side}")
        else:
            prob = Problem("poiseuille", side, side, {"kind": "uniform"}, {"kind": "tanh2", "beta": beta},
                           {"Re": Re, "tau": 0.8, "mach_max": 0.1}, name=f"r{k}_poiseuille_{side}")
        out.append({"arrival_s": t, "problem": prob, "budget": budget, "tol": tol})
    return out


def taylor_green(n: int = 64, a: float = 0.3, u0: float = 0.01, tau: float = 0.8) -> Problem:
    """Decaying Taylor-Green vortex on a sine-stretched periodic grid."""
    m = {"kind": "sine", "a": a} if a else {"kind": "uniform"}
    return Problem("taylor_green", n, n, dict(m), dict(m), {"u0": u0, "tau": tau}, name=f"tg_{n}")


def random_periodic_fields(nx: int, ny: int, seed: int, amp: float = 0.02):
    """Smooth random velocity field (a few Fourier modes) for parity tests."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx)[None, :] * 2 * math.pi / nx
    y = np.arange(ny)[:, None] * 2 * math.pi / ny
    u1 = np.zeros((ny, nx))
    u2 = np.zeros((ny, nx))
    for _ in range(4):
        kx, ky = rng.integers(0, 3, size=2)
        p1, p2 = rng.uniform(0, 2 * math.pi, size=2)
        c1, c2 = rng.normal(size=2) * amp / 4
        u1 += c1 * np.sin(kx * x + ky * y + p1)
        u2 += c2 * np.cos(kx * x - ky * y + p2)
    return u1, u2


def taylor_couette(n1: int = 256, n2: int = 6, r_in: float = 32.0, sectors: float = 60.0, Re: float = 50.0,
                   U0: float = 0.01, u_in: float = 1.0, u_out: float = 1.5) -> Problem:
    """Taylor-Couette flow in an annular sector (Sec. 8): inner radius r_in,
    outer r_in + n1, 2 pi / sectors of the circle on n2 periodic azimuthal
    nodes; wall speeds u_in U0 (inner) and u_out U0 (outer)."""
    m1 = {"kind": "annulus", "r_in": r_in, "r_out": r_in + n1, "sectors": sectors}
    return Problem("taylor_couette", n1, n2, m1, {"kind": "uniform"},
                   {"Re": Re, "U0": U0, "u_in": u_in * U0, "u_out": u_out * U0}, name=f"taylor_couette_{n1}x{n2}")


def taylor_couette_profile(r: np.ndarray, r1: float, r2: float, u1: float, u2: float) -> np.ndarray:
    """Azimuthal velocity of circular Couette flow between cylinders of radii
    r1 < r2 with wall speeds u1 = Omega1 r1, u2 = Omega2 r2 (Sec. 8.2)."""
    o1, o2, e2 = u1 / r1, u2 / r2, (r1 / r2) ** 2
    return ((o2 - o1 * e2) * r + r1 * r1 * (o1 - o2) / r) / (1.0 - e2)


def spiral_grid(nx: int, ny: int, c: float, phi: float) -> dict:
    """Node table of the orthogonal grid of the conformal map
    z = exp(a (w - w0)) / a, w = xi1 + i xi2, a = c e^{i phi}, w0 the lattice
    centre: h1 = h2 = h = exp(c (cos(phi) (xi1 - nx/2) - sin(phi) (xi2 - ny/2))),
    so theta11 = theta21 = c cos(phi)/h and theta12 = theta22 = -c sin(phi)/h
    (theta_ij = dh_i/dxi_j / (h_i h_j)); the lines of constant xi are
    logarithmic spirals.  Nodes at xi = (i + 1/2, j + 1/2), walls at xi1 = 0,
    nx and xi2 = 0, ny."""
    def h(x1, x2):
        return np.exp(c * (math.cos(phi) * (x1 - nx / 2.0) - math.sin(phi) * (x2 - ny / 2.0)))

    x1 = (np.arange(nx) + 0.5)[None, :]
    x2 = (np.arange(ny) + 0.5)[:, None]
    hn = h(x1, x2)
    ta, tb = c * math.cos(phi) / hn, -c * math.sin(phi) / hn
    i_, j_ = np.arange(nx) + 0.5, np.arange(ny) + 0.5
    wall = {"W": (h(0.0, j_),) * 2, "E": (h(float(nx), j_),) * 2, "S": (h(i_, 0.0),) * 2, "N": (h(i_, float(ny)),) * 2}
    return {"h1": hn, "h2": hn.copy(), "t11": ta, "t12": tb, "t21": ta.copy(), "t22": tb.copy(), "wall": wall}


def spiral_cavity(nx: int = 40, ny: int = 37, c: float | None = None, phi: float = 0.6, Re: float = 50.0,
                  u_lid: float = 0.05, mach_matched: bool = False) -> Problem:
    """Lid-driven cavity on the logarithmic-spiral grid (every theta_ij
    non-zero): walls on all sides, the N wall moving along xi1
    (mach_matched: the lid at the Mach number u_lid has on a standard
    lattice)."""
    c = 1.0 / math.hypot(nx, ny) if c is None else c
    return Problem("cavity", nx, ny, {"kind": "table"}, {"kind": "uniform"},
                   {"Re": Re, "u_lid": u_lid, "mach_matched": mach_matched},
                   metric=spiral_grid(nx, ny, c, phi), name=f"spiral_cavity_{nx}x{ny}")
