"""FP64 metric factors for the oracle (test infrastructure only).

This module belongs to the CPU oracle.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` leg of ``bench.py`` may import it; the CUDA library
computes its own metric tables and shares nothing with this file.

What it computes
----------------
For a straight orthogonal grid x = x(xi1), y = y(xi2) the metric (Lame) factors
are h1 = dx/dxi1, h2 = dy/dxi2 (Eq. metricfactor, Sec. 2.1) and the curvature
matrix is theta_ij = (1/(h_i h_j)) dh_i/dxi_j (Eq. curvaturematrix), so that
theta_11 = h1'/h1^2, theta_22 = h2'/h2^2 and theta_12 = theta_21 = 0
(Appendix B, case (i)).

Maps (Sec. 6):
* ``uniform``: x = xi, h = 1, theta = 0.
* ``tanh2``: clustering at both walls (Eq. hypertanh_transformation1 and
  Eq. metriccoefficient, Sec. 6.1).  Reading of the node placement: nodes are
  cell-centred, eta_j = (j + 1/2)/N, walls at eta = 0 and 1 (half a spacing
  outside the first and last fluid node, as the half-way bounce-back of
  Sec. 7.1 implies) and the physical length is N lattice units, so
  x = (N/2) [1 + tanh(beta (2 eta - 1)) / tanh(beta)],
  h = (beta / tanh beta) sech^2(beta (2 eta - 1)),
  theta = -(4 tanh(beta) / N) tanh(beta (2 eta - 1)) / sech^2(beta (2 eta - 1)).
* ``sine``: a periodic stretching x = xi + (a N / 2 pi) sin(2 pi xi / N)
  (not in the paper; used for Taylor-Green decay and mass conservation on a
  stretched periodic grid), h = 1 + a cos(2 pi xi / N),
  theta = -a (2 pi / N) sin(2 pi xi / N) / h^2.
* ``roberts``: Roberts boundary-layer map (Eq. y_Roberts, Eq. h2_Roberts,
  Sec. 6.2) with lambda = (gamma + 1)/(gamma - 1) (the printed
  (gamma+1)/(gamma+1) is garbled; only this reading gives y(0) = 0 and the
  printed h2).  Cell-centred nodes as above with L = N.
* ``tanh1``: clustering at the wall xi = 0 only (Eq. hypertanh_transformation,
  Eq. metriccoefficientB, Sec. 6.3).  The printed prefactor L_y/2 would map
  onto [0, L/2]; the printed h2 and theta22 belong to the prefactor L, so
  x = N [1 - tanh(beta (1 - eta)) / tanh(beta)],
  h = (beta / tanh beta) sech^2(beta (1 - eta)),
  theta = (2 tanh(beta) / N) tanh(beta (1 - eta)) / sech^2(beta (1 - eta)).
* ``sinh``: clustering around an interior point x_c = yc N (Eq.
  Holst_transformation, Eq. B_Holst, Eq. h_2_Holst, Sec. 6.4), the printed
  "sinh ]" read as sinh[...]:
  B = ln[(1 + (e^mu - 1) yc) / (1 + (e^-mu - 1) yc)] / (2 mu),
  x = x_c [1 + sinh(mu (eta - B)) / sinh(mu B)],
  h = (x_c / N) mu cosh(mu (eta - B)) / sinh(mu B),
  theta = (sinh(mu B) / x_c) tanh(mu (eta - B)) sech(mu (eta - B)).

Periodic axes place nodes at eta_i = i / N.

Curvilinear grid (Sec. 8.1): the annular sector between circles of radii a
and R_o spanning 2 pi / N_theta, by the conformal map Z = a exp(pi W / N_theta)
(Eq. 2_annularsector) scaled to the lattice (Eq. 5_annularsector) with
cell-centred radial nodes (walls at xi1 = 0 and N1) and periodic azimuthal
nodes xi2 = j:
  r = a exp(ln(R_o/a) xi1/N1),  phi = (pi/N_theta)(2 xi2/N2 - 1),
  h1 = r ln(R_o/a)/N1,  h2 = 2 pi r/(N_theta N2),
  theta11 = theta21 = 1/r,  theta12 = theta22 = 0.
"""
from __future__ import annotations

import math

import numpy as np


def _eta(n: int, periodic: bool) -> np.ndarray:
    j = np.arange(n, dtype=np.float64)
    return j / n if periodic else (j + 0.5) / n


def _holst_b(mu: float, yc: float) -> float:
    """B of the interior map (Eq. B_Holst) for x_c / L = yc."""
    return math.log((1.0 + (math.exp(mu) - 1.0) * yc) / (1.0 + (math.exp(-mu) - 1.0) * yc)) / (2.0 * mu)


def map_position(kind: str, n: int, xi: np.ndarray, *, beta: float = 0.0,
                 a: float = 0.0, gamma: float = 0.0, alpha: float = 0.5,
                 mu: float = 0.0, yc: float = 0.5) -> np.ndarray:
    """Physical coordinate x(xi) of the named map, xi in [0, n] (lattice units)."""
    xi = np.asarray(xi, dtype=np.float64)
    if kind == "uniform" or (kind == "tanh2" and beta == 0.0):
        return xi.copy()
    if kind == "tanh2":
        eta = xi / n
        return 0.5 * n * (1.0 + np.tanh(beta * (2.0 * eta - 1.0)) / math.tanh(beta))
    if kind == "sine":
        return xi + a * n / (2.0 * math.pi) * np.sin(2.0 * math.pi * xi / n)
    if kind == "roberts":
        lam = (gamma + 1.0) / (gamma - 1.0)
        s = (xi / n - alpha) / (1.0 - alpha)
        ls = lam ** s
        return n * ((gamma + 2 * alpha) * ls - gamma + 2 * alpha) / ((2 * alpha + 1) * (1 + ls))
    if kind == "tanh1":
        return n * (1.0 - np.tanh(beta * (1.0 - xi / n)) / math.tanh(beta))
    if kind == "sinh":
        B = _holst_b(mu, yc)
        return yc * n * (1.0 + np.sinh(mu * (xi / n - B)) / math.sinh(mu * B))
    raise ValueError(f"unknown map {kind!r}")


def map_metric(kind: str, n: int, xi: np.ndarray, *, beta: float = 0.0,
               a: float = 0.0, gamma: float = 0.0, alpha: float = 0.5,
               mu: float = 0.0, yc: float = 0.5):
    """Analytic (h, theta) of the named map at the points xi."""
    xi = np.asarray(xi, dtype=np.float64)
    if kind == "uniform" or (kind == "tanh2" and beta == 0.0):
        return np.ones_like(xi), np.zeros_like(xi)
    if kind == "tanh2":
        arg = beta * (2.0 * xi / n - 1.0)
        sech2 = 1.0 / np.cosh(arg) ** 2
        h = beta / math.tanh(beta) * sech2
        theta = -(4.0 * math.tanh(beta) / n) * np.tanh(arg) / sech2
        return h, theta
    if kind == "sine":
        ph = 2.0 * math.pi * xi / n
        h = 1.0 + a * np.cos(ph)
        dh = -a * (2.0 * math.pi / n) * np.sin(ph)
        return h, dh / h ** 2
    if kind == "roberts":
        lam = (gamma + 1.0) / (gamma - 1.0)
        s = (xi / n - alpha) / (1.0 - alpha)
        ls = lam ** s
        h = (2.0 * gamma / (2 * alpha + 1)) * math.log(lam) / (1.0 - alpha) * ls / (1.0 + ls) ** 2
        theta = (1.0 / n) * ((1.0 + 2 * alpha) / (2.0 * gamma)) * (1.0 / ls - ls)
        return h, theta
    if kind == "tanh1":
        arg = beta * (1.0 - xi / n)
        sech2 = 1.0 / np.cosh(arg) ** 2
        h = beta / math.tanh(beta) * sech2
        theta = (2.0 * math.tanh(beta) / n) * np.tanh(arg) / sech2
        return h, theta
    if kind == "sinh":
        B = _holst_b(mu, yc)
        arg = mu * (xi / n - B)
        h = yc * mu * np.cosh(arg) / math.sinh(mu * B)
        theta = math.sinh(mu * B) / (yc * n) * np.tanh(arg) / np.cosh(arg)
        return h, theta
    raise ValueError(f"unknown map {kind!r}")


def axis_tables(kind: str, n: int, periodic: bool, **kw):
    """Per-axis node tables (h, theta) and the wall values h(0), h(n)."""
    xi = _eta(n, periodic) * n
    h, th = map_metric(kind, n, xi, **kw)
    hw, _ = map_metric(kind, n, np.array([0.0, float(n)]), **kw)
    return h, th, hw


class Metric:
    """Metric of a straight grid as 2D node arrays (row-major [ny, nx])."""

    def __init__(self, nx: int, ny: int, map1: dict, map2: dict,
                 periodic1: bool, periodic2: bool):
        m1 = dict(map1)
        m2 = dict(map2)
        k1 = m1.pop("kind", "uniform")
        k2 = m2.pop("kind", "uniform")
        h1, t1, hw1 = axis_tables(k1, nx, periodic1, **m1)
        h2, t2, hw2 = axis_tables(k2, ny, periodic2, **m2)
        self.nx, self.ny = nx, ny
        self.h1_axis, self.h2_axis = h1, h2
        self.h1 = np.broadcast_to(h1[None, :], (ny, nx)).copy()
        self.h2 = np.broadcast_to(h2[:, None], (ny, nx)).copy()
        self.t11 = np.broadcast_to(t1[None, :], (ny, nx)).copy()
        self.t22 = np.broadcast_to(t2[:, None], (ny, nx)).copy()
        self.t12 = np.zeros((ny, nx))
        self.t21 = np.zeros((ny, nx))
        # metric at the wall points: W/E walls run along xi2 (arrays over j),
        # S/N walls along xi1 (arrays over i); each holds (h1, h2) there.
        self.wall = {
            "W": (np.full(ny, hw1[0]), h2.copy()),
            "E": (np.full(ny, hw1[1]), h2.copy()),
            "S": (h1.copy(), np.full(nx, hw2[0])),
            "N": (h1.copy(), np.full(nx, hw2[1])),
        }

    def q(self) -> float:
        """q = min(min h1, min h2) over all nodes (Eq. GOC-LBE_CFL)."""
        return float(min(self.h1.min(), self.h2.min()))

    def cs2(self) -> float:
        """c_s^2 = q^2 / 3 (Eq. GOC-LBE_CFL)."""
        return self.q() ** 2 / 3.0


def annulus_position(xi1, xi2, n1: int, n2: int, r_in: float, r_out: float, sectors: float):
    """Cartesian (x1, x2) of the annular-sector map at lattice coordinates."""
    r = r_in * np.exp(math.log(r_out / r_in) * np.asarray(xi1, dtype=np.float64) / n1)
    phi = math.pi / sectors * (2.0 * np.asarray(xi2, dtype=np.float64) / n2 - 1.0)
    return r * np.cos(phi), r * np.sin(phi)


def annulus_metric(n1: int, n2: int, r_in: float, r_out: float, sectors: float) -> "Metric":
    """Metric of the annular sector (Eq. h1, h2, theta of Sec. 8.1) as a
    Metric: radial axis xi1 with walls, azimuthal axis xi2 periodic."""
    lam = math.log(r_out / r_in)

    def radial(xi1):
        r = r_in * np.exp(lam * np.asarray(xi1, dtype=np.float64) / n1)
        return r, r * lam / n1, 2.0 * math.pi * r / (sectors * n2), 1.0 / r

    m = Metric.__new__(Metric)
    m.nx, m.ny = n1, n2
    r, h1, h2, th = radial(np.arange(n1) + 0.5)
    m.h1_axis, m.h2_axis = h1, h2
    m.radius = r
    shape = (n2, n1)
    m.h1 = np.broadcast_to(h1[None, :], shape).copy()
    m.h2 = np.broadcast_to(h2[None, :], shape).copy()
    m.t11 = np.broadcast_to(th[None, :], shape).copy()
    m.t21 = np.broadcast_to(th[None, :], shape).copy()
    m.t12 = np.zeros(shape)
    m.t22 = np.zeros(shape)
    _, hw1, hw2, _ = radial(np.array([0.0, float(n1)]))
    m.wall = {
        "W": (np.full(n2, hw1[0]), np.full(n2, hw2[0])),
        "E": (np.full(n2, hw1[1]), np.full(n2, hw2[1])),
        "S": (h1.copy(), h2.copy()),
        "N": (h1.copy(), h2.copy()),
    }
    return m


def table_metric(nx: int, ny: int, table: dict) -> "Metric":
    """Metric given node by node (a general orthogonal grid): table holds
    [ny, nx] arrays h1, h2, t11, t12, t21, t22 (theta_ij of Eq.
    curvaturematrix) and "wall": {"W", "E": (h1, h2) over j, "S", "N": (h1,
    h2) over i} at the wall points (used by moving walls; any values on
    periodic sides)."""
    m = Metric.__new__(Metric)
    m.nx, m.ny = nx, ny
    for k in ("h1", "h2", "t11", "t12", "t21", "t22"):
        a = np.ascontiguousarray(np.asarray(table[k], dtype=np.float64))
        if a.shape != (ny, nx):
            raise ValueError(f"{k}: shape {a.shape}, want {(ny, nx)}")
        setattr(m, k, a.copy())
    m.h1_axis, m.h2_axis = m.h1[0].copy(), m.h2[:, 0].copy()
    m.wall = {w: (np.asarray(table["wall"][w][0], dtype=np.float64).copy(),
                  np.asarray(table["wall"][w][1], dtype=np.float64).copy()) for w in ("W", "E", "S", "N")}
    return m
