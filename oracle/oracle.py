"""Python driver of the FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference legs may import this module.  It compiles ``goc_oracle.c`` with gcc
(no CUDA, no code shared with the library) and drives it through ctypes.

A problem is described by a plain dict ``spec`` (see ``goc_inputs``):

    nx, ny            lattice size
    map1, map2        {"kind": "uniform"|"tanh2"|"sine"|"roberts", parameters}
    walls             {"W","E","S","N"} -> None (periodic) or
                      {"u": tangential velocity, "B": (B1, B2) for the MIE}
    tau | nu          shear relaxation time (omega4 = omega5 = 1/tau) or the
                      kinematic viscosity nu = cs^2 (tau - 1/2) (Eq. 73, Eq. 76)
    tau_zeta          omega3 = 1/tau_zeta, zeta = cs^2 (tau_zeta - 1/2); default 1
    omega_free        omega0,1,2,6,7,8 (default 1, preparatory step (d))
    fext              (F_ext,1, F_ext,2)
    gi                1: full correction coefficients (default); 0: cubic terms dropped
    collision         "cm" (default): central-moment MRT of Appendix E; "srt": the
                      single-relaxation-time GOC-LBM in velocity space of Appendix F
                      (one rate 1/tau for every moment, zeta = nu); "raw": the
                      raw-moment MRT of Appendix D (rates as for "cm")
    mhd               None or {"tau_m" | "eta", "mu_m"}
    rho0              reference density (default 1)

Readings of the paper used here are listed in ``goc_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .metric import Metric, annulus_metric, table_metric

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "goc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgoc_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O3 -march=native, no fast-math, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O3", "-march=native", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_create.restype = ctypes.c_void_p
            lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int] + [_D] * 6 + [
                _I, _D, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D,
                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, ctypes.c_int]
            lib.orc_destroy.argtypes = [ctypes.c_void_p]
            lib.orc_init.argtypes = [ctypes.c_void_p] + [_D] * 5
            lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_fields.argtypes = [ctypes.c_void_p] + [_D] * 5
            lib.orc_get_state.argtypes = [ctypes.c_void_p] + [_D] * 4
            lib.orc_set_state.argtypes = [ctypes.c_void_p] + [_D] * 4
            lib.orc_frame_matrix.argtypes = [ctypes.c_double, ctypes.c_double, _D]
            lib.orc_p_matrix.argtypes = [ctypes.c_void_p, _D, _D]
            lib.orc_central_equilibria.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 7 + [_D]
            lib.orc_raw_equilibria.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 7 + [_D]
            lib.orc_corrections.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 13 + [_D]
            lib.orc_mie_diag.argtypes = [ctypes.c_void_p] + [_D] * 3
            lib.orc_mie_grad.argtypes = [ctypes.c_void_p, _D]
            lib.orc_set_collision.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_srt_equilibria.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 13 + [_D]
            lib.orc_srt_to_populations.argtypes = [_D, _D]
            lib.orc_threads.argtypes = [ctypes.c_void_p]
            lib.orc_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


_WALLS = ("W", "E", "S", "N")


def derived_parameters(spec: dict, metric: Metric) -> dict:
    """Lattice parameters of a spec: c_s^2 from the metric (Eq. GOC-LBE_CFL),
    omegas (preparatory step (d)), nu (Eq. 73), zeta (Eq. 76), eta (Eq.
    magneticresistivity) with c_sm = c_s (Eq. GOC-LBE_CFL-MIE)."""
    cs2 = metric.cs2()
    if "nu" in spec and spec["nu"] is not None:
        nu = float(spec["nu"])
        tau = nu / cs2 + 0.5
    else:
        tau = float(spec.get("tau", 1.0))
        nu = cs2 * (tau - 0.5)
    tz = float(spec.get("tau_zeta", 1.0))
    zeta = cs2 * (tz - 0.5)
    of = float(spec.get("omega_free", 1.0))
    om = [of] * 9
    om[3] = 1.0 / tz
    om[4] = om[5] = 1.0 / tau
    for k, v in (spec.get("omega_set") or {}).items():   # explicit per-moment rates
        om[int(k)] = float(v)
    if spec.get("collision", "cm") == "srt":   # Appendix F: one rate, zeta = nu
        om = [1.0 / tau] * 9
        zeta = nu
    out = {"cs2": cs2, "nu": nu, "zeta": zeta, "tau": tau, "omega": om}
    mhd = spec.get("mhd")
    if mhd:
        csm2 = cs2
        if "eta" in mhd and mhd["eta"] is not None:
            taum = float(mhd["eta"]) / csm2 + 0.5
        else:
            taum = float(mhd.get("tau_m", 1.0))
        out.update(csm2=csm2, tau_m=taum, eta=csm2 * (taum - 0.5), mu_m=float(mhd.get("mu_m", 1.0)))
    return out


def build_metric(spec: dict) -> Metric:
    m1 = spec.get("map1", {"kind": "uniform"})
    if m1.get("kind") == "table":     # metric given node by node (general orthogonal grid)
        return table_metric(int(spec["nx"]), int(spec["ny"]), spec["metric"])
    if m1.get("kind") == "annulus":   # curvilinear annular sector (Sec. 8.1)
        return annulus_metric(int(spec["nx"]), int(spec["ny"]), float(m1["r_in"]), float(m1["r_out"]),
                              float(m1["sectors"]))
    walls = spec["walls"]
    per1 = walls.get("W") is None
    per2 = walls.get("S") is None
    return Metric(spec["nx"], spec["ny"], spec.get("map1", {"kind": "uniform"}),
                  spec.get("map2", {"kind": "uniform"}), per1, per2)


class Oracle:
    """One lattice advanced by the FP64 oracle."""

    def __init__(self, spec: dict, threads: int | None = None,
                 q3_printed: bool = False, metric: Metric | None = None):
        """metric: the node metric to use instead of the one built from the
        spec's maps (a slab of a larger lattice, see oracle.slab)."""
        lib = _load()
        self.spec = spec
        nx, ny = int(spec["nx"]), int(spec["ny"])
        self.nx, self.ny = nx, ny
        self.metric = m = build_metric(spec) if metric is None else metric
        self.par = par = derived_parameters(spec, m)
        walls = spec["walls"]
        wall = np.array([0 if walls.get(w) is None else 1 for w in _WALLS], dtype=np.int32)
        if wall[0] != wall[1] or wall[2] != wall[3]:
            raise ValueError("opposite walls must both be periodic or both walls")
        uwall = np.array([0.0 if walls.get(w) is None else float(walls[w].get("u", 0.0))
                          for w in _WALLS])
        bwall = np.zeros(8)
        for k, w in enumerate(_WALLS):
            if walls.get(w) is not None and walls[w].get("B") is not None:
                bwall[2 * k:2 * k + 2] = walls[w]["B"]
        wh1 = np.concatenate([m.wall[w][0] for w in _WALLS])
        wh2 = np.concatenate([m.wall[w][1] for w in _WALLS])
        fext = spec.get("fext", (0.0, 0.0))
        mhd = spec.get("mhd")
        if threads is None:
            threads = int(os.environ.get("GOC_ORACLE_THREADS", "1"))
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in
                      (m.h1, m.h2, m.t11, m.t12, m.t21, m.t22)]
        om = np.array(par["omega"], dtype=np.float64)
        self._h = lib.orc_create(
            nx, ny, *[_p(a) for a in self._keep], wall.ctypes.data_as(_I), _p(uwall),
            _p(wh1), _p(wh2), par["cs2"], par["nu"], par["zeta"], _p(om),
            float(fext[0]), float(fext[1]), int(spec.get("gi", 1)), int(q3_printed),
            1 if mhd else 0, par.get("csm2", 0.0), par.get("tau_m", 1.0), par.get("mu_m", 1.0),
            _p(bwall), int(threads))
        self._lib = lib
        coll = spec.get("collision", "cm")
        kinds = {"cm": 0, "srt": 1, "raw": 2}
        if coll not in kinds:
            raise ValueError(f"unknown collision {coll!r}")
        lib.orc_set_collision(self._h, kinds[coll])
        self.steps_done = 0
        self.initialize()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def threads(self) -> int:
        return self._lib.orc_threads(self._h)

    def initialize(self, rho=None, u1=None, u2=None, b1=None, b2=None):
        nx, ny = self.nx, self.ny
        rho0 = float(self.spec.get("rho0", 1.0))
        init = self.spec.get("init") or {}
        rho = np.full((ny, nx), rho0) if rho is None else np.asarray(rho, dtype=np.float64)
        u1 = np.asarray(init.get("u1", 0.0) if u1 is None else u1, dtype=np.float64)
        u2 = np.asarray(init.get("u2", 0.0) if u2 is None else u2, dtype=np.float64)
        u1 = np.broadcast_to(u1, (ny, nx)).copy()
        u2 = np.broadcast_to(u2, (ny, nx)).copy()
        mhd = self.spec.get("mhd") or {}
        b0 = mhd.get("B_init", (0.0, 0.0))
        b1 = np.broadcast_to(np.asarray(b0[0] if b1 is None else b1, dtype=np.float64), (ny, nx)).copy()
        b2 = np.broadcast_to(np.asarray(b0[1] if b2 is None else b2, dtype=np.float64), (ny, nx)).copy()
        rho = np.ascontiguousarray(np.broadcast_to(rho, (ny, nx)))
        self._lib.orc_init(self._h, _p(rho), _p(u1), _p(u2), _p(b1), _p(b2))
        self.steps_done = 0

    def step(self, n: int = 1):
        self._lib.orc_step(self._h, int(n))
        self.steps_done += int(n)

    def fields(self):
        """(rho, U1, U2, B1, B2) of the current state, each [ny, nx]."""
        N = (self.ny, self.nx)
        out = [np.zeros(N) for _ in range(5)]
        self._lib.orc_fields(self._h, *[_p(a) for a in out])
        return tuple(out)

    def state(self):
        N = self.nx * self.ny
        f = np.zeros(9 * N)
        F1 = np.zeros(N)
        F2 = np.zeros(N)
        g = np.zeros(10 * N)
        self._lib.orc_get_state(self._h, _p(f), _p(F1), _p(F2), _p(g))
        s = (self.ny, self.nx)
        return (f.reshape((9,) + s), F1.reshape(s), F2.reshape(s), g.reshape((2, 5) + s))

    def set_state(self, f, F1, F2, g=None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        F1 = np.ascontiguousarray(F1, dtype=np.float64)
        F2 = np.ascontiguousarray(F2, dtype=np.float64)
        gp = _p(np.ascontiguousarray(g, dtype=np.float64)) if g is not None else None
        self._lib.orc_set_state(self._h, _p(f), _p(F1), _p(F2), gp)

    def mie_diag(self):
        N = self.nx * self.ny
        J3, FL1, FL2 = np.zeros(N), np.zeros(N), np.zeros(N)
        self._lib.orc_mie_diag(self._h, _p(J3), _p(FL1), _p(FL2))
        s = (self.ny, self.nx)
        return J3.reshape(s), FL1.reshape(s), FL2.reshape(s)

    def mie_grad(self):
        """The local gradients of B of the last step (Eqs. gradB1/gradB2):
        [4, ny, nx] dB1/dxi1, dB2/dxi1, dB1/dxi2, dB2/dxi2."""
        out = np.zeros(4 * self.nx * self.ny)
        self._lib.orc_mie_grad(self._h, _p(out))
        return out.reshape(4, self.ny, self.nx)

    # ---- single-node algebra exposed for pin tests --------------------
    def frame_matrix(self, u, v):
        out = np.zeros(81)
        self._lib.orc_frame_matrix(float(u), float(v), _p(out))
        return out.reshape(9, 9)

    def p_matrices(self):
        P = np.zeros(81)
        Pi = np.zeros(81)
        self._lib.orc_p_matrix(self._h, _p(P), _p(Pi))
        return P.reshape(9, 9), Pi.reshape(9, 9)

    def central_equilibria(self, rho, u1, u2, h1, h2, n3=0.0, n4=0.0):
        out = np.zeros(9)
        self._lib.orc_central_equilibria(self._h, rho, u1, u2, h1, h2, n3, n4, _p(out))
        return out

    def raw_equilibria(self, rho, u1, u2, h1, h2, n3=0.0, n4=0.0):
        out = np.zeros(9)
        self._lib.orc_raw_equilibria(self._h, rho, u1, u2, h1, h2, n3, n4, _p(out))
        return out

    def srt_equilibria(self, rho, u1, u2, h1, h2, t11, t12, t21, t22, dU1, dU2, dr1, dr2):
        out = np.zeros(9)
        self._lib.orc_srt_equilibria(self._h, rho, u1, u2, h1, h2, t11, t12, t21, t22,
                                     dU1, dU2, dr1, dr2, _p(out))
        return out

    def srt_to_populations(self, k):
        k = np.ascontiguousarray(k, dtype=np.float64)
        out = np.zeros(9)
        self._lib.orc_srt_to_populations(_p(k), _p(out))
        return out

    def corrections(self, rho, u1, u2, h1, h2, t11, t12, t21, t22, dU1, dU2, dr1, dr2):
        out = np.zeros(2)
        self._lib.orc_corrections(self._h, rho, u1, u2, h1, h2, t11, t12, t21, t22,
                                  dU1, dU2, dr1, dr2, _p(out))
        return out
