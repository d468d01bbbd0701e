"""Python view of the C ABI: Lattice and Batch (marshalling only; every step
runs in libgoc.so's CUDA kernels)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import GocExec, GocFlow, GocGrid, GocMap, GocMhd, check, lib

_SIDES = ("W", "E", "S", "N")


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def structs_from_spec(spec: dict):
    """goc_grid, goc_map, goc_flow, goc_mhd of a lattice spec (see goc_inputs):
    nx, ny; walls {"W", "E", "S", "N"} -> None (periodic) or {"u": tangential
    speed, "B": (B1, B2)}; map1, map2 {"kind": uniform | tanh2 | sine | roberts
    | tanh1 | sinh | annulus | table, with that map's parameters}; for kind
    "table" (map1), spec["metric"] holds [ny, nx] arrays h1, h2, t11, t12, t21,
    t22 and "wall": side -> (h1, h2) along that side; rho0, nu or tau,
    tau_zeta, omega_free, fext, gi; mhd {tau_m or eta, mu_m, B_init}."""
    g = GocGrid()
    g.nx, g.ny = int(spec["nx"]), int(spec["ny"])
    walls = spec["walls"]
    for k, s in enumerate(_SIDES):
        w = walls.get(s)
        g.bc[k] = 0 if w is None else 1
        if w is not None:
            g.wall_u[k] = float(w.get("u", 0.0))
            b = w.get("B")
            if b is not None:
                g.wall_b[k][0], g.wall_b[k][1] = float(b[0]), float(b[1])
    m = GocMap()
    for ax, key in enumerate(("map1", "map2")):
        mp = spec.get(key, {"kind": "uniform"})
        m.kind[ax] = _abi.MAPS[mp.get("kind", "uniform")]
        m.beta[ax] = float(mp.get("beta", 0.0))
        m.a[ax] = float(mp.get("a", 0.0))
        m.gamma[ax] = float(mp.get("gamma", 0.0))
        m.alpha[ax] = float(mp.get("alpha", 0.5))
        m.mu[ax] = float(mp.get("mu", 0.0))
        m.yc[ax] = float(mp.get("yc", 0.5))
        if mp.get("kind") == "annulus":
            m.r_inner, m.r_outer, m.sectors = float(mp["r_in"]), float(mp["r_out"]), float(mp["sectors"])
        if mp.get("kind") == "table" and ax == 0:   # general grid: spec["metric"] as in oracle.metric.table_metric
            t = spec["metric"]
            tab = np.ascontiguousarray(np.stack([np.asarray(t[k], dtype=np.float64).reshape(g.ny, g.nx)
                                                 for k in ("h1", "h2", "t11", "t12", "t21", "t22")]))
            wall = t["wall"]   # side -> (h1, h2) at the wall points
            wt = np.ascontiguousarray(np.concatenate(
                [np.asarray(wall[w][k], dtype=np.float64)
                 for w, k in (("W", 0), ("E", 0), ("S", 1), ("N", 1),     # wall-normal factor
                              ("W", 1), ("E", 1), ("S", 0), ("N", 0))]))  # tangential factor
            m.table = tab.ctypes.data
            m.wall_table = wt.ctypes.data
            m._keep = (tab, wt)   # alive as long as the struct
    f = GocFlow()
    f.rho0 = float(spec.get("rho0", 1.0))
    f.tau = float(spec.get("tau", 1.0)) if spec.get("tau") is not None else 1.0
    f.nu = float(spec["nu"]) if spec.get("nu") is not None else 0.0
    f.tau_zeta = float(spec.get("tau_zeta", 1.0))
    f.omega_free = float(spec.get("omega_free", 1.0))
    fe = spec.get("fext", (0.0, 0.0))
    f.fext[0], f.fext[1] = float(fe[0]), float(fe[1])
    f.gi_correction = int(spec.get("gi", 1))
    h = GocMhd()
    mhd = spec.get("mhd")
    if mhd:
        h.enabled = 1
        h.tau_m = float(mhd.get("tau_m", 1.0))
        h.eta = float(mhd["eta"]) if mhd.get("eta") is not None else 0.0
        h.mu_m = float(mhd.get("mu_m", 1.0))
        b = mhd.get("B_init", (0.0, 0.0))
        h.b_init[0], h.b_init[1] = float(b[0]), float(b[1])
    return g, m, f, h


def metric_info(spec: dict):
    """(q, cs^2) computed by the library's FP64 metric kernel."""
    g, m, _, _ = structs_from_spec(spec)
    q, cs2 = ctypes.c_double(), ctypes.c_double()
    check(lib().goc_metric_info(ctypes.byref(g), ctypes.byref(m), ctypes.byref(q), ctypes.byref(cs2)))
    return q.value, cs2.value


ROUNDING = {"stochastic": 0, "nearest": 1}
SCHEMES = {"goc": 0, "standard": 1, "goc_srt": 2, "goc_raw": 3}


STREAMING = {"two_buffers": 0, "in_place": 1}


def _exec(storage: str, stream, check_every: int, rounding: str = "stochastic", scheme: str = "goc",
          fixed_launch: bool = False, plateau_checks: int = 0, reference_every: int = 0,
          streaming: str = "two_buffers") -> GocExec:
    e = GocExec()
    e.storage = _abi.STORAGE[storage]
    e.cuda_stream = ctypes.c_void_p(int(stream)) if stream else None
    e.device = -1
    e.check_every = int(check_every)
    e.rounding = ROUNDING[rounding]
    e.scheme = SCHEMES[scheme]
    e.fixed_launch = 1 if fixed_launch else 0
    e.plateau_checks = int(plateau_checks)
    e.reference_every = int(reference_every)
    e.streaming = STREAMING[streaming]
    return e


class Lattice:
    """One lattice owned by libgoc."""

    def __init__(self, spec: dict, storage: str = "fp32", stream=None, check_every: int = 100,
                 rounding: str = "stochastic", scheme: str = "goc", fixed_launch: bool = False,
                 plateau_checks: int = 0, reference_every: int = 0, streaming: str = "two_buffers",
                 _handle=None, _owner=None):
        """scheme "standard": the uniform-grid central-moment LBM comparator
        (uniform maps, spec["gi"] = 0, no MIE).  reference_every: steps between
        refreshes of the per-row storage reference of 16-bit storage on
        straight grids (0: the library default, < 0: never).  streaming
        "in_place": one population buffer updated in place (straight grids;
        goc_exec.streaming)."""
        self.spec = spec
        self.nx, self.ny = int(spec["nx"]), int(spec["ny"])
        self.storage = storage
        self._owner = _owner
        if _handle is not None:
            self._h = _handle
        else:
            g, m, f, h = structs_from_spec(spec)
            e = _exec(storage, stream, check_every, rounding, scheme, fixed_launch, plateau_checks, reference_every,
                      streaming)
            out = ctypes.c_void_p()
            check(lib().goc_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(f),
                                   ctypes.byref(h), ctypes.byref(e), ctypes.byref(out)))
            self._h = out
        init = spec.get("init")
        if init and _handle is None:
            self.init_fields(u1=init.get("u1"), u2=init.get("u2"), rho=init.get("rho"))

    @classmethod
    def from_problem(cls, problem, storage: str = "fp32", **kw) -> "Lattice":
        spec0 = problem.lattice_spec(1.0)
        _, cs2 = metric_info(spec0)
        return cls(problem.lattice_spec(cs2), storage=storage, **kw)

    def close(self):
        if getattr(self, "_h", None) and self._owner is None:
            lib().goc_destroy(self._h)
        self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _field(self, a):
        if a is None:
            return None
        return np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (self.ny, self.nx)))

    def init_fields(self, rho=None, u1=None, u2=None, b1=None, b2=None):
        arrs = [self._field(x) for x in (rho, u1, u2, b1, b2)]
        check(lib().goc_init_fields(self._h, *[_dptr(a) for a in arrs]))

    def step(self, n: int = 1):
        check(lib().goc_step(self._h, int(n)))

    def sync(self):
        check(lib().goc_sync(self._h))

    def run_until(self, tol: float, max_steps: int):
        done, res = ctypes.c_longlong(), ctypes.c_double()
        check(lib().goc_run_until(self._h, float(tol), int(max_steps), ctypes.byref(done), ctypes.byref(res)))
        return done.value, res.value

    def moments(self, cartesian: bool = False, out=None):
        """(rho, U1, U2, B1, B2) as [ny, nx] float64 arrays.  out: five
        C-contiguous float64 arrays (or None entries to skip a field) to fill
        instead of new ones, e.g. page-locked buffers."""
        if out is None:
            out = [np.zeros((self.ny, self.nx)) for _ in range(5)]
        for a in out:
            if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous or a.size != self.nx * self.ny):
                raise ValueError("out arrays must be C-contiguous float64 of nx * ny elements")
        check(lib().goc_moments(self._h, int(cartesian), *[_dptr(a) for a in out]))
        return tuple(out)

    def moments_device(self, out_ptr: int):
        check(lib().goc_moments_device(self._h, ctypes.c_void_p(out_ptr)))

    def mass(self) -> float:
        m = ctypes.c_double()
        check(lib().goc_diagnostics(self._h, ctypes.byref(m), None, None))
        return m.value

    def residuals(self):
        ru, rb = ctypes.c_double(), ctypes.c_double()
        check(lib().goc_diagnostics(self._h, None, ctypes.byref(ru), ctypes.byref(rb)))
        return ru.value, rb.value

    @property
    def steps_done(self) -> int:
        return int(lib().goc_steps_done(self._h))

    def footprint(self):
        n, b = ctypes.c_longlong(), ctypes.c_longlong()
        check(lib().goc_footprint(self._h, ctypes.byref(n), ctypes.byref(b)))
        return n.value, b.value

    @property
    def launch_config(self) -> dict:
        d, p, t, b, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().goc_launch_config(self._h, ctypes.byref(d), ctypes.byref(p), ctypes.byref(t)))
        check(lib().goc_launch_grid(self._h, ctypes.byref(b)))
        check(lib().goc_tile_height(self._h, ctypes.byref(r)))
        return {"dynamic_tiles": bool(d.value), "pdl": bool(p.value), "balanced_grid": bool(b.value),
                "tile_rows": r.value, "tuned": bool(t.value)}

    def set_launch_config(self, dynamic_tiles: bool, pdl: bool, balanced_grid: bool = False, tile_rows: int = 8):
        """Fix the launch settings (and turn the autotuner off); tile_rows 16
        is for straight grids with the central-moment collision."""
        check(lib().goc_set_launch_config(self._h, int(dynamic_tiles), int(pdl)))
        check(lib().goc_set_launch_grid(self._h, int(balanced_grid)))
        check(lib().goc_set_tile_height(self._h, int(tile_rows)))

    @property
    def bytes_per_node(self) -> float:
        return float(lib().goc_bytes_per_node(self._h))

    def get_state(self) -> bytes:
        n = ctypes.c_size_t()
        check(lib().goc_get_state(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        check(lib().goc_get_state(self._h, buf, ctypes.byref(n)))
        return buf.raw

    def set_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        check(lib().goc_set_state(self._h, buf, len(data)))


def _vp(ptr):
    return ctypes.c_void_p(int(ptr)) if ptr else None


class Slab(Lattice):
    """The slab of the global rows [row_begin, row_end) of the lattice
    `spec` (goc_create_slab): a Lattice over its local rows -- ghost rows,
    owned rows, ghost rows -- whose ghost rows are refreshed from the
    neighbouring slabs after creation and after every step (pack, exchange,
    unpack; see paper_2607_15362_b300.slab)."""

    def __init__(self, spec: dict, row_begin: int, row_end: int, storage: str = "fp32", stream=None,
                 rounding: str = "stochastic", scheme: str = "goc", reference_every: int = 0):
        g, m, f, h = structs_from_spec(spec)
        e = _exec(storage, stream, 100, rounding, scheme, True, 0, reference_every)
        out = ctypes.c_void_p()
        check(lib().goc_create_slab(ctypes.byref(g), ctypes.byref(m), ctypes.byref(f), ctypes.byref(h),
                                    ctypes.byref(e), int(row_begin), int(row_end), ctypes.byref(out)))
        r0, r1, lo, hi = (ctypes.c_int() for _ in range(4))
        check(lib().goc_slab_info(out, ctypes.byref(r0), ctypes.byref(r1), ctypes.byref(lo), ctypes.byref(hi)))
        self.row_begin, self.row_end, self.ghost_lo, self.ghost_hi = r0.value, r1.value, lo.value, hi.value
        self.global_ny = int(spec["ny"])
        local = dict(spec, ny=self.row_end - self.row_begin + self.ghost_lo + self.ghost_hi)
        local.pop("init", None)
        super().__init__(local, storage=storage, _handle=out)
        self.global_spec = spec
        # global row of every local row (ghost rows of a periodic axis wrap)
        self.rows = (np.arange(self.ny) + self.row_begin - self.ghost_lo) % self.global_ny
        self.halo_bytes = int(lib().goc_slab_halo_bytes(out))
        init = spec.get("init")
        if init:
            self.init_fields(**{k: np.asarray(v)[self.rows] for k, v in init.items() if v is not None})

    @property
    def own(self) -> slice:
        """Local rows owned by this slab."""
        return slice(self.ghost_lo, self.ghost_lo + self.row_end - self.row_begin)

    def owned_moments(self, cartesian: bool = False):
        """(rho, U1, U2, B1, B2) of the owned rows."""
        return tuple(a[self.own] for a in self.moments(cartesian))

    def pack(self, send_lo, send_hi):
        """Rows nearest each cut into device buffers (addresses; None skips)."""
        check(lib().goc_slab_pack(self._h, _vp(send_lo), _vp(send_hi)))

    def unpack(self, recv_lo, recv_hi):
        """Ghost rows from the neighbours' messages (device addresses; None skips)."""
        check(lib().goc_slab_unpack(self._h, _vp(recv_lo), _vp(recv_hi)))


class Batch:
    """Many independent lattices advanced together (one persistent launch
    per time step, captured in CUDA graphs)."""

    def __init__(self, hbm_budget_bytes: int, max_lattices: int, storage: str = "fp32", stream=None,
                 rounding: str = "stochastic", reference_every: int = 0):
        e = _exec(storage, stream, 100, rounding, reference_every=reference_every)
        out = ctypes.c_void_p()
        check(lib().goc_batch_create(int(hbm_budget_bytes), int(max_lattices), ctypes.byref(e), ctypes.byref(out)))
        self._h = out
        self.storage = storage
        self.specs = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().goc_batch_destroy(self._h)
        self._h = None

    __del__ = close

    def add(self, spec: dict, storage: str | None = None) -> int:
        g, m, f, h = structs_from_spec(spec)
        slot = ctypes.c_int()
        check(lib().goc_batch_add(self._h, ctypes.byref(g), ctypes.byref(m), ctypes.byref(f), ctypes.byref(h),
                                  _abi.STORAGE[storage or self.storage], ctypes.byref(slot)))
        self.specs[slot.value] = spec
        init = spec.get("init")
        if init:
            self.lattice(slot.value).init_fields(u1=init.get("u1"), u2=init.get("u2"), rho=init.get("rho"))
        return slot.value

    def try_add(self, spec: dict, storage: str | None = None):
        """Slot id, or None when the batch is full or out of HBM budget."""
        try:
            return self.add(spec, storage)
        except _abi.GocError as e:
            if e.status == _abi.GOC_EBUSY:
                return None
            raise

    def remove(self, slot: int):
        check(lib().goc_batch_remove(self._h, int(slot)))
        self.specs.pop(slot, None)

    def step(self, n: int = 1):
        check(lib().goc_batch_step(self._h, int(n)))

    def check(self, slot: int, on: bool = True):
        """Record the residual of this slot at the end of every batch step."""
        check(lib().goc_batch_check(self._h, int(slot), int(bool(on))))

    def residual(self, slot: int):
        ru, rb = ctypes.c_double(), ctypes.c_double()
        check(lib().goc_batch_residual(self._h, int(slot), ctypes.byref(ru), ctypes.byref(rb)))
        return ru.value, rb.value

    def lattice(self, slot: int) -> Lattice:
        out = ctypes.c_void_p()
        check(lib().goc_batch_lattice(self._h, int(slot), ctypes.byref(out)))
        return Lattice(self.specs[slot], storage=self.storage, _handle=out, _owner=self)

    def usage(self):
        u, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
        check(lib().goc_batch_usage(self._h, ctypes.byref(u), ctypes.byref(b), ctypes.byref(c)))
        return u.value, b.value, c.value
