"""Continuous-batching request loop over the batched executor (libgoc).

Requests (a goc_inputs.Problem plus a step budget or a residual tolerance)
arrive over time.  The loop admits waiting requests, first come first
served, while the batch's HBM budget and slot count allow (goc_batch_add
reports GOC_EBUSY otherwise), advances every resident lattice together with
goc_batch_step (one persistent launch per time step under CUDA graphs), and
retires lattices whose budget is spent or whose residual (Sec. 7.3: 2-norm of
successive velocity fields, max with the field residual for MHD) fell below
the tolerance; retired slots free their memory for the next admissions.

Chunks end exactly at the next budget boundary of any resident request, so a
budget request runs exactly its budget and its result does not depend on
what else shares the batch.  Residual requests are tested at the end of
every chunk of at least two steps.

All numerical work happens in libgoc's kernels; this module only schedules.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from ._abi import GOC_EDIVERGED, GocError
from .lattice import Batch, Lattice, metric_info


@dataclass
class Request:
    rid: int
    arrival_s: float
    problem: object            # goc_inputs.Problem
    budget: int                # step budget (cap when tol is set)
    tol: float | None = None   # residual tolerance, or None for a pure budget
    storage: str = "fp32"


@dataclass
class Result:
    rid: int
    arrival_s: float
    admitted_s: float
    finished_s: float
    steps: int
    nodes: int
    residual: float | None
    status: str
    fields: tuple | None = None

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


def lattice_spec(problem) -> dict:
    """Lattice-unit spec of a problem with c_s^2 from the library's metric."""
    _, cs2 = metric_info(problem.lattice_spec(1.0))
    return problem.lattice_spec(cs2)


def summarize(results: list[Result], wall_s: float) -> dict:
    lat = np.array([r.latency_s for r in results if r.status == "done"])
    work = sum(r.nodes * r.steps for r in results)
    return {
        "requests": len(results),
        "done": int(sum(r.status == "done" for r in results)),
        "diverged": int(sum(r.status == "diverged" for r in results)),
        "cancelled": int(sum(r.status == "cancelled" for r in results)),
        "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
        "aggregate_mlups": work / wall_s / 1e6 if wall_s > 0 else None,
        "node_updates": int(work),
        "wall_s": wall_s,
    }


class Server:
    def __init__(self, hbm_budget_bytes: int, max_slots: int = 128, chunk: int = 500,
                 storage: str = "fp32", keep_fields: bool = False, stream=None, batch=None, spec_fn=None):
        self.batch = batch if batch is not None else Batch(hbm_budget_bytes, max_slots, storage=storage, stream=stream)
        self.spec_fn = spec_fn or lattice_spec
        self.chunk = int(chunk)
        self.keep_fields = keep_fields
        self._cancelled: set[int] = set()

    def cancel(self, rid: int):
        """Withdraw request rid: if it waits it is dropped, if it runs it is
        evicted at the next chunk boundary; either way it is reported as
        "cancelled".  Safe to call from another thread while run() serves."""
        self._cancelled.add(rid)

    def close(self):
        self.batch.close()

    def run(self, requests: list[Request], time_scale: float = 1.0, max_wall_s: float | None = None):
        """Serve requests arriving at arrival_s * time_scale seconds after the
        start; returns (results, summary)."""
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting: collections.deque = collections.deque()
        active: dict[int, dict] = {}
        results: list[Result] = []
        specs: dict[int, dict] = {}
        while pending or waiting or active:
            if max_wall_s is not None and now() > max_wall_s:
                break
            t = now()
            while pending and pending[0].arrival_s * time_scale <= t:
                waiting.append(pending.popleft())
            for r in [r for r in waiting if r.rid in self._cancelled]:   # withdrawn before admission
                waiting.remove(r)
                results.append(Result(r.rid, r.arrival_s * time_scale, float("nan"), now(), 0,
                                      r.problem.nodes, None, "cancelled"))
            for slot in [s_ for s_, a in active.items() if a["req"].rid in self._cancelled]:   # evicted
                a = active.pop(slot)
                r = a["req"]
                results.append(Result(r.rid, r.arrival_s * time_scale, a["admitted"], now(), a["steps"],
                                      r.problem.nodes, a["residual"], "cancelled"))
                self.batch.remove(slot)
            while waiting:                                   # first come, first served
                r = waiting[0]
                spec = specs.get(r.rid) or self.spec_fn(r.problem)
                specs[r.rid] = spec
                slot = self.batch.try_add(spec, r.storage)
                if slot is None:
                    break
                if r.tol is not None:
                    self.batch.check(slot)
                active[slot] = {"req": r, "admitted": now(), "steps": 0, "residual": None}
                waiting.popleft()
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival_s * time_scale - now())))
                continue
            k = self.chunk
            for a in active.values():
                k = min(k, a["req"].budget - a["steps"])
            k = max(1, k)
            self.batch.step(k)
            done = []
            for slot, a in active.items():
                a["steps"] += k
                r = a["req"]
                status = None
                if r.tol is not None and k >= 2:
                    try:
                        ru, rb = self.batch.residual(slot)
                        a["residual"] = max(ru, rb)
                        if a["residual"] < r.tol:
                            status = "done"
                    except Exception:
                        status = "diverged"
                if status is None and a["steps"] >= r.budget:
                    status = "done"
                if status:
                    done.append((slot, status))
            for slot, status in done:
                a = active.pop(slot)
                r = a["req"]
                fields = None
                try:   # a lattice that diverged is reported as such and evicted; the others go on
                    fields = self.batch.lattice(slot).moments() if self.keep_fields else None
                    if not self.keep_fields:
                        self.batch.lattice(slot).sync()
                except GocError as e:
                    if e.status != GOC_EDIVERGED:
                        raise
                    status, fields = "diverged", None
                results.append(Result(r.rid, r.arrival_s * time_scale, a["admitted"], now(), a["steps"],
                                      r.problem.nodes, a["residual"], status, fields))
                self.batch.remove(slot)
        wall = now()
        for r in list(waiting) + list(pending):
            results.append(Result(r.rid, r.arrival_s * time_scale, float("nan"), float("nan"), 0,
                                  r.problem.nodes, None, "not_admitted"))
        for a in active.values():
            r = a["req"]
            results.append(Result(r.rid, r.arrival_s * time_scale, a["admitted"], float("nan"), a["steps"],
                                  r.problem.nodes, a["residual"], "unfinished"))
        return results, summarize(results, wall)


def run_sequential(requests: list[Request], time_scale: float = 1.0, keep_fields: bool = False,
                   max_wall_s: float | None = None, check_every: int = 500, stream=None):
    """Baseline: one lattice at a time, in arrival order, each with its own
    launches (goc_step / goc_run_until)."""
    t0 = time.perf_counter()
    results = []
    for r in sorted(requests, key=lambda r: r.arrival_s):
        if max_wall_s is not None and time.perf_counter() - t0 > max_wall_s:
            results.append(Result(r.rid, r.arrival_s * time_scale, float("nan"), float("nan"), 0,
                                  r.problem.nodes, None, "not_admitted"))
            continue
        wait = r.arrival_s * time_scale - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        admitted = time.perf_counter() - t0
        lat = Lattice(lattice_spec(r.problem), storage=r.storage, check_every=check_every, stream=stream)
        residual, status, fields, steps = None, "done", None, r.budget
        try:
            if r.tol is None:
                lat.step(r.budget)
            else:
                steps, residual = lat.run_until(r.tol, r.budget)
            fields = lat.moments() if keep_fields else None
            lat.sync()
        except GocError as e:
            if e.status != GOC_EDIVERGED:
                raise
            status, fields = "diverged", None
        results.append(Result(r.rid, r.arrival_s * time_scale, admitted, time.perf_counter() - t0, steps,
                              r.problem.nodes, residual, status, fields))
        lat.close()
    return results, summarize(results, time.perf_counter() - t0)


def requests_from_trace(trace: list[dict], storage: str = "fp32") -> list[Request]:
    """Requests from goc_inputs.serving_trace entries."""
    return [Request(k, t["arrival_s"], t["problem"], int(t["budget"]), t["tol"], storage)
            for k, t in enumerate(trace)]
