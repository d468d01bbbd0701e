"""Benchmark of the GOC-LBM hot path (prints one JSON line).

Default workload: the lid-driven cavity of 512 x 512 nodes, tanh clustering
(beta = 2) toward all four walls, Re = 1000, lid velocity 0.05, D2Q9
central-moment MRT, FP32 storage.  One benchmark step is one solve chunk of
1000 fused time steps (graph-replayed launches of the step kernel) on data
resident in HBM; 20 chunks are the full 20000-step job.  Between timed steps
L2 is flushed by writing a 256 MiB buffer (the 23 MB lattice itself fits in
the 126 MB L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--storage fp32|fp16|bf16] [--chunk T]

Under torchrun every rank runs an independent replica (a single lattice is
not sharded); value is the sum over ranks, timed as the maximum over ranks.
--impl reference times the FP64 CPU oracle (the method as written) on this
host on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import goc_inputs as gi  # noqa: E402

METRIC = "MLUPS & % of HBM peak (FP32 vs FP16 store); batched p50/p99 solve latency"
PROFILE = os.path.join(ROOT, "profiles", "lean_step_kernel_cavity512_fp32.txt")
PROFILE_SPIRAL = os.path.join(ROOT, "profiles", "step_kernel_spiral512_fp32_table.txt")
KERNEL_SOURCES = ["paper_2607_15362_b300/csrc/goc_step.cuh", "paper_2607_15362_b300/csrc/goc_device.cuh",
                  "paper_2607_15362_b300/csrc/goc_vec.cuh", "paper_2607_15362_b300/csrc/goc_lean.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def step_kernel_name(storage: str, mie: bool, scheme: str, geom: int, tile_rows: int = 8) -> str:
    """The step kernel a lattice runs: straight grids with the central-moment
    collision run lean_step_kernel (lean2_step_kernel with 16-row tiles), the
    others step_kernel."""
    s = {"fp32": "float", "fp16": "__half", "bf16": "__nv_bfloat16"}[storage]
    if geom == 0 and scheme == "goc":
        return "goc::{}<{},{}>".format("lean2_step_kernel" if tile_rows == 16 else "lean_step_kernel", s, int(mie))
    return "goc::step_kernel<{},{},{},{}>".format(s, int(mie), int(scheme != "goc"), geom)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0}, "fallback"


def _profile_value(key: str, path: str = PROFILE):
    """A number from a committed ncu summary of the step kernel, if it was
    taken on the current kernel source."""
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = dict(line.split("=", 1) for line in txt.splitlines() if "=" in line and not line.startswith("#"))
    if vals.get("kernel_source_hash", "").strip() != kernel_hash():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def profile_traffic(path: str = PROFILE):
    """DRAM bytes per launch of the step kernel (ncu)."""
    return _profile_value("dram_bytes_per_launch", path)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def setup_dist(backend: str = "nccl"):
    """Ranks from the torchrun environment; a process group when there are
    several (NCCL on the GPUs; the host-side tests use gloo)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend, init_method="env://")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x: float, device: str = "cuda") -> float:
    """Maximum of x over the ranks (the job's time is the slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, ms_max: float) -> float:
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the slowest rank's time (units per second / 1e6)."""
    return world * units_per_rank / (ms_max * 1e-3) / 1e6


def _problem(args):
    """The workload of the main bench line: the clustered cavity (the
    benchmark), the cavity on a logarithmic-spiral node table, or
    Taylor-Couette flow in an annular sector (radius ratio 2, h2 = h1 at
    mid-radius)."""
    n = args.cavity_n
    if args.grid == "spiral":
        return gi.spiral_cavity(n, n, Re=args.cavity_re, u_lid=0.05, mach_matched=True)
    if args.grid == "annulus":
        return gi.taylor_couette(n1=n, n2=n, r_in=float(n), sectors=2 * math.pi / math.log(2.0), Re=200.0,
                                 u_in=1.0, u_out=1.5)
    return gi.lid_cavity(n=n, Re=args.cavity_re)


def _spec(args, prob, cs2):
    """Lattice spec of the workload for a given c_s^2 (the MIE and collision
    options included, in the form both the library binding and the oracle
    read)."""
    spec = prob.lattice_spec(cs2)
    if args.mie:   # the coupled MIE with an initial uniform field
        spec["mhd"] = {"tau_m": 0.9, "mu_m": 2.0, "B_init": (0.01, 0.004)}
    if args.scheme != "goc":
        spec["collision"] = {"goc_srt": "srt", "goc_raw": "raw"}[args.scheme]
    return spec


def run_ours(args):
    import numpy as np
    import torch

    import paper_2607_15362_b300 as goc

    world, rank, local = setup_dist()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    spiral, annulus = args.grid == "spiral", args.grid == "annulus"
    prob = _problem(args)
    _, cs2 = goc.metric_info(prob.lattice_spec(1.0))
    spec = _spec(args, prob, cs2)
    geom = 2 if spiral else 1 if annulus else 0
    in_place = args.streaming == "in_place"
    lat = goc.Lattice(spec, storage=args.storage, stream=stream.cuda_stream, scheme=args.scheme,
                      streaming=args.streaming)
    nodes = prob.nodes
    chunk = args.chunk
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def one_step():
        lat.step(chunk)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # ---- device-resident timed region ----------------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xff)          # L2 flush between timed steps (not timed)
            ev[k][0].record(stream)
            one_step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier(world)
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    ms_total = allmax(world, sum(ms_steps))
    ms_per_step = ms_total / args.steps
    mlups = job_rate(world, nodes * chunk * args.steps, ms_total)

    # ---- end to end through the C ABI with host buffers -------------------
    e2e = None
    h2d = d2h = 3 * nodes * 8   # rho, U1, U2 in FP64 each way
    if not args.no_e2e:
        def pinned(fill):
            t = torch.full((prob.ny, prob.nx), fill, dtype=torch.float64).pin_memory()
            return t, t.numpy()
        keep = [pinned(v) for v in (1.0, 0.0, 0.0, 0.0, 0.0, 0.0)]   # inputs rho, U1, U2; outputs rho, U1, U2
        rho_in, u1_in, u2_in, rho_out, u1_out, u2_out = [a for _, a in keep]
        barrier(world)
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for k in range(args.steps):
            lat.init_fields(rho=rho_in, u1=u1_in, u2=u2_in)   # H2D of the step's input fields (page-locked)
            one_step()
            lat.moments(out=[rho_out, u1_out, u2_out, None, None])   # D2H of the result fields (page-locked)
        torch.cuda.synchronize()
        e_wall = allmax(world, time.perf_counter() - e0)
        e2e = world * nodes * chunk * args.steps / e_wall / 1e6
        del keep

    # ---- roofline of the step kernel ----------------------------------------
    peaks, src = measured_peaks()
    bpn = lat.bytes_per_node
    launch_s = ms_per_step * 1e-3 / chunk
    achieved = bpn * nodes / launch_s / 1e9
    peak = float(peaks.get("hbm_gbs", 6400.0))
    prof = PROFILE_SPIRAL if spiral else PROFILE
    # the captures are of FP32 512^2 launches of the central-moment NSE step on the two cavity grids
    captured = (args.cavity_n == 512 and args.storage == "fp32" and not annulus and not args.mie
                and args.scheme == "goc" and not in_place)
    traffic = profile_traffic(prof) if captured else None
    clocks = clk.summary()
    # instruction-issue view of the same kernel: warp instructions per node
    # (ncu, current source) x node updates per second against one warp
    # instruction per scheduler per cycle at the SM clock seen under load
    issue = None
    ipn = _profile_value("warp_instructions_per_node", prof) if captured else None
    if ipn and clocks and clocks.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        ach = ipn * nodes / launch_s
        pk = sms * 4 * clocks["sm_mhz"] * 1e6
        issue = {"achieved": float(f"{ach:.4g}"), "peak": float(f"{pk:.4g}"), "unit": "warp instructions/s",
                 "frac": round(ach / pk, 4), "warp_instructions_per_node": ipn,
                 "peak_source": f"{sms} SMs x 4 schedulers x 1 warp instruction per cycle at {clocks['sm_mhz']:.0f} MHz"}

    # ---- CPU baseline: the FP64 oracle on this host (rank 0 only) ----------
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(prob, spec, budget_s=args.cpu_seconds)
    extras = None
    headline = (args.cavity_n == 512 and args.grid == "tanh" and args.storage == "fp32" and not args.mie
                and args.scheme == "goc" and not in_place)
    if rank == 0 and world == 1 and headline and not args.no_extras:
        extras = extra_numbers(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "fp32" else f"f32 arithmetic, {args.storage} storage",
            "data": ("synthetic (Taylor-Couette flow from rest)" if annulus
                     else "synthetic (lid-driven cavity from rest, seeded parameters)"),
            "config": {"workload": prob.name + f"_{args.storage}", "nodes": nodes,
                       "lb_steps_per_bench_step": chunk,
                       "map": ("logarithmic spiral given node by node (every theta_ij non-zero)" if spiral
                               else "annular sector, radius ratio 2 (Sec. 8.1)" if annulus
                               else "tanh beta=2 on both axes"),
                       "Re": 200.0 if annulus else args.cavity_re,
                       "u_lid": None if annulus else round(spec["walls"]["N"]["u"], 6),
                       "lid_mach": None if annulus else 0.087,
                       "mie": bool(args.mie), "collision": args.scheme,
                       "storage": args.storage,
                       "streaming": args.streaming,
                       "parallelism": f"replicas x{world}" if world > 1 else "single lattice",
                       "l2": f"flushed between timed steps (256 MiB write); lattice ({nodes * bpn / 1e6:.0f} MB) "
                             + ("is L2-resident within a step" if nodes * bpn < 100e6 else "exceeds L2")},
            "e2e": ({"value": round(e2e, 1), "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
                    if e2e is not None else None),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_source": src, "bytes_per_node": bpn,
                         "kernel": ("goc::aa_fields_kernel + goc::aa_collide_kernel (in place)" if in_place
                                    else step_kernel_name(args.storage, bool(args.mie), args.scheme, geom,
                                                          lat.launch_config.get("tile_rows", 8))),
                         "launch_us": round(launch_s * 1e6, 3),
                         "launch_config": lat.launch_config, "issue": issue},
            "cpu_baseline": cpu,
            "extras": extras,
            "gpu_launches": args.steps * chunk * (2 if in_place else 1),
            "clocks": clocks,
            "wall_s": round(wall, 3),
        }
        print(json.dumps(line))
    lat.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_sharded(args):
    """One lattice cut into slabs along xi2, one per rank and GPU
    (goc_create_slab), with one ghost-row exchange per LB step over NCCL
    (paper_2607_15362_b300.slab.Halo): the clustered cavity n x (n * ranks),
    so that every GPU holds an n x n slab (weak scaling)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2607_15362_b300 as goc
    from paper_2607_15362_b300.slab import Halo, rows_of

    world, rank, local = setup_dist()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    n = args.cavity_n
    prob = gi.Problem("cavity", n, n * world, {"kind": "tanh2", "beta": 2.0}, {"kind": "tanh2", "beta": 2.0},
                      {"Re": args.cavity_re, "u_lid": 0.05, "mach_matched": True},
                      name=f"lid_cavity_{n}x{n * world}_in_{world}_slabs")
    _, cs2 = goc.metric_info(prob.lattice_spec(1.0))
    spec = _spec(args, prob, cs2)
    r0, r1 = rows_of(rank, world, prob.ny)
    slab = goc.Slab(spec, r0, r1, storage=args.storage, stream=stream.cuda_stream)
    halo = Halo(slab, rank, world, False, f"cuda:{local}")
    halo.exchange(dist)
    chunk = args.chunk
    own_nodes = prob.nx * (r1 - r0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def one_step():
        for _ in range(chunk):
            slab.step(1)
            halo.exchange(dist)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            ev[k][0].record(stream)
            one_step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier(world)
    ms_total = allmax(world, sum(a.elapsed_time(b) for a, b in ev))
    ms_per_step = ms_total / args.steps
    mlups = job_rate(world, own_nodes * chunk * args.steps, ms_total)
    e2e = None
    nloc = slab.nx * slab.ny
    h2d = d2h = 3 * nloc * 8
    if not args.no_e2e:
        keep = [torch.full((slab.ny, slab.nx), v, dtype=torch.float64).pin_memory() for v in (1.0, 0, 0, 0, 0, 0)]
        rho_in, u1_in, u2_in, rho_out, u1_out, u2_out = [t.numpy() for t in keep]
        barrier(world)
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for _ in range(args.steps):
            slab.init_fields(rho=rho_in, u1=u1_in, u2=u2_in)
            halo.exchange(dist)
            one_step()
            slab.moments(out=[rho_out, u1_out, u2_out, None, None])
        torch.cuda.synchronize()
        e_wall = allmax(world, time.perf_counter() - e0)
        e2e = world * own_nodes * chunk * args.steps / e_wall / 1e6
        del keep
    peaks, src = measured_peaks()
    bpn = slab.bytes_per_node
    launch_s = ms_per_step * 1e-3 / chunk
    achieved = bpn * own_nodes / launch_s / 1e9
    peak = float(peaks.get("hbm_gbs", 6400.0))
    # launches per LB step: the step kernel, then per side with a neighbour the
    # pack and unpack kernels (plus the storage-reference rows and tables of
    # 16-bit storage)
    sides = (1 if r0 > 0 else 0) + (1 if r1 < prob.ny else 0)
    per_step = 1 + 2 * sides + (2 * sides + 1 if args.storage != "fp32" else 0)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "fp32" else f"f32 arithmetic, {args.storage} storage",
            "data": "synthetic (lid-driven cavity from rest, seeded parameters)",
            "config": {"workload": prob.name + f"_{args.storage}", "nodes": prob.nodes,
                       "nodes_per_gpu": own_nodes, "lb_steps_per_bench_step": chunk,
                       "map": "tanh beta=2 on both axes", "Re": args.cavity_re,
                       "u_lid": round(spec["walls"]["N"]["u"], 6), "storage": args.storage,
                       "parallelism": f"slabs along xi2 x{world}, one ghost-row exchange per LB step (NCCL)",
                       "l2": "flushed between timed steps (256 MiB write)"},
            "e2e": ({"value": round(e2e, 1), "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
                    if e2e is not None else None),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "peak_source": src,
                         "bytes_per_node": bpn, "kernel": "goc::step_kernel<float,0,0,0> (per slab)",
                         "launch_us": round(launch_s * 1e6, 3)},
            "cpu_baseline": None,
            "gpu_launches": args.steps * chunk * per_step,
            "clocks": clk.summary(),
            "wall_s": round(wall, 3),
        }
        print(json.dumps(line))
    slab.close()
    if world > 1:
        dist.destroy_process_group()


def batch_numbers(steps: int, storage16: str = "fp16") -> dict:
    """64 lattices (seed 7) advanced together by the persistent batched
    kernel (FP32 and 16-bit storage) vs one lattice at a time with its own
    launches (FP32): aggregate MLUPS of each."""
    import torch

    import paper_2607_15362_b300 as goc
    from paper_2607_15362_b300.serve import lattice_spec

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    probs = gi.batch_lattices(steps=steps)
    specs = [lattice_spec(p) for p in probs]
    nodes = sum(p.nodes for p in probs)
    out = {"lattices": len(probs), "nodes": nodes, "steps_each": steps}
    for storage in ("fp32", storage16):
        b = goc.Batch(200 << 30, len(probs), storage=storage, stream=stream.cuda_stream)
        for sp in specs:
            b.add(sp)
        b.step(64)                                   # warm-up: rebuild, graph capture
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[f"batched_{storage}_mlups"] = round(nodes * steps / ms / 1e3, 1)
        used, _, _ = b.usage()
        out[f"batched_{storage}_device_gb"] = round(used / 1e9, 3)
        b.close()
    total_ms = 0.0   # sequential: each lattice alone, same number of steps
    for sp in specs:
        lat = goc.Lattice(sp, stream=stream.cuda_stream)
        lat.step(64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        lat.close()
    out["sequential_fp32_mlups"] = round(nodes * steps / total_ms / 1e3, 1)
    out["speedup_batched_vs_sequential"] = round(out["batched_fp32_mlups"] / out["sequential_fp32_mlups"], 3)
    return out


def run_batch(args):
    line = {"metric": METRIC, "workload": "batch of 64 stretched-grid lattices (seed 7)", "unit": "MLUPS",
            **batch_numbers(args.batch_steps, args.storage if args.storage != "fp32" else "fp16")}
    print(json.dumps(line))


def serve_numbers(requests: int, storage: str, chunk: int, seconds: float) -> dict:
    """The first requests of the seed-11 Poisson trace served with
    continuous batching vs one solve at a time; p50/p99 latency and
    aggregate MLUPS."""
    import torch

    from paper_2607_15362_b300.serve import Server, requests_from_trace, run_sequential

    torch.cuda.set_device(0)
    trace = gi.serving_trace()[:requests]
    reqs = requests_from_trace(trace, storage=storage)
    offered = sum(r.problem.nodes * r.budget for r in reqs) / max(trace[-1]["arrival_s"], 1e-9) / 1e6
    srv = Server(150 * (1 << 30) // 1, max_slots=256, chunk=chunk, storage=storage)
    res_b, sum_b = srv.run(reqs, max_wall_s=seconds)
    srv.close()
    res_s, sum_s = run_sequential(reqs, max_wall_s=seconds)
    return {"workload": f"serving trace (seed 11), first {len(reqs)} requests", "unit": "MLUPS",
            "offered_mlups": round(offered, 1),
            "batched": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in sum_b.items()},
            "sequential": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in sum_s.items()}}


def run_serve(args):
    print(json.dumps({"metric": METRIC, **serve_numbers(args.requests, args.storage,
                                                        args.chunk if args.chunk != 1000 else 500,
                                                        args.serve_seconds)}))


def lattice_rate(spec: dict, storage: str, steps: int, init=None, streaming: str = "two_buffers") -> dict:
    """us per LB step (CUDA events around goc_step after a warm-up call that
    lets the launch autotuner run), node updates per second and the HBM
    fraction (algorithmic bytes / time over the measured copy bandwidth)."""
    import torch

    import paper_2607_15362_b300 as goc
    stream = torch.cuda.current_stream()
    lat = goc.Lattice(spec, storage=storage, stream=stream.cuda_stream, streaming=streaming)
    if init:
        lat.init_fields(**init)
    lat.step(max(200, steps // 4))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / steps
    nodes = spec["nx"] * spec["ny"]
    peaks, _ = measured_peaks()
    bpn = lat.bytes_per_node
    _, held = lat.footprint() if streaming != "two_buffers" else (None, None)
    out = {"us_per_step": round(us, 3), "mlups": round(nodes / us, 1),
           "hbm_frac": round(bpn * nodes / (us * 1e-6) / (float(peaks.get("hbm_gbs", 6400.0)) * 1e9), 4),
           "bytes_per_node": round(bpn, 2)}
    lat.close()
    if held is not None:
        out["resident_bytes_per_node"] = round(held / nodes, 2)
    return out


def extra_numbers(args) -> dict:
    """The rest of the metric, measured in the same run as the headline: 16-bit
    against FP32 storage and FP32 updated in place (the benchmark cavity, and
    at 2048^2 beyond L2), the
    coupled MHD Hartmann channel (256 x 1024, tanh beta = 3, Ha = 100), the
    64-lattice batch against sequential launches, and serving p50/p99."""
    import paper_2607_15362_b300 as goc
    t0 = time.perf_counter()
    out = {}
    storage = {}
    for n, re in ((512, 1000.0), (2048, 4000.0)):
        prob = gi.lid_cavity(n=n, Re=re)
        _, cs2 = goc.metric_info(prob.lattice_spec(1.0))
        spec = prob.lattice_spec(cs2)
        row = {st: lattice_rate(spec, st, 2000 if n == 512 else 400) for st in ("fp32", "fp16", "bf16")}
        row["fp16_over_fp32"] = round(row["fp16"]["mlups"] / row["fp32"]["mlups"], 3)
        # one population buffer updated in place (goc_exec.streaming = 1)
        row["fp32_in_place"] = lattice_rate(spec, "fp32", 2000 if n == 512 else 400, streaming="in_place")
        row["fp16_in_place"] = lattice_rate(spec, "fp16", 2000 if n == 512 else 400, streaming="in_place")
        storage[f"cavity_{n}x{n}" + ("" if n == 512 else f"_Re{re:g}")] = row
    out["storage"] = storage
    prob = gi.hartmann_channel()
    _, cs2 = goc.metric_info(prob.lattice_spec(1.0))
    spec = prob.lattice_spec(cs2)
    y = prob.ny * gi.wall_positions(prob.map2, prob.ny)
    ua, ba = gi.hartmann_profiles(spec, 100.0, y)
    shape = (prob.ny, prob.nx)
    import numpy as np
    init = {"u1": np.broadcast_to(ua[:, None], shape).copy(), "b1": np.broadcast_to(ba[:, None], shape).copy()}
    out["mie_hartmann_256x1024"] = {st: lattice_rate(spec, st, 2000, init) for st in ("fp32", "fp16")}
    out["mie_hartmann_256x1024"]["fp32_in_place"] = lattice_rate(spec, "fp32", 2000, init, streaming="in_place")
    out["batch"] = batch_numbers(500)
    out["serve"] = serve_numbers(args.requests, "fp32", 500, args.serve_seconds)
    out["extras_wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def _wall_positions(m, n):
    """Physical node positions of a wall axis as a fraction of the side (see
    goc_inputs.wall_positions)."""
    return gi.wall_positions(m, n)


def _centrelines(prob, fields, u_lid):
    """Velocity profiles of a square cavity along its two centrelines, at the
    physical node positions, normalised by the side and the lid speed:
    u1 on x = L/2 against y/L, u2 on y = L/2 against x/L.  With an even node
    count and a symmetric map the centreline lies half-way between the two
    middle columns (rows), whose average is taken."""
    import numpy as np

    positions = _wall_positions
    n = prob.nx
    assert n == prob.ny and n % 2 == 0
    y = positions(prob.map2, n)
    x = positions(prob.map1, n)
    u = 0.5 * (fields[1][:, n // 2 - 1] + fields[1][:, n // 2]) / u_lid
    v = 0.5 * (fields[2][n // 2 - 1, :] + fields[2][n // 2, :]) / u_lid
    return y, u, x, v


def run_accuracy(args):
    """Matched accuracy: the GOC cavity (512^2, tanh beta = 2) against the
    standard uniform-grid LBM at several sizes, all at the same Reynolds and
    Mach numbers and the same dimensionless time t* = t u_lid / L, each
    compared on the centreline profiles with a uniform 2048^2 run of the
    standard scheme (FP32) as the reference."""
    import numpy as np
    import torch

    import paper_2607_15362_b300 as goc

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    tstar = args.tstar

    def run(prob, scheme):
        if scheme == "standard":
            spec = prob.lattice_spec(1.0 / 3.0)
        else:
            _, cs2 = goc.metric_info(prob.lattice_spec(1.0))
            spec = prob.lattice_spec(cs2)
        u_lid = spec["walls"]["N"]["u"]
        steps = int(round(tstar * prob.nx / u_lid))
        lat = goc.Lattice(spec, scheme=scheme, stream=stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        fields = lat.moments()
        lat.close()
        return {"n": prob.nx, "steps": steps, "seconds": ms / 1e3, "mlups": prob.nodes * steps / ms / 1e3,
                "profiles": _centrelines(prob, fields, u_lid)}

    ref = run(gi.uniform_cavity(n=args.ref_n), "standard")
    ry, ru, rx, rv = ref["profiles"]

    def err(r):
        y, u, x, v = r["profiles"]
        # reference interpolated to the nodes, closed by the wall values (u = 1 at the lid)
        uref = np.interp(y, np.concatenate([[0.0], ry, [1.0]]), np.concatenate([[0.0], ru, [1.0]]))
        vref = np.interp(x, np.concatenate([[0.0], rx, [1.0]]), np.concatenate([[0.0], rv, [0.0]]))
        return float(np.sqrt((np.sum((u - uref) ** 2) + np.sum((v - vref) ** 2))
                             / (np.sum(uref ** 2) + np.sum(vref ** 2))))

    rows = []
    goc_r = run(gi.lid_cavity(n=512), "goc")
    rows.append({"scheme": "goc tanh beta=2", **{k: goc_r[k] for k in ("n", "steps", "seconds", "mlups")},
                 "centreline_rel_err": err(goc_r)})
    for n in args.uniform_sizes:
        r = run(gi.uniform_cavity(n=n), "standard")
        rows.append({"scheme": "standard uniform", **{k: r[k] for k in ("n", "steps", "seconds", "mlups")},
                     "centreline_rel_err": err(r)})
    for r in rows:
        r["seconds"] = round(r["seconds"], 3)
        r["mlups"] = round(r["mlups"], 1)
        r["centreline_rel_err"] = float(f"{r['centreline_rel_err']:.4g}")
    # uniform size and time at the GOC error (log-log interpolation between measured sizes)
    uni = sorted([r for r in rows if r["scheme"] == "standard uniform"], key=lambda r: r["n"])
    target = rows[0]["centreline_rel_err"]
    match = None
    for a, b in zip(uni, uni[1:]):
        ea, eb = a["centreline_rel_err"], b["centreline_rel_err"]
        if (ea - target) * (eb - target) <= 0 and ea != eb:
            w = (np.log(target) - np.log(ea)) / (np.log(eb) - np.log(ea))
            n = float(np.exp(np.log(a["n"]) + w * (np.log(b["n"]) - np.log(a["n"]))))
            t = float(np.exp(np.log(a["seconds"]) + w * (np.log(b["seconds"]) - np.log(a["seconds"]))))
            match = {"uniform_n": round(n, 1), "uniform_seconds": round(t, 3),
                     "goc_seconds": rows[0]["seconds"], "goc_speedup_at_matched_accuracy": round(t / rows[0]["seconds"], 3)}
            break
    line = {"metric": METRIC, "workload": f"512^2 cavity matched accuracy at t* = {tstar}", "unit": "MLUPS",
            "reference": {"scheme": "standard uniform FP32", "n": ref["n"], "steps": ref["steps"],
                          "mlups": round(ref["mlups"], 1)},
            "runs": rows, "matched": match}
    print(json.dumps(line))


def _vortex_centres(prob, fields):
    """Centres of the primary vortex (minimum of the stream function) and of
    the first secondary vortices at the bottom corners (local maxima), in
    units of the side, from U1 on the physical node positions of the tanh
    map.  psi(x, y) = integral of u from the bottom wall (u = 0 there) along
    y; the extremum node is refined by a parabola through its neighbours
    along each axis."""
    import numpy as np

    x, y = _wall_positions(prob.map1, prob.nx), _wall_positions(prob.map2, prob.ny)
    u = fields[1]
    psi = np.empty_like(u)
    psi[0] = 0.5 * u[0] * y[0]
    for j in range(1, prob.ny):
        psi[j] = psi[j - 1] + 0.5 * (u[j] + u[j - 1]) * (y[j] - y[j - 1])

    def refine(c, k, f):
        if 0 < k < len(c) - 1:
            x0, x1, x2 = c[k - 1], c[k], c[k + 1]
            f0, f1, f2 = f[k - 1], f[k], f[k + 1]
            den = (x0 - x1) * (x0 - x2) * (x1 - x2)
            a = (x2 * (f1 - f0) + x1 * (f0 - f2) + x0 * (f2 - f1)) / den
            b = (x2 * x2 * (f0 - f1) + x1 * x1 * (f2 - f0) + x0 * x0 * (f1 - f2)) / den
            if a != 0:
                return float(-b / (2 * a))
        return float(c[k])

    def centre(mask, sign):
        q = np.where(mask, sign * psi, -np.inf)
        j, i = np.unravel_index(np.argmax(q), q.shape)
        return [round(refine(x, i, psi[j]), 4), round(refine(y, j, psi[:, i]), 4)]

    X, Y = np.meshgrid(x, y)
    return {"primary": centre(np.ones_like(psi, bool), -1.0),
            "bottom_left": centre((X < 0.3) & (Y < 0.3), 1.0),
            "bottom_right": centre((X > 0.6) & (Y < 0.4), 1.0),
            "top_left": centre((X < 0.3) & (Y > 0.7), 1.0)}


def run_capacity(args):
    """The largest lattice one GPU holds with two population buffers and in
    place: a channel with the MIE (Hartmann flow, tanh beta = 3 across,
    Ha = 100), 40,000 rows and as many columns (a multiple of 32) as fill about
    80% of the free device memory in place (at most 2e9 nodes).  Each mode is
    created with uniform initial fields, stepped 2 + 10 times (the 10 timed with
    CUDA events) and its mass read, or reports why it could not be created."""
    import torch

    import paper_2607_15362_b300 as goc

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    free, total = torch.cuda.mem_get_info()
    ny = 40000
    nodes = min(int(0.8 * free / 96.0), 2_000_000_000)
    nx = max(32, nodes // ny // 32 * 32)
    prob = gi.Problem("hartmann", nx, ny, {"kind": "uniform"}, {"kind": "tanh2", "beta": 3.0},
                      {"Ha": 100.0, "Re": 100.0, "tau": 1.0, "tau_m": 1.0})
    _, cs2 = goc.metric_info(prob.lattice_spec(1.0))
    spec = prob.lattice_spec(cs2)
    runs = []
    for streaming in ("two_buffers", "in_place"):
        rec = {"streaming": streaming}
        try:
            lat = goc.Lattice(spec, stream=stream.cuda_stream, streaming=streaming, fixed_launch=True)
        except goc.GocError as e:
            rec.update(created=False, error=str(e))
            runs.append(rec)
            continue
        _, held = lat.footprint()
        lat.step(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(10)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        rec.update(created=True, device_gb=round(held / 1e9, 2), bytes_per_node=round(held / (nx * ny), 2),
                   ms_per_step=round(ms, 3), mlups=round(nx * ny / ms / 1e3, 1), mass=lat.mass(),
                   steps=lat.steps_done)
        lat.close()
        runs.append(rec)
    print(json.dumps({"metric": METRIC, "workload": f"capacity: Hartmann channel with the MIE, {nx} x {ny} "
                      f"({nx * ny / 1e9:.2f} G nodes), FP32", "device_free_gb": round(free / 1e9, 1),
                      "device_total_gb": round(total / 1e9, 1), "runs": runs}))


def run_vortex(args):
    """The cavity of Sec. 7.3 run to its steady state on the GPU, and the
    centres of its primary and bottom-corner vortices (the quantities of the
    paper's Tables 1 and 2)."""
    import torch

    import paper_2607_15362_b300 as goc

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    prob = gi.lid_cavity(n=args.cavity_n, beta=args.vortex_beta, Re=args.vortex_re,
                         u_lid=args.vortex_mach / math.sqrt(3.0))   # lid at this Mach number
    _, cs2 = goc.metric_info(prob.lattice_spec(1.0))
    spec = prob.lattice_spec(cs2)
    u_lid = spec["walls"]["N"]["u"]
    lat = goc.Lattice(spec, stream=stream.cuda_stream, check_every=1000)
    steps = int(round(args.tstar * prob.nx / u_lid))
    t0 = time.perf_counter()
    lat.step(steps)
    lat.sync()
    wall = time.perf_counter() - t0
    fields = lat.moments()
    lat.close()
    # the paper's GOC-LBM values (Table 1, Table 2), for context
    printed = {1000.0: {"primary": [0.5314, 0.5646], "bottom_left": [0.0855, 0.0779],
                        "bottom_right": [0.8581, 0.1104], "top_left": None},
               3200.0: {"primary": [0.5178, 0.5404], "bottom_left": [0.0813, 0.1194],
                        "bottom_right": [0.8249, 0.0845], "top_left": [0.05318, 0.89824]},
               5000.0: {"primary": [0.5151, 0.5356], "bottom_left": [0.0726, 0.1383],
                        "bottom_right": [0.8040, 0.0747], "top_left": [0.0646, 0.9060]}}.get(args.vortex_re)
    print(json.dumps({"metric": METRIC, "workload": f"cavity {prob.nx}^2, tanh beta = {args.vortex_beta}, "
                      f"Re = {args.vortex_re:g}, lid Mach {args.vortex_mach:g}, t* = {args.tstar}: vortex centres",
                      "steps": steps, "seconds": round(wall, 3), "mlups": round(prob.nodes * steps / wall / 1e6, 1),
                      "centres": _vortex_centres(prob, fields),
                      "paper_goc_lbm": printed}))


def _hartmann_analytic(spec, ny, positions):
    """u_x and B_x of the Hartmann flow (Sec. 7.4) at physical positions y in
    [0, ny] of a channel of half-width H = ny/2 (goc_inputs.hartmann_profiles)."""
    return gi.hartmann_profiles(spec, float(spec.get("_Ha")), positions)


def run_accuracy_mhd(args):
    """Matched accuracy for the Hartmann channel (Ha = 100, Re = 100, Pm = 1,
    256 periodic columns), scored by the column-mean u_x, B_x against the
    analytic profiles of Sec. 7.4.

    The GOC grid (wall-normal tanh beta = 3, 1024 rows) has c_s^2 = q^2/3 =
    3.0e-4, so nu = eta = 1.5e-4 and the Alfven crossing time 2 H^2/(Ha nu)
    is 3.5e7 steps: from rest it needs about 1e8 steps.  It therefore starts
    from the analytic profiles and runs until its own discrete steady state
    (residual 1e-9, no new smallest residual over 20 checks, or the step
    cap), which measures its discretisation error.  The uniform grids (the
    same library with h = 1 and the cubic terms dropped: the standard
    central-moment D2Q9 + D2Q5 scheme, c_s^2 = 1/3) run from rest for four
    crossing times.  The matched uniform size is interpolated (or
    extrapolated with the measured order) in log-log."""
    import numpy as np
    import torch

    import paper_2607_15362_b300 as goc

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    Ha, Re = args.mhd_ha, args.mhd_re
    roberts = args.mhd_map == "roberts"
    goc_name = f"goc roberts gamma={args.mhd_gamma}" if roberts else "goc tanh beta=3"

    def run(ny, stretched):
        if stretched:
            if roberts:   # clustering at both walls
                map2 = {"kind": "roberts", "gamma": args.mhd_gamma, "alpha": 0.5}
            else:
                map2 = {"kind": "tanh2", "beta": 3.0}
            y = ny * _wall_positions(map2, ny)
            prob = gi.Problem("hartmann", args.mhd_nx, ny, {"kind": "uniform"}, map2,
                              {"Ha": Ha, "Re": Re, "tau": 1.0, "tau_m": 1.0})
            _, cs2 = goc.metric_info(prob.lattice_spec(1.0))
        else:
            prob = gi.Problem("hartmann", args.mhd_nx, ny, {"kind": "uniform"}, {"kind": "uniform"},
                              {"Ha": Ha, "Re": Re, "tau": 1.0, "tau_m": 1.0, "gi": 0})
            cs2 = 1.0 / 3.0
            y = np.arange(ny) + 0.5
        spec = prob.lattice_spec(cs2)
        spec["_Ha"] = Ha
        d = spec["derived"]
        crossing = 2.0 * d["H"] ** 2 / (Ha * d["nu"])
        ua, ba = _hartmann_analytic(spec, ny, y)
        lat = goc.Lattice(spec, stream=stream.cuda_stream, check_every=5000 if stretched else 500,
                          plateau_checks=20 if stretched else 0,
                          streaming=args.streaming if stretched else "two_buffers")
        if stretched:
            shape = (ny, args.mhd_nx)
            lat.init_fields(u1=np.broadcast_to(ua[:, None], shape).copy(),
                            b1=np.broadcast_to(ba[:, None], shape).copy())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if stretched and args.mhd_goc_crossings > 0:   # a fixed number of crossing times
            steps = int(args.mhd_goc_crossings * crossing)
            lat.step(steps)
            lat.sync()
            res = None
        elif stretched:
            steps, res = lat.run_until(1e-9, args.mhd_goc_max_steps)
        else:
            steps = int(4 * crossing)
            lat.step(steps)
            lat.sync()
            res = None
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        f = lat.moments()
        lat.close()
        u, b = f[1].mean(axis=1), f[3].mean(axis=1)
        eu = float(np.linalg.norm(u - ua) / np.linalg.norm(ua))
        eb = float(np.linalg.norm(b - ba) / np.linalg.norm(ba))
        row = {"grid": goc_name if stretched else "uniform", "ny": ny,
               "streaming": args.streaming if stretched else "two_buffers",
               "start": "analytic" if stretched else "rest", "steps": int(steps),
               "crossing_steps": round(crossing), "seconds": round(wall, 3),
               "mlups": round(args.mhd_nx * ny * steps / wall / 1e6, 1),
               "err_u": float(f"{eu:.4g}"), "err_b": float(f"{eb:.4g}"), "err": float(f"{max(eu, eb):.4g}"),
               "err_sq": float(f"{max(eu, eb) ** 2:.4g}")}
        if res is not None:
            row["residual"] = float(f"{res:.3g}")
        return row

    rows = [run(args.mhd_goc_ny, True)]
    for ny in args.mhd_uniform_ny:
        rows.append(run(ny, False))
    uni = sorted(rows[1:], key=lambda r: r["ny"])
    target = rows[0]["err"]
    match = None
    for a, b in zip(uni, uni[1:]):
        ea, eb = a["err"], b["err"]
        if (ea - target) * (eb - target) <= 0 and ea != eb:
            w = (np.log(target) - np.log(ea)) / (np.log(eb) - np.log(ea))
            match = {"uniform_ny": round(float(np.exp(np.log(a["ny"]) + w * (np.log(b["ny"]) - np.log(a["ny"])))), 1),
                     "how": "interpolated"}
            break
    if match is None and len(uni) >= 2 and uni[-1]["err"] < uni[-2]["err"]:
        a, b = uni[-2], uni[-1]
        order = np.log(a["err"] / b["err"]) / np.log(b["ny"] / a["ny"])
        ny = b["ny"] * (b["err"] / target) ** (1.0 / order)
        match = {"uniform_ny": round(float(ny), 1), "how": f"extrapolated with the measured order {order:.2f}"}
    print(json.dumps({"metric": METRIC, "workload": f"Hartmann channel {args.mhd_nx} columns, Ha = {Ha:g}, Re = {Re:g}: "
                      "matched accuracy", "runs": rows, "matched": match}))


def cpu_baseline(prob, spec_lib, budget_s: float = 15.0):
    """FP64 oracle, as it stands, on this host's cores: a bounded number of
    time steps of the same workload (its own c_s^2; the MIE and collision
    settings of the GPU run), scaled to MLUPS."""
    import oracle
    cores = os.cpu_count() or 1
    cs2 = oracle.build_metric(prob.lattice_spec(1.0)).cs2()
    spec = prob.lattice_spec(cs2)
    for k in ("mhd", "collision"):
        if k in spec_lib:
            spec[k] = spec_lib[k]
    o = oracle.Oracle(spec, threads=cores)
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    n = max(1, min(200, int(budget_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    return {"value": round(prob.nodes * n / dt / 1e6, 3), "unit": "MLUPS", "cores": o.threads,
            "kind": "oracle", "sample": f"{n} time steps of {prob.name or prob.kind} ({prob.nx}x{prob.ny}) "
                                         "after 1 warm-up step"}


def run_oracle_timing(args):
    """The FP64 oracle on this host, single-threaded and on all cores, on the
    Poiseuille channel (32 x 64), the 512^2 cavity, an x-invariant strip of
    the Hartmann channel (4 x 1024) and the 8 smallest lattices of the batch;
    each a bounded number of steps (about args.cpu_seconds per entry)."""
    import oracle
    cores = os.cpu_count() or 1
    probs = [("poiseuille_channel_32x64", gi.poiseuille_channel()), ("lid_cavity_512x512", gi.lid_cavity()),
             ("hartmann_strip_4x1024", gi.hartmann_channel(nx=4))]
    batch = sorted(gi.batch_lattices(), key=lambda p: p.nodes)[:8]
    rows = []

    def time_one(prob, threads, budget):
        cs2 = oracle.build_metric(prob.lattice_spec(1.0)).cs2()
        o = oracle.Oracle(prob.lattice_spec(cs2), threads=threads)
        t0 = time.perf_counter()
        o.step(1)
        one = max(time.perf_counter() - t0, 1e-4)
        n = max(1, min(1000, int(budget / one)))
        t0 = time.perf_counter()
        o.step(n)
        return prob.nodes * n, time.perf_counter() - t0, n, o.threads

    for name, prob in probs:
        for threads in (1, cores):
            upd, dt, n, used = time_one(prob, threads, args.cpu_seconds / 4)
            rows.append({"workload": name, "threads": used, "steps": n, "mlups": round(upd / dt / 1e6, 3)})
    for threads in (1, cores):
        upd = dt = 0.0
        for prob in batch:
            u, d, n, used = time_one(prob, threads, args.cpu_seconds / 16)
            upd += u
            dt += d
        rows.append({"workload": "batch_8_smallest_lattices", "threads": used, "mlups": round(upd / dt / 1e6, 3)})
    print(json.dumps({"metric": METRIC, "workload": "oracle timing on the host cores", "unit": "MLUPS",
                      "cores": cores, "build": "gcc -O3 -march=native -fopenmp, no fast-math", "runs": rows}))


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    prob = _problem(args)   # the same workload as the main line, stepped by the oracle
    cores = os.cpu_count() or 1
    cs2 = oracle.build_metric(prob.lattice_spec(1.0)).cs2()
    o = oracle.Oracle(_spec(args, prob, cs2), threads=cores)
    per_step = max(1, args.ref_steps_per_step)
    for _ in range(args.warmup):
        o.step(per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(per_step)
    dt = time.perf_counter() - t0
    value = prob.nodes * per_step * args.steps / dt / 1e6
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": prob.name + f"_{args.storage}", "nodes": prob.nodes,
                   "lb_steps_per_bench_step": per_step, "parallelism": "host cores"},
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": o.threads, "kind": "oracle",
                         "sample": f"{per_step} time steps per benchmark step of {prob.name} ({prob.nx}x{prob.ny})"},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--chunk", type=int, default=1000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass (profiling runs)")
    ap.add_argument("--cavity-n", type=int, default=512, help="cavity side (512 is the benchmark workload)")
    ap.add_argument("--cavity-re", type=float, default=1000.0,
                    help="cavity Reynolds number (1000 is the benchmark workload; with the Mach-matched lid "
                         "tau - 1/2 grows as n/Re and the step is stable up to tau of about 2)")
    ap.add_argument("--grid", default="tanh", choices=["tanh", "spiral", "annulus"],
                    help="tanh map on both axes (the benchmark cavity), the cavity on a logarithmic-spiral node "
                         "table, or Taylor-Couette flow on the annular sector")
    ap.add_argument("--streaming", default="two_buffers", choices=["two_buffers", "in_place"],
                    help="in_place: one population buffer updated in place (straight grids)")
    ap.add_argument("--scheme", default="goc", choices=["goc", "goc_srt", "goc_raw"],
                    help="collision: central-moment MRT (the benchmark), SRT (Appendix F), raw-moment MRT (Appendix D)")
    ap.add_argument("--mie", action="store_true", help="couple the MIE (Appendix G)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-steps-per-step", type=int, default=4)
    ap.add_argument("--workload", default="cavity",
                    choices=["cavity", "batch", "serve", "accuracy", "accuracy_mhd", "oracle_timing", "vortex",
                             "capacity"])
    ap.add_argument("--mhd-nx", type=int, default=256)
    ap.add_argument("--mhd-ha", type=float, default=100.0)
    ap.add_argument("--mhd-re", type=float, default=100.0)
    ap.add_argument("--mhd-map", default="tanh", choices=["tanh", "roberts"],
                    help="wall-normal map of the GOC Hartmann grid (roberts: the paper's Table 3 grids)")
    ap.add_argument("--mhd-gamma", type=float, default=1.05)
    ap.add_argument("--vortex-re", type=float, default=1000.0)
    ap.add_argument("--vortex-beta", type=float, default=1.2)
    ap.add_argument("--vortex-mach", type=float, default=0.05 * math.sqrt(3.0))
    ap.add_argument("--mhd-goc-crossings", type=float, default=0.0,
                    help="run the GOC grid for this many crossing times instead of to its residual plateau")
    ap.add_argument("--mhd-goc-ny", type=int, default=1024)
    ap.add_argument("--mhd-goc-max-steps", type=int, default=1000000)
    ap.add_argument("--mhd-uniform-ny", type=int, nargs="+", default=[512, 1024, 2048])
    ap.add_argument("--tstar", type=float, default=5.0, help="accuracy workload: dimensionless time t u_lid / L")
    ap.add_argument("--ref-n", type=int, default=2048, help="accuracy workload: reference grid side")
    ap.add_argument("--uniform-sizes", type=int, nargs="+", default=[256, 384, 512, 768, 1024])
    ap.add_argument("--batch-steps", type=int, default=5000)
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra measurements of the main line (storage formats, sizes, MHD, batch, serving)")
    ap.add_argument("--replicas", action="store_true",
                    help="with several ranks: one independent lattice per rank instead of one lattice in slabs")
    ap.add_argument("--shard", action="store_true",
                    help="run the slab path (one lattice in slabs along xi2) even on one rank")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "accuracy":
        run_accuracy(args)
    elif args.workload == "accuracy_mhd":
        run_accuracy_mhd(args)
    elif args.workload == "oracle_timing":
        run_oracle_timing(args)
    elif args.workload == "vortex":
        run_vortex(args)
    elif args.workload == "capacity":
        run_capacity(args)
    elif args.shard or (int(os.environ.get("WORLD_SIZE", "1")) > 1 and not args.replicas and args.grid == "tanh"
                        and not args.mie and args.scheme == "goc"):
        run_sharded(args)   # one lattice over all ranks, slabs along xi2
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
