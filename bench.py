#!/usr/bin/env python
"""Throughput of the entropic (KBC) D3Q27 step on the deforming, self-propelled
anguilliform swimmer (arXiv 1608.04658, Sec. 4.3): 768x256x256 periodic box,
body length L = 128 (19,200-triangle mesh of elliptic cross sections), midline
wave with period T = 4000 steps, free along the swimming direction, refill of
uncovered nodes every step.  This is the largest of the paper's single-GPU
configurations (50,331,648 nodes).

One step = the whole hot path: body update and mesh pose, node marks and
boundary list, refill, bulk stream+collide, Grad boundary + collide,
momentum-exchange reduction.  The value is GLUPS over box nodes, FP32
storage; FP16 and BF16 storage and the exact stabilizer are reported under
"variants", and the two-way coupled sedimenting sphere (128x128x256, Sec. 4.1)
under "workloads" with the same measurement.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload swimmer|sphere|airfoil|tgv] [--shape n]

--workload selects another of the paper's configurations for the main line:
the sedimenting sphere, the plunging airfoil (1024x512x64, chord 128,
Sec. 4.2) or the bodiless periodic Taylor-Green box (256^3, or n^3 with
--shape n) that isolates the bulk kernel.

The CPU baseline is the FP64 oracle on the host: one thread, and under
"all_cores" one independent replica per host core, on a bounded sample of
the workload (the swimmer: one step of a 176x64x32 periodic crop around the
whole body; the sphere: two steps of the full box).

With N > 1 (torchrun) every rank runs an independent replica (the path has
no data-parallel split without a halo exchange); the value is all ranks'
node updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import datetime as _dt
import hashlib
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & % of HBM roofline, D3Q27 entropic step (FP32 vs 16-bit); adjoint/fwd time"
BYTES_PER_NODE = {"fp64": 432, "fp32": 216, "fp16": 108, "bf16": 108}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f32", "bf16": "f32"}
FALLBACK_HBM_GBS = 6800.0
PROFILES = os.path.join(ROOT, "profiles")
KERNEL_SOURCES = ["bulk.cu", "pull.cuh", "kbc.cuh", "kbcv.cuh", "lbm_internal.cuh"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="fp32", choices=list(BYTES_PER_NODE))
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-refinement", action="store_true",
                    help="skip the two-level block refinement line (key refinement)")
    ap.add_argument("--refinement-only", action="store_true",
                    help="print only the two-level block refinement line")
    ap.add_argument("--shape", default=None,
                    help="nx,ny,nz of a smaller box with the same sphere (profiling cases only); "
                         "n (or n,n,n) of the periodic Taylor-Green box (default 256)")
    ap.add_argument("--workload", default="swimmer", choices=["sphere", "airfoil", "swimmer", "tgv"])
    ap.add_argument("--parallel", default="auto", choices=["auto", "split", "replicas"],
                    help="several GPUs: split the box along z into one slab per rank (auto, split) or run "
                         "independent replicas; split on one GPU runs a single slab with halo exchange")
    ap.add_argument("--gamma", default="analytic", choices=["analytic", "exact"],
                    help="the stabilizer of the headline line: the analytic formula or the exact root "
                         "(the variants time the other storage forms and the exact root as well)")
    ap.add_argument("--launch-order", default="auto", choices=["auto", "split", "sequential"],
                    help="the step's launch order (lbm_set_launch_order); auto times both in the first steps "
                         "and keeps the faster (the results do not depend on it)")
    ap.add_argument("--slabs", type=int, default=2,
                    help="--parallel split on one GPU: slab lattices in this process")
    ap.add_argument("--second-workload", default="sphere", choices=["sphere", "airfoil", "swimmer", "tgv", "none"],
                    help="workload measured beside the main line, reported under 'workloads'")
    ap.add_argument("--accuracy-steps", type=int, default=2000,
                    help="steps of the FP64/FP32/FP16/BF16 sphere comparison (0 to skip it)")
    ap.add_argument("--adjoint-horizon", type=int, default=8000,
                    help="steps of the adjoint/forward measurement (0 to skip it)")
    ap.add_argument("--adjoint-checkpoint", type=int, default=0,
                    help="checkpoint spacing of the adjoint measurement (0: ceil(sqrt(horizon)))")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint measurement and print it (profiling runs)")
    return ap.parse_args(argv)


# ----------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        # LBM_DIST_BACKEND=gloo: a host-only group (the slab exchange is then
        # staged through host memory), e.g. to run several ranks on one GPU
        backend = os.environ.get("LBM_DIST_BACKEND") or ("nccl" if torch.cuda.is_available() else "gloo")
        if torch.cuda.is_available():
            torch.cuda.set_device(local % torch.cuda.device_count())
        dist.init_process_group(backend=backend)
    return world, rank, local


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(value: float, world: int) -> float:
    """Maximum of a float over ranks (identity for one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        # the raw samples go to LBM_CLOCKS_DIR (the system's temporary directory by default)
        import tempfile
        out = os.environ.get("LBM_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out, f"clocks_rank{device_index}.csv")
        self.proc = None
        self.windows = []
        self.dev = device_index

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "100"]
            bus = _pci_bus_id(self.dev)
            if bus:
                cmd += ["-i", bus]
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def mark(self, t0: float, t1: float):
        self.windows.append((t0, t1))

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = _dt.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        if not rows:
            return None
        inside = [r for r in rows if any(a - 0.15 <= r[0] <= b + 0.15 for a, b in self.windows)]
        sel = inside or rows
        mhz = sorted(r[1] for r in sel)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in sel for k in range(4) if r[3][k].lower() == "active"})
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": max(r[2] for r in sel), "reasons": reasons,
                "samples": len(sel), "in_timed_region": bool(inside)}


def _pci_bus_id(dev: int) -> str | None:
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


# ----------------------------------------------------------------- roofline inputs
def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs_sustained", "hbm_gbs", "hbm_GBps", "hbm_copy_gbs"):
                if key in d and d[key]:
                    return float(d[key]), f"measured ({key})"
        except (ValueError, OSError):
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1608_04658_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(storage: str, workload_name: str):
    """DRAM bytes per bulk launch from a committed ncu summary
    (profiles/bulk_kernel_*.md) taken on this workload with the current
    kernel sources, else None."""
    if not os.path.isdir(PROFILES):
        return None
    sha_now = kernel_sha()
    for fn in sorted(os.listdir(PROFILES)):
        if not (fn.startswith("bulk_kernel_") and fn.endswith(".md")):
            continue
        sha, val, name = None, None, None
        for line in open(os.path.join(PROFILES, fn)):
            line = line.strip().strip("`")
            if line.startswith("source_sha:"):
                sha = line.split(":", 1)[1].strip()
            if line.startswith("traffic_workload:"):
                name = line.split(":", 1)[1].strip()
            if line.startswith(f"traffic_bytes_per_launch[{storage}]:"):
                try:
                    val = float(line.split(":", 1)[1].strip())
                except ValueError:
                    val = None
        if sha == sha_now and name == workload_name and val is not None:
            return val
    return None


# ----------------------------------------------------------------- workload
def workload(shape=None, kind="sphere"):
    import synth
    if kind == "tgv":
        dims = {int(v) for v in shape.split(",")} if shape else {256}
        if len(dims) != 1:
            raise SystemExit("the Taylor-Green box is cubic: --shape n or n,n,n")
        wl = synth.tgv_periodic(dims.pop())
    elif kind == "airfoil":
        wl = synth.plunging_airfoil()
    elif kind == "swimmer":
        wl = synth.anguilliform_swimmer()
    elif shape:
        wl = synth.sedimenting_sphere(shape=tuple(int(v) for v in shape.split(",")))
    else:
        wl = synth.sedimenting_sphere()
    wl["kind"] = kind
    return wl


def initial_flow(wl):
    """Quiescent fluid, the inflow velocity everywhere for the airfoil, the
    Taylor-Green field for the bodiless box."""
    import synth
    if wl["kind"] == "tgv":
        return synth.taylor_green_fields(wl["shape"], wl["u0"])
    return synth.uniform_fields(wl["shape"], wl.get("u_face", (0.0, 0.0, 0.0)))


def geometry_for(wl):
    """The workload's body as the binding describes it (None without one)."""
    import paper_1608_04658_gb300 as lbm
    if wl["kind"] == "airfoil":
        return lbm.airfoil(wl["le"], wl["chord"], wl["ca"], wl["sa"], wl["h_amp"], wl["h_omega"],
                           wl["camber_m"], wl["camber_p"], wl["thick"])
    if wl["kind"] == "swimmer":
        return lbm.swimmer(wl["X"], wl["rest"], wl["tris"], wl["L"], wl["amp"], wl["wavelength"],
                           wl["period"], ramp=bool(wl["ramp"]), free=True, mass=wl["mass"])
    if wl["kind"] == "tgv":
        return None
    return lbm.sphere(wl["X"], wl["D"] / 2, free=True, rho_ratio=wl["rho_ratio"], g=wl["g"])


def make_lattice(storage, wl, device, gamma_mode=0, order="auto"):
    import numpy as np

    import paper_1608_04658_gb300 as lbm
    shape = wl["shape"]
    lat = lbm.Lattice(shape, wl["nu"], storage=storage, faces=wl["faces"], device=device,
                      u_face=wl.get("u_face", (0.0, 0.0, 0.0)), gamma_mode=gamma_mode)
    if order != "auto":
        lat.set_launch_order(order)
    geom = geometry_for(wl)
    if geom is not None:
        lat.set_geometry(geom)
    rho, u = initial_flow(wl)
    lat.init_state(rho, u)
    return lat, np


def time_storage(storage, wl, args, world, device, clocks, gamma_mode=0):
    import torch
    lat, np = make_lattice(storage, wl, device, gamma_mode, args.launch_order)
    K, W = args.steps, args.warmup
    lat.step(W)
    # the library times both launch orders in its first steps after
    # lbm_set_geometry; finish that trial before the timed region, so every
    # timed step runs the chosen order
    extra = 0
    while lat.launch_order() == "auto" and extra < 32:
        # the choice is made at the first step after the trial's last event
        torch.cuda.synchronize()
        lat.step(1)
        extra += 1
    torch.cuda.synchronize()
    dist_barrier(world)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    lat.profile_begin(K)
    t0 = time.time()
    start.record(lat.stream)
    lat.step(K)
    end.record(lat.stream)
    torch.cuda.synchronize()
    t1 = time.time()
    dist_barrier(world)
    clocks.mark(t0, t1)
    launches = lat.launches()
    bulk_ms, nbulk = lat.profile_end()
    ms = dist_max(start.elapsed_time(end), world)
    flags = lat.flags
    body = lat.body()
    # the timed launch: all bulk nodes, or those outside the body's sweep box
    # when the band's nodes have a launch of their own
    bulk_nodes = lat.N - body["n_band"] if body["n_band"] > 0 else int(((flags & 5) == 0).sum().item())
    F, _ = lat.forces()  # raises on an unstable run
    N = lat.N
    res = dict(ms=ms, glups=N * K * world / (ms * 1e-3) / 1e9, launches=launches,
               bulk_ms=bulk_ms / max(nbulk, 1), bulk_nodes=bulk_nodes, body=body, F=F,
               order=lat.launch_order(), trial_steps_after_warmup=extra)
    lat.close()
    del lat
    torch.cuda.empty_cache()
    return res


def _split_runner(storage, wl, args, world, device):
    """One slab per rank (DistSlab, NCCL between the GPUs); on one GPU
    (world 1), args.slabs slab lattices in this process (SlabSet, device
    copies between them)."""
    from paper_1608_04658_gb300.slab import DistSlab, SlabSet
    kw = dict(storage=storage, faces=wl["faces"], geometry=geometry_for(wl),
              u_face=wl.get("u_face", (0.0, 0.0, 0.0)))
    if world > 1:
        ds = DistSlab(wl["shape"], wl["nu"], device=device, two_phase=True, **kw)
        return ds, [ds.lat]
    ds = SlabSet(wl["shape"], wl["nu"], args.slabs, devices=device, two_phase=True, **kw)
    return ds, ds.slabs


def time_split(storage, wl, args, world, device, clocks):
    """The workload's box split along z into slabs (paper_1608_04658_gb300.slab,
    lbm_set_slab): every step the slabs swap two edge layers per side (NCCL
    send/recv of packed layers between ranks, device copies within one
    process) while the own layers that read no halo layer are updated
    (lbm_step_interior), then the rest of the step runs (lbm_step_edges) and
    the force records are added in slab order on the device
    (lbm_sum_body_force).  The value is the whole box's node updates over the
    slowest rank's time (strong scaling: the box is fixed, each rank updates
    its share).  The roofline figures are those of the first slab's interior
    launch, its nodes counted as the interior layers' less all of the sweep
    box's (a lower bound)."""
    import torch
    ds, lats = _split_runner(storage, wl, args, world, device)
    lat = lats[0]
    ds.init_state(*initial_flow(wl))
    K, W = args.steps, args.warmup
    ds.step(W)
    extra = 0
    while ds.body and any(q.launch_order() == "auto" for q in lats) and extra < 32:
        torch.cuda.synchronize()
        ds.step(1)
        extra += 1
    torch.cuda.synchronize()
    dist_barrier(world)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    lat.profile_begin(K)
    t0 = time.time()
    start.record(lat.stream)
    ds.step(K)
    end.record(lat.stream)
    torch.cuda.synchronize()
    t1 = time.time()
    dist_barrier(world)
    clocks.mark(t0, t1)
    launches = ds.launches
    bulk_ms, nbulk = lat.profile_end()
    ms = dist_max(start.elapsed_time(end), world)
    body = lat.body()
    nx, ny, nz = wl["shape"]
    own = lat.shape[2] - 2 * ds.halo
    interior = own - 2 if own >= 3 else 0
    bulk_nodes = max(nx * ny * interior - body["n_band"], 0)
    if ds.body:
        lat.forces()  # raises on an unstable run
    res = dict(ms=ms, glups=nx * ny * nz * K / (ms * 1e-3) / 1e9, launches=launches,
               bulk_ms=bulk_ms / max(nbulk, 1), bulk_nodes=bulk_nodes, body=body,
               order=",".join(q.launch_order() for q in lats), trial_steps_after_warmup=extra,
               slab_layers=lat.shape[2], slabs=len(lats) if world == 1 else world)
    for q in lats:
        q.close()
    del ds, lat, lats
    torch.cuda.empty_cache()
    return res


def e2e_split(storage, wl, args, world, device):
    """e2e_storage for the z-slab split: each slab copies its rows of the
    pinned initial fields (halo rows included) to the device and builds its
    state from them, then K steps with the exchanges and force hand-overs,
    each step's summed force record read by the host at most two steps later;
    the value is the whole box's node updates over the slowest rank's time."""
    import torch

    from paper_1608_04658_gb300.slab import slab_rows
    ds, lats = _split_runner(storage, wl, args, world, device)
    rho, u = initial_flow(wl)
    nz = wl["shape"][2]
    parts = world if world > 1 else len(lats)
    ks = [ds.rank] if world > 1 else list(range(parts))
    rows = [slab_rows(nz, parts, k, 2) for k in ks]
    ds.init_state(rho, u)
    ds.step(max(args.warmup, 1))
    extra = 0
    while ds.body and any(q.launch_order() == "auto" for q in lats) and extra < 32:
        torch.cuda.synchronize()
        ds.step(1)
        extra += 1
    import numpy as np
    fdt = np.float64 if storage == "fp64" else np.float32
    h_rho = [torch.from_numpy(rho[r].astype(fdt)).pin_memory() for r in rows]
    h_u = [torch.from_numpy(u[r].astype(fdt)).pin_memory() for r in rows]
    del rho, u
    K = args.steps
    lat = lats[0]
    torch.cuda.synchronize()
    dist_barrier(world)
    t0 = time.perf_counter()
    for q, a, b in zip(lats, h_rho, h_u):
        q.init_state(a, b)
    pending = []
    for _ in range(K):
        ds.step(1)
        if ds.body:
            pending.append(lat.forces_async())
            if len(pending) > 2:
                lat.forces_wait(pending.pop(0))
    for tk in pending:
        lat.forces_wait(tk)
    torch.cuda.synchronize()
    t = dist_max(time.perf_counter() - t0, world)
    for q in lats:
        q.close()
    del ds, lat, lats
    torch.cuda.empty_cache()
    nx, ny, _ = wl["shape"]
    h2d = sum(a.numel() * a.element_size() + b.numel() * b.element_size() for a, b in zip(h_rho, h_u))
    return {"value": round(nx * ny * nz * K / t / 1e9, 4), "unit": "GLUPS",
            "h2d_bytes_per_step": int(round(h2d / K)), "d2h_bytes_per_step": 60 if wl["kind"] != "tgv" else 0,
            "note": "each slab: its rows of the initial density and velocity fields (pinned, FP32 for FP32 and "
                    "16-bit storage, halo rows included) read across the host link by lbm_init_state(_f32), which turns them "
                    "into its state, once per run; every step's summed force record (60 bytes) read by the host "
                    "at most two steps later; h2d counted on this rank"}


def e2e_storage(storage, wl, args, device):
    """Same workload through the public API from host memory: the initial
    density and velocity fields (pinned FP64, 4 doubles per node) are read
    across the host link by lbm_init_state, which builds the state from them
    (the device reads the pinned pages in place), then K steps run
    with every step's force, torque, time and status record (60 bytes) copied
    to pinned host memory and read by the host at most two steps later; all of
    it inside the timed region.  The lattice and its body are set up, and the
    launch order chosen, before it."""
    import torch
    lat, _ = make_lattice(storage, wl, device)
    lat.step(max(args.warmup, 1))
    extra = 0
    while lat.launch_order() == "auto" and extra < 32:
        torch.cuda.synchronize()
        lat.step(1)
        extra += 1
    rho, u = initial_flow(wl)
    # the fields in the collision's precision: FP32 for FP32 and 16-bit storage
    import numpy as np
    fdt = np.float64 if storage == "fp64" else np.float32
    h_rho = torch.from_numpy(rho.astype(fdt)).pin_memory()
    h_u = torch.from_numpy(u.astype(fdt)).pin_memory()
    del rho, u
    K = args.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.init_state(h_rho, h_u)
    # each step's force record is copied to pinned host memory while the
    # next steps are enqueued; the host reads it at most two steps later
    pending = []
    for _ in range(K):
        lat.step(1)
        pending.append(lat.forces_async())
        if len(pending) > 2:
            lat.forces_wait(pending.pop(0))
    for tk in pending:
        lat.forces_wait(tk)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    N = lat.N
    lat.close()
    del lat
    torch.cuda.empty_cache()
    h2d = h_rho.numel() * h_rho.element_size() + h_u.numel() * h_u.element_size()
    return {"value": round(N * K / t / 1e9, 4), "unit": "GLUPS",
            "h2d_bytes_per_step": int(round(h2d / K)), "d2h_bytes_per_step": 60,
            "note": "initial density and velocity fields (pinned, in the collision's precision: FP32 for FP32 and "
                    "16-bit storage, 16 bytes per node) read across the host link by lbm_init_state(_f32), which "
                    "turns them into the state, once per run (amortised over the steps); every "
                    "step's force, torque, time and status (60 bytes) copied to pinned host memory and read by "
                    "the host at most two steps later (lbm_body_forces_async / lbm_body_forces_wait)"}


def oracle_body(wl):
    import oracle
    if wl["kind"] == "tgv":
        return None
    if wl["kind"] == "airfoil":
        return oracle.airfoil_body(wl["le"], wl["chord"], wl["ca"], wl["sa"], wl["h_amp"], wl["h_omega"],
                                   wl["camber_m"], wl["camber_p"], wl["thick"])
    if wl["kind"] == "swimmer":
        return oracle.mesh_body(wl["X"], wl["rest"], wl["tris"], wl["L"], wl["amp"], wl["wavelength"],
                                wl["period"], ramp=bool(wl["ramp"]), free=True, mass=wl["mass"])
    return oracle.sphere_body(wl["X"], wl["D"] / 2, free=True, rho_ratio=wl["rho_ratio"], g=wl["g"])


def adjoint_bench(args, world, device):
    """Adjoint/forward time on the differentiated swimmer (256x128x128,
    L = 64, FP32, held): lbm_step over the horizon vs lbm_adjoint_step over
    the same horizon (forward with checkpoints, recompute, reverse sweep),
    objective = mean thrust, gradient w.r.t. (amplitude, wavelength, period)."""
    import torch

    import paper_1608_04658_gb300 as lbm
    import synth
    wl = synth.differentiated_swimmer()
    H = args.adjoint_horizon
    lat = lbm.Lattice(wl["shape"], wl["nu"], storage="fp32", faces=wl["faces"], device=device)
    lat.set_geometry(lbm.swimmer(wl["X"], wl["rest"], wl["tris"], wl["L"], wl["amp"], wl["wavelength"],
                                 wl["period"], mass=wl["mass"]))
    lat.init_state(*synth.uniform_fields(wl["shape"]))
    lat.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    dist_barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    lat.step(H)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    fwd_ms = dist_max(e0.elapsed_time(e1), world)
    dist_barrier(world)
    t0 = time.perf_counter()
    K = args.adjoint_checkpoint if args.adjoint_checkpoint > 0 else int(math.ceil(math.sqrt(H)))
    out = lat.adjoint(H, (-1.0, 0.0, 0.0), checkpoint_every=K)
    torch.cuda.synchronize()
    adj_ms = dist_max(1e3 * (time.perf_counter() - t0), world)
    nx, ny, nz = wl["shape"]
    lat.close()
    del lat
    torch.cuda.empty_cache()
    return {"workload": wl["name"], "storage": "fp32", "horizon": H, "checkpoint_every": K,
            "objective": "mean thrust -F_x over the horizon",
            "theta": "(wave amplitude, wavelength, period)",
            "fwd_ms_per_step": round(fwd_ms / H, 5), "adjoint_ms_per_step": round(adj_ms / H, 5),
            "adjoint_over_forward": round(adj_ms / fwd_ms, 3),
            "J": out["J"], "dJ_dtheta": [float(v) for v in out["dJ_dtheta"]],
            "checkpoint_bytes": int((math.ceil(H / K) + K + 3) * 27 * nx * ny * nz * 4)}


def accuracy_bench(args, device):
    """The sedimenting sphere run for N steps with FP64, FP32, FP16 and BF16
    storage on the GPU: mean hydrodynamic force over the second half and the
    final settling velocity of each form against the FP64 run (the FP64 GPU
    path is itself within 1e-12 of the FP64 oracle over 10 steps); also FP32
    with the exact stabilizer, whose difference is that of the stabilizer
    choice, not a rounding error."""
    import numpy as np
    import torch
    N = args.accuracy_steps
    wl = workload(None, "sphere")
    res, t_ms = {}, {}
    for st in ("fp64", "fp32", "fp16", "bf16", "fp32_exact_gamma"):
        lat, _ = make_lattice(st.split("_")[0], wl, device, gamma_mode=1 if "exact" in st else 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.step(N // 2)
        lat.reset_average()
        lat.step(N - N // 2)
        F, _ = lat.forces(averaged=True)
        t_ms[st] = 1e3 * (time.perf_counter() - t0) / N
        b = lat.body()
        res[st] = (np.array(F), np.array(b["U"]))
        lat.close()
        del lat
        torch.cuda.empty_cache()
    F64, U64 = res["fp64"]
    out = {"workload": wl["name"], "steps": N, "force_window": "mean over the second half",
           "reference": "fp64 storage on the GPU", "fp64": {"F_mean_z": F64[2], "U_z": U64[2],
                                                           "ms_per_step": round(t_ms["fp64"], 4)}}
    for st in ("fp32", "fp16", "bf16", "fp32_exact_gamma"):
        F, U = res[st]
        out[st] = {"F_mean_z": F[2], "U_z": U[2], "drag_rel_err": abs(F[2] - F64[2]) / abs(F64[2]),
                   "U_rel_err": abs(U[2] - U64[2]) / abs(U64[2]), "ms_per_step": round(t_ms[st], 4)}
    return out


def refined_counts(shape, lo, hi):
    """(coarse nodes updated, fine interior nodes, node updates per coarse
    step) of a refined step: the coarse level skips the block's inside
    (closed axes strictly between lo and hi, a spanned axis - lo = 0, hi = n
    - whole), the fine level updates its interior twice (closed axes 1 .. 2m
    - 1 of its 2m + 2 nodes, a spanned axis all 2n)."""
    full = [l == 0 and h == n for l, h, n in zip(lo, hi, shape)]
    inside = fine_interior = 1
    for a in range(3):
        m = hi[a] - lo[a]
        inside *= shape[a] if full[a] else m - 1
        fine_interior *= 2 * shape[a] if full[a] else 2 * m - 1
    coarse_updated = shape[0] * shape[1] * shape[2] - inside
    return coarse_updated, fine_interior, coarse_updated + 2 * fine_interior


def refine_bench(args, world, device, clocks):
    """The two-level block refinement (lbm_refine_step; Sec. 4.2's two-level
    grid) on two workloads: the bodiless refined block (FP32 and FP16) and
    the plunging airfoil on the fine level of a block spanning the periodic
    span (FP32).  Per coarse step: the coarse launch off the block's inside,
    two fine steps over the block's interior (with the airfoil's chain) and
    the surface/restriction kernels.  GLUPS counts every node update (coarse
    nodes updated + 2 x fine interior nodes per coarse step); the fine-grid
    equivalent counts the updates a uniform fine grid over the whole coarse
    box would make in the same simulated time (16 per coarse node and coarse
    step).  The roofline is that of the fine bulk launches (CUDA events on
    the shared stream around each)."""
    import synth
    out = {}
    for wl, storages in ((synth.refined_block(), ("fp32", "fp16")), (synth.refined_airfoil(), ("fp32",))):
        out[wl["name"]] = refine_run(args, world, device, clocks, wl, storages)
        if world == 1 and not args.no_cpu_baseline:
            out[wl["name"]]["cpu_baseline"] = refine_cpu_baseline(wl, "airfoil" in wl["name"])
    return out


def refine_run(args, world, device, clocks, wl, storages):
    import numpy as np
    import torch

    import paper_1608_04658_gb300 as lbm
    import synth
    (nx, ny, nz), lo, hi = wl["shape"], wl["lo"], wl["hi"]
    full = [l == 0 and h == n for l, h, n in zip(lo, hi, wl["shape"])]
    coarse_updated, fine_interior, per_step = refined_counts(wl["shape"], lo, hi)
    K, W = args.steps, args.warmup
    peak, peak_kind = measured_hbm_peak()
    body = "airfoil" in wl["name"]
    out = {"coarse_nodes_updated_per_step": coarse_updated, "fine_interior_nodes": fine_interior,
           "node_updates_per_coarse_step": per_step, "faces": list(wl["faces"]), "nu_coarse": wl["nu"],
           "spanned_axes": [a for a in range(3) if full[a]], "steps": K, "warmup": W}
    for st in storages:
        lat = lbm.Lattice(wl["shape"], wl["nu"], storage=st, faces=wl["faces"], u_face=wl["u_face"], device=device)
        ref = lbm.Refinement(lat, lo, hi)
        if body:
            ref.fine.set_geometry(lbm.airfoil(wl["le"], wl["chord"], wl["ca"], wl["sa"], wl["h_amp"], wl["h_omega"],
                                              wl["camber_m"], wl["camber_p"], wl["thick"]))
            lat.init_state(*synth.uniform_fields(wl["shape"], wl["u_face"]))
            ref.fine.init_state(*synth.uniform_fields(wl["fine_shape"], wl["u_face"]))
        else:
            lat.init_state(*synth.refined_fields(wl, "coarse"))
            ref.fine.init_state(*synth.refined_fields(wl, "fine"))
        ref.init()
        ref.step(W)
        torch.cuda.synchronize()
        dist_barrier(world)
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        ref.fine.profile_begin(2 * K)
        t0 = time.time()
        start.record(lat.stream)
        ref.step(K)
        end.record(lat.stream)
        torch.cuda.synchronize()
        t1 = time.time()
        dist_barrier(world)
        clocks.mark(t0, t1)
        fine_ms, nfine = ref.fine.profile_end()
        ms = dist_max(start.elapsed_time(end), world)
        tot = lat.totals()  # raises if a node went unstable
        if not np.all(np.isfinite(tot)):
            raise RuntimeError("refined run went unstable")
        res = {}
        if body:
            F, _ = ref.fine.forces()  # raises if the band reached the block's surface
            res["airfoil_force_fine_units"] = [float(v) for v in F]
        fine_ms /= max(nfine, 1)
        bytes_launch = fine_interior * BYTES_PER_NODE[st]
        achieved = bytes_launch / (fine_ms * 1e-3) / 1e9
        res.update({"value": round(per_step * K * world / (ms * 1e-3) / 1e9, 4), "unit": "GLUPS",
                    "dtype": DTYPE[st], "ms_per_step": round(ms / K, 5),
                    "fine_grid_equivalent_glups": round(16 * nx * ny * nz * K * world / (ms * 1e-3) / 1e9, 4),
                    "gpu_launches": lat.launches(),
                    "roofline": {"bound": "hbm", "kernel": "bulk_pair_kernel (fine level)",
                                 "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                                 "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                                 "traffic": ncu_traffic(st, wl["name"]),
                                 "algorithmic_bytes_per_launch": bytes_launch,
                                 "bulk_ms_per_launch": round(fine_ms, 5),
                                 "note": "the coarse launch and the coupling kernels run beside the fine launches"},
                    "step_algorithmic_gbs": round(per_step * BYTES_PER_NODE[st] / (ms / K) / 1e6, 1),
                    "step_frac_of_peak": round(per_step * BYTES_PER_NODE[st] / (ms / K) / 1e6 / peak, 4)})
        out[st] = res
        ref.close()
        ref.fine.close()
        lat.close()
        del ref, lat
        torch.cuda.empty_cache()
    return out


def cpu_sample(wl):
    """Bounded sample of a workload for the FP64 oracle on the host:
    (workload of the sample, steps, description).  The swimmer's sample is one
    step of a periodic crop around the whole body (same mesh, kinematics and
    viscosity; the oracle's brute-force mesh geometry costs about as much as
    the crop's bulk nodes); the sphere's two steps and the other boxes' one
    step of the full box."""
    if wl["kind"] == "swimmer":
        import synth
        L = wl["L"]
        shape = (int(round(L)) + 48, 2 * int(math.ceil(0.165 * L)) + 20, 2 * int(math.ceil(0.08 * L)) + 10)
        head = (16.137, shape[1] / 2 + 0.371, shape[2] / 2 + 0.293)
        smp = synth.anguilliform_swimmer(shape=shape, L=L, period=wl["period"], amp=wl["amp"],
                                         wavelength=wl["wavelength"], ramp=bool(wl["ramp"]), head=head)
        smp["kind"] = "swimmer"
        return smp, 1, (f"one step of a {shape[0]}x{shape[1]}x{shape[2]} periodic crop around the whole "
                        f"swimmer (same mesh, kinematics and viscosity)")
    n = 2 if wl["kind"] == "sphere" else 1
    nx, ny, nz = wl["shape"]
    return wl, n, f"{n} step(s) of the full {nx}x{ny}x{nz} box"


def cpu_baseline(wl):
    """The FP64 oracle, single-threaded, on the bounded sample of the
    workload (cpu_sample)."""
    import oracle
    smp, nsteps, desc = cpu_sample(wl)
    shape = smp["shape"]
    orc = oracle.Oracle(shape, nu=smp["nu"], faces=smp["faces"], u_face=smp.get("u_face", (0.0, 0.0, 0.0)),
                        body=oracle_body(smp))
    orc.init_state(*initial_flow(smp))
    t0 = time.perf_counter()
    orc.step(nsteps)
    t = time.perf_counter() - t0
    n = shape[0] * shape[1] * shape[2]
    return {"value": n * nsteps / t / 1e9, "unit": "GLUPS", "cores": 1, "kind": "oracle",
            "sample": desc + ", FP64, one thread", "seconds": round(t, 2)}


def refine_cpu_baseline(wl, body: bool):
    """The FP64 oracle's refined step (RefinedOracle), single-threaded, on a
    bounded sample of a refined workload: the same faces, viscosity and flow
    on a crop with a block of the same kind (closed, or spanning z with the
    airfoil on the fine level, chord scaled to the crop), a few coarse steps;
    the value counts node updates as the GPU line does."""
    import math as _m

    import oracle
    import synth
    if body:
        shape, lo, hi, steps = (64, 48, 4), (8, 8, 0), (55, 39, 4), 24
        chord, le = 32.0, (16.37, 32.29)
        f = 3.93 * wl["u_inf"] / (_m.pi * chord)
        fb = oracle.airfoil_body(le, chord, wl["ca"], wl["sa"], 0.05 * chord, 2 * _m.pi * f,
                                 wl["camber_m"], wl["camber_p"], wl["thick"])
        desc = (f"{steps} coarse steps of a {shape[0]}x{shape[1]}x{shape[2]} box, block [8, 55] x [8, 39] "
                f"spanning z, the airfoil (chord {chord:g}) on the fine level")
    else:
        shape, lo, hi, steps, fb = (64, 32, 16), (16, 8, 2), (47, 23, 13), 24, None
        desc = f"{steps} coarse steps of a {shape[0]}x{shape[1]}x{shape[2]} box, block [16, 47] x [8, 23] x [2, 13]"
    o = oracle.Oracle(shape, nu=wl["nu"], faces=wl["faces"], u_face=wl["u_face"])
    o.init_state(*synth.uniform_fields(shape, wl["u_face"]))
    r = oracle.RefinedOracle(o, lo, hi, fine_body=fb)
    r.fine.init_state(*synth.uniform_fields(r.fine.shape, wl["u_face"]))
    r.init()
    per_step = refined_counts(shape, lo, hi)[2]
    t0 = time.perf_counter()
    r.step(steps)
    t = time.perf_counter() - t0
    return {"value": per_step * steps / t / 1e9, "unit": "GLUPS", "cores": 1, "kind": "oracle",
            "sample": desc + ", FP64, one thread", "seconds": round(t, 2)}


def _oracle_replica(wl, nsteps, barrier, out, warm=0):
    """One independent FP64 oracle replica of the workload, in a spawned
    process: set up, run `warm` untimed steps, wait for the others, time its
    steps."""
    import oracle
    orc = oracle.Oracle(wl["shape"], nu=wl["nu"], faces=wl["faces"], u_face=wl.get("u_face", (0.0, 0.0, 0.0)),
                        body=oracle_body(wl))
    orc.init_state(*initial_flow(wl))
    if warm:
        orc.step(warm)
    barrier.wait(timeout=900)
    t0 = time.perf_counter()
    orc.step(nsteps)
    out.put((t0, time.perf_counter()))


def _replica_cap(wl, cores):
    """Replicas whose buffers (about 650 bytes per node each) fit in half of
    the free host memory, at most one per core."""
    nx, ny, nz = wl["shape"]
    free = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    return max(1, min(cores, int(0.5 * free // (650 * nx * ny * nz))))


def _run_replicas(wl, steps_each, warm_each=None):
    """Starts one spawned oracle process per entry of steps_each, together
    behind a barrier; returns the span from the first timed start to the last
    finish."""
    import multiprocessing as mp
    import queue
    procs = len(steps_each)
    warm_each = warm_each or [0] * procs
    ctx = mp.get_context("spawn")   # the parent may hold a CUDA context
    barrier, out = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_replica, args=(wl, steps_each[k], barrier, out, warm_each[k]))
          for k in range(procs)]
    for p in ps:
        p.start()
    spans, deadline = [], time.monotonic() + 1800
    try:
        while len(spans) < procs:
            try:
                spans.append(out.get(timeout=2))
            except queue.Empty:
                dead = [p.exitcode for p in ps if p.exitcode not in (None, 0)]
                if dead or time.monotonic() > deadline:
                    raise RuntimeError(f"oracle replicas failed (exit codes {dead})")
    finally:
        for p in ps:
            p.join(timeout=60 if len(spans) == procs else 0)
            if p.is_alive():
                p.terminate()
                p.join(timeout=10)
    return max(b for _, b in spans) - min(a for a, _ in spans)


def cpu_baseline_all_cores(wl, nsteps=None, procs=None):
    """The same oracle on every host core the process may use: one
    independent single-threaded replica of the workload's bounded sample per
    core (the oracle has no threads of its own), started together; the value
    is all replicas' node updates over the span from the first start to the
    last finish.  Replicas are capped so that their buffers fit in half of the
    free host memory."""
    smp, n_default, desc = cpu_sample(wl)
    nsteps = n_default if nsteps is None else nsteps
    nx, ny, nz = smp["shape"]
    n = nx * ny * nz
    cores = len(os.sched_getaffinity(0))
    if procs is None:
        procs = _replica_cap(smp, cores)
    t = _run_replicas(smp, [nsteps] * procs)
    return {"value": procs * n * nsteps / t / 1e9, "unit": "GLUPS", "cores": procs, "kind": "oracle",
            "sample": f"{procs} independent replicas (one process each) of {nsteps} step(s) of the "
                      f"{nx}x{ny}x{nz} sample ({desc}), FP64, started together",
            "seconds": round(t, 2)}


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the compute path is liblbm.so)")
    import paper_1608_04658_gb300 as lbm
    lbm.build()
    local = local % torch.cuda.device_count()
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    if args.adjoint_only:
        adj = adjoint_bench(args, world, device)
        if rank == 0:
            print(json.dumps({"adjoint": adj}), flush=True)
        return
    if args.refinement_only:
        clocks = ClockSampler(local)
        clocks.start()
        ref = refine_bench(args, world, device, clocks)
        clk = clocks.stop()
        if rank == 0:
            print(json.dumps({"refinement": ref, "clocks": clk}), flush=True)
        return
    wl = workload(args.shape, args.workload)
    # several GPUs split the box along z (one slab per rank, halo exchange);
    # --parallel replicas runs independent copies instead
    split = args.parallel == "split" or (args.parallel == "auto" and world > 1)
    clocks = ClockSampler(local)
    clocks.start()
    if split:
        return run_split(args, wl, world, rank, device, clocks)
    main = time_storage(args.storage, wl, args, world, device, clocks, gamma_mode=1 if args.gamma == "exact" else 0)
    variants = {}
    if not args.no_variants:
        for st in ("fp16", "bf16", "fp32"):
            if st == args.storage:
                continue
            r = time_storage(st, wl, args, world, device, clocks)
            variants[st] = r
        # the exact stabilizer (root of Eq. gamma_min per node) instead of the analytic one
        variants[args.storage + "_exact_gamma"] = time_storage(args.storage, wl, args, world, device, clocks,
                                                               gamma_mode=1)
    second = {}
    if args.second_workload != "none" and args.second_workload != args.workload:
        wl2 = workload(None, args.second_workload)
        second[wl2["name"]] = (wl2, {st: time_storage(st, wl2, args, world, device, clocks)
                                     for st in (["fp32", "fp16", "bf16"] if not args.no_variants else ["fp32"])})
    refined = refine_bench(args, world, device, clocks) if not args.no_refinement else None
    adj = adjoint_bench(args, world, device) if args.adjoint_horizon > 0 else None
    acc = accuracy_bench(args, device) if args.accuracy_steps > 0 and rank == 0 else None
    clk = clocks.stop()
    e2e = None if args.no_e2e else e2e_storage(args.storage, wl, args, device)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)
        try:
            cpu["all_cores"] = cpu_baseline_all_cores(wl)
        except (RuntimeError, OSError) as e:   # the single-thread figure stands alone
            cpu["all_cores"] = {"unavailable": str(e)}
    if rank != 0:
        return
    peak, peak_kind = measured_hbm_peak()

    def roofline(st, r, key=None, name=wl["name"]):
        bytes_launch = r["bulk_nodes"] * BYTES_PER_NODE[st]
        achieved = bytes_launch / (r["bulk_ms"] * 1e-3) / 1e9
        # counters committed for this storage form (key: the variant, e.g.
        # fp32_exact_gamma for the exact stabilizer's kernel)
        tr = ncu_traffic(key or st, name)
        return {"bound": "hbm", "kernel": "bulk_kernel", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "traffic": tr, "algorithmic_bytes_per_launch": bytes_launch,
                "bulk_ms_per_launch": round(r["bulk_ms"], 5)}

    nx, ny, nz = wl["shape"]
    N = nx * ny * nz
    line = {
        "metric": METRIC, "value": round(main["glups"], 4), "unit": "GLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(main["ms"] / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.storage],
        "data": "synthetic",
        "config": {"workload": wl["name"], "storage": args.storage, "stabilizer": args.gamma, "nodes": N,
                   "bytes_per_node_update": BYTES_PER_NODE[args.storage],
                   "hbm_roofline_glups": round(peak / BYTES_PER_NODE[args.storage], 3),
                   "percent_of_hbm_roofline_step": round(100 * main["glups"] * BYTES_PER_NODE[args.storage]
                                                         / world / peak, 2),
                   "l2": "inputs larger than L2 (population buffers %d MB each)"
                         % (27 * N * (BYTES_PER_NODE[args.storage] // 54) // 2 ** 20),
                   "parallelism": "replicas" if world > 1 else "single",
                   "boundary_nodes": main["body"]["n_boundary"], "links": main["body"]["n_links"],
                   "launch_order": main["order"],
                   "trial_steps_after_warmup": main["trial_steps_after_warmup"]},
        "roofline": roofline(args.storage, main, key=args.storage + ("_exact_gamma" if args.gamma == "exact" else "")),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": main["launches"],
        "clocks": clk,
        "adjoint": adj,
        "accuracy": acc,
        "refinement": refined,
        "variants": {st: {"value": round(r["glups"], 4), "unit": "GLUPS", "dtype": DTYPE[st.split("_")[0]],
                          "ms_per_step": round(r["ms"] / args.steps, 5),
                          "percent_of_hbm_roofline_step": round(100 * r["glups"] * BYTES_PER_NODE[st.split("_")[0]]
                                                                / world / peak, 2),
                          "roofline": roofline(st.split("_")[0], r, key=st),
                          "gpu_launches": r["launches"]}
                     for st, r in variants.items()},
        "workloads": {name: {st: {"value": round(r["glups"], 4), "unit": "GLUPS", "dtype": DTYPE[st],
                                  "ms_per_step": round(r["ms"] / args.steps, 5),
                                  "percent_of_hbm_roofline_step": round(100 * r["glups"] * BYTES_PER_NODE[st]
                                                                        / world / peak, 2),
                                  "roofline": roofline(st, r, name=name), "gpu_launches": r["launches"],
                                  "launch_order": r["order"]}
                             for st, r in res.items()}
                      for name, (w2, res) in second.items()},
    }
    print(json.dumps(line))


def run_split(args, wl, world, rank, device, clocks):
    """The JSON line of the z-slab split: the headline storage form on the
    workload's box and, unless left out, the second workload's box in FP32;
    the variants, the adjoint and the accuracy runs are single-GPU figures and
    are not repeated here."""
    main = time_split(args.storage, wl, args, world, device, clocks)
    second = {}
    if args.second_workload != "none" and args.second_workload != args.workload:
        wl2 = workload(None, args.second_workload)
        second[wl2["name"]] = {"fp32": time_split("fp32", wl2, args, world, device, clocks)}
    clk = clocks.stop()
    e2e = None if args.no_e2e else e2e_split(args.storage, wl, args, world, device)
    if rank != 0:
        return
    peak, peak_kind = measured_hbm_peak()
    B = BYTES_PER_NODE[args.storage]

    def roofline(st, r):
        if r["bulk_nodes"] <= 0 or r["bulk_ms"] <= 0:
            return None
        bytes_launch = r["bulk_nodes"] * BYTES_PER_NODE[st]
        achieved = bytes_launch / (r["bulk_ms"] * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": "bulk_kernel (rank 0's slab, interior layers)",
                "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "traffic": None, "algorithmic_bytes_per_launch": bytes_launch,
                "bulk_ms_per_launch": round(r["bulk_ms"], 5)}

    nx, ny, nz = wl["shape"]
    N = nx * ny * nz
    line = {
        "metric": METRIC, "value": round(main["glups"], 4), "unit": "GLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(main["ms"] / args.steps, 5),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": DTYPE[args.storage],
        "data": "synthetic",
        "config": {"workload": wl["name"], "storage": args.storage, "nodes": N, "bytes_per_node_update": B,
                   "hbm_roofline_glups": round(peak / B, 3),
                   "percent_of_hbm_roofline_step": round(100 * main["glups"] * B / world / peak, 2),
                   "l2": "inputs larger than L2 (population buffers %d MB per rank)"
                         % (27 * N // world * (B // 54) // 2 ** 20),
                   "parallelism": f"z slabs x{main['slabs']}" + (" (one GPU)" if world == 1 else ""),
                   "slab_layers_rank0": main["slab_layers"],
                   "halo_layers": 2, "launch_order": main["order"],
                   "trial_steps_after_warmup": main["trial_steps_after_warmup"]},
        "roofline": roofline(args.storage, main),
        "cpu_baseline": None,
        "e2e": e2e,
        "gpu_launches": main["launches"],
        "clocks": clk,
        "workloads": {name: {st: {"value": round(r["glups"], 4), "unit": "GLUPS", "dtype": DTYPE[st],
                                  "ms_per_step": round(r["ms"] / args.steps, 5),
                                  "roofline": roofline(st, r), "gpu_launches": r["launches"]}
                             for st, r in res.items()}
                      for name, res in second.items()},
    }
    print(json.dumps(line))


def run_reference(args):
    """The FP64 oracle as the reference arm, on the host cores: the K timed
    steps are oracle steps of the workload's bounded sample (cpu_sample),
    shared out over one process per core (at most K, capped by host memory),
    each of which first runs its share of the W warm-up steps; the value is
    all timed node updates over the span from the first timed start to the
    last finish."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.shape, args.workload)
    smp, _, desc = cpu_sample(wl)
    K, W = max(1, args.steps), max(0, args.warmup)
    P = min(_replica_cap(smp, len(os.sched_getaffinity(0))), K)
    shares = [K // P + (1 if k < K % P else 0) for k in range(P)]
    warm = [-(-W // P)] * P
    t = _run_replicas(smp, shares, warm)
    nx, ny, nz = smp["shape"]
    v = nx * ny * nz * K / t / 1e9
    sample = (f"{desc}; the {K} timed steps shared out over {P} single-threaded processes started together "
              f"(each after {warm[0]} untimed warm-up step(s)), FP64")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "sample_box": list(smp["shape"]), "processes": P},
        "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": P, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }))


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
