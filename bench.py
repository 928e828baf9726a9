#!/usr/bin/env python
"""Benchmark of the SD-MHD hot path on one GB300 (or N independent replicas).

Workload (default): the 6th-order cubed-sphere shell of 6 x 24^2 x 12 =
41,472 hexahedra (8,957,952 solution points per variable), polytrope with
N_rho = 3, GM = 1, Omega = 1, density noise 1e-4 (seed 0) and a dipole of
1e-6 of the internal energy.  A step is one full SSP-RK3 step through
sd_step: lambda_max -> dt, c_h on the device, then the three fused stages.

Headline `value`: DOF-updates/s of the FP32-mixed path (whole job);
`fp64` holds the same metric for the plain FP64 path.  Inputs are resident
in HBM and larger than L2.  `e2e` repeats the mixed step through the C ABI
with the state copied host->device before and device->host after every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SD-MHD DOF-updates/s at 6th order (FP64 vs FP32-mixed); serve p50/p99 latency"
UNIT = "DOF-updates/s"

WORKLOADS = {
    "shell41k": dict(nz=24, nr=12, N=6, Nrho=3.0,
                     desc="cubed-sphere shell 6 x 24^2 x 12 = 41,472 hexahedra, N=6 (8,957,952 DOF), "
                          "r in [0.70, 0.98], polytrope n=1.5 N_rho=3, GM=1, Omega=1, noise 1e-4 seed 0, "
                          "dipole 1e-6 of internal energy"),
    "shell221k": dict(nz=48, nr=16, N=6, Nrho=3.0,
                      desc="cubed-sphere shell 6 x 48^2 x 16 = 221,184 hexahedra, N=6 (47,775,744 DOF), "
                           "polytrope N_rho=3, same recipe"),
    "shell12k": dict(nz=16, nr=8, N=6, Nrho=3.0,
                     desc="cubed-sphere shell 6 x 16^2 x 8 = 12,288 hexahedra, N=6 (2,654,208 DOF), "
                          "polytrope N_rho=3, same recipe (profiling size: state 191 MB > L2)"),
    "shell1536": dict(nz=8, nr=4, N=6, Nrho=1.0,
                      desc="cubed-sphere shell 6 x 8^2 x 4 = 1,536 hexahedra, N=6 (331,776 DOF), N_rho=1"),
}
CFL = 0.2
GLM_ALPHA = 1.0
# coefficients of the viscous legs and their step limits: the advective CFL of the other legs and the
# library's diffusive limit dt <= visc_cfl dx_min^2 / nu_max (sd_phys.visc_cfl).  With these coefficients
# the stiff modes of the viscous stress near the top of the N_rho = 3 shell (nu = mu / rho largest) grow
# under the advective limit alone: at CFL 0.2 to NaN within 10 steps, at 0.05 and 0.02 slowly (over
# 200 steps the kinetic energy 200 and 6 times that of the inviscid run), at 0.01 barely (1.5 times);
# visc_cfl 0.0157 gives the step of CFL 0.01 on this shell.  The work of a step does not depend on dt,
# so neither does DOF-updates/s.
VISCOUS = dict(viscous=1, mu=1e-4, eta=1e-4, kappa=1e-4, kappa_r=1e-4, R_gas=1.0, visc_cfl=0.015)
VISCOUS_CFL = CFL


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="shell41k", choices=sorted(WORKLOADS))
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-rk53", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-viscous", action="store_true")
    ap.add_argument("--no-largest", action="store_true")
    ap.add_argument("--accuracy-steps", type=int, default=200)
    ap.add_argument("--accuracy-oracle-steps", type=int, default=0,
                    help="steps of the FP32-mixed path against the FP64 oracle itself on the workload's shell "
                         "(off by default: the oracle takes about 0.9 s per step of the 41,472-element shell)")
    ap.add_argument("--viscous-accuracy-steps", type=int, default=0,
                    help="steps of the viscous FP32-mixed path against the viscous FP64 path on the workload's "
                         "shell at the viscous legs' CFL (off by default: about 0.14 s of FP64 per step of the "
                         "41,472-element shell)")
    ap.add_argument("--largest-steps", type=int, default=50)
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-budget-gb", type=float, default=24.0)
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

def dist_info():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of per-rank timings (ms) over all ranks of the process group (the
    slowest rank times the job); the values unchanged when there is no process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(dof_per_rank: int, steps: int, world: int, ms: float) -> float:
    """DOF-updates/s of the whole job: every rank advances its own replica of dof_per_rank points by
    `steps` steps in the slowest rank's ms (weak scaling)."""
    return dof_per_rank * steps * world / (ms / 1e3)


def algorithmic_bytes_per_dof_step(mixed: bool) -> int:
    """State streams of one SSP-RK3 step: stage 0 reads q^n and writes q^1; stages 1 and 2 read q^n and
    q^(s) and write q^(s+1): 8 passes of 9 FP64 values (576 B).  The mixed path also reads the
    background residual R0 (3 momentum components, counted as FP64) in each of the 3 stages: 648 B."""
    b = 8 * 9 * 8
    if mixed:
        b += 3 * 3 * 8
    return b


# FP64 flops of one residual evaluation per solution point at N = 6 (extrapolation and derivative
# 163k, interior fluxes 54k, face fluxes 32k, div B 13k, sources 9k, RK sum 8k per element: 280k / 216)
ALGORITHMIC_FLOP_PER_DOF_STAGE = 1300


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources the mixed stage kernel is compiled from (its DRAM counters stay valid while these are unchanged)
KERNEL_SOURCES = ("sd_internal.h", "sd_physics.cuh", "sd_physics2.cuh", "sd_stage.cuh", "sd_stage_v2.cuh",
                  "sd_stage_mixed.cu")
# the sources of the FP64 stage (face-flux and element kernels)
FP64_SOURCES = ("sd_internal.h", "sd_physics.cuh", "sd_stage.cuh", "sd_viscous.cuh", "sd_stage_f64.cuh",
                "sd_stage_fp64.cu")


def source_hash(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_2502_17805_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def fp64_peak_tflops(n_sm: int, sm_mhz: float) -> float:
    """FP64 peak from unit counts and clocks: 2 FP64 FMA per SM and clock on GB300 (its nominal
    1.25 TFLOP/s over 152 SMs at about 2 GHz), 2 flop per FMA."""
    return n_sm * 2 * 2 * sm_mhz * 1e6 / 1e12


# the workload the committed per-launch counters were taken at (or scaled to)
COUNTER_WORKLOAD = "shell41k"


def committed_traffic(kernel_key: str, sources=KERNEL_SOURCES, workload: str = COUNTER_WORKLOAD):
    """A per-launch counter of a kernel (DRAM bytes, FP64 flops) from a committed ncu summary, if it
    was taken on these sources and the bench runs the workload it was taken at."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if workload != COUNTER_WORKLOAD or not os.path.exists(path):
        return None
    cur = source_hash(sources)
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel_key and parts[2] == cur:
                return float(parts[1])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.file.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def bench_config(wl, world: int) -> dict:
    """The workload description both arms print (the reference arm runs a bounded sample of it)."""
    return {"workload": wl["desc"], "cfl": CFL, "rk": "SSP-RK3 (Shu-Osher)",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (one FP64 state is %.0f MB)" % (
                9 * 8 * 6 * wl["nz"] ** 2 * wl["nr"] * wl["N"] ** 3 / 1e6)}


# ----------------------------------------------------------------------------- our arm

def make_case(wl, device_stream=None, timing=None):
    """Mesh, physics, initial state and background of a workload; with a dict `timing`, the wall
    time of sd_mesh_create (host face matching and the device geometry, row a1) goes to
    timing["mesh_create_ms"]."""
    import time

    import torch

    from paper_2502_17805_gb300 import inputs, sdmhd
    v, h = inputs.shell_mesh(wl["nz"], wl["nr"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh = sdmhd.Mesh(wl["N"], v, h, geom=1, r_in=0.70, r_out=0.98, bc_in=sdmhd.BC_WALL_CONDUCTING,
                      bc_out=sdmhd.BC_WALL_RADIAL)
    torch.cuda.synchronize()
    if timing is not None:
        timing["mesh_create_ms"] = (time.perf_counter() - t0) * 1e3
    phys = sdmhd.Phys(gamma=5.0 / 3.0, GM=1.0, omega=1.0, glm_alpha=GLM_ALPHA, c_h=0.0, powell=1, gravity=1,
                      coriolis=1)
    params = [wl["Nrho"], 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-6]
    bgs = mesh.empty_state()
    q0 = mesh.state_init(phys, sdmhd.INIT_SHELL_POLYTROPE, params, seed=0, background=bgs)
    bg = mesh.background(phys, bgs)
    del bgs
    return mesh, phys, q0, bg, params


def time_steps(mesh, phys, q, work, prec, bg, steps, warmup, sampler=None, barrier=None, reset_to=None, cfl=CFL):
    """The timed steps run as one sd_advance call: each step's lambda_max and face traces come from
    the last stage of the step before (one trace pass per call instead of one per step).  With
    reset_to, q is set back to that state after the warm-up steps."""
    import torch
    mesh.advance(phys, cfl, warmup, q, work, prec=prec, bg=bg)
    if reset_to is not None:
        q.copy_(reset_to)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    mesh.profile(True)
    if sampler:
        sampler.start()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    mesh.advance(phys, cfl, steps, q, work, prec=prec, bg=bg)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop() if sampler else None
    prof = mesh.profile_read()
    mesh.profile(False)
    if barrier:
        barrier()
    return ms, prof, clocks


def rk53_leg(mesh, phys, q0, bg, steps, warmup, cfl53=0.5):
    """The five-stage third-order SSP method (SSPRK(5,3), SSP coefficient r = 2.65) on the FP32-mixed
    path beside the three-stage method at the bench's CFL: the rate per step and the simulated time
    per wall-clock second of each (sd_advance from the same state, device dt)."""
    import torch

    from paper_2502_17805_gb300 import sdmhd
    out = {}
    for name, scheme, cfl in (("ssp33", sdmhd.RK_SSP33, CFL), ("ssp53", sdmhd.RK_SSP53, cfl53)):
        ph = sdmhd.Phys(**dict(vars(phys), rk_scheme=scheme))
        q, work = q0.clone(), mesh.empty_state()
        mesh.advance(ph, cfl, warmup, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg)
        dts = torch.zeros(2 * steps, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mesh.advance(ph, cfl, steps, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        dt_mean = float(dts.view(steps, 2)[:, 0].mean())
        out[name] = {"cfl": cfl, "stages": 3 if scheme == sdmhd.RK_SSP33 else 5, "steps": steps,
                     "ms_per_step": ms / steps, "value": mesh.info["n_points"] * steps / (ms / 1e3),
                     "dt_mean": dt_mean, "sim_time_per_s": dt_mean * steps / (ms / 1e3)}
        del q, work
    out["unit"] = UNIT
    out["sim_time_ratio_ssp53_vs_ssp33"] = out["ssp53"]["sim_time_per_s"] / out["ssp33"]["sim_time_per_s"]
    out["note"] = ("cfl 0.5 for the five-stage method: within r = 2.65 times the three-stage method's 0.2 "
                   "(the same strong-stability bound per forward-Euler step)")
    return out


def time_e2e(mesh, phys, q_dev, work, bg, steps, warmup, chunks=16):
    """Through the C ABI with host buffers: every step copies the whole state from pinned host memory
    to the device, runs sd_step, and copies the whole new state (and dt, c_h) back.  The copies run
    in `chunks` pieces on two copy streams: piece i of a step's input goes up as soon as piece i of
    the previous step's result has come down, so the two directions overlap; the step waits for all
    of its input."""
    import torch

    from paper_2502_17805_gb300 import sdmhd
    host = torch.empty(q_dev.shape, dtype=torch.float64, pin_memory=True)
    host.copy_(q_dev)
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    dts_h = torch.zeros(2, dtype=torch.float64, pin_memory=True)
    s = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    hflat, dflat = host.view(-1), q_dev.view(-1)
    bounds = [len(hflat) * k // chunks for k in range(chunks + 1)]
    came_down = [torch.cuda.Event() for _ in range(chunks)]
    for ev in came_down:
        ev.record(down)

    def one():
        # this step's input, piece by piece behind the previous step's result
        up.wait_stream(s)
        for k in range(chunks):
            up.wait_event(came_down[k])
            with torch.cuda.stream(up):
                dflat[bounds[k]:bounds[k + 1]].copy_(hflat[bounds[k]:bounds[k + 1]], non_blocking=True)
        s.wait_stream(up)
        mesh.step(phys, CFL, q_dev, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
        down.wait_stream(s)
        with torch.cuda.stream(down):
            for k in range(chunks):
                hflat[bounds[k]:bounds[k + 1]].copy_(dflat[bounds[k]:bounds[k + 1]], non_blocking=True)
                came_down[k].record(down)
            dts_h.copy_(dts, non_blocking=True)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        one()
    s.wait_stream(down)
    e1.record(s)
    torch.cuda.synchronize()
    nbytes = q_dev.numel() * 8
    return e0.elapsed_time(e1), nbytes, nbytes + 16


def sequential_fifo(srv, reqs, prec=None):
    """The same requests served one at a time, first in first out, without batching: each request
    (initial state, background, then its K steps in one sd_advance call) is issued once it has
    arrived and the request before it has been issued; at most two are in flight.  Latency =
    completion (device event after its last step) - arrival."""
    import numpy as np
    import torch

    from paper_2502_17805_gb300 import sdmhd, serve
    prec = sdmhd.SD_FP32_MIXED if prec is None else prec
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t0 = time.perf_counter()
    inflight, lat, dof = [], [], 0
    for r in sorted(reqs, key=lambda x: x.arrival):
        wait = r.arrival - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        run = serve._Running(r, srv.mesh(r.nz, r.nr, r.N))
        run.mesh.advance(run.phys, r.cfl, r.steps, run.q, run.work, prec=prec,
                         bg=run.bg if prec == sdmhd.SD_FP32_MIXED else None)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        inflight.append((ev, r, run))
        dof += r.dof * r.steps
        if len(inflight) >= 2:
            e, rr, _ = inflight.pop(0)
            e.synchronize()
            lat.append(ev0.elapsed_time(e) / 1e3 - rr.arrival)
    done = 0.0
    for e, rr, _ in inflight:
        e.synchronize()
        lat.append(ev0.elapsed_time(e) / 1e3 - rr.arrival)
        done = ev0.elapsed_time(e) / 1e3
    lat = np.array(lat)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "aggregate": dof / done, "wall_s": done}


def run_serving(n_requests: int, budget_gb: float, tight_budget_gb: float = 4.0):
    """Serving workload: n requests arriving Poisson (mean gap 20 ms), 6 Nz^2 Nr in {384, 1536, 6144, 24576}
    elements, N in {4, 5, 6}, N_rho ~ U[1, 3], Omega ~ U[0.5, 2], seeds 0..n-1, 50 FP32-mixed steps each,
    admitted by HBM footprint under `budget_gb`.  Latency = completion - arrival.

    Beside it: the same requests all arriving at t = 0 (saturating: the aggregate then measures capacity,
    not the arrival rate), once under `budget_gb` and once under `tight_budget_gb`; and a sequential
    first-in first-out server without batching (one request at a time through sd_advance) under both
    arrival traces.  The sequential FP64 rate is measured on a bounded sample (one request of each size,
    5 steps each)."""
    import dataclasses

    import torch

    from paper_2502_17805_gb300 import sdmhd, serve
    reqs = serve.poisson_requests(n_requests, 0.020, steps=50)
    srv = serve.Server(int(budget_gb * 1e9), max_running=max(n_requests, 1))
    srv.warm(reqs)
    torch.cuda.synchronize()

    def fresh(rs, at_zero=False):
        return [dataclasses.replace(r, arrival=0.0 if at_zero else r.arrival) for r in rs]

    def served(server, rs):
        server.peak_bytes, server.ticks = 0, 0
        o = server.run(rs)
        torch.cuda.synchronize()
        return {"p50_ms": o["p50_ms"], "p99_ms": o["p99_ms"], "mean_ms": o["mean_ms"], "aggregate": o["aggregate"],
                "wall_s": o["wall_s"], "ticks": o["ticks"], "budget_gb": o["budget_bytes"] / 1e9,
                "peak_gb": o["peak_bytes"] / 1e9}

    out = served(srv, fresh(reqs))
    sat = served(srv, fresh(reqs, at_zero=True))
    tight_srv = serve.Server(int(tight_budget_gb * 1e9), max_running=max(n_requests, 1))
    tight_srv.meshes = srv.meshes
    tight = served(tight_srv, fresh(reqs, at_zero=True))
    share = serve.Server(int(budget_gb * 1e9), max_running=max(n_requests, 1), policy="all")
    share.meshes = srv.meshes
    share_poisson = served(share, fresh(reqs))
    share_sat = served(share, fresh(reqs, at_zero=True))
    srpt = serve.Server(int(budget_gb * 1e9), max_running=max(n_requests, 1), policy="srpt")
    srpt.meshes = srv.meshes
    srpt_poisson = served(srpt, fresh(reqs))
    srpt_sat = served(srpt, fresh(reqs, at_zero=True))
    bf = serve.Server(int(budget_gb * 1e9), max_running=max(n_requests, 1), policy="backfill")
    bf.meshes = srv.meshes
    bf_poisson = served(bf, fresh(reqs))
    bf_sat = served(bf, fresh(reqs, at_zero=True))
    # a fresh server: each shape's mesh (host face matching and device geometry) is built when its
    # first request is admitted, inside that request's latency
    cold = serve.Server(int(budget_gb * 1e9), max_running=max(n_requests, 1))
    cold_poisson = served(cold, fresh(reqs))
    fifo = sequential_fifo(srv, fresh(reqs))
    fifo_sat = sequential_fifo(srv, fresh(reqs, at_zero=True))
    sample = []
    for shape in ((4, 4), (8, 4), (16, 4), (32, 4)):
        cand = [r for r in reqs if (r.nz, r.nr) == shape]
        if cand:
            sample.append(cand[0])
    dof, ms = 0, 0.0
    for r in sample:
        run = serve._Running(dataclasses.replace(r, steps=5, arrival=0.0), srv.mesh(r.nz, r.nr, r.N))
        run.mesh.step(run.phys, r.cfl, run.q, run.work, prec=sdmhd.SD_FP64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run.mesh.advance(run.phys, r.cfl, 5, run.q, run.work, prec=sdmhd.SD_FP64)
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        dof += r.dof * 5
    seq64 = dof / (ms / 1e3)
    res = dict(out)
    res.update({
        "requests": n_requests, "unit": UNIT,
        "policy": "least remaining work first, each request's remaining work less %.1f x %.2g DOF/s x its "
                  "waiting time, up to %d DOF per tick" % (srv.aging, srv.dof_rate, srv.tick_dof),
        "saturating": sat, "saturating_tight_budget": tight,
        "every_request_every_tick": {"poisson": share_poisson, "saturating": share_sat},
        "least_remaining_work_first": {"poisson": srpt_poisson, "saturating": srpt_sat},
        "oldest_first_with_backfill": {"poisson": bf_poisson, "saturating": bf_sat},
        "cold_meshes": dict(cold_poisson, note="a fresh server: every shape's mesh built on its first request's "
                                               "admission, inside the latency"),
        "sequential_fifo": fifo, "sequential_fifo_saturating": fifo_sat,
        "sequential_mixed": fifo_sat["aggregate"], "sequential_fp64": seq64,
        "sequential_fp64_sample": "one request of each of the four sizes, 5 FP64 steps each (sd_advance)",
        "vs_sequential_fp64": out["aggregate"] / seq64,
        "saturating_vs_sequential_mixed": sat["aggregate"] / fifo_sat["aggregate"],
        "p50_vs_sequential_fifo": out["p50_ms"] / fifo["p50_ms"], "p99_vs_sequential_fifo": out["p99_ms"] / fifo["p99_ms"],
        "workload": "%d requests, Poisson arrivals mean 20 ms, 6 Nz^2 x 4 shells with Nz in {4, 8, 16, 32}, "
                    "N in {4, 5, 6}, N_rho ~ U[1,3], Omega ~ U[0.5,2], seeds 0-%d, 50 FP32-mixed steps each; "
                    "saturating: the same requests all at t = 0" % (n_requests, n_requests - 1)})
    return res


def accuracy_report(steps: int = 20):
    """Error of the FP32-mixed path against the FP64 oracle over `steps` SSP-RK3 steps of the
    1,536-element shell (N = 6, N_rho = 1 recipe), both advanced with the dt and c_h sequence of the
    mixed run; per variable max |mixed - oracle| / max |oracle change|.  Also the relative drift of
    the total energy and the final max|div B| for both GPU paths."""
    import numpy as np
    import torch

    from oracle import sdref
    from paper_2502_17805_gb300 import sdmhd
    wl = WORKLOADS["shell1536"]
    mesh, phys, q0, bg, params = make_case(wl)
    from paper_2502_17805_gb300 import inputs
    v, h = inputs.shell_mesh(wl["nz"], wl["nr"])
    om = sdref.Mesh(wl["N"], v, h, geom=1, r_in=0.70, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING,
                    bc_out=sdref.BC_WALL_RADIAL)
    oph = sdref.Phys(gamma=phys.gamma, GM=phys.GM, omega=phys.omega, glm_alpha=phys.glm_alpha, c_h=0.0,
                     powell=1, gravity=1, coriolis=1)
    qo = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, params, seed=0)
    q, work = mesh.to_device(qo), mesh.empty_state()
    q64 = q.clone()
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    d0 = mesh.diagnostics(phys, q)
    for _ in range(steps):
        mesh.step(phys, CFL, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
        dt, ch = (float(x) for x in dts.cpu().numpy())
        oph.c_h = ch
        qo = om.rk_step(oph, dt, qo)
        ph64 = sdmhd.Phys(**{k: getattr(phys, k) for k in ("gamma", "GM", "omega", "glm_alpha", "powell",
                                                          "gravity", "coriolis")})
        ph64.c_h = ch
        mesh.rk_step(ph64, dt, q64, work)
    qm = mesh.to_host(q)
    q_init = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, params, seed=0)
    err = np.abs(qm - qo).max(axis=(1, 2)) / np.maximum(np.abs(qo - q_init).max(axis=(1, 2)), 1e-300)
    dm, d64 = mesh.diagnostics(phys, q), mesh.diagnostics(phys, q64)
    names = ["rho", "mx", "my", "mz", "E", "Bx", "By", "Bz", "psi"]
    return {"workload": wl["desc"], "steps": steps,
            "mixed_vs_oracle_rel_err_of_change": {k: float(x) for k, x in zip(names, err)},
            "energy_drift_mixed": dm["energy"] / d0["energy"] - 1.0,
            "energy_drift_fp64": d64["energy"] / d0["energy"] - 1.0,
            "ke_mixed": dm["ke"], "ke_fp64": d64["ke"], "eb_mixed": dm["eb"], "eb_fp64": d64["eb"],
            "max_divb_mixed": dm["max_divb"], "max_divb_fp64": d64["max_divb"]}


def accuracy_viscous_mixed_vs_fp64(mesh, phys, q0, params, steps: int):
    """The viscous FP32-mixed path against the viscous FP64 path over `steps` SSP-RK3 steps at the
    viscous legs' coefficients and CFL: the mixed run takes dt and c_h from its own lambda_max (one
    sd_advance call), the FP64 run repeats that sequence with fixed-dt steps.  Per variable
    max|dq_mixed - dq_fp64| / max|dq_fp64|, dq the change over the steps; energy, KE, magnetic
    energy and max|div B| of both."""
    import torch

    from paper_2502_17805_gb300 import sdmhd
    phys_v = sdmhd.Phys(**{k: getattr(phys, k) for k in ("gamma", "GM", "omega", "glm_alpha", "c_h", "powell",
                                                        "gravity", "coriolis")}, **VISCOUS)
    work, bgs = mesh.empty_state(), mesh.empty_state()
    mesh.state_init(phys_v, sdmhd.INIT_SHELL_POLYTROPE, params, seed=0, q=work, background=bgs)
    bg_v = mesh.background(phys_v, bgs)
    del bgs
    q = q0.clone()
    dts = torch.zeros(2 * steps, dtype=torch.float64, device="cuda")
    d0 = mesh.diagnostics(phys_v, q0)
    mesh.advance(phys_v, VISCOUS_CFL, steps, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg_v, dt_out=dts)
    d = dts.cpu().numpy()
    q64 = q0.clone()
    for k in range(steps):
        mesh.rk_step(sdmhd.Phys(**dict(vars(phys_v), c_h=float(d[2 * k + 1]))), float(d[2 * k]), q64, work)
    n3 = mesh.N ** 3
    dm = (q - q0)[:, :, :n3].reshape(9, -1)
    d64 = (q64 - q0)[:, :, :n3].reshape(9, -1)
    err = ((dm - d64).abs().amax(dim=1) / d64.abs().amax(dim=1).clamp_min(1e-300)).cpu().tolist()
    gm, g64 = mesh.diagnostics(phys_v, q), mesh.diagnostics(phys_v, q64)
    names = ["rho", "mx", "my", "mz", "E", "Bx", "By", "Bz", "psi"]
    return {"steps": steps, "cfl": VISCOUS_CFL, "t_end": float(d[0::2].sum()),
            "coefficients": {k: v for k, v in VISCOUS.items() if k not in ("viscous", "visc_cfl")},
            "visc_cfl": VISCOUS["visc_cfl"],
            "mixed_vs_fp64_rel_err_of_change": dict(zip(names, err)), "max_rel_err_of_change": max(err),
            "energy_drift_mixed": gm["energy"] / d0["energy"] - 1.0,
            "energy_drift_fp64": g64["energy"] / d0["energy"] - 1.0,
            "ke_mixed": gm["ke"], "ke_fp64": g64["ke"], "eb_mixed": gm["eb"], "eb_fp64": g64["eb"],
            "max_divb_mixed": gm["max_divb"], "max_divb_fp64": g64["max_divb"]}


def accuracy_vs_oracle_shell(wl_key: str, steps: int):
    """The FP32-mixed path against the FP64 oracle itself (OpenMP over elements on the host cores)
    over `steps` SSP-RK3 steps of a workload's shell from the oracle's initial state: the mixed run
    takes dt and c_h from its own lambda_max (one sd_advance call), the oracle repeats that sequence.
    Per variable max|mixed - oracle| / max|oracle change|, and the relative drift of the total energy
    of both (each by its own diagnostics).  Off by default: about 0.9 s of oracle per step of the
    41,472-element shell on 16 cores."""
    import time

    import numpy as np
    import torch

    from oracle import sdref
    from paper_2502_17805_gb300 import inputs, sdmhd
    wl = WORKLOADS[wl_key]
    mesh, phys, _, bg, params = make_case(wl)
    v, h = inputs.shell_mesh(wl["nz"], wl["nr"])
    om = sdref.Mesh(wl["N"], v, h, geom=1, r_in=0.70, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING,
                    bc_out=sdref.BC_WALL_RADIAL)
    oph = sdref.Phys(gamma=phys.gamma, GM=phys.GM, omega=phys.omega, glm_alpha=phys.glm_alpha, c_h=0.0,
                     powell=1, gravity=1, coriolis=1)
    q_init = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, params, seed=0)
    q, work = mesh.to_device(q_init), mesh.empty_state()
    dts = torch.zeros(2 * steps, dtype=torch.float64, device="cuda")
    mesh.advance(phys, CFL, steps, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
    d = dts.cpu().numpy()
    qm = mesh.to_host(q)
    t0 = time.perf_counter()
    qo = q_init
    for k in range(steps):
        oph.c_h = float(d[2 * k + 1])
        qo = om.rk_step(oph, float(d[2 * k]), qo)
    secs = time.perf_counter() - t0
    err = np.abs(qm - qo).max(axis=(1, 2)) / np.maximum(np.abs(qo - q_init).max(axis=(1, 2)), 1e-300)
    e0 = om.diagnostics(oph, q_init)["energy"]
    names = ["rho", "mx", "my", "mz", "E", "Bx", "By", "Bz", "psi"]
    return {"workload": wl["desc"], "steps": steps, "t_end": float(d[0::2].sum()),
            "reference": "the FP64 oracle (OpenMP over elements, %d host threads, %.0f s)" % (os.cpu_count(), secs),
            "mixed_vs_oracle_rel_err_of_change": {k: float(x) for k, x in zip(names, err)},
            "max_rel_err_of_change": float(err.max()),
            "energy_drift_mixed": mesh.diagnostics(phys, q)["energy"] / e0 - 1.0,
            "energy_drift_oracle": om.diagnostics(oph, qo)["energy"] / e0 - 1.0}


def accuracy_fp32_vs_fp64(mesh, phys, q0, bg, steps: int):
    """FP32-mixed against the FP64 path on the GPU (parity-checked against the oracle to 1e-12 per
    entry) over `steps` SSP-RK3 steps of the same shell: the mixed run takes dt and c_h from its own
    lambda_max each step (sd_advance); the FP64 run repeats that dt and c_h sequence through
    sd_rk_stage.  Per variable max|mixed - FP64| / max|FP64 - initial|; relative drift of the total
    energy, KE, E_B and max|div B| (GLM cleaning on) of both, at the start and the end."""
    import torch

    from paper_2502_17805_gb300 import sdmhd
    qm, q64, work = q0.clone(), q0.clone(), mesh.empty_state()
    dts = torch.zeros(2 * steps, dtype=torch.float64, device="cuda")
    d0 = mesh.diagnostics(phys, q0)
    mesh.advance(phys, CFL, steps, qm, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
    d = dts.cpu().numpy()
    ph64 = sdmhd.Phys(**{k: getattr(phys, k) for k in ("gamma", "GM", "omega", "glm_alpha", "powell", "gravity",
                                                       "coriolis")})
    for k in range(steps):
        ph64.c_h = float(d[2 * k + 1])
        mesh.rk_step(ph64, float(d[2 * k]), q64, work)
    torch.cuda.synchronize()
    n3 = mesh.N ** 3
    change = (q64[:, :, :n3] - q0[:, :, :n3]).abs().amax(dim=(1, 2))
    err = (qm[:, :, :n3] - q64[:, :, :n3]).abs().amax(dim=(1, 2))
    rel = (err / change.clamp_min(1e-300)).cpu().tolist()
    dm, d64 = mesh.diagnostics(phys, qm), mesh.diagnostics(phys, q64)
    del qm, q64, work
    names = ["rho", "mx", "my", "mz", "E", "Bx", "By", "Bz", "psi"]
    return {"steps": steps, "reference": "FP64 GPU path (parity-checked against the FP64 oracle), same dt and c_h",
            "mixed_vs_fp64_rel_err_of_change": dict(zip(names, rel)),
            "max_rel_err_of_change": max(rel), "t_end": float(d[0::2].sum()),
            "energy_drift_mixed": dm["energy"] / d0["energy"] - 1.0,
            "energy_drift_fp64": d64["energy"] / d0["energy"] - 1.0,
            "ke_mixed": dm["ke"], "ke_fp64": d64["ke"], "eb_start": d0["eb"], "eb_mixed": dm["eb"], "eb_fp64": d64["eb"],
            "max_divb_start": d0["max_divb"], "max_divb_mixed": dm["max_divb"], "max_divb_fp64": d64["max_divb"]}


def largest_shell_leg(steps: int, fp64_steps: int, peak: float, peak_kind: str):
    """The largest single-GPU configuration: the 221,184-element shell (N = 6, N_rho = 3), `steps`
    FP32-mixed steps and `fp64_steps` FP64 steps from the initial state (after untimed warm-up steps
    on the same state, which is then reset), DOF-updates/s, the mixed stage kernel against the HBM
    roofline, and max|div B| under GLM cleaning before and after."""
    import torch

    from paper_2502_17805_gb300 import sdmhd
    wl = WORKLOADS["shell221k"]
    mesh, phys, q0, bg, _ = make_case(wl)
    n_pts = mesh.info["n_points"]
    d0 = mesh.diagnostics(phys, q0)
    q, work = q0.clone(), mesh.empty_state()
    ms, prof, _ = time_steps(mesh, phys, q, work, sdmhd.SD_FP32_MIXED, bg, steps, 3, reset_to=q0)
    dm = mesh.diagnostics(phys, q)
    q.copy_(q0)
    ms64, prof64, _ = time_steps(mesh, phys, q, work, sdmhd.SD_FP64, None, fp64_steps, 1, reset_to=q0)
    d64 = mesh.diagnostics(phys, q)
    stage_ms = prof["stage_ms"] / max(prof["stage_launches"], 1)
    bpl = algorithmic_bytes_per_dof_step(True) / 3.0 * n_pts
    achieved = bpl / (stage_ms / 1e3) / 1e9
    del q, work, q0, bg, mesh
    torch.cuda.empty_cache()
    return {"workload": wl["desc"], "dof": n_pts,
            "mixed": {"value": n_pts * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
                      "roofline": {"kernel": "stage_kernel_v2<6>", "bound": "hbm", "achieved": achieved,
                                   "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                                   "avg_launch_ms": stage_ms, "algorithmic_bytes_per_launch": bpl},
                      "max_divb": dm["max_divb"], "energy_drift": dm["energy"] / d0["energy"] - 1.0},
            "fp64": {"value": n_pts * fp64_steps / (ms64 / 1e3), "unit": UNIT, "steps": fp64_steps,
                     "ms_per_step": ms64 / fp64_steps, "max_divb": d64["max_divb"],
                     "energy_drift": d64["energy"] / d0["energy"] - 1.0},
            "max_divb_start": d0["max_divb"], "eb_start": d0["eb"]}


class OracleSample:
    """The CPU oracle, as it stands, on a bounded sample of the workload: one step is the work of one
    SSP-RK3 step (three residual evaluations) on `n_elems` random elements of the same shell, from the
    workload's initial state.  Set-up (mesh, geometry, state) is not timed."""

    def __init__(self, wl, n_elems: int, seed: int = 1):
        import numpy as np

        from oracle import sdref
        from paper_2502_17805_gb300 import inputs
        v, h = inputs.shell_mesh(wl["nz"], wl["nr"])
        self.om = sdref.Mesh(wl["N"], v, h, geom=1, r_in=0.70, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING,
                             bc_out=sdref.BC_WALL_RADIAL)
        self.ph = sdref.Phys(gamma=5.0 / 3.0, GM=1.0, omega=1.0, glm_alpha=GLM_ALPHA, c_h=1.0, powell=1,
                             gravity=1, coriolis=1)
        rng = np.random.default_rng(seed)
        self.elems = np.sort(rng.choice(self.om.n_e, size=min(n_elems, self.om.n_e), replace=False))
        self.q = self.om.state_init(self.ph, sdref.INIT_SHELL_POLYTROPE,
                                    [wl["Nrho"], 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-6], seed=0)
        self.dof_per_step = self.elems.size * wl["N"] ** 3
        self.threads = sdref.get_threads()

    def run(self, steps: int):
        t0 = time.perf_counter()
        for _ in range(steps):
            for _stage in range(3):
                self.om.residual_elements(self.ph, self.q, self.elems)
        secs = time.perf_counter() - t0
        return self.dof_per_step * steps / secs if steps else 0.0, secs


def fp64_roofline(stage_ms: float, clocks, n_pts: int, workload: str = COUNTER_WORKLOAD):
    """The FP64 stage kernel against the FP64 pipe: the algorithmic FP64 flops of one stage (1,300 per
    solution point at N = 6) over its live average launch time, against a peak derived from unit
    counts and clocks (no measured FP64 peak is available).  The committed ncu count of the kernel's
    DFMA, DADD, DMUL (scaled to the bench shell) is reported beside it when it was taken on these
    sources."""
    import torch
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clocks["sm_max_mhz"] if clocks else 2070.0
    peak = fp64_peak_tflops(n_sm, mhz)
    flops = ALGORITHMIC_FLOP_PER_DOF_STAGE * n_pts
    achieved = flops / (stage_ms / 1e3) / 1e12
    counted = committed_traffic("stage_fp64_N6_flops", FP64_SOURCES, workload)
    return {"kernel": "face_flux_kernel<6> + stage_kernel_f64<6> (FP64 stage)", "bound": "alu", "pipe": "fp64",
            "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": "derived: %d SMs x 2 FP64 FMA/clk x 2 flop x %.0f MHz" % (n_sm, mhz),
            "algorithmic_flops_per_launch": flops, "counted_flops_per_launch": counted,
            "counted_tflops": counted / (stage_ms / 1e3) / 1e12 if counted else None}


def run_ours(args):
    import torch

    from paper_2502_17805_gb300 import build, sdmhd
    rank, world, local = dist_info()
    barrier = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        barrier = dist.barrier
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        build.build()
    if barrier:
        barrier()
    sdmhd.lib()
    wl = WORKLOADS[args.workload]
    setup = {}
    mesh, phys, q0, bg, params = make_case(wl, timing=setup)
    n_pts = mesh.info["n_points"]
    q = q0.clone()
    work = mesh.empty_state()
    sampler = ClockSampler(local)

    # headline: FP32-mixed path
    ms, prof, clocks = time_steps(mesh, phys, q, work, sdmhd.SD_FP32_MIXED, bg, args.steps, args.warmup, sampler,
                                  barrier)
    # FP64 path, same workload and initial state
    q64 = q0.clone()
    k64 = max(1, min(args.steps, args.fp64_steps))
    ms64, prof64, _ = time_steps(mesh, phys, q64, work, sdmhd.SD_FP64, None, k64, min(args.warmup, 3), None, barrier)
    # the viscous, resistive and thermal fluxes: FP64 path (BR1 gradient pass before every stage) and
    # FP32-mixed path (perturbation gradients and viscous fluxes before every stage, about a background
    # built with the same coefficients), the same steps from the same state; the mixed path's change of
    # the state against the FP64 path's, per variable
    visc = visc_mixed = None
    if not args.no_viscous:
        phys_v = sdmhd.Phys(**{k: getattr(phys, k) for k in ("gamma", "GM", "omega", "glm_alpha", "c_h", "powell",
                                                            "gravity", "coriolis")}, **VISCOUS)
        coef = {k: v for k, v in VISCOUS.items() if k not in ("viscous", "visc_cfl")}
        wv = min(args.warmup, 3)
        qv = q0.clone()
        msv, profv, _ = time_steps(mesh, phys_v, qv, work, sdmhd.SD_FP64, None, k64, wv, None, barrier,
                                   cfl=VISCOUS_CFL)
        bgs = mesh.empty_state()
        mesh.state_init(phys_v, sdmhd.INIT_SHELL_POLYTROPE, params, seed=0, q=work, background=bgs)
        bg_v = mesh.background(phys_v, bgs)
        del bgs
        qm = q0.clone()
        msm, profm, _ = time_steps(mesh, phys_v, qm, work, sdmhd.SD_FP32_MIXED, bg_v, k64, wv, None, barrier,
                                   cfl=VISCOUS_CFL)
        dv, dm = qv - q0, qm - q0
        rel = ((dm - dv).abs().amax(dim=(1, 2)) / dv.abs().amax(dim=(1, 2)).clamp_min(1e-300)).cpu().tolist()
        msv, msm = max_over_ranks([msv, msm], device="cuda")
        # against the derived FP64 peak on the inviscid path's 1,300 flop per point and stage (the
        # viscous terms' own flops on top): a lower bound of the FP64 pipe's share
        import torch as _t
        n_sm = _t.cuda.get_device_properties(_t.cuda.current_device()).multi_processor_count
        peak64 = fp64_peak_tflops(n_sm, 2070.0)
        visc64_roof = {"bound": "alu", "pipe": "fp64", "basis": "1,300 flop per point and stage (the inviscid count)",
                       "achieved": 3 * ALGORITHMIC_FLOP_PER_DOF_STAGE * n_pts * k64 / (msv / 1e3) / 1e12,
                       "peak": peak64, "unit": "TFLOP/s",
                       "peak_source": "derived: %d SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz" % n_sm}
        visc64_roof["frac"] = visc64_roof["achieved"] / peak64
        # the committed ncu count of the viscous stage's DFMA, DADD, DMUL (viscous kernel, face-flux
        # kernel with the common viscous flux, element kernel; scaled to the bench shell), when it was
        # taken on these sources: the FP64 pipe's share of the whole step
        counted_v = committed_traffic("stage_fp64_visc_N6_flops", FP64_SOURCES, args.workload)
        visc64_roof["counted_flops_per_stage"] = counted_v
        visc64_roof["counted_tflops"] = 3 * counted_v * k64 / (msv / 1e3) / 1e12 if counted_v else None
        visc64_roof["counted_frac"] = visc64_roof["counted_tflops"] / peak64 if counted_v else None
        visc = {"value": whole_job_rate(n_pts, k64, world, msv), "unit": UNIT, "steps": k64, "ms_per_step": msv / k64,
                "roofline": visc64_roof,
                "dtype": "f64", "coefficients": coef, "cfl": VISCOUS_CFL, "visc_cfl": VISCOUS["visc_cfl"],
                "kernel_ms_per_step": {"stage": profv["stage_ms"] / k64,
                                       "gradients_and_control": profv["other_ms"] / k64,
                                       "trace_lambda": profv["trace_ms"] / k64}}
        peak_v, peak_kind_v = measured_peaks()
        # against the HBM roofline on the state streams alone (the 648 B per DOF and step of the
        # inviscid mixed path): the gradient record, its traces and the viscous residual are this
        # design's own traffic on top
        visc_roof = {"bound": "hbm", "basis": "algorithmic state streams, 648 B per DOF and step",
                     "achieved": algorithmic_bytes_per_dof_step(True) * n_pts * k64 / (msm / 1e3) / 1e9,
                     "peak": peak_v, "unit": "GB/s", "peak_source": peak_kind_v}
        visc_roof["frac"] = visc_roof["achieved"] / peak_v
        visc_mixed = {"value": whole_job_rate(n_pts, k64, world, msm), "unit": UNIT, "steps": k64,
                      "roofline": visc_roof,
                      "ms_per_step": msm / k64, "dtype": "f32 (perturbation) + f64 (background, RK state)",
                      "coefficients": coef, "cfl": VISCOUS_CFL, "visc_cfl": VISCOUS["visc_cfl"],
                      "kernel_ms_per_step": {"stage": profm["stage_ms"] / k64,
                                             "viscous_gradients_fluxes_and_control": profm["other_ms"] / k64,
                                             "trace_lambda": profm["trace_ms"] / k64},
                      "change_vs_fp64": {"steps": wv + k64, "max_rel_per_variable": rel,
                                         "basis": "max |dq_mixed - dq_fp64| / max |dq_fp64| per variable, "
                                                  "dq the change of the state over the steps"}}
        del qv, qm, bg_v

    rk53 = None
    if rank == 0 and world == 1 and not args.no_rk53:
        rk53 = rk53_leg(mesh, phys, q0, bg, max(1, min(args.steps, 10)), min(args.warmup, 3))

    ms, ms64 = max_over_ranks([ms, ms64], device="cuda")
    value = whole_job_rate(n_pts, args.steps, world, ms)
    value64 = whole_job_rate(n_pts, k64, world, ms64)
    peak, peak_kind = measured_peaks()
    # dominant kernel: the fused element kernel (three launches per step)
    stage_avg_ms = prof["stage_ms"] / max(prof["stage_launches"], 1)
    bytes_per_launch = (algorithmic_bytes_per_dof_step(True) / 3.0) * n_pts
    achieved = bytes_per_launch / (stage_avg_ms / 1e3) / 1e9
    step_achieved = algorithmic_bytes_per_dof_step(True) * n_pts * args.steps / (ms / 1e3) / 1e9
    stage64_ms = prof64["stage_ms"] / max(prof64["stage_launches"], 1)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (SD operators) + f64 (background, RK state, reductions)",
        "data": "synthetic",
        "config": bench_config(wl, world), "precision": "FP32-mixed (headline); FP64 under fp64",
        "roofline": {"kernel": "stage_kernel_v2<6> (FP32-mixed fused stage)", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                     "traffic": committed_traffic("stage_mixed_N6", KERNEL_SOURCES, args.workload),
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "avg_launch_ms": stage_avg_ms,
                     "step_frac": step_achieved / peak},
        "fp64": {"value": value64, "unit": UNIT, "steps": k64, "ms_per_step": ms64 / k64, "dtype": "f64",
                 "stage_avg_ms": stage64_ms, "roofline": fp64_roofline(stage64_ms, clocks, n_pts, args.workload)},
        "viscous_fp64": visc,
        "viscous_mixed": visc_mixed,
        "ssprk53": rk53,
        "gpu_launches": int(prof["stage_launches"] + prof["trace_launches"] + prof["other_launches"]),
        "kernel_ms_per_step": {"stage": prof["stage_ms"] / args.steps, "trace_lambda": prof["trace_ms"] / args.steps,
                               "control": prof["other_ms"] / args.steps},
        # one-off, outside the rate: sd_mesh_create of this shell (host face matching, device geometry)
        "mesh_create_ms": setup.get("mesh_create_ms"),
    }
    if clocks:
        out["clocks"] = clocks
    q2 = None
    if not args.no_e2e:
        q2 = q0.clone()
        ems, h2d, d2h = time_e2e(mesh, phys, q2, work, bg, max(1, min(args.steps, 10)), 1)
        ke = max(1, min(args.steps, 10))
        out["e2e"] = {"value": n_pts * ke * world / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h, "ms_per_step": ems / ke}
    if rank == 0 and world == 1 and not args.no_accuracy:
        out["accuracy_vs_oracle"] = accuracy_report()
        out["accuracy"] = accuracy_fp32_vs_fp64(mesh, phys, q0, bg, args.accuracy_steps)
        if args.accuracy_oracle_steps > 0:
            out["accuracy_oracle"] = accuracy_vs_oracle_shell(args.workload, args.accuracy_oracle_steps)
        if args.viscous_accuracy_steps > 0:
            out["accuracy_viscous"] = accuracy_viscous_mixed_vs_fp64(mesh, phys, q0, params,
                                                                   args.viscous_accuracy_steps)
        out["accuracy"]["workload"] = wl["desc"]
    if rank == 0 and world == 1 and not args.no_largest:
        del q, work, q64, q2
        q = work = q64 = q2 = None
        import torch
        torch.cuda.empty_cache()
        out["largest"] = largest_shell_leg(args.largest_steps, args.largest_steps, peak, peak_kind)
    if rank == 0 and world == 1 and not args.no_serve:
        del q, work, q64, q2, mesh, bg, q0
        import torch
        torch.cuda.empty_cache()
        out["serve"] = run_serving(args.serve_requests, args.serve_budget_gb)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ors = OracleSample(wl, WORKLOADS[args.workload]["nz"] ** 2 * 6 * WORKLOADS[args.workload]["nr"])
        ors.run(1)
        rate, secs = ors.run(3)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": ors.threads, "kind": "oracle",
                               "sample": "3 steps, each 3 residual evaluations on all %d elements of the "
                                         "shell (%.1f s wall)" % (ors.elems.size, secs)}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The CPU oracle as it stands, on the host cores: each step is the work of one SSP-RK3 step (three
    residual evaluations) on a bounded random sample of the workload's elements."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from oracle import build as obuild
    obuild.build()
    wl = WORKLOADS[args.workload]
    ors = OracleSample(wl, 4096, seed=3)
    ors.run(args.warmup)
    rate, secs = ors.run(args.steps)
    cores, nel = ors.threads, ors.elems.size
    n_pts = 6 * wl["nz"] ** 2 * wl["nr"] * wl["N"] ** 3
    # value and ms_per_step on the same basis: one SSP-RK3 step of the whole shell at the sample's rate
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": n_pts / rate * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "precision": "FP64 oracle", "config": bench_config(wl, world),
           "sample_ms_per_step": secs * 1e3 / args.steps,
           "cpu_baseline": {"value": rate, "unit": UNIT, "kind": "oracle", "cores": cores,
                            "sample": "per step: 3 residual evaluations on %d random elements of the shell; "
                                      "ms_per_step scales the sample's time to the whole shell" % nel},
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
