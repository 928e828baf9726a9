"""Continuous-batching server of independent SD-MHD shell solves.

Each request is a shell solve (its own mesh shape, order N, density scale
height N_rho, rotation Omega and seed) that must advance K SSP-RK3 steps of
the FP32-mixed path.  The server

* admits arrived requests first-in first-out while their device footprint
  (two FP64 states, FP32 face traces, background tables and the transient of
  building the background) fits in the HBM budget next to the running ones;
* keeps every admitted state resident on the device;
* advances running requests together: each tick is one sd_step_packed call,
  i.e. per order N one launch of each kernel over the elements of every
  request the tick steps; by default a tick takes the requests with the least
  remaining work first, up to a solution-point budget that fills the GPU, so
  small requests are not held back behind large ones and several small ones
  share launches; requests that arrive meanwhile join at the next tick, so
  their work overlaps with the others' on the device;
* retires a request after K steps, records its latency (completion minus
  arrival, the completion taken from a CUDA event after its last tick) and
  frees its memory, which may admit waiting requests;
* never waits for the device between ticks: admission only enqueues work, up
  to two ticks are in flight, and the host blocks only on the oldest tick's
  event.

Meshes (geometry) are cached per (Nz, Nr, N) and shared between requests;
everything a step writes (states, traces, dt) belongs to the request.
"""
from __future__ import annotations

import dataclasses
import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import inputs, sdmhd

R_IN, R_OUT = 0.70, 0.98


@dataclass
class Request:
    rid: int
    nz: int
    nr: int
    N: int
    n_rho: float
    omega: float
    seed: int
    steps: int
    arrival: float  # seconds after the start of the run
    cfl: float = 0.2
    noise: float = 1e-4
    dipole: float = 1e-6
    # filled in by the server
    admitted: float = float("nan")
    done: float = float("nan")

    @property
    def n_elements(self) -> int:
        return 6 * self.nz * self.nz * self.nr

    @property
    def dof(self) -> int:
        return self.n_elements * self.N ** 3

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def poisson_requests(n: int, mean_gap_s: float, seed: int = 1234, steps: int = 50,
                     shapes: Sequence[Tuple[int, int]] = ((4, 4), (8, 4), (16, 4), (32, 4)),
                     orders: Sequence[int] = (4, 5, 6)) -> List[Request]:
    """The serving workload: Poisson arrivals, element counts 6 Nz^2 Nr from `shapes`,
    orders from `orders`, N_rho ~ U[1, 3], Omega ~ U[0.5, 2]; request i uses seed i for
    both its parameter draws and its initial noise."""
    gaps = np.random.default_rng(seed).exponential(mean_gap_s, size=n)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n):
        r = np.random.default_rng(i)
        nz, nr = shapes[int(r.integers(len(shapes)))]
        out.append(Request(rid=i, nz=nz, nr=nr, N=int(orders[int(r.integers(len(orders)))]),
                           n_rho=float(r.uniform(1.0, 3.0)), omega=float(r.uniform(0.5, 2.0)), seed=i,
                           steps=steps, arrival=float(t[i])))
    return out


class _Running:
    def __init__(self, req: Request, mesh: sdmhd.Mesh):
        import torch
        self.req = req
        self.mesh = mesh
        self.phys = sdmhd.Phys(gamma=5.0 / 3.0, GM=1.0, omega=req.omega, glm_alpha=1.0, c_h=0.0, powell=1,
                               gravity=1, coriolis=1)
        params = [req.n_rho, R_IN, R_OUT, 1.0, 1.0, req.noise, req.dipole]
        bgs = mesh.empty_state()
        self.q = mesh.state_init(self.phys, sdmhd.INIT_SHELL_POLYTROPE, params, seed=req.seed, background=bgs)
        self.bg = mesh.background(self.phys, bgs)
        del bgs
        self.work = mesh.empty_state()
        self.traces = torch.empty(mesh.info["trace_bytes"] // 4, dtype=torch.float32, device="cuda")
        self.dyn = torch.zeros(4, dtype=torch.float64, device="cuda")
        self.steps_done = 0
        self.ready = False  # the previous step left the traces and lambda_max of q
        self._rec = None

    def keep(self) -> bool:
        """another step of this request follows the one about to be issued"""
        return self.steps_done + 1 < self.req.steps

    def flags(self) -> int:
        return (sdmhd.REQ_KEEP_TRACES if self.keep() else 0) | (sdmhd.REQ_TRACES_READY if self.ready else 0)

    def as_packed(self):
        return (self.mesh, self.phys, self.bg, self.q, self.work, self.traces, self.dyn, self.req.cfl, self.flags())

    def record(self):
        """the request's C record for the next step (built once, its flags updated)"""
        if self._rec is None:
            self._rec = sdmhd.Packer.request(*self.as_packed())
        self._rec.flags = self.flags()
        return self._rec

    def advanced(self):
        """after the step from as_packed() has been issued"""
        self.ready = self.keep()
        self.steps_done += 1


def footprint_bytes(info: dict, n_pts: int) -> int:
    """Device bytes a running request holds, counting the transient of building its background
    (one more state and an FP64 residual).  The background holds rho0, p0, R0 (5 FP32 values per
    point), the face jumps and the step's FP32 scratch D and q' (18 values per point)."""
    state = info["state_bytes"]
    bg = (5 + 18) * n_pts * 4 + info["n_elements"] * 6 * 2 * info["order"] ** 2 * 4
    return 4 * state + info["trace_bytes"] + bg + 64


class Server:
    def __init__(self, hbm_budget_bytes: int, max_running: int = 256, policy: str = "aged",
                 tick_dof: int = 2_000_000, backfill_frac: float = 0.25):
        """Which running requests a tick steps (the others stay resident and wait):
        "backfill": the oldest running request every tick, so that no request waits
            behind later ones, plus the others in order of least remaining work (steps left x
            DOF) while the tick holds at most max(tick_dof, (1 + backfill_frac) x the oldest
            request's DOF) solution points: small requests ride along in the capacity a large
            one leaves, and several small ones fill one tick;
        "srpt": least remaining work first up to tick_dof solution points (at least one
            request): the smallest mean latency, but a large request waits while smaller ones
            keep arriving;
        "aged" (default): least remaining work first, each request's remaining work reduced by
            aging x dof_rate x its waiting time (the work the GPU could have done for it
            meanwhile), so that a request passed over long enough moves to the front;
        "all": every running request every tick (processor sharing)."""
        if policy not in ("backfill", "srpt", "aged", "all"):
            raise ValueError("policy must be 'backfill', 'srpt', 'aged' or 'all'")
        self.budget = int(hbm_budget_bytes)
        # backgrounds come from the stream-ordered pool: keep what retired requests free for reuse
        sdmhd.memory_pool_keep(self.budget)
        self.policy = policy
        self.tick_dof = int(tick_dof)
        self.backfill_frac = float(backfill_frac)
        # multi-step ticks: a tick of small requests takes several steps (see steps_per_tick)
        self.tick_seconds = 0.4e-3
        self.dof_rate = 2.9e9
        self.step_overhead_s = 30e-6
        self.aging = 1.0
        self._now = 0.0  # seconds since the start of the current run (the "aged" policy)
        self.packer = sdmhd.Packer(max_running)
        self.max_running = max_running
        self.meshes: Dict[Tuple[int, int, int], sdmhd.Mesh] = {}
        self.peak_bytes = 0
        self.ticks = 0

    def mesh(self, nz: int, nr: int, N: int) -> sdmhd.Mesh:
        key = (nz, nr, N)
        if key not in self.meshes:
            v, h = inputs.shell_mesh(nz, nr, R_IN, R_OUT)
            self.meshes[key] = sdmhd.Mesh(N, v, h, geom=1, r_in=R_IN, r_out=R_OUT, bc_in=sdmhd.BC_WALL_CONDUCTING,
                                          bc_out=sdmhd.BC_WALL_RADIAL)
        return self.meshes[key]

    def warm(self, requests: Sequence[Request]):
        """Build the meshes of every shape the workload uses and step one request of each shape once,
        so that the kernels' set-up and the pool's memory are in place before requests arrive (a
        running service keeps its meshes and is warm)."""
        import torch
        seen = set()
        for r in requests:
            key = (r.nz, r.nr, r.N)
            self.mesh(*key)
            if key not in seen:
                seen.add(key)
                run = _Running(dataclasses.replace(r, steps=2, arrival=0.0), self.meshes[key])
                for _ in range(2):
                    self.packer.step_records([run.record()])
                    run.advanced()
        torch.cuda.synchronize()

    def run(self, requests: Sequence[Request], depth: int = 2, states: Optional[dict] = None) -> dict:
        """Serve `requests` (arrival times relative to the call) to completion.

        Ticks are issued without waiting for the device: up to `depth` ticks are in
        flight, and admitting a request (initial state, background tables) only
        enqueues work, so the host prepares the next tick while the device runs the
        current one.  A request's completion time is the device time of the event
        recorded after its last tick.  With `states` (a dict), each finished
        request's final device state is stored there under its rid."""
        import torch
        self.peak_bytes, self.ticks = 0, 0
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: List[Request] = []
        running: List[Tuple[_Running, int]] = []
        # (event, requests completing at that tick, their _Running objects, their footprint)
        inflight: list = []
        used = 0  # footprint of the running requests and of finished ones still held by a tick in flight
        peak_running = 0
        finished: List[Request] = []
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        t0 = time.perf_counter()

        def retire_oldest():
            nonlocal used
            ev, reqs, runs_done, fp_done = inflight.pop(0)
            ev.synchronize()
            used -= fp_done  # their tensors are dropped with this tick's record
            if states is not None:
                for run in runs_done:
                    states[run.req.rid] = run.q
            t_done = ev0.elapsed_time(ev) / 1e3
            for r in reqs:
                r.done = t_done
                finished.append(r)

        i = 0
        while i < len(pending) or queue or running or inflight:
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i].arrival <= now:
                queue.append(pending[i])
                i += 1
            # admission: FIFO while the footprint fits next to the running requests and the finished
            # ones whose memory a tick in flight still holds (a request is always admitted when
            # nothing else holds memory)
            while queue and len(running) < self.max_running:
                r = queue[0]
                m = self.mesh(r.nz, r.nr, r.N)
                fp = footprint_bytes(m.info, m.info["n_points"])
                if used > 0 and used + fp > self.budget:
                    break
                queue.pop(0)
                r.admitted = time.perf_counter() - t0
                running.append((_Running(r, m), fp))
                used += fp
                self.peak_bytes = max(self.peak_bytes, used)
                peak_running = max(peak_running, len(running))
            if not running:
                if inflight:
                    retire_oldest()
                elif i < len(pending):
                    time.sleep(max(0.0, pending[i].arrival - (time.perf_counter() - t0)))
                continue
            # one tick: the chosen running requests advance one step, or several when their step is
            # short (fewer host round trips per unit of GPU work; none of them finishes early)
            self._now = time.perf_counter() - t0
            chosen = self.choose(running)
            n_steps = self.steps_per_tick([running[k][0] for k in chosen])
            for _ in range(n_steps):
                self.packer.step_records([running[k][0].record() for k in chosen])
                for k in chosen:
                    running[k][0].advanced()
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            self.ticks += 1
            keep, done_reqs, done_runs, fp_done = [], [], [], 0
            for run, fp in running:
                if run.steps_done >= run.req.steps:
                    done_reqs.append(run.req)
                    done_runs.append(run)  # released (stream-ordered) once retired
                    fp_done += fp
                else:
                    keep.append((run, fp))
            running = keep
            inflight.append((ev, done_reqs, done_runs, fp_done))
            if len(inflight) >= depth:
                retire_oldest()
        wall = max(r.done for r in finished) if finished else time.perf_counter() - t0
        lat = np.array([r.latency for r in finished])
        dof_updates = sum(r.dof * r.steps for r in finished)
        return {"requests": len(finished), "wall_s": wall, "dof_updates": dof_updates,
                "aggregate": dof_updates / wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                "peak_bytes": self.peak_bytes, "budget_bytes": self.budget, "ticks": self.ticks,
                "peak_running": peak_running}

    def steps_per_tick(self, runs) -> int:
        """Steps a tick takes: enough for about `tick_seconds` of GPU work at `dof_rate` DOF-updates/s
        (with `step_overhead_s` of launches per step), at most the fewest steps any chosen request
        has left."""
        dof = sum(r.req.dof for r in runs)
        per_step = dof / self.dof_rate + self.step_overhead_s
        k = max(1, int(self.tick_seconds / per_step))
        return min(k, min(r.req.steps - r.steps_done for r in runs))

    def choose(self, running) -> List[int]:
        """Indices into `running` ((_Running, footprint) pairs) of the requests the next tick steps."""
        if self.policy == "all":
            return list(range(len(running)))
        def work(k):
            r = running[k][0]
            w = (r.req.steps - r.steps_done) * r.req.dof
            if self.policy == "aged":
                w -= self.aging * self.dof_rate * max(0.0, self._now - r.req.arrival)
            return (w, r.req.arrival)

        order = sorted(range(len(running)), key=work)
        chosen, dof, cap = [], 0, self.tick_dof
        if self.policy == "backfill":
            head = min(range(len(running)), key=lambda k: (running[k][0].req.arrival, running[k][0].req.rid))
            chosen, dof = [head], running[head][0].req.dof
            cap = max(self.tick_dof, (1.0 + self.backfill_frac) * dof)
            order = [k for k in order if k != head]
        for k in order:
            if chosen and dof + running[k][0].req.dof > cap:
                continue  # a smaller request further on may still fit
            chosen.append(k)
            dof += running[k][0].req.dof
        return sorted(chosen)

    def final_state(self, req: Request):
        """Run one request alone to completion (for checks); returns its final state on the device."""
        m = self.mesh(req.nz, req.nr, req.N)
        run = _Running(req, m)
        for _ in range(req.steps):
            self.packer.step([run.as_packed()])
            run.advanced()
        return run.q


def run_mix(server: Server, reqs: Sequence[Request]):
    """Advance a fixed set of requests together (all admitted at once), one packed step per tick;
    returns their final states (for the alone-versus-mix check)."""
    runs = [_Running(r, server.mesh(r.nz, r.nr, r.N)) for r in reqs]
    for _ in range(max(r.steps for r in reqs)):
        active = [run for run in runs if run.steps_done < run.req.steps]
        server.packer.step([run.as_packed() for run in active])
        for run in active:
            run.advanced()
    return [run.q for run in runs]
