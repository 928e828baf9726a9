"""Serving: packed steps of independent solves (sd_step_packed) and the
continuous-batching server.  A request's result must not depend on which other
requests share its launches."""
import dataclasses
import math

import numpy as np
import pytest

from paper_2502_17805_gb300 import serve


def test_poisson_workload_recipe():
    reqs = serve.poisson_requests(64, 0.020, steps=50)
    assert len(reqs) == 64
    assert [r.seed for r in reqs] == list(range(64))
    assert {r.n_elements for r in reqs} <= {384, 1536, 6144, 24576}
    assert {r.N for r in reqs} <= {4, 5, 6}
    assert all(1.0 <= r.n_rho <= 3.0 and 0.5 <= r.omega <= 2.0 for r in reqs)
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) >= 0) and arr[0] == 0.0
    assert 0.5 * 0.020 < np.diff(arr).mean() < 2.0 * 0.020
    # request i draws its parameters from seed i: the same request in another workload is identical
    again = serve.poisson_requests(8, 0.5, seed=99, steps=50)
    assert (again[3].nz, again[3].N, again[3].n_rho) == (reqs[3].nz, reqs[3].N, reqs[3].n_rho)


def test_footprint_grows_with_the_mesh():
    info_small = {"state_bytes": 9 * 384 * 64 * 8, "trace_bytes": 2 * 384 * 6 * 9 * 16 * 4, "n_elements": 384,
                  "order": 4}
    info_big = {"state_bytes": 9 * 1536 * 64 * 8, "trace_bytes": 2 * 1536 * 6 * 9 * 16 * 4, "n_elements": 1536,
                "order": 4}
    assert serve.footprint_bytes(info_big, 1536 * 64) > 3 * serve.footprint_bytes(info_small, 384 * 64)


def test_tick_policy_takes_least_remaining_work_first_up_to_the_budget():
    from types import SimpleNamespace as NS

    def run(dof, steps_left, arrival=0.0):
        return (NS(req=NS(dof=dof, steps=steps_left, arrival=arrival), steps_done=0), 0)

    srv = serve.Server.__new__(serve.Server)
    srv.policy, srv.tick_dof, srv.backfill_frac = "srpt", 1000, 0.25
    running = [run(900, 10), run(100, 50), run(300, 2), run(50, 1), run(600, 1)]
    # remaining work: 9000, 5000, 600, 50, 600 -> order 3, 2, 4 (ties keep their order), 1, 0
    assert srv.choose(running) == [2, 3, 4]  # 50 + 300 + 600 DOF; 100 more would pass the 1000 budget
    srv.tick_dof = 10
    assert srv.choose(running) == [3]  # a lone request always runs, even above the budget
    srv.policy = "all"
    assert srv.choose(running) == [0, 1, 2, 3, 4]


def test_backfill_policy_always_steps_the_oldest_request():
    from types import SimpleNamespace as NS

    def run(rid, dof, steps_left, arrival):
        return (NS(req=NS(rid=rid, dof=dof, steps=steps_left, arrival=arrival), steps_done=0), 0)

    srv = serve.Server.__new__(serve.Server)
    srv.policy, srv.tick_dof, srv.backfill_frac = "backfill", 1000, 0.25
    # the oldest (index 1) is large: the tick may hold 1.25 x its 4000 DOF, smallest remaining work first
    running = [run(0, 300, 5, 0.2), run(1, 4000, 40, 0.0), run(2, 800, 1, 0.3), run(3, 200, 2, 0.1)]
    assert srv.choose(running) == [1, 2, 3]  # 4000 + 200 (rid 3) + 800 (rid 2) = 5000; rid 0 no longer fits
    # a small oldest request: the tick fills up to tick_dof
    running[1] = run(1, 100, 3, 0.0)
    assert srv.choose(running) == [0, 1, 3]  # 100 + 200 + 300 = 600; rid 2 would make 1400


gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_17805_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


@gpu
@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_packed_step_equals_sd_step(torch_dev, N):
    """The packed launches (parameters from a device table, one launch over all requests) and sd_step
    do the same arithmetic in the same order: the same bits, for each order."""
    torch = torch_dev
    from paper_2502_17805_gb300 import sdmhd
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=8)
    req = serve.Request(rid=0, nz=3, nr=2, N=N, n_rho=2.0, omega=1.3, seed=5, steps=3, arrival=0.0)
    q_packed = srv.final_state(req)
    run = serve._Running(req, srv.mesh(req.nz, req.nr, req.N))
    for _ in range(req.steps):
        run.mesh.step(run.phys, req.cfl, run.q, run.work, prec=sdmhd.SD_FP32_MIXED, bg=run.bg)
    torch.cuda.synchronize()
    assert torch.equal(q_packed, run.q)


@gpu
def test_each_result_is_the_same_alone_and_in_the_mix(torch_dev):
    torch = torch_dev
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=8)
    reqs = [serve.Request(rid=0, nz=2, nr=2, N=4, n_rho=1.5, omega=0.7, seed=1, steps=4, arrival=0.0),
            serve.Request(rid=1, nz=3, nr=2, N=6, n_rho=2.5, omega=1.9, seed=2, steps=3, arrival=0.0),
            serve.Request(rid=2, nz=4, nr=1, N=5, n_rho=1.1, omega=1.0, seed=3, steps=5, arrival=0.0),
            serve.Request(rid=3, nz=2, nr=1, N=4, n_rho=2.9, omega=0.6, seed=4, steps=2, arrival=0.0)]
    alone = [srv.final_state(r).clone() for r in reqs]
    mixed = serve.run_mix(srv, reqs)
    torch.cuda.synchronize()
    for a, m in zip(alone, mixed):
        assert torch.equal(a, m)


@gpu
def test_admission_respects_the_hbm_budget(torch_dev):
    reqs = serve.poisson_requests(10, 0.002, steps=3, shapes=((2, 2), (4, 2)), orders=(4, 5))
    srv = serve.Server(hbm_budget_bytes=1 << 20, max_running=16)  # smaller than any two requests
    srv.warm(reqs)
    out = srv.run(reqs)
    assert out["requests"] == 10
    biggest = max(serve.footprint_bytes(m.info, m.info["n_points"]) for m in srv.meshes.values())
    assert out["peak_bytes"] <= max(srv.budget, biggest)
    assert out["peak_running"] == 1
    # all arrived at once: a roomy budget runs them together (they share ticks), the tight one in turn
    at_once = [dataclasses.replace(r, arrival=0.0) for r in reqs]
    roomy = serve.Server(hbm_budget_bytes=1 << 34, max_running=16)
    roomy.warm(reqs)
    out2 = roomy.run(at_once)
    out3 = srv.run([dataclasses.replace(r) for r in at_once])
    assert out2["requests"] == 10 and out2["peak_running"] == 10 and out3["peak_running"] == 1
    assert out2["ticks"] < out3["ticks"]


@gpu
def test_packed_step_matches_the_oracle(torch_dev):
    """One packed step of a stratified shell against the FP64 oracle, given the packed dt and c_h."""
    torch = torch_dev
    from oracle import sdref
    from paper_2502_17805_gb300 import inputs
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=4)
    req = serve.Request(rid=0, nz=3, nr=2, N=5, n_rho=2.0, omega=1.3, seed=5, steps=1, arrival=0.0)
    run = serve._Running(req, srv.mesh(req.nz, req.nr, req.N))
    q_before = run.mesh.to_host(run.q)
    srv.packer.step([run.as_packed()])
    dt, ch = run.dyn.cpu().numpy()[:2]
    v, h = inputs.shell_mesh(req.nz, req.nr)
    om = sdref.Mesh(req.N, v, h, geom=1, r_in=0.70, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING,
                    bc_out=sdref.BC_WALL_RADIAL)
    oph = sdref.Phys(gamma=5.0 / 3.0, GM=1.0, omega=req.omega, glm_alpha=1.0, c_h=float(ch), powell=1, gravity=1,
                     coriolis=1)
    qo = om.rk_step(oph, float(dt), q_before)
    dg, do = run.mesh.to_host(run.q) - q_before, qo - q_before
    # every variable within 1e-5 of its largest change over the step
    err = np.abs(dg - do).max(axis=(1, 2))
    strict = 1e-5 * np.abs(do).max(axis=(1, 2))
    print("packed step vs oracle: max|g-o|/(1e-5 max|change|) = %s" % (err / strict))
    assert np.all(err <= strict), (err, strict)
    lam = om.diagnostics(oph, q_before)["lambda_max"]
    xs = sdref.nodes(req.N)[0]
    assert abs(dt / (req.cfl * om.info()["h_min"] * (xs[1] - xs[0]) / lam) - 1.0) < 1e-6


@gpu
def test_requests_may_not_share_a_background(torch_dev):
    """The background holds the step's FP32 scratch (D and q'), so a pack with two requests on one
    background is refused before any launch."""
    from paper_2502_17805_gb300 import sdmhd
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=4)
    req = serve.Request(rid=0, nz=2, nr=1, N=4, n_rho=2.0, omega=1.0, seed=5, steps=1, arrival=0.0)
    run = serve._Running(req, srv.mesh(req.nz, req.nr, req.N))
    other = serve._Running(req, srv.mesh(req.nz, req.nr, req.N))
    a, b = run.as_packed(), list(other.as_packed())
    b[2] = a[2]  # other's states, run's background
    with pytest.raises(sdmhd.SDError, match="share a background"):
        srv.packer.step([a, tuple(b)])


@gpu
@pytest.mark.parametrize("N", [4, 6])
def test_kept_traces_give_the_same_bits(torch_dev, N):
    """With SD_REQ_KEEP_TRACES / SD_REQ_TRACES_READY the last stage of one call leaves the traces and
    lambda_max of the new state and the next call skips its trace pass; the states and (dt, c_h, lambda)
    are the same bits as plain calls (each with its own trace pass)."""
    torch = torch_dev
    from paper_2502_17805_gb300 import sdmhd
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=4)
    req = serve.Request(rid=0, nz=3, nr=2, N=N, n_rho=2.0, omega=1.3, seed=5, steps=4, arrival=0.0)
    fused = serve._Running(req, srv.mesh(req.nz, req.nr, req.N))
    plain = serve._Running(req, srv.mesh(req.nz, req.nr, req.N))
    assert fused.mesh.info["trace_bytes"] == 3 * fused.mesh.n_e * 6 * 9 * N * N * 4 + 128
    flags_seen = []
    for _ in range(req.steps):
        pf = fused.as_packed()
        flags_seen.append(pf[8])
        srv.packer.step([pf])
        fused.advanced()
        srv.packer.step([plain.as_packed()[:8]])  # flags 0
        plain.advanced()
        torch.cuda.synchronize()
        assert torch.equal(fused.q, plain.q) and torch.equal(fused.dyn[:3], plain.dyn[:3])
    K, R = sdmhd.REQ_KEEP_TRACES, sdmhd.REQ_TRACES_READY
    assert flags_seen == [K, K | R, K | R, R]


@gpu
def test_unknown_request_flags_are_refused(torch_dev):
    from paper_2502_17805_gb300 import sdmhd
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=4)
    req = serve.Request(rid=0, nz=2, nr=1, N=4, n_rho=2.0, omega=1.0, seed=5, steps=1, arrival=0.0)
    run = serve._Running(req, srv.mesh(req.nz, req.nr, req.N))
    with pytest.raises(sdmhd.SDError, match="unknown flags"):
        srv.packer.step([run.as_packed()[:8] + (4,)])


@gpu
def test_an_empty_pack_is_a_no_op(torch_dev):
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=4)
    srv.packer.step([])


@gpu
def test_staggered_arrivals_give_each_result_alone(torch_dev):
    """Requests arriving while others run (staggered arrival times through Server.run, so they join
    at different ticks and share launches with different partners) end with the same bits as each
    request run alone."""
    torch = torch_dev
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=8)
    shapes = [(2, 2, 4), (3, 2, 6), (4, 1, 5), (2, 1, 4), (3, 1, 6), (2, 2, 5)]
    reqs = [serve.Request(rid=i, nz=nz, nr=nr, N=N, n_rho=1.2 + 0.3 * i, omega=0.6 + 0.2 * i, seed=10 + i,
                          steps=6 + (i % 3), arrival=0.004 * i)
            for i, (nz, nr, N) in enumerate(shapes)]
    srv.warm(reqs)
    alone = {r.rid: srv.final_state(serve.Request(**{k: getattr(r, k) for k in
                                                     ("rid", "nz", "nr", "N", "n_rho", "omega", "seed", "steps",
                                                      "arrival")})).clone() for r in reqs}
    states = {}
    out = srv.run(reqs, states=states)
    torch.cuda.synchronize()
    assert out["requests"] == len(reqs) and sorted(states) == sorted(alone)
    for rid, q in states.items():
        assert torch.equal(q, alone[rid]), rid


@gpu
def test_packed_calls_alternating_streams(torch_dev):
    """Consecutive sd_step_packed calls on two streams in turn (the packer's double-buffered device
    tables are then reused by a call on another stream than the one whose kernels read them last) give
    the bits of the same calls on one stream."""
    torch = torch_dev
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=4)
    reqs = [serve.Request(rid=0, nz=3, nr=2, N=6, n_rho=2.0, omega=1.3, seed=5, steps=5, arrival=0.0),
            serve.Request(rid=1, nz=2, nr=2, N=4, n_rho=1.5, omega=0.8, seed=6, steps=5, arrival=0.0)]
    one = [serve._Running(r, srv.mesh(r.nz, r.nr, r.N)) for r in reqs]
    two = [serve._Running(r, srv.mesh(r.nz, r.nr, r.N)) for r in reqs]
    torch.cuda.synchronize()
    for _ in range(5):
        srv.packer.step([run.as_packed() for run in one])
        for run in one:
            run.advanced()
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    prev = torch.cuda.current_stream()
    for k in range(5):
        s = streams[k % 2]
        s.wait_stream(prev)  # the step reads the state the previous call wrote
        srv.packer.step([run.as_packed() for run in two], stream=s)
        for run in two:
            run.advanced()
        prev = s
    torch.cuda.synchronize()
    for a, b in zip(one, two):
        assert torch.equal(a.q, b.q)


def test_small_ticks_take_several_steps():
    from types import SimpleNamespace as NS
    srv = serve.Server.__new__(serve.Server)
    srv.tick_seconds, srv.dof_rate, srv.step_overhead_s = 0.4e-3, 2.9e9, 30e-6
    small = [NS(req=NS(dof=24_576, steps=50), steps_done=0), NS(req=NS(dof=48_000, steps=50), steps_done=47)]
    big = [NS(req=NS(dof=5_308_416, steps=50), steps_done=0)]
    assert srv.steps_per_tick(small) == 3          # several steps, but no more than a request has left
    assert srv.steps_per_tick(small[:1]) == 10     # 0.4 ms / (8.5 us + 30 us)
    assert srv.steps_per_tick(big) == 1            # one step of a large request already fills a tick


def test_aged_policy_moves_a_long_waiting_request_forward():
    """The aged order is that of remaining work + aging x rate x arrival time: a request that arrived
    early enough goes first even with more work left."""
    from types import SimpleNamespace as NS
    srv = serve.Server.__new__(serve.Server)
    srv.policy, srv.tick_dof, srv.backfill_frac = "aged", 1000, 0.25
    srv.aging, srv.dof_rate = 1.0, 1000.0

    def run(rid, dof, steps, arrival):
        return (NS(req=NS(rid=rid, dof=dof, steps=steps, arrival=arrival), steps_done=0), 0)

    big = run(0, 900, 10, 0.0)                 # 9000 DOF-steps left, arrived at 0
    srv._now = 9.0
    assert srv.choose([big, run(1, 800, 2, 5.0)]) == [1]  # 1600 + 5000 < 9000 + 0
    assert srv.choose([big, run(1, 800, 2, 8.0)]) == [0]  # 1600 + 8000 > 9000: the early one first


@gpu
def test_five_stage_method_is_refused_in_packed_steps(torch_dev):
    """sd_step_packed runs the three-stage stages; a request asking for SSPRK(5,3) is refused
    (sd_step runs it)."""
    import dataclasses

    from paper_2502_17805_gb300 import sdmhd
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=4)
    req = serve.Request(rid=0, nz=2, nr=1, N=4, n_rho=2.0, omega=1.0, seed=5, steps=1, arrival=0.0)
    run = serve._Running(req, srv.mesh(req.nz, req.nr, req.N))
    packed = list(run.as_packed())
    packed[1] = dataclasses.replace(packed[1], rk_scheme=sdmhd.RK_SSP53)
    with pytest.raises(sdmhd.SDError) as exc:
        srv.packer.step([tuple(packed)])
    assert exc.value.code == 2 and "three-stage" in str(exc.value)
