"""Every call of the library enqueues all of its work on the stream it is given
(each entry point of include/sdmhd.h takes a cudaStream_t).  PyTorch's side
streams do not synchronise with the default stream, so any work of a call that
went to another stream would race with the work the caller ordered on its own:
a run on a side stream, while the default stream is kept busy, must give the
same bits as the same run on the default stream."""
import pytest

from paper_2502_17805_gb300 import serve

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


def _shell_case(N):
    from paper_2502_17805_gb300 import inputs, sdmhd
    v, h = inputs.shell_mesh(4, 2)
    mesh = sdmhd.Mesh(N, v, h, geom=1, r_in=0.70, r_out=0.98, bc_in=sdmhd.BC_WALL_CONDUCTING,
                      bc_out=sdmhd.BC_WALL_RADIAL)
    phys = sdmhd.Phys(gamma=5.0 / 3.0, GM=1.0, omega=1.0, glm_alpha=1.0, c_h=0.0, powell=1, gravity=1,
                      coriolis=1)
    q0bg = mesh.empty_state()
    q0 = mesh.state_init(phys, sdmhd.INIT_SHELL_POLYTROPE, [2.0, 0.70, 0.98, 1.0, 1.0, 1e-3, 1e-4], seed=3,
                         background=q0bg)
    bg = mesh.background(phys, q0bg)
    return mesh, phys, q0, bg


def _keep_default_stream_busy(torch):
    """a chain of dense products on the default stream (tens of milliseconds), returned so that it
    stays alive until the end of the test"""
    a = torch.randn(4096, 4096, device="cuda")
    for _ in range(24):
        a = torch.tanh(a @ a * (1.0 / 64.0))
    return a


@gpu
@pytest.mark.parametrize("mixed", [False, True])
def test_advance_and_diagnostics_on_a_side_stream(torch_dev, mixed):
    torch = torch_dev
    from paper_2502_17805_gb300 import sdmhd
    mesh, phys, q0, bg = _shell_case(4)
    prec = sdmhd.SD_FP32_MIXED if mixed else sdmhd.SD_FP64
    b = bg if mixed else None
    qa, wa = q0.clone(), mesh.empty_state()
    mesh.advance(phys, 0.2, 4, qa, wa, prec=prec, bg=b)
    da = mesh.diagnostics(phys, qa)
    torch.cuda.synchronize()

    qb, wb = q0.clone(), mesh.empty_state()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())  # qb, wb and the background are ready
    busy = _keep_default_stream_busy(torch)
    mesh.advance(phys, 0.2, 4, qb, wb, prec=prec, bg=b, stream=side)
    db = mesh.diagnostics(phys, qb, stream=side)
    torch.cuda.synchronize()
    del busy
    assert torch.equal(qa, qb)
    assert da == db


@gpu
def test_packed_steps_on_a_side_stream(torch_dev):
    """sd_step_packed over two requests of different orders (one packed launch per kernel and order)"""
    torch = torch_dev
    srv = serve.Server(hbm_budget_bytes=1 << 34, max_running=4)
    reqs = [serve.Request(rid=0, nz=3, nr=2, N=4, n_rho=2.0, omega=1.3, seed=5, steps=3, arrival=0.0),
            serve.Request(rid=1, nz=2, nr=2, N=6, n_rho=1.5, omega=0.7, seed=6, steps=3, arrival=0.0)]

    def run(stream):
        runs = [serve._Running(r, srv.mesh(r.nz, r.nr, r.N)) for r in reqs]
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())
        busy = _keep_default_stream_busy(torch) if stream is not None else None
        for _ in range(3):
            srv.packer.step([x.as_packed() for x in runs], stream=stream)
            for x in runs:
                x.advanced()
        torch.cuda.synchronize()
        del busy
        return [x.q for x in runs] + [x.dyn[:3] for x in runs]

    plain = run(None)
    side = run(torch.cuda.Stream())
    for a, b in zip(plain, side):
        assert torch.equal(a, b)


@gpu
def test_two_meshes_from_two_threads_on_two_streams(torch_dev):
    """Distinct mesh objects may be used from distinct host threads: two solves (N = 4 on the FP64
    path, N = 6 on the FP32-mixed path), each from its own thread on its own stream at the same
    time, give the same bits as each alone (no scratch, lambda slot or error state is shared)."""
    torch = torch_dev
    import threading
    from paper_2502_17805_gb300 import sdmhd
    cases = [(_shell_case(4), sdmhd.SD_FP64), (_shell_case(6), sdmhd.SD_FP32_MIXED)]

    def solve(case, prec, stream, out, i):
        (mesh, phys, q, bg), w = case, out[i][1]
        mesh.advance(phys, 0.2, 6, out[i][0], w, prec=prec, bg=bg if prec == sdmhd.SD_FP32_MIXED else None,
                     stream=stream)
        out[i].append(mesh.diagnostics(phys, out[i][0], stream=stream))

    alone = [[c[0][2].clone(), c[0][0].empty_state()] for c in cases]
    for i, (case, prec) in enumerate(cases):
        solve(case, prec, None, alone, i)
    torch.cuda.synchronize()

    both = [[c[0][2].clone(), c[0][0].empty_state()] for c in cases]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for s in streams:
        s.wait_stream(torch.cuda.current_stream())
    errors = []

    def worker(i):
        try:
            solve(cases[i][0], cases[i][1], streams[i], both, i)
        except Exception as exc:  # reported below, on the test's thread
            errors.append(exc)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    assert not errors, errors
    for a, b in zip(alone, both):
        assert torch.equal(a[0], b[0])
        assert a[2] == b[2]
