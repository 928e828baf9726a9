"""Failure detection without a GPU fault: the bounded device-side waits of the
FP32-mixed stage kernels (on the shared-memory bulk copies) report a time-out
through the mesh's error word, which sd_diagnostics returns as SD_ERR_TIMEOUT.

The test makes every wait run out by setting the mesh's poll limit to zero
polls.  A wait that runs out records the time-out and then waits (again bounded)
for its copies to land, so nothing hangs, no memory is touched out of turn and
the step's results are still those of a normal step."""
import pytest

torch = pytest.importorskip("torch")

from paper_2502_17805_gb300 import inputs, sdmhd  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_17805_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _case(N):
    v, h = inputs.shell_mesh(2, 2)
    gm = sdmhd.Mesh(N, v, h, geom=1, r_in=0.7, r_out=0.98, bc_in=sdmhd.BC_WALL_CONDUCTING,
                    bc_out=sdmhd.BC_WALL_RADIAL)
    ph = sdmhd.Phys(powell=1, c_h=0.0, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0)
    bgs = gm.empty_state()
    q0 = gm.state_init(ph, sdmhd.INIT_SHELL_POLYTROPE, [2.0, 0.7, 0.98, 1.0, 1.0, 1e-4, 1e-6], seed=0,
                       background=bgs)
    return gm, ph, q0, gm.background(ph, bgs)


@pytest.mark.parametrize("N", [4, 6])
def test_wait_that_runs_out_is_reported_and_cleared(N):
    gm, ph, q0, bg = _case(N)
    ref, work = q0.clone(), gm.empty_state()
    gm.step(ph, 0.2, ref, work, prec=sdmhd.SD_FP32_MIXED, bg=bg)
    assert gm.diagnostics(ph, ref)["status"] == 0

    q = q0.clone()
    gm.set_wait_limit(0)  # every bounded wait of the next stage launches runs out at once
    gm.step(ph, 0.2, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg)
    gm.set_wait_limit(-1)
    with pytest.raises(sdmhd.SDError) as exc:
        gm.diagnostics(ph, q)
    assert exc.value.code == 8 and "wait" in str(exc.value)  # SD_ERR_TIMEOUT
    # the copies still landed before the kernels went on: the step is the normal one
    torch.cuda.synchronize()
    assert torch.equal(q, ref)
    # reported once: with the default limit the next step and diagnostics are clean
    gm.step(ph, 0.2, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg)
    d = gm.diagnostics(ph, q)
    assert d["status"] == 0 and d["min_rho"] > 0.0
