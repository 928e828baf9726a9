"""sd_residual_noalloc: the FP64 residual for callers that cannot allocate device
memory when they need it (a memory pool that already owns the device budget, or
a latency-bound loop that must not block on an allocation).  It runs the same
kernels as sd_residual, so it must give the same bits, on consecutive calls that
reuse its fixed scratch, and reject meshes whose scratch would not fit, viscous
physics and an output that aliases the input.

This file is collected last on purpose: a failure here leaves every other test
already run."""
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


def _shell_case(N):
    v, h = inputs.shell_mesh(3, 2)
    gm = sdmhd.Mesh(N, v, inputs.reorient(h, seed=3), geom=1, r_in=0.7, r_out=0.98,
                    bc_in=sdmhd.BC_WALL_CONDUCTING, bc_out=sdmhd.BC_WALL_RADIAL)
    ph = sdmhd.Phys(powell=1, c_h=0.9, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.2)
    return gm, ph


def _box_case(N):
    v, h, per = inputs.box_mesh(3, jitter=0.1, seed=4)
    gm = sdmhd.Mesh(N, v, inputs.reorient(h, seed=5), periodic=per, geom=0)
    ph = sdmhd.Phys(powell=1, c_h=0.7, glm_alpha=0.3)
    return gm, ph


@pytest.mark.parametrize("case,N", [("shell", 6), ("box", 3)])
def test_noalloc_residual_matches_sd_residual_on_consecutive_calls(case, N):
    """The same trace and stage kernels run on the same layout as sd_residual, so the output is the
    same bits, on two calls in a row (the second finds the first call's traces in the scratch)."""
    gm, ph = _shell_case(N) if case == "shell" else _box_case(N)
    for seed in (21, 22):
        q = gm.to_device(inputs.random_state(gm.n_e, N, seed=seed))
        ref = gm.residual(ph, q)
        out = gm.residual_noalloc(ph, q, gm.empty_state())
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (case, N, seed)


def test_noalloc_rejects_meshes_beyond_its_scratch():
    N = 6
    v, h = inputs.shell_mesh(4, 6)  # 576 elements: traces and face fluxes need 14.2 MB > 8 MiB
    gm = sdmhd.Mesh(N, v, h, geom=1, r_in=0.7, r_out=0.98)
    q = gm.empty_state()
    with pytest.raises(sdmhd.SDError) as exc:
        gm.residual_noalloc(sdmhd.Phys(), q, gm.empty_state())
    assert exc.value.code == 1 and "too large" in str(exc.value)


def test_noalloc_rejects_viscous_physics_and_aliased_output():
    gm, ph = _box_case(3)
    q = gm.to_device(inputs.random_state(gm.n_e, 3, seed=7))
    visc = sdmhd.Phys(powell=1, c_h=0.7, viscous=1, mu=1e-3, eta=1e-3, kappa=1e-3, R_gas=1.0)
    with pytest.raises(sdmhd.SDError) as exc:
        gm.residual_noalloc(visc, q, gm.empty_state())
    assert exc.value.code == 2  # SD_ERR_UNSUPPORTED: the viscous fluxes need gradient buffers
    with pytest.raises(sdmhd.SDError) as exc:
        gm.residual_noalloc(ph, q, q)
    assert exc.value.code == 1  # SD_ERR_INVALID_ARGUMENT: dqdt may not alias q
