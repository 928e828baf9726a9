"""sd_residual_noalloc: the FP64 residual for callers that cannot allocate device
memory when they need it (a memory pool that already owns the device budget, or
a latency-bound loop that must not block on an allocation).  It must give the
residual of sd_residual within the FP64 parity tolerance, on consecutive calls
that reuse its fixed scratch, and reject meshes whose scratch would not fit.

This file is collected last on purpose: a failure here leaves every other test
already run."""
import numpy as np
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


def _close(a, b, tol=1e-12):
    # FP64 parity tolerance of the suite, relative to each variable's magnitude
    scale = np.maximum(np.abs(b).max(axis=(1, 2)), 1e-300)
    return (np.abs(a - b).max(axis=(1, 2)) / scale).max() <= tol


def test_noalloc_residual_matches_sd_residual_on_consecutive_calls():
    N = 6
    v, h = inputs.shell_mesh(3, 2)
    gm = sdmhd.Mesh(N, v, inputs.reorient(h, seed=3), geom=1, r_in=0.7, r_out=0.98,
                    bc_in=sdmhd.BC_WALL_CONDUCTING, bc_out=sdmhd.BC_WALL_RADIAL)
    ph = sdmhd.Phys(powell=1, c_h=0.9, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.2)
    for seed in (21, 22):  # the second call finds the first call's traces in the scratch
        q = gm.to_device(inputs.random_state(gm.n_e, N, seed=seed))
        ref = gm.to_host(gm.residual(ph, q))
        out = gm.to_host(gm.residual_noalloc(ph, q, gm.empty_state()))
        torch.cuda.synchronize()
        assert _close(out, ref), seed


def test_noalloc_rejects_meshes_beyond_its_scratch():
    N = 6
    v, h = inputs.shell_mesh(4, 6)  # 576 elements: traces need 8.96 MB > 8 MiB
    gm = sdmhd.Mesh(N, v, h, geom=1, r_in=0.7, r_out=0.98)
    q = gm.empty_state()
    with pytest.raises(sdmhd.SDError) as exc:
        gm.residual_noalloc(sdmhd.Phys(), q, gm.empty_state())
    assert exc.value.code == 1 and "too large" in str(exc.value)
