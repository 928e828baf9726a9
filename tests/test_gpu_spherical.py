"""Parity of sd_spherical_sums (longitude averages of Sec. Results) with the oracle's fixed-order sums
on the shell, for bin tables that fit an element's window in shared memory and for tables that do not
(point-by-point global additions)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sdref  # noqa: E402
from paper_2502_17805_gb300 import inputs, sdmhd  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_17805_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("N,n_r,n_t", [(4, 3, 7), (6, 2, 5), (5, 4, 256)])
def test_spherical_sums_match_the_oracle(N, n_r, n_t):
    v, h = inputs.shell_mesh(8, 4)
    kw = dict(geom=1, r_in=0.70, r_out=0.98)
    gm, om = sdmhd.Mesh(N, v, h, **kw), sdref.Mesh(N, v, h, **kw)
    q0 = inputs.random_state(gm.n_e, N, seed=12)
    G = gm.spherical_sums(gm.to_device(q0), 0.70, 0.98, n_r, n_t).cpu().numpy()
    O = om.spherical_sums(q0, n_r, n_t)
    # per quantity: round-off of sums whose terms are bounded by the largest bin sum of |values|
    scale = np.abs(O).reshape(-1, 8).max(axis=0)
    err = np.abs(G - O).reshape(-1, 8).max(axis=0)
    assert np.all(err <= 1e-12 * scale), (err, scale)
    assert abs(G[..., 0].sum() / O[..., 0].sum() - 1.0) < 1e-13


def test_spherical_sums_reject_bad_arguments():
    v, h = inputs.shell_mesh(2, 1)
    gm = sdmhd.Mesh(4, v, h, geom=1, r_in=0.7, r_out=0.98)
    q = gm.empty_state()
    with pytest.raises(sdmhd.SDError, match="r_min < r_max"):
        gm.spherical_sums(q, 0.98, 0.70, 2, 2)
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(sdmhd.SDError, match="n_r"):
        gm.spherical_sums(q, 0.70, 0.98, 0, 2, out=out)
    with pytest.raises(sdmhd.SDError, match="out is NULL"):
        gm.spherical_sums(q, 0.70, 0.98, 2, 2, out=torch.zeros(0, dtype=torch.float64, device="cuda"))


def test_spherical_sums_repeat_to_round_off():
    """The bin sums use atomic additions (no fixed order): two calls on the same state agree to
    round-off of each bin's sum of magnitudes."""
    N = 5
    v, h = inputs.shell_mesh(8, 4)
    gm = sdmhd.Mesh(N, v, h, geom=1, r_in=0.70, r_out=0.98)
    q = gm.to_device(inputs.random_state(gm.n_e, N, seed=13))
    a = gm.spherical_sums(q, 0.70, 0.98, 4, 16).cpu().numpy()
    b = gm.spherical_sums(q, 0.70, 0.98, 4, 16).cpu().numpy()
    scale = np.abs(a).reshape(-1, 8).max(axis=0)
    assert np.all(np.abs(a - b).reshape(-1, 8).max(axis=0) <= 1e-13 * scale)
