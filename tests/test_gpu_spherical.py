"""Parity of sd_spherical_sums (longitude averages of Sec. Results) with the oracle's fixed-order sums
on the shell, for bin tables that fit an element's window in shared memory and for tables that do not
(point-by-point global additions); the sums' independence of the element order (bitwise)."""
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


@pytest.mark.parametrize("N,n_r,n_t", [(2, 2, 3), (3, 3, 4), (4, 3, 7), (6, 2, 5), (5, 4, 256), (7, 2, 6), (8, 3, 5)])
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


def test_spherical_sums_do_not_depend_on_the_element_order():
    """The sums are exact in fixed point before one conversion: the same mesh with its elements
    listed in another order (the same geometry per element, the state permuted alike) gives the
    same bits, and so do repeated calls."""
    N = 5
    v, h = inputs.shell_mesh(8, 4)
    kw = dict(geom=1, r_in=0.70, r_out=0.98)
    q0 = inputs.random_state(len(h), N, seed=13)
    perm = np.random.default_rng(5).permutation(len(h))
    ga, gb = sdmhd.Mesh(N, v, h, **kw), sdmhd.Mesh(N, v, np.ascontiguousarray(h[perm]), **kw)
    qa, qb = ga.to_device(q0), gb.to_device(np.ascontiguousarray(q0[:, perm]))
    for n_r, n_t in [(4, 16), (3, 300)]:  # element windows in shared memory; point-by-point additions
        a = ga.spherical_sums(qa, 0.70, 0.98, n_r, n_t)
        b = gb.spherical_sums(qb, 0.70, 0.98, n_r, n_t)
        assert torch.equal(a, b), (n_r, n_t)
        assert torch.equal(a, ga.spherical_sums(qa, 0.70, 0.98, n_r, n_t))


def test_spherical_sums_of_terms_far_apart_in_size():
    """Terms of very different size in one bin: the fixed-point sum keeps the small ones (the
    density of one element raised by 1e12 leaves the other bins' mass sums as the oracle's)."""
    N = 4
    v, h = inputs.shell_mesh(4, 2)
    kw = dict(geom=1, r_in=0.70, r_out=0.98)
    gm, om = sdmhd.Mesh(N, v, h, **kw), sdref.Mesh(N, v, h, **kw)
    q0 = inputs.random_state(gm.n_e, N, seed=21)
    q0[:, 0] *= 1e12  # every component of element 0, so the velocities stay as they were
    G = gm.spherical_sums(gm.to_device(q0), 0.70, 0.98, 2, 6).cpu().numpy()
    O = om.spherical_sums(q0, 2, 6)
    for c in (0, 4, 5, 6, 7):  # non-negative terms; per bin: round-off of that bin's own sum
        mag = np.abs(O[..., c])
        assert np.all(np.abs(G[..., c] - O[..., c]) <= 1e-12 * np.maximum(mag, 1e-300)), c


def test_spherical_sums_nan_term():
    """A NaN momentum at one point: the velocity quantities and the kinetic energy sum to NaN; the
    volume, magnetic energies and mass stay finite."""
    N = 3
    v, h = inputs.shell_mesh(2, 1)
    gm = sdmhd.Mesh(N, v, h, geom=1, r_in=0.7, r_out=0.98)
    q0 = inputs.random_state(gm.n_e, N, seed=2)
    q0[1, 3, 5] = np.nan
    out = gm.spherical_sums(gm.to_device(q0), 0.70, 0.98, 2, 3).cpu().numpy().reshape(-1, 8)
    assert np.all(np.isnan(out[:, [1, 2, 3, 7]]))
    assert np.all(np.isfinite(out[:, [0, 4, 5, 6]]))
