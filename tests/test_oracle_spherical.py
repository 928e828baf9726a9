"""Pins of the oracle's spherical diagnostics (longitude averages of Sec. Results) against closed forms,
exact zeros and the independent volume diagnostics.

The shell 6 x 8^2 x 4 has element layers at r = 0.70 + 0.07 k and element faces on the equator, so
radial bins of width 0.14 and the two hemispheres hold whole elements: the bin sums are quadratures
of smooth integrands over exact shell sections and converge to the closed forms with the mesh."""
import math

import numpy as np

from paper_2502_17805_gb300 import inputs

R_IN, R_OUT = 0.70, 0.98


def _shell(oracle, N=4, nz=8, nr=4):
    v, h = inputs.shell_mesh(nz, nr)
    return oracle.Mesh(N, v, h, geom=1, r_in=R_IN, r_out=R_OUT)


def _points(m):
    return np.stack([m.geometry(e)[2] for e in range(m.n_e)])  # [n_e, N^3, 3]


def _state(X, u, B, rho=None):
    x = X[..., 0]
    rho = np.ones_like(x) if rho is None else rho
    q = np.zeros((9,) + x.shape)
    q[0] = rho
    for d in range(3):
        q[1 + d] = rho * u[d]
        q[5 + d] = B[d]
    q[4] = 1.0 / (5.0 / 3.0 - 1.0) + 0.5 * rho * sum(c ** 2 for c in u) + 0.5 * sum(c ** 2 for c in B)
    return q


def test_radial_bins_hold_exact_shell_volumes(oracle):
    m = _shell(oracle)
    X = _points(m)
    zero = np.zeros_like(X[..., 0])
    S = m.spherical_sums(_state(X, [zero] * 3, [zero] * 3), 2, 1)
    for k in range(2):
        r1, r2 = R_IN + 0.14 * k, R_IN + 0.14 * (k + 1)
        exact = 4.0 * math.pi / 3.0 * (r2 ** 3 - r1 ** 3)
        assert abs(S[k, 0, 0] / exact - 1.0) < 1e-4, (k, S[k, 0, 0], exact)


def test_solid_body_rotation(oracle):
    """U = Omega z x x: V_r = V_theta = 0 at every point, V_phi = Omega s (s the distance from the
    axis), whose shell integral is Omega pi^2 (r2^4 - r1^4) / 4."""
    m = _shell(oracle)
    X = _points(m)
    Om = 0.8
    u = [-Om * X[..., 1], Om * X[..., 0], np.zeros_like(X[..., 0])]
    zero = np.zeros_like(X[..., 0])
    S = m.spherical_sums(_state(X, u, [zero] * 3), 2, 1)
    speed = np.abs(Om) * np.sqrt(X[..., 0] ** 2 + X[..., 1] ** 2).max()
    assert np.abs(S[..., 1]).max() < 1e-14 * speed and np.abs(S[..., 2]).max() < 1e-14 * speed
    for k in range(2):
        r1, r2 = R_IN + 0.14 * k, R_IN + 0.14 * (k + 1)
        exact = Om * math.pi ** 2 * (r2 ** 4 - r1 ** 4) / 4.0
        assert abs(S[k, 0, 3] / exact - 1.0) < 1e-4, (k, S[k, 0, 3], exact)


def test_colatitude_bins_separate_the_hemispheres(oracle):
    """V_phi = Omega s (1 + z): the northern half (first colatitude bin) carries the extra
    Omega int s z dV = Omega 2 pi (r2^5 - r1^5) / 15 and the southern half loses it."""
    m = _shell(oracle)
    X = _points(m)
    Om = 0.5
    f = 1.0 + X[..., 2]
    u = [-Om * X[..., 1] * f, Om * X[..., 0] * f, np.zeros_like(f)]
    zero = np.zeros_like(f)
    S = m.spherical_sums(_state(X, u, [zero] * 3), 1, 2)
    half = Om * math.pi ** 2 * (R_OUT ** 4 - R_IN ** 4) / 8.0
    extra = Om * 2.0 * math.pi * (R_OUT ** 5 - R_IN ** 5) / 15.0
    assert abs(S[0, 0, 3] / (half + extra) - 1.0) < 1e-4, (S[0, 0, 3], half + extra)
    assert abs(S[0, 1, 3] / (half - extra) - 1.0) < 1e-4, (S[0, 1, 3], half - extra)


def test_poloidal_and_toroidal_energies(oracle):
    """A field along phi has no poloidal energy and one in the meridional plane no toroidal energy,
    point by point; for any field the two add up to the volume integral of B^2 / 2 that the
    ordinary diagnostics compute."""
    m = _shell(oracle)
    X = _points(m)
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    zero = np.zeros_like(x)
    s = np.sqrt(x ** 2 + y ** 2)
    tor = [-0.3 * y / s, 0.3 * x / s, zero]
    r = np.sqrt(x ** 2 + y ** 2 + z ** 2)
    pol = [0.2 * x / r + 0.1 * x * z / (r * s), 0.2 * y / r + 0.1 * y * z / (r * s), 0.2 * z / r - 0.1 * s / r]
    S = m.spherical_sums(_state(X, [zero] * 3, tor), 2, 3)
    assert np.abs(S[..., 4]).max() < 1e-15 * np.abs(S[..., 5]).max()
    S = m.spherical_sums(_state(X, [zero] * 3, pol), 2, 3)
    assert np.abs(S[..., 5]).max() < 1e-15 * np.abs(S[..., 4]).max()
    rng = np.random.default_rng(4)
    B = [rng.normal(size=x.shape) for _ in range(3)]
    U = [0.1 * rng.normal(size=x.shape) for _ in range(3)]
    rho = 1.0 + 0.2 * rng.random(size=x.shape)
    q = _state(X, U, B, rho)
    S = m.spherical_sums(q, 3, 5)
    d = m.diagnostics(oracle.Phys(powell=0), q)
    assert abs((S[..., 4].sum() + S[..., 5].sum()) / (d["eb"] * d["volume"]) - 1.0) < 1e-13
    assert abs(S[..., 6].sum() / d["mass"] - 1.0) < 1e-13
    assert abs(S[..., 7].sum() / (d["ke"] * d["volume"]) - 1.0) < 1e-13
    assert abs(S[..., 0].sum() / d["volume"] - 1.0) < 1e-13
