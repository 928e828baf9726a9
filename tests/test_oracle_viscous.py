"""Pins of the oracle's viscous, resistive and thermal fluxes (F_vis of Sec. MHD Governing Equations,
BR1 gradients of Sec. SD Method) against closed forms.

Each closed-form test takes a one-dimensional field on a periodic box and compares
dR = R(with the coefficient) - R(without) at the solution points with the exact contribution of that
term, at two resolutions: the inviscid part cancels exactly in dR, and the error must fall at high
order.  A wrong sign, a dropped factor (the -2/3 mu of Stokes' hypothesis, C_p, the gas constant)
or a transposed gradient fails one of them.
"""
import math

import numpy as np
import pytest

from paper_2502_17805_gb300 import inputs

GAMMA = 5.0 / 3.0
K = 2.0 * math.pi


def _box(oracle, n, N, jitter=0.0):
    v, h, per = inputs.box_mesh(n, jitter=jitter, seed=5)
    return oracle.Mesh(N, v, h, periodic=per, geom=0)


def _points(m):
    return np.stack([m.geometry(e)[2] for e in range(m.n_e)])  # [n_e, N^3, 3]


def _state(rho, u, p, B):
    """conserved state [9, n_e, N^3] from primitive fields (psi = 0)"""
    q = np.zeros((9,) + rho.shape)
    q[0] = rho
    for d in range(3):
        q[1 + d] = rho * u[d]
        q[5 + d] = B[d]
    q[4] = p / (GAMMA - 1.0) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) + 0.5 * (B[0] ** 2 + B[1] ** 2 + B[2] ** 2)
    return q


def _dR(oracle, m, q, **coef):
    base = dict(gamma=GAMMA, powell=0, glm_alpha=0.0, c_h=0.0, R_gas=coef.pop("R_gas", 1.0))
    R0, _ = m.residual(oracle.Phys(**base), q)
    R1, _ = m.residual(oracle.Phys(viscous=1, **base, **coef), q)
    return R1 - R0


def _err(oracle, n, N, build, **coef):
    """max error of dR against the closed form, per variable, relative to the closed form's amplitude"""
    m = _box(oracle, n, N)
    x = _points(m)[..., 0]  # [n_e, N^3]
    q, exact = build(x)
    d = _dR(oracle, m, q, **coef)
    out = {}
    for v, ex in exact.items():
        out[v] = np.abs(d[v] - ex).max() / np.abs(ex).max()
    others = [v for v in range(9) if v not in exact]
    out["others"] = max(np.abs(d[v]).max() for v in others)
    return out


def _converges(oracle, build, N=6, **coef):
    """BR1 second derivatives converge at about order N - 2 in the maximum norm (the central average
    of both sides' gradients): at N = 6, 4^3 -> 8^3 elements must gain at least 2^3."""
    coarse, fine = _err(oracle, 4, N, build, **coef), _err(oracle, 8, N, build, **coef)
    for v in coarse:
        if v == "others":
            continue
        assert fine[v] < 1e-3 and fine[v] < coarse[v] / 8.0, (v, coarse[v], fine[v])
    assert coarse["others"] < 1e-9 and fine["others"] < 1e-9, (coarse["others"], fine["others"])


def test_resistive_diffusion_of_a_shear_field(oracle):
    """B = (B0, d sin kx, 0): the induction equation gains eta d_xx B_y, the total energy the divergence
    of the resistive Poynting flux eta J x B: d_t E = eta d_x (B_y d_x B_y)."""
    eta, d0 = 0.02, 0.3

    def build(x):
        one = np.ones_like(x)
        By = d0 * np.sin(K * x)
        q = _state(one, [0 * x, 0 * x, 0 * x], one, [0.7 * one, By, 0 * x])
        dBy, ddBy = d0 * K * np.cos(K * x), -K * K * By
        return q, {6: eta * ddBy, 4: eta * (dBy ** 2 + By * ddBy)}

    _converges(oracle, build, eta=eta)


def test_shear_viscosity(oracle):
    """U = (0, d sin kx, 0) at uniform rho, p: d_t(rho v) = mu v'', d_t E = mu (v'^2 + v v'')."""
    mu, d0 = 0.05, 0.2

    def build(x):
        one = np.ones_like(x)
        v = d0 * np.sin(K * x)
        q = _state(one, [0 * x, v, 0 * x], one, [0 * x, 0 * x, 0 * x])
        dv, ddv = d0 * K * np.cos(K * x), -K * K * v
        return q, {2: mu * ddv, 4: mu * (dv ** 2 + v * ddv)}

    _converges(oracle, build, mu=mu)


def test_bulk_part_of_the_stress_follows_stokes(oracle):
    """U = (d sin kx, 0, 0): tau_xx = (2 - 2/3) mu u' (lambda = -2/3 mu), so d_t(rho u) = 4/3 mu u''
    and d_t E = 4/3 mu (u'^2 + u u'')."""
    mu, d0 = 0.05, 0.1

    def build(x):
        one = np.ones_like(x)
        u = d0 * np.sin(K * x)
        q = _state(one, [u, 0 * x, 0 * x], one, [0 * x, 0 * x, 0 * x])
        du, ddu = d0 * K * np.cos(K * x), -K * K * u
        return q, {1: 4.0 / 3.0 * mu * ddu, 4: 4.0 / 3.0 * mu * (du ** 2 + u * ddu)}

    _converges(oracle, build, mu=mu)


@pytest.mark.parametrize("term", ["kappa_r", "kappa"])
def test_heat_flux(oracle, term):
    """rho = 1, U = B = 0, T = T0 + d sin kx with p = rho R T (R = 0.7): the radiative term gives
    d_t E = kappa_r C_p T''; the entropy term -kappa rho T grad S with grad S = (C_p / gamma) grad T / T
    gives d_t E = kappa (C_p / gamma) T'' (C_p = gamma R / (gamma - 1))."""
    R, kap, d0 = 0.7, 0.03, 0.1
    cp = GAMMA * R / (GAMMA - 1.0)
    factor = cp if term == "kappa_r" else cp / GAMMA

    def build(x):
        one = np.ones_like(x)
        T = 1.0 + d0 * np.sin(K * x)
        q = _state(one, [0 * x, 0 * x, 0 * x], R * T, [0 * x, 0 * x, 0 * x])
        return q, {4: kap * factor * (-K * K * d0 * np.sin(K * x))}

    _converges(oracle, build, R_gas=R, **{term: kap})


def test_gradients_exact_for_linear_fields(oracle):
    """On straight (jittered) hexahedra the BR1 gradient of a field linear in x is exact: the
    extrapolation reproduces it on both sides of every face and D differentiates S^d w exactly."""
    N = 4
    v, h, per = inputs.box_mesh(3, jitter=0.15, seed=2)
    m = oracle.Mesh(N, v, h, periodic=per, geom=0)
    X = _points(m)
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    one = np.ones_like(x)
    u = [0.1 + 0.2 * x - 0.1 * y, 0.05 * z, -0.3 * x + 0.2 * z]
    B = [0.4 + 0.1 * y, 0.2 - 0.3 * z, 0.1 * x]
    R = 0.8
    T = 1.0 + 0.2 * x + 0.1 * y - 0.05 * z
    q = _state(one, u, R * T, B)
    # the field is not periodic: only the middle element of the 3^3 box sees it continuous on all
    # six faces (its neighbours' points are not wrapped)
    ph = oracle.Phys(gamma=GAMMA, R_gas=R, viscous=1)
    g = m.gradients(ph, q)
    centre = X.mean(axis=1)
    mid = [int(np.argmin(((centre - 0.5) ** 2).sum(axis=1)))]
    exact = {0: (0.2, -0.1, 0.0), 1: (0.0, 0.0, 0.05), 2: (-0.3, 0.0, 0.2), 3: (0.2, 0.1, -0.05),
             5: (0.0, 0.1, 0.0), 6: (0.0, 0.0, -0.3), 7: (0.1, 0.0, 0.0)}
    for e in mid:
        for c, ex in exact.items():
            for j in range(3):
                assert np.abs(g[e, c, j] - ex[j]).max() < 1e-12, (e, c, j, g[e, c, j].min(), g[e, c, j].max())


@pytest.mark.parametrize("kr", [(0.02, 0.0, 0.0), (0.004, 0.012, 0.006)])
def test_viscous_fluxes_conserve_on_a_curved_periodic_box(oracle, kr):
    """Random state on a jittered periodic box with every coefficient on: the face fluxes are averages
    along the owner's normal, so sum w |J| R = 0 to round-off for mass, momentum, energy and B.  With
    kappa_r(r) the two sides of a periodic face lie at different radii: the common flux takes the
    owner's face point (reading V7), one value per face point."""
    N = 4
    v, h, per = inputs.box_mesh(3, jitter=0.2, seed=8)
    m = oracle.Mesh(N, v, h, periodic=per, geom=0)
    q = inputs.random_state(m.n_e, N, seed=3)
    ph = oracle.Phys(gamma=GAMMA, powell=0, glm_alpha=0.0, c_h=0.5, viscous=1, mu=0.03, eta=0.02, kappa=0.01,
                     kappa_r=kr[0], kappa_r1=kr[1], kappa_r2=kr[2], R_gas=0.9)
    R, s = m.residual(ph, q)
    xs, xf, E, D, w = oracle.nodes(N)
    W = np.einsum("i,j,k->kji", w, w, w).ravel()
    tot, mag = np.zeros(9), np.zeros(9)
    for e in range(m.n_e):
        J = m.geometry(e)[1]
        tot += (R[:, e] * W * J).sum(axis=1)
        mag += (np.abs(R[:, e]) * W * J).sum(axis=1)
    assert np.all(np.abs(tot[:8]) <= 1e-13 * mag[:8]), (tot, mag)
    # and the viscous part is not negligible here
    R0, _ = m.residual(oracle.Phys(gamma=GAMMA, powell=0, glm_alpha=0.0, c_h=0.5), q)
    assert np.abs(R - R0).max() > 1e-3 * np.abs(R0).max()


def test_br1_gradient_integrates_to_zero_on_a_periodic_box(oracle):
    """With the BR1 common value on every face, sum w |J| grad w over a periodic box is a sum of face
    terms S w^ that cancel pairwise (the discrete divergence theorem): zero to round-off even for a
    random, discontinuous state.  One-sided face values leave the jumps in it."""
    N = 4
    v, h, per = inputs.box_mesh(3, jitter=0.2, seed=4)
    m = oracle.Mesh(N, v, h, periodic=per, geom=0)
    q = inputs.random_state(m.n_e, N, seed=9)
    g = m.gradients(oracle.Phys(gamma=GAMMA, viscous=1, R_gas=0.9), q)  # [n_e, 8, 3, N^3]
    xs, xf, E, D, w = oracle.nodes(N)
    W = np.einsum("i,j,k->kji", w, w, w).ravel()
    tot, mag = np.zeros((8, 3)), np.zeros((8, 3))
    for e in range(m.n_e):
        J = m.geometry(e)[1]
        tot += (g[e] * W * J).sum(axis=-1)
        mag += (np.abs(g[e]) * W * J).sum(axis=-1)
    assert np.all(np.abs(tot) <= 1e-13 * mag), np.abs(tot / mag).max()
