"""Pins of the oracle's almost flux-balanced initial profile (Sec. Initial Conditions).

The profile solves dS/dr = (L / (4 pi r^2) + kappa_r rho_p C_p dT_p/dr) / (kappa rho_p T_p) and the
hydrostatic density equation; these tests check it against what fixes it independently: the
classical polytrope is the isentropic solution (L = kappa_r = 0), the result is in hydrostatic
balance, carries the prescribed entropy gradient, starts from the polytrope's bottom state and
has converged in the number of integration nodes."""
import math

import numpy as np

GAMMA, GM = 5.0 / 3.0, 1.0
RB, RT = 0.70, 0.98


def _params(L, kappa, kappa_r, N_rho=3.0, R=1.0):
    return [N_rho, RB, RT, 1.0, R, 0.0, 0.0, L, kappa, kappa_r]


def test_isentropic_limit_is_the_polytrope(oracle):
    r = np.linspace(RB, RT, 57)
    rho, p = oracle.flux_balanced(_params(0.0, 1.0, 0.0), r, GAMMA, GM)
    for i, ri in enumerate(r):
        rp, pp, _ = oracle.polytrope(ri, 3.0, RB, RT, 1.0, 1.0, GAMMA, GM)
        assert abs(rho[i] / rp - 1.0) < 1e-12 and abs(p[i] / pp - 1.0) < 1e-12, (ri, rho[i], rp, p[i], pp)


P_FB = _params(L=0.02, kappa=0.05, kappa_r=0.01)
H = 2e-4


def _d(oracle, f, r):
    """fourth-order central difference of f(rho, p) along r"""
    vals = [f(*oracle.flux_balanced(P_FB, r + k * H, GAMMA, GM)) for k in (-2, -1, 1, 2)]
    return (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * H)


def test_hydrostatic_balance(oracle):
    r = np.linspace(RB + 3 * H, RT - 3 * H, 41)
    rho, p = oracle.flux_balanced(P_FB, r, GAMMA, GM)
    dpdr = _d(oracle, lambda rr, pr: pr, r)
    assert np.all(np.abs(dpdr + rho * GM / r ** 2) <= 1e-8 * rho * GM / r ** 2)


def test_entropy_gradient_carries_the_luminosity(oracle):
    P = P_FB
    r = np.linspace(RB + 3 * H, RT - 3 * H, 41)
    L, kappa, kappa_r, R = P[7], P[8], P[9], P[4]
    cp = GAMMA * R / (GAMMA - 1.0)
    dSdr = _d(oracle, lambda rr, pr: cp * np.log(pr ** (1.0 / GAMMA) / rr), r)
    want = []
    for ri in r:
        rho_poly, _, T_poly = oracle.polytrope(ri, 3.0, RB, RT, 1.0, R, GAMMA, GM)
        dT = -GM / (cp * ri * ri)
        want.append((L / (4 * math.pi * ri * ri) + kappa_r * rho_poly * cp * dT) / (kappa * rho_poly * T_poly))
    want = np.array(want)
    assert np.all(np.abs(dSdr - want) <= 1e-8 * np.abs(want)), np.abs(dSdr / want - 1.0).max()


def test_bottom_state_and_node_convergence(oracle):
    P = _params(L=0.02, kappa=0.05, kappa_r=0.01)
    rho, p = oracle.flux_balanced(P, [RB], GAMMA, GM)
    _, pb, _ = oracle.polytrope(RB, 3.0, RB, RT, 1.0, 1.0, GAMMA, GM)
    assert abs(rho[0] - 1.0) < 1e-15 and abs(p[0] / pb - 1.0) < 1e-14
    r = np.linspace(RB, RT, 33)
    a = oracle.flux_balanced(P, r, GAMMA, GM, n_nodes=2048)
    b = oracle.flux_balanced(P, r, GAMMA, GM, n_nodes=4096)
    for x, y in zip(a, b):
        assert np.abs(x / y - 1.0).max() < 1e-11


def test_state_init_uses_the_profile(oracle):
    from paper_2502_17805_gb300 import inputs
    v, h = inputs.shell_mesh(2, 2)
    m = oracle.Mesh(4, v, h, geom=1, r_in=RB, r_out=RT)
    P = _params(L=0.02, kappa=0.05, kappa_r=0.01)
    ph = oracle.Phys(gamma=GAMMA, GM=GM)
    q = m.state_init(ph, oracle.INIT_SHELL_FLUX_BALANCED, P, seed=0)
    X = np.stack([m.geometry(e)[2] for e in range(m.n_e)])
    r = np.sqrt((X ** 2).sum(axis=-1)).ravel()
    rho, p = oracle.flux_balanced(P, r, GAMMA, GM)
    assert np.abs(q[0].ravel() / rho - 1.0).max() < 1e-14
    assert np.abs(q[4].ravel() * (GAMMA - 1.0) / p - 1.0).max() < 1e-14


def test_entropy_gradient_with_radius_dependent_kappa_r(oracle):
    """With kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2 (reading V7) the profile's entropy gradient
    carries the luminosity with that diffusivity at each radius."""
    kr0, kr1, kr2 = 0.004, 0.01, -0.003
    P = _params(L=0.02, kappa=0.05, kappa_r=kr0) + [kr1, kr2]
    r = np.linspace(RB + 3 * H, RT - 3 * H, 41)
    L, kappa, R = P[7], P[8], P[4]
    cp = GAMMA * R / (GAMMA - 1.0)

    def f(rr):
        rho, p = oracle.flux_balanced(P, rr, GAMMA, GM)
        return cp * np.log(p ** (1.0 / GAMMA) / rho)
    dSdr = (f(r - 2 * H) - 8 * f(r - H) + 8 * f(r + H) - f(r + 2 * H)) / (12 * H)
    want = []
    for ri in r:
        rho_poly, _, T_poly = oracle.polytrope(ri, 3.0, RB, RT, 1.0, R, GAMMA, GM)
        dT = -GM / (cp * ri * ri)
        kr = kr0 + kr1 * ri + kr2 * ri * ri
        want.append((L / (4 * math.pi * ri * ri) + kr * rho_poly * cp * dT) / (kappa * rho_poly * T_poly))
    want = np.array(want)
    assert np.all(np.abs(dSdr - want) <= 1e-8 * np.abs(want)), np.abs(dSdr / want - 1.0).max()
    # and it differs from the constant-kappa_r profile
    rho_c, _ = oracle.flux_balanced(_params(L=0.02, kappa=0.05, kappa_r=kr0), r, GAMMA, GM)
    rho_v, _ = oracle.flux_balanced(P, r, GAMMA, GM)
    assert np.abs(rho_v / rho_c - 1.0).max() > 1e-4
