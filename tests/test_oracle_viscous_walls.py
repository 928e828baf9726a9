"""Pins of the oracle's viscous wall conditions (Sec. Problem Formulation: stress-free, impenetrable
walls, a heat flux through the inner sphere, a fixed temperature on the outer sphere) on the shell.

Integral checks take dR = R(viscous) - R(inviscid) over the shell, weighted by w |J|: the interior
viscous fluxes cancel between elements, so what remains is what the walls let through."""
import math

import numpy as np
import pytest

from paper_2502_17805_gb300 import inputs

GAMMA = 5.0 / 3.0
RB, RT = 0.70, 0.98


def _shell(oracle, N=5, nz=6, nr=4):
    v, h = inputs.shell_mesh(nz, nr)
    return oracle.Mesh(N, v, h, geom=1, r_in=RB, r_out=RT, bc_in=oracle.BC_WALL_CONDUCTING,
                       bc_out=oracle.BC_WALL_RADIAL)


def _points(m):
    return np.stack([m.geometry(e)[2] for e in range(m.n_e)])


def _weights(oracle, m):
    xs, xf, E, D, w = oracle.nodes(m.N)
    W = np.einsum("i,j,k->kji", w, w, w).ravel()
    return np.stack([W * m.geometry(e)[1] for e in range(m.n_e)])  # [n_e, N^3]


def _state(X, u, T, R):
    x = X[..., 0]
    q = np.zeros((9,) + x.shape)
    q[0] = 1.0
    for d in range(3):
        q[1 + d] = u[d]
    q[4] = R * T / (GAMMA - 1.0) + 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    return q


def _dR(oracle, m, q, **kw):
    base = dict(gamma=GAMMA, powell=0, glm_alpha=0.0, c_h=0.5, R_gas=kw.get("R_gas", 1.0))
    R0, _ = m.residual(oracle.Phys(**base), q)
    R1, _ = m.residual(oracle.Phys(viscous=1, **dict(base, **kw)), q)
    return R1 - R0


def test_heat_through_the_inner_wall(oracle):
    """Steady conduction T = A + C / r (rho = 1, kappa_r): raising the inner flux from q to 2 q adds
    4 pi r_b^2 q to the shell's energy per unit time (the outer wall is treated alike in both); with the
    walls passing their own conducted flux the steady field gains nothing."""
    m = _shell(oracle)
    X = _points(m)
    r = np.sqrt((X ** 2).sum(axis=-1))
    R, kr, A, Cc = 0.8, 0.02, 0.5, 0.3
    cp = GAMMA * R / (GAMMA - 1.0)
    zero = np.zeros_like(r)
    q = _state(X, [zero] * 3, A + Cc / r, R)
    W = _weights(oracle, m)
    qb = kr * cp * Cc / RB ** 2
    common = dict(kappa_r=kr, R_gas=R, T_top=A + Cc / RT, visc_walls=1)
    g1 = (W * _dR(oracle, m, q, q_bottom=qb, **common)[4]).sum()
    g2 = (W * _dR(oracle, m, q, q_bottom=2 * qb, **common)[4]).sum()
    exact = 4 * math.pi * RB ** 2 * qb
    assert abs((g2 - g1) / exact - 1.0) < 1e-3, (g2 - g1, exact)
    own = (W * _dR(oracle, m, q, **dict(common, visc_walls=0))[4]).sum()
    assert abs(own) < 1e-4 * exact, own


def test_top_temperature_is_held(oracle):
    """Uniform T equal to T_top conducts nothing anywhere (the metric identity makes the gradient of a
    constant vanish); a higher T_top heats the outermost layer through the outer wall, and the layers
    two or more elements away do not see it (the viscous face fluxes couple neighbours only)."""
    m = _shell(oracle)
    X = _points(m)
    r = np.sqrt((X ** 2).sum(axis=-1))
    R, kr, T0 = 0.8, 0.02, 0.7
    zero = np.zeros_like(r)
    q = _state(X, [zero] * 3, T0 + zero, R)
    kw = dict(kappa_r=kr, R_gas=R, visc_walls=1, q_bottom=0.0)
    # round-off scale of the conduction terms: kappa_r C_p T0 over the square of the point spacing
    scale = kr * GAMMA * R / (GAMMA - 1.0) * T0 / (0.07 / 5) ** 2
    d0 = _dR(oracle, m, q, T_top=T0, **kw)[4]
    assert np.abs(d0).max() < 1e-12 * scale, np.abs(d0).max() / scale
    d1 = _dR(oracle, m, q, T_top=T0 + 0.05, **kw)[4]
    W = _weights(oracle, m)
    top = r > RT - 0.07
    # at least a thousandth of the flux of a 0.05 drop across one element layer
    assert (W * d1)[top].sum() > 1e-3 * kr * GAMMA * R / (GAMMA - 1.0) * 0.05 / 0.07 * 4 * math.pi * RT ** 2
    far = r < RT - 0.14
    assert np.abs(d1[far]).max() < 1e-12 * scale


def test_stress_free_walls_exert_no_torque(oracle):
    """Differential rotation U = (O0 + O1 r) z x x: the viscous torque about z integrates to the
    torque of the walls.  Stress-free walls exert none; a wall that passes its own shear stress
    exerts (8 pi / 3) mu O1 (r_t^4 - r_b^4)."""
    m = _shell(oracle)
    X = _points(m)
    x, y = X[..., 0], X[..., 1]
    r = np.sqrt((X ** 2).sum(axis=-1))
    mu, O0, O1 = 0.01, 0.3, 0.5
    Om = O0 + O1 * r
    q = _state(X, [-Om * y, Om * x, np.zeros_like(x)], np.ones_like(x), 1.0)
    W = _weights(oracle, m)
    exact = 8 * math.pi / 3 * mu * O1 * (RT ** 4 - RB ** 4)
    for walls, want in ((1, 0.0), (0, exact)):
        d = _dR(oracle, m, q, mu=mu, visc_walls=walls, T_top=1.0)
        torque = (W * (x * d[2] - y * d[1])).sum()
        assert abs(torque - want) < 2e-3 * exact, (walls, torque, want)


def _mhd_state(X):
    """rho = 1, U = 0, p = 1 and a smooth field with tangential components and current at both walls"""
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    B = [0.2 * z - 0.3 * y, 0.3 * x + 0.1 * z * z, 0.2 * x * y]
    q = np.zeros((9,) + x.shape)
    q[0] = 1.0
    for d in range(3):
        q[5 + d] = B[d]
    q[4] = 1.0 / (GAMMA - 1.0) + 0.5 * (B[0] ** 2 + B[1] ** 2 + B[2] ** 2)
    return q


def _resistive_integrals(oracle, bc_in, bc_out, walls):
    v, h = inputs.shell_mesh(6, 4)
    m = oracle.Mesh(5, v, h, geom=1, r_in=RB, r_out=RT, bc_in=bc_in, bc_out=bc_out)
    X = _points(m)
    q = _mhd_state(X)
    W = _weights(oracle, m)
    d = _dR(oracle, m, q, eta=0.02, visc_walls=walls, q_bottom=0.0, T_top=1.0)
    return np.array([(W * d[v]).sum() for v in (4, 5, 6, 7)])


def test_conducting_walls_pass_no_resistive_flux(oracle):
    """A perfectly conducting wall has J = J_r r^ (Sec. Problem Formulation): neither the resistive
    induction flux eta J x n nor the resistive energy flux eta (B x J).n passes it, so with both walls
    conducting the shell integrals of the resistive residual of E and B vanish (the interior fluxes
    cancel between elements).  A wall that passes its own tangential current lets them through."""
    cond = oracle.BC_WALL_CONDUCTING
    own = _resistive_integrals(oracle, cond, cond, 0)
    scale = np.abs(own).max()
    assert scale > 1e-4, own
    held = _resistive_integrals(oracle, cond, cond, 1)
    assert np.abs(held).max() < 1e-12 * scale, (held, own)


def test_radial_field_walls_carry_surface_current(oracle):
    """A radial-field wall holds B_theta = B_phi = 0 on its face: it passes no resistive energy
    (B x J is tangential to the wall) but a surface current, i.e. resistive induction flux."""
    rad = oracle.BC_WALL_RADIAL
    held = _resistive_integrals(oracle, rad, rad, 1)
    assert abs(held[0]) < 1e-12 * np.abs(held[1:]).max(), held
    assert np.abs(held[1:]).max() > 1e-4, held


def _conducted_net(oracle, T_of_r, **kw):
    """shell integral of the conductive energy residual (rho = 1, U = 0) with each wall passing its
    own conducted flux: minus the net heat flowing out through the two spheres"""
    m = _shell(oracle)
    X = _points(m)
    r = np.sqrt((X ** 2).sum(axis=-1))
    zero = np.zeros_like(r)
    R = 0.8
    q = _state(X, [zero] * 3, T_of_r(r), R)
    W = _weights(oracle, m)
    return (W * _dR(oracle, m, q, R_gas=R, visc_walls=0, **kw)[4]).sum()


@pytest.mark.parametrize("power", [1, 2])
def test_radius_dependent_radiative_diffusivity(oracle, power):
    """kappa_r(r) = k r^power (reading V7): T = A - C / ((power + 1) k r^(power + 1)) makes
    r^2 kappa_r dT/dr constant, so as much heat leaves through the outer sphere as enters through the
    inner one and the shell gains nothing; the same profile with a constant kappa_r (its value at mid
    radius) does not conduct a constant flux and the shell gains or loses heat."""
    k, A, C = 0.02, 1.0, 0.004
    T = lambda r: A - C / ((power + 1) * k * r ** (power + 1))  # noqa: E731
    coef = {1: dict(kappa_r1=k), 2: dict(kappa_r2=k)}[power]
    steady = _conducted_net(oracle, T, **coef)
    rm = 0.5 * (RB + RT)
    flat = _conducted_net(oracle, T, kappa_r=k * rm ** power)
    assert abs(flat) > 1e-3 * GAMMA * 0.8 / (GAMMA - 1.0) * C, flat
    assert abs(steady) < 1e-4 * abs(flat), (steady, flat)
