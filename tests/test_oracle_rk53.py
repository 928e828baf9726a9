"""Pins of the five-stage third-order SSP method (SSPRK(5,3), reading R23) and of the oracle's step.

The coefficients are those oracle/ssprk53.py derives; these tests check them against what defines
the method, not against themselves: the third-order conditions, the non-negative (strong-stability-
preserving) canonical form with coefficient r, the stability polynomial the oracle's step produces
on a linear problem, and third-order convergence in time on the nonlinear Alfven wave."""
import math

import numpy as np
import pytest

from oracle import ssprk53
from paper_2502_17805_gb300 import inputs

R_SSP = 2.6506291914393882
A43, A54, A61, A62 = 0.47329099097408517, 0.85150069298830050, 0.16614637524614647, 0.063691005655456475
A65 = 1.0 - A61 - A62
# the circularly polarised Alfven wave of the oracle pins: rho, amplitude, |B0|, p, wave vector
ALFVEN = [1.0, 0.1, 1.0, 0.1, 2 * math.pi, 2 * math.pi, 2 * math.pi]


def _tableau():
    A, b = ssprk53._butcher(1.0 / R_SSP, A43, A54, A61, A62)
    return np.array(A, dtype=float), np.array(b, dtype=float)


def test_third_order_conditions():
    A, b = _tableau()
    c = A.sum(1)
    assert abs(b.sum() - 1) < 1e-15
    assert abs(b @ c - 1 / 2) < 1e-15
    assert abs(b @ c ** 2 - 1 / 3) < 1e-15
    assert abs(b @ (A @ c) - 1 / 6) < 1e-15
    # and not of order 4: the tall tree b.A.A.c = 1/24 fails
    assert abs(b @ (A @ (A @ c)) - 1 / 24) > 1e-3


def test_strong_stability_preserving_with_coefficient_r():
    """Every stage a convex combination of forward-Euler steps of size dt/r: with K = [[A, 0],
    [b^T, 0]], K (I + r K)^-1 >= 0 and (I + r K)^-1 e >= 0 hold at r and fail just above it."""
    A, b = _tableau()
    K = np.zeros((6, 6))
    K[:5, :5] = A
    K[5, :5] = b

    def worst(r):
        M = np.linalg.inv(np.eye(6) + r * K)
        return min((K @ M)[np.tril_indices(6, -1)].min(), (M @ np.ones(6)).min())
    assert worst(R_SSP) > -1e-14
    assert worst(R_SSP * (1 + 1e-6)) < 0
    assert min(A43, A54, A61, A62, A65, 1 - A43, 1 - A54) > 0
    # r / 5 stages: more than twice the 1/3 per residual evaluation of the three-stage method
    assert R_SSP / 5 > 1.5 / 3


def test_stability_polynomial_of_the_oracle_step(oracle):
    """psi' = -a psi on a uniform periodic state: one step multiplies by R(z), z = -a dt, a degree-5
    polynomial with coefficients 1, 1, 1/2, 1/6 (order 3), b.A^3.e and b.A^4.e."""
    v, h, per = inputs.box_mesh(3)
    m = oracle.Mesh(3, v, h, periodic=per, geom=0)
    a = 2.0
    ph = oracle.Phys(powell=1, c_h=0.0, glm_alpha=a)
    q = m.state_init(ph, oracle.INIT_UNIFORM, [1.0, 0.1, 0.2, 0.3, 0.6, 0.2, 0.1, 0.3, 0.05])
    zs = np.array([-0.25, -0.5, -0.75, -1.0, -1.25, -1.5])
    Rz = np.array([m.rk53_step(ph, -z / a, q)[8].mean() / q[8].mean() for z in zs])
    coef = np.linalg.solve(np.vander(zs, 6, increasing=True), Rz)
    A, b = _tableau()
    e = np.ones(5)
    want = [1, 1, 1 / 2, 1 / 6, b @ A @ A @ A @ e, b @ A @ A @ A @ A @ e]
    np.testing.assert_allclose(coef, want, rtol=1e-8, atol=1e-10)


def _alfven_error(oracle, dt, T, N=4, n=3):
    v, h, per = inputs.box_mesh(n)
    m = oracle.Mesh(N, v, h, periodic=per, geom=0)
    ph = oracle.Phys(powell=1, c_h=0.0)
    q = m.state_init(ph, oracle.INIT_ALFVEN, ALFVEN + [0.0])
    for _ in range(int(round(T / dt))):
        q = m.rk53_step(ph, dt, q)
    return q


def test_third_order_in_time_on_the_alfven_wave(oracle):
    """The nonlinear circularly polarised Alfven wave on a fixed mesh: halving dt cuts the time
    error eightfold (against a run at dt/16); this exercises every order condition, the bushy tree
    b.c^2 = 1/3 among them, which linear problems do not see."""
    T, dt = 0.06, 0.015
    ref = _alfven_error(oracle, dt / 16, T)
    errs = [np.abs(_alfven_error(oracle, dt / k, T) - ref).max() for k in (1, 2, 4)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 2.7, (errs, rates)
