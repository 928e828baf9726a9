"""Derivation of the five-stage, third-order SSP Runge-Kutta method the oracle and the library use
(test infrastructure: its results are typed into both, it runs in no product path).

The paper integrates with SSPRK(5,3), the method of a table in Ruuth's study of optimal strong-
stability-preserving methods, which is not available here.  That table is the result of an
optimisation with a published statement: among explicit s-stage methods of order p, maximise the
SSP coefficient r, the largest r for which every stage is a convex combination of forward-Euler
steps of size dt/r.  This script solves that problem for s = 5, p = 3 from its statement:

1. search: over all explicit 5-stage methods (Butcher matrix A, weights b), maximise r subject to
   the four third-order conditions and absolute monotonicity of the method at r (with
   K = [[A, 0], [b^T, 0]]: K (I + r K)^-1 >= 0 and (I + r K)^-1 e >= 0), by SLSQP from many random
   starts.  The optimum (r = 2.6506...) has canonical Shu-Osher coefficients
   alpha = r K (I + r K)^-1 that vanish except on this pattern:
       y2 = y1 + c dt F(y1),   y3 = y2 + c dt F(y2),
       y4 = (1 - a43) y1 + a43 (y3 + c dt F(y3)),   y5 = (1 - a54) y1 + a54 (y4 + c dt F(y4)),
       u^{n+1} = a61 y2 + a62 y3 + a65 (y5 + c dt F(y5)),   a65 = 1 - a61 - a62,
   with y1 = u^n and c = 1/r;
2. refinement: on that pattern the order conditions are four equations in (c, a43, a54, a61, a62).
   Solved for (c, a43, a54, a61) at a given a62 (Newton, 40 digits) they give the same c = 1/r for
   every a62 in [0, 0.2374] (where every coefficient is non-negative): the optimal methods form a
   one-parameter family, and the optimisation alone does not fix the table;
3. choice: the member with the least principal error, the 2-norm of the four fourth-order error
   coefficients (Phi(t) - 1/gamma(t)) / sigma(t) over the rooted trees t of order 4, the usual
   second criterion among methods of equal SSP coefficient (a62 = 0.0646...: 1.468e-2, against
   1.488e-2 and 1.644e-2 at the two ends of the family).

Run as a script it prints them."""
import numpy as np


def _butcher(c, a43, a54, a61, a62):
    a65 = 1 - a61 - a62
    A = [[0, 0, 0, 0, 0], [c, 0, 0, 0, 0], [c, c, 0, 0, 0], [a43 * c] * 3 + [0, 0],
         [a54 * a43 * c] * 3 + [a54 * c, 0]]
    b = [c * (a61 + a62 + a65 * a54 * a43), c * (a62 + a65 * a54 * a43), c * a65 * a54 * a43, c * a65 * a54,
         c * a65]
    return A, b


def search(trials=200, seed=1):
    """Step 1: the SSP coefficient of the best 5-stage third-order method found, its (A, b)."""
    from scipy.optimize import minimize
    s, nA = 5, 10

    def unpack(x):
        A = np.zeros((s, s))
        A[np.tril_indices(s, -1)] = x[:nA]
        return A, x[nA:nA + s], x[-1]

    def K(A, b):
        k = np.zeros((s + 1, s + 1))
        k[:s, :s] = A
        k[s, :s] = b
        return k

    def eq(x):
        A, b, _ = unpack(x)
        cv = A.sum(1)
        return np.array([b.sum() - 1, b @ cv - 0.5, b @ cv ** 2 - 1 / 3, b @ (A @ cv) - 1 / 6])

    def ineq(x):
        A, b, r = unpack(x)
        k = K(A, b)
        M = np.linalg.inv(np.eye(s + 1) + r * k)
        return np.concatenate([(k @ M)[np.tril_indices(s + 1, -1)], M @ np.ones(s + 1)])

    rng = np.random.default_rng(seed)
    best = None
    for _ in range(trials):
        x0 = np.concatenate([rng.uniform(0, 0.5, nA), rng.uniform(0, 0.4, s), [rng.uniform(0.5, 2.5)]])
        res = minimize(lambda x: -x[-1], x0, method="SLSQP",
                       constraints=[{"type": "eq", "fun": eq}, {"type": "ineq", "fun": ineq}],
                       options={"maxiter": 500, "ftol": 1e-14})
        if res.success and np.abs(eq(res.x)).max() < 1e-10 and ineq(res.x).min() > -1e-10:
            if best is None or res.x[-1] > best[-1]:
                best = res.x
    A, b, r = unpack(best)
    return r, A, b


def _solve(a62, start, mp):
    """(c, a43, a54, a61) from the four order conditions at the given a62."""
    def g(c, a43, a54, a61):
        A, b = _butcher(c, a43, a54, a61, a62)
        cv = [sum(row) for row in A]
        Ac = [sum(A[i][j] * cv[j] for j in range(5)) for i in range(5)]
        return [sum(b) - 1, sum(b[i] * cv[i] for i in range(5)) - mp.mpf(1) / 2,
                sum(b[i] * cv[i] ** 2 for i in range(5)) - mp.mpf(1) / 3,
                sum(b[i] * Ac[i] for i in range(5)) - mp.mpf(1) / 6]
    sol = mp.findroot(g, [mp.mpf(v) for v in start])
    return [sol[i] for i in range(4)]


def principal_error(c, a43, a54, a61, a62):
    """2-norm of the fourth-order error coefficients (Phi(t) - 1/gamma(t)) / sigma(t), t the four
    rooted trees of order 4 (b.A.A.c, b.A.c^2, b.(c * A.c), b.c^3)."""
    A, b = _butcher(c, a43, a54, a61, a62)
    cv = [sum(row) for row in A]
    Ac = [sum(A[i][j] * cv[j] for j in range(5)) for i in range(5)]
    AAc = [sum(A[i][j] * Ac[j] for j in range(5)) for i in range(5)]
    Ac2 = [sum(A[i][j] * cv[j] ** 2 for j in range(5)) for i in range(5)]
    import mpmath as mp
    one = mp.mpf(1)
    t = [sum(b[i] * AAc[i] for i in range(5)) - one / 24, (sum(b[i] * Ac2[i] for i in range(5)) - one / 12) / 2,
         sum(b[i] * cv[i] * Ac[i] for i in range(5)) - one / 8, (sum(b[i] * cv[i] ** 3 for i in range(5)) - one / 4) / 6]
    return mp.sqrt(sum(x * x for x in t))


def refine(start, digits=40):
    """Steps 2 and 3: the family of optimal methods and its member of least principal error:
    (c, a43, a54, a61, a62) to `digits` digits, and c over the family (its spread)."""
    import mpmath as mp
    mp.mp.dps = digits + 15
    guess = list(start[:4])
    cs = []
    for k in range(0, 24, 4):  # the family: c at a62 = 0, 0.04, ..., 0.2
        guess = _solve(mp.mpf(k) / 100, guess, mp)
        cs.append(guess[0])

    def err2(a62):
        return principal_error(*_solve(a62, guess, mp), a62) ** 2
    a62 = mp.findroot(lambda x: mp.diff(err2, x), mp.mpf("0.065"), tol=mp.mpf(10) ** (-digits))
    c, a43, a54, a61 = _solve(a62, guess, mp)
    return [c, a43, a54, a61, a62], max(cs) - min(cs)


def coefficients():
    """(r, a43, a54, a61, a62, a65) from the search, the family and the choice."""
    r, A, b = search()
    K = np.zeros((6, 6))
    K[:5, :5] = A
    K[5, :5] = b
    alpha = r * K @ np.linalg.inv(np.eye(6) + r * K)
    start = [1 / r, alpha[3, 2], alpha[4, 3], alpha[5, 0], alpha[5, 1]]
    (c, a43, a54, a61, a62), spread = refine(start)
    return 1 / c, a43, a54, a61, a62, 1 - a61 - a62, spread


if __name__ == "__main__":
    import mpmath as mp
    *vals, spread = coefficients()
    for name, v in zip(("r", "a43", "a54", "a61", "a62", "a65"), vals):
        print("%-4s %s" % (name, mp.nstr(v, 25)))
    print("spread of c over the family: %s" % mp.nstr(spread, 3))
    c, a43, a54, a61, a62 = 1 / vals[0], vals[1], vals[2], vals[3], vals[4]
    print("principal error norm: %s" % mp.nstr(principal_error(c, a43, a54, a61, a62), 8))
