"""Kantorovich certificates for tracked endpoints (test infrastructure).

For a square polynomial system f and a point x0 let, in the infinity norm
(complex moduli),

    B   >= ||J(x0)^-1||,
    eta >= ||J(x0)^-1 f(x0)||   (the Newton step),
    K   >= Lipschitz constant of J on the ball |y - x0| <= 2 eta.

Kantorovich's theorem: if h = B K eta <= 1/2, f has a root x* with
|x* - x0| <= r0 = (1 - sqrt(1 - 2h)) / (B K) = 2 eta / (1 + sqrt(1 - 2h)) <= 2 eta, and J(x*) is invertible
(|J(x0)^-1 (J(x*) - J(x0))| <= B K r0 < 1), so x* is isolated.  Endpoints that
are more than r0(p) + r0(q) apart certify different roots.  With as many such
endpoints as the Bezout number prod(d_i), which bounds the number of isolated
roots in C^n, the tracked endpoints are all the roots of f.

K is bounded from the second derivatives: for every row i,
|J_i.(y) - J_i.(z)| <= sum_j sum_k sup |d^2 f_i / dx_j dx_k| |y - z|, and on the
ball every partial derivative of a monomial is bounded by the same partial of
sum |c| x^a evaluated at |x0| + r (all its coefficients are nonnegative).

Everything here is numpy in double precision; the certificates below hold
with margins of many orders of magnitude, far above the rounding of these
estimates.
"""
from __future__ import annotations

import numpy as np


def _power_product(X, a, sup):
    """prod_j X[:, j] ** a[j] over the support `sup` (ones if empty)."""
    out = np.ones(X.shape[0], X.dtype)
    for j in sup:
        if a[j] > 0:
            out = out * X[:, j] ** int(a[j])
    return out


def _values_and_jacobian(system, X):
    """f and J at the points X [m][n] (complex), straight from the monomials."""
    m, n = X.shape
    F = np.zeros((m, system.n_polys), complex)
    J = np.zeros((m, system.n_polys, n), complex)
    c = system.coef[:, 0] + 1j * system.coef[:, 1]
    row = 0
    for i, k in enumerate(system.n_terms):
        for t in range(row, row + k):
            a = system.exps[t].astype(int)
            sup = np.nonzero(a)[0]
            F[:, i] += c[t] * _power_product(X, a, sup)
            for j in sup:
                e = a.copy()
                e[j] -= 1
                J[:, i, j] += c[t] * a[j] * _power_product(X, e, sup)
        row += k
    return F, J


def _second_derivative_bound(system, R):
    """max_i sum_{j,k} sum_t |c_t| |d^2 x^a_t / dx_j dx_k| at the moduli R [m][n]."""
    m, n = R.shape
    rows = np.zeros((m, system.n_polys))
    mod = np.hypot(system.coef[:, 0], system.coef[:, 1])
    row = 0
    for i, k in enumerate(system.n_terms):
        for t in range(row, row + k):
            a = system.exps[t].astype(int)
            sup = np.nonzero(a)[0]
            for j in sup:
                for l in sup:
                    e = a.copy()
                    if j == l:
                        if a[j] < 2:
                            continue
                        mult = a[j] * (a[j] - 1)
                        e[j] -= 2
                    else:
                        mult = a[j] * a[l]
                        e[j] -= 1
                        e[l] -= 1
                    rows[:, i] += mod[t] * mult * _power_product(R, e, sup)
        row += k
    return rows.max(axis=1)


def _min_separation(X, radius):
    """The smallest infinity-norm distance between two rows of X when it is
    below `radius`, else a value >= radius (inf if no projections are close).
    Every pair closer than `radius` is compared, since a real projection
    shrinks distances by at most |w|_1: |Re w.(x - y)| <= |w|_1 |x - y|_inf;
    sorting the projections leaves only neighbours within that width."""
    m, n = X.shape
    if m < 2:
        return np.inf
    w = np.exp(2j * np.pi * np.arange(1, n + 1) / (n + 1.618))
    proj = (X @ w).real
    order = np.argsort(proj, kind="stable")
    ps, Xs = proj[order], X[order]
    width = radius * np.abs(w).sum()
    best = np.inf
    for off in range(1, m):
        near = (ps[off:] - ps[:-off]) < width
        if not near.any():
            break
        idx = np.nonzero(near)[0]
        d = np.max(np.abs(Xs[idx + off] - Xs[idx]), axis=1)
        best = min(best, float(d.min()))
    return best


def certify_roots(system, X):
    """Kantorovich certificate of the endpoints X [m][n] (leading limbs).
    Returns a dict: h (max B K eta), r0 (max radius), separation (the
    smallest distance between two endpoints if below 1e-3, else >= 1e-3), and
    `distinct_roots` = m when every endpoint is certified and no two balls
    meet, else 0."""
    X = np.asarray(X, complex)
    F, J = _values_and_jacobian(system, X)
    Jinv = np.linalg.inv(J)
    B = np.abs(Jinv).sum(axis=2).max(axis=1)
    eta = np.abs(np.einsum("mij,mj->mi", Jinv, F)).max(axis=1)
    K = _second_derivative_bound(system, np.abs(X) + 2.0 * eta[:, None])
    h = B * K * eta
    ok = bool(np.all(h <= 0.5))
    # (1 - sqrt(1 - 2h)) / (B K), written without cancellation; eta when K = 0
    r0 = 2.0 * eta / (1.0 + np.sqrt(np.clip(1.0 - 2.0 * h, 0.0, 1.0)))
    sep = _min_separation(X, max(1e-3, 4.0 * float(r0.max())))
    distinct = ok and sep > 2.0 * float(r0.max())
    return dict(h=float(h.max()), r0=float(r0.max()), separation=sep, distinct_roots=X.shape[0] if distinct else 0)
