"""Exact rational helpers for pinning the oracle (Python fractions only)."""
from fractions import Fraction as Fr

import numpy as np


def fr(limbs) -> Fr:
    """Exact value of an L-limb number."""
    return sum((Fr(float(v)) for v in np.ravel(limbs)), Fr(0))


class Cx:
    """Exact complex rational."""

    __slots__ = ("re", "im")

    def __init__(self, re, im=Fr(0)):
        self.re = Fr(re)
        self.im = Fr(im)

    def __add__(self, o):
        return Cx(self.re + o.re, self.im + o.im)

    def __sub__(self, o):
        return Cx(self.re - o.re, self.im - o.im)

    def __mul__(self, o):
        if not isinstance(o, Cx):
            o = Cx(o)
        return Cx(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)

    def __truediv__(self, o):
        if not isinstance(o, Cx):
            o = Cx(o)
        den = o.re * o.re + o.im * o.im
        n = self * Cx(o.re, -o.im)
        return Cx(n.re / den, n.im / den)

    def abs2(self):
        return self.re * self.re + self.im * self.im

    def absf(self) -> float:
        return float(self.abs2()) ** 0.5


def cx_from(arr2L) -> Cx:
    """arr2L: [2][L] limbs -> exact complex."""
    return Cx(fr(arr2L[0]), fr(arr2L[1]))


def cx_pow(z: Cx, e: int) -> Cx:
    r = Cx(1)
    for _ in range(e):
        r = r * z
    return r


def poly_value(coefs, exps, x):
    """sum_m c_m prod_i x_i^a_mi, exactly."""
    v = Cx(0)
    for c, a in zip(coefs, exps):
        t = c
        for i, e in enumerate(a):
            if e:
                t = t * cx_pow(x[i], int(e))
        v = v + t
    return v


def poly_partial_by_interpolation(coefs, exps, x, i, degree):
    """Exact d/dx_i of the polynomial at x, from values only: p(h) = f(x + h e_i)
    is a polynomial of degree <= degree in h; its slope at h = 0 follows from the
    Lagrange basis derivatives at 0 over the nodes h = 0..degree."""
    nodes = [Fr(k) for k in range(degree + 1)]
    vals = []
    for h in nodes:
        xs = list(x)
        xs[i] = x[i] + Cx(h)
        vals.append(poly_value(coefs, exps, xs))
    d = Cx(0)
    for k, hk in enumerate(nodes):
        # l_k'(0) = sum_{j != k} [1/(hk - hj)] prod_{m != k, j} (0 - hm)/(hk - hm)
        w = Fr(0)
        for j, hj in enumerate(nodes):
            if j == k:
                continue
            term = Fr(1) / (hk - hj)
            for m, hm in enumerate(nodes):
                if m in (k, j):
                    continue
                term *= (0 - hm) / (hk - hm)
            w += term
        d = d + vals[k] * Cx(w)
    return d
