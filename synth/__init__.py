"""Seeded synthetic inputs for the many-path homotopy tracker.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no evaluation, differentiation, Newton or tracking).  Both
the CPU oracle (``oracle/``) and the CUDA library take their inputs from here,
so a parity test feeds the two sides bit-identical data.

Every draw comes from one SplitMix64 stream (Steele, Lea, Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), written out below
with numpy uint64 arithmetic so that the same seed gives the same bits on any
machine and any numpy version.  Floating point work here is limited to
correctly rounded IEEE operations (+, *, /, sqrt), which are also identical on
x86 and Arm.

Data layout (the "vertical" layout of the paper's Section 3, Table tabtranspose:
path index fastest):

* a system is ``n_terms[n_polys]`` (int32), ``exps[M][n_vars]`` (int8, M = sum of
  n_terms, monomials of polynomial 0 first) and ``coef[M][2]`` (float64 re, im);
* a batch of points is ``x[n_vars][2][L][n_pts]`` (float64), L limbs per real
  number (1 = double, 2 = double double, 4 = quad double), limb 0 the leading one.

The workload shapes follow the paper's synthetic benchmark families; see
``CONFIGS`` for the five workload families, the three stand-ins shaped like
the paper's benchmark applications, and their seeds.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """SplitMix64 stream: state += golden; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            steps = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + steps * _GOLDEN
            self.state = self.state + np.uint64(n) * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers uniform in [lo, hi] (inclusive) by the multiply-shift map."""
        span = np.uint64(hi - lo + 1)
        top = self.u64(n) >> np.uint64(32)
        return ((top * span) >> np.uint64(32)).astype(np.int64) + lo

    def choice_without_replacement(self, pool_size: int, k: int) -> np.ndarray:
        """k distinct indices from range(pool_size), partial Fisher-Yates."""
        idx = np.arange(pool_size)
        for i in range(k):
            j = int(self.integers(i, pool_size - 1, 1)[0])
            idx[i], idx[j] = idx[j], idx[i]
        return idx[:k].copy()


def unit_circle(rng: SplitMix64, n: int) -> tuple[np.ndarray, np.ndarray]:
    """n complex numbers of modulus 1 (to rounding) with uniform phase.

    Rejection sampling in the square [-1,1]^2 keeps points with
    0.01 <= r^2 <= 1 and scales them by 1/r; the phase of the kept points is
    uniform.  Only correctly rounded operations are used.
    """
    re = np.empty(n)
    im = np.empty(n)
    filled = 0
    while filled < n:
        need = n - filled
        u = rng.uniform(2 * need + 16) * 2.0 - 1.0
        a, b = u[0::2], u[1::2]
        m = min(a.size, b.size)
        a, b = a[:m], b[:m]
        r2 = a * a + b * b
        keep = (r2 <= 1.0) & (r2 >= 0.01)
        a, b, r2 = a[keep], b[keep], r2[keep]
        r = np.sqrt(r2)
        take = min(need, a.size)
        re[filled:filled + take] = a[:take] / r[:take]
        im[filled:filled + take] = b[:take] / r[:take]
        filled += take
    return re, im


def random_tails(rng: SplitMix64, lead: np.ndarray, limbs: int) -> np.ndarray:
    """Extend doubles ``lead`` to ``limbs``-limb numbers with random tails.

    Limb j+1 is uniform in (-ulp(limb j)/2, ulp(limb j)/2), so the limbs do not
    overlap and the value differs from ``lead`` by less than one ulp.
    Returns an array of shape (limbs, len(lead)).
    """
    out = np.zeros((limbs,) + lead.shape)
    out[0] = lead
    for j in range(1, limbs):
        ulp = np.abs(np.spacing(out[j - 1]))
        out[j] = ulp * (rng.uniform(lead.size).reshape(lead.shape) - 0.5)
    return out


@dataclass
class System:
    """A polynomial system f(x) = 0: n_polys polynomials in n_vars variables."""

    n_vars: int
    n_polys: int
    n_terms: np.ndarray  # int32 [n_polys]
    exps: np.ndarray  # int8 [M][n_vars]
    coef: np.ndarray  # float64 [M][2]
    meta: dict = field(default_factory=dict)

    @property
    def n_monomials(self) -> int:
        return int(self.n_terms.sum())

    def coef_limbs(self, limbs: int) -> np.ndarray:
        """Coefficients as [M][2][limbs]: the doubles in limb 0, zeros below."""
        out = np.zeros((self.n_monomials, 2, limbs))
        out[:, :, 0] = self.coef
        return np.ascontiguousarray(out)

    def degrees(self) -> np.ndarray:
        """Total degree of each polynomial."""
        deg = self.exps.astype(np.int64).sum(axis=1)
        off = np.concatenate([[0], np.cumsum(self.n_terms)])
        return np.array([deg[off[i]:off[i + 1]].max() for i in range(self.n_polys)], dtype=np.int32)


def _exponent_vectors(n: int, max_degree: int) -> list[tuple[int, ...]]:
    """All exponent vectors in n variables with total degree 1..max_degree."""
    out = []
    for d in range(1, max_degree + 1):
        for combo in itertools.combinations_with_replacement(range(n), d):
            a = [0] * n
            for v in combo:
                a[v] += 1
            out.append(tuple(a))
    return out


def total_degree_system(seed: int, n: int, degree: int, n_monomials: int) -> System:
    """Random system whose i-th equation holds x_i^degree, the constant 1 and
    n_monomials - 2 further distinct monomials drawn uniformly from all exponent
    vectors of total degree 1..degree.  Coefficients are uniform on the unit
    circle.  Every equation then has total degree ``degree``, so the total-degree
    start system x_i^degree - 1 = 0 gives degree^n paths.
    """
    rng = SplitMix64(seed)
    pool_all = _exponent_vectors(n, degree)
    exps = []
    for i in range(n):
        lead = [0] * n
        lead[i] = degree
        lead = tuple(lead)
        pool = [a for a in pool_all if a != lead]
        k = n_monomials - 2
        if k > len(pool):
            raise ValueError("not enough distinct monomials of this degree")
        pick = rng.choice_without_replacement(len(pool), k)
        eq = [lead, tuple([0] * n)] + [pool[j] for j in sorted(pick.tolist())]
        exps.extend(eq)
    M = n * n_monomials
    re, im = unit_circle(rng, M)
    return System(
        n_vars=n,
        n_polys=n,
        n_terms=np.full(n, n_monomials, dtype=np.int32),
        exps=np.array(exps, dtype=np.int8).reshape(M, n),
        coef=np.ascontiguousarray(np.stack([re, im], axis=1)),
        meta={"seed": seed, "family": "total_degree", "degree": degree},
    )


def sparse_support_system(seed: int, n_vars: int, n_polys: int, n_monomials: int,
                          k_min: int, k_max: int, e_min: int, e_max: int) -> System:
    """Random system for the standalone evaluation sweep: every monomial has a
    support of k ~ U{k_min..k_max} distinct variables, each with exponent
    ~ U{e_min..e_max}; supports (exponent vectors) are distinct within a
    polynomial; coefficients are uniform on the unit circle."""
    rng = SplitMix64(seed)
    exps = np.zeros((n_polys * n_monomials, n_vars), dtype=np.int8)
    row = 0
    for _ in range(n_polys):
        seen = set()
        while len(seen) < n_monomials:
            k = int(rng.integers(k_min, k_max, 1)[0])
            vars_ = rng.choice_without_replacement(n_vars, k)
            e = rng.integers(e_min, e_max, k)
            a = [0] * n_vars
            for v, ev in zip(vars_.tolist(), e.tolist()):
                a[v] = ev
            a = tuple(a)
            if a in seen:
                continue
            seen.add(a)
            exps[row] = a
            row += 1
    M = n_polys * n_monomials
    re, im = unit_circle(rng, M)
    return System(
        n_vars=n_vars,
        n_polys=n_polys,
        n_terms=np.full(n_polys, n_monomials, dtype=np.int32),
        exps=exps,
        coef=np.ascontiguousarray(np.stack([re, im], axis=1)),
        meta={"seed": seed, "family": "sparse_support"},
    )


def deficient_system() -> System:
    """f = (xy - 1, xy + x - 2): total degrees (2, 2), Bezout number 4, but the
    only finite root is (1, 1) (subtracting gives x = 1), where
    det J = det [[1, 1], [2, 1]] = -1: regular.  The leading forms xy, xy
    vanish at [1:0:0] and [0:1:0], so three paths of the total-degree
    homotopy must leave every bounded set."""
    exps = np.array([[1, 1], [0, 0], [1, 1], [1, 0], [0, 0]], np.int8)
    coef = np.array([[1, 0], [-1, 0], [1, 0], [1, 0], [-2, 0]], float)
    return System(n_vars=2, n_polys=2, n_terms=np.array([2, 3], np.int32), exps=exps, coef=coef,
                  meta={"family": "deficient"})


def extreme_system(seed: int, n_vars: int, n_polys: int) -> System:
    """A system at the limits of the format: random supports over n_vars
    variables (6 monomials per polynomial, supports of 1..min(n_vars, 20)
    variables, exponents 1..3), in which five monomials are replaced by a
    support of the last 64 variables, x_{n/2}^127 (the largest exponent), a
    constant, the first 64 variables squared, and the last variable alone.
    Needs n_vars >= 64 and n_polys >= 3."""
    if n_vars < 64 or n_polys < 3:
        raise ValueError("extreme_system needs n_vars >= 64 and n_polys >= 3")
    base = sparse_support_system(seed, n_vars, n_polys, 6, 1, min(n_vars, 20), 1, 3)
    exps = base.exps.copy()
    exps[0] = 0
    exps[0, n_vars - 64:] = 1
    exps[1] = 0
    exps[1, n_vars // 2] = 127
    exps[6] = 0
    exps[7] = 0
    exps[7, :64] = 2
    exps[12] = 0
    exps[12, n_vars - 1] = 1
    return System(n_vars=n_vars, n_polys=n_polys, n_terms=base.n_terms, exps=exps, coef=base.coef,
                  meta={"seed": seed, "family": "extreme"})


def _multilinear(rng: SplitMix64, n: int, k: int) -> tuple[int, ...]:
    """An exponent vector with k distinct variables, each to the power 1."""
    a = [0] * n
    for v in rng.choice_without_replacement(n, k).tolist():
        a[v] = 1
    return tuple(a)


def paper_shaped_system(kind: str, seed: int) -> System:
    """Random systems with the shapes the paper reports for its three benchmark
    applications (Section 4.2, Table tabsumchar): the dimension, the number of
    monomials of each polynomial and their degrees.  The monomials are drawn
    at random (products of distinct variables, exponent 1: the paper gives
    degrees, not exponents); coefficients are uniform on the unit circle.

    * "cyclic10": 10 variables; polynomial k = 1..9 has 10 distinct monomials
      of degree k; the last has one monomial of degree 10 and a constant
      (92 monomials);
    * "nash8": 8 variables, 8 polynomials of 130 distinct monomials whose
      degrees are uniform in 1..7 (1,040 monomials);
    * "pieri44": 16 variables, 16 polynomials of 246 distinct monomials of
      degree 4 (3,936 monomials).
    """
    rng = SplitMix64(seed)
    polys: list[list[tuple[int, ...]]] = []
    if kind == "cyclic10":
        n = 10
        for k in range(1, n):
            seen: list[tuple[int, ...]] = []
            while len(seen) < 10:
                a = _multilinear(rng, n, k)
                if a not in seen:
                    seen.append(a)
            polys.append(seen)
        polys.append([tuple([1] * n), tuple([0] * n)])
    elif kind in ("nash8", "pieri44"):
        n, per, kmin, kmax = (8, 130, 1, 7) if kind == "nash8" else (16, 246, 4, 4)
        for _ in range(n):
            seen = []
            have = set()
            while len(seen) < per:
                k = int(rng.integers(kmin, kmax, 1)[0])
                a = _multilinear(rng, n, k)
                if a not in have:
                    have.add(a)
                    seen.append(a)
            polys.append(seen)
    else:
        raise ValueError("unknown paper shape %r" % kind)
    exps = np.array([a for p in polys for a in p], dtype=np.int8)
    M = exps.shape[0]
    re, im = unit_circle(rng, M)
    return System(
        n_vars=n, n_polys=n, n_terms=np.array([len(p) for p in polys], dtype=np.int32), exps=exps,
        coef=np.ascontiguousarray(np.stack([re, im], axis=1)),
        meta={"seed": seed, "family": "paper_shape", "kind": kind},
    )


def unit_points(seed: int, n_vars: int, n_pts: int, limbs: int) -> np.ndarray:
    """Points with |x_i| = 1 (to rounding in limb 0) and uniform phase; lower
    limbs are random non-overlapping tails.  Shape [n_vars][2][limbs][n_pts]."""
    rng = SplitMix64(seed)
    re, im = unit_circle(rng, n_vars * n_pts)
    x = np.empty((n_vars, 2, limbs, n_pts))
    x[:, 0] = random_tails(rng, re.reshape(n_vars, n_pts), limbs).transpose(1, 0, 2)
    x[:, 1] = random_tails(rng, im.reshape(n_vars, n_pts), limbs).transpose(1, 0, 2)
    return np.ascontiguousarray(x)


def random_gamma(seed: int) -> tuple[float, float]:
    """The homotopy's random complex constant: a double on the unit circle."""
    re, im = unit_circle(SplitMix64(seed ^ 0x5DEECE66D), 1)
    return float(re[0]), float(im[0])


# The five workload families (seed = 1000 * family + instance).
CONFIGS = {
    "plain_n6_d": dict(kind="track", n=6, degree=2, n_monomials=8, limbs=1, seed=0),
    "evaldiff_n32": dict(kind="evaldiff", n_vars=32, n_polys=32, n_monomials=64, k_min=2, k_max=8,
                        e_min=1, e_max=3, n_pts=65536, seed=1000),
    "batched_n12_dd": dict(kind="track", n=12, degree=2, n_monomials=16, limbs=2, seed=2000),
    "learned_n16_d": dict(kind="track", n=16, degree=2, n_monomials=24, limbs=1, seed=3000,
                         train_seeds=(3000, 3200), heldout_seeds=(3500, 3520)),
    "stress_n10_qd": dict(kind="track", n=10, degree=3, n_monomials=32, limbs=4, seed=4000),
    # stand-ins with the shapes of the paper's benchmark applications (Table
    # tabsumchar), for evaluation sweeps over 10..3000 points
    "cyclic10_shape": dict(kind="paper_shape", shape="cyclic10", n=10, monomials=92, seed=5000),
    "nash8_shape": dict(kind="paper_shape", shape="nash8", n=8, monomials=1040, seed=6000),
    "pieri44_shape": dict(kind="paper_shape", shape="pieri44", n=16, monomials=3936, seed=7000),
}

# numbers of points of the paper's evaluation tables (Tables tabevalcyclic10,
# tabevalnash8, tabevalpieri44)
PAPER_SWEEP_POINTS = (10, 20, 50, 100, 200, 500, 1000, 2000, 3000)


def config_system(name: str, seed: int | None = None) -> System:
    c = CONFIGS[name]
    s = c["seed"] if seed is None else seed
    if c["kind"] == "paper_shape":
        return paper_shaped_system(c["shape"], s)
    if c["kind"] == "evaldiff":
        return sparse_support_system(s, c["n_vars"], c["n_polys"], c["n_monomials"],
                                     c["k_min"], c["k_max"], c["e_min"], c["e_max"])
    return total_degree_system(s, c["n"], c["degree"], c["n_monomials"])
