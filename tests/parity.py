"""Element-wise comparison of L-limb complex SoA arrays against the oracle."""
import numpy as np

import oracle

TOL = {1: 1e-12, 2: 1e-26, 4: 1e-55}  # relative to the sum of term moduli


def cerr(got, ref):
    """got, ref: [..., 2, L, n] -> |got - ref| per complex entry, [..., n], using
    the exact difference of the limb sums."""
    g = np.ascontiguousarray(got)
    r = np.ascontiguousarray(ref)
    dre = oracle.value_diff(np.moveaxis(g[..., 0, :, :], -2, -1), np.moveaxis(r[..., 0, :, :], -2, -1))
    dim = oracle.value_diff(np.moveaxis(g[..., 1, :, :], -2, -1), np.moveaxis(r[..., 1, :, :], -2, -1))
    return np.hypot(dre, dim)


def rel_err(got, ref, mag):
    """Maximum of |got - ref| / mag (mag: the oracle's sum of term moduli)."""
    e = cerr(got, ref)
    return float(np.max(e / np.maximum(mag, 1e-300)))
