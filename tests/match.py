"""Endpoint-set comparison: endpoints are a multiset (their order is
irrelevant), so two runs agree when a one-to-one pairing exists with every pair
within tol * max(1, |a|_inf)."""
import numpy as np
from scipy.optimize import linear_sum_assignment


def to_complex(x):
    """[n][2][L][m] limbs -> [m][n] complex (leading limbs)."""
    return (x[:, 0, 0, :] + 1j * x[:, 1, 0, :]).T


def match_sets(A, B, tol):
    """A, B: [m][n] complex. Returns (ok, max scaled distance of the pairing)."""
    A = np.asarray(A)
    B = np.asarray(B)
    if A.shape != B.shape:
        return False, np.inf
    if A.shape[0] == 0:
        return True, 0.0
    scale = np.maximum(1.0, np.max(np.abs(A), axis=1))
    D = np.max(np.abs(A[:, None, :] - B[None, :, :]), axis=2) / scale[:, None]
    r, c = linear_sum_assignment(D)
    worst = float(np.max(D[r, c]))
    return worst <= tol, worst
