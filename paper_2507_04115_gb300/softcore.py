"""Soft-core parameter fit on the GPU (arXiv:2507.04115 Sec. 3.1: a is chosen so that the
ground-state energy of H0 = p^2/2 - Z/sqrt(x^2 + a^2) equals the target of the atom).

The ground-state energy increases monotonically with a (the well gets shallower everywhere), so
the fit brackets the root and narrows it by evaluating many candidate values of a in one batched
ground-state call (one class, one CTA each), shrinking the bracket 32-fold per round.
"""
from __future__ import annotations

import numpy as np

from . import tdse


def ground_energies(a_values, N, dx, charge=1.0, scheme=tdse.TDSE_FULL_CN, device=0, dtau=0.1, max_iter=20000,
                    tol=1e-14):
    a_values = np.asarray(a_values, dtype=np.float64)
    n = a_values.size
    b = tdse.Batch([N] * n, dx, a_values, [0] * n, 0.05, charge=charge, absorber=None, scheme=scheme, device=device)
    try:
        e, _ = b.ground_state(dtau=dtau, max_iter=max_iter, tol=tol)
    finally:
        b.close()
    return e


def fit_softening(target, N, dx, charge=1.0, scheme=tdse.TDSE_FULL_CN, device=0, lo=0.3, hi=4.0, rounds=6,
                  width=33):
    """a such that the discrete ground-state energy equals ``target`` (bracketing search)."""
    for _ in range(rounds):
        grid = np.linspace(lo, hi, width)
        e = ground_energies(grid, N, dx, charge, scheme, device)
        above = np.nonzero(e > target)[0]
        if above.size == 0 or above[0] == 0:
            raise ValueError("target energy %.6f not bracketed by a in [%g, %g]" % (target, lo, hi))
        k = above[0]
        lo, hi = grid[k - 1], grid[k]
        e_lo, e_hi = e[k - 1], e[k]
        if hi - lo < 1e-13:
            break
    # final linear interpolation inside the bracket
    return float(lo + (target - e_lo) * (hi - lo) / (e_hi - e_lo))
