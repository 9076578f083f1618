"""The truncated sweeps the propagation kernels run per grid segment (no GPU).

Each warp solves A y = psi on its own segment [lo, hi) only: the forward elimination starts K rows
before lo from zero multipliers, the back substitution K rows after hi from zero.  A =
1 + i dt/2 H(Ebar) is diagonally dominant with Re(pivot) >= 1, so a perturbation at the start of a
sweep shrinks by |gamma| <= beta = dt/(4 dx^2) per row, and K is chosen with beta^K < 1e-18
(halo_for_beta).  This file restates that segmented algorithm in numpy and compares it with an
exact banded solve on the volume configuration: the segments agree with the exact solution to
rounding, and they do not with a halo far shorter than the rule's (so the comparison can fail).
"""
import math

import numpy as np
from scipy.linalg import solve_banded


def _halo(beta):
    # the rule of the planner: smallest K >= 8 with beta^K < 1e-18
    return max(8, math.ceil(math.log(1e-18) / math.log(beta)))


def _segment_solve(lo_c, di, up_c, r, lo, hi, K):
    """y on [lo, hi) from sweeps over [lo - K, hi + K) clipped to the walls (Thomas algorithm)."""
    N = di.size
    a, b = max(0, lo - K), min(N, hi + K)
    cp = np.zeros(b - a, dtype=complex)
    dp = np.zeros(b - a, dtype=complex)
    for k, j in enumerate(range(a, b)):
        piv = di[j] - (lo_c * cp[k - 1] if k > 0 else 0.0)
        cp[k] = up_c / piv
        dp[k] = (r[j] - (lo_c * dp[k - 1] if k > 0 else 0.0)) / piv
    y = np.zeros(b - a, dtype=complex)
    y[-1] = dp[-1]
    for k in range(b - a - 2, -1, -1):
        y[k] = dp[k] - cp[k] * y[k + 1]
    return y[lo - a: hi - a]


def _system(N, dx, dt, a, Ebar):
    x = (np.arange(N) - 0.5 * (N - 1)) * dx
    V = -1.0 / np.sqrt(x * x + a * a)
    h = 0.5 * dt
    di = 1.0 + 1j * h * (1.0 / dx ** 2 + V + x * Ebar)
    off = -1j * h * 0.5 / dx ** 2        # = -i beta
    return di, off


def test_segments_match_the_exact_solve_at_the_rule_halo():
    N, dx, dt, a = 4096, 0.15, 0.02, 1.19     # the volume batch's grid and step
    beta = dt / (4 * dx * dx)
    K = _halo(beta)
    assert abs(beta - 0.2222) < 1e-3 and K == 28
    rng = np.random.default_rng(3)
    r = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    for Ebar in (0.0, 0.08, -0.15):
        di, off = _system(N, dx, dt, a, Ebar)
        ab = np.zeros((3, N), dtype=complex)
        ab[0, 1:] = off
        ab[1] = di
        ab[2, :-1] = off
        y = solve_banded((1, 1), ab, r)
        P = 12                                  # segments of the volume launch (12 warps)
        m = -(-N // P)
        ys = np.concatenate([_segment_solve(off, di, off, r, w * m, min(N, (w + 1) * m), K) for w in range(P)])
        assert np.max(np.abs(ys - y)) < 1e-14 * np.max(np.abs(y)), Ebar
        # a halo of 5 rows leaves errors near beta^5 ~ 5e-4
        ys5 = np.concatenate([_segment_solve(off, di, off, r, w * m, min(N, (w + 1) * m), 5) for w in range(P)])
        assert np.max(np.abs(ys5 - y)) > 1e-6 * np.max(np.abs(y))


def test_numerov_substitutions_with_exact_factors():
    """NUMEROV_SPLIT factors its constant A = M2 + i h (-Delta2/2 + M2 V) once over the whole grid;
    the kernels truncate only the two substitutions, whose errors shrink by |L_j| and |C_j| per
    row, so the halo comes from rho = max_j max(|L_j|, |C_j|)."""
    N, dx, dt, a = 4096, 0.15, 0.02, 1.19
    x = (np.arange(N) - 0.5 * (N - 1)) * dx
    V = -1.0 / np.sqrt(x * x + a * a)
    h = 0.5 * dt
    lo_c = 1 / 12 + 1j * h * (-0.5 / dx ** 2 + np.concatenate([[0.0], V[:-1]]) / 12)   # A[j, j-1]
    up_c = 1 / 12 + 1j * h * (-0.5 / dx ** 2 + np.concatenate([V[1:], [0.0]]) / 12)    # A[j, j+1]
    di = 10 / 12 + 1j * h * (1.0 / dx ** 2 + 10 / 12 * V)
    # exact factors over the whole grid, scaled as the kernels store them: pivots p_j,
    # L_j = A[j, j-1] / p_j, C_j = A[j, j+1] / p_j
    p = np.empty(N, dtype=complex)
    p[0] = di[0]
    for j in range(1, N):
        p[j] = di[j] - lo_c[j] * up_c[j - 1] / p[j - 1]
    L = np.zeros(N, dtype=complex)
    L[1:] = lo_c[1:] / p[1:]
    C = up_c / p
    rho = max(np.max(np.abs(L)), np.max(np.abs(C[:-1])))
    K = _halo(rho)
    assert rho < 0.85
    rng = np.random.default_rng(4)
    r = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ab = np.zeros((3, N), dtype=complex)
    ab[0, 1:] = up_c[:-1]
    ab[1] = di
    ab[2, :-1] = lo_c[1:]
    y = solve_banded((1, 1), ab, r)

    def seg(lo, hi, K):
        a0, b0 = max(0, lo - K), min(N, hi + K)
        z = np.zeros(b0 - a0, dtype=complex)              # forward: z_j = r_j / p_j - L_j z_{j-1}
        for k, j in enumerate(range(a0, b0)):
            z[k] = r[j] / p[j] - (L[j] * z[k - 1] if k > 0 else 0.0)
        u = np.zeros(b0 - a0, dtype=complex)              # back: u_j = z_j - C_j u_{j+1}
        for k in range(b0 - a0 - 1, -1, -1):
            u[k] = z[k] - (C[a0 + k] * u[k + 1] if k + 1 < b0 - a0 else 0.0)
        return u[lo - a0: hi - a0]

    P = 12
    m = -(-N // P)
    ys = np.concatenate([seg(w * m, min(N, (w + 1) * m), K) for w in range(P)])
    assert np.max(np.abs(ys - y)) < 1e-14 * np.max(np.abs(y))
    ys5 = np.concatenate([seg(w * m, min(N, (w + 1) * m), 5) for w in range(P)])
    assert np.max(np.abs(ys5 - y)) > 1e-6 * np.max(np.abs(y))


def _halo_double_rows(beta, K):
    # a split of a halo: the rows nearest the segment in double, enough for an error of float
    # rounding (1e-7 of the values) to shrink below 1e-18 (beta^K2 < 1e-11); the rest in float
    return min(K, max(4, math.ceil(math.log(1e-11) / math.log(beta))))


def _segment_solve_split(di, off, r, lo, hi, K, K2):
    """As _segment_solve, but the outer K - K2 rows of each halo run in float32 (complex64): the
    forward sweep from the top of the halo to K2 rows before the segment, and both sweeps over the
    bottom halo's rows beyond K2 after the segment.  (The MIXED path runs its whole halo in float;
    an FP64 variant with this split was measured slower than the all-double sweep and not kept.)"""
    N = di.size
    a, b = max(0, lo - K), min(N, hi + K)
    tf, bd = max(a, lo - K2), min(b, hi + K2)
    c32, d32 = np.complex64(0), np.complex64(0)
    for j in range(a, tf):                                   # float forward rows
        piv = np.complex64(di[j]) - np.complex64(off) * c32
        c32 = np.complex64(off) / piv
        d32 = (np.complex64(r[j]) - np.complex64(off) * d32) / piv
    cp = np.zeros(b - a, dtype=complex)
    dp = np.zeros(b - a, dtype=complex)
    c64, d64 = complex(c32), complex(d32)
    for j in range(tf, bd):                                  # double forward rows
        piv = di[j] - off * c64
        c64 = off / piv
        d64 = (r[j] - off * d64) / piv
        cp[j - a], dp[j - a] = c64, d64
    c32, d32 = np.complex64(c64), np.complex64(d64)
    cf = np.zeros(b - bd, dtype=np.complex64)
    df = np.zeros(b - bd, dtype=np.complex64)
    for j in range(bd, b):                                   # float forward rows after the segment
        piv = np.complex64(di[j]) - np.complex64(off) * c32
        c32 = np.complex64(off) / piv
        d32 = (np.complex64(r[j]) - np.complex64(off) * d32) / piv
        cf[j - bd], df[j - bd] = c32, d32
    y32 = np.complex64(0)
    for j in range(b - 1, bd - 1, -1):                       # float back substitution
        y32 = df[j - bd] - cf[j - bd] * y32
    y = np.zeros(b - a, dtype=complex)
    yn = complex(y32)
    for j in range(bd - 1, lo - 1, -1):                      # double back substitution
        yn = dp[j - a] - cp[j - a] * yn
        y[j - a] = yn
    return y[lo - a: hi - a]


def test_float_outer_halo_rows_stay_at_double_rounding():
    """Running the outer K - K2 rows of every halo in float leaves the segments at double rounding
    against the exact solve: the float error (~1e-7 of the values) enters K2 rows before the
    segment and shrinks by beta^K2 < 1e-11; with too few double rows it shows."""
    N, dx, dt, a = 4096, 0.15, 0.02, 1.19
    beta = dt / (4 * dx * dx)
    K = _halo(beta)
    K2 = _halo_double_rows(beta, K)
    assert (K, K2) == (28, 17)
    rng = np.random.default_rng(5)
    r = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    P = 12
    m = -(-N // P)
    for Ebar in (0.0, 0.08, -0.15):
        di, off = _system(N, dx, dt, a, Ebar)
        ab = np.zeros((3, N), dtype=complex)
        ab[0, 1:] = off
        ab[1] = di
        ab[2, :-1] = off
        y = solve_banded((1, 1), ab, r)
        ys = np.concatenate([_segment_solve_split(di, off, r, w * m, min(N, (w + 1) * m), K, K2) for w in range(P)])
        assert np.max(np.abs(ys - y)) < 1e-14 * np.max(np.abs(y)), Ebar
        # four double rows leave the float rounding at beta^4 ~ 2e-3 of ~1e-7
        ys4 = np.concatenate([_segment_solve_split(di, off, r, w * m, min(N, (w + 1) * m), K, 4) for w in range(P)])
        assert np.max(np.abs(ys4 - y)) > 1e-12 * np.max(np.abs(y))
