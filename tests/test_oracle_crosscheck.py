"""Cross-check of the C oracle's stepping against an independent formulation (no GPU).

The oracle sweeps a hand-written Thomas solver over coefficient arrays; here the same schemes are
written as banded matrices built from the readings (cell-centred grid, Dirichlet walls, FULL_CN with
the midpoint field, NUMEROV_SPLIT as Sec. 4.2's three substeps) and stepped with
scipy.linalg.solve_banded.  The two share no code: an index shift in the off-diagonals, a wrong
time level of the field, a dropped potential term or a transposed band would separate them far
beyond rounding.  This complements the pins in test_oracle_pins.py (closed forms, invariants,
eigensolvers), which fix the mathematics; this file fixes the bookkeeping on a generic input
(complex initial state, field with noise, mask on).
"""
import numpy as np
import pytest
from scipy.linalg import solve_banded

FULL_CN, NUMEROV = 0, 1


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def _banded(lo, di, up):
    """(3, N) array in solve_banded's layout for the tridiagonal matrix with sub-diagonal lo[1:],
    diagonal di and super-diagonal up[:-1] (row j: lo[j] psi_{j-1} + di[j] psi_j + up[j] psi_{j+1})."""
    N = di.size
    ab = np.zeros((3, N), dtype=np.complex128)
    ab[0, 1:] = up[:-1]
    ab[1, :] = di
    ab[2, :-1] = lo[1:]
    return ab


def _apply(lo, di, up, v):
    r = di * v
    r[1:] += lo[1:] * v[:-1]
    r[:-1] += up[:-1] * v[1:]
    return r


def _reference(psi0, E, dx, dt, a, m, scheme):
    N = psi0.size
    x = (np.arange(N) - 0.5 * (N - 1)) * dx
    V = -1.0 / np.sqrt(x * x + a * a)
    dV = x / (x * x + a * a) ** 1.5
    h = 0.5 * dt
    lap_off = np.full(N, 1.0 / dx ** 2)
    lap_di = np.full(N, -2.0 / dx ** 2)
    psi = psi0.astype(np.complex128).copy()
    d = np.empty(E.size)
    acc = np.empty(E.size)

    def obs(p, En):
        rho = np.abs(p) ** 2
        return np.sum(x * rho) * dx, (np.sum(dV * rho) + En * np.sum(rho)) * dx

    d[0], acc[0] = obs(psi, E[0])
    for n in range(E.size - 1):
        if scheme == FULL_CN:
            Eb = 0.5 * (E[n] + E[n + 1])
            Hlo, Hdi, Hup = -0.5 * lap_off, -0.5 * lap_di + V + x * Eb, -0.5 * lap_off
            rhs = _apply(-1j * h * Hlo, 1 - 1j * h * Hdi, -1j * h * Hup, psi)
            psi = solve_banded((1, 1), _banded(1j * h * Hlo, 1 + 1j * h * Hdi, 1j * h * Hup), rhs)
        else:
            # M2 = tridiag(1, 10, 1)/12; K = -Delta2/2 + M2 diag(V): K_{j,j+-1} = -1/(2dx^2) + V_{j+-1}/12
            Mlo, Mdi, Mup = np.full(N, 1 / 12), np.full(N, 10 / 12), np.full(N, 1 / 12)
            Klo = -0.5 * lap_off + np.concatenate([[0.0], V[:-1]]) / 12
            Kup = -0.5 * lap_off + np.concatenate([V[1:], [0.0]]) / 12
            Kdi = -0.5 * lap_di + 10 / 12 * V
            rhs = _apply(Mlo - 1j * h * Klo, Mdi - 1j * h * Kdi, Mup - 1j * h * Kup, psi)
            psi = solve_banded((1, 1), _banded(Mlo + 1j * h * Klo, Mdi + 1j * h * Kdi, Mup + 1j * h * Kup), rhs)
            psi = psi * np.exp(-1j * dt * E[n] * x)
        psi = psi * m
        d[n + 1], acc[n + 1] = obs(psi, E[n + 1])
    return psi, d, acc


@pytest.mark.parametrize("scheme", [FULL_CN, NUMEROV])
def test_oracle_stepping_matches_banded_formulation(oracle_mod, scheme):
    rng = np.random.default_rng(11)
    N, dx, dt, a = 96, 0.25, 0.05, 1.3
    x = (np.arange(N) - 0.5 * (N - 1)) * dx
    psi0 = np.exp(-((x - 1.5) ** 2) / 4 + 0.8j * x) * (1 + 0.1 * rng.standard_normal(N))
    psi0 /= np.sqrt(np.sum(np.abs(psi0) ** 2) * dx)
    nt = 60
    E = 0.05 * np.sin(0.3 * np.arange(nt + 1) * dt) + 0.01 * rng.standard_normal(nt + 1)
    m = oracle_mod.mask(N, dx, 4.0, 0.125)
    psi_o, d_o, a_o = oracle_mod.propagate(psi0, E, dx, dt, a, scheme=scheme, mask_values=m)
    psi_r, d_r, a_r = _reference(psi0, E, dx, dt, a, m, scheme)
    assert np.max(np.abs(psi_o - psi_r)) < 1e-12
    assert np.max(np.abs(d_o - d_r)) < 1e-12 * max(1.0, np.max(np.abs(d_r)))
    assert np.max(np.abs(a_o - a_r)) < 1e-12 * max(1.0, np.max(np.abs(a_r)))
