"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test would fail on a plausible mistake in the oracle: a dropped term, a wrong sign or
index, a transposed operand, the wrong time level of the field.  None of them re-types the
oracle's own formulas: they compare against closed forms, brute-force eigensolvers,
invariants, symmetry and convergence orders.
"""
import numpy as np
import pytest
from scipy.fft import dst, idst
from scipy.linalg import eigh

FULL_CN, NUMEROV = 0, 1


def _gauss(x, x0, sigma, p0):
    return (2 * np.pi * sigma ** 2) ** -0.25 * np.exp(-((x - x0) ** 2) / (4 * sigma ** 2) + 1j * p0 * (x - x0))


def _norm(psi, dx):
    return float(np.sum(np.abs(psi) ** 2) * dx)


def _sin2_pulse(Nt, dt, E0, w, ncyc):
    t = np.arange(Nt + 1) * dt
    Tp = ncyc * 2 * np.pi / w
    return np.where(t <= Tp, E0 * np.sin(np.pi * t / Tp) ** 2 * np.cos(w * (t - Tp / 2)), 0.0)


# ---------------------------------------------------------------- free propagation: exact discrete pin

@pytest.mark.parametrize("scheme", [FULL_CN, NUMEROV])
def test_free_propagation_matches_dst_eigenbasis(oracle_mod, scheme):
    """V = 0, E = 0, no mask.  -Delta2/2 (and M2^{-1}(-Delta2/2)) on the Dirichlet grid are diagonal in
    the DST-I basis with eigenvalues lam_k = (2/dx^2) sin^2(k pi / (2(N+1))) (Numerov: lam_k / (1 - s_k/3),
    s_k = sin^2(...)); Crank-Nicolson multiplies mode k by (1 - i h lam_k)/(1 + i h lam_k) per step."""
    N, dx, dt, nsteps = 200, 0.3, 0.05, 100
    x, _, _ = oracle_mod.grid(N, dx, 1.0, Z=0.0)
    psi0 = _gauss(x, -5.0, 2.0, 1.5)
    E = np.zeros(nsteps + 1)
    psi, _, _ = oracle_mod.propagate(psi0, E, dx, dt, 1.0, Z=0.0, scheme=scheme)
    k = np.arange(1, N + 1)
    s = np.sin(k * np.pi / (2 * (N + 1))) ** 2
    lam = 2.0 / dx ** 2 * s
    if scheme == NUMEROV:
        lam = lam / (1.0 - s / 3.0)
    h = dt / 2
    fac = ((1 - 1j * h * lam) / (1 + 1j * h * lam)) ** nsteps
    coef = dst(psi0.real, type=1, norm="ortho") + 1j * dst(psi0.imag, type=1, norm="ortho")
    coef = coef * fac
    exact = idst(coef.real, type=1, norm="ortho") + 1j * idst(coef.imag, type=1, norm="ortho")
    assert np.max(np.abs(psi - exact)) < 1e-12


def test_free_gaussian_closed_form_second_order(oracle_mod):
    """Continuous free Gaussian packet: the FULL_CN error falls ~4x when dx and dt are halved."""
    T, x0, sigma, p0 = 4.0, -3.0, 1.5, 1.0
    errs = []
    for dx, dt in [(0.2, 0.1), (0.1, 0.05), (0.05, 0.025)]:
        N = int(round(80 / dx))
        x, _, _ = oracle_mod.grid(N, dx, 1.0, Z=0.0)
        nsteps = int(round(T / dt))
        psi, _, _ = oracle_mod.propagate(_gauss(x, x0, sigma, p0), np.zeros(nsteps + 1), dx, dt, 1.0, Z=0.0)
        c = 1 + 1j * T / (2 * sigma ** 2)
        exact = ((2 * np.pi * sigma ** 2) ** -0.25 * c ** -0.5
                 * np.exp(-((x - x0 - p0 * T) ** 2) / (4 * sigma ** 2 * c) + 1j * p0 * (x - x0) - 1j * p0 ** 2 * T / 2))
        errs.append(np.sqrt(np.sum(np.abs(psi - exact) ** 2) * dx))
    assert errs[0] < 5e-2
    assert 3.5 < errs[0] / errs[1] < 4.5
    assert 3.5 < errs[1] / errs[2] < 4.5


# ---------------------------------------------------------------- norm, reversibility, symmetry

@pytest.mark.parametrize("scheme", [FULL_CN, NUMEROV])
def test_norm_conserved_with_field(oracle_mod, scheme):
    N, dx, dt = 800, 0.2, 0.05
    a = 1.19
    psi0, _, _ = oracle_mod.ground_state(N, dx, a, scheme=scheme, tol=1e-12)
    E = _sin2_pulse(1500, dt, 0.05, 0.057, 1)
    psi, d, acc = oracle_mod.propagate(psi0, E, dx, dt, a, scheme=scheme)
    assert abs(_norm(psi, dx) - 1.0) < 1e-12
    assert np.all(np.isfinite(d)) and np.all(np.isfinite(acc))


def test_mask_reduces_norm_monotonically(oracle_mod):
    N, dx, dt = 600, 0.2, 0.05
    a = 1.19
    psi0, _, _ = oracle_mod.ground_state(N, dx, a, tol=1e-12)
    E = _sin2_pulse(1200, dt, 0.12, 0.057, 1)
    m = oracle_mod.mask(N, dx, 20.0, 0.125)
    norms = []
    psi = psi0
    for c in range(4):
        psi, _, _ = oracle_mod.propagate(psi, E, dx, dt, a, mask_values=m, n_begin=c * 300, n_end=(c + 1) * 300)
        norms.append(_norm(psi, dx))
    assert norms[-1] < 1.0 - 1e-7
    assert all(b <= a_ + 1e-13 for a_, b in zip([1.0] + norms[:-1], norms))


def test_reversibility_full_cn(oracle_mod):
    """FULL_CN is exactly reversible: stepping back with -dt and the reversed field inverts each step."""
    N, dx, dt = 500, 0.2, 0.05
    a = 1.19
    psi0, _, _ = oracle_mod.ground_state(N, dx, a, tol=1e-12)
    E = _sin2_pulse(800, dt, 0.08, 0.057, 1)
    psi1, _, _ = oracle_mod.propagate(psi0, E, dx, dt, a)
    psi2, _, _ = oracle_mod.propagate(psi1, E[::-1].copy(), dx, -dt, a)
    assert np.max(np.abs(psi2 - psi0)) < 1e-12


@pytest.mark.parametrize("scheme", [FULL_CN, NUMEROV])
def test_field_reversal_symmetry(oracle_mod, scheme):
    """Symmetric grid and potential: E -> -E maps x -> -x, so d -> -d and a -> -a."""
    N, dx, dt = 500, 0.2, 0.05
    a = 1.19
    psi0, _, _ = oracle_mod.ground_state(N, dx, a, scheme=scheme, tol=1e-12)
    E = _sin2_pulse(600, dt, 0.08, 0.057, 1)
    m = oracle_mod.mask(N, dx, 20.0, 0.125)
    _, d1, a1 = oracle_mod.propagate(psi0, E, dx, dt, a, scheme=scheme, mask_values=m)
    _, d2, a2 = oracle_mod.propagate(psi0, -E, dx, dt, a, scheme=scheme, mask_values=m)
    assert np.max(np.abs(d1 + d2)) < 1e-11 * np.max(np.abs(d1))
    assert np.max(np.abs(a1 + a2)) < 1e-11 * np.max(np.abs(a1))


# ---------------------------------------------------------------- ground state

@pytest.mark.parametrize("scheme", [FULL_CN, NUMEROV])
def test_ground_state_matches_dense_eigensolver(oracle_mod, scheme):
    """Imaginary time vs. dense diagonalisation of the discrete H0 on a tiny grid."""
    N, dx, a = 96, 0.25, 1.19
    x, V, _ = oracle_mod.grid(N, dx, a)
    lap = (np.diag(np.full(N - 1, 1.0), -1) - 2 * np.eye(N) + np.diag(np.full(N - 1, 1.0), 1)) / dx ** 2
    if scheme == FULL_CN:
        H = -0.5 * lap + np.diag(V)
    else:
        M2 = np.eye(N) + dx ** 2 / 12.0 * lap
        H = np.linalg.solve(M2, -0.5 * lap) + np.diag(V)
        H = 0.5 * (H + H.T)
    w, U = eigh(H)
    psi, e, it = oracle_mod.ground_state(N, dx, a, scheme=scheme, tol=1e-15, max_iter=20000)
    assert abs(e - w[0]) < 1e-12
    assert psi[N // 2].real > 0 and np.all(np.abs(psi.imag) == 0)   # reading GS: real, positive at the centre
    u = U[:, 0] / np.sqrt(dx)
    overlap = abs(np.sum(np.conj(psi) * u) * dx)
    assert overlap > 1 - 1e-12
    assert abs(oracle_mod.lowest_eigenvalue(N, dx, a, scheme=scheme) - w[0]) < 1e-12


def test_softcore_fit_and_discretisation_orders(oracle_mod):
    """a^2 = 2 soft-core: three-point energies converge at order 2, Numerov at order 4, and both
    Richardson limits agree with each other (two independent discretisations, same continuum value)."""
    a = np.sqrt(2.0)
    e_fd, e_nu = [], []
    for dx in (0.2, 0.1, 0.05):
        N = int(round(400 / dx))
        e_fd.append(oracle_mod.lowest_eigenvalue(N, dx, a, scheme=FULL_CN))
        e_nu.append(oracle_mod.lowest_eigenvalue(N, dx, a, scheme=NUMEROV))
    r_fd = (e_fd[0] - e_fd[1]) / (e_fd[1] - e_fd[2])
    r_nu = (e_nu[0] - e_nu[1]) / (e_nu[1] - e_nu[2])
    assert 3.8 < r_fd < 4.2
    assert 15.0 < r_nu < 17.0
    lim_fd = e_fd[2] + (e_fd[2] - e_fd[1]) / 3.0
    lim_nu = e_nu[2] + (e_nu[2] - e_nu[1]) / 15.0
    assert abs(lim_fd - lim_nu) < 1e-8
    assert abs(lim_nu + 0.5) < 1e-7           # the hydrogen-like soft-core model
    # the fit helper reproduces its target on the discrete operator
    a_fit = oracle_mod.fit_softening(-0.579, 400, 0.2)
    assert abs(oracle_mod.lowest_eigenvalue(400, 0.2, a_fit) + 0.579) < 1e-12


def test_stationarity_of_discrete_eigenstate(oracle_mod):
    """Field off, mask off: an exact eigenvector of the discrete H0 only acquires the CN phase
    ((1 - i h E)/(1 + i h E))^n; <x> and <dV/dx> vanish by parity."""
    from scipy.linalg import eigh_tridiagonal
    N, dx, dt, a, n = 400, 0.2, 0.05, 1.19, 300
    x, V, _ = oracle_mod.grid(N, dx, a)
    w, U = eigh_tridiagonal(1 / dx ** 2 + V, np.full(N - 1, -0.5 / dx ** 2), select="i", select_range=(0, 0))
    psi0 = (U[:, 0] / np.sqrt(dx)).astype(np.complex128)
    psi, d, acc = oracle_mod.propagate(psi0, np.zeros(n + 1), dx, dt, a)
    h = dt / 2
    ph = ((1 - 1j * h * w[0]) / (1 + 1j * h * w[0])) ** n
    assert np.max(np.abs(psi - ph * psi0)) < 1e-12
    assert np.max(np.abs(d)) < 1e-12 and np.max(np.abs(acc)) < 1e-12


# ---------------------------------------------------------------- field coupling, observables

def test_ramped_field_free_electron_midpoint_order(oracle_mod):
    """V = 0, E(t) = alpha t:  <x>(t) = x0 + p0 t - alpha t^3 / 6 exactly in the continuum.
    FULL_CN takes the field at the midpoint of each step; feeding it the field shifted by half a
    step (which is what taking E_n instead of the midpoint would amount to) gives a first-order
    error that is an order of magnitude larger and halves with dt."""
    alpha, T, x0, sigma, p0 = 0.02, 6.0, 0.0, 2.0, 0.3
    dx = 0.02
    N = int(round(90 / dx))
    x, _, _ = oracle_mod.grid(N, dx, 1.0, Z=0.0)
    exact = x0 + p0 * T - alpha * T ** 3 / 6
    good, shifted = [], []
    for dt in (0.2, 0.1):
        n = int(round(T / dt))
        E = alpha * np.arange(n + 1) * dt
        _, d, _ = oracle_mod.propagate(_gauss(x, x0, sigma, p0), E, dx, dt, 1.0, Z=0.0)
        good.append(abs(d[-1] - exact))
        _, d2, _ = oracle_mod.propagate(_gauss(x, x0, sigma, p0), E - alpha * dt / 2, dx, dt, 1.0, Z=0.0)
        shifted.append(abs(d2[-1] - exact))
    assert good[0] < 0.1 * shifted[0] and good[1] < 0.1 * shifted[1]
    assert 1.8 < shifted[0] / shifted[1] < 2.2
    assert good[0] / good[1] > 3.0


@pytest.mark.parametrize("scheme", [FULL_CN, NUMEROV])
def test_ehrenfest_acceleration(oracle_mod, scheme):
    """a_n = <dV/dx> + E_n equals -d^2<x>/dt^2 (App. A, Eq. "Current_der_TDSE1D" with Ehrenfest's
    theorem), up to the discretisation error, which shrinks when dx and dt are refined.  The window
    ends before any part of the packet reaches the walls (no mask here)."""
    res = []
    for dx, dt in [(0.2, 0.05), (0.1, 0.025)]:
        N = int(round(240 / dx))
        a = 1.19
        psi0, _, _ = oracle_mod.ground_state(N, dx, a, scheme=scheme, tol=1e-13)
        n = int(round(200.0 / dt))
        E = _sin2_pulse(n, dt, 0.06, 0.057, 2)
        _, d, acc = oracle_mod.propagate(psi0, E, dx, dt, a, scheme=scheme)
        dd = (d[2:] - 2 * d[1:-1] + d[:-2]) / dt ** 2
        res.append(np.max(np.abs(dd + acc[1:-1])) / np.max(np.abs(acc)))
    assert res[0] < 2e-2
    assert res[0] / res[1] > 2.0


@pytest.mark.parametrize("scheme", [FULL_CN, NUMEROV])
def test_dipole_sign_under_static_field(oracle_mod, scheme):
    """A weak static field E > 0 pushes the electron (charge -1) towards negative x: <x> < 0
    while the acceleration-form source <dV/dx> + E stays consistent with it."""
    N, dx, dt, a = 600, 0.2, 0.05, 1.19
    psi0, _, _ = oracle_mod.ground_state(N, dx, a, scheme=scheme, tol=1e-13)
    n = 400
    E = 0.002 * np.minimum(1.0, np.arange(n + 1) * dt / 10.0)
    _, d, acc = oracle_mod.propagate(psi0, E, dx, dt, a, scheme=scheme)
    assert d[-1] < 0.0
    assert acc[5] > 0.0


def test_schemes_agree_to_discretisation_error(oracle_mod):
    """FULL_CN and the paper's NUMEROV_SPLIT discretise the same equation: their dipoles agree up to
    the discretisation errors, and the gap shrinks when dx and dt are halved."""
    gaps = []
    for dx, dt in [(0.2, 0.05), (0.1, 0.025)]:
        N = int(round(200 / dx))
        n = int(round(150.0 / dt))
        E = _sin2_pulse(n, dt, 0.05, 0.057, 1)
        out = []
        for scheme in (FULL_CN, NUMEROV):
            a = oracle_mod.fit_softening(-0.579, N, dx, scheme=scheme)
            psi0, _, _ = oracle_mod.ground_state(N, dx, a, scheme=scheme, tol=1e-13)
            _, d, _ = oracle_mod.propagate(psi0, E, dx, dt, a, scheme=scheme)
            out.append(d)
        gaps.append(np.max(np.abs(out[0] - out[1])) / np.max(np.abs(out[0])))
    assert gaps[0] < 5e-2
    assert gaps[0] / gaps[1] > 2.0


# ---------------------------------------------------------------- harmonic cutoff (Sec. 7.1)

def test_harmonic_cutoff_law(oracle_mod):
    """The single-atom configuration (800 nm, 4-cycle sin^2, 1e14 W/cm^2, E_g = -0.579) gives a
    harmonic plateau that ends near the semi-classical cutoff q_cut = (I_p + 3.17 U_p)/w = 22.4
    (Sec. 7.1), U_p = E0^2/(4 w^2): the yield first drops below 1 % of the plateau within ten orders
    above q_cut and is down by 1e5 at q ~ 35-41.  A wrong field coupling moves or removes the
    cutoff."""
    from paper_2507_04115_gb300 import inputs
    wl = inputs.single_atom()
    N, dx, dt = int(wl.N[0]), float(wl.dx[0]), wl.dt
    w, E0 = float(wl.omega[0]), float(wl.E0[0])
    a = oracle_mod.fit_softening(-0.579, N, dx)
    psi0, _, _ = oracle_mod.ground_state(N, dx, a, tol=1e-12)
    _, _, acc = oracle_mod.propagate(psi0, wl.field_rows()[0], dx, dt, a,
                                     mask_values=oracle_mod.mask(N, dx, 20.0, 0.125))
    S = oracle_mod.spectrum(acc * np.hanning(acc.size), dt)
    q = 2 * np.pi * np.arange(acc.size) / (acc.size * dt) / w

    def band(q0):
        return S[np.abs(q - q0) < 0.5].sum()

    q_cut = (0.579 + 3.17 * E0 ** 2 / (4 * w ** 2)) / w
    assert abs(q_cut - 22.4) < 0.1
    plateau = np.mean([band(k) for k in range(11, 22, 2)])
    assert plateau > 1e5 * np.mean([band(k) for k in range(35, 42, 2)])
    drop = next(k for k in range(11, 61, 2) if band(k) < 1e-2 * plateau)
    assert q_cut <= drop <= q_cut + 10, drop


# ---------------------------------------------------------------- mask and spectrum

def test_mask_shape(oracle_mod):
    N, dx, w, p = 2000, 0.2, 20.0, 0.125
    x, _, _ = oracle_mod.grid(N, dx, 1.0)
    m = oracle_mod.mask(N, dx, w, p)
    xb = N * dx / 2 - w
    assert np.all(m[np.abs(x) <= xb] == 1.0)
    edge = np.abs(x) > xb
    assert np.all((m[edge] < 1.0) & (m[edge] >= 0.0))
    right = x > xb
    assert np.all(np.diff(m[right]) <= 0.0)
    assert np.allclose(m, m[::-1], atol=0, rtol=0)
    j = np.argmin(np.abs(x - (xb + w / 2)))
    assert abs(m[j] - np.cos(np.pi / 2 * (x[j] - xb) / w) ** p) < 1e-15
    assert abs(np.interp(xb + w / 2, x, m) - 2 ** (-p / 2)) < 2e-3
    assert np.all(oracle_mod.mask(N, dx, 0.0, p) == 1.0)


def test_spectrum_against_direct_sum(oracle_mod):
    rng = np.random.default_rng(5)
    L, dt = 37, 0.3
    a = rng.standard_normal(L)
    S = oracle_mod.spectrum(a, dt)
    for k in range(L):
        s = 0j
        for n in range(L):
            s += a[n] * np.exp(-2j * np.pi * k * n / L)
        assert abs(S[k] - abs(s) ** 2 * dt * dt) < 1e-12 * (1 + abs(s) ** 2)
    k0 = 5
    tone = np.cos(2 * np.pi * k0 * np.arange(L) / L)
    St = oracle_mod.spectrum(tone, dt)
    assert abs(St[k0] - (L / 2) ** 2 * dt * dt) < 1e-10
    assert np.max(np.delete(St, [k0, L - k0])) < 1e-20


# ---------------------------------------------------------------- discrete adjoint

def test_adjoint_matches_central_differences(oracle_mod):
    """dL/dE of a loss L = sum gd_n d_n + ga_n a_n (random weights) against central finite
    differences of the forward oracle on several field samples, mask on."""
    rng = np.random.default_rng(7)
    N, dx, dt, a = 300, 0.2, 0.05, 1.19
    nt = 240
    psi0, _, _ = oracle_mod.ground_state(N, dx, a, tol=1e-13)
    E = _sin2_pulse(nt, dt, 0.07, 0.057, 1) + 0.01 * rng.standard_normal(nt + 1)
    m = oracle_mod.mask(N, dx, 15.0, 0.125)
    gd = rng.standard_normal(nt + 1)
    ga = rng.standard_normal(nt + 1)

    def loss(Ev):
        _, d, acc = oracle_mod.propagate(psi0, Ev, dx, dt, a, mask_values=m)
        return float(np.dot(gd, d) + np.dot(ga, acc))

    gE = oracle_mod.adjoint(psi0, E, dx, dt, a, gd, ga, mask_values=m)
    for k in [0, 1, 17, 120, 239, 240]:
        eps = 1e-5
        Ep, Em = E.copy(), E.copy()
        Ep[k] += eps
        Em[k] -= eps
        fd = (loss(Ep) - loss(Em)) / (2 * eps)
        assert abs(fd - gE[k]) < 1e-6 * (abs(fd) + 1e-3), (k, fd, gE[k])
    # directional derivative along a random field perturbation
    v = rng.standard_normal(nt + 1)
    eps = 1e-6
    fd = (loss(E + eps * v) - loss(E - eps * v)) / (2 * eps)
    assert abs(fd - np.dot(gE, v)) < 1e-6 * abs(fd)


def test_adjoint_with_strong_absorption(oracle_mod):
    """A packet running into the absorber (the norm falls to 1 %), loss = a at the last sample with a
    large final field: dL/dE_k then goes mostly through E_Nt times the norm's dependence on E_k,
    which the unitary part cannot see.  Central differences at several samples."""
    N, dx, dt, a = 300, 0.2, 0.05, 1.19
    nt = 160
    x, _, _ = oracle_mod.grid(N, dx, a)
    psi0 = np.exp(-(x - 14.0) ** 2 / 4.0 + 2.0j * x)
    psi0 /= np.sqrt(np.sum(np.abs(psi0) ** 2) * dx)
    rng = np.random.default_rng(11)
    E = 0.05 * rng.standard_normal(nt + 1)
    E[-1] = 0.4
    m = oracle_mod.mask(N, dx, 15.0, 0.125)
    gd = np.zeros(nt + 1)
    ga = np.zeros(nt + 1)
    ga[-1] = 1.0

    def loss(Ev):
        return float(oracle_mod.propagate(psi0, Ev, dx, dt, a, mask_values=m)[2][-1])

    psi_end = oracle_mod.propagate(psi0, E, dx, dt, a, mask_values=m)[0]
    assert _norm(psi_end, dx) < 0.02
    gE = oracle_mod.adjoint(psi0, E, dx, dt, a, gd, ga, mask_values=m)
    for k in [0, 40, 100, 159, 160]:
        eps = 1e-5
        Ep, Em = E.copy(), E.copy()
        Ep[k] += eps
        Em[k] -= eps
        fd = (loss(Ep) - loss(Em)) / (2 * eps)
        assert abs(fd - gE[k]) < 1e-6 * (abs(fd) + 1e-3), (k, fd, gE[k])


# ---------------------------------------------------------------- energy distribution (Sec. 6.1)

def _dense_h0(oracle_mod, N, dx, a, scheme):
    x, V, _ = oracle_mod.grid(N, dx, a)
    lap = (np.diag(np.full(N - 1, 1.0), -1) - 2 * np.eye(N) + np.diag(np.full(N - 1, 1.0), 1)) / dx ** 2
    if scheme == FULL_CN:
        return -0.5 * lap + np.diag(V)
    M2 = np.eye(N) + dx ** 2 / 12.0 * lap
    H = np.linalg.solve(M2, -0.5 * lap) + np.diag(V)   # M2 and lap commute: symmetric
    return 0.5 * (H + H.T)


@pytest.mark.parametrize("scheme", [FULL_CN, NUMEROV])
def test_energy_distribution_equals_eigen_expansion(oracle_mod, scheme):
    """P(E) of any state equals its expansion over the eigenpairs (w_k, u_k) of the discrete H0:
    P(E) = sum_k |<u_k|psi>|^2 (eps/pi) / ((E - w_k)^2 + eps^2) (the resolvent is diagonal in the
    eigenbasis).  Brute force by dense diagonalisation against the oracle's tridiagonal solves, for
    an eigenstate (a single Lorentzian) and a random complex state."""
    rng = np.random.default_rng(23)
    N, dx, a, eps = 96, 0.25, 1.19, 0.07
    w, U = eigh(_dense_h0(oracle_mod, N, dx, a, scheme))
    u = U / np.sqrt(dx)                      # sum |u_k|^2 dx = 1
    E_grid = np.concatenate([np.linspace(-1.2, 2.0, 40), w[[0, 1, 5]], [w[0] + 0.5 * eps]])
    states = [u[:, 0].astype(np.complex128), u[:, 3].astype(np.complex128),
              rng.standard_normal(N) + 1j * rng.standard_normal(N)]
    for psi in states:
        c = (u.T @ psi) * dx                 # <u_k|psi> in the sum-dx inner product
        ref = np.array([np.sum(np.abs(c) ** 2 * (eps / np.pi) / ((E - w) ** 2 + eps ** 2)) for E in E_grid])
        P = oracle_mod.energy_distribution(psi, E_grid, dx, a, eps, scheme=scheme)
        assert np.max(np.abs(P - ref) / ref) < 1e-9
    # an eigenstate at its own energy: the peak of a unit Lorentzian, 1/(pi eps)
    P0 = oracle_mod.energy_distribution(u[:, 0], [w[0]], dx, a, eps, scheme=scheme)
    assert abs(P0[0] * np.pi * eps - 1.0) < 1e-9


def test_energy_distribution_sum_rule(oracle_mod):
    """The integral of P over energy is the norm of the state (Sec. 6.1: the integral gives the
    probability), up to the Lorentzian tails beyond a wide grid."""
    rng = np.random.default_rng(29)
    N, dx, a, eps = 80, 0.5, 1.19, 0.05
    psi = np.exp(-((np.arange(N) - 40.0) * dx) ** 2 / 8 + 0.6j * np.arange(N) * dx) * (1 + 0.2 * rng.standard_normal(N))
    norm = np.sum(np.abs(psi) ** 2) * dx
    E_grid = np.linspace(-60.0, 70.0, 26001)
    P = oracle_mod.energy_distribution(psi, E_grid, dx, a, eps)
    integral = np.sum(P) * (E_grid[1] - E_grid[0])
    assert abs(integral / norm - 1.0) < 2e-3


@pytest.mark.parametrize("scheme", [FULL_CN, NUMEROV])
def test_ionisation_equals_integrated_eigen_expansion(oracle_mod, scheme):
    """The ionisation probability (Sec. 6.1: the energy integral of P) of any state equals the
    exact integral of its eigen-expansion, a sum of Lorentzians:
        int_{E_a}^{E_b} P dE = sum_k |<u_k|psi>|^2 (atan((E_b - w_k)/eps) - atan((E_a - w_k)/eps)) / pi,
    up to the trapezoidal rule's error, bounded here by (E_b - E_a) h^2 max|P''| / 12 with
    max|P''| <= 2 ||psi||^2 / (pi eps^3).  The state is mostly the ground state (the lower node sits
    at its Lorentzian's peak, so wrong end weights would show) plus a continuum part.  The
    ground state alone gives atan(eps / |w_0|)/pi over [0, inf) -- not zero at finite eps: that is
    the Lorentzian tail of a bound state above the threshold."""
    rng = np.random.default_rng(31)
    N, dx, a, eps = 96, 0.25, 1.19, 0.07
    w, U = eigh(_dense_h0(oracle_mod, N, dx, a, scheme))
    u = U / np.sqrt(dx)
    cont = np.nonzero(w > 0.3)[0][:6]
    psi = (0.9 * u[:, 0] + (0.1 + 0.05j) * u[:, cont] @ rng.standard_normal(cont.size)).astype(np.complex128)
    norm = np.sum(np.abs(psi) ** 2) * dx
    c2 = np.abs((u.T @ psi) * dx) ** 2
    for E_a, E_b, h in ((w[0], 3.0, eps / 200), (0.0, 4.0, eps / 100)):
        nodes = np.linspace(E_a, E_b, int(round((E_b - E_a) / h)) + 1)
        hh = nodes[1] - nodes[0]
        exact = np.sum(c2 * (np.arctan((E_b - w) / eps) - np.arctan((E_a - w) / eps))) / np.pi
        bound = (E_b - E_a) * hh ** 2 / 12 * 2 * norm / (np.pi * eps ** 3)
        ion = oracle_mod.ionisation(psi, nodes, dx, a, eps, scheme=scheme)
        assert abs(ion - exact) <= bound, (E_a, ion, exact, bound)
        # the end weights matter at this resolution: a plain Riemann sum is off by far more
        P_end = oracle_mod.energy_distribution(psi, nodes[[0, -1]], dx, a, eps, scheme=scheme)
        assert 0.5 * hh * (P_end[0] + P_end[1]) > 3 * bound or E_a == 0.0
    # ground state over the continuum up to far above the spectrum's top
    nodes = np.linspace(0.0, 6.0, 12001)
    ion0 = oracle_mod.ionisation(u[:, 0].astype(np.complex128), nodes, dx, a, eps, scheme=scheme)
    ref0 = (np.arctan(eps / abs(w[0])) - np.arctan(eps / (6.0 - w[0]))) / np.pi
    assert abs(ion0 - ref0) < 1e-4 * ref0


# ---------------------------------------------------------------- far field (Sec. 3.2, Sec. 4.3)

def test_dipole_spectrum_convention_and_closed_form(oracle_mod):
    """The source transform uses the paper's convention F^(w) = (2 pi)^(-1/2) int F(t) e^{+i w t} dt.
    (i) At the DFT bins w_k = 2 pi k / (L dt) the rectangle rule is numpy's FFT with the opposite
    sign: dt / sqrt(2 pi) * conj(FFT(a))_k for real a.  (ii) A Gaussian-enveloped cosine
    exp(-(t - t0)^2 / (2 s^2)) cos(W t) has the closed-form transform
    (s/2) [exp(i (w+W) t0 - s^2 (w+W)^2 / 2) + exp(i (w-W) t0 - s^2 (w-W)^2 / 2)], which the rectangle
    rule reaches to rounding for a well-sampled pulse decaying inside the window (t0 != 0 fixes
    the sign of the exponent); a density weight scales the result."""
    rng = np.random.default_rng(41)
    L, dt = 600, 0.05
    a = rng.standard_normal(L)
    k = np.array([0, 1, 7, 123, 299])
    S = oracle_mod.dipole_spectrum(a, dt, 2 * np.pi * k / (L * dt))
    ref = dt / np.sqrt(2 * np.pi) * np.conj(np.fft.fft(a))[k]
    assert np.max(np.abs(S - ref)) < 1e-12 * np.max(np.abs(ref))
    s, W, t0, dt2 = 12.0, 1.3, 150.0, 0.02
    t = np.arange(int(300.0 / dt2) + 1) * dt2
    sig = np.exp(-((t - t0) ** 2) / (2 * s * s)) * np.cos(W * t)
    w = np.array([0.0, 0.9, 1.25, 1.3, 1.4, 2.0])
    ref = 0.5 * s * (np.exp(1j * (w + W) * t0 - s * s * (w + W) ** 2 / 2) + np.exp(1j * (w - W) * t0 - s * s * (w - W) ** 2 / 2))
    got = oracle_mod.dipole_spectrum(sig, dt2, w, weight=2.5)
    assert np.max(np.abs(got - 2.5 * ref)) < 1e-12 * s


def _gauss_hankel(k, D, w, rho):
    """int_0^inf exp(i k r^2 / (2 D)) exp(-r^2 / w^2) J0(k rho r / D) r dr = exp(-kap^2 / (4 al)) / (2 al),
    al = 1/w^2 - i k / (2 D), kap = k rho / D (the Gaussian Hankel transform with a complex width)."""
    al = 1.0 / w ** 2 - 1j * k / (2.0 * D)
    kap = k * np.asarray(rho) / D
    return np.exp(-kap ** 2 / (4.0 * al)) / (2.0 * al)


def test_hankel_thin_gaussian_source_closed_form(oracle_mod):
    """A thin Gaussian source plane (one z' node): the direct integration equals the paraxial
    propagation of a Gaussian, -(mu0/4pi) e^{ik(z - z0)} e^{i k rho^2/(2D)}/D times the Gaussian Hankel
    transform with complex width (closed form), to the trapezoid rule's h^2/12 error on a fine rho'
    grid.  Fixes the J0 argument k rho rho'/D, the sign of both Fresnel phases, the rho' weight, the
    1/D and the prefactor."""
    lam, w, z0, z_obs = 40e-9, 20e-6, 1e-3, 0.5
    k = np.array([2 * np.pi / lam, 2 * np.pi / (1.3 * lam)])
    rho_src = np.linspace(0.0, 8 * w, 1601)
    rho_obs = np.linspace(0.0, 1.2e-3, 64)
    S = (3.0 - 1.0j) * np.exp(-rho_src ** 2 / w ** 2)[:, None, None] * np.ones((1, 1, k.size))
    E = oracle_mod.hankel_far_field(S, rho_src, [z0], k, z_obs, rho_obs)
    D = z_obs - z0
    for q in range(k.size):
        ref = (-oracle_mod.MU0 / (4 * np.pi) * np.exp(1j * k[q] * (z_obs - z0)) * np.exp(1j * k[q] * rho_obs ** 2 / (2 * D))
               / D * (3.0 - 1.0j) * _gauss_hankel(k[q], D, w, rho_obs))
        assert np.max(np.abs(E[q] - ref)) < 2e-5 * np.max(np.abs(ref)), q


def test_hankel_long_phase_matched_medium_against_adaptive_quadrature(oracle_mod):
    """A long homogeneous medium driven in phase, S(rho', z') = exp(-rho'^2/w^2) exp(i k z'): the
    e^{-ikz'} of the propagator cancels the source phase and the field is the z' integral of the
    thin closed form over the medium, here by adaptive quadrature (scipy.integrate.quad).  The
    direct grid integration (trapezoid in rho' and z') must agree to its discretisation error; a
    wrong sign of the propagator phase leaves an e^{2ikz'} that the z' grid cannot resolve."""
    from scipy.integrate import quad
    lam, w, Lm, z_obs = 40e-9, 20e-6, 10e-3, 0.5
    k = 2 * np.pi / lam
    rho_src = np.linspace(0.0, 8 * w, 1601)   # rho' trapezoid: h^2/12 / (w^2/2) = 4.2e-6 of the field
    z_src = np.linspace(-Lm / 2, Lm / 2, 129)
    rho_obs = np.array([0.0, 1.5e-4, 3e-4, 6e-4])
    S = np.exp(-rho_src ** 2 / w ** 2)[:, None] * np.exp(1j * k * z_src)[None, :]
    E = oracle_mod.hankel_far_field(S[:, :, None], rho_src, z_src, [k], z_obs, rho_obs)[0]
    ref = np.zeros(rho_obs.size, dtype=np.complex128)
    for o, r in enumerate(rho_obs):
        def f(zp, part):
            D = z_obs - zp
            v = np.exp(1j * k * r * r / (2 * D)) / D * _gauss_hankel(k, D, w, r)
            return v.real if part == 0 else v.imag
        re = quad(f, -Lm / 2, Lm / 2, args=(0,), epsabs=0, epsrel=1e-12, limit=200)[0]
        im = quad(f, -Lm / 2, Lm / 2, args=(1,), epsabs=0, epsrel=1e-12, limit=200)[0]
        ref[o] = -oracle_mod.MU0 / (4 * np.pi) * np.exp(1j * k * z_obs) * (re + 1j * im)
    # the rho' trapezoid's h^2/12 term does not decay with rho, so the bound is on the field's scale
    assert np.max(np.abs(E - ref)) < 1e-5 * np.max(np.abs(ref)), (E, ref)


def test_hankel_thin_medium_is_the_limit_of_a_thin_slab(oracle_mod):
    """Three source planes 2 delta apart in total (trapezoid weights delta/2, delta, delta/2) carrying
    the same in-phase source give 2 delta times the single-plane (thin-medium) result, up to the
    O(delta / D) change of the propagator across the slab."""
    rng = np.random.default_rng(43)
    lam, z_obs, delta = 50e-9, 0.8, 1e-7
    k = np.array([2 * np.pi / lam])
    rho_src = np.linspace(0.0, 1e-4, 65)
    rho_obs = np.linspace(0.0, 2e-3, 17)
    prof = (rng.standard_normal(rho_src.size) + 1j * rng.standard_normal(rho_src.size)) * np.exp(-(rho_src / 4e-5) ** 2)
    z3 = np.array([-delta, 0.0, delta])
    S3 = prof[:, None, None] * np.exp(1j * k[0] * z3)[None, :, None]
    E3 = oracle_mod.hankel_far_field(S3, rho_src, z3, k, z_obs, rho_obs)
    E1 = oracle_mod.hankel_far_field(prof[:, None, None], rho_src, [0.0], k, z_obs, rho_obs)
    assert np.max(np.abs(E3 / (2 * delta) - E1)) < 1e-6 * np.max(np.abs(E1))


# ---------------------------------------------------------------- field ingestion (Sec. 4.2)

def test_resampling_is_exact_at_coarse_samples_and_for_band_limited_fields(oracle_mod):
    """Zero-padding the DFT is the trigonometric interpolant: it passes through every coarse sample,
    and a field made of harmonics of the window below the Nyquist frequency comes back exactly at
    every fine time (odd and even numbers of samples)."""
    rng = np.random.default_rng(31)
    for M in (64, 75):
        dtc, r = 0.4, 8
        T = M * dtc
        c = rng.standard_normal(M)
        fine = oracle_mod.resample_field(c, dtc, dtc / r, M * r)
        assert np.max(np.abs(fine[::r] - c)) < 1e-12
        tm = np.arange(M) * dtc
        f = lambda t: 0.3 + np.cos(2 * np.pi * 3 * t / T) + 0.5 * np.sin(2 * np.pi * 7 * t / T + 0.3)
        tf = np.arange(M * r) * dtc / r
        got = oracle_mod.resample_field(f(tm), dtc, dtc / r, M * r)
        assert np.max(np.abs(got - f(tf))) < 1e-12


def test_resampling_equals_zero_padded_inverse_fft(oracle_mod):
    """When the window holds a whole number L of fine steps, the interpolant equals the inverse FFT
    of the spectrum zero-padded to L bins (Nyquist bin split in two), times L / M."""
    rng = np.random.default_rng(37)
    for M, L in ((64, 512), (75, 600)):
        dtc = 0.4
        c = rng.standard_normal(M)
        Eh = np.fft.fft(c)
        pad = np.zeros(L, dtype=np.complex128)
        h = M // 2
        if M % 2 == 0:
            pad[:h] = Eh[:h]
            pad[h] = 0.5 * Eh[h]
            pad[L - h] = 0.5 * Eh[h]
            pad[L - h + 1:] = Eh[h + 1:]
        else:
            pad[:h + 1] = Eh[:h + 1]
            pad[L - h:] = Eh[h + 1:]
        ref = np.real(np.fft.ifft(pad)) * L / M
        got = oracle_mod.resample_field(c, dtc, M * dtc / L, L)
        assert np.max(np.abs(got - ref)) < 1e-12


# ---------------------------------------------------------------- populations (Sec. 7.5)

def test_populations_of_eigenstates_and_superpositions(oracle_mod):
    """The ground-state population is 1 for the ground state, 0 for an excited eigenstate, |c0|^2
    for a superposition c0 u0 + c1 u1 of orthonormal eigenstates (dense diagonalisation of the
    discrete H0); the near-core probability tends to the norm for a radius beyond the box, and for
    a Gaussian equals the discrete sum of its closed form."""
    N, dx, a = 200, 0.25, 1.19
    w, U = eigh(_dense_h0(oracle_mod, N, dx, a, FULL_CN))
    u = U / np.sqrt(dx)
    p0, _ = oracle_mod.populations(u[:, 0], u[:, 0], dx, a, 5.0)
    assert abs(p0 - 1.0) < 1e-12
    p1, _ = oracle_mod.populations(u[:, 3], u[:, 0], dx, a, 5.0)
    assert p1 < 1e-24
    c0, c1 = 0.6 * np.exp(1j * np.pi / 3), 0.8j   # complex c0: |<u0|psi>|^2, not Re(<u0|psi>)^2
    pm, core_all = oracle_mod.populations(c0 * u[:, 0] + c1 * u[:, 1], u[:, 0], dx, a, 1e9)
    assert abs(pm - 0.36) < 1e-12
    assert abs(core_all - 1.0) < 1e-12
    x, _, _ = oracle_mod.grid(N, dx, a)
    g = np.exp(-x ** 2 / 2) + 0j
    _, core = oracle_mod.populations(g, u[:, 0], dx, a, 2.0)
    assert abs(core - np.sum(np.exp(-x[np.abs(x) < 2.0] ** 2)) * dx) < 1e-13
    # the core region is open: on an odd grid x = +-2 are grid points (x_j = (j - 100) dx) and are
    # left out; a unit spike there and nowhere else has no near-core probability at r = 2
    x1, _, _ = oracle_mod.grid(201, dx, a)
    spike = np.zeros(201, dtype=complex)
    spike[[92, 108]] = 1.0
    assert x1[108] == 2.0 and x1[92] == -2.0
    assert oracle_mod.populations(spike, np.zeros(201), dx, a, 2.0)[1] == 0.0
    assert abs(oracle_mod.populations(spike, np.zeros(201), dx, a, 2.0 + 1e-12)[1] - 2 * dx) < 1e-15
