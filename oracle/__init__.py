"""FP64 CPU oracle for the batched 1D-TDSE hot path (arXiv:2507.04115, Sec. 3.1 and 4.2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA path.

Contents
  * ctypes bindings of ``tdse_oracle.c`` (grid, mask, ground state, energy, propagation);
  * ``spectrum``: |DFT(a)|^2 dt^2 with numpy's FFT as the library primitive (reading F:
    plain FFT over the Nt+1 samples, no window; the paper warns that the periodic FFT makes
    the dipole, current and acceleration forms differ, App. A, last paragraph);
  * ``lowest_eigenvalue`` / ``fit_softening``: the soft-core parameter a such that the
    ground-state energy of the discrete field-free Hamiltonian equals a target (Sec. 3.1,
    the sentence after Eq. "SC potential"), by a bracketing root finder;
  * ``propagate_many``: one oracle instance per worker process (spawned), for baselines.

``adjoint``: the exact discrete adjoint of the FULL_CN forward map (gradient of a loss of d and a
with respect to every field sample).

``energy_distribution``: the time-dependent electron energy distribution P(E) of a state through the
resolvent of the field-free Hamiltonian (Sec. 6.1).

``ionisation``: the energy integral of P(E, t) over the continuum, the time-dependent ionisation
probability (Sec. 6.1, last paragraph).

``populations``: the ground-state population and the near-core probability of a state (Sec. 7.5).

``dipole_spectrum`` and ``hankel_far_field``: the output side, the Fourier transform of a(t) in the
paper's convention and the far field of a homogeneous medium by direct grid integration of
Eq. "Hankel long homogeneous" (Sec. 3.2, Sec. 4.3).

``resample_field``: the input step of Sec. 4.2, a coarsely sampled field moved to t = 0 and
interpolated to the propagation step by zero-padding its DFT.

Scheme ids: 0 = FULL_CN (E in the diagonal at the midpoint field), 1 = NUMEROV_SPLIT
(the paper's Eqs. "CN - step 4/2/3").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

FULL_CN = 0
NUMEROV_SPLIT = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdse_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile tdse_oracle.c into oracle/_liboracle.so with gcc (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_grid.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
        L.oracle_mask.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
        L.oracle_energy.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    _dp, _dp]
        L.oracle_ground_state.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_long, ctypes.c_double,
                                          _dp, _dp, _lp]
        L.oracle_propagate.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_long, ctypes.c_long,
                                       _dp, _dp, _dp]
        L.oracle_adjoint.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     _dp, _dp, ctypes.c_long, _dp, _dp, _dp, _dp]
        L.oracle_energy_distribution.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_double, _dp]
        for f in (L.oracle_grid, L.oracle_mask, L.oracle_energy, L.oracle_ground_state, L.oracle_propagate,
                  L.oracle_adjoint, L.oracle_energy_distribution):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _check(rc, what):
    if rc != 0:
        raise ValueError("%s failed (rc=%d)" % (what, rc))


def grid(N, dx, a, Z=1.0):
    """x_j, V_j and dV/dx at x_j on the cell-centred grid (reading G)."""
    x = np.empty(N); V = np.empty(N); dV = np.empty(N)
    _check(lib().oracle_grid(N, dx, a, Z, _ptr(x), _ptr(V), _ptr(dV)), "oracle_grid")
    return x, V, dV


def mask(N, dx, width=20.0, exponent=0.125):
    """cos^p edge mask (reading D); width <= 0 returns ones."""
    m = np.empty(N)
    _check(lib().oracle_mask(N, dx, width, exponent, _ptr(m)), "oracle_mask")
    return m


def energy(psi, dx, a, Z=1.0, scheme=FULL_CN):
    """<psi|H0|psi>/<psi|psi> for the scheme's discrete field-free Hamiltonian."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    e = np.zeros(1)
    _check(lib().oracle_energy(psi.size, dx, a, Z, scheme, psi.view(np.float64).ctypes.data_as(_dp), _ptr(e)),
           "oracle_energy")
    return float(e[0])


def ground_state(N, dx, a, Z=1.0, scheme=FULL_CN, dtau=0.1, max_iter=20000, tol=1e-13):
    """Imaginary-time Crank-Nicolson ground state (reading GS). Returns (psi, E, iterations)."""
    psi = np.zeros(N, dtype=np.complex128)
    e = np.zeros(1)
    it = ctypes.c_long(0)
    _check(lib().oracle_ground_state(N, dx, a, Z, scheme, dtau, max_iter, tol,
                                     psi.view(np.float64).ctypes.data_as(_dp), _ptr(e), ctypes.byref(it)),
           "oracle_ground_state")
    return psi, float(e[0]), int(it.value)


def propagate(psi0, E, dx, dt, a, Z=1.0, scheme=FULL_CN, mask_values=None, n_begin=0, n_end=None):
    """Propagate one instance over steps [n_begin, n_end) of the sampled field E[0..Nt].

    Returns (psi, d, acc) with d, acc of length len(E): entries n_begin+1..n_end are written
    (and n_begin when n_begin == 0); others are NaN."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    Nt = E.size - 1
    if n_end is None:
        n_end = Nt
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    d = np.full(E.size, np.nan)
    acc = np.full(E.size, np.nan)
    m = None if mask_values is None else np.ascontiguousarray(mask_values, dtype=np.float64)
    _check(lib().oracle_propagate(psi.size, dx, a, Z, scheme, dt, _ptr(m), _ptr(E), n_begin, n_end,
                                  psi.view(np.float64).ctypes.data_as(_dp), _ptr(d), _ptr(acc)),
           "oracle_propagate")
    return psi, d, acc


def adjoint(psi0, E, dx, dt, a, gd, ga, Z=1.0, mask_values=None):
    """dL/dE_n for a loss with gradients gd = dL/dd_n, ga = dL/da_n through the FULL_CN forward map
    (exact discrete adjoint; see oracle_adjoint)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    gd = np.ascontiguousarray(gd, dtype=np.float64)
    ga = np.ascontiguousarray(ga, dtype=np.float64)
    if gd.size != E.size or ga.size != E.size:
        raise ValueError("gd and ga need one entry per field sample")
    gE = np.zeros(E.size)
    m = None if mask_values is None else np.ascontiguousarray(mask_values, dtype=np.float64)
    _check(lib().oracle_adjoint(psi0.size, dx, a, Z, dt, _ptr(m), _ptr(E), E.size - 1,
                                psi0.view(np.float64).ctypes.data_as(_dp), _ptr(gd), _ptr(ga), _ptr(gE)),
           "oracle_adjoint")
    return gE


def energy_distribution(psi, E_grid, dx, a, eps, Z=1.0, scheme=FULL_CN):
    """P(E_k) = N_eps eps^2 ||(E_k - H0 - i eps)^{-1} psi||^2, N_eps = 1/(pi eps), with the inversion in
    the scheme's representation of H0 (Sec. 6.1; see oracle_energy_distribution)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    Eg = np.ascontiguousarray(E_grid, dtype=np.float64)
    P = np.zeros(Eg.size)
    _check(lib().oracle_energy_distribution(psi.size, dx, a, Z, scheme, psi.view(np.float64).ctypes.data_as(_dp),
                                            _ptr(Eg), Eg.size, eps, _ptr(P)), "oracle_energy_distribution")
    return P


def ionisation(psi, E_nodes, dx, a, eps, Z=1.0, scheme=FULL_CN):
    """Time-dependent ionisation probability of a state (Sec. 6.1, last paragraph: the integral of
    P(E, t) over energy).  Reading: the integral runs over the continuum, E >= 0 (the soft-core
    potential vanishes at infinity, so the bound states lie below 0), and is taken by the
    trapezoidal rule on the caller's ascending nodes E_nodes (at least two; the first one is the
    threshold, the last one an energy beyond which P is negligible):
        Ion = sum_k w_k P(E_k),  w_0 = (E_1 - E_0)/2,  w_k = (E_{k+1} - E_{k-1})/2,  w_last = (E_last - E_{last-1})/2,
    with P from ``energy_distribution`` at resolution eps."""
    E = np.asarray(E_nodes, dtype=np.float64)
    if E.size < 2 or np.any(np.diff(E) <= 0):
        raise ValueError("need at least two strictly ascending energy nodes")
    P = energy_distribution(psi, E, dx, a, eps, Z, scheme)
    w = np.empty(E.size)
    w[0] = 0.5 * (E[1] - E[0])
    w[-1] = 0.5 * (E[-1] - E[-2])
    w[1:-1] = 0.5 * (E[2:] - E[:-2])
    return float(np.sum(w * P))


def populations(psi, psi0, dx, a, r_core, Z=1.0):
    """Sec. 7.5's populations of a state psi: the ground-state population |<psi0|psi>|^2 with
    <u|v> = sum_j conj(u_j) v_j dx (psi0 the normalised field-free ground state), and the
    probability of finding the electron within |x| < r_core of the nucleus, sum_{|x_j|<r_core} |psi_j|^2 dx."""
    psi = np.asarray(psi, dtype=np.complex128)
    psi0 = np.asarray(psi0, dtype=np.complex128)
    x, _, _ = grid(psi.size, dx, a, Z)
    ov = np.sum(np.conj(psi0) * psi) * dx
    core = np.sum(np.abs(psi[np.abs(x) < r_core]) ** 2) * dx
    return float(np.abs(ov) ** 2), float(core)


def resample_field(coarse, dt_coarse, dt_fine, n_fine):
    """Field ingestion (Sec. 4.2): the coarse samples E(t_min + m dt_coarse), m = 0..M-1, moved to the
    time origin t = 0 and interpolated to t_n = n dt_fine, n = 0..n_fine-1, by zero-padding the DFT:
        E(t) = (1/M) sum_{k=-floor(M/2)}^{floor(M/2)} w_k Ehat_k exp(2 pi i k t / T),  T = M dt_coarse,
    Ehat = DFT of the samples (numpy's FFT as the library primitive), w_k = 1/2 for |k| = M/2 (even M,
    the Nyquist bin split between the two ends of the padded spectrum), otherwise 1."""
    c = np.asarray(coarse, dtype=np.float64)
    M = c.size
    Eh = np.fft.fft(c)
    k = np.arange(-(M // 2), M // 2 + 1)
    w = np.ones(k.size)
    if M % 2 == 0:
        w[0] = w[-1] = 0.5
    coef = w * Eh[k % M] / M
    t = np.arange(n_fine) * dt_fine
    T = M * dt_coarse
    out = np.empty(n_fine)
    for s0 in range(0, n_fine, 4096):   # bounded memory for the explicit sum
        tt = t[s0:s0 + 4096]
        out[s0:s0 + 4096] = np.real(np.exp(2j * np.pi * np.outer(tt, k) / T) @ coef)
    return out


# ------------------------------------------------------------------ far field (Sec. 3.2, Sec. 4.3)

MU0 = 1.25663706212e-6   # vacuum permeability (H/m, CODATA 2018)


def dipole_spectrum(acc, dt, omegas, weight=1.0):
    """Source term of the far-field integral (Sec. 3.2): the temporal Fourier transform of the dipole
    acceleration in the paper's convention (Sec. 2: F^(omega) = (2 pi)^(-1/2) int F(t) exp(i omega t) dt),
    by the rectangle rule over the samples t_n = n dt, times a weight (the gas density at the
    instance's point, since the macroscopic source is the density times the microscopic one):
        weight * dt / sqrt(2 pi) * sum_n a_n exp(i omega t_n)   for every omega in ``omegas``."""
    a = np.asarray(acc, dtype=np.float64)
    om = np.atleast_1d(np.asarray(omegas, dtype=np.float64))
    t = np.arange(a.size) * dt
    out = np.zeros(om.size, dtype=np.complex128)
    for s0 in range(0, a.size, 8192):   # bounded memory for the explicit sum
        out += np.exp(1j * np.outer(om, t[s0:s0 + 8192])) @ a[s0:s0 + 8192]
    return weight * dt / np.sqrt(2.0 * np.pi) * out


def trapezoid_weights(x):
    """Weights of the trapezoidal rule on the ascending nodes x (one node: weight 1)."""
    x = np.asarray(x, dtype=np.float64)
    if x.size == 1:
        return np.ones(1)
    w = np.empty(x.size)
    w[0] = 0.5 * (x[1] - x[0])
    w[-1] = 0.5 * (x[-1] - x[-2])
    w[1:-1] = 0.5 * (x[2:] - x[:-2])
    return w


def hankel_far_field(S, rho_src, z_src, k, z_obs, rho_obs):
    """Far field of a homogeneous generating medium, Eq. "Hankel long homogeneous" (Sec. 3.2), by
    direct grid integration over the source points (Sec. 4.3):
        E(rho, z, w) = -(mu0/(4 pi)) exp(i k z) sum_i wz_i exp(-i k z'_i) exp(i k rho^2 / (2 D_i)) / D_i
                       * sum_j wr_j rho'_j exp(i k rho'_j^2 / (2 D_i)) S[j, i, w] J0(k rho rho'_j / D_i),
    D_i = z - z'_i, k = k(omega_w).  Readings: the integrals are the trapezoidal rule on the source
    nodes (wr, wz: trapezoid weights of rho' and z'); a single z' plane is the thin medium (weight 1,
    the source then being the plane's source integrated over its thickness).  S[j, i, w] is the
    macroscopic source (density times the microscopic dJ/dt transform) at (rho'_j, z'_i, omega_w);
    SI units (lengths in m, k in 1/m).  Returns E[w, o] at the radii rho_obs[o] of the plane z = z_obs.
    J0 is scipy.special.j0 (library primitive)."""
    from scipy.special import j0
    S = np.asarray(S, dtype=np.complex128)
    rho = np.asarray(rho_src, dtype=np.float64)
    z = np.asarray(z_src, dtype=np.float64)
    kk = np.atleast_1d(np.asarray(k, dtype=np.float64))
    ro = np.atleast_1d(np.asarray(rho_obs, dtype=np.float64))
    if S.shape != (rho.size, z.size, kk.size):
        raise ValueError("S must be (n_rho, n_z, n_omega)")
    if np.any(z >= z_obs):
        raise ValueError("the observation plane must lie beyond every source plane")
    wr = trapezoid_weights(rho)
    wz = trapezoid_weights(z)
    E = np.zeros((kk.size, ro.size), dtype=np.complex128)
    for w in range(kk.size):
        kw = kk[w]
        acc = np.zeros(ro.size, dtype=np.complex128)
        for i in range(z.size):
            D = z_obs - z[i]
            src = wr * rho * np.exp(1j * kw * rho ** 2 / (2.0 * D)) * S[:, i, w]
            inner = j0(kw * np.outer(ro, rho) / D) @ src
            acc += wz[i] * np.exp(-1j * kw * z[i]) * np.exp(1j * kw * ro ** 2 / (2.0 * D)) / D * inner
        E[w] = -MU0 / (4.0 * np.pi) * np.exp(1j * kw * z_obs) * acc
    return E


def spectrum(acc, dt):
    """S_k = |sum_n a_n exp(-2 pi i k n / L)|^2 dt^2, L = number of samples (reading F)."""
    acc = np.asarray(acc, dtype=np.float64)
    return np.abs(np.fft.fft(acc)) ** 2 * dt * dt


# ------------------------------------------------------------------ soft-core parameter (Sec. 3.1)

def _numerov_solve_shifted(N, dx, V, sigma, rhs):
    """Solve (M2^{-1}(-Delta2/2) + V - sigma) y = rhs  <=>  (-Delta2/2 + M2 V - sigma M2) y = M2 rhs."""
    from scipy.linalg import solve_banded
    inv = 1.0 / (dx * dx)
    diag = inv + (10.0 / 12.0) * (V - sigma)
    sup = -0.5 * inv + (V[1:] - sigma) / 12.0      # row j, column j+1 carries V_{j+1}
    sub = -0.5 * inv + (V[:-1] - sigma) / 12.0     # row j+1, column j carries V_j
    ab = np.zeros((3, N))
    ab[0, 1:] = sup
    ab[1, :] = diag
    ab[2, :-1] = sub
    m2rhs = (10.0 / 12.0) * rhs
    m2rhs[1:] += rhs[:-1] / 12.0
    m2rhs[:-1] += rhs[1:] / 12.0
    return solve_banded((1, 1), ab, m2rhs)


def lowest_eigenvalue(N, dx, a, Z=1.0, scheme=FULL_CN):
    """Lowest eigenvalue of the scheme's discrete field-free Hamiltonian.

    FULL_CN: symmetric tridiagonal eigensolver.  NUMEROV_SPLIT: shifted inverse iteration on
    M2^{-1}(-Delta2/2) + V, started at the three-point value, with Rayleigh quotients."""
    from scipy.linalg import eigh_tridiagonal
    x, V, _ = grid(N, dx, a, Z)
    inv = 1.0 / (dx * dx)
    w = eigh_tridiagonal(inv + V, np.full(N - 1, -0.5 * inv), select="i", select_range=(0, 0),
                         eigvals_only=True)
    e_fd = float(w[0])
    if scheme == FULL_CN:
        return e_fd
    sigma = e_fd - 1e-3
    y = np.exp(-x * x)
    e = e_fd
    for _ in range(200):
        y = _numerov_solve_shifted(N, dx, V, sigma, y)
        y /= np.linalg.norm(y)
        e_new = energy(y.astype(np.complex128), dx, a, Z, NUMEROV_SPLIT)
        if abs(e_new - e) < 1e-15:
            e = e_new
            break
        e = e_new
    return e


def fit_softening(target, N, dx, Z=1.0, scheme=FULL_CN, lo=0.2, hi=6.0):
    """Soft-core a such that the discrete ground-state energy equals ``target``."""
    from scipy.optimize import brentq
    return brentq(lambda a: lowest_eigenvalue(N, dx, a, Z, scheme) - target, lo, hi, xtol=1e-14, rtol=1e-15,
                  maxiter=200)


# ------------------------------------------------------------------ many instances, one per process

def _propagate_job(args):
    (psi0, E, dx, dt, a, Z, scheme, mask_values) = args
    _, d, acc = propagate(psi0, E, dx, dt, a, Z, scheme, mask_values)
    return d, acc


def propagate_many(jobs, workers):
    """Run ``propagate`` for each job tuple (psi0, E, dx, dt, a, Z, scheme, mask) in a spawned pool."""
    import multiprocessing as mp
    build()
    if workers <= 1 or len(jobs) <= 1:
        return [_propagate_job(j) for j in jobs]
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=workers) as pool:
        return pool.map(_propagate_job, jobs, chunksize=1)
