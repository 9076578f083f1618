"""The oracle's pins catch plausible mistakes (no GPU).

Each mutant is a copy of ``oracle/`` with one planted mistake: a dropped term, a wrong sign, a
wrong index or time level, a transposed operand, a missing factor.  The pins and the independent
cross-check (test_oracle_pins.py, test_oracle_crosscheck.py) run against every copy in a
subprocess and must fail on each one; against an unmodified copy they must pass.  This keeps the
claim that the pins fix the oracle reproducible as the oracle and its pins change.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C_SRC = "tdse_oracle.c"
PY_SRC = "__init__.py"

# (file in oracle/, text, replacement, what the mistake is)
MUTANTS = [
    (C_SRC, "Kdi[j] = inv_dx2 + V[j];", "Kdi[j] = inv_dx2;", "FULL_CN: potential dropped from H0"),
    (C_SRC, "Klo[j] = -0.5 * inv_dx2;", "Klo[j] = 0.5 * inv_dx2;", "FULL_CN: sign of the kinetic sub-diagonal"),
    (C_SRC, "Kdi[j] = inv_dx2 + (10.0 / 12.0) * V[j];", "Kdi[j] = inv_dx2 + V[j];",
     "NUMEROV: M2 V diagonal weight"),
    (C_SRC, "(j > 0 ? V[j - 1] / 12.0 : 0.0)", "(j > 0 ? V[j] / 12.0 : 0.0)", "NUMEROV: index of V in M2 V"),
    (C_SRC, "Mdi[j] = 10.0 / 12.0;\n", "Mdi[j] = 1.0;\n", "NUMEROV: M2 diagonal"),
    (C_SRC, "double Ebar = 0.5 * (E[n] + E[n + 1]);", "double Ebar = E[n];", "FULL_CN: field time level"),
    (C_SRC, "double kd = K[1][j] + x[j] * Ebar;   /* diagonal", "double kd = K[1][j] - x[j] * Ebar;   /* diagonal",
     "FULL_CN: sign of the field term"),
    (C_SRC, "cexp(-I * dt * E[n] * x[j])", "cexp(I * dt * E[n] * x[j])", "NUMEROV: sign of the field phase"),
    (C_SRC, "cexp(-I * dt * E[n] * x[j])", "cexp(-I * dt * E[n + 1] * x[j])", "NUMEROV: time level of the phase"),
    (C_SRC, "double complex piv = di[j] - lo[j] * cp[j - 1];", "double complex piv = di[j] - up[j] * cp[j - 1];",
     "Thomas: transposed operand in the pivot"),
    (C_SRC, "for (int j = N - 2; j >= 0; --j) y[j] = dp[j] - cp[j] * y[j + 1];",
     "for (int j = N - 2; j >= 0; --j) y[j] = dp[j] + cp[j] * y[j + 1];", "Thomas: sign of the back substitution"),
    (C_SRC, "*a = (sa + E * sn) * dx;", "*a = (sa - E * sn) * dx;", "observables: sign of E in a(t)"),
    (C_SRC, "*a = (sa + E * sn) * dx;", "*a = sa * dx;", "observables: E term dropped from a(t)"),
    (C_SRC, "*d = sd * dx;", "*d = sd;", "observables: dx missing in d(t)"),
    (C_SRC, "if (dV) dV[j] = Z * xj / (r2 * sqrt(r2));", "if (dV) dV[j] = -Z * xj / (r2 * sqrt(r2));",
     "grid: sign of dV/dx"),
    (C_SRC, "double xj = (j - 0.5 * (N - 1)) * dx;\n        double r2", "double xj = (j - 0.5 * N) * dx;\n        double r2",
     "grid: off-centre x_j"),
    (C_SRC, "for (int j = 0; j < N; ++j) psi[j] *= mask[j];", "for (int j = 0; j < N; ++j) psi[j] *= mask[j] * mask[j];",
     "absorber applied twice"),
    (C_SRC, "double c = cos(0.5 * 3.14159265358979323846 * (ax - xb) / width);",
     "double c = cos(0.5 * 3.14159265358979323846 * (ax - xb) / (2.0 * width));", "mask: width of the ramp"),
    (C_SRC, "lo[j] = M[0][j] + c * K[0][j];  di[j] = M[1][j] + c * K[1][j];  up[j] = M[2][j] + c * K[2][j];\n"
            "        blo[j] = M[0][j] - c * K[0][j]; bdi[j] = M[1][j] - c * K[1][j]; bup[j] = M[2][j] - c * K[2][j];\n"
            "    }\n    for (int j = 0; j < N; ++j) psi[j] = exp",
     "lo[j] = M[0][j] + c * K[0][j];  di[j] = M[1][j] + c * K[1][j];  up[j] = M[2][j] + c * K[2][j];\n"
     "        blo[j] = M[0][j] - c * K[0][j]; bdi[j] = M[1][j] - c * K[1][j]; bup[j] = M[2][j] + c * K[2][j];\n"
     "    }\n    for (int j = 0; j < N; ++j) psi[j] = exp", "ground state: sign in the explicit half-step"),
    (C_SRC, "gE[n] += 0.5 * gbar;", "gE[n] += gbar;", "adjoint: midpoint split of the field gradient"),
    (C_SRC, "lam[j] = 2.0 * dx * (gd[Nt] * x[j] + ga[Nt] * (dV[j] + E[Nt])) * p[j];",
     "lam[j] = 2.0 * dx * (gd[Nt] * x[j] + ga[Nt] * dV[j]) * p[j];", "adjoint: field dropped from the terminal source"),
    (C_SRC, "if (creal(psi[N / 2]) < 0.0)", "if (creal(psi[N / 2]) > 0.0)", "ground state: sign convention"),
    (C_SRC, "tri_solve(N, blo, bdi, bup, r, mu, work);", "tri_solve(N, lo, di, up, r, mu, work);",
     "adjoint: A_n instead of its adjoint B_n"),
    (C_SRC, "const double norm = 1.0 / (3.14159265358979323846 * eps);", "const double norm = 1.0 / eps;",
     "energy distribution: N_eps"),
    (C_SRC, "tri_apply(N, mlo, mdi, mup, psi, r);                         /* M psi */",
     "memcpy(r, psi, sizeof(double complex) * N);", "energy distribution: M dropped from the right-hand side"),
    (C_SRC, "lo[j] = z * M[0][j] - K[0][j];", "lo[j] = z * M[0][j] + K[0][j];",
     "energy distribution: sign of K's sub-diagonal"),
    (C_SRC, "if (j > 0) s += lo[j] * v[j - 1];", "if (j > 0) s += up[j] * v[j - 1];",
     "tridiagonal product: transposed operand"),
    (C_SRC, "m[j] = (c > 0.0) ? pow(c, exponent) : 0.0;", "m[j] = (c > 0.0) ? c : 0.0;", "mask: exponent ignored"),
    (C_SRC, "double xb = 0.5 * N * dx - width;", "double xb = 0.5 * (N - 1) * dx - width;",
     "mask: plateau edge off by half a cell"),
    (C_SRC, "tri_solve(N, lo, di, up, t1, t2, work);", "memcpy(t2, t1, sizeof(double complex) * N);",
     "NUMEROV energy: M2^-1 dropped"),
    (C_SRC, "sn += rho;", "sn += 1.0;", "observables: norm sum"),
    (C_SRC, "const double complex c = I * 0.5 * dt;", "const double complex c = I * dt;", "propagation: h = dt"),
    (C_SRC, "nrm = sqrt(nrm * dx);", "nrm = sqrt(nrm);", "ground state: normalisation without dx"),
    (C_SRC, "gE[Nt] += ga[Nt] * dx * nrm;", "gE[Nt] += 0.0 * nrm;", "adjoint: terminal direct field term"),
    (C_SRC, "num += conj(psi[j]) * (t2[j] + V[j] * psi[j]);", "num += conj(psi[j]) * t2[j];",
     "energy: potential dropped"),
    (C_SRC, "lo[j] = -0.5 * inv_dx2; di[j] = inv_dx2; up[j] = -0.5 * inv_dx2; }",
     "lo[j] = -0.5 * inv_dx2; di[j] = 2.0 * inv_dx2; up[j] = -0.5 * inv_dx2; }", "energy: kinetic diagonal"),
    (C_SRC, "if (d && acc) observables(N, dx, x, dV, E[n + 1], psi, &d[n + 1], &acc[n + 1]);",
     "if (d && acc) observables(N, dx, x, dV, E[n], psi, &d[n + 1], &acc[n + 1]);", "observables: field time level"),
    (C_SRC, "gbar += x[j] * cimag(conj(mu[j]) * (p[j] + q[j]));", "gbar += x[j] * cimag(conj(mu[j]) * (p[j] - q[j]));",
     "adjoint: sign of the new state in the field gradient"),
    (C_SRC, "for (int j = 0; j < N; ++j) r[j] = (mask ? mask[j] : 1.0) * lam[j];",
     "for (int j = 0; j < N; ++j) r[j] = lam[j];", "adjoint: mask dropped from the backward step"),
    (PY_SRC, "diag = inv + (10.0 / 12.0) * (V - sigma)", "diag = inv + (V - sigma)",
     "Numerov eigenvalue: M2 weight of the diagonal"),
    (PY_SRC, "lowest_eigenvalue(N, dx, a, Z, scheme) - target", "lowest_eigenvalue(N, dx, a, Z, scheme) + target",
     "soft-core fit: sign of the target"),
    (PY_SRC, "w = eigh_tridiagonal(inv + V,", "w = eigh_tridiagonal(inv + 0.5 * V,", "FD eigenvalue: potential weight"),
    (PY_SRC, "return np.abs(np.fft.fft(acc)) ** 2 * dt * dt", "return np.abs(np.fft.fft(acc)) ** 2 * dt",
     "spectrum: dt^2"),
    (PY_SRC, "return np.abs(np.fft.fft(acc)) ** 2 * dt * dt", "return np.abs(np.fft.ifft(acc)) ** 2 * dt * dt",
     "spectrum: inverse transform"),
    (PY_SRC, "coef = w * Eh[k % M] / M", "coef = w * Eh[k % M]", "field ingestion: 1/M"),
    (PY_SRC, "t = np.arange(n_fine) * dt_fine", "t = np.arange(1, n_fine + 1) * dt_fine",
     "field ingestion: time origin"),
    (PY_SRC, "        w[0] = w[-1] = 0.5\n", "        pass\n", "field ingestion: Nyquist bin not split"),
    (PY_SRC, "ov = np.sum(np.conj(psi0) * psi) * dx", "ov = np.sum(np.conj(psi0) * psi)", "populations: dx missing"),
    (PY_SRC, "psi[np.abs(x) < r_core]", "psi[np.abs(x) <= r_core]", "populations: closed core interval"),
    (PY_SRC, "return float(np.abs(ov) ** 2), float(core)", "return float(np.real(ov) ** 2), float(core)",
     "populations: real part for the modulus"),
    (PY_SRC, "w[0] = 0.5 * (E[1] - E[0])", "w[0] = E[1] - E[0]", "ionisation: first trapezoid weight"),
    (PY_SRC, "out += np.exp(1j * np.outer(om, t[s0:s0 + 8192]))", "out += np.exp(-1j * np.outer(om, t[s0:s0 + 8192]))",
     "dipole spectrum: sign of the Fourier exponent"),
    (PY_SRC, "return weight * dt / np.sqrt(2.0 * np.pi) * out", "return weight * dt * out",
     "dipole spectrum: 1/sqrt(2 pi) of the convention"),
    (PY_SRC, "inner = j0(kw * np.outer(ro, rho) / D) @ src", "inner = j0(kw * np.outer(ro, rho) / z_obs) @ src",
     "Hankel: J0 argument over z instead of z - z'"),
    (PY_SRC, "src = wr * rho * np.exp(1j * kw * rho ** 2 / (2.0 * D)) * S[:, i, w]",
     "src = wr * rho * np.exp(-1j * kw * rho ** 2 / (2.0 * D)) * S[:, i, w]", "Hankel: sign of the source Fresnel phase"),
    (PY_SRC, "src = wr * rho * np.exp(1j * kw * rho ** 2 / (2.0 * D)) * S[:, i, w]",
     "src = wr * np.exp(1j * kw * rho ** 2 / (2.0 * D)) * S[:, i, w]", "Hankel: rho' of the area element dropped"),
    (PY_SRC, "acc += wz[i] * np.exp(-1j * kw * z[i])", "acc += wz[i] * np.exp(1j * kw * z[i])",
     "Hankel: sign of the propagator phase"),
    (PY_SRC, "np.exp(1j * kw * ro ** 2 / (2.0 * D)) / D * inner", "np.exp(1j * kw * ro ** 2 / (2.0 * D)) * inner",
     "Hankel: 1/(z - z') dropped"),
    (PY_SRC, "    wz = trapezoid_weights(z)\n", "    wz = np.ones(z.size)\n", "Hankel: z' weights"),
    (PY_SRC, "w[1:-1] = 0.5 * (E[2:] - E[:-2])", "w[1:-1] = 0.5 * (E[2:] - E[1:-1])",
     "ionisation: interior weights from one neighbour"),
]

PIN_FILES = ["conftest.py", "test_oracle_pins.py", "test_oracle_crosscheck.py"]


def _make_copy(dest, mutant):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dest, "oracle"),
                    ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    os.makedirs(os.path.join(dest, "tests"))
    for f in PIN_FILES:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dest, "tests", f))
    # the seeded input generators some pins draw their workloads from (no method arithmetic)
    pkg = "paper_2507_04115_gb300"
    os.makedirs(os.path.join(dest, pkg))
    for f in ("__init__.py", "inputs.py"):
        shutil.copy(os.path.join(ROOT, pkg, f), os.path.join(dest, pkg, f))
    if mutant is not None:
        fname, old, new, _ = mutant
        path = os.path.join(dest, "oracle", fname)
        src = open(path).read()
        assert old in src, "mutation target not found: %r" % old
        with open(path, "w") as fh:
            fh.write(src.replace(old, new, 1))


def _run_pins(dest):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
           os.path.join(dest, "tests", "test_oracle_pins.py"), os.path.join(dest, "tests", "test_oracle_crosscheck.py")]
    r = subprocess.run(cmd, cwd=dest, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


def test_pins_pass_on_the_oracle_and_fail_on_every_mutant(tmp_path):
    for fname, old, _, _ in MUTANTS:
        assert old in open(os.path.join(ROOT, "oracle", fname)).read(), old
    jobs = [(None, tmp_path / "control")] + [(m, tmp_path / ("m%02d" % i)) for i, m in enumerate(MUTANTS)]
    for mutant, dest in jobs:
        _make_copy(str(dest), mutant)
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda j: _run_pins(str(j[1])), jobs))
    rc0, out0 = results[0]
    assert rc0 == 0, "pins fail on the unmodified oracle:\n" + out0
    missed = []
    for (mutant, _), (rc, out) in zip(jobs[1:], results[1:]):
        # 1 = some test failed; anything else (collection error, crash) is not a caught mistake
        if rc != 1:
            missed.append("%s (exit %d)\n%s" % (mutant[3], rc, out[-600:]))
    assert not missed, "mutants the pins did not catch:\n" + "\n".join(missed)
