/*
 * tdse_oracle.c -- plain, slow, FP64 CPU reference of the batched 1D-TDSE hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's library.  It shares no code with the CUDA
 * path: no headers, tables, helpers or generated constants.
 *
 * Every routine follows the paper's statement of the problem (arXiv:2507.04115):
 *   - Hamiltonian H(t) = p^2/2 + V_C + x E(t), length gauge         (Sec. 3.1, Eq. "Hamiltonian (a)")
 *   - soft-core potential V_C = -Z / sqrt(x^2 + a^2), Z = 1           (Sec. 3.1, Eq. "SC potential")
 *   - space/time grids, field time origin at t = 0                    (Sec. 4.2)
 *   - the paper's three-substep Numerov Crank-Nicolson scheme          (Sec. 4.2, Eqs. "CN - step 4/2/3")
 *   - dipole <x> and dipole acceleration <dV/dx + E>                  (Sec. 3.1 Eq. "dipole acceleration";
 *                                                                       App. A Eq. "Current_der_TDSE1D")
 * and, where the paper is silent, the readings listed in the design notes:
 *   - FULL_CN: Crank-Nicolson with E in the diagonal at the midpoint field (E_n + E_{n+1})/2;
 *   - cell-centred grid x_j = (j - (N-1)/2) dx, Dirichlet walls psi_{-1} = psi_N = 0;
 *   - cos^p edge mask applied after every full step;
 *   - ground state by imaginary-time Crank-Nicolson with per-iteration renormalisation;
 *   - rectangle-rule quadrature, sum |psi|^2 dx = 1.
 *
 * Linear algebra is written out: a three-point stencil for every tridiagonal product and
 * the textbook Thomas algorithm (forward elimination, back substitution) for every solve.
 * No blocking, fusion or reordering beyond those definitions.
 *
 * Complex vectors cross the C boundary as interleaved doubles (re, im), which is the
 * memory layout of C99 "double complex".
 *
 * Return codes: 0 = ok, -1 = bad argument, -2 = out of memory.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_FULL_CN 0
#define ORACLE_NUMEROV_SPLIT 1

/* ---------------------------------------------------------------- grid and potential (Sec. 3.1, 4.2) */

/* x_j = (j - (N-1)/2) dx; V_j = -Z/sqrt(x_j^2 + a^2); dV_j = dV/dx at x_j = Z x_j/(x_j^2 + a^2)^{3/2}. */
int oracle_grid(int N, double dx, double a, double Z, double* x, double* V, double* dV)
{
    if (N < 3 || !(dx > 0.0) || !(a > 0.0)) return -1;
    for (int j = 0; j < N; ++j) {
        double xj = (j - 0.5 * (N - 1)) * dx;
        double r2 = xj * xj + a * a;
        if (x) x[j] = xj;
        if (V) V[j] = -Z / sqrt(r2);
        if (dV) dV[j] = Z * xj / (r2 * sqrt(r2));
    }
    return 0;
}

/* Edge mask: m_j = cos(pi/2 * (|x_j| - x_b)/w)^p for |x_j| > x_b = N dx/2 - w, else 1.
 * width <= 0 gives m = 1 everywhere (mask off). */
int oracle_mask(int N, double dx, double width, double exponent, double* m)
{
    if (N < 1 || !(dx > 0.0) || !m) return -1;
    double xb = 0.5 * N * dx - width;
    for (int j = 0; j < N; ++j) {
        double xj = (j - 0.5 * (N - 1)) * dx;
        double ax = fabs(xj);
        if (width > 0.0 && ax > xb) {
            double c = cos(0.5 * 3.14159265358979323846 * (ax - xb) / width);
            m[j] = (c > 0.0) ? pow(c, exponent) : 0.0;
        } else {
            m[j] = 1.0;
        }
    }
    return 0;
}

/* ---------------------------------------------------------------- tridiagonal helpers */

/* y = T v for the tridiagonal T with sub-diagonal lo[j] (= T_{j,j-1}), diagonal di[j] and
 * super-diagonal up[j] (= T_{j,j+1}); entries outside the matrix are ignored (Dirichlet). */
static void tri_apply(int N, const double complex* lo, const double complex* di, const double complex* up,
                      const double complex* v, double complex* y)
{
    for (int j = 0; j < N; ++j) {
        double complex s = di[j] * v[j];
        if (j > 0) s += lo[j] * v[j - 1];
        if (j < N - 1) s += up[j] * v[j + 1];
        y[j] = s;
    }
}

/* Thomas algorithm: solve T y = r (same storage as tri_apply).  work needs 2N entries. */
static void tri_solve(int N, const double complex* lo, const double complex* di, const double complex* up,
                      const double complex* r, double complex* y, double complex* work)
{
    double complex* cp = work;      /* modified super-diagonal */
    double complex* dp = work + N;  /* modified right-hand side */
    cp[0] = up[0] / di[0];
    dp[0] = r[0] / di[0];
    for (int j = 1; j < N; ++j) {
        double complex piv = di[j] - lo[j] * cp[j - 1];
        cp[j] = (j < N - 1) ? up[j] / piv : 0.0;
        dp[j] = (r[j] - lo[j] * dp[j - 1]) / piv;
    }
    y[N - 1] = dp[N - 1];
    for (int j = N - 2; j >= 0; --j) y[j] = dp[j] - cp[j] * y[j + 1];
}

/* ---------------------------------------------------------------- observables (Sec. 3.1, App. A) */

/* d = sum_j x_j |psi_j|^2 dx  (position expectation; the paper's dipole is q<x> with q = -1)
 * a = sum_j (dV_j + E) |psi_j|^2 dx  (Eq. "Current_der_TDSE1D", rectangle rule) */
static void observables(int N, double dx, const double* x, const double* dV, double E,
                        const double complex* psi, double* d, double* a)
{
    double sd = 0.0, sa = 0.0, sn = 0.0;
    for (int j = 0; j < N; ++j) {
        double rho = creal(psi[j]) * creal(psi[j]) + cimag(psi[j]) * cimag(psi[j]);
        sd += x[j] * rho;
        sa += dV[j] * rho;
        sn += rho;
    }
    *d = sd * dx;
    *a = (sa + E * sn) * dx;
}

/* ---------------------------------------------------------------- operator assembly */

/* Coefficients of the field-free operator used by each scheme, as a tridiagonal "K" and the
 * tridiagonal "M" it is paired with, so that both schemes read
 *      (M + c K) psi_new = (M - c K) psi_old,
 * with c = i dt/2 in real time and c = dtau/2 in imaginary time.
 *   FULL_CN  : M = 1,  K = H0 = -Delta2/2 + V           (three-point Laplacian)
 *   NUMEROV  : M = M2 = tridiag(1/12, 10/12, 1/12),  K = -Delta2/2 + M2 V   (Sec. 4.2, Eqs. step 4/2)
 * Delta2 = tridiag(1, -2, 1)/dx^2.  (M2 V)_{j,k} = (M2)_{j,k} V_k. */
static void assemble(int N, double dx, const double* V, int scheme,
                     double* Klo, double* Kdi, double* Kup, double* Mlo, double* Mdi, double* Mup)
{
    double inv_dx2 = 1.0 / (dx * dx);
    for (int j = 0; j < N; ++j) {
        if (scheme == ORACLE_NUMEROV_SPLIT) {
            Mlo[j] = 1.0 / 12.0;
            Mdi[j] = 10.0 / 12.0;
            Mup[j] = 1.0 / 12.0;
            Kdi[j] = inv_dx2 + (10.0 / 12.0) * V[j];
            Klo[j] = -0.5 * inv_dx2 + (j > 0 ? V[j - 1] / 12.0 : 0.0);
            Kup[j] = -0.5 * inv_dx2 + (j < N - 1 ? V[j + 1] / 12.0 : 0.0);
        } else {
            Mlo[j] = 0.0;
            Mdi[j] = 1.0;
            Mup[j] = 0.0;
            Kdi[j] = inv_dx2 + V[j];
            Klo[j] = -0.5 * inv_dx2;
            Kup[j] = -0.5 * inv_dx2;
        }
    }
}

/* ---------------------------------------------------------------- energy of the field-free Hamiltonian */

/* <psi|H0|psi> dx / (<psi|psi> dx) for the scheme's H0:
 *   FULL_CN : H0 = -Delta2/2 + V
 *   NUMEROV : H0 = M2^{-1}(-Delta2/2) + V   (the Hamiltonian the Numerov pencil represents) */
int oracle_energy(int N, double dx, double a, double Z, int scheme, const double* psi_ri, double* energy)
{
    if (N < 3 || !(dx > 0.0) || !psi_ri || !energy) return -1;
    const double complex* psi = (const double complex*)psi_ri;
    double* x = malloc(sizeof(double) * N);
    double* V = malloc(sizeof(double) * N);
    double complex* t1 = malloc(sizeof(double complex) * N);
    double complex* t2 = malloc(sizeof(double complex) * N);
    double complex* lo = malloc(sizeof(double complex) * N);
    double complex* di = malloc(sizeof(double complex) * N);
    double complex* up = malloc(sizeof(double complex) * N);
    double complex* work = malloc(sizeof(double complex) * 2 * N);
    if (!x || !V || !t1 || !t2 || !lo || !di || !up || !work) {
        free(x); free(V); free(t1); free(t2); free(lo); free(di); free(up); free(work);
        return -2;
    }
    oracle_grid(N, dx, a, Z, x, V, NULL);
    double inv_dx2 = 1.0 / (dx * dx);
    /* t1 = (-Delta2/2) psi */
    for (int j = 0; j < N; ++j) { lo[j] = -0.5 * inv_dx2; di[j] = inv_dx2; up[j] = -0.5 * inv_dx2; }
    tri_apply(N, lo, di, up, psi, t1);
    if (scheme == ORACLE_NUMEROV_SPLIT) {
        for (int j = 0; j < N; ++j) { lo[j] = 1.0 / 12.0; di[j] = 10.0 / 12.0; up[j] = 1.0 / 12.0; }
        tri_solve(N, lo, di, up, t1, t2, work);
    } else {
        memcpy(t2, t1, sizeof(double complex) * N);
    }
    double complex num = 0.0;
    double den = 0.0;
    for (int j = 0; j < N; ++j) {
        num += conj(psi[j]) * (t2[j] + V[j] * psi[j]);
        den += creal(psi[j]) * creal(psi[j]) + cimag(psi[j]) * cimag(psi[j]);
    }
    *energy = creal(num) / den;
    free(x); free(V); free(t1); free(t2); free(lo); free(di); free(up); free(work);
    return 0;
}

/* ---------------------------------------------------------------- ground state by imaginary time */

/* Imaginary-time Crank-Nicolson, dt -> -i dtau:
 *     (M + dtau/2 K) psi' = (M - dtau/2 K) psi,  then psi' <- psi' / sqrt(sum |psi'|^2 dx).
 * Start from exp(-x^2); stop once |E_k - E_{k-1}| < tol or after max_iter iterations.
 * The sign is fixed so that psi is positive at the centre of the grid. */
int oracle_ground_state(int N, double dx, double a, double Z, int scheme, double dtau, long max_iter,
                        double tol, double* psi_ri, double* energy, long* iters)
{
    if (N < 3 || !(dx > 0.0) || !(a > 0.0) || !(dtau > 0.0) || max_iter < 1 || !psi_ri) return -1;
    double complex* psi = (double complex*)psi_ri;
    double* x = malloc(sizeof(double) * N);
    double* V = malloc(sizeof(double) * N);
    double* K[3]; double* M[3];
    for (int k = 0; k < 3; ++k) { K[k] = malloc(sizeof(double) * N); M[k] = malloc(sizeof(double) * N); }
    double complex* lo = malloc(sizeof(double complex) * N);
    double complex* di = malloc(sizeof(double complex) * N);
    double complex* up = malloc(sizeof(double complex) * N);
    double complex* blo = malloc(sizeof(double complex) * N);
    double complex* bdi = malloc(sizeof(double complex) * N);
    double complex* bup = malloc(sizeof(double complex) * N);
    double complex* r = malloc(sizeof(double complex) * N);
    double complex* work = malloc(sizeof(double complex) * 2 * N);
    int ok = x && V && lo && di && up && blo && bdi && bup && r && work;
    for (int k = 0; k < 3; ++k) ok = ok && K[k] && M[k];
    if (!ok) {
        free(x); free(V); free(lo); free(di); free(up); free(blo); free(bdi); free(bup); free(r); free(work);
        for (int k = 0; k < 3; ++k) { free(K[k]); free(M[k]); }
        return -2;
    }
    oracle_grid(N, dx, a, Z, x, V, NULL);
    assemble(N, dx, V, scheme, K[0], K[1], K[2], M[0], M[1], M[2]);
    double c = 0.5 * dtau;
    for (int j = 0; j < N; ++j) {
        lo[j] = M[0][j] + c * K[0][j];  di[j] = M[1][j] + c * K[1][j];  up[j] = M[2][j] + c * K[2][j];
        blo[j] = M[0][j] - c * K[0][j]; bdi[j] = M[1][j] - c * K[1][j]; bup[j] = M[2][j] - c * K[2][j];
    }
    for (int j = 0; j < N; ++j) psi[j] = exp(-x[j] * x[j]);
    double e_prev = 0.0, e = 0.0;
    long it = 0;
    for (it = 1; it <= max_iter; ++it) {
        tri_apply(N, blo, bdi, bup, psi, r);
        tri_solve(N, lo, di, up, r, psi, work);
        double nrm = 0.0;
        for (int j = 0; j < N; ++j) nrm += creal(psi[j]) * creal(psi[j]) + cimag(psi[j]) * cimag(psi[j]);
        nrm = sqrt(nrm * dx);
        for (int j = 0; j < N; ++j) psi[j] /= nrm;
        oracle_energy(N, dx, a, Z, scheme, (const double*)psi, &e);
        if (it > 1 && fabs(e - e_prev) < tol) break;
        e_prev = e;
    }
    if (it > max_iter) it = max_iter;
    if (creal(psi[N / 2]) < 0.0)
        for (int j = 0; j < N; ++j) psi[j] = -psi[j];
    if (energy) *energy = e;
    if (iters) *iters = it;
    free(x); free(V); free(lo); free(di); free(up); free(blo); free(bdi); free(bup); free(r); free(work);
    for (int k = 0; k < 3; ++k) { free(K[k]); free(M[k]); }
    return 0;
}

/* ---------------------------------------------------------------- real-time propagation */

/* Propagate one instance over the steps n = n_begin .. n_end-1 (t_n -> t_{n+1}, t_n = n dt).
 *
 * E[n] is the field at t_n for n = 0..n_end (absolute indexing).  mask is NULL (off) or N values.
 * d[n], acc[n] are written for n = n_begin+1 .. n_end from the state after each step, and also
 * for n = n_begin when n_begin == 0 (the initial state).
 *
 * FULL_CN step (midpoint field Ebar = (E_n + E_{n+1})/2):
 *     (1 + i dt/2 H(Ebar)) psi~ = (1 - i dt/2 H(Ebar)) psi^n,   psi^{n+1} = m * psi~
 * NUMEROV_SPLIT step (Sec. 4.2, Eqs. "CN - step 4", "CN - step 2", "CN - step 3"):
 *     psi1 = (M2 - i dt/2 K) psi^n;  psi2 = (M2 + i dt/2 K)^{-1} psi1;
 *     psi3_j = exp(-i dt E(t_n) x_j) psi2_j;  psi^{n+1} = m * psi3.               */
int oracle_propagate(int N, double dx, double a, double Z, int scheme, double dt, const double* mask,
                     const double* E, long n_begin, long n_end, double* psi_ri, double* d, double* acc)
{
    if (N < 3 || !(dx > 0.0) || !(a > 0.0) || n_begin < 0 || n_end < n_begin || !E || !psi_ri) return -1;
    if (scheme != ORACLE_FULL_CN && scheme != ORACLE_NUMEROV_SPLIT) return -1;
    double complex* psi = (double complex*)psi_ri;
    double* x = malloc(sizeof(double) * N);
    double* V = malloc(sizeof(double) * N);
    double* dV = malloc(sizeof(double) * N);
    double* K[3]; double* M[3];
    for (int k = 0; k < 3; ++k) { K[k] = malloc(sizeof(double) * N); M[k] = malloc(sizeof(double) * N); }
    double complex* lo = malloc(sizeof(double complex) * N);
    double complex* di = malloc(sizeof(double complex) * N);
    double complex* up = malloc(sizeof(double complex) * N);
    double complex* blo = malloc(sizeof(double complex) * N);
    double complex* bdi = malloc(sizeof(double complex) * N);
    double complex* bup = malloc(sizeof(double complex) * N);
    double complex* r = malloc(sizeof(double complex) * N);
    double complex* work = malloc(sizeof(double complex) * 2 * N);
    int ok = x && V && dV && lo && di && up && blo && bdi && bup && r && work;
    for (int k = 0; k < 3; ++k) ok = ok && K[k] && M[k];
    if (!ok) {
        free(x); free(V); free(dV); free(lo); free(di); free(up); free(blo); free(bdi); free(bup); free(r);
        free(work);
        for (int k = 0; k < 3; ++k) { free(K[k]); free(M[k]); }
        return -2;
    }
    oracle_grid(N, dx, a, Z, x, V, dV);
    assemble(N, dx, V, scheme, K[0], K[1], K[2], M[0], M[1], M[2]);
    const double complex c = I * 0.5 * dt;

    if (scheme == ORACLE_NUMEROV_SPLIT) {
        /* the Numerov matrices do not depend on time: assemble them once */
        for (int j = 0; j < N; ++j) {
            lo[j] = M[0][j] + c * K[0][j];  di[j] = M[1][j] + c * K[1][j];  up[j] = M[2][j] + c * K[2][j];
            blo[j] = M[0][j] - c * K[0][j]; bdi[j] = M[1][j] - c * K[1][j]; bup[j] = M[2][j] - c * K[2][j];
        }
    }
    if (n_begin == 0) {
        if (d && acc) observables(N, dx, x, dV, E[0], psi, &d[0], &acc[0]);
    }
    for (long n = n_begin; n < n_end; ++n) {
        if (scheme == ORACLE_FULL_CN) {
            double Ebar = 0.5 * (E[n] + E[n + 1]);
            for (int j = 0; j < N; ++j) {
                double kd = K[1][j] + x[j] * Ebar;   /* diagonal of H(Ebar) */
                lo[j] = c * K[0][j];       di[j] = 1.0 + c * kd;  up[j] = c * K[2][j];
                blo[j] = -c * K[0][j];     bdi[j] = 1.0 - c * kd; bup[j] = -c * K[2][j];
            }
            tri_apply(N, blo, bdi, bup, psi, r);
            tri_solve(N, lo, di, up, r, psi, work);
        } else {
            tri_apply(N, blo, bdi, bup, psi, r);
            tri_solve(N, lo, di, up, r, psi, work);
            for (int j = 0; j < N; ++j) psi[j] *= cexp(-I * dt * E[n] * x[j]);
        }
        if (mask)
            for (int j = 0; j < N; ++j) psi[j] *= mask[j];
        if (d && acc) observables(N, dx, x, dV, E[n + 1], psi, &d[n + 1], &acc[n + 1]);
    }
    free(x); free(V); free(dV); free(lo); free(di); free(up); free(blo); free(bdi); free(bup); free(r); free(work);
    for (int k = 0; k < 3; ++k) { free(K[k]); free(M[k]); }
    return 0;
}

/* ---------------------------------------------------------------- discrete adjoint of FULL_CN */

/* Gradient of a loss L(d, a) with respect to every field sample, through the FULL_CN forward map
 * (the exact derivative of the discrete scheme, so it matches finite differences of the scheme).
 * Inputs: the initial state psi0 (N complex), the field E[0..Nt], the mask (NULL = off), and the
 * loss gradients gd[n] = dL/dd_n, ga[n] = dL/da_n for n = 0..Nt.  Output: gE[n] = dL/dE_n.
 *
 * With lambda^n = 2 dL/d conj(psi^n) (so that dL = Re sum conj(lambda) dpsi):
 *   forward   A_n psi~^{n+1} = B_n psi^n,  psi^{n+1} = M psi~^{n+1},
 *             A_n = 1 + i h H(Ebar_n), B_n = 1 - i h H(Ebar_n), h = dt/2, M = diag(m)
 *   terminal  lambda^{Nt} = g^{Nt}
 *   backward  mu = B_n^{-1} M lambda^{n+1}   (A_n^H = B_n because H is real symmetric)
 *             lambda^n = A_n mu + g^n
 *   local     g^n_j = 2 dx (gd_n x_j + ga_n (dV_j + E_n)) psi^n_j
 *   field     dL/dEbar_n = h sum_j x_j Im(conj(mu_j) (psi^n_j + psi~^{n+1}_j)), split half to E_n and
 *             half to E_{n+1} (Ebar_n = (E_n + E_{n+1})/2); plus dL/dE_n += ga_n dx sum_j |psi^n_j|^2. */
int oracle_adjoint(int N, double dx, double a, double Z, double dt, const double* mask, const double* E, long Nt,
                   const double* psi0_ri, const double* gd, const double* ga, double* gE)
{
    if (N < 3 || !(dx > 0.0) || !(a > 0.0) || Nt < 0 || !E || !psi0_ri || !gd || !ga || !gE) return -1;
    const double h = 0.5 * dt;
    const double complex c = I * h;
    double* x = malloc(sizeof(double) * N);
    double* V = malloc(sizeof(double) * N);
    double* dV = malloc(sizeof(double) * N);
    double* K[3]; double* M[3];
    for (int k = 0; k < 3; ++k) { K[k] = malloc(sizeof(double) * N); M[k] = malloc(sizeof(double) * N); }
    double complex* psi = malloc(sizeof(double complex) * (size_t)N * (Nt + 1));     /* psi^n, n = 0..Nt */
    double complex* pt = malloc(sizeof(double complex) * (size_t)N * (Nt + 1));      /* psi~^n, n = 1..Nt */
    double complex* lo = malloc(sizeof(double complex) * N);
    double complex* di = malloc(sizeof(double complex) * N);
    double complex* up = malloc(sizeof(double complex) * N);
    double complex* blo = malloc(sizeof(double complex) * N);
    double complex* bdi = malloc(sizeof(double complex) * N);
    double complex* bup = malloc(sizeof(double complex) * N);
    double complex* r = malloc(sizeof(double complex) * N);
    double complex* lam = malloc(sizeof(double complex) * N);
    double complex* mu = malloc(sizeof(double complex) * N);
    double complex* work = malloc(sizeof(double complex) * 2 * N);
    int ok = x && V && dV && psi && pt && lo && di && up && blo && bdi && bup && r && lam && mu && work;
    for (int k = 0; k < 3; ++k) ok = ok && K[k] && M[k];
    if (!ok) {
        free(x); free(V); free(dV); free(psi); free(pt); free(lo); free(di); free(up); free(blo); free(bdi);
        free(bup); free(r); free(lam); free(mu); free(work);
        for (int k = 0; k < 3; ++k) { free(K[k]); free(M[k]); }
        return -2;
    }
    oracle_grid(N, dx, a, Z, x, V, dV);
    assemble(N, dx, V, ORACLE_FULL_CN, K[0], K[1], K[2], M[0], M[1], M[2]);
    memcpy(psi, psi0_ri, sizeof(double complex) * N);
    /* forward pass, keeping every state */
    for (long n = 0; n < Nt; ++n) {
        double Ebar = 0.5 * (E[n] + E[n + 1]);
        for (int j = 0; j < N; ++j) {
            double kd = K[1][j] + x[j] * Ebar;
            lo[j] = c * K[0][j];   di[j] = 1.0 + c * kd;  up[j] = c * K[2][j];
            blo[j] = -c * K[0][j]; bdi[j] = 1.0 - c * kd; bup[j] = -c * K[2][j];
        }
        tri_apply(N, blo, bdi, bup, psi + (size_t)n * N, r);
        tri_solve(N, lo, di, up, r, pt + (size_t)(n + 1) * N, work);
        for (int j = 0; j < N; ++j)
            psi[(size_t)(n + 1) * N + j] = (mask ? mask[j] : 1.0) * pt[(size_t)(n + 1) * N + j];
    }
    for (long n = 0; n <= Nt; ++n) gE[n] = 0.0;
    /* terminal adjoint and the direct field term of a_Nt */
    {
        const double complex* p = psi + (size_t)Nt * N;
        double nrm = 0.0;
        for (int j = 0; j < N; ++j) {
            lam[j] = 2.0 * dx * (gd[Nt] * x[j] + ga[Nt] * (dV[j] + E[Nt])) * p[j];
            nrm += creal(p[j]) * creal(p[j]) + cimag(p[j]) * cimag(p[j]);
        }
        gE[Nt] += ga[Nt] * dx * nrm;
    }
    for (long n = Nt - 1; n >= 0; --n) {
        double Ebar = 0.5 * (E[n] + E[n + 1]);
        for (int j = 0; j < N; ++j) {
            double kd = K[1][j] + x[j] * Ebar;
            lo[j] = c * K[0][j];   di[j] = 1.0 + c * kd;  up[j] = c * K[2][j];
            blo[j] = -c * K[0][j]; bdi[j] = 1.0 - c * kd; bup[j] = -c * K[2][j];
        }
        for (int j = 0; j < N; ++j) r[j] = (mask ? mask[j] : 1.0) * lam[j];
        tri_solve(N, blo, bdi, bup, r, mu, work);               /* mu = B_n^{-1} M lambda^{n+1} */
        const double complex* p = psi + (size_t)n * N;
        const double complex* q = pt + (size_t)(n + 1) * N;
        double gbar = 0.0;
        for (int j = 0; j < N; ++j) gbar += x[j] * cimag(conj(mu[j]) * (p[j] + q[j]));
        gbar *= h;
        gE[n] += 0.5 * gbar;
        gE[n + 1] += 0.5 * gbar;
        tri_apply(N, lo, di, up, mu, lam);                      /* lambda^n = A_n mu + g^n */
        double nrm = 0.0;
        for (int j = 0; j < N; ++j) {
            lam[j] += 2.0 * dx * (gd[n] * x[j] + ga[n] * (dV[j] + E[n])) * p[j];
            nrm += creal(p[j]) * creal(p[j]) + cimag(p[j]) * cimag(p[j]);
        }
        gE[n] += ga[n] * dx * nrm;
    }
    free(x); free(V); free(dV); free(psi); free(pt); free(lo); free(di); free(up); free(blo); free(bdi);
    free(bup); free(r); free(lam); free(mu); free(work);
    for (int k = 0; k < 3; ++k) { free(K[k]); free(M[k]); }
    return 0;
}

/* ---------------------------------------------------------------- energy distribution (Sec. 6.1) */

/* Time-dependent electron energy distribution of a state psi (Sec. 6.1, the equations defining
 * P(E, t) through the resolvent of the field-free Hamiltonian and its factorised form):
 *     P(E) = N_eps eps^2 <psi| ((E - H0)^2 + eps^2)^{-1} |psi> = N_eps eps^2 || (E - H0 - i eps)^{-1} psi ||^2,
 * with N_eps = 1 / (pi eps), the normalisation of a Lorentzian of half-width eps (so that the
 * distribution of an eigenstate integrates to its norm), and || v ||^2 = sum_j |v_j|^2 dx.
 * The inversion follows each scheme's representation of H0 = M^{-1} K (M, K from assemble):
 *     (E - i eps - H0)^{-1} psi = ((E - i eps) M - K)^{-1} (M psi),
 * i.e. the identity and the three-point H0 for FULL_CN, and the Numerov pencil for NUMEROV_SPLIT,
 * solved with the Thomas algorithm.  Writes P[k] for the n_E energies E_grid[k]. */
int oracle_energy_distribution(int N, double dx, double a, double Z, int scheme, const double* psi_ri,
                               const double* E_grid, int n_E, double eps, double* P)
{
    if (N < 3 || !(dx > 0.0) || !(a > 0.0) || !(eps > 0.0) || n_E < 0 || !psi_ri || (n_E > 0 && (!E_grid || !P)))
        return -1;
    if (scheme != ORACLE_FULL_CN && scheme != ORACLE_NUMEROV_SPLIT) return -1;
    const double complex* psi = (const double complex*)psi_ri;
    double* x = malloc(sizeof(double) * N);
    double* V = malloc(sizeof(double) * N);
    double* dV = malloc(sizeof(double) * N);
    double* K[3]; double* M[3];
    for (int k = 0; k < 3; ++k) { K[k] = malloc(sizeof(double) * N); M[k] = malloc(sizeof(double) * N); }
    double complex* mlo = malloc(sizeof(double complex) * N);
    double complex* mdi = malloc(sizeof(double complex) * N);
    double complex* mup = malloc(sizeof(double complex) * N);
    double complex* lo = malloc(sizeof(double complex) * N);
    double complex* di = malloc(sizeof(double complex) * N);
    double complex* up = malloc(sizeof(double complex) * N);
    double complex* r = malloc(sizeof(double complex) * N);
    double complex* y = malloc(sizeof(double complex) * N);
    double complex* work = malloc(sizeof(double complex) * 2 * N);
    int ok = x && V && dV && mlo && mdi && mup && lo && di && up && r && y && work;
    for (int k = 0; k < 3; ++k) ok = ok && K[k] && M[k];
    if (ok) {
        oracle_grid(N, dx, a, Z, x, V, dV);
        assemble(N, dx, V, scheme, K[0], K[1], K[2], M[0], M[1], M[2]);
        for (int j = 0; j < N; ++j) { mlo[j] = M[0][j]; mdi[j] = M[1][j]; mup[j] = M[2][j]; }
        tri_apply(N, mlo, mdi, mup, psi, r);                         /* M psi */
        const double norm = 1.0 / (3.14159265358979323846 * eps);   /* N_eps */
        for (int k = 0; k < n_E; ++k) {
            const double complex z = E_grid[k] - I * eps;
            for (int j = 0; j < N; ++j) {
                lo[j] = z * M[0][j] - K[0][j];
                di[j] = z * M[1][j] - K[1][j];
                up[j] = z * M[2][j] - K[2][j];
            }
            tri_solve(N, lo, di, up, r, y, work);
            double s = 0.0;
            for (int j = 0; j < N; ++j) s += creal(y[j]) * creal(y[j]) + cimag(y[j]) * cimag(y[j]);
            P[k] = norm * eps * eps * s * dx;
        }
    }
    free(x); free(V); free(dV); free(mlo); free(mdi); free(mup); free(lo); free(di); free(up); free(r); free(y);
    free(work);
    for (int k = 0; k < 3; ++k) { free(K[k]); free(M[k]); }
    return ok ? 0 : -2;
}
