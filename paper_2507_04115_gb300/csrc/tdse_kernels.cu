// CUDA kernels of the batched 1D-TDSE engine (sm_103a).
//
// Hot path: lane-batched segmented Thomas Crank-Nicolson (FULL_CN, FP64).
//   * one CTA = 32 instances of one grid class (one per lane) x P warps;
//   * warp w owns the contiguous grid segment [w m, (w+1) m) of all 32 instances;
//   * every step solves A y = psi^n with A = 1 + i dt/2 H(Ebar) and sets psi^{n+1} = m (2 y - psi^n),
//     which equals A^{-1} (2 - A) psi^n = A^{-1} (1 - i dt/2 H) psi^n, the Crank-Nicolson update,
//     without the explicit right-hand-side product;
//   * the tridiagonal solve of a segment is a Thomas sweep started K points before the segment
//     and closed K points after it.  A is strictly diagonally dominant with Re(pivot) >= 1, so
//     the forward coefficients forget their start and the back substitution forgets its seed
//     at a rate <= beta = dt/(4 dx^2) per point; K is chosen so that beta^K < 1e-17, which puts
//     the truncation below double rounding.  Segments at the walls use the exact Dirichlet ends.
// Layouts: psi [group][j][lane] (complex double, 512 B per grid point per group: one coalesced
// warp access), scratch [group][warp][row][g|d][lane].
#include "tdse_internal.h"

#include <cstdint>

namespace tdse {

// ------------------------------------------------------------------------------------ helpers

// 1/n for finite n >= 1: hardware seed (rcp.approx.ftz.f64) refined by one third-order step of
// the Newton-Raphson family, y = y0 (1 + e + e^2) with e = 1 - n y0, which leaves a relative
// error of e^3 (seed error ~2^-20 gives ~2^-60, below double rounding).
__device__ __forceinline__ double rcp_ge1(double n)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(n));
    const double e = fma(-n, y, 1.0);
    const double t = fma(e, e, e);
    return fma(y, t, y);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block reduction (fixed order): every thread returns the total.
__device__ double block_sum(double v, double* red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    return t;
}

// ------------------------------------------------------------------------------------ tables

// Per-class tables: x_j, V_j = -Z/sqrt(x_j^2 + a^2), dV/dx = Z x_j / (x_j^2 + a^2)^{3/2} (Sec. 3.1,
// Eq. "SC potential"), the FULL_CN diagonal pieces and the edge mask.
__global__ void k_build_tables(const ClassDesc* cls, int n_cls, double dt, double mw, double mp, int mask_on,
                               double* tab)
{
    const int c = blockIdx.y;
    if (c >= n_cls) return;
    const ClassDesc C = cls[c];
    const double h = 0.5 * dt;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < C.N; j += gridDim.x * blockDim.x) {
        const double x = (j - 0.5 * (C.N - 1)) * C.dx;
        const double r2 = fma(x, x, C.a * C.a);
        const double r = sqrt(r2);
        const double V = -C.Z / r;
        const double dV = C.Z * x / (r2 * r);
        double* ab = tab + tab_ab(C);
        double* xv = tab + tab_xv(C);
        double* mk = tab + tab_mk(C);
        ab[2 * j] = h * (1.0 / (C.dx * C.dx) + V);
        ab[2 * j + 1] = h * x;
        xv[2 * j] = x;
        xv[2 * j + 1] = dV;
        double m = 1.0;
        const double xb = 0.5 * C.N * C.dx - mw;
        const double ax = fabs(x);
        if (mask_on && mw > 0.0 && ax > xb) {
            const double cs = cospi(0.5 * (ax - xb) / mw);
            m = cs > 0.0 ? pow(cs, mp) : 0.0;
        }
        mk[j] = m;
    }
}

cudaError_t launch_build_tables(const ClassDesc* d_cls, int n_cls, int max_N, double dt, double mask_width,
                                double mask_exp, int mask_on, double* d_tab, cudaStream_t st)
{
    dim3 grid((max_N + 255) / 256, n_cls);
    k_build_tables<<<grid, 256, 0, st>>>(d_cls, n_cls, dt, mask_width, mask_exp, mask_on, d_tab);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ ground state

// Imaginary-time Crank-Nicolson for the field-free Hamiltonian of one class per CTA.
//   FULL_CN  : A = 1 + dtau/2 H0,   y = A^{-1} psi,       psi' = 2 y - psi
//   NUMEROV  : A = M2 + dtau/2 K,   y = A^{-1} (M2 psi),  psi' = 2 y - psi   (K = -Delta2/2 + M2 V)
// since A + B = 2M with B = M - dtau/2 K.  Then psi' is normalised and E = <psi|H0|psi> dx.
// The tridiagonal sweeps run in thread 0 over global work arrays (the ground state is computed
// once per class); normalisation and energy use the whole block.
// Work block per class (4N doubles): psi | inverse pivots w | lower multipliers l | y.
__global__ void k_ground_state(const ClassDesc* cls, int scheme, double dtau, int64_t max_iter, double tol,
                               double* work, const int64_t* work_off, double* energy, int64_t* iters)
{
    __shared__ double red[32];
    __shared__ int stop;
    const ClassDesc C = cls[blockIdx.x];
    const int N = C.N;
    double* psi = work + work_off[blockIdx.x];
    double* w = psi + N;
    double* l = w + N;
    double* y = l + N;
    const double inv_dx2 = 1.0 / (C.dx * C.dx);
    const double c = 0.5 * dtau;
    const bool numerov = (scheme == 1);

    auto V_at = [&](int j) {
        const double x = (j - 0.5 * (N - 1)) * C.dx;
        return -C.Z / sqrt(fma(x, x, C.a * C.a));
    };
    // A's diagonal and off-diagonals (row j: lo_j psi_{j-1} + di_j psi_j + up_j psi_{j+1})
    auto A_di = [&](int j) {
        return numerov ? 10.0 / 12.0 + c * (inv_dx2 + (10.0 / 12.0) * V_at(j)) : 1.0 + c * (inv_dx2 + V_at(j));
    };
    auto A_lo = [&](int j) { return numerov ? 1.0 / 12.0 + c * (-0.5 * inv_dx2 + V_at(j - 1) / 12.0) : -c * 0.5 * inv_dx2; };
    auto A_up = [&](int j) { return numerov ? 1.0 / 12.0 + c * (-0.5 * inv_dx2 + V_at(j + 1) / 12.0) : -c * 0.5 * inv_dx2; };

    // initial state exp(-x^2) and the LU factors of A (Thomas): w_j = 1/(di_j - lo_j up_{j-1} w_{j-1}),
    // l_j = lo_j w_{j-1} ... stored as w (inverse pivot) and the products needed by the sweeps.
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double x = (j - 0.5 * (N - 1)) * C.dx;
        psi[j] = exp(-x * x);
    }
    if (threadIdx.x == 0) {
        double wprev = 0.0;
        for (int j = 0; j < N; ++j) {
            const double piv = j == 0 ? A_di(0) : A_di(j) - A_lo(j) * A_up(j - 1) * wprev;
            w[j] = 1.0 / piv;
            l[j] = j == 0 ? 0.0 : A_lo(j);
            wprev = w[j];
        }
    }
    __syncthreads();

    double e_prev = 0.0, e = 0.0;
    int64_t it = 1;
    for (;; ++it) {
        // right-hand side r = psi (FD) or M2 psi (Numerov), kept in y
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            double r = psi[j];
            if (numerov) {
                r = (10.0 / 12.0) * psi[j] + ((j > 0 ? psi[j - 1] : 0.0) + (j < N - 1 ? psi[j + 1] : 0.0)) / 12.0;
            }
            y[j] = r;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // forward: y_j <- (r_j - lo_j y_{j-1}) w_j ; backward: y_j <- y_j - up_j w_j y_{j+1}
            double prev = 0.0;
            for (int j = 0; j < N; ++j) {
                prev = (y[j] - l[j] * prev) * w[j];
                y[j] = prev;
            }
            double nxt = 0.0;
            for (int j = N - 1; j >= 0; --j) {
                nxt = y[j] - (j < N - 1 ? A_up(j) * w[j] * nxt : 0.0);
                y[j] = nxt;
            }
        }
        __syncthreads();
        double s = 0.0;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            const double v = 2.0 * y[j] - psi[j];
            psi[j] = v;
            s += v * v;
        }
        const double nrm = sqrt(block_sum(s, red) * C.dx);
        for (int j = threadIdx.x; j < N; j += blockDim.x) psi[j] /= nrm;
        __syncthreads();
        // energy: kinetic part T psi = -Delta2/2 psi (FD) or M2^{-1}(-Delta2/2 psi) (Numerov)
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            const double lap = ((j > 0 ? psi[j - 1] : 0.0) - 2.0 * psi[j] + (j < N - 1 ? psi[j + 1] : 0.0)) * inv_dx2;
            y[j] = -0.5 * lap;
        }
        __syncthreads();
        if (numerov && threadIdx.x == 0) {
            // solve M2 t = y in place (constant-coefficient Thomas, coefficients recomputed on the fly)
            double cp_prev = 0.0, prev = 0.0;
            for (int j = 0; j < N; ++j) {
                const double piv = 10.0 / 12.0 - (j > 0 ? (1.0 / 12.0) * cp_prev : 0.0);
                const double cp = (1.0 / 12.0) / piv;
                prev = (y[j] - (j > 0 ? (1.0 / 12.0) * prev : 0.0)) / piv;
                y[j] = prev;
                l[j] = cp;   // l is free once the solve above is done; reuse it for M2's c'
                cp_prev = cp;
            }
            double nxt = 0.0;
            for (int j = N - 1; j >= 0; --j) {
                nxt = y[j] - (j < N - 1 ? l[j] * nxt : 0.0);
                y[j] = nxt;
            }
        }
        __syncthreads();
        double se = 0.0;
        for (int j = threadIdx.x; j < N; j += blockDim.x) se += psi[j] * (y[j] + V_at(j) * psi[j]);
        e = block_sum(se, red) * C.dx;
        if (numerov) {
            // restore the lower multipliers of A for the next iteration
            for (int j = threadIdx.x; j < N; j += blockDim.x) l[j] = j == 0 ? 0.0 : A_lo(j);
        }
        if (threadIdx.x == 0) stop = (it > 1 && fabs(e - e_prev) < tol) || it >= max_iter;
        __syncthreads();
        if (stop) break;
        e_prev = e;
    }
    // sign: positive at the centre
    const double sgn = psi[N / 2] < 0.0 ? -1.0 : 1.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) psi[j] *= sgn;
    if (threadIdx.x == 0) {
        energy[blockIdx.x] = e;
        iters[blockIdx.x] = it;
    }
}

cudaError_t launch_ground_state(const ClassDesc* d_cls, int n_cls, int scheme, double dtau, int64_t max_iter,
                                double tol, double* d_work, const int64_t* d_work_off, double* d_energy,
                                int64_t* d_iters, cudaStream_t st)
{
    k_ground_state<<<n_cls, 256, 0, st>>>(d_cls, scheme, dtau, max_iter, tol, d_work, d_work_off, d_energy, d_iters);
    return cudaGetLastError();
}

__global__ void k_broadcast_psi(const GroupDesc* groups, int64_t n_groups, const double* work,
                                const int64_t* work_off, const int64_t* slot_valid, double2* psi)
{
    const int lane = threadIdx.x & 31;
    for (int64_t g = blockIdx.y; g < n_groups; g += gridDim.y) {
        const GroupDesc G = groups[g];
        if (!slot_valid[G.slot0 + lane]) continue;
        const double* src = work + work_off[G.cls];
        double2* dst = psi + G.psi_off;
        for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < G.N; j += gridDim.x * (blockDim.x >> 5))
            dst[(int64_t)j * kLanes + lane] = make_double2(src[j], 0.0);
    }
}

cudaError_t launch_broadcast_psi(const GroupDesc* d_groups, int64_t n_groups, const double* d_work,
                                 const int64_t* d_work_off, const int64_t* d_slot_valid, double2* d_psi,
                                 cudaStream_t st)
{
    if (n_groups == 0) return cudaSuccess;
    dim3 grid(16, (unsigned)(n_groups < 65535 ? n_groups : 65535));
    k_broadcast_psi<<<grid, 256, 0, st>>>(d_groups, n_groups, d_work, d_work_off, d_slot_valid, d_psi);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ propagation

// Observables of the state held in psi for one group: partial sums over the warp's segment,
// combined across warps through shared memory by warp 0.  Returns (in warp 0) sums of
// |psi|^2, x |psi|^2, dV/dx |psi|^2.
struct ObsSums {
    double n, x, v;
};

__device__ __forceinline__ ObsSums reduce_obs(ObsSums s, double* red, int P)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    red[(w * 3 + 0) * 32 + lane] = s.n;
    red[(w * 3 + 1) * 32 + lane] = s.x;
    red[(w * 3 + 2) * 32 + lane] = s.v;
    __syncthreads();
    ObsSums t{0.0, 0.0, 0.0};
    if (w == 0) {
        for (int q = 0; q < P; ++q) {
            t.n += red[(q * 3 + 0) * 32 + lane];
            t.x += red[(q * 3 + 1) * 32 + lane];
            t.v += red[(q * 3 + 2) * 32 + lane];
        }
    }
    return t;
}

__global__ void __launch_bounds__(512, 1)
k_propagate_fp64(const GroupDesc* __restrict__ groups, int64_t g_begin, const ClassDesc* __restrict__ cls,
                 const double* __restrict__ tab, const int64_t* __restrict__ slot_row,
                 const int64_t* __restrict__ slot_nt, double2* __restrict__ psi_all,
                 double2* __restrict__ scratch_all, const double* __restrict__ E, double* __restrict__ d_out,
                 double* __restrict__ a_out, int64_t sample_base, int64_t step_begin, int64_t step_end,
                 int mask_on, int* __restrict__ status)
{
    extern __shared__ double red[];   // [P][3][32]
    const GroupDesc G = groups[g_begin + blockIdx.x];
    const ClassDesc C = cls[G.cls];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int N = G.N, P = G.P, K = G.K, m = G.m;
    const int64_t slot = G.slot0 + lane;
    const int64_t nt = slot_nt[slot];          // 0 for padding lanes
    const int64_t row = slot_row[slot];
    const double beta = C.beta;
    const double b2 = beta * beta;
    const double dx = C.dx;

    const int s = min(N, w * m);
    const int e = min(N, s + m);
    const int lo = max(0, s - K);
    const int hi = min(N, e + K);
    double2* __restrict__ ps = psi_all + G.psi_off;
    double2* __restrict__ sc = scratch_all + G.scratch_off + (int64_t)w * G.rows * (2 * kLanes);
    const double2* __restrict__ tab_ab2 = reinterpret_cast<const double2*>(tab + tab_ab(C));
    const double2* __restrict__ tab_xv2 = reinterpret_cast<const double2*>(tab + tab_xv(C));
    const double* __restrict__ tab_m = tab + tab_mk(C);
    const int jm_lo = mask_on ? C.jm_lo : 0;
    const int jm_hi = mask_on ? C.jm_hi : N - 1;

    const int64_t n_last = min(step_end, G.nt_max);

    // observables of the initial state
    if (step_begin == 0) {
        ObsSums o{0.0, 0.0, 0.0};
        for (int j = s; j < e; ++j) {
            const double2 p = ps[(int64_t)j * kLanes + lane];
            const double rho = fma(p.x, p.x, p.y * p.y);
            const double2 xv = tab_xv2[j];
            o.n += rho;
            o.x = fma(xv.x, rho, o.x);
            o.v = fma(xv.y, rho, o.v);
        }
        const ObsSums t = reduce_obs(o, red, P);
        if (w == 0 && nt >= 0) {
            const double E0 = E[row - sample_base];
            d_out[row - sample_base] = t.x * dx;
            a_out[row - sample_base] = fma(E0, t.n, t.v) * dx;
        }
        __syncthreads();
    }

    for (int64_t n = step_begin; n < n_last; ++n) {
        const bool active = n < nt;
        double En = 0.0, En1 = 0.0;
        if (active) {
            En = E[row + n - sample_base];
            En1 = E[row + n + 1 - sample_base];
        }
        const double Eb = 0.5 * (En + En1);

        // forward elimination over [lo, hi): g_j = 1/q_j, q_j = 1 + i s_j + beta^2 g_{j-1};
        // d_j = g_j (psi_j + i beta d_{j-1})
        double gr = 0.0, gi = 0.0, dr = 0.0, di = 0.0;
        for (int j = lo; j < hi; ++j) {
            const double2 p = ps[(int64_t)j * kLanes + lane];
            const double2 t = tab_ab2[j];
            const double sj = fma(t.y, Eb, t.x);
            const double qr = fma(b2, gr, 1.0);
            const double qi = fma(b2, gi, sj);
            const double inv = rcp_ge1(fma(qr, qr, qi * qi));
            gr = qr * inv;
            gi = -qi * inv;
            const double ur = fma(-beta, di, p.x);
            const double ui = fma(beta, dr, p.y);
            dr = fma(gr, ur, -gi * ui);
            di = fma(gr, ui, gi * ur);
            double2* r = sc + (int64_t)(j - lo) * (2 * kLanes);
            r[lane] = make_double2(gr, gi);
            r[kLanes + lane] = make_double2(dr, di);
        }
        __syncthreads();   // every read of psi^n (own segment and halos) precedes any write of psi^{n+1}

        // back substitution y_j = d_j + i beta g_j y_{j+1}, seeded with 0 at hi (exact at the wall)
        double yr = 0.0, yi = 0.0;
        for (int j = hi - 1; j >= e; --j) {
            const double2* r = sc + (int64_t)(j - lo) * (2 * kLanes);
            const double2 g = r[lane];
            const double2 d = r[kLanes + lane];
            const double pr = fma(g.x, yr, -g.y * yi);
            const double pi = fma(g.x, yi, g.y * yr);
            yr = fma(-beta, pi, d.x);
            yi = fma(beta, pr, d.y);
        }
        ObsSums o{0.0, 0.0, 0.0};
        for (int j = e - 1; j >= s; --j) {
            const double2* r = sc + (int64_t)(j - lo) * (2 * kLanes);
            const double2 g = r[lane];
            const double2 d = r[kLanes + lane];
            const double pr = fma(g.x, yr, -g.y * yi);
            const double pi = fma(g.x, yi, g.y * yr);
            yr = fma(-beta, pi, d.x);
            yi = fma(beta, pr, d.y);
            double2* pp = ps + (int64_t)j * kLanes + lane;
            const double2 old = *pp;
            double xr = fma(2.0, yr, -old.x);
            double xi = fma(2.0, yi, -old.y);
            if (j < jm_lo || j > jm_hi) {
                const double mm = tab_m[j];
                xr *= mm;
                xi *= mm;
            }
            if (active) *pp = make_double2(xr, xi);
            const double rho = fma(xr, xr, xi * xi);
            const double2 xv = tab_xv2[j];
            o.n += rho;
            o.x = fma(xv.x, rho, o.x);
            o.v = fma(xv.y, rho, o.v);
        }
        const ObsSums t = reduce_obs(o, red, P);   // contains the barrier after the psi writes
        if (w == 0 && active) {
            const int64_t k = row + n + 1 - sample_base;
            d_out[k] = t.x * dx;
            a_out[k] = fma(En1, t.n, t.v) * dx;
            const double nrm = t.n * dx;
            if (!(nrm <= 1.0 + 1e-6)) status[slot] = 1;
        }
    }
}

cudaError_t launch_propagate_fp64(const GroupDesc* d_groups, int64_t g_begin, int64_t n_groups, int P,
                                  const ClassDesc* d_cls, const double* d_tab, const int64_t* d_slot_row,
                                  const int64_t* d_slot_nt, double2* d_psi, double2* d_scratch, const double* E,
                                  double* d_out, double* a_out, int64_t sample_base, int64_t step_begin,
                                  int64_t step_end, int mask_on, int* d_status, cudaStream_t st)
{
    if (n_groups == 0) return cudaSuccess;
    const size_t smem = (size_t)P * 3 * kLanes * sizeof(double);
    k_propagate_fp64<<<(unsigned)n_groups, P * kLanes, smem, st>>>(
        d_groups, g_begin, d_cls, d_tab, d_slot_row, d_slot_nt, d_psi, d_scratch, E, d_out, a_out, sample_base,
        step_begin, step_end, mask_on, d_status);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ psi access

__global__ void k_get_psi(const double2* psi, int64_t off, int N, int lane, double* out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const double2 v = psi[off + (int64_t)j * kLanes + lane];
        out[2 * j] = v.x;
        out[2 * j + 1] = v.y;
    }
}

__global__ void k_set_psi(double2* psi, int64_t off, int N, int lane, const double* in)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x)
        psi[off + (int64_t)j * kLanes + lane] = make_double2(in[2 * j], in[2 * j + 1]);
}

cudaError_t launch_get_psi(const double2* d_psi, int64_t psi_off, int N, int lane, double* out, cudaStream_t st)
{
    k_get_psi<<<(N + 255) / 256, 256, 0, st>>>(d_psi, psi_off, N, lane, out);
    return cudaGetLastError();
}

cudaError_t launch_set_psi(double2* d_psi, int64_t psi_off, int N, int lane, const double* in, cudaStream_t st)
{
    k_set_psi<<<(N + 255) / 256, 256, 0, st>>>(d_psi, psi_off, N, lane, in);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ spectrum

// S_i[k] = dt^2 |sum_n a_i[n] exp(-2 pi i k n / L_i)|^2 for k in [k_begin, k_end); one thread per
// bin, the row staged through shared memory in tiles.  The twiddle advances by complex
// multiplication and is re-seeded from sincospi every 64 samples (index k n mod L in integers).
__global__ void k_spectrum(const double* a, const int64_t* offs, int64_t row0, double dt, int64_t k_begin,
                           int64_t k_end, double* S)
{
    __shared__ double tile[512];
    const int64_t row = row0 + blockIdx.y;
    const int64_t base = offs[row];
    const int64_t L = offs[row + 1] - base;
    const int64_t nb = k_end - k_begin;
    const int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = kk < nb && L > 0;
    const int64_t k = k_begin + (live ? kk : 0);
    const int64_t kmod = L > 0 ? k % L : 0;
    double wr = 1.0, wi = 0.0;
    if (L > 0) sincospi(-2.0 * (double)kmod / (double)L, &wi, &wr);
    double ar = 0.0, ai = 0.0, zr = 1.0, zi = 0.0;
    int64_t idx = 0;   // (k n) mod L
    for (int64_t t0 = 0; t0 < L; t0 += 512) {
        const int cnt = (int)(L - t0 < 512 ? L - t0 : 512);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) tile[i] = a[base + t0 + i];
        __syncthreads();
        for (int i = 0; i < cnt; ++i) {
            const int64_t n = t0 + i;
            if ((n & 63) == 0) sincospi(-2.0 * (double)idx / (double)L, &zi, &zr);
            const double v = tile[i];
            ar = fma(v, zr, ar);
            ai = fma(v, zi, ai);
            const double nr = fma(zr, wr, -zi * wi);
            const double ni = fma(zr, wi, zi * wr);
            zr = nr;
            zi = ni;
            idx += kmod;
            if (idx >= L) idx -= L;
        }
    }
    if (live) S[row * nb + kk] = (ar * ar + ai * ai) * dt * dt;
}

cudaError_t launch_spectrum(const double* a, const int64_t* d_offsets, int64_t n_rows, double dt, int64_t k_begin,
                            int64_t k_end, double* S, cudaStream_t st)
{
    if (n_rows == 0) return cudaSuccess;
    const int64_t nb = k_end - k_begin;
    for (int64_t r0 = 0; r0 < n_rows; r0 += 65535) {
        const int64_t nr = n_rows - r0 < 65535 ? n_rows - r0 : 65535;
        dim3 grid((unsigned)((nb + 127) / 128), (unsigned)nr);
        k_spectrum<<<grid, 128, 0, st>>>(a, d_offsets, r0, dt, k_begin, k_end, S);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace tdse
