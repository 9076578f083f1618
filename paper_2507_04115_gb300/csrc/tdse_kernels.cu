// Set-up and auxiliary kernels of libtdse (sm_103a): per-class tables, imaginary-time ground
// state, wavefunction broadcast and access, the populations of the states, and the DFT power
// spectrum.  The propagation kernels
// live in tdse_full_cn.cu and tdse_numerov.cu, the adjoint in tdse_adjoint.cu, the energy
// distribution in tdse_resolvent.cu.
#include "tdse_device.cuh"
#include "tdse_internal.h"

#include <cooperative_groups.h>
#include <cstdint>

namespace tdse {

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
        ab[2 * j] = h * (1.0 / (C.dx * C.dx) + V) / C.beta;
        ab[2 * j + 1] = h * x / C.beta;
        reinterpret_cast<float2*>(tab + tab_af(C))[j] = make_float2((float)ab[2 * j], (float)ab[2 * j + 1]);
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
        reinterpret_cast<float4*>(tab + tab_fx(C))[j] = make_float4((float)x, (float)dV, (float)m, 0.0f);
        const float xh = (float)x, vh = (float)dV;
        reinterpret_cast<float4*>(tab + tab_xff(C))[j] = make_float4(xh, (float)(x - (double)xh), vh, (float)(dV - (double)vh));
        tab[tab_vv(C) + j] = V;
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

// First-order linear recurrence x_j = a_j x_{j-1} + b_j over j = 0..N-1 with x_{-1} = 0 (rev: over
// j = N-1..0 with x_N = 0), solved in place by the whole block (x holds b on entry, the solution on
// exit): each thread runs the recurrence over its chunk of the index range from zero, the chunk maps
// x_out = P x_in + v (P the product of the chunk's a) are composed by an inclusive scan over the
// threads, and each chunk adds its incoming value times the running product of its a.  The result
// equals the sequential sweep up to the order of rounding.  sp, sv: blockDim.x doubles each.
__device__ void block_recurrence(double* __restrict__ x, const double* __restrict__ a, int N, bool rev, double* sp,
                                 double* sv)
{
    const int T = blockDim.x, t = threadIdx.x;
    const int c = (N + T - 1) / T;
    const int k0 = min(N, t * c), k1 = min(N, k0 + c);
    double y = 0.0, P = 1.0;
    for (int k = k0; k < k1; ++k) {
        const int j = rev ? N - 1 - k : k;
        y = fma(a[j], y, x[j]);
        P *= a[j];
        x[j] = y;
    }
    sp[t] = P;
    sv[t] = y;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        double pl = 1.0, vl = 0.0;
        if (t >= off) {
            pl = sp[t - off];
            vl = sv[t - off];
        }
        __syncthreads();
        if (t >= off) {
            const double pr = sp[t], vr = sv[t];
            sp[t] = pr * pl;
            sv[t] = fma(pr, vl, vr);
        }
        __syncthreads();
    }
    const double carry = t > 0 ? sv[t - 1] : 0.0;   // x at the end of the previous chunk
    double Q = 1.0;
    for (int k = k0; k < k1; ++k) {
        const int j = rev ? N - 1 - k : k;
        Q *= a[j];
        x[j] = fma(Q, carry, x[j]);
    }
    __syncthreads();
}

// Imaginary-time Crank-Nicolson for the field-free Hamiltonian of one class per CTA.
//   FULL_CN  : A = 1 + dtau/2 H0,   y = A^{-1} psi,       psi' = 2 y - psi
//   NUMEROV  : A = M2 + dtau/2 K,   y = A^{-1} (M2 psi),  psi' = 2 y - psi   (K = -Delta2/2 + M2 V)
// since A + B = 2M with B = M - dtau/2 K.  Then psi' is normalised and E = <psi|H0|psi> dx.
// A is factored once (Thomas pivots, thread 0); every iteration's solve is then two first-order
// linear recurrences with fixed coefficients, solved block-parallel (block_recurrence), as are the
// two sweeps of Numerov's M2 solve in the energy.
// Work block per class (kGsWork N doubles): psi | 1/pivot of A | forward a | backward a | y |
// 1/pivot of M2 | M2 forward a | M2 backward a.
__global__ void k_ground_state(const ClassDesc* cls, int scheme, double dtau, int64_t max_iter, double tol,
                               double* work, const int64_t* work_off, double* energy, int64_t* iters)
{
    __shared__ double red[32];
    __shared__ double sp[kGsThreads], sv[kGsThreads];
    __shared__ int stop;
    const ClassDesc C = cls[blockIdx.x];
    const int N = C.N;
    double* psi = work + work_off[blockIdx.x];
    double* w = psi + N;
    double* fa = w + N;
    double* ba = fa + N;
    double* y = ba + N;
    double* mw = y + N;
    double* mfa = mw + N;
    double* mba = mfa + N;
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

    // initial state exp(-x^2); the Thomas factors of A: w_j = 1/(di_j - lo_j up_{j-1} w_{j-1}), and
    // the recurrence coefficients of the two sweeps, forward y_j = w_j r_j - lo_j w_j y_{j-1} and
    // backward y_j = y_j - up_j w_j y_{j+1}; for Numerov also those of M2 = tridiag(1, 10, 1)/12
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double x = (j - 0.5 * (N - 1)) * C.dx;
        psi[j] = exp(-x * x);
    }
    if (threadIdx.x == 0) {
        double wprev = 0.0, mprev = 0.0;
        for (int j = 0; j < N; ++j) {
            const double piv = j == 0 ? A_di(0) : A_di(j) - A_lo(j) * A_up(j - 1) * wprev;
            w[j] = 1.0 / piv;
            wprev = w[j];
            if (numerov) {
                const double mp = 10.0 / 12.0 - (j > 0 ? (1.0 / 144.0) * mprev : 0.0);
                mw[j] = 1.0 / mp;
                mprev = mw[j];
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        fa[j] = j == 0 ? 0.0 : -A_lo(j) * w[j];
        ba[j] = j == N - 1 ? 0.0 : -A_up(j) * w[j];
        if (numerov) {
            mfa[j] = j == 0 ? 0.0 : -(1.0 / 12.0) * mw[j];
            mba[j] = j == N - 1 ? 0.0 : -(1.0 / 12.0) * mw[j];
        }
    }
    __syncthreads();

    double e_prev = 0.0, e = 0.0;
    int64_t it = 1;
    for (;; ++it) {
        // right-hand side w_j r_j with r = psi (FD) or M2 psi (Numerov), then the two sweeps
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            double r = psi[j];
            if (numerov) {
                r = (10.0 / 12.0) * psi[j] + ((j > 0 ? psi[j - 1] : 0.0) + (j < N - 1 ? psi[j + 1] : 0.0)) / 12.0;
            }
            y[j] = w[j] * r;
        }
        __syncthreads();
        block_recurrence(y, fa, N, false, sp, sv);
        block_recurrence(y, ba, N, true, sp, sv);
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
            y[j] = -0.5 * lap * (numerov ? mw[j] : 1.0);
        }
        __syncthreads();
        if (numerov) {
            // M2 t = y: forward t'_j = y_j/p_j - (1/12) t'_{j-1}/p_j, backward t_j = t'_j - (1/12)/p_j t_{j+1}
            block_recurrence(y, mfa, N, false, sp, sv);
            block_recurrence(y, mba, N, true, sp, sv);
        }
        double se = 0.0;
        for (int j = threadIdx.x; j < N; j += blockDim.x) se += psi[j] * (y[j] + V_at(j) * psi[j]);
        e = block_sum(se, red) * C.dx;
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
    k_ground_state<<<n_cls, kGsThreads, 0, st>>>(d_cls, scheme, dtau, max_iter, tol, d_work, d_work_off, d_energy,
                                                  d_iters);
    return cudaGetLastError();
}

__device__ __forceinline__ void store_cx(double2* p, double a, double b) { *p = make_double2(a, b); }
__device__ __forceinline__ void store_cx(float2* p, double a, double b) { *p = make_float2((float)a, (float)b); }

template <class Cx>
__global__ void k_broadcast_psi(const GroupDesc* groups, int64_t n_groups, const double* work,
                                const int64_t* work_off, const int64_t* slot_valid, Cx* psi)
{
    const int lane = threadIdx.x & 31;
    for (int64_t g = blockIdx.y; g < n_groups; g += gridDim.y) {
        const GroupDesc G = groups[g];
        // a warp covers 32 / I consecutive points of the [N][I] layout
        const int i = lane % G.I, jq = lane / G.I, per_warp = kLanes / G.I;
        if (!slot_valid[G.slot0 + i]) continue;
        const double* src = work + work_off[G.cls];
        Cx* dst = psi + G.psi_off;
        for (int j0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * per_warp; j0 < G.N;
             j0 += gridDim.x * (blockDim.x >> 5) * per_warp) {
            const int j = j0 + jq;
            if (j < G.N) store_cx(dst + (int64_t)j * G.I + i, src[j], 0.0);
        }
    }
}

cudaError_t launch_broadcast_psi(int mixed, const GroupDesc* d_groups, int64_t n_groups, const double* d_work,
                                 const int64_t* d_work_off, const int64_t* d_slot_valid, void* d_psi,
                                 cudaStream_t st)
{
    if (n_groups == 0) return cudaSuccess;
    dim3 grid(16, (unsigned)(n_groups < 65535 ? n_groups : 65535));
    if (mixed)
        k_broadcast_psi<float2><<<grid, 256, 0, st>>>(d_groups, n_groups, d_work, d_work_off, d_slot_valid,
                                                       static_cast<float2*>(d_psi));
    else
        k_broadcast_psi<double2><<<grid, 256, 0, st>>>(d_groups, n_groups, d_work, d_work_off, d_slot_valid,
                                                        static_cast<double2*>(d_psi));
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ psi access

template <class Cx>
__global__ void k_get_psi(const Cx* psi, int64_t off, int N, int lane, int I, double* out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const Cx v = psi[off + (int64_t)j * I + lane];
        out[2 * j] = v.x;
        out[2 * j + 1] = v.y;
    }
}

template <class Cx>
__global__ void k_set_psi(Cx* psi, int64_t off, int N, int lane, int I, const double* in)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x)
        store_cx(psi + off + (int64_t)j * I + lane, in[2 * j], in[2 * j + 1]);
}

cudaError_t launch_get_psi(int mixed, const void* d_psi, int64_t psi_off, int N, int lane, int I, double* out,
                           cudaStream_t st)
{
    if (mixed)
        k_get_psi<float2><<<(N + 255) / 256, 256, 0, st>>>(static_cast<const float2*>(d_psi), psi_off, N, lane, I, out);
    else
        k_get_psi<double2><<<(N + 255) / 256, 256, 0, st>>>(static_cast<const double2*>(d_psi), psi_off, N, lane, I, out);
    return cudaGetLastError();
}

cudaError_t launch_set_psi(int mixed, void* d_psi, int64_t psi_off, int N, int lane, int I, const double* in, cudaStream_t st)
{
    if (mixed)
        k_set_psi<float2><<<(N + 255) / 256, 256, 0, st>>>(static_cast<float2*>(d_psi), psi_off, N, lane, I, in);
    else
        k_set_psi<double2><<<(N + 255) / 256, 256, 0, st>>>(static_cast<double2*>(d_psi), psi_off, N, lane, I, in);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ populations

// Support of psi0: one warp per class scans 32 points at a time from each end, with an inclusive
// warp prefix sum of psi0_j^2 dx, and stops at the first point whose running tail exceeds
// kSupportTail^2 / 2.  The overlap with any psi then misses at most kSupportTail ||psi|| (Cauchy-
// Schwarz over the two tails), below the rounding of a population.
__global__ void k_gs_support(const ClassDesc* cls, const double* work, const int64_t* work_off, int64_t* support)
{
    const int lane = threadIdx.x & 31;
    const ClassDesc C = cls[blockIdx.x];
    const int N = C.N;
    const double* p0 = work + work_off[blockIdx.x];
    const double thr = 0.5 * kSupportTail * kSupportTail;
    int bound[2] = {0, N};
    for (int side = 0; side < 2; ++side) {
        double run = 0.0;
        int found = side == 0 ? N : 0;   // psi0 negligible everywhere: empty support
        for (int k0 = 0; k0 < N; k0 += kLanes) {
            const int k = k0 + lane;   // k-th point from this side's end
            const int j = side == 0 ? k : N - 1 - k;
            double v = k < N ? p0[j] * p0[j] * C.dx : 0.0;
            for (int o = 1; o < kLanes; o <<= 1) {
                const double t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            const unsigned over = __ballot_sync(0xffffffffu, k < N && run + v > thr);
            if (over) {
                const int kk = k0 + __ffs(over) - 1;   // first point that must be kept
                found = side == 0 ? kk : N - kk;
                break;
            }
            run += __shfl_sync(0xffffffffu, v, kLanes - 1);
        }
        bound[side] = found;
    }
    if (lane == 0) {
        support[2 * blockIdx.x] = bound[0];
        support[2 * blockIdx.x + 1] = bound[1] > bound[0] ? bound[1] : bound[0];
    }
}

cudaError_t launch_gs_support(const ClassDesc* d_cls, int n_cls, const double* d_work, const int64_t* d_work_off,
                              int64_t* d_support, cudaStream_t st)
{
    if (n_cls == 0) return cudaSuccess;
    k_gs_support<<<n_cls, kLanes, 0, st>>>(d_cls, d_work, d_work_off, d_support);
    return cudaGetLastError();
}

// Ground-state population |sum_j psi0_j psi_j dx|^2 and near-core probability
// sum_{|x_j| < r_core} |psi_j|^2 dx of every instance (Sec. 7.5).
//   Only the rows j in the hull of psi0's support [s_lo, s_hi) and of the core interval are read:
//   outside the support the overlap's terms sum to less than kSupportTail ||psi||, outside the core
//   interval the second sum has no terms.  The core interval is {j : |x_j| < r_core} with
//   x_j = (j - (N-1)/2) dx, the same expression (and rounding) as the tables; x is odd about the
//   centre in floating point too, so the interval is [c_lo, N - c_lo), c_lo found from an estimate
//   corrected by exact comparisons.
//   A group is handled by a thread-block cluster of S CTAs (S <= 8, chosen on the host so that the
//   grid fills the SMs); CTA r of the cluster takes the r-th chunk of the rows.  A warp reads 32
//   consecutive elements of the [N][I] layout per load (32 / I points of all I instances),
//   kPopDepth loads in flight per thread; lane l accumulates instance l % I.
//   Sums: shuffles over the lanes of an instance, the CTA's warps in a fixed order into shared
//   memory, then CTA 0 of the cluster adds the S CTAs' partials in rank order through distributed
//   shared memory -- deterministic, no scratch, no atomics.
constexpr int kPopWarps = 8;
constexpr int kPopDepth = 4;
constexpr int kPopMaxCluster = 8;

__device__ __forceinline__ double grid_x(int j, int N, double dx) { return (j - 0.5 * (N - 1)) * dx; }

// float -> double from the IEEE-754 fields with integer operations only (a conversion instruction
// would occupy the FP64 pipe, which the sums already saturate).  Normal numbers: exponent rebiased
// by 1023 - 127 = 896, the 23 mantissa bits moved to the top of the 52.  Subnormal floats m 2^-149
// are normal doubles: with p the position of m's top bit, exponent p - 149 + 1023 and the bits
// below it as mantissa.  Zero keeps its sign; infinities and NaN (payload kept) map to 2047.
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    const uint32_t p = 31u - (uint32_t)__clz((int)(m | 1u));   // top bit of m (m = 0: unused)
    const uint32_t E = e == 0xffu ? 2047u : (e != 0u ? e + 896u : (m != 0u ? p + 874u : 0u));
    const uint32_t M = e != 0u ? m : ((m << (23u - p)) & 0x7fffffu);
    const uint32_t hi = (u & 0x80000000u) | (E << 20) | (M >> 3);
    return __hiloint2double((int)hi, (int)(M << 29));
}

// First j of the core interval; the interval is empty when the result exceeds (N - 1) / 2.
__device__ int core_lo(int N, double dx, double r_core)
{
    const int mid = (N - 1) / 2;   // last point with x <= 0
    if (!(r_core > 0.0)) return mid + 1;
    const double t = 0.5 * (N - 1) - r_core / dx;
    int lo = t <= 0.0 ? 0 : (t >= (double)mid ? mid : (int)ceil(t));
    while (lo > 0 && fabs(grid_x(lo - 1, N, dx)) < r_core) --lo;
    while (lo <= mid && !(fabs(grid_x(lo, N, dx)) < r_core)) ++lo;
    return lo;
}

template <class Cx>
__global__ void __launch_bounds__(kPopWarps * 32) k_populations(const GroupDesc* __restrict__ groups,
                                                                const ClassDesc* __restrict__ cls,
                                                                const int64_t* __restrict__ slot_inst,
                                                                const Cx* __restrict__ psi_all,
                                                                const double* __restrict__ gs_work,
                                                                const int64_t* __restrict__ gs_off,
                                                                const int64_t* __restrict__ support, double r_core,
                                                                double* __restrict__ out)
{
    namespace cg = cooperative_groups;
    __shared__ double part[kPopWarps][3][kLanes];
    __shared__ double cta_sum[3][kLanes];
    __shared__ int s_core_lo;
    cg::cluster_group cluster = cg::this_cluster();
    const int S = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const GroupDesc G = groups[blockIdx.x / S];
    const ClassDesc C = cls[G.cls];
    const int N = G.N, I = G.I, per_warp = kLanes / I;
    const int i = lane % I, jq = lane / I;
    // rows to read: hull of the support and the core interval (its bound found by one thread: the
    // division and the comparisons would otherwise cost every thread as much FP64 work as its sums)
    if (threadIdx.x == 0) s_core_lo = core_lo(N, C.dx, r_core);
    __syncthreads();
    const int c_lo = s_core_lo;
    const bool core_on = c_lo <= (N - 1) / 2;
    const int c_hi = N - c_lo;
    int h_lo = (int)support[2 * G.cls], h_hi = (int)support[2 * G.cls + 1];
    if (core_on) {
        h_lo = min(h_lo, c_lo);
        h_hi = max(h_hi, c_hi);
    }
    // chunk of this CTA: whole rows of per_warp points, the first row aligned to per_warp
    const int r_lo = h_lo / per_warp, r_hi = (h_hi + per_warp - 1) / per_warp;
    const int chunk_rows = (r_hi - r_lo + S - 1) / S;
    const int lo = max(h_lo, (r_lo + rank * chunk_rows) * per_warp);
    const int hi = min(h_hi, (r_lo + (rank + 1) * chunk_rows) * per_warp);
    const Cx* __restrict__ ps = psi_all + G.psi_off + i;   // point j at ps[j * I]
    const double* __restrict__ psi0 = gs_work + gs_off[G.cls];
    const int stride = kPopWarps * per_warp;
    double ovr = 0.0, ovi = 0.0, core = 0.0;
    for (int jb = (r_lo + rank * chunk_rows + warp) * per_warp; jb < hi; jb += kPopDepth * stride) {
        Cx v[kPopDepth];
        double p0[kPopDepth];
#pragma unroll
        for (int u = 0; u < kPopDepth; ++u) {
            const int j = jb + u * stride + jq;
            const bool ok = j >= lo && j < hi;
            v[u] = ok ? ps[(int64_t)j * I] : Cx{0, 0};
            p0[u] = ok ? psi0[j] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kPopDepth; ++u) {
            ovr = fma(p0[u], to_f64(v[u].x), ovr);
            ovi = fma(p0[u], to_f64(v[u].y), ovi);
        }
    }
    // the core rows of this chunk once more (from L1/L2): |psi|^2 only where it is summed
    const int k_lo = max(lo, c_lo), k_hi = min(hi, c_hi);
    for (int jb = (r_lo + rank * chunk_rows + warp) * per_warp; jb < k_hi; jb += stride) {
        const int j = jb + jq;
        if (j >= k_lo && j < k_hi) {
            const Cx v = ps[(int64_t)j * I];
            const double vr = to_f64(v.x), vi = to_f64(v.y);
            core = fma(vr, vr, fma(vi, vi, core));
        }
    }
    for (int o = I; o < kLanes; o <<= 1) {
        ovr += __shfl_xor_sync(0xffffffffu, ovr, o);
        ovi += __shfl_xor_sync(0xffffffffu, ovi, o);
        core += __shfl_xor_sync(0xffffffffu, core, o);
    }
    part[warp][0][lane] = ovr;
    part[warp][1][lane] = ovi;
    part[warp][2][lane] = core;
    __syncthreads();
    if (threadIdx.x < 3 * kLanes) {
        const int q = threadIdx.x / kLanes, l = threadIdx.x % kLanes;
        double t = 0.0;
        for (int w = 0; w < kPopWarps; ++w) t += part[w][q][l];
        cta_sum[q][l] = t;
    }
    cluster.sync();   // every CTA's partials are visible to the cluster
    if (rank == 0 && threadIdx.x < I) {
        double sr = 0.0, si = 0.0, sc = 0.0;
        for (int r = 0; r < S; ++r) {
            const double* rs = cluster.map_shared_rank(&cta_sum[0][0], r);
            sr += rs[0 * kLanes + i];
            si += rs[1 * kLanes + i];
            sc += rs[2 * kLanes + i];
        }
        const int64_t inst = slot_inst[G.slot0 + i];
        if (inst >= 0) {
            const double dx = C.dx;
            out[2 * inst] = (sr * sr + si * si) * (dx * dx);
            out[2 * inst + 1] = sc * dx;
        }
    }
    cluster.sync();   // the partials stay alive until CTA 0 has read them
}

cudaError_t launch_populations(int mixed, const GroupDesc* d_groups, int64_t n_groups, const ClassDesc* d_cls,
                               const int64_t* d_slot_inst, const void* d_psi, const double* d_gs_work,
                               const int64_t* d_gs_off, const int64_t* d_support, double r_core, double* out,
                               int sm_count, cudaStream_t st)
{
    if (n_groups == 0) return cudaSuccess;
    if (n_groups > (int64_t(1) << 27)) return cudaErrorInvalidValue;
    // CTAs per group: enough for about 8 resident CTAs of 8 warps per SM
    const int64_t want = (int64_t)std::max(sm_count, 1) * 8;
    const int S = (int)std::min<int64_t>(kPopMaxCluster, std::max<int64_t>(1, (want + n_groups - 1) / n_groups));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_groups * S));
    cfg.blockDim = dim3(kPopWarps * 32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (mixed)
        e = cudaLaunchKernelEx(&cfg, k_populations<float2>, d_groups, d_cls, d_slot_inst,
                               static_cast<const float2*>(d_psi), d_gs_work, d_gs_off, d_support, r_core, out);
    else
        e = cudaLaunchKernelEx(&cfg, k_populations<double2>, d_groups, d_cls, d_slot_inst,
                               static_cast<const double2*>(d_psi), d_gs_work, d_gs_off, d_support, r_core, out);
    if (e != cudaSuccess) return e;
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
