// Real-time propagation kernels of libtdse (sm_103a): FULL_CN in FP64 and MIXED precision.
//
// Numerical scheme (one step t_n -> t_{n+1}, h = dt/2, Ebar = (E_n + E_{n+1})/2):
//   A = 1 + i h H(Ebar) = tridiag(-i beta, 1 + i s_j, -i beta),  beta = dt/(4 dx^2),
//   s_j = h (1/dx^2 + V_j + x_j Ebar);  psi^{n+1} = m (A^{-1}(1 - i h H) psi^n) = m (2 A^{-1} psi^n - psi^n)
// because (1 - i h H) = 2 - A.  So each step is one tridiagonal solve A y = psi^n (Thomas: forward
// elimination, back substitution) and a pointwise update -- no right-hand-side product.
//
// Parallel layout (lane-batched segmented Thomas):
//   * a group = 32 instances of one grid class, one per lane, so every warp instruction works on
//     32 independent systems (the FP64 pipe costs the same per warp instruction whatever the
//     number of active lanes, so full warps matter);
//   * a CTA of P warps owns one group at a time; warp w owns the grid segment [w m, (w+1) m);
//   * a segment's sweep starts K points before the segment and closes K points after it.  A is
//     strictly diagonally dominant with Re(pivot) >= 1, so both the forward coefficients and the
//     back substitution forget their starting values by a factor <= beta per point; K is chosen so
//     that beta^K < 1e-18, below double rounding.  The outermost segments use the exact walls.
//   * scheduling: a persistent grid of CTAs picks groups dynamically, one time slice (a few tens
//     of steps) at a time, always the free group with the most remaining slices.  A group is
//     claimed with an atomic compare-and-swap and released after its slice; a CTA that finds no
//     free unfinished group exits.  No CTA ever waits on another, so there is nothing to time out.
//     Dynamic slices balance the load when the number of groups is not a multiple of the SM count
//     (8192 instances = 256 groups on 152 SMs) and when groups have different lengths.
// HBM layouts: psi [group][j][lane] (16 B per point, a warp reads 512 contiguous bytes), scratch per
// CTA [warp][row][gamma | D][lane].
#include "tdse_device.cuh"
#include "tdse_internal.h"

namespace tdse {

namespace {

// Storage and arithmetic types per precision: FP64 keeps everything in double; MIXED keeps psi,
// the solve's right-hand side and back substitution, and the pointwise update in float, while the
// elimination recurrence (the pivots and gamma) and the observable sums stay in double.
template <bool kMixed> struct Prec;
template <> struct Prec<false> {
    using R = double;
    using C = double2;
};
template <> struct Prec<true> {
    using R = float;
    using C = float2;
};

__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

// double -> float on the integer pipe for values well inside float's normal range: on GB300 a
// hardware conversion costs as much as an FP64 multiply-add.  The 52-bit mantissa is rounded to 23
// bits to nearest (ties away from zero; a carry into the exponent is the correct result), so the
// rounding is unbiased -- truncation would perturb every step's elimination coefficients in the
// same direction and the error would grow linearly with the number of steps.  Values outside the
// range (including 0) take the hardware conversion.
__device__ __forceinline__ float d2f(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
    if (e - 897u < 253u) {
        const unsigned bits = ((unsigned)hi & 0x80000000u) | ((e - 896u) << 23) | (((unsigned)hi & 0xfffffu) << 3) |
                              (lo >> 29);
        return __uint_as_float(bits + ((lo >> 28) & 1u));
    }
    return __double2float_rn(x);
}

struct ObsSums {
    double n, x, v;
};

// Per-warp partial sums of |psi|^2, x |psi|^2 and dV/dx |psi|^2 combined over the CTA's warps
// through shared memory; warp 0 receives the totals (the barrier inside also orders the psi
// writes of the step before any read of the next one).
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

__device__ __forceinline__ int64_t group_slices(const GroupDesc& G, int64_t step_begin, int64_t step_end, int slice)
{
    const int64_t n_end = min(step_end, G.nt_max);
    if (n_end > step_begin) return (n_end - step_begin + slice - 1) / slice;
    return step_begin == 0 ? 1 : 0;   // only the initial observables
}

// Warp 0 picks and claims the free group with the most remaining slices; ties go to the group
// closest after this CTA's index (cyclically), so that CTAs starting together claim different
// groups instead of all racing for the same one.  Returns the group (its slice index in *k_out) or
// -1 when no free unfinished group is left.  Every failed claim means another CTA claimed a group,
// so the retries are bounded by the total number of claims.
__device__ int pick_group(const GroupDesc* groups, int64_t n_groups, int* busy, int* progress, int64_t step_begin,
                          int64_t step_end, int slice, int* k_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t me = (int64_t)blockIdx.x % n_groups;
    for (int64_t attempt = 0; attempt < 4 * n_groups + 64; ++attempt) {
        int64_t best_rem = 0, best_d = n_groups, best_g = -1;
        for (int64_t g = lane; g < n_groups; g += 32) {
            const int64_t rem = group_slices(groups[g], step_begin, step_end, slice) -
                                *(volatile int*)(progress + g);
            const int64_t dist = (g - me + n_groups) % n_groups;
            if (rem > 0 && *(volatile int*)(busy + g) == 0 && (rem > best_rem || (rem == best_rem && dist < best_d))) {
                best_rem = rem;
                best_d = dist;
                best_g = g;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t r2 = __shfl_xor_sync(0xffffffffu, best_rem, o);
            const int64_t d2 = __shfl_xor_sync(0xffffffffu, best_d, o);
            const int64_t g2 = __shfl_xor_sync(0xffffffffu, best_g, o);
            if (g2 >= 0 && (best_g < 0 || r2 > best_rem || (r2 == best_rem && d2 < best_d))) {
                best_rem = r2;
                best_d = d2;
                best_g = g2;
            }
        }
        if (best_g < 0) return -1;
        int got = 0, k = 0;
        if (lane == 0) {
            if (atomicCAS(busy + best_g, 0, 1) == 0) {
                __threadfence();   // acquire: the previous owner's psi writes precede its release
                k = *(volatile int*)(progress + best_g);
                if (k < group_slices(groups[best_g], step_begin, step_end, slice)) {
                    got = 1;
                } else {           // finished in the meantime: give it back
                    atomicExch(busy + best_g, 0);
                }
            }
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (got) {
            *k_out = k;
            return (int)best_g;
        }
    }
    return -1;
}

}  // namespace

template <bool kMixed>
__global__ void __launch_bounds__(512, 1)
k_propagate_full_cn(const GroupDesc* __restrict__ groups, int64_t n_groups, const ClassDesc* __restrict__ cls,
                    const double* __restrict__ tab, const int64_t* __restrict__ slot_row,
                    const int64_t* __restrict__ slot_nt, void* __restrict__ psi_raw, void* __restrict__ scratch_raw,
                    int rows, const double* __restrict__ E, double* __restrict__ d_out, double* __restrict__ a_out,
                    int64_t sample_base, int64_t step_begin, int64_t step_end, int slice, int mask_on,
                    int* __restrict__ busy, int* __restrict__ progress, int* __restrict__ status)
{
    using R = typename Prec<kMixed>::R;
    using Cx = typename Prec<kMixed>::C;
    extern __shared__ double red[];   // [P][3][32]
    __shared__ int s_g, s_k;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int P = blockDim.x >> 5;
    Cx* __restrict__ psi_all = static_cast<Cx*>(psi_raw);
    Cx* __restrict__ sc = static_cast<Cx*>(scratch_raw) + ((int64_t)blockIdx.x * P + w) * rows * (2 * kLanes);

    for (;;) {
        if (w == 0) {
            int k = 0;
            const int g = pick_group(groups, n_groups, busy, progress, step_begin, step_end, slice, &k);
            if (lane == 0) {
                s_g = g;
                s_k = k;
            }
        }
        __syncthreads();
        const int g = s_g;
        const int kslice = s_k;
        __threadfence();   // order this CTA's reads of the group's psi after the claim
        __syncthreads();   // s_g / s_k are rewritten only after every warp has read them
        if (g < 0) break;

        const GroupDesc G = groups[g];
        const ClassDesc C = cls[G.cls];
        const int N = G.N, Pg = G.P, K = G.K, m = G.m;
        const int64_t slot = G.slot0 + lane;
        const int64_t nt = slot_nt[slot];   // -1 for padding lanes
        const int64_t row = slot_row[slot];
        const double beta = C.beta;
        const double inv_beta = 1.0 / beta;
        const R two_over_beta = (R)(2.0 / beta);
        const double dx = C.dx;
        // warps beyond the group's segment count own an empty segment
        const int s = w < Pg ? min(N, w * m) : N;
        const int e = w < Pg ? min(N, s + m) : N;
        const int lo = w < Pg ? max(0, s - K) : N;
        const int hi = w < Pg ? min(N, e + K) : N;
        Cx* __restrict__ ps = psi_all + G.psi_off;
        const double2* __restrict__ tab_ab2 = reinterpret_cast<const double2*>(tab + tab_ab(C));
        const double2* __restrict__ tab_xv2 = reinterpret_cast<const double2*>(tab + tab_xv(C));
        const double* __restrict__ tab_m = tab + tab_mk(C);
        const int jm_lo = mask_on ? C.jm_lo : 0;
        const int jm_hi = mask_on ? C.jm_hi : N - 1;
        const int64_t n_end = min(step_end, G.nt_max);
        const int64_t n0 = step_begin + (int64_t)kslice * slice;
        const int64_t n1 = min(n_end, n0 + slice);

        if (kslice == 0 && step_begin == 0) {
            // observables of the initial state
            ObsSums o{0.0, 0.0, 0.0};
            for (int j = s; j < e; ++j) {
                const Cx p = ld_cg(ps + (int64_t)j * kLanes + lane);
                const double rho = fma((double)p.x, (double)p.x, (double)p.y * (double)p.y);
                const double2 xv = __ldg(tab_xv2 + j);
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

        for (int64_t n = n0; n < n1; ++n) {
            const bool active = n < nt;
            double En = 0.0, En1 = 0.0;
            if (active) {
                En = E[row + n - sample_base];
                En1 = E[row + n + 1 - sample_base];
            }
            const double Eb = 0.5 * (En + En1);

            // Forward elimination over [lo, hi) in scaled variables: Q = q/beta with
            // q_j = 1 + i s_j + beta^2 g_{j-1} the Thomas pivot, gamma = i beta g = i conj(Q)/|Q|^2,
            // D = beta d = -i gamma u with u = psi + i D_{j-1}.  Tables hold s_j/beta split as
            // (S0_j, Xh_j)/beta; Re Q = 1/beta + Im gamma_{j-1}, Im Q = s_j/beta - Re gamma_{j-1}.
            // The recurrence for Q and gamma always runs in double.
            double cr = 0.0, ci = 0.0;
            R Dr = 0, Di = 0;
            {
                const Cx* pj = ps + (int64_t)lo * kLanes + lane;
                Cx pa = lo < hi ? ld_cg(pj) : mk(R(0), R(0));
                Cx pb = lo + 1 < hi ? ld_cg(pj + kLanes) : mk(R(0), R(0));
                Cx* r = sc;
#pragma unroll 2
                for (int j = lo; j < hi; ++j) {
                    const Cx p = pa;
                    pa = pb;
                    if (j + 2 < hi) pb = ld_cg(ps + (int64_t)(j + 2) * kLanes + lane);
                    const double2 t = __ldg(tab_ab2 + j);
                    const double Qr = inv_beta + ci;
                    const double Qi = fma(t.y, Eb, t.x) - cr;
                    const double inv = rcp_pos(fma(Qr, Qr, Qi * Qi));
                    cr = Qi * inv;
                    ci = Qr * inv;
                    R gr, gi;
                    if constexpr (kMixed) {
                        gr = d2f(cr);
                        gi = d2f(ci);
                    } else {
                        gr = cr;
                        gi = ci;
                    }
                    const R ur = p.x - Di;
                    const R ui = p.y + Dr;
                    Dr = fma(gr, ui, gi * ur);
                    Di = fma(gi, ui, -gr * ur);
                    r[lane] = mk(gr, gi);
                    r[kLanes + lane] = mk(Dr, Di);
                    r += 2 * kLanes;
                }
            }
            __syncthreads();   // every read of psi^n (own segment and halos) precedes any write of psi^{n+1}

            // Back substitution Y_j = D_j + gamma_j Y_{j+1} (Y = beta y), seeded with 0 at hi (exact at
            // the wall), then psi^{n+1}_j = m_j (2 Y_j / beta - psi^n_j) on the own segment.
            R Yr = 0, Yi = 0;
            ObsSums o{0.0, 0.0, 0.0};
            {
                const Cx* r = sc + (int64_t)(hi - 1 - lo) * (2 * kLanes);
                for (int j = hi - 1; j >= e; --j) {
                    const Cx g2 = r[lane];
                    const Cx d2 = r[kLanes + lane];
                    r -= 2 * kLanes;
                    const R nr = fma(g2.x, Yr, fma(-g2.y, Yi, d2.x));
                    Yi = fma(g2.x, Yi, fma(g2.y, Yr, d2.y));
                    Yr = nr;
                }
                // own segment, with the scratch row and the old psi prefetched two points ahead
                Cx ga = mk(R(0), R(0)), da = ga, gb = ga, db = ga, pa = ga, pb = ga;
                if (e - 1 >= s) {
                    ga = r[lane];
                    da = r[kLanes + lane];
                    pa = ld_cg(ps + (int64_t)(e - 1) * kLanes + lane);
                }
                if (e - 2 >= s) {
                    gb = r[-2 * kLanes + lane];
                    db = r[-kLanes + lane];
                    pb = ld_cg(ps + (int64_t)(e - 2) * kLanes + lane);
                }
                // MIXED: |psi|^2 and its weighted sums run in float over blocks of 8 points, each
                // block total is added to the double accumulators
                R fn = 0, fx = 0, fv = 0;
                int blk = 0;
#pragma unroll 2
                for (int j = e - 1; j >= s; --j) {
                    const Cx g2 = ga, d2 = da, old = pa;
                    ga = gb;
                    da = db;
                    pa = pb;
                    if (j - 2 >= s) {
                        gb = r[-4 * kLanes + lane];
                        db = r[-3 * kLanes + lane];
                        pb = ld_cg(ps + (int64_t)(j - 2) * kLanes + lane);
                    }
                    r -= 2 * kLanes;
                    const R nr = fma(g2.x, Yr, fma(-g2.y, Yi, d2.x));
                    Yi = fma(g2.x, Yi, fma(g2.y, Yr, d2.y));
                    Yr = nr;
                    R xr = fma(two_over_beta, Yr, -old.x);
                    R xi = fma(two_over_beta, Yi, -old.y);
                    if (j < jm_lo || j > jm_hi) {
                        const R mm = (R)__ldg(tab_m + j);
                        xr *= mm;
                        xi *= mm;
                    }
                    if (active) ps[(int64_t)j * kLanes + lane] = mk(xr, xi);
                    const R rho = fma(xr, xr, xi * xi);
                    const double2 xv = __ldg(tab_xv2 + j);
                    if constexpr (kMixed) {
                        fn += rho;
                        fx = fma((R)xv.x, rho, fx);
                        fv = fma((R)xv.y, rho, fv);
                        if (++blk == 8) {
                            o.n += (double)fn;
                            o.x += (double)fx;
                            o.v += (double)fv;
                            fn = fx = fv = 0;
                            blk = 0;
                        }
                    } else {
                        o.n += rho;
                        o.x = fma(xv.x, rho, o.x);
                        o.v = fma(xv.y, rho, o.v);
                    }
                }
                if constexpr (kMixed) {
                    o.n += (double)fn;
                    o.x += (double)fx;
                    o.v += (double)fv;
                }
            }
            const ObsSums t = reduce_obs(o, red, P);   // its barrier also orders this step's psi writes
            if (w == 0 && active) {
                const int64_t kk = row + n + 1 - sample_base;
                d_out[kk] = t.x * dx;
                a_out[kk] = fma(En1, t.n, t.v) * dx;
                // the norm never grows in exact arithmetic (unitary step, mask <= 1); the allowance
                // covers rounding: 1e-6 in FP64, 1e-3 in MIXED where float psi random-walks ~1e-5
                if (!(t.n * dx <= (kMixed ? 1.0 + 1e-3 : 1.0 + 1e-6))) status[slot] = 1;
            }
        }

        // release the group: its psi writes become visible before the next owner's claim
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            *(volatile int*)(progress + g) = kslice + 1;
            __threadfence();
            atomicExch(busy + g, 0);
        }
    }
}

// NUMEROV_SPLIT step (the paper's three substeps, Sec. 4.2, Eqs. "CN - step 4/2/3"):
//   psi1 = (M2 - i h K) psi,  psi2 = (M2 + i h K)^{-1} psi1,  psi3_j = exp(-i dt E_n x_j) psi2_j,
// with K = -Delta2/2 + M2 V, M2 = tridiag(1, 10, 1)/12, h = dt/2.  Since A + B = 2 M2 for
// A = M2 + i h K and B = M2 - i h K, psi2 = 2 A^{-1} (M2 psi) - psi: one solve with the
// time-independent A, whose LU factors (W = 1/pivot folded with the 1/12 of M2, L, C) are tabulated
// once per class in double.  Forward d_j = W_j (psi_{j-1} + 10 psi_j + psi_{j+1}) - L_j d_{j-1},
// backward y_j = d_j - C_j y_{j+1}.  Segments start their sweeps K points early / close K points
// late with the exact factors; both recurrences forget their truncated start by max|L|, max|C| per
// point, and K is chosen from that bound.  Then psi^{n+1} = m exp(-i dt E_n x) (2y - psi).
// The phase exp(-i dt E_n x_j) runs as a complex rotation from the segment end, re-seeded from
// sincos every 64 points (double) or 8 points (float).
template <bool kMixed>
__global__ void __launch_bounds__(512, 1)
k_propagate_numerov(const GroupDesc* __restrict__ groups, int64_t n_groups, const ClassDesc* __restrict__ cls,
                    const double* __restrict__ tab, const int64_t* __restrict__ slot_row,
                    const int64_t* __restrict__ slot_nt, void* __restrict__ psi_raw, void* __restrict__ scratch_raw,
                    int rows, const double* __restrict__ E, double* __restrict__ d_out, double* __restrict__ a_out,
                    int64_t sample_base, int64_t step_begin, int64_t step_end, int slice, int mask_on, double dt,
                    int* __restrict__ busy, int* __restrict__ progress, int* __restrict__ status)
{
    using R = typename Prec<kMixed>::R;
    using Cx = typename Prec<kMixed>::C;
    extern __shared__ double red[];   // [P][3][32]
    __shared__ int s_g, s_k;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int P = blockDim.x >> 5;
    Cx* __restrict__ psi_all = static_cast<Cx*>(psi_raw);
    // scratch rows: d_j only (one complex per row per lane)
    Cx* __restrict__ sc = static_cast<Cx*>(scratch_raw) + ((int64_t)blockIdx.x * P + w) * rows * (2 * kLanes);

    for (;;) {
        if (w == 0) {
            int k = 0;
            const int g = pick_group(groups, n_groups, busy, progress, step_begin, step_end, slice, &k);
            if (lane == 0) {
                s_g = g;
                s_k = k;
            }
        }
        __syncthreads();
        const int g = s_g;
        const int kslice = s_k;
        __threadfence();
        __syncthreads();
        if (g < 0) break;

        const GroupDesc G = groups[g];
        const ClassDesc C = cls[G.cls];
        const int N = G.N, Pg = G.P, K = G.K, m = G.m;
        const int64_t slot = G.slot0 + lane;
        const int64_t nt = slot_nt[slot];
        const int64_t row = slot_row[slot];
        const double dx = C.dx;
        const int s = w < Pg ? min(N, w * m) : N;
        const int e = w < Pg ? min(N, s + m) : N;
        const int lo = w < Pg ? max(0, s - K) : N;
        const int hi = w < Pg ? min(N, e + K) : N;
        Cx* __restrict__ ps = psi_all + G.psi_off;
        const double2* __restrict__ tab_xv2 = reinterpret_cast<const double2*>(tab + tab_xv(C));
        const double* __restrict__ tab_m = tab + tab_mk(C);
        const double2* __restrict__ tW = reinterpret_cast<const double2*>(tab + tab_nw(C));
        const double2* __restrict__ tL = reinterpret_cast<const double2*>(tab + tab_nl(C));
        const double2* __restrict__ tC = reinterpret_cast<const double2*>(tab + tab_nc(C));
        const float2* __restrict__ tF = reinterpret_cast<const float2*>(tab + tab_nf(C));
        const int jm_lo = mask_on ? C.jm_lo : 0;
        const int jm_hi = mask_on ? C.jm_hi : N - 1;
        const int64_t n_end = min(step_end, G.nt_max);
        const int64_t n0 = step_begin + (int64_t)kslice * slice;
        const int64_t n1 = min(n_end, n0 + slice);
        const double x0 = -0.5 * (N - 1) * dx;

        if (kslice == 0 && step_begin == 0) {
            ObsSums o{0.0, 0.0, 0.0};
            for (int j = s; j < e; ++j) {
                const Cx p = ld_cg(ps + (int64_t)j * kLanes + lane);
                const double rho = fma((double)p.x, (double)p.x, (double)p.y * (double)p.y);
                const double2 xv = __ldg(tab_xv2 + j);
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

        for (int64_t n = n0; n < n1; ++n) {
            const bool active = n < nt;
            double En = 0.0, En1 = 0.0;
            if (active) {
                En = E[row + n - sample_base];
                En1 = E[row + n + 1 - sample_base];
            }

            // forward: d_j = W_j r_j - L_j d_{j-1}, r_j = psi_{j-1} + 10 psi_j + psi_{j+1}
            {
                const Cx zero = mk(R(0), R(0));
                Cx pm = lo > 0 && lo < hi ? ld_cg(ps + (int64_t)(lo - 1) * kLanes + lane) : zero;
                Cx pc = lo < hi ? ld_cg(ps + (int64_t)lo * kLanes + lane) : zero;
                Cx pn = lo + 1 < N && lo < hi ? ld_cg(ps + (int64_t)(lo + 1) * kLanes + lane) : zero;
                R dr = 0, di = 0;
                Cx* r = sc;
#pragma unroll 2
                for (int j = lo; j < hi; ++j) {
                    const Cx nx = (j + 2 < N && j + 1 < hi) ? ld_cg(ps + (int64_t)(j + 2) * kLanes + lane) : zero;
                    const R rr = fma(R(10), pc.x, pm.x + pn.x);
                    const R ri = fma(R(10), pc.y, pm.y + pn.y);
                    R wr, wi, lr, li;
                    if constexpr (kMixed) {
                        const float2 fw = __ldg(tF + 3 * j), fl = __ldg(tF + 3 * j + 1);
                        wr = fw.x; wi = fw.y; lr = fl.x; li = fl.y;
                    } else {
                        const double2 tw = __ldg(tW + j), tl = __ldg(tL + j);
                        wr = tw.x; wi = tw.y; lr = tl.x; li = tl.y;
                    }
                    const R nr = fma(wr, rr, fma(-wi, ri, fma(-lr, dr, li * di)));
                    const R ni = fma(wr, ri, fma(wi, rr, fma(-lr, di, -li * dr)));
                    dr = nr;
                    di = ni;
                    r[lane] = mk(dr, di);
                    r += 2 * kLanes;
                    pm = pc;
                    pc = pn;
                    pn = nx;
                }
            }
            __syncthreads();

            // backward: y_j = d_j - C_j y_{j+1}; psi^{n+1}_j = m_j phase_j (2 y_j - psi^n_j)
            ObsSums o{0.0, 0.0, 0.0};
            {
                R yr = 0, yi = 0;
                const Cx* r = sc + (int64_t)(hi - 1 - lo) * (2 * kLanes);
                for (int j = hi - 1; j >= e; --j) {
                    const Cx d2 = r[0 + lane];
                    r -= 2 * kLanes;
                    R cr_, ci_;
                    if constexpr (kMixed) {
                        const float2 fc = __ldg(tF + 3 * j + 2);
                        cr_ = fc.x; ci_ = fc.y;
                    } else {
                        const double2 tc = __ldg(tC + j);
                        cr_ = tc.x; ci_ = tc.y;
                    }
                    const R nr = fma(-cr_, yr, fma(ci_, yi, d2.x));
                    yi = fma(-cr_, yi, fma(-ci_, yr, d2.y));
                    yr = nr;
                }
                // phase rotation per point: exp(+i dt E_n dx) steps x_j down by dx
                R wr_, wi_;
                if constexpr (kMixed) {
                    sincosf((float)(dt * En * dx), &wi_, &wr_);
                } else {
                    sincos(dt * En * dx, &wi_, &wr_);
                }
                const R mdtE = (R)(-dt * En);
                const R x0r = (R)x0, dxr = (R)dx;
                R phr = 1, phi = 0;
                const int reseed = kMixed ? 8 : 64;
                R fn = 0, fx = 0, fv = 0;
                int blk = 0;
                for (int j = e - 1; j >= s; --j) {
                    const Cx d2 = r[lane];
                    r -= 2 * kLanes;
                    R cr_, ci_;
                    if constexpr (kMixed) {
                        const float2 fc = __ldg(tF + 3 * j + 2);
                        cr_ = fc.x; ci_ = fc.y;
                    } else {
                        const double2 tc = __ldg(tC + j);
                        cr_ = tc.x; ci_ = tc.y;
                    }
                    const R nr = fma(-cr_, yr, fma(ci_, yi, d2.x));
                    yi = fma(-cr_, yi, fma(-ci_, yr, d2.y));
                    yr = nr;
                    if (((e - 1 - j) % reseed) == 0) {
                        if constexpr (kMixed) {
                            sincosf(mdtE * fmaf((float)j, dxr, x0r), &phi, &phr);
                        } else {
                            sincos(-dt * En * (x0 + j * dx), &phi, &phr);
                        }
                    }
                    const Cx old = ld_cg(ps + (int64_t)j * kLanes + lane);
                    const R tr = fma(R(2), yr, -old.x);
                    const R ti = fma(R(2), yi, -old.y);
                    R xr = fma(tr, phr, -ti * phi);
                    R xi = fma(tr, phi, ti * phr);
                    // next point (x smaller by dx): phase times exp(+i dt E dx)
                    const R qr = fma(phr, wr_, -phi * wi_);
                    phi = fma(phr, wi_, phi * wr_);
                    phr = qr;
                    if (j < jm_lo || j > jm_hi) {
                        const R mm = (R)__ldg(tab_m + j);
                        xr *= mm;
                        xi *= mm;
                    }
                    if (active) ps[(int64_t)j * kLanes + lane] = mk(xr, xi);
                    const R rho = fma(xr, xr, xi * xi);
                    const double2 xv = __ldg(tab_xv2 + j);
                    if constexpr (kMixed) {
                        fn += rho;
                        fx = fma((R)xv.x, rho, fx);
                        fv = fma((R)xv.y, rho, fv);
                        if (++blk == 8) {
                            o.n += (double)fn;
                            o.x += (double)fx;
                            o.v += (double)fv;
                            fn = fx = fv = 0;
                            blk = 0;
                        }
                    } else {
                        o.n += rho;
                        o.x = fma(xv.x, rho, o.x);
                        o.v = fma(xv.y, rho, o.v);
                    }
                }
                if constexpr (kMixed) {
                    o.n += (double)fn;
                    o.x += (double)fx;
                    o.v += (double)fv;
                }
            }
            const ObsSums t = reduce_obs(o, red, P);
            if (w == 0 && active) {
                const int64_t kk = row + n + 1 - sample_base;
                d_out[kk] = t.x * dx;
                a_out[kk] = fma(En1, t.n, t.v) * dx;
                if (!(t.n * dx <= (kMixed ? 1.0 + 1e-3 : 1.0 + 1e-6))) status[slot] = 1;
            }
        }

        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            *(volatile int*)(progress + g) = kslice + 1;
            __threadfence();
            atomicExch(busy + g, 0);
        }
    }
}

cudaError_t launch_propagate_numerov(int mixed, const GroupDesc* d_groups, int64_t n_groups, int P, int ctas,
                                     const ClassDesc* d_cls, const double* d_tab, const int64_t* d_slot_row,
                                     const int64_t* d_slot_nt, void* d_psi, void* d_scratch, int rows,
                                     const double* E, double* d_out, double* a_out, int64_t sample_base,
                                     int64_t step_begin, int64_t step_end, int slice, int mask_on, double dt,
                                     int* d_busy, int* d_progress, int* d_status, cudaStream_t st)
{
    if (n_groups == 0 || ctas == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(d_busy, 0, sizeof(int) * n_groups, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d_progress, 0, sizeof(int) * n_groups, st);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)P * 3 * kLanes * sizeof(double);
    if (mixed)
        k_propagate_numerov<true><<<(unsigned)ctas, P * kLanes, smem, st>>>(
            d_groups, n_groups, d_cls, d_tab, d_slot_row, d_slot_nt, d_psi, d_scratch, rows, E, d_out, a_out,
            sample_base, step_begin, step_end, slice, mask_on, dt, d_busy, d_progress, d_status);
    else
        k_propagate_numerov<false><<<(unsigned)ctas, P * kLanes, smem, st>>>(
            d_groups, n_groups, d_cls, d_tab, d_slot_row, d_slot_nt, d_psi, d_scratch, rows, E, d_out, a_out,
            sample_base, step_begin, step_end, slice, mask_on, dt, d_busy, d_progress, d_status);
    return cudaGetLastError();
}

cudaError_t launch_propagate_full_cn(int mixed, const GroupDesc* d_groups, int64_t n_groups, int P, int ctas,
                                     const ClassDesc* d_cls, const double* d_tab, const int64_t* d_slot_row,
                                     const int64_t* d_slot_nt, void* d_psi, void* d_scratch, int rows,
                                     const double* E, double* d_out, double* a_out, int64_t sample_base,
                                     int64_t step_begin, int64_t step_end, int slice, int mask_on, int* d_busy,
                                     int* d_progress, int* d_status, cudaStream_t st)
{
    if (n_groups == 0 || ctas == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(d_busy, 0, sizeof(int) * n_groups, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d_progress, 0, sizeof(int) * n_groups, st);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)P * 3 * kLanes * sizeof(double);
    if (mixed) {
        k_propagate_full_cn<true><<<(unsigned)ctas, P * kLanes, smem, st>>>(
            d_groups, n_groups, d_cls, d_tab, d_slot_row, d_slot_nt, d_psi, d_scratch, rows, E, d_out, a_out,
            sample_base, step_begin, step_end, slice, mask_on, d_busy, d_progress, d_status);
    } else {
        k_propagate_full_cn<false><<<(unsigned)ctas, P * kLanes, smem, st>>>(
            d_groups, n_groups, d_cls, d_tab, d_slot_row, d_slot_nt, d_psi, d_scratch, rows, E, d_out, a_out,
            sample_base, step_begin, step_end, slice, mask_on, d_busy, d_progress, d_status);
    }
    return cudaGetLastError();
}

int propagate_max_ctas_per_sm(int mixed, int P)
{
    int n = 0;
    const size_t smem = (size_t)P * 3 * kLanes * sizeof(double);
    const cudaError_t e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_propagate_full_cn<true>, P * kLanes, smem)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_propagate_full_cn<false>, P * kLanes, smem);
    if (e != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace tdse
