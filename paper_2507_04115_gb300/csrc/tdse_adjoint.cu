// Discrete adjoint of the FULL_CN propagation (FP64): the gradient of a loss L(d, a) with respect to
// every field sample E_n, exact for the discrete scheme (so it agrees with finite differences of
// the forward map).
//
// With lambda^n = 2 dL/d conj(psi^n) (dL = Re sum conj(lambda) dpsi), A_n = 1 + i h H(Ebar_n),
// B_n = 1 - i h H(Ebar_n) = conj(A_n) (H is real), M = diag(m):
//   forward   psi~^{n+1} = A_n^{-1} B_n psi^n,  psi^{n+1} = M psi~^{n+1}
//   backward  mu = B_n^{-1} M lambda^{n+1} = conj(A_n^{-1} conj(M lambda^{n+1}))
//             lambda^n = A_n mu + g^n = 2 mu - M lambda^{n+1} + g^n      (A_n + B_n = 2)
//             g^n_j = 2 dx (gd_n x_j + ga_n (dV_j + E_n)) psi^n_j
//   field     dL/dEbar_n = h sum_j x_j Im(conj(mu_j) (psi^n_j + psi~^{n+1}_j)), half to E_n and half
//             to E_{n+1}; dL/dE_n += ga_n dx sum_j |psi^n_j|^2 (the E_n in a_n)
// The solve with A_n reuses the forward kernel's segmented, halo-truncated Thomas sweep.
//
// Memory: the forward states are recomputed from checkpoints every K steps; within a checkpoint
// interval the pre-mask states psi~ are kept on a per-CTA tape.  One CTA owns a group for the whole
// call: first a forward pass writing the checkpoints (unless a checkpointed forward propagation has
// written them already, tdse_propagate_checkpointed), then the intervals from last to first
// (recompute the interval onto the tape, then sweep it backwards).
//
// Lane geometry (any group width I = 32/L, see GroupDesc): lane l of warp w holds instance l % I
// and sweeps segment sigma = w L + l / I over rows r = 0 .. m + 2K - 1 at points sigma m - K + r;
// rows outside the grid restart the recurrences at the walls, so every lane of a warp runs the
// same trip counts; the own segment is rows K .. K + m - 1.
#include "tdse_sched.cuh"

namespace tdse {

namespace {

struct AdjGeom {
    int N, I, i, q, base, nrows, K, m, s, e;
    double inv_beta, two_over_beta;
    Fma64 F;
    __device__ __forceinline__ int64_t at(int j) const { return (int64_t)j * I + i; }
};

__device__ __forceinline__ AdjGeom adj_geom(const GroupDesc& G, const ClassDesc& C)
{
    const double beta = C.beta;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    AdjGeom g;
    g.N = G.N;
    g.I = G.I;
    const int L = kLanes / G.I;
    g.i = lane & (G.I - 1);
    g.q = lane / G.I;
    g.K = G.K;
    g.m = G.m;
    const int sigma = w * L + g.q;
    g.nrows = w < G.P ? G.m + 2 * G.K : 0;
    g.base = sigma * G.m - G.K;
    g.s = w < G.P ? min(G.N, sigma * G.m) : G.N;
    g.e = w < G.P ? min(G.N, sigma * G.m + G.m) : G.N;
    g.inv_beta = 1.0 / beta;
    g.two_over_beta = 2.0 / beta;
    g.F = Fma64{C.one, C.nzero};
    return g;
}

// sum over the L lanes of an instance, then over the warps (warp 0 lanes q == 0 get the totals)
__device__ __forceinline__ ObsSums adj_reduce(ObsSums o, const AdjGeom& g, double* red, int P)
{
    for (int off = g.I; off < kLanes; off <<= 1) {
        o.n += __shfl_xor_sync(0xffffffffu, o.n, off);
        o.x += __shfl_xor_sync(0xffffffffu, o.x, off);
        o.v += __shfl_xor_sync(0xffffffffu, o.v, off);
    }
    return reduce_obs(o, red, P);
}

// Forward elimination of A y = v over the lane's sweep rows (v from `rhs`, a callable giving the
// right-hand side at point j), writing (gamma, D) rows to the scratch.  The right-hand side and the
// table entry are loaded two rows ahead of the recurrence (they do not depend on it).
template <class Rhs>
__device__ __forceinline__ void eliminate(const AdjGeom& g, double Eb, const double2* __restrict__ tab_ab2,
                                          double2* __restrict__ sc, Rhs rhs, double2* __restrict__ gout = nullptr)
{
    const int lane = threadIdx.x & 31;
    auto fetch = [&](int rr) {
        const int j = g.base + rr;
        return (rr < g.nrows && (unsigned)j < (unsigned)g.N) ? rhs(j) : make_double2(0.0, 0.0);
    };
    double cr = 0.0, ci = 0.0, Dr = 0.0, Di = 0.0;
    double2* r = sc;
    double2 va = fetch(0), vb = fetch(1);
    for (int rr = 0; rr < g.nrows; ++rr) {
        const double2 v = va;
        va = vb;
        vb = fetch(rr + 2);
        const int j = g.base + rr;
        const bool in = (unsigned)j < (unsigned)g.N;
        const int jc = min(max(j, 0), g.N - 1);
        const double2 t = __ldg(tab_ab2 + jc);
        const Fma64& F = g.F;
        const double Qr = F.add(ci, g.inv_beta);
        const double Qi = F.sub(fma(t.y, Eb, t.x), cr);
        const double inv = rcp_pos(fma(Qr, Qr, F.mul(Qi, Qi)));
        cr = in ? F.mul(Qi, inv) : 0.0;
        ci = in ? F.mul(Qr, inv) : 0.0;
        const double ur = F.sub(v.x, Di);
        const double ui = F.add(v.y, Dr);
        Dr = in ? fma(cr, ui, F.mul(ci, ur)) : 0.0;
        Di = in ? fma(ci, ui, F.mul(-cr, ur)) : 0.0;
        r[lane] = make_double2(cr, ci);
        r[kLanes + lane] = make_double2(Dr, Di);
        r += 2 * kLanes;
        if (gout) gout[rr * kLanes + lane] = make_double2(cr, ci);
    }
}

// The same elimination with the coefficients gamma of every sweep row given (written by the
// recomputation of this step, `eliminate` with gout): only the D recurrence is evaluated.  gamma
// depends on the step's field and the class only, so the result is bitwise that of `eliminate`.
template <class Rhs>
__device__ __forceinline__ void eliminate_given(const AdjGeom& g, const double2* __restrict__ gin,
                                                double2* __restrict__ sc, Rhs rhs)
{
    const int lane = threadIdx.x & 31;
    auto fetch = [&](int rr) {
        const int j = g.base + rr;
        return (rr < g.nrows && (unsigned)j < (unsigned)g.N) ? rhs(j) : make_double2(0.0, 0.0);
    };
    auto gam = [&](int rr) { return rr < g.nrows ? gin[rr * kLanes + lane] : make_double2(0.0, 0.0); };
    double Dr = 0.0, Di = 0.0;
    double2* r = sc;
    double2 va = fetch(0), vb = fetch(1);
    double2 ca = gam(0), cb = gam(1);
    for (int rr = 0; rr < g.nrows; ++rr) {
        const double2 v = va, c = ca;
        va = vb;
        vb = fetch(rr + 2);
        ca = cb;
        cb = gam(rr + 2);
        const int j = g.base + rr;
        const bool in = (unsigned)j < (unsigned)g.N;
        const Fma64& F = g.F;
        const double ur = F.sub(v.x, Di);
        const double ui = F.add(v.y, Dr);
        Dr = in ? fma(c.x, ui, F.mul(c.y, ur)) : 0.0;
        Di = in ? fma(c.y, ui, F.mul(-c.x, ur)) : 0.0;
        r[lane] = c;
        r[kLanes + lane] = make_double2(Dr, Di);
        r += 2 * kLanes;
    }
}

// Back substitution over rows nrows-1 .. K.  On the own segment's points, fetch(j) loads what the
// update needs (independent of Y, so it is issued one row ahead together with the next scratch
// row) and own(j, Yr, Yi, payload) consumes it.
template <class Fetch, class Own>
__device__ __forceinline__ void substitute(const AdjGeom& g, const double2* __restrict__ sc, Fetch fetch, Own own)
{
    const int lane = threadIdx.x & 31;
    auto is_own = [&](int rr) { return rr >= g.K && rr < g.K + g.m && g.base + rr < g.N; };
    using Payload = decltype(fetch(0));
    double Yr = 0.0, Yi = 0.0;
    if (g.nrows <= g.K) return;
    const double2* r = sc + (int64_t)(g.nrows - 1) * (2 * kLanes);
    double2 ga = r[lane], da = r[kLanes + lane];
    Payload pa{};
    if (is_own(g.nrows - 1)) pa = fetch(g.base + g.nrows - 1);
    for (int rr = g.nrows - 1; rr >= g.K; --rr) {
        const int j = g.base + rr;
        const double2 g2 = ga, d2 = da;
        const Payload pl = pa;
        r -= 2 * kLanes;
        if (rr - 1 >= g.K) {
            ga = r[lane];
            da = r[kLanes + lane];
            if (is_own(rr - 1)) pa = fetch(j - 1);
        }
        const double nr = fma(g2.x, Yr, fma(-g2.y, Yi, d2.x));
        const double ni = fma(g2.x, Yi, fma(g2.y, Yr, d2.y));
        Yr = j < g.N ? nr : 0.0;
        Yi = j < g.N ? ni : 0.0;
        if (is_own(rr)) own(j, Yr, Yi, pl);
    }
}

// One FULL_CN step on the work state ps (layout [N][I]); optionally stores the pre-mask state into
// tape.  Ends with a barrier so that the next step sees every segment's writes.
__device__ __forceinline__ void fwd_step(double2* __restrict__ ps, const AdjGeom& g, double Eb,
                                         const double2* __restrict__ tab_ab2, const double* __restrict__ tab_m,
                                         int jm_lo, int jm_hi, double2* __restrict__ sc, bool active,
                                         double2* __restrict__ tape, double2* __restrict__ gout = nullptr)
{
    eliminate(g, Eb, tab_ab2, sc, [&](int j) { return ld_cg(ps + g.at(j)); }, gout);
    __syncthreads();
    substitute(g, sc, [&](int j) { return ld_cg(ps + g.at(j)); }, [&](int j, double Yr, double Yi, const double2& old) {
        double2* pp = ps + g.at(j);
        double xr = fma(g.two_over_beta, Yr, -old.x);
        double xi = fma(g.two_over_beta, Yi, -old.y);
        if (tape) tape[g.at(j)] = active ? make_double2(xr, xi) : old;
        if (j < jm_lo || j > jm_hi) {
            const double mm = __ldg(tab_m + j);
            xr = g.F.mul(xr, mm);
            xi = g.F.mul(xi, mm);
        }
        if (active) *pp = make_double2(xr, xi);
    });
    __syncthreads();
}

__device__ __forceinline__ void copy_state(double2* __restrict__ dst, const double2* __restrict__ src, int64_t n)
{
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) dst[k] = ld_cg(src + k);
}

}  // namespace

__global__ void __launch_bounds__(512, 1)
k_adjoint_full_cn(const GroupDesc* __restrict__ groups, int64_t n_groups, const ClassDesc* __restrict__ cls,
                  const double* __restrict__ tab, const int64_t* __restrict__ slot_row,
                  const int64_t* __restrict__ slot_nt, const double2* __restrict__ psi0_all,
                  double2* __restrict__ lam_all, double2* __restrict__ ckpt_all, const int64_t* __restrict__ ckpt_off,
                  double2* __restrict__ work_all, double2* __restrict__ tape_all, double2* __restrict__ scratch_all,
                  int rows, int n_max, int kc, const double* __restrict__ E, const double* __restrict__ gd,
                  const double* __restrict__ ga, double* __restrict__ gE, int mask_on, int* __restrict__ busy,
                  int* __restrict__ progress, int have_ckpt, double2* __restrict__ gtape_all)
{
    extern __shared__ double red[];
    __shared__ int s_g;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int P = blockDim.x >> 5;
    double2* __restrict__ sc = scratch_all + ((int64_t)blockIdx.x * P + w) * rows * (2 * kLanes);
    double2* __restrict__ work = work_all + (int64_t)blockIdx.x * n_max * kLanes;
    double2* __restrict__ tape = tape_all + (int64_t)blockIdx.x * kc * n_max * kLanes;
    // gamma tape (optional): the elimination coefficients of every recomputed step, this warp's
    // rows at gtape + (n - na) * gstep + w * rows * 32
    const int64_t gstep = (int64_t)P * rows * kLanes;
    double2* __restrict__ gtape = gtape_all ? gtape_all + (int64_t)blockIdx.x * kc * gstep + (int64_t)w * rows * kLanes
                                            : nullptr;
    const int64_t whole = int64_t(1) << 40;   // one scheduling slice per group

    for (;;) {
        if (w == 0) {
            int k = 0;
            const int g = pick_group(groups, n_groups, busy, progress, 0, whole, (int)(whole >> 10), &k);
            if (lane == 0) s_g = g;
        }
        __syncthreads();
        const int gi = s_g;
        __threadfence();
        __syncthreads();
        if (gi < 0) break;

        const GroupDesc G = groups[gi];
        const ClassDesc C = cls[G.cls];
        const AdjGeom geo = adj_geom(G, C);
        const int N = G.N, L = kLanes / G.I;
        const int64_t slot = G.slot0 + geo.i;
        const int64_t nt = slot_nt[slot];
        const int64_t row = slot_row[slot];
        const int64_t nt_max = G.nt_max;
        const int64_t state = (int64_t)N * G.I;   // elements of one state of the group
        const double dx = C.dx, h = 2.0 * C.beta * dx * dx;   // h = dt/2 = 2 beta dx^2
        const double2* __restrict__ tab_ab2 = reinterpret_cast<const double2*>(tab + tab_ab(C));
        const double2* __restrict__ tab_xv2 = reinterpret_cast<const double2*>(tab + tab_xv(C));
        const double* __restrict__ tab_m = tab + tab_mk(C);
        const int jm_lo = mask_on ? C.jm_lo : 0;
        const int jm_hi = mask_on ? C.jm_hi : N - 1;
        double2* __restrict__ lam = lam_all + G.psi_off;
        double2* __restrict__ ck = ckpt_all + ckpt_off[gi];
        const int64_t n_int = (nt_max + kc - 1) / kc;   // checkpoint intervals

        // gE rows start at zero (the L lanes of an instance and the warps share the row)
        if (nt >= 0)
            for (int64_t n = w * L + geo.q; n <= nt; n += P * L) gE[row + n] = 0.0;

        // forward pass from psi^0, checkpoint every kc steps (skipped when a checkpointed forward
        // propagation already wrote them)
        if (!have_ckpt) {
            copy_state(work, psi0_all + G.psi_off, state);
            copy_state(ck, psi0_all + G.psi_off, state);
            __syncthreads();
            for (int64_t n = 0; n < nt_max; ++n) {
                const bool active = n < nt;
                const double Eb = active ? 0.5 * (E[row + n] + E[row + n + 1]) : 0.0;
                fwd_step(work, geo, Eb, tab_ab2, tab_m, jm_lo, jm_hi, sc, active, nullptr);
                if ((n + 1) % kc == 0 && n + 1 < nt_max) {
                    copy_state(ck + ((n + 1) / kc) * state, work, state);
                    __syncthreads();
                }
            }
        }
        for (int64_t k = threadIdx.x; k < state; k += blockDim.x) lam[k] = make_double2(0.0, 0.0);
        __syncthreads();

        // backward over the checkpoint intervals, last first
        for (int64_t c = n_int - 1; c >= 0; --c) {
            const int64_t na = c * kc, nb = min(nt_max, na + kc);
            const double2* __restrict__ cks = ck + c * state;
            copy_state(work, cks, state);
            __syncthreads();
            for (int64_t n = na; n < nb; ++n) {
                const bool active = n < nt;
                const double Eb = active ? 0.5 * (E[row + n] + E[row + n + 1]) : 0.0;
                fwd_step(work, geo, Eb, tab_ab2, tab_m, jm_lo, jm_hi, sc, active, tape + (n - na) * (int64_t)n_max * kLanes,
                         gtape ? gtape + (n - na) * gstep : nullptr);
            }
            for (int64_t n = nb - 1; n >= na; --n) {
                const bool term = (n + 1 == nt);     // this instance's last sample: lambda starts here
                const bool active = n < nt;
                const double2* __restrict__ pt1 = tape + (n - na) * (int64_t)n_max * kLanes;              // psi~^{n+1}
                const double2* __restrict__ pt0 = n > na ? tape + (n - na - 1) * (int64_t)n_max * kLanes : nullptr;
                double En = 0.0, En1 = 0.0, gdn = 0.0, gan = 0.0, gd1 = 0.0, ga1 = 0.0;
                if (active) {
                    En = E[row + n];
                    En1 = E[row + n + 1];
                    gdn = gd[row + n];
                    gan = ga[row + n];
                    gd1 = gd[row + n + 1];
                    ga1 = ga[row + n + 1];
                }
                // A: terminal adjoint lambda^{Nt} = g^{Nt}, own segment
                double norm_term = 0.0;
                if (term) {
                    for (int j = geo.s; j < geo.e; ++j) {
                        const double2 q = ld_cg(pt1 + geo.at(j));
                        const double mm = (j < jm_lo || j > jm_hi) ? __ldg(tab_m + j) : 1.0;
                        const double2 xv = __ldg(tab_xv2 + j);
                        const double pr = mm * q.x, pi = mm * q.y;
                        const double wgt = 2.0 * dx * fma(gd1, xv.x, ga1 * (xv.y + En1));
                        lam[geo.at(j)] = make_double2(wgt * pr, wgt * pi);
                        norm_term = fma(pr, pr, fma(pi, pi, norm_term));
                    }
                }
                __syncthreads();
                // B: solve A_n y = conj(M lambda^{n+1}) -- forward elimination over the sweep rows
                const double Eb = 0.5 * (En + En1);
                auto rhs_b = [&](int j) {
                    const double2 lv = ld_cg(lam + geo.at(j));
                    const double mm = (j < jm_lo || j > jm_hi) ? __ldg(tab_m + j) : 1.0;
                    return make_double2(mm * lv.x, -mm * lv.y);   // conj(M lambda)
                };
                if (gtape)   // A_n's coefficients as the recomputation of step n left them
                    eliminate_given(geo, gtape + (n - na) * gstep, sc, rhs_b);
                else
                    eliminate(geo, Eb, tab_ab2, sc, rhs_b);
                __syncthreads();
                // C: back substitution, mu = conj(y), lambda^n = 2 mu - M lambda^{n+1} + g^n, field gradient
                ObsSums o{0.0, 0.0, norm_term};
                // mu = conj(y) = (Y_r, -Y_i) / beta; the 1/beta is folded into the constants below:
                // 2 mu = tb (Y_r, -Y_i) with tb = 2/beta, and x Im(conj(mu)(psi + psi~)) sums
                // x (Y_r s_i + Y_i s_r) with the 1/beta applied to the total.  The local gradient
                // weight 2 dx (gd_n x_j + ga_n (dV_j + E_n)) = cx x_j + (cv dV_j + cE).
                const double tb = 2.0 * geo.inv_beta;
                const double cx = 2.0 * dx * gdn, cv = 2.0 * dx * gan, cE = cv * En;
                const Fma64& F = geo.F;
                struct Row {
                    double2 v, p0, p1, xv;
                };
                auto fetch = [&](int j) {
                    Row q;
                    q.v = ld_cg(lam + geo.at(j));                                  // lambda^{n+1}
                    q.p0 = pt0 ? ld_cg(pt0 + geo.at(j)) : ld_cg(cks + geo.at(j));  // psi~^n or psi^n
                    q.p1 = ld_cg(pt1 + geo.at(j));                                 // psi~^{n+1}
                    q.xv = __ldg(tab_xv2 + j);
                    return q;
                };
                substitute(geo, sc, fetch, [&](int j, double Yr, double Yi, const Row& q) {
                    double2* lp = lam + geo.at(j);
                    double2 v = q.v;     // M lambda^{n+1}
                    double2 p0 = q.p0;   // psi^n = M psi~^n (the checkpoint at the interval start)
                    if (j < jm_lo || j > jm_hi) {
                        const double mm = __ldg(tab_m + j);
                        v = make_double2(F.mul(mm, v.x), F.mul(mm, v.y));
                        if (pt0) p0 = make_double2(F.mul(mm, p0.x), F.mul(mm, p0.y));
                    }
                    const double2 p1 = q.p1;
                    const double2 xv = q.xv;
                    const double wgt = fma(cx, xv.x, fma(cv, xv.y, cE));
                    if (active)
                        *lp = make_double2(fma(tb, Yr, fma(wgt, p0.x, -v.x)), fma(-tb, Yi, fma(wgt, p0.y, -v.y)));
                    const double sr = F.add(p0.x, p1.x), si = F.add(p0.y, p1.y);
                    o.n = fma(xv.x, fma(Yr, si, F.mul(Yi, sr)), o.n);
                    o.x = fma(p0.x, p0.x, fma(p0.y, p0.y, o.x));
                });
                const ObsSums t = adj_reduce(o, geo, red, P);
                if (w == 0 && geo.q == 0) {
                    if (term) gE[row + nt] += ga1 * dx * t.v;
                    if (active) {
                        const double gbar = h * geo.inv_beta * t.n;
                        gE[row + n] += 0.5 * gbar + gan * dx * t.x;
                        gE[row + n + 1] += 0.5 * gbar;
                    }
                }
                __syncthreads();
            }
        }
        // an instance without steps: only the direct term of a_0 (the reduction runs for every lane
        // so that all threads meet the same barriers)
        {
            double s0 = 0.0;
            if (nt == 0) {
                const double2* p0 = have_ckpt ? ck : psi0_all + G.psi_off;   // psi^0
                for (int j = geo.s; j < geo.e; ++j) {
                    const double2 p = ld_cg(p0 + geo.at(j));
                    s0 = fma(p.x, p.x, fma(p.y, p.y, s0));
                }
            }
            const ObsSums t = adj_reduce(ObsSums{s0, 0.0, 0.0}, geo, red, P);
            if (w == 0 && geo.q == 0 && nt == 0) gE[row] = ga[row] * dx * t.n;
            __syncthreads();
        }

        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            *(volatile int*)(progress + gi) = 1;
            __threadfence();
            atomicExch(busy + gi, 0);
        }
    }
}

cudaError_t launch_adjoint_full_cn(const GroupDesc* d_groups, int64_t n_groups, int P, int ctas, const ClassDesc* d_cls,
                                   const double* d_tab, const int64_t* d_slot_row, const int64_t* d_slot_nt,
                                   const void* d_psi0, void* d_lam, void* d_ckpt, const int64_t* d_ckpt_off,
                                   void* d_work, void* d_tape, void* d_scratch, int rows, int n_max, int kc,
                                   const double* E, const double* gd, const double* ga, double* gE, int mask_on,
                                   int* d_busy, int* d_progress, cudaStream_t st, int have_ckpt, void* d_gtape)
{
    if (n_groups == 0 || ctas == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(d_busy, 0, sizeof(int) * n_groups, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d_progress, 0, sizeof(int) * n_groups, st);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)P * 3 * kLanes * sizeof(double);
    k_adjoint_full_cn<<<(unsigned)ctas, P * kLanes, smem, st>>>(
        d_groups, n_groups, d_cls, d_tab, d_slot_row, d_slot_nt, static_cast<const double2*>(d_psi0),
        static_cast<double2*>(d_lam), static_cast<double2*>(d_ckpt), d_ckpt_off, static_cast<double2*>(d_work),
        static_cast<double2*>(d_tape), static_cast<double2*>(d_scratch), rows, n_max, kc, E, gd, ga, gE, mask_on,
        d_busy, d_progress, have_ckpt, static_cast<double2*>(d_gtape));
    return cudaGetLastError();
}

}  // namespace tdse
