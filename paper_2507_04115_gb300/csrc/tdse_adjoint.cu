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
// interval the pre-mask states psi~ are kept on a per-CTA tape.  One CTA owns a group (32
// instances) for the whole call: first a forward pass writing the checkpoints, then the intervals
// from last to first (recompute the interval onto the tape, then sweep it backwards).
#include "tdse_sched.cuh"

namespace tdse {

namespace {

struct AdjGeom {
    int N, s, e, lo, hi;
    double beta, inv_beta, two_over_beta;
};

// One FULL_CN step on the work state ps (layout [N][32]); optionally stores the pre-mask state into
// tape.  Ends with a barrier so that the next step sees every segment's writes.
__device__ __forceinline__ void fwd_step(double2* __restrict__ ps, const AdjGeom& g, double Eb,
                                         const double2* __restrict__ tab_ab2, const double* __restrict__ tab_m,
                                         int jm_lo, int jm_hi, double2* __restrict__ sc, bool active,
                                         double2* __restrict__ tape)
{
    const int lane = threadIdx.x & 31;
    double cr = 0.0, ci = 0.0, Dr = 0.0, Di = 0.0;
    double2* r = sc;
    for (int j = g.lo; j < g.hi; ++j) {
        const double2 p = ld_cg(ps + (int64_t)j * kLanes + lane);
        const double2 t = __ldg(tab_ab2 + j);
        const double Qr = g.inv_beta + ci;
        const double Qi = fma(t.y, Eb, t.x) - cr;
        const double inv = rcp_pos(fma(Qr, Qr, Qi * Qi));
        cr = Qi * inv;
        ci = Qr * inv;
        const double ur = p.x - Di;
        const double ui = p.y + Dr;
        Dr = fma(cr, ui, ci * ur);
        Di = fma(ci, ui, -cr * ur);
        r[lane] = make_double2(cr, ci);
        r[kLanes + lane] = make_double2(Dr, Di);
        r += 2 * kLanes;
    }
    __syncthreads();
    double Yr = 0.0, Yi = 0.0;
    const double2* q = sc + (int64_t)(g.hi - 1 - g.lo) * (2 * kLanes);
    for (int j = g.hi - 1; j >= g.s; --j) {
        const double2 g2 = q[lane];
        const double2 d2 = q[kLanes + lane];
        q -= 2 * kLanes;
        const double nr = fma(g2.x, Yr, fma(-g2.y, Yi, d2.x));
        Yi = fma(g2.x, Yi, fma(g2.y, Yr, d2.y));
        Yr = nr;
        if (j < g.e) {
            double2* pp = ps + (int64_t)j * kLanes + lane;
            const double2 old = *pp;
            double xr = fma(g.two_over_beta, Yr, -old.x);
            double xi = fma(g.two_over_beta, Yi, -old.y);
            if (tape) tape[(int64_t)j * kLanes + lane] = active ? make_double2(xr, xi) : old;
            if (j < jm_lo || j > jm_hi) {
                const double mm = __ldg(tab_m + j);
                xr *= mm;
                xi *= mm;
            }
            if (active) *pp = make_double2(xr, xi);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void copy_state(double2* __restrict__ dst, const double2* __restrict__ src, int N)
{
    for (int64_t k = threadIdx.x; k < (int64_t)N * kLanes; k += blockDim.x) dst[k] = ld_cg(src + k);
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
                  int* __restrict__ progress)
{
    extern __shared__ double red[];
    __shared__ int s_g;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int P = blockDim.x >> 5;
    double2* __restrict__ sc = scratch_all + ((int64_t)blockIdx.x * P + w) * rows * (2 * kLanes);
    double2* __restrict__ work = work_all + (int64_t)blockIdx.x * n_max * kLanes;
    double2* __restrict__ tape = tape_all + (int64_t)blockIdx.x * kc * n_max * kLanes;
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
        const int N = G.N, Pg = G.P, K = G.K, m = G.m;
        const int64_t slot = G.slot0 + lane;
        const int64_t nt = slot_nt[slot];
        const int64_t row = slot_row[slot];
        const int64_t nt_max = G.nt_max;
        const double dx = C.dx, h = 2.0 * C.beta * dx * dx;   // h = dt/2 = 2 beta dx^2
        AdjGeom geo;
        geo.N = N;
        geo.s = w < Pg ? min(N, w * m) : N;
        geo.e = w < Pg ? min(N, geo.s + m) : N;
        geo.lo = w < Pg ? max(0, geo.s - K) : N;
        geo.hi = w < Pg ? min(N, geo.e + K) : N;
        geo.beta = C.beta;
        geo.inv_beta = 1.0 / C.beta;
        geo.two_over_beta = 2.0 / C.beta;
        const double2* __restrict__ tab_ab2 = reinterpret_cast<const double2*>(tab + tab_ab(C));
        const double2* __restrict__ tab_xv2 = reinterpret_cast<const double2*>(tab + tab_xv(C));
        const double* __restrict__ tab_m = tab + tab_mk(C);
        const int jm_lo = mask_on ? C.jm_lo : 0;
        const int jm_hi = mask_on ? C.jm_hi : N - 1;
        double2* __restrict__ lam = lam_all + G.psi_off;
        double2* __restrict__ ck = ckpt_all + ckpt_off[gi];
        const int64_t n_int = (nt_max + kc - 1) / kc;   // checkpoint intervals

        // gE rows start at zero
        if (nt >= 0)
            for (int64_t n = w; n <= nt; n += P) gE[row + n] = 0.0;

        // forward pass from psi^0, checkpoint every kc steps
        copy_state(work, psi0_all + G.psi_off, N);
        copy_state(ck, psi0_all + G.psi_off, N);
        __syncthreads();
        for (int64_t n = 0; n < nt_max; ++n) {
            const bool active = n < nt;
            const double Eb = active ? 0.5 * (E[row + n] + E[row + n + 1]) : 0.0;
            fwd_step(work, geo, Eb, tab_ab2, tab_m, jm_lo, jm_hi, sc, active, nullptr);
            if ((n + 1) % kc == 0 && n + 1 < nt_max) {
                copy_state(ck + ((n + 1) / kc) * (int64_t)N * kLanes, work, N);
                __syncthreads();
            }
        }
        for (int64_t k = threadIdx.x; k < (int64_t)N * kLanes; k += blockDim.x) lam[k] = make_double2(0.0, 0.0);
        __syncthreads();

        // backward over the checkpoint intervals, last first
        for (int64_t c = n_int - 1; c >= 0; --c) {
            const int64_t na = c * kc, nb = min(nt_max, na + kc);
            const double2* __restrict__ cks = ck + c * (int64_t)N * kLanes;
            copy_state(work, cks, N);
            __syncthreads();
            for (int64_t n = na; n < nb; ++n) {
                const bool active = n < nt;
                const double Eb = active ? 0.5 * (E[row + n] + E[row + n + 1]) : 0.0;
                fwd_step(work, geo, Eb, tab_ab2, tab_m, jm_lo, jm_hi, sc, active, tape + (n - na) * (int64_t)n_max * kLanes);
            }
            for (int64_t n = nb - 1; n >= na; --n) {
                const bool term = (n + 1 == nt);     // this lane's last sample: lambda starts here
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
                        const double2 q = ld_cg(pt1 + (int64_t)j * kLanes + lane);
                        const double mm = (j < jm_lo || j > jm_hi) ? __ldg(tab_m + j) : 1.0;
                        const double2 xv = __ldg(tab_xv2 + j);
                        const double pr = mm * q.x, pi = mm * q.y;
                        const double wgt = 2.0 * dx * fma(gd1, xv.x, ga1 * (xv.y + En1));
                        lam[(int64_t)j * kLanes + lane] = make_double2(wgt * pr, wgt * pi);
                        norm_term = fma(pr, pr, fma(pi, pi, norm_term));
                    }
                }
                __syncthreads();
                // B: solve A_n y = conj(M lambda^{n+1}) -- forward elimination over the halo range
                const double Eb = 0.5 * (En + En1);
                {
                    double cr = 0.0, ci = 0.0, Dr = 0.0, Di = 0.0;
                    double2* r = sc;
                    for (int j = geo.lo; j < geo.hi; ++j) {
                        const double2 lv = ld_cg(lam + (int64_t)j * kLanes + lane);
                        const double mm = (j < jm_lo || j > jm_hi) ? __ldg(tab_m + j) : 1.0;
                        const double vr = mm * lv.x, vi = -mm * lv.y;   // conj(M lambda)
                        const double2 t = __ldg(tab_ab2 + j);
                        const double Qr = geo.inv_beta + ci;
                        const double Qi = fma(t.y, Eb, t.x) - cr;
                        const double inv = rcp_pos(fma(Qr, Qr, Qi * Qi));
                        cr = Qi * inv;
                        ci = Qr * inv;
                        const double ur = vr - Di;
                        const double ui = vi + Dr;
                        Dr = fma(cr, ui, ci * ur);
                        Di = fma(ci, ui, -cr * ur);
                        r[lane] = make_double2(cr, ci);
                        r[kLanes + lane] = make_double2(Dr, Di);
                        r += 2 * kLanes;
                    }
                }
                __syncthreads();
                // C: back substitution, mu = conj(y), lambda^n = 2 mu - M lambda^{n+1} + g^n, field gradient
                ObsSums o{0.0, 0.0, norm_term};
                {
                    double Yr = 0.0, Yi = 0.0;
                    const double2* q = sc + (int64_t)(geo.hi - 1 - geo.lo) * (2 * kLanes);
                    for (int j = geo.hi - 1; j >= geo.s; --j) {
                        const double2 g2 = q[lane];
                        const double2 d2 = q[kLanes + lane];
                        q -= 2 * kLanes;
                        const double nr = fma(g2.x, Yr, fma(-g2.y, Yi, d2.x));
                        Yi = fma(g2.x, Yi, fma(g2.y, Yr, d2.y));
                        Yr = nr;
                        if (j < geo.e) {
                            const double mur = Yr * geo.inv_beta, mui = -Yi * geo.inv_beta;
                            const double mm = (j < jm_lo || j > jm_hi) ? __ldg(tab_m + j) : 1.0;
                            double2* lp = lam + (int64_t)j * kLanes + lane;
                            const double2 lv = *lp;
                            const double vr = mm * lv.x, vi = mm * lv.y;
                            double2 p0;
                            if (pt0) {
                                const double2 q0 = ld_cg(pt0 + (int64_t)j * kLanes + lane);
                                p0 = make_double2(mm * q0.x, mm * q0.y);
                            } else {
                                p0 = ld_cg(cks + (int64_t)j * kLanes + lane);
                            }
                            const double2 p1 = ld_cg(pt1 + (int64_t)j * kLanes + lane);
                            const double2 xv = __ldg(tab_xv2 + j);
                            const double wgt = 2.0 * dx * fma(gdn, xv.x, gan * (xv.y + En));
                            if (active)
                                *lp = make_double2(fma(2.0, mur, fma(wgt, p0.x, -vr)), fma(2.0, mui, fma(wgt, p0.y, -vi)));
                            const double sr = p0.x + p1.x, si = p0.y + p1.y;
                            o.n = fma(xv.x, fma(mur, si, -mui * sr), o.n);
                            o.x = fma(p0.x, p0.x, fma(p0.y, p0.y, o.x));
                        }
                    }
                }
                const ObsSums t = reduce_obs(o, red, P);
                if (w == 0) {
                    if (term) gE[row + nt] += ga1 * dx * t.v;
                    if (active) {
                        const double gbar = h * t.n;
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
                for (int j = geo.s; j < geo.e; ++j) {
                    const double2 p = ld_cg(psi0_all + G.psi_off + (int64_t)j * kLanes + lane);
                    s0 = fma(p.x, p.x, fma(p.y, p.y, s0));
                }
            }
            const ObsSums t = reduce_obs(ObsSums{s0, 0.0, 0.0}, red, P);
            if (w == 0 && nt == 0) gE[row] = ga[row] * dx * t.n;
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
                                   int* d_busy, int* d_progress, cudaStream_t st)
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
        d_busy, d_progress);
    return cudaGetLastError();
}

}  // namespace tdse
