// Time-dependent electron energy distribution (Sec. 6.1): for every instance state psi and every
// energy E_k of a grid,
//     P(E_k) = N_eps eps^2 || (E_k - H0 - i eps)^{-1} psi ||^2 = (eps / pi) || y ||^2,
//     ((E_k - i eps) M - K) y = M psi,   || y ||^2 = sum_j |y_j|^2 dx,
// with (M, K) = (1, -Delta2/2 + V) for FULL_CN and (M2, -Delta2/2 + M2 V) for NUMEROV_SPLIT (the
// inversion uses each scheme's own representation of H0 = M^{-1} K).  Each system is solved by the
// Thomas algorithm over the whole grid: the matrix is not diagonally dominant (E_k lies inside the
// spectrum of H0), so the segmented halo sweeps of the propagation do not apply.  No pivot comes
// near zero: for FULL_CN each pivot is z - H_jj - b^2 / (previous pivot) with b = 1/(2 dx^2)
// real, so Im(pivot) <= -eps by induction; on the Numerov pencil the first pivot has
// Im = -(10/12) eps and, on the grids checked, none rises above that.
//
// The pivots depend on the class and the energy only, not on psi, so they are computed once:
//   k_ed_pivots  one lane per (class, energy): w_j = b_j - a_j c'_{j-1}, stores 1/w_j and
//                c'_j = c_j / w_j, layout [class][j][energy] (32 lanes read 32 consecutive energies);
//   k_ed_solve   one warp per (instance, block of 32 energies), one lane per energy:
//                d'_j = (r_j - a_j d'_{j-1}) / w_j forward (r = M psi), y_j = d'_j - c'_j y_{j+1}
//                backward, summing |y_j|^2; d' rows go to a per-warp scratch [j][lane].
// Work per point of a (instance, energy) solve: 13 FP64 operations (the pivot work is amortised
// over the class's instances).
#include "tdse_sched.cuh"

namespace tdse {

namespace {

// Sub-diagonal, diagonal and super-diagonal of (z M - K) at point j (z = E - i eps), FULL_CN or
// NUMEROV_SPLIT; V from the class table.
struct EdRow {
    double2 a, b, c;
};

__device__ __forceinline__ EdRow ed_row(int scheme, double zr, double zi, double inv_dx2, const double* __restrict__ V,
                                        int j, int N)
{
    EdRow r;
    if (scheme == 0) {
        r.a = make_double2(j > 0 ? 0.5 * inv_dx2 : 0.0, 0.0);
        r.c = make_double2(j < N - 1 ? 0.5 * inv_dx2 : 0.0, 0.0);
        r.b = make_double2(zr - (inv_dx2 + V[j]), zi);
    } else {
        const double k12 = 1.0 / 12.0;
        r.a = j > 0 ? make_double2(fma(zr, k12, 0.5 * inv_dx2 - V[j - 1] * k12), zi * k12) : make_double2(0.0, 0.0);
        r.c = j < N - 1 ? make_double2(fma(zr, k12, 0.5 * inv_dx2 - V[j + 1] * k12), zi * k12) : make_double2(0.0, 0.0);
        r.b = make_double2(fma(zr, 10.0 * k12, -(inv_dx2 + 10.0 * k12 * V[j])), zi * (10.0 * k12));
    }
    return r;
}

__device__ __forceinline__ double2 cmul(double2 x, double2 y)
{
    return make_double2(fma(x.x, y.x, -x.y * y.y), fma(x.x, y.y, x.y * y.x));
}

// 1/w for w with |w| bounded away from zero (|Im w| >= eps)
__device__ __forceinline__ double2 cinv(double2 w)
{
    const double r = rcp_pos(fma(w.x, w.x, w.y * w.y));
    return make_double2(w.x * r, -w.y * r);
}

__global__ void k_ed_pivots(const ClassDesc* __restrict__ cls, int n_cls, const double* __restrict__ tab,
                            const double* __restrict__ E_grid, int nE, int nE_pad, double eps, int scheme,
                            double2* __restrict__ pivW, double2* __restrict__ pivC, const int64_t* __restrict__ piv_off)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (c >= n_cls || k >= nE_pad) return;
    const ClassDesc C = cls[c];
    const int N = C.N;
    const double inv_dx2 = 1.0 / (C.dx * C.dx);
    const double* V = tab + tab_vv(C);
    const double zr = k < nE ? E_grid[k] : 0.0, zi = -eps;
    double2* W = pivW + piv_off[c];
    double2* Cp = pivC + piv_off[c];
    double2 cprev = make_double2(0.0, 0.0);
    for (int j = 0; j < N; ++j) {
        const EdRow r = ed_row(scheme, zr, zi, inv_dx2, V, j, N);
        const double2 ac = cmul(r.a, cprev);
        const double2 w = make_double2(r.b.x - ac.x, r.b.y - ac.y);
        const double2 iw = cinv(w);
        cprev = cmul(r.c, iw);
        W[(int64_t)j * nE_pad + k] = iw;
        Cp[(int64_t)j * nE_pad + k] = cprev;
    }
}

template <class Cx>
__global__ void k_ed_solve(const GroupDesc* __restrict__ groups, const ClassDesc* __restrict__ cls,
                           const double* __restrict__ tab, const int64_t* __restrict__ slot_group,
                           const int64_t* __restrict__ slot_inst, int64_t n_slots, const Cx* __restrict__ psi_all,
                           const double* __restrict__ E_grid, int nE, int nE_pad, double eps, int scheme,
                           const double2* __restrict__ pivW, const double2* __restrict__ pivC,
                           const int64_t* __restrict__ piv_off, double2* __restrict__ scratch, int n_max,
                           double* __restrict__ P_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nkb = nE_pad / kLanes;
    double2* __restrict__ sc = scratch + warp * (int64_t)n_max * kLanes;
    for (int64_t task = warp; task < n_slots * nkb; task += n_warps) {
        const int64_t slot = task / nkb;
        const int kb = (int)(task % nkb);
        const int64_t inst = slot_inst[slot];
        if (inst < 0) continue;   // padding slot (warp-uniform)
        const GroupDesc G = groups[slot_group[slot]];
        const ClassDesc C = cls[G.cls];
        const Fma64 F{C.one, C.nzero};
        const int N = G.N, I = G.I;
        const int64_t i = slot - G.slot0;
        const Cx* __restrict__ ps = psi_all + G.psi_off + i;   // point j at ps[j * I]
        const int k = kb * kLanes + lane;
        const double zr = k < nE ? E_grid[k] : 0.0, zi = -eps;
        const double inv_dx2 = 1.0 / (C.dx * C.dx);
        const double* V = tab + tab_vv(C);
        const double2* W = pivW + piv_off[G.cls] + k;
        const double2* Cp = pivC + piv_off[G.cls] + k;
        // forward: d'_j = (r_j - a_j d'_{j-1}) / w_j
        double dr = 0.0, di = 0.0;
        Cx pm = Cx{0, 0}, pc = ps[0], pn = N > 1 ? ps[I] : Cx{0, 0};
        // 1/w rows and (below) the scratch and c' rows are loaded two rows ahead of the recurrence
        double2 wa = W[0], wb = N > 1 ? W[nE_pad] : make_double2(0.0, 0.0);
        for (int j = 0; j < N; ++j) {
            double rr, ri;
            if (scheme == 0) {
                rr = pc.x;
                ri = pc.y;
            } else {   // M2 psi
                const double k12 = 1.0 / 12.0;
                rr = k12 * fma(10.0, (double)pc.x, F.add((double)pm.x, (double)pn.x));
                ri = k12 * fma(10.0, (double)pc.y, F.add((double)pm.y, (double)pn.y));
            }
            double2 a;
            if (scheme == 0) {
                a = make_double2(j > 0 ? 0.5 * inv_dx2 : 0.0, 0.0);
            } else {
                a = j > 0 ? make_double2(fma(zr, 1.0 / 12.0, 0.5 * inv_dx2 - V[j - 1] * (1.0 / 12.0)), zi * (1.0 / 12.0))
                          : make_double2(0.0, 0.0);
            }
            // u = r - a d'
            const double ur = fma(-a.x, dr, fma(a.y, di, rr));
            const double ui = fma(-a.x, di, fma(-a.y, dr, ri));
            const double2 iw = wa;
            wa = wb;
            if (j + 2 < N) wb = W[(int64_t)(j + 2) * nE_pad];
            dr = fma(ur, iw.x, F.mul(-ui, iw.y));
            di = fma(ur, iw.y, F.mul(ui, iw.x));
            sc[(int64_t)j * kLanes + lane] = make_double2(dr, di);
            pm = pc;
            pc = pn;
            pn = j + 2 < N ? ps[(int64_t)(j + 2) * I] : Cx{0, 0};
        }
        // backward: y_j = d'_j - c'_j y_{j+1}, sum |y|^2 (|y|^2 and the sum as float pairs on the FP32
        // pipe, widened to double every kObsBlock points, as the propagation kernels' observables)
        double yr = 0.0, yi = 0.0, s = 0.0;
        float sh = 0.f, sl = 0.f;
        int blk = 0;
        double2 da = sc[(int64_t)(N - 1) * kLanes + lane], ca = Cp[(int64_t)(N - 1) * nE_pad];
        double2 db = make_double2(0.0, 0.0), cb = db;
        if (N > 1) {
            db = sc[(int64_t)(N - 2) * kLanes + lane];
            cb = Cp[(int64_t)(N - 2) * nE_pad];
        }
        for (int j = N - 1; j >= 0; --j) {
            const double2 d2 = da, cp = ca;
            da = db;
            ca = cb;
            if (j - 2 >= 0) {
                db = sc[(int64_t)(j - 2) * kLanes + lane];
                cb = Cp[(int64_t)(j - 2) * nE_pad];
            }
            const double nr = fma(-cp.x, yr, fma(cp.y, yi, d2.x));
            yi = fma(-cp.x, yi, fma(-cp.y, yr, d2.y));
            yr = nr;
            float rh, rl;
            sq_mod_ff(yr, yi, rh, rl);
            ff_acc(sh, sl, rh, rl);
            if (++blk == kObsBlock) {
                s = F.add(f2d_int(sh), F.add(f2d_int(sl), s));
                sh = sl = 0.f;
                blk = 0;
            }
        }
        s = F.add(f2d_int(sh), F.add(f2d_int(sl), s));
        if (k < nE) P_out[inst * (int64_t)nE + k] = (eps / 3.14159265358979323846) * s * C.dx;
    }
}

// Ionisation probability (Sec. 6.1, last paragraph): Ion_i = sum_k w_k P_i(E_k), the quadrature of
// the energy distribution over the caller's nodes.  One warp per instance, lanes striding over the
// energies, FP64 sums combined by shuffles (fixed order: deterministic).
__global__ void k_ionisation(const double* __restrict__ P, int64_t n_inst, int nE, const double* __restrict__ w,
                             double* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n_inst; i += n_warps) {
        const double* row = P + i * (int64_t)nE;
        double s = 0.0;
        for (int k = lane; k < nE; k += kLanes) s = fma(w[k], row[k], s);
        s = warp_sum(s);
        if (lane == 0) out[i] = s;
    }
}

}  // namespace

cudaError_t launch_ionisation(const double* d_P, int64_t n_inst, int nE, const double* d_w, double* d_out,
                              int sm_count, cudaStream_t st)
{
    if (n_inst == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n_inst + 7) / 8, (int64_t)sm_count * 8);
    k_ionisation<<<(unsigned)blocks, 256, 0, st>>>(d_P, n_inst, nE, d_w, d_out);
    return cudaGetLastError();
}

int64_t energy_distribution_scratch_elems(int sm_count, int n_max) { return (int64_t)sm_count * 8 * kLanes * n_max; }

cudaError_t launch_energy_distribution(int mixed, const GroupDesc* d_groups, const ClassDesc* d_cls, int n_cls,
                                       const double* d_tab, const int64_t* d_slot_group, const int64_t* d_slot_inst,
                                       int64_t n_slots, const void* d_psi, const double* d_E_grid, int nE, double eps,
                                       int scheme, void* d_piv, const int64_t* d_piv_off, int64_t piv_elems,
                                       void* d_scratch, int n_max, int sm_count, double* P_out, cudaStream_t st)
{
    if (nE == 0 || n_slots == 0) return cudaSuccess;
    const int nE_pad = (nE + kLanes - 1) / kLanes * kLanes;
    double2* pivW = static_cast<double2*>(d_piv);
    double2* pivC = pivW + piv_elems;
    dim3 pg((nE_pad + 127) / 128, n_cls);
    k_ed_pivots<<<pg, 128, 0, st>>>(d_cls, n_cls, d_tab, d_E_grid, nE, nE_pad, eps, scheme, pivW, pivC, d_piv_off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int blocks = sm_count;   // 8 warps per block: the scratch holds sm_count * 8 warps
    if (mixed)
        k_ed_solve<float2><<<blocks, 256, 0, st>>>(d_groups, d_cls, d_tab, d_slot_group, d_slot_inst, n_slots,
                                                   static_cast<const float2*>(d_psi), d_E_grid, nE, nE_pad, eps, scheme,
                                                   pivW, pivC, d_piv_off, static_cast<double2*>(d_scratch), n_max,
                                                   P_out);
    else
        k_ed_solve<double2><<<blocks, 256, 0, st>>>(d_groups, d_cls, d_tab, d_slot_group, d_slot_inst, n_slots,
                                                    static_cast<const double2*>(d_psi), d_E_grid, nE, nE_pad, eps,
                                                    scheme, pivW, pivC, d_piv_off, static_cast<double2*>(d_scratch),
                                                    n_max, P_out);
    return cudaGetLastError();
}

}  // namespace tdse
