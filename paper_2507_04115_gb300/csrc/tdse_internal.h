// Internal declarations shared by the C-ABI layer (tdse_api.cu) and the kernels (tdse_kernels.cu).
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <limits>
#include <vector>
#include <cuda_runtime.h>

#include "tdse.h"

namespace tdse {

constexpr int kLanes = 32;          // instances per group: one per lane of a warp
constexpr int kMaxSegments = 16;    // warps per CTA at most (512 threads)

// Per-class tables (one class = one distinct (N, dx, a, Z)), all of length N, in doubles:
//   ab[j]  = (S0_j/beta, Xh_j/beta), S0_j = dt/2 (1/dx^2 + V_j), Xh_j = dt/2 x_j  (FULL_CN diagonal)
//   xv[j]  = (x_j, dV_j)                                                  (observables)
//   mk[j]  = m_j                                                          (edge mask)
//   nw[j], nl[j], nc[j]: NUMEROV_SPLIT factors of A = M2 + i dt/2 (-Delta2/2 + M2 V) (complex):
//            W_j/12 = 1/(12 pivot_j), L_j = A_{j,j-1}/pivot_j, C_j = A_{j,j+1}/pivot_j
//   nf[3j..3j+2] = the same three factors rounded to float2 (MIXED)
//   fx[j]  = (x_j, dV_j, m_j, 0) rounded to float4 (MIXED observables and mask)
//   vv[j]  = V_j                                                          (energy distribution)
//   af[j]  = ab[j] rounded to float2                                      (float halo rows)
//   xff[j] = (x_j, dV_j) as float pairs (hi, lo), hi = x rounded to float, lo = x - hi rounded
//            to float: a float4 (x_hi, x_lo, dV_hi, dV_lo)
struct ClassDesc {
    int64_t tab_off;      // offset (in doubles) of the class block in the table buffer
    int32_t N;
    int32_t jm_lo, jm_hi; // m_j == 1 exactly for jm_lo <= j <= jm_hi
    double dx, a, Z;
    double beta;          // dt / (4 dx^2): magnitude of the off-diagonal of 1 + i dt/2 H
    double rho;           // NUMEROV_SPLIT: max_j max(|L_j|, |C_j|), the decay rate of its sweeps
    double one, nzero;    // 1.0 and -0.0 as data, for adds and multiplies issued as FMAs (Fma64)
};

// A group = I instances of one class.  With I = 32 every lane of a warp carries its own instance;
// with I = 32/L each instance spans L lanes of every warp, lane l holding instance l % I and the
// segment l / I of the warp's L (lane split, for batches too small to fill the GPU with 32-wide
// groups).  The propagation kernel processes a group with one CTA at a time (P warps, the group
// uses the first P_g of them), so an instance is cut into P_g * L segments of m points.
struct GroupDesc {
    int64_t psi_off;      // complex-element offset of the group's wavefunctions, layout [N][I]
    int64_t slot0;        // first slot (slot = slot0 + instance index within the group)
    int64_t nt_max;       // largest Nt over the group's real instances
    int32_t cls;          // class index
    int32_t N, P, K, m;   // grid size, warps carrying segments, halo, segment length
    int32_t I;            // instances per group (32, 16, 8, 4, 2 or 1)
    int32_t w;            // cost of one time step (units of group_step_cost / 64, >= 1): the
                          // scheduler's priority is remaining slices x w
};

// Device-side tables offsets inside a class block (in doubles).
__host__ __device__ inline int64_t tab_ab(const ClassDesc& c) { return c.tab_off; }
__host__ __device__ inline int64_t tab_xv(const ClassDesc& c) { return c.tab_off + 2 * (int64_t)c.N; }
__host__ __device__ inline int64_t tab_mk(const ClassDesc& c) { return c.tab_off + 4 * (int64_t)c.N; }
__host__ __device__ inline int64_t tab_nw(const ClassDesc& c) { return c.tab_off + 5 * (int64_t)c.N; }
__host__ __device__ inline int64_t tab_nl(const ClassDesc& c) { return c.tab_off + 7 * (int64_t)c.N; }
__host__ __device__ inline int64_t tab_nc(const ClassDesc& c) { return c.tab_off + 9 * (int64_t)c.N; }
__host__ __device__ inline int64_t tab_nf(const ClassDesc& c) { return c.tab_off + 11 * (int64_t)c.N; }
__host__ __device__ inline int64_t tab_fx(const ClassDesc& c) { return c.tab_off + 14 * (int64_t)c.N; }
__host__ __device__ inline int64_t tab_vv(const ClassDesc& c) { return c.tab_off + 16 * (int64_t)c.N; }
__host__ __device__ inline int64_t tab_af(const ClassDesc& c) { return c.tab_off + 17 * (int64_t)c.N; }
__host__ __device__ inline int64_t tab_xff(const ClassDesc& c) { return c.tab_off + 18 * (int64_t)c.N; }
inline int64_t tab_doubles(int N) { return 20 * (int64_t)N; }

// ---- host-side planning rules shared by the allocating and the static entry points ----

// Halo length K such that beta^K < tol (1e-18 by default): the truncated sweeps then agree with the
// exact Thomas solve below double rounding (|gamma| <= |beta| per point, see tdse_full_cn.cu); 0 when
// beta is too close to 1 for truncation to pay off.  The MIXED FULL_CN path, whose wavefunctions
// are rounded to float every step, takes tol = kMixedHaloTol.
constexpr double kMixedHaloTol = 1e-13;
inline int halo_for_beta(double beta, double tol = 1e-18)
{
    const double b = std::fabs(beta);
    if (b >= 0.85) return 0;
    if (b < 1e-3) return 8;
    const int K = (int)std::ceil(std::log(tol) / std::log(b));
    return std::max(K, 8);
}

// Segments of a class: at most the CTA's warps, and every segment at least four halos long
// (otherwise the halo work dominates); one exact segment when no halo applies.
inline int class_segments(int N, int K, int warps)
{
    if (K == 0) return 1;
    const int max_P = std::max(1, N / std::max(4 * K, 16));
    return std::max(1, std::min(warps, max_P));
}

// Segment length of a group: P_g warps x L lanes per instance share the N points.
inline int group_segment_length(int N, int P, int L) { return (N + P * L - 1) / (P * L); }

// Warps carrying segments in a group of a class (N points, halo K) at L lanes per instance: the
// class's segment rule for 32-wide groups; every warp of the CTA for lane-split groups (short
// segments are the price of spreading an instance over more lanes).
inline int group_warps(int N, int K, int L, int warps)
{
    return L == 1 ? class_segments(N, K, warps) : std::max(1, std::min(warps, N / L));
}

// Cost model of one time step of a group: ceil(P/4) x (27 m + 36 K) FP64 warp instructions on its
// busiest SM sub-partition (27 per own point: forward elimination 16, back substitution and update
// 11; 36 per halo point: 2K forward rows and K back-substitution rows), m = N / (P L).  One group
// runs on one SM at a time.
inline double group_step_cost(int N, int K, int L, int warps)
{
    const int P = group_warps(N, K, L, warps);
    const int m = group_segment_length(N, P, L);
    return std::ceil(P / 4.0) * (27.0 * m + 36.0 * (P * L > 1 ? K : 0));
}

// Group widths by the whole job's makespan.  A group of instances with Nt_max steps keeps one SM
// busy for Nt_max x cost; groups migrate between SMs only between slices, so the job takes at least
// max(sum of the groups' work / SMs, longest group).  When a few groups are much longer than the
// rest (an uneven batch: long pulses on large grids), the longest group bounds the job; spreading
// those instances over more lanes (L x 2 halves the instances per group, the group's step gets
// cheaper at the price of more halo rows) shortens it.
//   Per class c: N[c], K[c] (0: no halo, L stays 1), base L[c] (the per-step model's choice) and
//   the instances' Nt sorted in decreasing order.  Groups are cut greedily from the longest
//   instance: the group takes the smallest L >= base with Nt_first x cost <= T (32 at most) and
//   the next 32/L instances.  T runs over S0 x 0.95^j (S0: the longest group of the base plan);
//   the plan with the smallest makespan estimate is kept if it beats the base plan's by 5 %.
//   widths[c] receives the L of every group of class c, in order.  Returns the estimate.
struct WidthClass {
    int N, K, L_base;
    std::vector<int64_t> nt_desc;
};

inline double plan_widths_at(const std::vector<WidthClass>& cls, int warps, int sm_count, double T,
                             std::vector<std::vector<int>>* widths, double* work_out = nullptr,
                             double* longest_out = nullptr)
{
    double work = 0.0, longest = 0.0;
    if (widths) widths->assign(cls.size(), {});
    for (size_t c = 0; c < cls.size(); ++c) {
        const WidthClass& C = cls[c];
        const int64_t n = (int64_t)C.nt_desc.size();
        for (int64_t k = 0; k < n;) {
            int L = C.L_base;
            const double nt = (double)std::max<int64_t>(C.nt_desc[k], 1);
            if (C.K > 0)
                while (L < 32 && nt * group_step_cost(C.N, C.K, L, warps) > T) L *= 2;
            const double t = nt * group_step_cost(C.N, C.K, L, warps);
            work += t;
            longest = std::max(longest, t);
            if (widths) (*widths)[c].push_back(L);
            k += 32 / L;
        }
    }
    if (work_out) *work_out = work;
    if (longest_out) *longest_out = longest;
    return std::max(work / std::max(1, sm_count), longest);
}

inline double plan_widths(const std::vector<WidthClass>& cls, int warps, int sm_count,
                          std::vector<std::vector<int>>* widths, double* work_out = nullptr,
                          double* longest_out = nullptr)
{
    const double inf = std::numeric_limits<double>::infinity();
    double S0 = 0.0;
    for (const WidthClass& C : cls)
        if (!C.nt_desc.empty())
            S0 = std::max(S0, (double)std::max<int64_t>(C.nt_desc[0], 1) * group_step_cost(C.N, C.K, C.L_base, warps));
    const double M0 = plan_widths_at(cls, warps, sm_count, inf, nullptr);
    double best = M0, best_T = inf;
    for (int j = 1; j <= 90; ++j) {
        const double T = S0 * std::pow(0.95, j);
        const double M = plan_widths_at(cls, warps, sm_count, T, nullptr);
        if (M < best) {
            best = M;
            best_T = T;
        }
    }
    if (!(best < 0.95 * M0)) best_T = inf;
    return plan_widths_at(cls, warps, sm_count, best_T, widths, work_out, longest_out);
}

// Function attributes (the dynamic shared memory limit) belong to a device: a launcher that raises
// one keeps a flag per device ordinal and sets it on the first launch on each device.
constexpr int kMaxAttrDevices = 64;
inline bool attr_needed(const std::atomic<bool>* flags, int* dev)
{
    *dev = 0;
    cudaGetDevice(dev);
    return *dev < 0 || *dev >= kMaxAttrDevices || !flags[*dev].load(std::memory_order_acquire);
}
inline void attr_done(std::atomic<bool>* flags, int dev)
{
    if (dev >= 0 && dev < kMaxAttrDevices) flags[dev].store(true, std::memory_order_release);
}

// Stores the calling thread's last-error message (tdse_api.cu).
const char* set_error_message(const char* msg);

// CUDA device a batch was created on (for host code layered on the public calls).
int batch_device(const tdse_batch* b);

// ---- kernel launchers (tdse_kernels.cu); all return cudaGetLastError() after the launch ----

cudaError_t launch_build_tables(const ClassDesc* d_cls, int n_cls, int max_N, double dt, double mask_width,
                                double mask_exp, int mask_on, double* d_tab, cudaStream_t st);

// Imaginary-time ground state, one CTA of kGsThreads threads per class.  Work buffers: kGsWork * N
// doubles per class at work + cls_work_off[c], the ground state psi0 in the first N.  Results:
// psi0, energy, iters.
constexpr int kGsThreads = 1024;
constexpr int kGsWork = 8;
cudaError_t launch_ground_state(const ClassDesc* d_cls, int n_cls, int scheme, double dtau, int64_t max_iter,
                                double tol, double* d_work, const int64_t* d_work_off, double* d_energy,
                                int64_t* d_iters, cudaStream_t st);

// Copy each class's real ground state (first N doubles of its work block) into every slot of the class.
cudaError_t launch_broadcast_psi(int mixed, const GroupDesc* d_groups, int64_t n_groups, const double* d_work,
                                 const int64_t* d_work_off, const int64_t* d_slot_valid, void* d_psi,
                                 cudaStream_t st);

// Persistent FULL_CN propagation (tdse_full_cn.cu): `ctas` CTAs of P warps pick groups
// dynamically, `slice` steps at a time.  mixed = 0: psi and scratch are double2; mixed = 1:
// float2.  Scratch holds ctas * P * rows rows of 2 * 32 complex values.  ring: MIXED bulk-copy
// slots per warp in [2, 4] (full_cn_ring_slots for the CTAs per SM of the launch); wait_polls:
// polls before a MIXED bulk-copy wait gives up (the batch reports TDSE_ERR_TIMEOUT).  d_ckpt (FP64
// only, NULL = none): the state after every kc-th step is also written to the adjoint's checkpoint
// layout (group g at d_ckpt_off[g], checkpoint c at + c * N * I; c = 0 is the state at step 0).
cudaError_t launch_propagate_full_cn(int mixed, const GroupDesc* d_groups, int64_t n_groups, int P, int ctas,
                                     const ClassDesc* d_cls, const double* d_tab, const int64_t* d_slot_row,
                                     const int64_t* d_slot_nt, void* d_psi, void* d_scratch, int rows,
                                     const double* E, double* d_out, double* a_out, int64_t sample_base,
                                     int64_t step_begin, int64_t step_end, int slice, int mask_on, int* d_busy,
                                     int* d_progress, int* d_status, int ring, uint32_t wait_polls,
                                     cudaStream_t st, void* d_ckpt = nullptr, const int64_t* d_ckpt_off = nullptr,
                                     int kc = 0);
// CTAs of P warps that fit on one SM (MIXED: with the shallowest bulk-copy ring).
int propagate_max_ctas_per_sm(int mixed, int P);
// MIXED bulk-copy slots per warp when per_sm CTAs of P warps share an SM.
int propagate_ring_slots(int P, int per_sm);

// Discrete adjoint of FULL_CN in FP64 (tdse_adjoint.cu): one CTA per group for the whole call.
// lam: psi-shaped; ckpt: per group (intervals + 1) states at ckpt_off[g]; work: ctas * n_max * 32;
// tape: ctas * kc * n_max * 32; scratch as for the propagation; gtape (NULL = none): ctas * kc * P *
// rows * 32 complex doubles, the elimination coefficients of the recomputed steps, which the
// backward sweeps then reuse instead of recomputing them.
cudaError_t launch_adjoint_full_cn(const GroupDesc* d_groups, int64_t n_groups, int P, int ctas, const ClassDesc* d_cls,
                                   const double* d_tab, const int64_t* d_slot_row, const int64_t* d_slot_nt,
                                   const void* d_psi0, void* d_lam, void* d_ckpt, const int64_t* d_ckpt_off,
                                   void* d_work, void* d_tape, void* d_scratch, int rows, int n_max, int kc,
                                   const double* E, const double* gd, const double* ga, double* gE, int mask_on,
                                   int* d_busy, int* d_progress, cudaStream_t st, int have_ckpt = 0,
                                   void* d_gtape = nullptr);

// Energy distribution of every instance state (tdse_resolvent.cu): pivots per (class, energy) into
// d_piv (2 * piv_elems complex doubles, class c at d_piv_off[c], N_c rows of nE rounded up to 32),
// then one warp per (instance, 32 energies) with a scratch of energy_distribution_scratch_elems.
int64_t energy_distribution_scratch_elems(int sm_count, int n_max);
cudaError_t launch_energy_distribution(int mixed, const GroupDesc* d_groups, const ClassDesc* d_cls, int n_cls,
                                       const double* d_tab, const int64_t* d_slot_group, const int64_t* d_slot_inst,
                                       int64_t n_slots, const void* d_psi, const double* d_E_grid, int nE, double eps,
                                       int scheme, void* d_piv, const int64_t* d_piv_off, int64_t piv_elems,
                                       void* d_scratch, int n_max, int sm_count, double* P_out, cudaStream_t st);

// Ionisation probability: out[i] = sum_k w[k] P[i * nE + k] (one warp per instance).
cudaError_t launch_ionisation(const double* d_P, int64_t n_inst, int nE, const double* d_w, double* d_out,
                              int sm_count, cudaStream_t st);

// Field ingestion (tdse_field.cu): DFT coefficients of every coarse row (n_rows x (M/2 + 1) complex
// doubles in d_coef), then the zero-padded interpolant at n_fine samples per row.
cudaError_t launch_resample_field(const double* coarse, int64_t n_rows, int M, double dt_c, double dt_f,
                                  int64_t n_fine, int64_t out_stride, double* out, void* d_coef, cudaStream_t st);

// Persistent NUMEROV_SPLIT propagation (same scheduler, scratch and layouts; tables nw/nl/nc/nf).
cudaError_t launch_propagate_numerov(int mixed, const GroupDesc* d_groups, int64_t n_groups, int P, int ctas,
                                     const ClassDesc* d_cls, const double* d_tab, const int64_t* d_slot_row,
                                     const int64_t* d_slot_nt, void* d_psi, void* d_scratch, int rows,
                                     const double* E, double* d_out, double* a_out, int64_t sample_base,
                                     int64_t step_begin, int64_t step_end, int slice, int mask_on, double dt,
                                     int* d_busy, int* d_progress, int* d_status, cudaStream_t st);

// Support of each class's ground state (first N doubles of work + work_off[c]): support[2c..2c+1]
// = [lo, hi), the largest lo and smallest hi with sum_{j<lo} psi0_j^2 dx and sum_{j>=hi} psi0_j^2 dx
// each at most kSupportTail^2 / 2 (one warp per class).
constexpr double kSupportTail = 1e-17;
cudaError_t launch_gs_support(const ClassDesc* d_cls, int n_cls, const double* d_work, const int64_t* d_work_off,
                              int64_t* d_support, cudaStream_t st);

// Ground-state population and near-core probability of every instance (a cluster of CTAs per
// group, sized for sm_count SMs), read over the hull of the class's psi0 support and the points
// with |x_j| < r_core; psi0 of class c: the first N doubles of gs_work + gs_off[c]; out: n_inst x 2.
cudaError_t launch_populations(int mixed, const GroupDesc* d_groups, int64_t n_groups, const ClassDesc* d_cls,
                               const int64_t* d_slot_inst, const void* d_psi, const double* d_gs_work,
                               const int64_t* d_gs_off, const int64_t* d_support, double r_core, double* out,
                               int sm_count, cudaStream_t st);

cudaError_t launch_get_psi(int mixed, const void* d_psi, int64_t psi_off, int N, int lane, int I, double* out,
                           cudaStream_t st);
cudaError_t launch_set_psi(int mixed, void* d_psi, int64_t psi_off, int N, int lane, int I, const double* in, cudaStream_t st);

cudaError_t launch_spectrum(const double* a, const int64_t* d_offsets, int64_t n_rows, double dt, int64_t k_begin,
                            int64_t k_end, double* S, cudaStream_t st);

}  // namespace tdse
