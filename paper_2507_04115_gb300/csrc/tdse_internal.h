// Internal declarations shared by the C-ABI layer (tdse_api.cu) and the kernels (tdse_kernels.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tdse {

constexpr int kLanes = 32;          // instances per group: one per lane of a warp
constexpr int kMaxSegments = 16;    // warps per CTA at most (512 threads)

// Per-class tables (one class = one distinct (N, dx, a, Z)), all length N:
//   ab[j]  = (S0_j, Xh_j)  with S0_j = dt/2 (1/dx^2 + V_j), Xh_j = dt/2 x_j   (FULL_CN diagonal)
//   xv[j]  = (x_j, dV_j)                                                   (observables)
//   mk[j]  = m_j                                                           (edge mask)
struct ClassDesc {
    int64_t tab_off;      // offset (in doubles) of the class block in the table buffer
    int32_t N;
    int32_t jm_lo, jm_hi; // m_j == 1 exactly for jm_lo <= j <= jm_hi
    double dx, a, Z;
    double beta;          // dt / (4 dx^2): magnitude of the off-diagonal of 1 + i dt/2 H
};

// One CTA of the propagation kernel = one group of 32 instances of one class.
struct GroupDesc {
    int64_t psi_off;      // complex-element offset of the group's wavefunctions, layout [N][32]
    int64_t scratch_off;  // complex-element offset of the group's scratch, layout [P][rows][2][32]
    int64_t slot0;        // first slot (slot = group * 32 + lane)
    int64_t nt_max;       // largest Nt over the group's real instances
    int32_t cls;          // class index
    int32_t N, P, K, m;   // grid size, segments (warps), halo, segment length
    int32_t rows;         // scratch rows per warp = m + 2K (clamped to N)
    int32_t pad;
};

// Device-side tables offsets inside a class block (in doubles).
__host__ __device__ inline int64_t tab_ab(const ClassDesc& c) { return c.tab_off; }
__host__ __device__ inline int64_t tab_xv(const ClassDesc& c) { return c.tab_off + 2 * (int64_t)c.N; }
__host__ __device__ inline int64_t tab_mk(const ClassDesc& c) { return c.tab_off + 4 * (int64_t)c.N; }
inline int64_t tab_doubles(int N) { return 5 * (int64_t)N; }

// ---- kernel launchers (tdse_kernels.cu); all return cudaGetLastError() after the launch ----

cudaError_t launch_build_tables(const ClassDesc* d_cls, int n_cls, int max_N, double dt, double mask_width,
                                double mask_exp, int mask_on, double* d_tab, cudaStream_t st);

// Imaginary-time ground state, one CTA per class.  Work buffers: 4 * N doubles per class at
// work + cls_work_off[c].  Results: psi0 (N doubles per class at the same offsets / 4), energy, iters.
cudaError_t launch_ground_state(const ClassDesc* d_cls, int n_cls, int scheme, double dtau, int64_t max_iter,
                                double tol, double* d_work, const int64_t* d_work_off, double* d_energy,
                                int64_t* d_iters, cudaStream_t st);

// Copy each class's real ground state (first N doubles of its work block) into every slot of the class.
cudaError_t launch_broadcast_psi(const GroupDesc* d_groups, int64_t n_groups, const double* d_work,
                                 const int64_t* d_work_off, const int64_t* d_slot_valid, double2* d_psi,
                                 cudaStream_t st);

cudaError_t launch_propagate_fp64(const GroupDesc* d_groups, int64_t g_begin, int64_t n_groups, int P,
                                  const ClassDesc* d_cls, const double* d_tab, const int64_t* d_slot_row,
                                  const int64_t* d_slot_nt, double2* d_psi, double2* d_scratch, const double* E,
                                  double* d_out, double* a_out, int64_t sample_base, int64_t step_begin,
                                  int64_t step_end, int mask_on, int* d_status, cudaStream_t st);

cudaError_t launch_get_psi(const double2* d_psi, int64_t psi_off, int N, int lane, double* out, cudaStream_t st);
cudaError_t launch_set_psi(double2* d_psi, int64_t psi_off, int N, int lane, const double* in, cudaStream_t st);

cudaError_t launch_spectrum(const double* a, const int64_t* d_offsets, int64_t n_rows, double dt, int64_t k_begin,
                            int64_t k_end, double* S, cudaStream_t st);

}  // namespace tdse
