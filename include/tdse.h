/*
 * tdse.h -- C ABI of libtdse.so, a GB300 (sm_103a) engine for batches of independent
 * one-dimensional time-dependent Schroedinger equations in the length gauge
 * (arXiv:2507.04115, Sec. 3.1 Eqs. "Hamiltonian (a)" and "SC potential"; Sec. 4.2):
 *
 *     i d/dt psi(x,t) = [ -1/2 d^2/dx^2 - Z / sqrt(x^2 + a^2) + x E(t) ] psi(x,t)
 *
 * one per macroscopic point, each driven by its own sampled field E(t), each emitting the
 * position expectation d(t) = <x> and the dipole acceleration a(t) = <dV/dx + E(t)>
 * (Sec. 3.1 Eq. "dipole acceleration"; App. A Eq. "Current_der_TDSE1D").
 *
 * Discretisation shared by every entry point
 *   grid      x_j = (j - (N-1)/2) dx, j = 0..N-1, Dirichlet walls psi_{-1} = psi_N = 0
 *             (Sec. 4.2 uses a symmetric grid; the cell-centred variant keeps N even)
 *   time      t_n = n dt, n = 0..Nt; E_n = E(t_n); the field's time origin is t = 0 (Sec. 4.2)
 *   schemes   TDSE_FULL_CN: Crank-Nicolson with the field in the diagonal at the midpoint
 *                 (1 + i dt/2 H(Ebar)) psi~ = (1 - i dt/2 H(Ebar)) psi^n, Ebar = (E_n + E_{n+1})/2,
 *                 H = -Delta2/2 + V + x Ebar, Delta2 = tridiag(1,-2,1)/dx^2
 *             TDSE_NUMEROV_SPLIT: the paper's three substeps (Sec. 4.2, Eqs. "CN - step 4",
 *                 "CN - step 2", "CN - step 3"): Numerov-corrected field-free CN, then the phase
 *                 exp(-i dt E_n x_j)
 *   absorber  after every step psi_j *= m_j, m_j = cos(pi/2 (|x_j| - x_b)/w)^p for |x_j| > x_b,
 *             x_b = N dx/2 - w (the paper has none, Sec. 4.2; width <= 0 disables it)
 *   output    d_n = dx sum_j x_j |psi_j|^2,  a_n = dx sum_j (dV/dx(x_j) + E_n) |psi_j|^2
 *             for n = 0..Nt (n = 0 is the initial state); rectangle rule, sum |psi|^2 dx = 1
 *
 * Conventions
 *   - "_dev" pointers are CUDA device memory owned by the caller; "_host" pointers are host
 *     memory owned by the caller.  The batch owns its wavefunctions, tables and scratch.
 *   - Compute entry points are asynchronous on the given stream (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream) and return a status, never abort.  The library
 *     sets the batch's device before it launches.
 *   - Errors: every entry point validates its arguments on the host and returns
 *     TDSE_ERR_ARG without launching anything; a failed CUDA call returns TDSE_ERR_CUDA.
 *     tdse_last_error() gives a message for the calling thread's last failure.
 *   - A batch handle is not thread-safe.  Separate handles are independent.
 *   - All floating-point values cross the boundary as IEEE double, whatever the precision.
 */
#ifndef TDSE_H
#define TDSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TDSE_OK = 0,
    TDSE_ERR_ARG = 1,        /* invalid argument; nothing was launched */
    TDSE_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    TDSE_ERR_NONFINITE = 3,  /* an instance's norm became non-finite or grew above 1 + 1e-6 (FP64),
                                1 + 1e-3 (MIXED) */
    TDSE_ERR_TIMEOUT = 4,    /* a bounded device wait gave up (MIXED bulk copies, see
                                tdse_set_wait_limit); reported by tdse_check */
    TDSE_ERR_NOMEM = 5,      /* device or host allocation failed */
    TDSE_ERR_STATE = 6       /* call out of order (e.g. propagate before any initial state) */
} tdse_status;

typedef enum {
    TDSE_FP64 = 0,   /* the solve and the wavefunctions in IEEE double; |psi|^2 and the observable
                        sums as float pairs (about 2^-44 relative per point) over blocks of 16
                        points, added in double across blocks */
    TDSE_MIXED = 1   /* psi, the solve's right-hand side and back substitution in float; the
                        elimination recurrence (pivots) in double; the observables as float
                        partial sums over 16 points, added in double across blocks */
} tdse_precision;

typedef enum {
    TDSE_FULL_CN = 0,
    TDSE_NUMEROV_SPLIT = 1
} tdse_scheme;

/* One TDSE instance: grid size and spacing, soft-core parameter a and charge Z. */
typedef struct {
    int32_t N;          /* grid points, 16 <= N <= 1 << 20 */
    double dx;          /* grid spacing (a.u.), > 0 */
    double softening;   /* a (a.u.), > 0 */
    double charge;      /* Z; 1 for the paper's model, 0 gives a free electron */
} tdse_instance;

/* Edge absorber: width w (a.u.) and exponent p; width <= 0 disables the mask. */
typedef struct {
    double width;
    double exponent;
} tdse_absorber;

typedef struct tdse_batch tdse_batch;

/* Create a batch of n_inst independent instances sharing the time step dt.
 *   inst_host[n_inst]          per-instance grid, soft-core a and charge
 *   n_steps_host[n_inst]       Nt_i, the number of time steps of instance i (>= 0)
 *   row_offsets_host[n_inst+1] layout of every per-sample array (field E, outputs d and a):
 *                              instance i owns elements [row_offsets[i], row_offsets[i+1]) of
 *                              each; element k of the row holds sample n = sample_base + k, with
 *                              sample_base given per call.  Non-decreasing, row_offsets[0] >= 0.
 *   absorber                   NULL or the edge mask parameters
 *   device                     CUDA device ordinal the batch lives on
 * Allocates the wavefunctions (uninitialised until tdse_ground_state or tdse_set_psi), the
 * per-instance tables and the propagation scratch on that device.  On success *out receives
 * the handle; on failure *out is NULL and nothing stays allocated. */
tdse_status tdse_batch_create(const tdse_instance* inst_host, int64_t n_inst, double dt,
                              const int64_t* n_steps_host, const int64_t* row_offsets_host,
                              const tdse_absorber* absorber, tdse_precision precision,
                              tdse_scheme scheme, int device, tdse_batch** out);

/* Release everything the batch owns.  Synchronises the batch's device first.  NULL is a no-op. */
void tdse_batch_destroy(tdse_batch* batch);

/* Ground state of the field-free Hamiltonian H0 of every instance (the paper leaves the method
 * open, Sec. 3.1 defines E_g only): imaginary-time Crank-Nicolson with the scheme's H0,
 *     (M + dtau/2 K) psi' = (M - dtau/2 K) psi,  psi' <- psi'/sqrt(sum |psi'|^2 dx),
 * started from exp(-x^2), stopped when |E_k - E_{k-1}| < tol or after max_iter iterations,
 * sign fixed so that psi is positive at the grid centre.  It runs once per distinct
 * (N, dx, a, Z) and the result is copied into every instance of that class, which also
 * resets each instance's time to n = 0.
 *   energies_host[n_inst]  NULL or receives E_g per instance (the call then synchronises)
 *   iters_host[n_inst]     NULL or receives the iteration count per instance (synchronises) */
tdse_status tdse_ground_state(tdse_batch* batch, double dtau, int64_t max_iter, double tol,
                              double* energies_host, int64_t* iters_host, void* stream);

/* Advance every instance i over the steps n = step_begin .. min(step_end, Nt_i) - 1.
 *   E_dev   field samples: E_n of instance i at E_dev[row_offsets[i] + n - sample_base]; the call
 *           reads n = step_begin .. min(step_end, Nt_i)
 *   d_dev, a_dev  outputs in the same layout: d_{n+1}, a_{n+1} for every step taken, and d_n, a_n
 *           for n = step_begin when step_begin == 0 (the initial state)
 *   sample_base <= step_begin; every row must hold the samples the call touches.
 * Instances with Nt_i <= step_begin are left untouched.  Chunked calls with consecutive ranges
 * continue the same propagation. */
tdse_status tdse_propagate(tdse_batch* batch, const double* E_dev, double* d_dev, double* a_dev,
                           int64_t sample_base, int64_t step_begin, int64_t step_end, void* stream);

/* Copy the wavefunction of instance `inst` out of / into the batch: 2N doubles, interleaved
 * (re, im), device memory of the caller (the paper exposes psi for user post-processing,
 * Sec. 4.2).  tdse_set_psi also marks the batch as initialised (resume from a checkpoint). */
tdse_status tdse_get_psi(tdse_batch* batch, int64_t inst, double* psi_dev, void* stream);
tdse_status tdse_set_psi(tdse_batch* batch, int64_t inst, const double* psi_dev, void* stream);

/* Copy the whole wavefunction state of the batch to (direction 0) or from (direction 1) a caller
 * device buffer of tdse_plan's psi_bytes bytes (layout internal to the library; use it to
 * checkpoint and resume a batch).  Loading marks the batch as initialised. */
tdse_status tdse_copy_state(tdse_batch* batch, void* buffer_dev, int32_t direction, void* stream);

/* Gradient of a loss L(d, a) with respect to every field sample, through the FULL_CN propagation
 * (FP64 batches): the exact discrete adjoint of the scheme, i.e. the backward sweep with the
 * conjugate-transposed step.  The batch's current wavefunctions are taken as the initial state
 * psi^0 (call after tdse_ground_state, tdse_set_psi or tdse_copy_state, before propagating), and
 * are left unchanged.  The loss gradients gd_n = dL/dd_n and ga_n = dL/da_n, the field E and the
 * output gE_n = dL/dE_n use the batch's row layout with sample_base 0 and n = 0..Nt_i.
 *   ckpt_every  states are checkpointed every ckpt_every steps and recomputed in between (one
 *               interval of states is kept per CTA); memory ~ (Nt/ckpt_every + ckpt_every) states.
 * With lambda^n = 2 dL/d conj(psi^n): lambda^Nt = g^Nt; mu = B_n^{-1} M lambda^{n+1};
 * lambda^n = A_n mu + g^n, g^n_j = 2 dx (gd_n x_j + ga_n (dV_j + E_n)) psi^n_j; and
 * dL/dEbar_n = dt/2 sum_j x_j Im(conj(mu_j)(psi^n_j + psi~^{n+1}_j)) split evenly to E_n, E_{n+1},
 * plus ga_n dx sum_j |psi^n_j|^2 on E_n (A_n = 1 + i dt/2 H(Ebar_n), B_n = conj(A_n), M the mask). */
tdse_status tdse_adjoint(tdse_batch* batch, const double* E_dev, const double* gd_dev, const double* ga_dev,
                         double* gE_dev, int32_t ckpt_every, void* stream);

/* tdse_propagate that also records the adjoint's checkpoints: the state after every ckpt_every-th
 * step (and the state at step 0) is copied into the batch's checkpoint buffers, in the layout
 * tdse_adjoint's own forward pass writes.  A recording starts with step_begin = 0 and may continue
 * over further calls, each beginning where the previous one ended, with the same ckpt_every; once it
 * covers every instance's last step, tdse_adjoint_checkpointed can start from it.  FP64 FULL_CN
 * only.  Allocates the adjoint's buffers on first use (as tdse_adjoint); the arguments are
 * tdse_propagate's.  TDSE_ERR_STATE for a continuation that does not follow the recording. */
tdse_status tdse_propagate_checkpointed(tdse_batch* batch, const double* E_dev, double* d_dev, double* a_dev,
                                        int64_t sample_base, int64_t step_begin, int64_t step_end, int32_t ckpt_every,
                                        void* stream);

/* tdse_adjoint from the checkpoints of a complete tdse_propagate_checkpointed recording: the same
 * gradient, without the adjoint's own forward pass (the intervals are recomputed from the recorded
 * checkpoints, then swept backwards).  E_dev must hold the field of the recorded propagation; the
 * batch's current state is not used.  TDSE_ERR_STATE when no complete recording exists (none, or
 * the launch shape or layout changed since). */
tdse_status tdse_adjoint_checkpointed(tdse_batch* batch, const double* E_dev, const double* gd_dev, const double* ga_dev,
                                      double* gE_dev, void* stream);

/* Synchronise the stream and report TDSE_ERR_NONFINITE if any instance's norm became non-finite
 * or exceeded 1 + 1e-6 (FP64; 1 + 1e-3 in MIXED) during a propagation since the batch was created
 * or last checked, or TDSE_ERR_TIMEOUT if a bounded bulk-copy wait gave up for it (MIXED, see
 * tdse_set_wait_limit);
 * *first_bad_host (may be NULL) receives the first such instance or -1.  Clears the flags. */
tdse_status tdse_check(tdse_batch* batch, int64_t* first_bad_host, void* stream);

/* Time-dependent electron energy distribution of every instance's current state (Sec. 6.1, the
 * resolvent of the field-free Hamiltonian and its factorised form):
 *     P_i(E_k) = N_eps eps^2 || (E_k - H0 - i eps)^{-1} psi_i ||^2,  N_eps = 1/(pi eps),
 * the normalisation of a Lorentzian of half-width eps (an eigenstate of H0 gives a Lorentzian of
 * unit area times its norm), || v ||^2 = sum_j |v_j|^2 dx.  The inversion is done in the batch
 * scheme's representation of H0 = M^{-1} K: ((E_k - i eps) M - K)^{-1} (M psi), with M = 1 and the
 * three-point H0 for FULL_CN, and the Numerov pencil M2, K = -Delta2/2 + M2 V for NUMEROV_SPLIT.
 * Integrating P over E gives the norm (the ionised part is the integral above the threshold).
 *   E_grid_host   n_energies energies in a.u. (host, any order, |E| <= 1e12)
 *   epsilon       resolution eps >= 1e-12 a.u.
 *   P_dev         out: n_inst x n_energies doubles, row i = instance i in creation order
 * Works on FP64 and MIXED batches (the solves always run in FP64).  Synchronous: allocates the
 * pivot tables (2 x 16 B x N x n_energies per class) for the call, keeps a solve scratch of
 * 8 x SMs x 32 x N_max x 16 B on the batch, and synchronises the stream before returning. */
tdse_status tdse_energy_distribution(tdse_batch* batch, const double* E_grid_host, int32_t n_energies,
                                     double epsilon, double* P_dev, void* stream);

/* Time-dependent ionisation probability of every instance's current state (Sec. 6.1, last
 * paragraph: integrating P(E, t) over energy gives the ionisation probability, i.e. the electron
 * density the TDSE itself predicts):
 *     ion_i = sum_k w_k P_i(E_k),  w = trapezoid weights of the nodes: w_0 = (E_1 - E_0)/2,
 *             w_k = (E_{k+1} - E_{k-1})/2, w_last = (E_last - E_{last-1})/2,
 * with P_i(E_k) exactly as tdse_energy_distribution computes it at resolution epsilon.  The
 * integral is meant over the continuum: the soft-core potential vanishes at infinity, so the nodes
 * should start at the threshold E = 0 and reach an energy beyond which P is negligible, with a
 * spacing well below epsilon (P varies on that scale).  At finite epsilon a bound state contributes
 * the Lorentzian tail above the threshold, atan(epsilon / |E_b|) / pi for an eigenstate at E_b.
 *   E_nodes_host  n_nodes >= 2 strictly ascending energies (a.u., host)
 *   P_dev         NULL, or out: n_inst x n_nodes doubles, the distribution at the nodes
 *   ion_dev       out: n_inst doubles, row i = instance i in creation order
 * FP64 and MIXED batches (FP64 solves and sums).  Synchronous, with the allocations of
 * tdse_energy_distribution plus the weights (and P when P_dev is NULL) for the call. */
tdse_status tdse_ionisation(tdse_batch* batch, const double* E_nodes_host, int32_t n_nodes, double epsilon,
                            double* P_dev, double* ion_dev, void* stream);

/* Populations of every instance's current state (Sec. 7.5: the time-dependent ground-state
 * population and the probability of finding the electron near the nucleus):
 *     out[2 i]     = | sum_j psi0_j psi_i,j dx |^2        (ground-state population)
 *     out[2 i + 1] = sum_{|x_j| < r_core} |psi_i,j|^2 dx  (near-core probability)
 * psi0 is the class's real field-free ground state from the batch's last tdse_ground_state call
 * (normalised to sum_j psi0_j^2 dx = 1), x_j = (j - (N-1)/2) dx.  r_core >= 0 (+inf gives the
 * norm).  out_dev: device, n_inst x 2 doubles, row i = instance i in creation order.  Sums run in
 * FP64 on FP64 and MIXED batches.  TDSE_ERR_STATE before the first tdse_ground_state, and after a
 * tdse_set_layout until a state is set again.
 * Asynchronous on the stream; allocates nothing (graph-capturable). */
tdse_status tdse_populations(tdse_batch* batch, double r_core, double* out_dev, void* stream);

/* Field ingestion (Sec. 4.2: the input interval is shifted to start at t = 0 and the coarsely
 * sampled field is interpolated to the propagation step by zero-padding in the Fourier domain).
 * Row r of coarse_dev holds M samples E(t_min + m dt_coarse), m = 0..M-1 (rows contiguous, M
 * apart); row r of out_dev (at r * out_stride) receives n_fine samples at t = n dt_fine, t measured
 * from the row's first sample:
 *     E(t) = (1/M) sum_{k=-floor(M/2)}^{floor(M/2)} w_k Ehat_k exp(2 pi i k t / T),  T = M dt_coarse,
 * Ehat the DFT of the row, w_k = 1/2 for |k| = M/2 (even M: the Nyquist bin split between the two
 * ends of the padded spectrum), else 1 -- the trigonometric interpolant, which reproduces the coarse
 * samples exactly.  It is T-periodic: times beyond the window wrap around, so pad the coarse row
 * with zeros past the pulse.  With out_stride equal to a batch's row stride the output feeds
 * tdse_propagate directly.  M in [2, 8192]; computed in FP64; synchronous (allocates
 * n_rows x (M/2+1) x 16 bytes for the call). */
tdse_status tdse_resample_field(const double* coarse_dev, int64_t n_rows, int32_t M, double dt_coarse, double dt_fine,
                                int64_t n_fine, int64_t out_stride, double* out_dev, int device, void* stream);

/* Macroscopic source spectrum of every dipole-acceleration row (Sec. 3.2: the far-field integral
 * takes the temporal Fourier transform of the macroscopic source, the gas density times the
 * microscopic dJ/dt = a(t); Sec. 2 fixes the convention F^(w) = (2 pi)^(-1/2) int F(t) e^{+i w t} dt),
 * by the rectangle rule over the samples t_n = n dt, n = 0..L_r-1:
 *     out[r][w] = weight_r dt / sqrt(2 pi) sum_n a_r,n exp(i omega_w n dt)
 *   a_dev          device, rows r at [offsets[r], offsets[r+1]) (a batch's a(t) rows with sample_base 0)
 *   omega_host     n_omega angular frequencies (same time unit as dt; |omega| <= 1e6)
 *   weight_dev     NULL (weight 1) or device n_rows doubles: the gas density of each row's point
 *   out_dev        device, n_rows x n_omega complex values as (re, im) double pairs, row-major
 * FP64.  Asynchronous on the stream (stream-ordered allocation of the offsets and frequencies).
 * The rows of a volume laid out radius-major (row = i_rho * n_z + i_z) give the source layout of
 * tdse_hankel directly. */
tdse_status tdse_dipole_spectrum(const double* a_dev, const int64_t* offsets_host, int64_t n_rows, double dt,
                                 const double* omega_host, int32_t n_omega, const double* weight_dev,
                                 double* out_dev, void* stream);

/* Far field of a homogeneous generating medium, Eq. "Hankel long homogeneous" (Sec. 3.2), evaluated
 * by direct grid integration over the source points as the paper's HANKEL module does (Sec. 4.3):
 *     E(rho_o, z, w) = -(mu0/(4 pi)) e^{i k z} sum_i wz_i e^{-i k z'_i} e^{i k rho_o^2/(2 D_i)} / D_i
 *                      * sum_j wr_j rho'_j e^{i k rho'_j^2/(2 D_i)} S[j][i][w] J0(k rho_o rho'_j / D_i),
 * D_i = z - z'_i, k = k(omega_w), wr and wz the trapezoidal weights of the source radii and planes
 * (a single plane, n_z = 1, is the thin medium with weight 1: its source is the plane's source
 * integrated over the thickness).  SI units: lengths in m, k in 1/m, mu0 = 1.25663706212e-6 H/m;
 * E takes the source's units times H.
 *   S_dev          device, n_rho x n_z x n_omega complex (re, im) values, S[j][i][w] at
 *                  ((j * n_z + i) * n_omega + w): the macroscopic source (density times the
 *                  transformed dipole acceleration, see tdse_dipole_spectrum) at (rho'_j, z'_i, omega_w)
 *   rho_src_host   n_rho radii, >= 0, strictly ascending (n_rho <= 2048)
 *   z_src_host     n_z planes, strictly ascending, all below z_obs
 *   k_host         n_omega wave numbers k(omega_w) > 0 (n_omega <= 65535)
 *   rho_obs_host   n_obs observation radii >= 0 in the plane z = z_obs
 *   E_dev          device, n_omega x n_obs complex (re, im) values, E[w][o]
 * FP64 throughout (the phases k z' reach 1e6 rad).  Asynchronous on the stream on `device`
 * (stream-ordered allocation of the grids). */
tdse_status tdse_hankel(const double* S_dev, const double* rho_src_host, int32_t n_rho, const double* z_src_host,
                        int32_t n_z, const double* k_host, int32_t n_omega, double z_obs, const double* rho_obs_host,
                        int32_t n_obs, double* E_dev, int device, void* stream);

/* Power spectrum of sampled signals (Sec. 3.1 / App. A: the source term enters Maxwell's
 * equations through its Fourier transform):
 *     S_i[k] = dt^2 |sum_{n=0}^{L_i - 1} a_i[n] exp(-2 pi i k n / L_i)|^2,  k = k_begin .. k_end - 1,
 * a plain DFT over the L_i = row length samples of row i (no window, no padding).
 *   a_dev     rows: row i is a_dev[offsets[i] .. offsets[i+1])   (offsets_host: host, n_rows+1)
 *   S_dev     [n_rows][k_end - k_begin] row-major
 * Requires 0 <= k_begin < k_end. */
tdse_status tdse_spectrum(const double* a_dev, const int64_t* offsets_host, int64_t n_rows, double dt,
                          int64_t k_begin, int64_t k_end, double* S_dev, void* stream);

/* Plan chosen for the batch (for benchmarks and tests): number of instance groups, warps
 * carrying grid segments per instance (largest over the classes), halo length in points (largest),
 * warps per CTA, CTAs of the persistent propagation grid, time steps per scheduling slice, the
 * bytes of the propagation scratch and of the wavefunctions, and the lanes per instance of the
 * layout (largest over the classes; see tdse_set_layout).  An instance is cut into
 * segments x lanes_per_instance segments. */
typedef struct {
    int64_t n_groups;
    int32_t segments;
    int32_t halo;
    int32_t warps_per_cta;
    int32_t ctas;
    int32_t slice_steps;
    int64_t scratch_bytes;
    int64_t psi_bytes;
    int32_t lanes_per_instance;
    double longest_share;   /* the planner's model: the longest group's time / (the whole batch's work
                               / SMs); above 0.5 the longest group bounds the job at 2 CTAs per SM */
} tdse_plan_info;

tdse_status tdse_plan(const tdse_batch* batch, tdse_plan_info* info_host);

/* How instances map onto the lanes of a warp.  The paper has no counterpart (its solver is serial
 * per MPI rank); this is the GPU layout choice.  With lanes_per_instance L = 1 a warp carries 32
 * instances, one per lane, each cut into as many segments as the CTA has warps.  With L in
 * {2, 4, 8, 16, 32} a warp carries 32/L instances and each spans L lanes, so every instance is cut
 * into L times more segments: more halo work per point, but 32/L-instance groups occupy L times
 * more SMs, which pays when the batch is too small to fill the GPU.  L = 0 (the default at
 * creation) picks L from a cost model of the batch: FP64 warp instructions of a step per group
 * against the number of SMs.  Classes whose sweeps cannot be truncated (decay rate per point
 * dt/(4 dx^2) for FULL_CN, the largest Numerov factor for NUMEROV_SPLIT, >= 0.85) always use L = 1.  The wavefunction state is discarded (call before
 * tdse_ground_state, tdse_set_psi or tdse_copy_state); synchronises the device and reallocates.
 * Returns TDSE_ERR_ARG for L outside {0, 1, 2, 4, 8, 16, 32}. */
tdse_status tdse_set_layout(tdse_batch* batch, int32_t lanes_per_instance);

/* Override the launch configuration for later calls (0 keeps the default of each):
 * warps_per_cta in [1, 16] (default 8 for FP64, 12 for MIXED FULL_CN, 16 for MIXED NUMEROV_SPLIT; also
 * the largest number of segments per instance),
 * ctas_per_sm in [1, 32] (default 1; clamped to the occupancy limit), slice_steps >= 1 (default 16),
 * max_ctas >= 1 caps the persistent grid (default: no cap beyond SMs x ctas_per_sm and the number
 * of groups).  Synchronises the device; the scratch is reallocated. */
tdse_status tdse_set_launch(tdse_batch* batch, int32_t warps_per_cta, int32_t ctas_per_sm, int32_t slice_steps,
                            int32_t max_ctas);

/* The layout (lanes per instance) that the per-step cost model of tdse_set_layout would pick for a
 * batch of these instances on a GPU with sm_count SMs, computed on the host without a GPU and
 * without creating anything, for capacity planning and tests.  It takes no step counts: when the
 * instances' Nt differ, tdse_batch_create may also widen the longest groups beyond this L so that
 * no group outlasts the rest of the batch (tdse_plan reports the widest).  The paper has no
 * counterpart.  Arguments as tdse_batch_create; *lanes_out receives L. */
tdse_status tdse_model_layout(const tdse_instance* inst_host, int64_t n_inst, double dt, tdse_precision precision,
                              tdse_scheme scheme, int32_t sm_count, int32_t* lanes_out);

/* Adjoint gamma tape (tdse_adjoint, tdse_adjoint_checkpointed).  The backward sweep of step n solves
 * with the same matrix A_n as the recomputation of that step, so the recomputation can store the
 * elimination coefficients gamma of every sweep row of a checkpoint interval and the backward sweep
 * reuse them (the pivot recurrence is then evaluated once per step instead of twice).  The tape
 * takes ctas x ckpt_every x warps x rows x 32 complex doubles (tdse_plan: ctas, warps_per_cta; rows
 * = segment + 2 halos); it is allocated at the next adjoint call when it takes at most half of the
 * device's free memory, and left out otherwise.  Results are bitwise the same with and without it.
 * enable: 1 (default) uses it when it fits, 0 never (and frees it).  The paper has no counterpart. */
tdse_status tdse_set_adjoint_gamma_tape(tdse_batch* batch, int32_t enable);

/* Bound on the MIXED kernels' waits for their bulk copies (global -> shared memory), in mbarrier
 * polls; default 2^22 (a copy lands within microseconds).  A wait that runs out drains the copies
 * still in flight (with the default bound), stops using bulk copies for the rest of the launch and
 * flags the group's instances, so tdse_check then returns TDSE_ERR_TIMEOUT; the results of that
 * launch are invalid but the context stays usable.  polls = 0 makes every wait give up at once:
 * the test of this path (there is no way to make a real copy fail without faulting the GPU).
 * The paper has no counterpart.  Applies to later calls; polls in [0, 2^30]. */
tdse_status tdse_set_wait_limit(tdse_batch* batch, int64_t polls);

/* Launch-shape autotuner.  The paper runs one solver per MPI rank and has no counterpart; this
 * picks, by timing, the shape tdse_set_launch sets: warps per CTA (also the number of segments
 * each instance's tridiagonal solve is split into, i.e. the depth of the parallel split), CTAs per
 * SM and the scheduling slice.  It times tdse_propagate over steps [step_begin, step_end) of the
 * given field rows (same arguments as tdse_propagate) for each candidate, every trial starting
 * from the batch's current state, which is restored afterwards: a coordinate search over
 * warps {4, 6, 8, 12, 16} x CTAs per SM {1, 2} at a 16-step slice, then slices {8, 32, 64} at the
 * best pair; shapes that the occupancy clamp makes identical are timed once.  The fastest shape
 * stays set on the batch.
 *   d_dev, a_dev    rows over the probed steps are scratch: overwritten by the probes
 *   repeats         timed runs per candidate in [1, 100] (the minimum counts); the first
 *                   candidate also gets one untimed run
 *   trials_host     optional (max_trials may be 0): receives up to max_trials trials in the order
 *                   run; *n_trials_host (may be NULL) receives how many were run.
 * Synchronous: it synchronises the stream and the device (tdse_set_launch), allocates a device
 * copy of the state for the duration of the call, and must not be called during stream capture. */
typedef struct {
    int32_t warps_per_cta;
    int32_t ctas_per_sm;
    int32_t slice_steps;
    int32_t ctas;   /* resulting persistent grid size */
    float ms;       /* fastest of the timed runs, milliseconds */
} tdse_tune_trial;

tdse_status tdse_autotune(tdse_batch* batch, const double* E_dev, double* d_dev, double* a_dev, int64_t sample_base,
                          int64_t step_begin, int64_t step_end, int32_t repeats, tdse_tune_trial* trials_host,
                          int32_t max_trials, int32_t* n_trials_host, void* stream);

/* FULL_CN FP64 propagation that allocates nothing, for callers that cannot call cudaMalloc: code
 * embedded in a host application that owns the whole device-memory budget (a pre-sized pool it
 * hands out itself), or code on a path that must not allocate at all.  The paper has no
 * counterpart; it is the same kernel as tdse_propagate with every piece of scratch (tables,
 * scheduler state, group descriptors, solver rows) in one fixed 64 MiB array compiled into the
 * library, which every GPU that loads the library holds until the process exits.
 *   inst_host       one instance description shared by all n_inst instances (one grid class)
 *   n_steps         Nt of every instance; row_stride: E, d and a hold row i at [i*row_stride, ...),
 *                   element k of a row being sample n = sample_base + k
 *   psi_dev         in/out, caller-owned, 32*ceil(n_inst/32)*N complex doubles (re, im) in the
 *                   lane-interleaved layout: instance i, point j at complex index
 *                   ((i/32)*N + j)*32 + i%32.  The padding lanes of the last group (i >= n_inst)
 *                   must be allocated and hold finite values: they are read by the sweeps but
 *                   never written, and they never mix with the real instances' lanes
 *   other arguments as tdse_propagate; no non-finite flags are reported.
 * Sizes whose scratch does not fit the array return TDSE_ERR_ARG with the limit in the message;
 * up to that limit the grid is shrunk to what fits (fewer CTAs, so slower than tdse_propagate).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress), so make
 * that first call before any stream capture.  Every call shares the array and leaves its contents
 * behind (the call clears what has to start at zero); calls that overlap on the GPU -- on
 * different streams, or concurrent host threads -- race on it and must be serialised. */
tdse_status tdse_propagate_static(const tdse_instance* inst_host, int64_t n_inst, double dt,
                                  const tdse_absorber* absorber, int64_t n_steps, int64_t row_stride,
                                  double* psi_dev, const double* E_dev, double* d_dev, double* a_dev,
                                  int64_t sample_base, int64_t step_begin, int64_t step_end, void* stream);

/* Measured rates of the arithmetic pipes the engine is bound by (the FP64 pipe of GB300 is not in a
 * copy/GEMM peak table): FP64 and FP32 fused multiply-add throughput with every SM busy, FP64 warp
 * instructions per second with one active lane per warp (the cost is per warp instruction), FP64
 * throughput with 1, 2 and 4 warps per SM (one FP64 unit per SM sub-partition), and
 * double->float->double conversion pairs per second, and the cost of a reciprocal seed in FP64 FMA
 * slots: the hardware double approximation (rcp.approx.ftz.f64, the seed the kernels use) and a
 * float-based alternative (float approximation of the truncated value, integer exponent shifts),
 * each measured as the extra time of a loop that adds one seed per FMA over the FMA-only loop.
 * Runs a few short bounded launches on `device` (synchronous; allocates a small buffer). */
typedef struct {
    double fp64_fma_tflops;
    double fp64_warp_instr_per_s;
    double fp64_one_lane_warp_instr_per_s;
    double fp64_tflops_warps_per_sm[3];
    double fp32_fma_tflops;
    double cvt_pairs_per_s;
    int32_t sm_count;
    double sm_clock_mhz;
    double rcp_f64_approx_fma_slots;
    double rcp_seed_fma_slots;
    double dadd_fma_slots;   /* time of an FP64 add, a multiply, in units of an FP64 FMA */
    double dmul_fma_slots;
    double add_as_fma_slots; /* the add as fma(x, 1, y), the multiply as fma(x, y, -0), with 1 and -0 not known at compile time */
    double mul_as_fma_slots;
    double fma_repeat_slots; /* the FMA loop timed again last (clock drift check) */
} tdse_pipe_rates;

tdse_status tdse_probe_pipes(int device, tdse_pipe_rates* out_host);

/* Message for the calling thread's last failed call ("" if none). */
const char* tdse_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TDSE_H */
