// C ABI of libtdse.so (declared in include/tdse.h): argument validation, instance grouping,
// planning, memory ownership and kernel launches.  Host logic only; kernels live in
// tdse_kernels.cu.
#include "tdse.h"
#include "tdse_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

using namespace tdse;

namespace {

thread_local std::string g_last_error;

tdse_status fail(tdse_status st, const std::string& msg)
{
    g_last_error = msg;
    return st;
}

}  // namespace

namespace tdse {
const char* set_error_message(const char* msg)
{
    g_last_error = msg ? msg : "";
    return g_last_error.c_str();
}
}  // namespace tdse

namespace {

tdse_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(TDSE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define TDSE_CUDA(call, what)                          \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <class T>
cudaError_t dev_alloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

}  // namespace

struct tdse_batch {
    int device = 0;
    int64_t n_inst = 0;
    double dt = 0.0;
    tdse_precision precision = TDSE_FP64;
    tdse_scheme scheme = TDSE_FULL_CN;
    int mask_on = 0;
    double mask_width = 0.0, mask_exp = 0.0;
    std::vector<tdse_instance> inst;
    std::vector<int64_t> n_steps, row_off;
    // classes and slots
    std::vector<ClassDesc> classes;
    std::vector<int> inst_class;
    std::vector<int64_t> slot_of_inst;
    std::vector<GroupDesc> groups;
    std::vector<int> class_P, class_K, class_L;
    std::vector<int64_t> slot_group;   // group of every slot
    int64_t n_slots = 0;
    int lanes_request = 0;             // tdse_set_layout's lanes per instance (0 = cost model)
    double longest_share = 0.0;        // longest group's modelled time / (total work / SMs)
    // launch configuration of the persistent propagation kernel
    int warps_override = 0, ctas_per_sm_override = 0, slice_override = 0, max_ctas_override = 0;
    int warps = 8, ctas = 0, rows = 0, slice = 16, ring = 4;
    uint32_t wait_polls = 1u << 22;   // MIXED bulk-copy wait bound (tdse_set_wait_limit)
    int sm_count = 0;
    bool initialized = false;
    bool gs_done = false;             // a ground state was computed (psi0 in d_gs_work)
    // device memory
    ClassDesc* d_cls = nullptr;
    GroupDesc* d_groups = nullptr;
    double* d_tab = nullptr;
    int64_t* d_slot_row = nullptr;
    int64_t* d_slot_nt = nullptr;
    int64_t* d_slot_valid = nullptr;
    int64_t* d_slot_group = nullptr;   // group of every slot
    int64_t* d_slot_inst = nullptr;    // instance of every slot (-1 for padding)
    void* d_psi = nullptr;       // double2 (FP64) or float2 (MIXED) elements
    void* d_scratch = nullptr;
    int* d_busy = nullptr;
    int* d_progress = nullptr;
    int* d_status = nullptr;
    double* d_gs_work = nullptr;
    int64_t* d_gs_off = nullptr;
    double* d_gs_energy = nullptr;
    int64_t* d_gs_iters = nullptr;
    int64_t* d_gs_support = nullptr;   // per class: [lo, hi) outside which psi0 has tail norm < 1e-17
    int64_t psi_elems = 0, scratch_elems = 0;
    // adjoint buffers (allocated on the first tdse_adjoint call, resized when the interval changes)
    void* d_lam = nullptr;
    void* d_ckpt = nullptr;
    int64_t* d_ckpt_off = nullptr;
    void* d_work = nullptr;
    void* d_tape = nullptr;
    void* d_gtape = nullptr;           // adjoint gamma tape (optional, see ensure_gamma_tape)
    size_t gtape_bytes = 0;
    bool use_gtape = true;             // tdse_set_adjoint_gamma_tape
    int adj_kc = 0, adj_ctas = 0;
    // checkpoints recorded by tdse_propagate_checkpointed: steps [0, ckpt_next) are covered (-1: none)
    int64_t ckpt_next = -1;
    // energy-distribution buffers (allocated on first use, grown as needed)
    void* d_ed_scratch = nullptr;
    int64_t ed_scratch_elems = 0;
    int mixed() const { return precision == TDSE_MIXED ? 1 : 0; }
    size_t cx_bytes() const { return precision == TDSE_MIXED ? sizeof(float2) : sizeof(double2); }
};

namespace {

void free_device(tdse_batch* b)
{
    cudaFree(b->d_cls);
    cudaFree(b->d_groups);
    cudaFree(b->d_tab);
    cudaFree(b->d_slot_row);
    cudaFree(b->d_slot_nt);
    cudaFree(b->d_slot_valid);
    cudaFree(b->d_psi);
    cudaFree(b->d_scratch);
    cudaFree(b->d_busy);
    cudaFree(b->d_progress);
    cudaFree(b->d_status);
    cudaFree(b->d_gs_work);
    cudaFree(b->d_gs_off);
    cudaFree(b->d_gs_energy);
    cudaFree(b->d_gs_iters);
    cudaFree(b->d_gs_support);
    cudaFree(b->d_lam);
    cudaFree(b->d_ckpt);
    cudaFree(b->d_ckpt_off);
    cudaFree(b->d_work);
    cudaFree(b->d_tape);
    cudaFree(b->d_gtape);
    b->d_gtape = nullptr;
    b->gtape_bytes = 0;
    cudaFree(b->d_slot_group);
    cudaFree(b->d_slot_inst);
    cudaFree(b->d_ed_scratch);
    b->d_slot_group = b->d_slot_inst = nullptr;
    b->d_ed_scratch = nullptr;
    b->ed_scratch_elems = 0;
    b->d_lam = b->d_ckpt = b->d_work = b->d_tape = nullptr;
    b->d_ckpt_off = nullptr;
    b->d_cls = nullptr;
    b->d_groups = nullptr;
    b->d_tab = nullptr;
    b->d_slot_row = b->d_slot_nt = b->d_slot_valid = nullptr;
    b->d_psi = b->d_scratch = nullptr;
    b->d_busy = b->d_progress = nullptr;
    b->d_status = nullptr;
    b->d_gs_work = nullptr;
    b->d_gs_off = nullptr;
    b->d_gs_energy = nullptr;
    b->d_gs_iters = nullptr;
    b->d_gs_support = nullptr;
}

// NUMEROV_SPLIT: LU factors of the time-independent A = M2 + i h (-Delta2/2 + M2 V), h = dt/2
// (Sec. 4.2, Eq. "CN - step 2"), M2 = tridiag(1, 10, 1)/12, (M2 V)_{jk} = (M2)_{jk} V_k:
//   A_{j,j-1} = 1/12 + i h (-1/(2dx^2) + V_{j-1}/12), A_{jj} = 10/12 + i h (1/dx^2 + 10 V_j/12),
//   A_{j,j+1} = 1/12 + i h (-1/(2dx^2) + V_{j+1}/12);
// Thomas from j = 0: pivot_j = A_jj - A_{j,j-1} C_{j-1}, W_j = 1/pivot_j, L_j = A_{j,j-1} W_j,
// C_j = A_{j,j+1} W_j.  Writes (W_j/12, L_j, C_j) as double pairs and float pairs into the host
// images of the nw/nl/nc/nf tables and returns max(|L|, |C|).
double numerov_factors(const ClassDesc& C, double dt, std::vector<double>& nw, std::vector<double>& nl,
                       std::vector<double>& nc, std::vector<float>& nf)
{
    using cd = std::complex<double>;
    const int N = C.N;
    const double h = 0.5 * dt, inv = 1.0 / (C.dx * C.dx);
    std::vector<double> V(N);
    for (int j = 0; j < N; ++j) {
        const double x = (j - 0.5 * (N - 1)) * C.dx;
        V[j] = -C.Z / std::sqrt(x * x + C.a * C.a);
    }
    nw.assign(2 * (size_t)N, 0.0);
    nl.assign(2 * (size_t)N, 0.0);
    nc.assign(2 * (size_t)N, 0.0);
    nf.assign(6 * (size_t)N, 0.0f);
    double rho = 0.0;
    cd cprev(0.0, 0.0);
    for (int j = 0; j < N; ++j) {
        const cd lo = j > 0 ? cd(1.0 / 12.0, h * (-0.5 * inv + V[j - 1] / 12.0)) : cd(0.0, 0.0);
        const cd di(10.0 / 12.0, h * (inv + (10.0 / 12.0) * V[j]));
        const cd up = j < N - 1 ? cd(1.0 / 12.0, h * (-0.5 * inv + V[j + 1] / 12.0)) : cd(0.0, 0.0);
        const cd piv = di - lo * cprev;
        const cd W = 1.0 / piv;
        const cd L = lo * W;
        const cd Cj = up * W;
        const cd W12 = W / 12.0;
        nw[2 * j] = W12.real();
        nw[2 * j + 1] = W12.imag();
        nl[2 * j] = L.real();
        nl[2 * j + 1] = L.imag();
        nc[2 * j] = Cj.real();
        nc[2 * j + 1] = Cj.imag();
        nf[6 * j + 0] = (float)W12.real();
        nf[6 * j + 1] = (float)W12.imag();
        nf[6 * j + 2] = (float)L.real();
        nf[6 * j + 3] = (float)L.imag();
        nf[6 * j + 4] = (float)Cj.real();
        nf[6 * j + 5] = (float)Cj.imag();
        rho = std::max(rho, std::max(std::abs(L), std::abs(Cj)));
        cprev = Cj;
    }
    return rho;
}

// Classes: distinct (N, dx, a, Z), compared bit for bit; fills b->classes and b->inst_class.
void build_classes(tdse_batch* b, const tdse_instance* inst_host, int64_t n_inst, double dt)
{
    std::map<std::tuple<int32_t, uint64_t, uint64_t, uint64_t>, int> cmap;
    b->inst_class.resize(n_inst);
    for (int64_t i = 0; i < n_inst; ++i) {
        const tdse_instance& I = inst_host[i];
        uint64_t kdx, ka, kz;
        std::memcpy(&kdx, &I.dx, 8);
        std::memcpy(&ka, &I.softening, 8);
        std::memcpy(&kz, &I.charge, 8);
        auto key = std::make_tuple(I.N, kdx, ka, kz);
        auto it = cmap.find(key);
        int c;
        if (it == cmap.end()) {
            c = (int)b->classes.size();
            cmap.emplace(key, c);
            ClassDesc C{};
            C.N = I.N;
            C.dx = I.dx;
            C.a = I.softening;
            C.Z = I.charge;
            C.beta = dt / (4.0 * I.dx * I.dx);
            C.one = 1.0;
            C.nzero = -0.0;
            b->classes.push_back(C);
        } else {
            c = it->second;
        }
        b->inst_class[i] = c;
    }
}

int default_warps(const tdse_batch* b)
{
    // measured on the 8192 x 4096 volume batch: FP64 is FP64-pipe bound with two warps per
    // sub-partition; the MIXED kernels need more warps to cover latency
    if (b->precision == TDSE_MIXED) return b->scheme == TDSE_NUMEROV_SPLIT ? 16 : 12;
    return 8;
}

// Lanes per instance for the lane-split layout, from the cost model of one time step
// (group_step_cost): the step time is the larger of (total work / SMs) and the longest single
// group (one group runs on one SM).  L = 1 keeps 32 instances per warp; a larger L is taken only
// when it is clearly faster, i.e. when the batch has too few groups to occupy the SMs.  Classes
// without a usable halo keep L = 1.  build_groups then widens single groups further where the
// whole job's makespan asks for it (plan_widths).
// Decay rate per point of a class's truncated sweeps: |gamma| <= beta for FULL_CN, max(|L|, |C|)
// of the factors for NUMEROV_SPLIT.
double class_decay(const tdse_batch* b, const ClassDesc& C)
{
    return b->scheme == TDSE_NUMEROV_SPLIT ? C.rho : C.beta;
}

// Halo of a class: exact to double rounding, except on the MIXED FULL_CN path, whose float
// wavefunctions need it only far below float rounding (kMixedHaloTol).
int class_halo(const tdse_batch* b, const ClassDesc& C)
{
    const bool mixed_cn = b->precision == TDSE_MIXED && b->scheme == TDSE_FULL_CN;
    return halo_for_beta(class_decay(b, C), mixed_cn ? kMixedHaloTol : 1e-18);
}

int model_lanes(const tdse_batch* b, const std::vector<int64_t>& class_count)
{
    const int warps = b->warps_override > 0 ? b->warps_override : default_warps(b);
    double best_t = 0.0;
    int best_L = 1;
    for (int L = 1; L <= kLanes; L *= 2) {
        double work = 0.0, longest = 0.0;
        for (size_t c = 0; c < b->classes.size(); ++c) {
            const ClassDesc& C = b->classes[c];
            const int K = class_halo(b, C);
            const int Lc = K == 0 ? 1 : L;
            const double cost = group_step_cost(C.N, K, Lc, warps);
            const double groups = std::ceil((double)class_count[c] * Lc / kLanes);
            work += groups * cost;
            longest = std::max(longest, cost);
        }
        const double t = std::max(work / std::max(1, b->sm_count), longest);
        if (L == 1 || t < 0.9 * best_t) {
            best_t = t;
            best_L = L;
        }
    }
    return best_L;
}

// Slots and groups: instances ordered by class, then by decreasing Nt (long groups first), cut
// into groups of I = 32/L instances, L per group: the per-step model's L (model_lanes) or the
// caller's (tdse_set_layout) for every group, widened for the longest groups where the makespan
// estimate asks for it (plan_widths; not under tdse_set_layout).  (Re)allocates everything sized by
// the grouping.  The state is lost.
tdse_status build_groups(tdse_batch* b)
{
    const int n_cls = (int)b->classes.size();
    const int64_t n_inst = b->n_inst;
    std::vector<int64_t> class_count(n_cls, 0);
    for (int64_t i = 0; i < n_inst; ++i) ++class_count[b->inst_class[i]];
    const int L = b->lanes_request > 0 ? b->lanes_request : model_lanes(b, class_count);

    std::vector<int64_t> order(n_inst);
    for (int64_t i = 0; i < n_inst; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t p, int64_t q) {
        if (b->inst_class[p] != b->inst_class[q]) return b->inst_class[p] < b->inst_class[q];
        return b->n_steps[p] > b->n_steps[q];
    });
    const int warps = b->warps_override > 0 ? b->warps_override : default_warps(b);
    std::vector<WidthClass> wc(n_cls);
    for (int c = 0; c < n_cls; ++c) {
        wc[c].N = b->classes[c].N;
        wc[c].K = class_halo(b, b->classes[c]);
        wc[c].L_base = wc[c].K == 0 ? 1 : L;
    }
    for (int64_t k = 0; k < n_inst; ++k) wc[b->inst_class[order[k]]].nt_desc.push_back(b->n_steps[order[k]]);
    std::vector<std::vector<int>> widths;
    double work = 0.0, longest = 0.0;
    if (b->lanes_request > 0)
        plan_widths_at(wc, warps, b->sm_count, std::numeric_limits<double>::infinity(), &widths, &work, &longest);
    else
        plan_widths(wc, warps, b->sm_count, &widths, &work, &longest);
    b->longest_share = work > 0.0 ? longest / (work / std::max(1, b->sm_count)) : 0.0;
    b->class_L.assign(n_cls, 1);
    for (int c = 0; c < n_cls; ++c)
        for (int Lg : widths[c]) b->class_L[c] = std::max(b->class_L[c], Lg);
    b->groups.clear();
    b->slot_group.clear();
    b->slot_of_inst.assign(n_inst, -1);
    std::vector<int64_t> slot_row, slot_nt, slot_valid;
    int64_t psi_elems = 0;
    for (int64_t k = 0; k < n_inst;) {
        const int c = b->inst_class[order[k]];
        size_t gk = 0;   // group index within the class
        while (k < n_inst && b->inst_class[order[k]] == c) {
            const int I = kLanes / (gk < widths[c].size() ? widths[c][gk] : widths[c].back());
            ++gk;
            GroupDesc G{};
            G.cls = c;
            G.N = b->classes[c].N;
            G.I = I;
            G.slot0 = (int64_t)slot_row.size();
            G.psi_off = psi_elems;
            psi_elems += (int64_t)G.N * I;
            G.nt_max = 0;
            for (int q = 0; q < I; ++q) {
                b->slot_group.push_back((int64_t)b->groups.size());
                if (k < n_inst && b->inst_class[order[k]] == c) {
                    const int64_t i = order[k++];
                    b->slot_of_inst[i] = (int64_t)slot_row.size();
                    slot_row.push_back(b->row_off[i]);
                    slot_nt.push_back(b->n_steps[i]);
                    slot_valid.push_back(1);
                    G.nt_max = std::max(G.nt_max, b->n_steps[i]);
                } else {
                    slot_row.push_back(0);
                    slot_nt.push_back(-1);
                    slot_valid.push_back(0);
                }
            }
            b->groups.push_back(G);
        }
    }
    b->n_slots = (int64_t)slot_row.size();
    b->psi_elems = psi_elems;
    b->initialized = false;

    cudaFree(b->d_groups);
    cudaFree(b->d_slot_row);
    cudaFree(b->d_slot_nt);
    cudaFree(b->d_slot_valid);
    cudaFree(b->d_slot_group);
    cudaFree(b->d_slot_inst);
    cudaFree(b->d_psi);
    cudaFree(b->d_status);
    cudaFree(b->d_busy);
    cudaFree(b->d_progress);
    b->d_slot_group = b->d_slot_inst = nullptr;
    b->d_groups = nullptr;
    b->d_slot_row = b->d_slot_nt = b->d_slot_valid = nullptr;
    b->d_psi = nullptr;
    b->d_status = b->d_busy = b->d_progress = nullptr;
    // adjoint buffers are sized by the grouping: dropped, reallocated by the next tdse_adjoint
    cudaFree(b->d_lam);
    cudaFree(b->d_ckpt);
    cudaFree(b->d_ckpt_off);
    cudaFree(b->d_work);
    cudaFree(b->d_tape);
    cudaFree(b->d_gtape);
    b->d_gtape = nullptr;
    b->gtape_bytes = 0;
    b->d_lam = b->d_ckpt = b->d_work = b->d_tape = nullptr;
    b->d_ckpt_off = nullptr;
    b->adj_kc = 0;
    b->ckpt_next = -1;
    TDSE_CUDA(dev_alloc(&b->d_groups, b->groups.size()), "cudaMalloc(groups)");
    TDSE_CUDA(dev_alloc(&b->d_slot_row, (size_t)b->n_slots), "cudaMalloc(slots)");
    TDSE_CUDA(dev_alloc(&b->d_slot_nt, (size_t)b->n_slots), "cudaMalloc(slots)");
    TDSE_CUDA(dev_alloc(&b->d_slot_valid, (size_t)b->n_slots), "cudaMalloc(slots)");
    TDSE_CUDA(cudaMalloc(&b->d_psi, (size_t)std::max<int64_t>(psi_elems, 1) * b->cx_bytes()), "cudaMalloc(psi)");
    TDSE_CUDA(dev_alloc(&b->d_status, (size_t)b->n_slots), "cudaMalloc(status)");
    TDSE_CUDA(dev_alloc(&b->d_busy, b->groups.size()), "cudaMalloc(sched)");
    TDSE_CUDA(dev_alloc(&b->d_progress, b->groups.size()), "cudaMalloc(sched)");
    TDSE_CUDA(cudaMemcpy(b->d_slot_row, slot_row.data(), sizeof(int64_t) * b->n_slots, cudaMemcpyHostToDevice), "cudaMemcpy(slots)");
    TDSE_CUDA(cudaMemcpy(b->d_slot_nt, slot_nt.data(), sizeof(int64_t) * b->n_slots, cudaMemcpyHostToDevice), "cudaMemcpy(slots)");
    TDSE_CUDA(cudaMemcpy(b->d_slot_valid, slot_valid.data(), sizeof(int64_t) * b->n_slots, cudaMemcpyHostToDevice), "cudaMemcpy(slots)");
    std::vector<int64_t> slot_inst(b->n_slots, -1);
    for (int64_t i = 0; i < n_inst; ++i) slot_inst[b->slot_of_inst[i]] = i;
    TDSE_CUDA(dev_alloc(&b->d_slot_group, (size_t)b->n_slots), "cudaMalloc(slots)");
    TDSE_CUDA(dev_alloc(&b->d_slot_inst, (size_t)b->n_slots), "cudaMalloc(slots)");
    TDSE_CUDA(cudaMemcpy(b->d_slot_group, b->slot_group.data(), sizeof(int64_t) * b->n_slots, cudaMemcpyHostToDevice), "cudaMemcpy(slots)");
    TDSE_CUDA(cudaMemcpy(b->d_slot_inst, slot_inst.data(), sizeof(int64_t) * b->n_slots, cudaMemcpyHostToDevice), "cudaMemcpy(slots)");
    TDSE_CUDA(cudaMemset(b->d_status, 0, sizeof(int) * b->n_slots), "cudaMemset(status)");
    TDSE_CUDA(cudaMemset(b->d_psi, 0, b->cx_bytes() * (size_t)std::max<int64_t>(psi_elems, 1)), "cudaMemset(psi)");
    return TDSE_OK;
}

// (Re)compute the launch configuration, the group descriptors and the scratch, and (re)allocate.
tdse_status build_plan(tdse_batch* b)
{
    const int n_cls = (int)b->classes.size();
    b->warps = b->warps_override > 0 ? b->warps_override : default_warps(b);
    b->slice = b->slice_override > 0 ? b->slice_override : 16;
    b->class_P.assign(n_cls, 1);
    b->class_K.assign(n_cls, 0);
    int rows = 1;
    for (auto& G : b->groups) {
        const ClassDesc& C = b->classes[G.cls];
        const int L = kLanes / G.I;
        int K = class_halo(b, C);
        const int P = group_warps(C.N, K, L, b->warps);
        if (P == 1 && L == 1) K = 0;   // one exact segment
        G.P = P;
        G.K = K;
        G.m = group_segment_length(G.N, P, L);
        G.w = std::max(1, (int)std::lround(group_step_cost(C.N, K, L, b->warps) / 64.0));
        b->class_P[G.cls] = std::max(b->class_P[G.cls], P);
        b->class_K[G.cls] = std::max(b->class_K[G.cls], K);
        // a sweep covers its segment and a halo on each side (m + 2K rows; the 32-wide propagation
        // clips it at the walls); a single exact segment covers the N points
        rows = std::max(rows, P * (kLanes / G.I) == 1 ? G.N : G.m + 2 * K);
    }
    b->rows = rows;
    const int per_sm_max = propagate_max_ctas_per_sm(b->mixed(), b->warps);
    const int per_sm = b->ctas_per_sm_override > 0 ? std::min(b->ctas_per_sm_override, per_sm_max) : 1;
    b->ring = propagate_ring_slots(b->warps, per_sm);
    b->ctas = (int)std::min<int64_t>((int64_t)b->groups.size(), (int64_t)b->sm_count * per_sm);
    if (b->max_ctas_override > 0) b->ctas = std::min(b->ctas, b->max_ctas_override);
    const int64_t sc = (int64_t)b->ctas * b->warps * rows * 2 * kLanes;
    cudaFree(b->d_scratch);
    b->d_scratch = nullptr;
    TDSE_CUDA(cudaMalloc(&b->d_scratch, (size_t)std::max<int64_t>(sc, 1) * b->cx_bytes()), "cudaMalloc(scratch)");
    b->scratch_elems = sc;
    TDSE_CUDA(cudaMemcpy(b->d_groups, b->groups.data(), sizeof(GroupDesc) * b->groups.size(), cudaMemcpyHostToDevice),
              "cudaMemcpy(groups)");
    return TDSE_OK;
}

bool is_finite(double v) { return std::isfinite(v); }

}  // namespace

namespace {

// Adjoint buffers (lambda, checkpoints and their offsets, the per-CTA work state and tape), sized by
// the grouping, the persistent grid and the checkpoint interval; reallocated when either changes,
// which drops any recorded checkpoints.
tdse_status ensure_adjoint_buffers(tdse_batch* b, int ckpt_every, cudaStream_t st, int* n_max_out)
{
    int n_max = 1;
    for (auto& G : b->groups) n_max = std::max(n_max, G.N);
    *n_max_out = n_max;
    if (!b->d_lam || b->adj_kc != ckpt_every || b->adj_ctas != b->ctas) {
        b->ckpt_next = -1;
        TDSE_CUDA(cudaStreamSynchronize(st), "tdse_adjoint: synchronize");
        cudaFree(b->d_lam);
        cudaFree(b->d_ckpt);
        cudaFree(b->d_ckpt_off);
        cudaFree(b->d_work);
        cudaFree(b->d_tape);
        b->d_lam = b->d_ckpt = b->d_work = b->d_tape = nullptr;
        b->d_ckpt_off = nullptr;
        b->adj_kc = 0;
        std::vector<int64_t> off(b->groups.size());
        int64_t total = 0;
        for (size_t g = 0; g < b->groups.size(); ++g) {
            off[g] = total;
            const int64_t n_int = (b->groups[g].nt_max + ckpt_every - 1) / ckpt_every;
            total += (n_int + 1) * (int64_t)b->groups[g].N * b->groups[g].I;
        }
        const size_t cx = sizeof(double2);
        TDSE_CUDA(cudaMalloc(&b->d_lam, (size_t)std::max<int64_t>(b->psi_elems, 1) * cx), "cudaMalloc(adjoint lambda)");
        TDSE_CUDA(cudaMalloc(&b->d_ckpt, (size_t)std::max<int64_t>(total, 1) * cx), "cudaMalloc(adjoint checkpoints)");
        TDSE_CUDA(dev_alloc(&b->d_ckpt_off, off.size()), "cudaMalloc(adjoint offsets)");
        TDSE_CUDA(cudaMalloc(&b->d_work, (size_t)b->ctas * n_max * kLanes * cx), "cudaMalloc(adjoint work)");
        TDSE_CUDA(cudaMalloc(&b->d_tape, (size_t)b->ctas * ckpt_every * (size_t)n_max * kLanes * cx),
                  "cudaMalloc(adjoint tape)");
        TDSE_CUDA(cudaMemcpy(b->d_ckpt_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice),
                  "cudaMemcpy(adjoint offsets)");
        b->adj_kc = ckpt_every;
        b->adj_ctas = b->ctas;
    }
    return TDSE_OK;
}

// The adjoint's gamma tape: the elimination coefficients of every recomputed step of a checkpoint
// interval (ctas x kc x warps x rows x 32 complex doubles), which spare the backward sweeps the
// pivot recurrence.  It is an accelerator only (the coefficients are recomputed bitwise the same
// without it): allocated when it takes at most half of the device's free memory, else left out.
void ensure_gamma_tape(tdse_batch* b, int kc)
{
    const size_t need = (size_t)b->ctas * kc * (size_t)b->warps * b->rows * kLanes * sizeof(double2);
    if (b->d_gtape && b->gtape_bytes == need) return;
    cudaFree(b->d_gtape);
    b->d_gtape = nullptr;
    b->gtape_bytes = 0;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || need > free_b / 2) {
        cudaGetLastError();
        return;
    }
    if (cudaMalloc(&b->d_gtape, need) != cudaSuccess) {
        cudaGetLastError();
        b->d_gtape = nullptr;
        return;
    }
    b->gtape_bytes = need;
}

}  // namespace

namespace tdse {
int batch_device(const tdse_batch* b) { return b->device; }
}  // namespace tdse

extern "C" {

const char* tdse_last_error(void) { return g_last_error.c_str(); }

tdse_status tdse_batch_create(const tdse_instance* inst_host, int64_t n_inst, double dt, const int64_t* n_steps_host,
                              const int64_t* row_offsets_host, const tdse_absorber* absorber,
                              tdse_precision precision, tdse_scheme scheme, int device, tdse_batch** out)
{
    if (!out) return fail(TDSE_ERR_ARG, "tdse_batch_create: out is NULL");
    *out = nullptr;
    if (!inst_host || !n_steps_host || !row_offsets_host) return fail(TDSE_ERR_ARG, "tdse_batch_create: NULL array");
    if (n_inst < 1 || n_inst > (int64_t(1) << 31)) return fail(TDSE_ERR_ARG, "tdse_batch_create: n_inst out of range");
    if (!is_finite(dt) || dt == 0.0) return fail(TDSE_ERR_ARG, "tdse_batch_create: dt must be finite and non-zero");
    if (precision != TDSE_FP64 && precision != TDSE_MIXED) return fail(TDSE_ERR_ARG, "tdse_batch_create: unknown precision");
    if (scheme != TDSE_FULL_CN && scheme != TDSE_NUMEROV_SPLIT) return fail(TDSE_ERR_ARG, "tdse_batch_create: unknown scheme");
    if (absorber && (!is_finite(absorber->width) || !is_finite(absorber->exponent) || absorber->exponent < 0.0))
        return fail(TDSE_ERR_ARG, "tdse_batch_create: bad absorber");
    if (row_offsets_host[0] < 0) return fail(TDSE_ERR_ARG, "tdse_batch_create: row_offsets[0] < 0");
    for (int64_t i = 0; i < n_inst; ++i) {
        const tdse_instance& I = inst_host[i];
        if (I.N < 16 || I.N > (1 << 20)) return fail(TDSE_ERR_ARG, "tdse_batch_create: N out of [16, 2^20] at instance " + std::to_string(i));
        if (!is_finite(I.dx) || I.dx <= 0.0) return fail(TDSE_ERR_ARG, "tdse_batch_create: dx <= 0 at instance " + std::to_string(i));
        if (!is_finite(I.softening) || I.softening <= 0.0) return fail(TDSE_ERR_ARG, "tdse_batch_create: softening <= 0 at instance " + std::to_string(i));
        if (!is_finite(I.charge)) return fail(TDSE_ERR_ARG, "tdse_batch_create: non-finite charge");
        if (n_steps_host[i] < 0) return fail(TDSE_ERR_ARG, "tdse_batch_create: negative n_steps");
        if (row_offsets_host[i + 1] < row_offsets_host[i]) return fail(TDSE_ERR_ARG, "tdse_batch_create: row_offsets decreasing");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(TDSE_ERR_ARG, "tdse_batch_create: no such CUDA device");
    DeviceGuard guard(device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "tdse_batch_create: cudaSetDevice failed");

    tdse_batch* b = new tdse_batch();
    b->device = device;
    b->n_inst = n_inst;
    b->dt = dt;
    b->precision = precision;
    b->scheme = scheme;
    b->mask_on = absorber && absorber->width > 0.0;
    b->mask_width = absorber ? absorber->width : 0.0;
    b->mask_exp = absorber ? absorber->exponent : 0.0;
    b->inst.assign(inst_host, inst_host + n_inst);
    b->n_steps.assign(n_steps_host, n_steps_host + n_inst);
    b->row_off.assign(row_offsets_host, row_offsets_host + n_inst + 1);

    build_classes(b, inst_host, n_inst, dt);
    const int n_cls = (int)b->classes.size();
    // mask plateau [jm_lo, jm_hi] and table offsets
    int64_t tab_total = 0;
    int max_N = 0;
    for (auto& C : b->classes) {
        C.tab_off = tab_total;
        tab_total += tab_doubles(C.N);
        max_N = std::max(max_N, C.N);
        C.jm_lo = 0;
        C.jm_hi = C.N - 1;
        if (b->mask_on) {
            const double xb = 0.5 * C.N * C.dx - b->mask_width;
            int lo_j = C.N, hi_j = -1;
            for (int j = 0; j < C.N; ++j) {
                const double x = (j - 0.5 * (C.N - 1)) * C.dx;
                if (!(std::fabs(x) > xb)) {
                    lo_j = std::min(lo_j, j);
                    hi_j = std::max(hi_j, j);
                }
            }
            C.jm_lo = lo_j;
            C.jm_hi = hi_j;   // empty plateau (lo > hi) masks every point
        }
    }
    // device allocations
    tdse_status st = TDSE_OK;
    auto bail = [&](tdse_status s) {
        free_device(b);
        delete b;
        return s;
    };
    cudaError_t e;
    if ((e = dev_alloc(&b->d_cls, n_cls)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(classes)"));
    if ((e = dev_alloc(&b->d_tab, (size_t)tab_total)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(tables)"));
    if ((e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaDeviceGetAttribute"));
    int64_t gs_total = 0;
    std::vector<int64_t> gs_off(n_cls);
    for (int c = 0; c < n_cls; ++c) {
        gs_off[c] = gs_total;
        gs_total += kGsWork * (int64_t)b->classes[c].N;
    }
    if ((e = dev_alloc(&b->d_gs_work, (size_t)gs_total)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(gs)"));
    if ((e = dev_alloc(&b->d_gs_off, (size_t)n_cls)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(gs)"));
    if ((e = dev_alloc(&b->d_gs_energy, (size_t)n_cls)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(gs)"));
    if ((e = dev_alloc(&b->d_gs_iters, (size_t)n_cls)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(gs)"));
    if ((e = dev_alloc(&b->d_gs_support, 2 * (size_t)n_cls)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(gs)"));
    if ((e = cudaMemcpy(b->d_cls, b->classes.data(), sizeof(ClassDesc) * n_cls, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_gs_off, gs_off.data(), sizeof(int64_t) * n_cls, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMemcpy(setup)"));
    if ((e = launch_build_tables(b->d_cls, n_cls, max_N, dt, b->mask_width, b->mask_exp, b->mask_on, b->d_tab, 0)) != cudaSuccess)
        return bail(cuda_fail(e, "build_tables launch"));
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(cuda_fail(e, "build_tables"));
    if (scheme == TDSE_NUMEROV_SPLIT) {
        std::vector<double> nw, nl, nc;
        std::vector<float> nf;
        for (auto& C : b->classes) {
            C.rho = numerov_factors(C, dt, nw, nl, nc, nf);
            if ((e = cudaMemcpy(b->d_tab + tab_nw(C), nw.data(), sizeof(double) * nw.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(b->d_tab + tab_nl(C), nl.data(), sizeof(double) * nl.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(b->d_tab + tab_nc(C), nc.data(), sizeof(double) * nc.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(b->d_tab + tab_nf(C), nf.data(), sizeof(float) * nf.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
                return bail(cuda_fail(e, "cudaMemcpy(numerov tables)"));
        }
        if ((e = cudaMemcpy(b->d_cls, b->classes.data(), sizeof(ClassDesc) * n_cls, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMemcpy(classes)"));
    }
    // the grouping (lanes per instance) needs each class's halo, which for NUMEROV_SPLIT comes from
    // the factors just computed
    if ((st = build_groups(b)) != TDSE_OK) return bail(st);
    if ((st = build_plan(b)) != TDSE_OK) return bail(st);
    *out = b;
    return TDSE_OK;
}

void tdse_batch_destroy(tdse_batch* b)
{
    if (!b) return;
    DeviceGuard guard(b->device);
    cudaDeviceSynchronize();
    free_device(b);
    delete b;
}

tdse_status tdse_plan(const tdse_batch* b, tdse_plan_info* info)
{
    if (!b || !info) return fail(TDSE_ERR_ARG, "tdse_plan: NULL argument");
    info->n_groups = (int64_t)b->groups.size();
    info->segments = b->class_P.empty() ? 0 : *std::max_element(b->class_P.begin(), b->class_P.end());
    info->halo = b->class_K.empty() ? 0 : *std::max_element(b->class_K.begin(), b->class_K.end());
    info->warps_per_cta = b->warps;
    info->ctas = b->ctas;
    info->slice_steps = b->slice;
    info->scratch_bytes = b->scratch_elems * (int64_t)b->cx_bytes();
    info->psi_bytes = b->psi_elems * (int64_t)b->cx_bytes();
    info->lanes_per_instance = b->class_L.empty() ? 1 : *std::max_element(b->class_L.begin(), b->class_L.end());
    info->longest_share = b->longest_share;
    return TDSE_OK;
}

tdse_status tdse_model_layout(const tdse_instance* inst_host, int64_t n_inst, double dt, tdse_precision precision,
                              tdse_scheme scheme, int32_t sm_count, int32_t* lanes_out)
{
    if (!inst_host || !lanes_out) return fail(TDSE_ERR_ARG, "tdse_model_layout: NULL argument");
    if (n_inst < 1 || n_inst > (int64_t(1) << 31)) return fail(TDSE_ERR_ARG, "tdse_model_layout: n_inst out of range");
    if (!is_finite(dt) || dt == 0.0) return fail(TDSE_ERR_ARG, "tdse_model_layout: dt must be finite and non-zero");
    if (precision != TDSE_FP64 && precision != TDSE_MIXED) return fail(TDSE_ERR_ARG, "tdse_model_layout: unknown precision");
    if (scheme != TDSE_FULL_CN && scheme != TDSE_NUMEROV_SPLIT) return fail(TDSE_ERR_ARG, "tdse_model_layout: unknown scheme");
    if (sm_count < 1 || sm_count > 4096) return fail(TDSE_ERR_ARG, "tdse_model_layout: sm_count out of [1, 4096]");
    for (int64_t i = 0; i < n_inst; ++i) {
        const tdse_instance& I = inst_host[i];
        if (I.N < 16 || I.N > (1 << 20) || !is_finite(I.dx) || I.dx <= 0.0 || !is_finite(I.softening) ||
            I.softening <= 0.0 || !is_finite(I.charge))
            return fail(TDSE_ERR_ARG, "tdse_model_layout: bad instance " + std::to_string(i));
    }
    tdse_batch tmp;   // host fields only: no device state is created
    tmp.n_inst = n_inst;
    tmp.dt = dt;
    tmp.precision = precision;
    tmp.scheme = scheme;
    tmp.sm_count = sm_count;
    build_classes(&tmp, inst_host, n_inst, dt);
    if (scheme == TDSE_NUMEROV_SPLIT) {
        std::vector<double> nw, nl, nc;
        std::vector<float> nf;
        for (auto& C : tmp.classes) C.rho = numerov_factors(C, dt, nw, nl, nc, nf);
    }
    std::vector<int64_t> count(tmp.classes.size(), 0);
    for (int64_t i = 0; i < n_inst; ++i) ++count[tmp.inst_class[i]];
    *lanes_out = model_lanes(&tmp, count);
    return TDSE_OK;
}

tdse_status tdse_set_adjoint_gamma_tape(tdse_batch* b, int32_t enable)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_set_adjoint_gamma_tape: NULL batch");
    if (enable != 0 && enable != 1) return fail(TDSE_ERR_ARG, "tdse_set_adjoint_gamma_tape: enable must be 0 or 1");
    b->use_gtape = enable != 0;
    if (!b->use_gtape && b->d_gtape) {
        DeviceGuard guard(b->device);
        if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
        TDSE_CUDA(cudaDeviceSynchronize(), "tdse_set_adjoint_gamma_tape: synchronize");
        cudaFree(b->d_gtape);
        b->d_gtape = nullptr;
        b->gtape_bytes = 0;
    }
    return TDSE_OK;
}

tdse_status tdse_set_wait_limit(tdse_batch* b, int64_t polls)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_set_wait_limit: NULL batch");
    if (polls < 0 || polls > (int64_t(1) << 30)) return fail(TDSE_ERR_ARG, "tdse_set_wait_limit: polls out of [0, 2^30]");
    b->wait_polls = (uint32_t)polls;
    return TDSE_OK;
}

tdse_status tdse_set_layout(tdse_batch* b, int32_t lanes_per_instance)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_set_layout: NULL batch");
    const int L = lanes_per_instance;
    if (L < 0 || L > kLanes || (L & (L - 1)) != 0)
        return fail(TDSE_ERR_ARG, "tdse_set_layout: lanes_per_instance must be 0, 1, 2, 4, 8, 16 or 32");
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    TDSE_CUDA(cudaDeviceSynchronize(), "tdse_set_layout: synchronize");
    b->lanes_request = L;
    tdse_status st = build_groups(b);
    if (st != TDSE_OK) return st;
    return build_plan(b);
}

tdse_status tdse_set_launch(tdse_batch* b, int32_t warps_per_cta, int32_t ctas_per_sm, int32_t slice_steps,
                            int32_t max_ctas)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_set_launch: NULL batch");
    if (warps_per_cta < 0 || warps_per_cta > kMaxSegments) return fail(TDSE_ERR_ARG, "tdse_set_launch: warps_per_cta out of [0, 16]");
    if (ctas_per_sm < 0 || ctas_per_sm > 32) return fail(TDSE_ERR_ARG, "tdse_set_launch: ctas_per_sm out of [0, 32]");
    if (slice_steps < 0) return fail(TDSE_ERR_ARG, "tdse_set_launch: slice_steps < 0");
    if (max_ctas < 0) return fail(TDSE_ERR_ARG, "tdse_set_launch: max_ctas < 0");
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    TDSE_CUDA(cudaDeviceSynchronize(), "tdse_set_launch: synchronize");
    b->warps_override = warps_per_cta;
    b->ctas_per_sm_override = ctas_per_sm;
    b->slice_override = slice_steps;
    b->max_ctas_override = max_ctas;
    return build_plan(b);
}

tdse_status tdse_ground_state(tdse_batch* b, double dtau, int64_t max_iter, double tol, double* energies_host,
                              int64_t* iters_host, void* stream)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_ground_state: NULL batch");
    if (!is_finite(dtau) || dtau <= 0.0) return fail(TDSE_ERR_ARG, "tdse_ground_state: dtau must be > 0");
    if (max_iter < 1) return fail(TDSE_ERR_ARG, "tdse_ground_state: max_iter < 1");
    if (!is_finite(tol) || tol < 0.0) return fail(TDSE_ERR_ARG, "tdse_ground_state: tol must be >= 0");
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    const int n_cls = (int)b->classes.size();
    TDSE_CUDA(launch_ground_state(b->d_cls, n_cls, (int)b->scheme, dtau, max_iter, tol, b->d_gs_work, b->d_gs_off,
                                  b->d_gs_energy, b->d_gs_iters, st),
              "ground_state launch");
    TDSE_CUDA(launch_gs_support(b->d_cls, n_cls, b->d_gs_work, b->d_gs_off, b->d_gs_support, st), "support launch");
    TDSE_CUDA(launch_broadcast_psi(b->mixed(), b->d_groups, (int64_t)b->groups.size(), b->d_gs_work, b->d_gs_off,
                                   b->d_slot_valid, b->d_psi, st),
              "broadcast launch");
    b->initialized = true;
    b->gs_done = true;
    if (energies_host || iters_host) {
        std::vector<double> e(n_cls);
        std::vector<int64_t> it(n_cls);
        TDSE_CUDA(cudaMemcpyAsync(e.data(), b->d_gs_energy, sizeof(double) * n_cls, cudaMemcpyDeviceToHost, st), "copy energies");
        TDSE_CUDA(cudaMemcpyAsync(it.data(), b->d_gs_iters, sizeof(int64_t) * n_cls, cudaMemcpyDeviceToHost, st), "copy iters");
        TDSE_CUDA(cudaStreamSynchronize(st), "ground_state");
        for (int64_t i = 0; i < b->n_inst; ++i) {
            if (energies_host) energies_host[i] = e[b->inst_class[i]];
            if (iters_host) iters_host[i] = it[b->inst_class[i]];
        }
    }
    return TDSE_OK;
}

static tdse_status propagate_impl(tdse_batch* b, const double* E_dev, double* d_dev, double* a_dev, int64_t sample_base,
                                  int64_t step_begin, int64_t step_end, void* stream, int ckpt_every)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_propagate: NULL batch");
    if (!E_dev || !d_dev || !a_dev) return fail(TDSE_ERR_ARG, "tdse_propagate: NULL buffer");
    if (step_begin < 0 || step_end < step_begin) return fail(TDSE_ERR_ARG, "tdse_propagate: bad step range");
    if (sample_base < 0 || sample_base > step_begin) return fail(TDSE_ERR_ARG, "tdse_propagate: need 0 <= sample_base <= step_begin");
    if (!b->initialized) return fail(TDSE_ERR_STATE, "tdse_propagate: no initial state (call tdse_ground_state or tdse_set_psi)");
    for (int64_t i = 0; i < b->n_inst; ++i) {
        const int64_t n_end = std::min(step_end, b->n_steps[i]);
        int64_t top = -1;
        if (step_begin == 0) top = 0;
        if (n_end > step_begin) top = n_end;
        if (top < 0) continue;
        const int64_t len = b->row_off[i + 1] - b->row_off[i];
        if (top - sample_base >= len)
            return fail(TDSE_ERR_ARG, "tdse_propagate: row of instance " + std::to_string(i) + " too short for the step range");
    }
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    if (b->scheme == TDSE_NUMEROV_SPLIT)
        TDSE_CUDA(launch_propagate_numerov(b->mixed(), b->d_groups, (int64_t)b->groups.size(), b->warps, b->ctas,
                                           b->d_cls, b->d_tab, b->d_slot_row, b->d_slot_nt, b->d_psi, b->d_scratch,
                                           b->rows, E_dev, d_dev, a_dev, sample_base, step_begin, step_end, b->slice,
                                           b->mask_on, b->dt, b->d_busy, b->d_progress, b->d_status, st),
                  "propagate launch");
    else
        TDSE_CUDA(launch_propagate_full_cn(b->mixed(), b->d_groups, (int64_t)b->groups.size(), b->warps, b->ctas,
                                           b->d_cls, b->d_tab, b->d_slot_row, b->d_slot_nt, b->d_psi, b->d_scratch,
                                           b->rows, E_dev, d_dev, a_dev, sample_base, step_begin, step_end, b->slice,
                                           b->mask_on, b->d_busy, b->d_progress, b->d_status, b->ring, b->wait_polls, st,
                                           ckpt_every > 0 ? b->d_ckpt : nullptr, b->d_ckpt_off, ckpt_every),
                  "propagate launch");
    return TDSE_OK;
}

tdse_status tdse_propagate(tdse_batch* b, const double* E_dev, double* d_dev, double* a_dev, int64_t sample_base,
                           int64_t step_begin, int64_t step_end, void* stream)
{
    return propagate_impl(b, E_dev, d_dev, a_dev, sample_base, step_begin, step_end, stream, 0);
}

static tdse_status locate(const tdse_batch* b, int64_t inst, int64_t* off, int* N, int* lane, int* I)
{
    if (inst < 0 || inst >= b->n_inst) return fail(TDSE_ERR_ARG, "instance index out of range");
    const int64_t slot = b->slot_of_inst[inst];
    const GroupDesc& G = b->groups[b->slot_group[slot]];
    *off = G.psi_off;
    *N = G.N;
    *lane = (int)(slot - G.slot0);
    *I = G.I;
    return TDSE_OK;
}

tdse_status tdse_get_psi(tdse_batch* b, int64_t inst, double* psi_dev, void* stream)
{
    if (!b || !psi_dev) return fail(TDSE_ERR_ARG, "tdse_get_psi: NULL argument");
    int64_t off;
    int N, lane, I;
    tdse_status s = locate(b, inst, &off, &N, &lane, &I);
    if (s != TDSE_OK) return s;
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    TDSE_CUDA(launch_get_psi(b->mixed(), b->d_psi, off, N, lane, I, psi_dev, (cudaStream_t)stream), "get_psi launch");
    return TDSE_OK;
}

tdse_status tdse_set_psi(tdse_batch* b, int64_t inst, const double* psi_dev, void* stream)
{
    if (!b || !psi_dev) return fail(TDSE_ERR_ARG, "tdse_set_psi: NULL argument");
    int64_t off;
    int N, lane, I;
    tdse_status s = locate(b, inst, &off, &N, &lane, &I);
    if (s != TDSE_OK) return s;
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    TDSE_CUDA(launch_set_psi(b->mixed(), b->d_psi, off, N, lane, I, psi_dev, (cudaStream_t)stream), "set_psi launch");
    b->initialized = true;
    return TDSE_OK;
}

tdse_status tdse_check(tdse_batch* b, int64_t* first_bad, void* stream)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_check: NULL batch");
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> flags((size_t)b->n_slots);
    TDSE_CUDA(cudaMemcpyAsync(flags.data(), b->d_status, sizeof(int) * b->n_slots, cudaMemcpyDeviceToHost, st), "copy status");
    TDSE_CUDA(cudaMemsetAsync(b->d_status, 0, sizeof(int) * b->n_slots, st), "clear status");
    TDSE_CUDA(cudaStreamSynchronize(st), "tdse_check");
    int64_t bad = -1;
    int kind = 0;
    for (int64_t i = 0; i < b->n_inst && bad < 0; ++i)
        if (flags[b->slot_of_inst[i]]) {
            bad = i;
            kind = flags[b->slot_of_inst[i]];
        }
    if (first_bad) *first_bad = bad;
    if (bad >= 0 && kind == 2)
        return fail(TDSE_ERR_TIMEOUT, "instance " + std::to_string(bad) + ": a bulk copy wait gave up");
    if (bad >= 0) return fail(TDSE_ERR_NONFINITE, "instance " + std::to_string(bad) + ": norm non-finite or above its rounding allowance");
    return TDSE_OK;
}

tdse_status tdse_copy_state(tdse_batch* b, void* buffer_dev, int32_t direction, void* stream)
{
    if (!b || !buffer_dev) return fail(TDSE_ERR_ARG, "tdse_copy_state: NULL argument");
    if (direction != 0 && direction != 1) return fail(TDSE_ERR_ARG, "tdse_copy_state: direction must be 0 or 1");
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    const size_t bytes = (size_t)b->psi_elems * b->cx_bytes();
    if (direction == 0)
        TDSE_CUDA(cudaMemcpyAsync(buffer_dev, b->d_psi, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "tdse_copy_state");
    else {
        TDSE_CUDA(cudaMemcpyAsync(b->d_psi, buffer_dev, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "tdse_copy_state");
        b->initialized = true;
    }
    return TDSE_OK;
}

tdse_status tdse_adjoint(tdse_batch* b, const double* E_dev, const double* gd_dev, const double* ga_dev, double* gE_dev,
                         int32_t ckpt_every, void* stream)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_adjoint: NULL batch");
    if (!E_dev || !gd_dev || !ga_dev || !gE_dev) return fail(TDSE_ERR_ARG, "tdse_adjoint: NULL buffer");
    if (b->precision != TDSE_FP64 || b->scheme != TDSE_FULL_CN)
        return fail(TDSE_ERR_ARG, "tdse_adjoint: only FP64 FULL_CN batches have an adjoint");
    if (ckpt_every < 1 || ckpt_every > 65536) return fail(TDSE_ERR_ARG, "tdse_adjoint: ckpt_every out of [1, 65536]");
    if (!b->initialized) return fail(TDSE_ERR_STATE, "tdse_adjoint: no initial state");
    for (int64_t i = 0; i < b->n_inst; ++i)
        if (b->row_off[i + 1] - b->row_off[i] < b->n_steps[i] + 1)
            return fail(TDSE_ERR_ARG, "tdse_adjoint: row of instance " + std::to_string(i) + " shorter than Nt + 1");
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    int n_max = 1;
    tdse_status s = ensure_adjoint_buffers(b, ckpt_every, st, &n_max);
    if (s != TDSE_OK) return s;
    b->ckpt_next = -1;   // the adjoint's own forward pass rewrites the checkpoints
    if (b->use_gtape) ensure_gamma_tape(b, ckpt_every);
    TDSE_CUDA(launch_adjoint_full_cn(b->d_groups, (int64_t)b->groups.size(), b->warps, b->ctas, b->d_cls, b->d_tab,
                                     b->d_slot_row, b->d_slot_nt, b->d_psi, b->d_lam, b->d_ckpt, b->d_ckpt_off,
                                     b->d_work, b->d_tape, b->d_scratch, b->rows, n_max, ckpt_every, E_dev, gd_dev,
                                     ga_dev, gE_dev, b->mask_on, b->d_busy, b->d_progress, st, 0,
                                     b->use_gtape ? b->d_gtape : nullptr),
              "adjoint launch");
    return TDSE_OK;
}

tdse_status tdse_propagate_checkpointed(tdse_batch* b, const double* E_dev, double* d_dev, double* a_dev,
                                        int64_t sample_base, int64_t step_begin, int64_t step_end, int32_t ckpt_every,
                                        void* stream)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_propagate_checkpointed: NULL batch");
    if (b->precision != TDSE_FP64 || b->scheme != TDSE_FULL_CN)
        return fail(TDSE_ERR_ARG, "tdse_propagate_checkpointed: only FP64 FULL_CN batches have an adjoint");
    if (ckpt_every < 1 || ckpt_every > 65536) return fail(TDSE_ERR_ARG, "tdse_propagate_checkpointed: ckpt_every out of [1, 65536]");
    if (step_begin != 0 && (b->ckpt_next != step_begin || b->adj_kc != ckpt_every))
        return fail(TDSE_ERR_STATE, "tdse_propagate_checkpointed: a recording starts at step 0 and continues where the "
                                    "previous checkpointed call ended, with the same ckpt_every");
    {
        DeviceGuard guard(b->device);
        if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
        int n_max = 1;
        const int64_t before = b->ckpt_next;
        tdse_status s = ensure_adjoint_buffers(b, ckpt_every, (cudaStream_t)stream, &n_max);
        if (s != TDSE_OK) return s;
        if (step_begin != 0 && b->ckpt_next != before)
            return fail(TDSE_ERR_STATE, "tdse_propagate_checkpointed: the launch shape changed during the recording");
    }
    tdse_status s = propagate_impl(b, E_dev, d_dev, a_dev, sample_base, step_begin, step_end, stream, ckpt_every);
    if (s != TDSE_OK) {
        b->ckpt_next = -1;
        return s;
    }
    b->ckpt_next = step_end;
    return TDSE_OK;
}

tdse_status tdse_adjoint_checkpointed(tdse_batch* b, const double* E_dev, const double* gd_dev, const double* ga_dev,
                                      double* gE_dev, void* stream)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_adjoint_checkpointed: NULL batch");
    if (!E_dev || !gd_dev || !ga_dev || !gE_dev) return fail(TDSE_ERR_ARG, "tdse_adjoint_checkpointed: NULL buffer");
    if (b->precision != TDSE_FP64 || b->scheme != TDSE_FULL_CN)
        return fail(TDSE_ERR_ARG, "tdse_adjoint_checkpointed: only FP64 FULL_CN batches have an adjoint");
    for (int64_t i = 0; i < b->n_inst; ++i)
        if (b->row_off[i + 1] - b->row_off[i] < b->n_steps[i] + 1)
            return fail(TDSE_ERR_ARG, "tdse_adjoint_checkpointed: row of instance " + std::to_string(i) + " shorter than Nt + 1");
    if (b->adj_kc < 1) return fail(TDSE_ERR_STATE, "tdse_adjoint_checkpointed: nothing recorded");
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    int n_max = 1;
    // the recording allocated the buffers; a changed launch shape reallocates them and drops it
    tdse_status s = ensure_adjoint_buffers(b, b->adj_kc, st, &n_max);
    if (s != TDSE_OK) return s;
    int64_t nt_all = 0;
    for (int64_t i = 0; i < b->n_inst; ++i) nt_all = std::max(nt_all, b->n_steps[i]);
    if (b->ckpt_next < nt_all || !b->d_ckpt)
        return fail(TDSE_ERR_STATE, "tdse_adjoint_checkpointed: no complete checkpointed forward propagation "
                                    "(tdse_propagate_checkpointed from step 0 through every instance's last step)");
    if (b->use_gtape) ensure_gamma_tape(b, b->adj_kc);
    TDSE_CUDA(launch_adjoint_full_cn(b->d_groups, (int64_t)b->groups.size(), b->warps, b->ctas, b->d_cls, b->d_tab,
                                     b->d_slot_row, b->d_slot_nt, b->d_psi, b->d_lam, b->d_ckpt, b->d_ckpt_off,
                                     b->d_work, b->d_tape, b->d_scratch, b->rows, n_max, b->adj_kc, E_dev, gd_dev,
                                     ga_dev, gE_dev, b->mask_on, b->d_busy, b->d_progress, st, 1,
                                     b->use_gtape ? b->d_gtape : nullptr),
              "adjoint launch");
    return TDSE_OK;
}


tdse_status tdse_energy_distribution(tdse_batch* b, const double* E_grid_host, int32_t n_energies, double epsilon,
                                     double* P_dev, void* stream)
{
    if (!b) return fail(TDSE_ERR_ARG, "tdse_energy_distribution: NULL batch");
    if (n_energies < 0 || n_energies > (1 << 20)) return fail(TDSE_ERR_ARG, "tdse_energy_distribution: n_energies out of [0, 2^20]");
    if (n_energies > 0 && (!E_grid_host || !P_dev)) return fail(TDSE_ERR_ARG, "tdse_energy_distribution: NULL buffer");
    if (!is_finite(epsilon) || !(epsilon >= 1e-12)) return fail(TDSE_ERR_ARG, "tdse_energy_distribution: epsilon must be >= 1e-12");
    for (int k = 0; k < n_energies; ++k)
        if (!is_finite(E_grid_host[k]) || std::fabs(E_grid_host[k]) > 1e12)
            return fail(TDSE_ERR_ARG, "tdse_energy_distribution: energy " + std::to_string(k) + " not finite or beyond 1e12");
    if (!b->initialized) return fail(TDSE_ERR_STATE, "tdse_energy_distribution: no state");
    if (n_energies == 0) return TDSE_OK;
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    const int n_cls = (int)b->classes.size();
    const int nE_pad = (n_energies + kLanes - 1) / kLanes * kLanes;
    std::vector<int64_t> piv_off(n_cls);
    int64_t piv_elems = 0;
    int n_max = 1;
    for (int c = 0; c < n_cls; ++c) {
        piv_off[c] = piv_elems;
        piv_elems += (int64_t)b->classes[c].N * nE_pad;
        n_max = std::max(n_max, b->classes[c].N);
    }
    const int64_t sc = energy_distribution_scratch_elems(b->sm_count, n_max);
    if (sc > b->ed_scratch_elems) {
        TDSE_CUDA(cudaStreamSynchronize(st), "tdse_energy_distribution: synchronize");
        cudaFree(b->d_ed_scratch);
        b->d_ed_scratch = nullptr;
        b->ed_scratch_elems = 0;
        TDSE_CUDA(cudaMalloc(&b->d_ed_scratch, sizeof(double2) * (size_t)sc), "cudaMalloc(energy distribution scratch)");
        b->ed_scratch_elems = sc;
    }
    // per-call buffers: energies, pivot tables and their offsets (freed after the stream drains)
    double* d_E = nullptr;
    void* d_piv = nullptr;
    int64_t* d_off = nullptr;
    auto release = [&]() {
        cudaFree(d_E);
        cudaFree(d_piv);
        cudaFree(d_off);
    };
    cudaError_t e = cudaMalloc(&d_E, sizeof(double) * n_energies);
    if (e == cudaSuccess) e = cudaMalloc(&d_piv, sizeof(double2) * 2 * (size_t)piv_elems);
    if (e == cudaSuccess) e = cudaMalloc(&d_off, sizeof(int64_t) * n_cls);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_E, E_grid_host, sizeof(double) * n_energies, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, piv_off.data(), sizeof(int64_t) * n_cls, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_energy_distribution(b->mixed(), b->d_groups, b->d_cls, n_cls, b->d_tab, b->d_slot_group,
                                       b->d_slot_inst, b->n_slots, b->d_psi, d_E, n_energies, epsilon, (int)b->scheme,
                                       d_piv, d_off, piv_elems, b->d_ed_scratch, n_max, b->sm_count, P_dev, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_fail(e, "tdse_energy_distribution");
    return TDSE_OK;
}

tdse_status tdse_ionisation(tdse_batch* b, const double* E_nodes_host, int32_t n_nodes, double epsilon,
                            double* P_dev, double* ion_dev, void* stream)
{
    if (!b || !E_nodes_host || !ion_dev) return fail(TDSE_ERR_ARG, "tdse_ionisation: NULL argument");
    if (n_nodes < 2 || n_nodes > (1 << 20)) return fail(TDSE_ERR_ARG, "tdse_ionisation: n_nodes out of [2, 2^20]");
    for (int k = 1; k < n_nodes; ++k)
        if (!(E_nodes_host[k] > E_nodes_host[k - 1]))
            return fail(TDSE_ERR_ARG, "tdse_ionisation: energy nodes must be strictly ascending (node " + std::to_string(k) + ")");
    if (!b->initialized) return fail(TDSE_ERR_STATE, "tdse_ionisation: no state");
    // trapezoid weights of the nodes
    std::vector<double> w(n_nodes);
    w[0] = 0.5 * (E_nodes_host[1] - E_nodes_host[0]);
    w[n_nodes - 1] = 0.5 * (E_nodes_host[n_nodes - 1] - E_nodes_host[n_nodes - 2]);
    for (int k = 1; k < n_nodes - 1; ++k) w[k] = 0.5 * (E_nodes_host[k + 1] - E_nodes_host[k - 1]);
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    double* d_w = nullptr;
    double* d_P = nullptr;
    auto release = [&]() {
        cudaFree(d_w);
        if (!P_dev) cudaFree(d_P);
    };
    cudaError_t e = cudaMalloc(&d_w, sizeof(double) * n_nodes);
    if (e == cudaSuccess && !P_dev) e = cudaMalloc(&d_P, sizeof(double) * (size_t)b->n_inst * n_nodes);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "tdse_ionisation: cudaMalloc");
    }
    double* P = P_dev ? P_dev : d_P;
    tdse_status s = tdse_energy_distribution(b, E_nodes_host, n_nodes, epsilon, P, stream);   // synchronises
    if (s != TDSE_OK) {
        release();
        return s;
    }
    e = cudaMemcpyAsync(d_w, w.data(), sizeof(double) * n_nodes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_ionisation(P, b->n_inst, n_nodes, d_w, ion_dev, b->sm_count, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_fail(e, "tdse_ionisation");
    return TDSE_OK;
}

tdse_status tdse_populations(tdse_batch* b, double r_core, double* out_dev, void* stream)
{
    if (!b || !out_dev) return fail(TDSE_ERR_ARG, "tdse_populations: NULL argument");
    if (std::isnan(r_core) || r_core < 0.0) return fail(TDSE_ERR_ARG, "tdse_populations: r_core must be >= 0");
    if (!b->gs_done) return fail(TDSE_ERR_STATE, "tdse_populations: no ground state (call tdse_ground_state)");
    if (!b->initialized) return fail(TDSE_ERR_STATE, "tdse_populations: no state (the layout changed since)");
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    TDSE_CUDA(launch_populations(b->mixed(), b->d_groups, (int64_t)b->groups.size(), b->d_cls,
                                 b->d_slot_inst, b->d_psi, b->d_gs_work, b->d_gs_off, b->d_gs_support, r_core,
                                 out_dev, b->sm_count, (cudaStream_t)stream),
              "populations launch");
    return TDSE_OK;
}

tdse_status tdse_resample_field(const double* coarse_dev, int64_t n_rows, int32_t M, double dt_coarse, double dt_fine,
                                int64_t n_fine, int64_t out_stride, double* out_dev, int device, void* stream)
{
    if (!coarse_dev || !out_dev) return fail(TDSE_ERR_ARG, "tdse_resample_field: NULL buffer");
    if (n_rows < 1 || n_rows > (int64_t(1) << 31)) return fail(TDSE_ERR_ARG, "tdse_resample_field: n_rows out of range");
    if (M < 2 || M > 8192) return fail(TDSE_ERR_ARG, "tdse_resample_field: M out of [2, 8192]");
    if (!is_finite(dt_coarse) || !(dt_coarse > 0.0) || !is_finite(dt_fine) || !(dt_fine > 0.0))
        return fail(TDSE_ERR_ARG, "tdse_resample_field: steps must be finite and > 0");
    if (n_fine < 1 || out_stride < n_fine) return fail(TDSE_ERR_ARG, "tdse_resample_field: need 1 <= n_fine <= out_stride");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(TDSE_ERR_ARG, "tdse_resample_field: no such CUDA device");
    DeviceGuard guard(device);
    if (!guard.ok) return fail(TDSE_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    void* d_coef = nullptr;
    cudaError_t e = cudaMalloc(&d_coef, sizeof(double2) * (size_t)n_rows * (M / 2 + 1));
    if (e == cudaSuccess) e = launch_resample_field(coarse_dev, n_rows, M, dt_coarse, dt_fine, n_fine, out_stride, out_dev,
                                                    d_coef, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_coef);
    if (e != cudaSuccess) return cuda_fail(e, "tdse_resample_field");
    return TDSE_OK;
}

tdse_status tdse_spectrum(const double* a_dev, const int64_t* offsets_host, int64_t n_rows, double dt, int64_t k_begin,
                          int64_t k_end, double* S_dev, void* stream)
{
    if (!a_dev || !offsets_host || !S_dev) return fail(TDSE_ERR_ARG, "tdse_spectrum: NULL argument");
    if (n_rows < 1 || n_rows > (int64_t(1) << 31)) return fail(TDSE_ERR_ARG, "tdse_spectrum: n_rows out of range");
    if (k_begin < 0 || k_end <= k_begin) return fail(TDSE_ERR_ARG, "tdse_spectrum: need 0 <= k_begin < k_end");
    if (!is_finite(dt)) return fail(TDSE_ERR_ARG, "tdse_spectrum: dt not finite");
    for (int64_t r = 0; r < n_rows; ++r)
        if (offsets_host[r + 1] < offsets_host[r] || offsets_host[r] < 0)
            return fail(TDSE_ERR_ARG, "tdse_spectrum: offsets must be non-decreasing and >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t* d_off = nullptr;
    TDSE_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d_off), sizeof(int64_t) * (n_rows + 1), st), "cudaMallocAsync(offsets)");
    cudaError_t e = cudaMemcpyAsync(d_off, offsets_host, sizeof(int64_t) * (n_rows + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_spectrum(a_dev, d_off, n_rows, dt, k_begin, k_end, S_dev, st);
    cudaError_t e2 = cudaFreeAsync(d_off, st);
    if (e != cudaSuccess) return cuda_fail(e, "tdse_spectrum");
    if (e2 != cudaSuccess) return cuda_fail(e2, "tdse_spectrum free");
    return TDSE_OK;
}

}  // extern "C"
