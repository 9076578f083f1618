// tdse_propagate_static: the FULL_CN FP64 propagation for callers that cannot allocate device
// memory.  Everything the kernel needs beyond the caller's buffers (tables, scheduler state, group
// descriptors, solver scratch) lives in one file-scope __device__ array of fixed size, so the
// library holds that much memory on every GPU it touches until the process exits.
#include "tdse.h"
#include "tdse_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

using namespace tdse;

namespace {

constexpr size_t kStaticBytes = size_t(64) << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code this name is only a stand-in for the symbol: its device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_mutex;
void* g_static_ptr[kMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

tdse_status err(tdse_status st, const char* msg)
{
    set_error_message(msg);
    return st;
}

// Device address of the static scratch on the current device (set up on the first call per device).
tdse_status static_scratch(int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices) return err(TDSE_ERR_ARG, "tdse_propagate_static: device ordinal too large");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) return err(TDSE_ERR_CUDA, "tdse_propagate_static: cudaGetSymbolAddress failed");
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return TDSE_OK;
}

// Descriptors of a uniform batch written straight into the static scratch.
__global__ void k_static_setup(ClassDesc C, int64_t n_inst, int64_t n_groups, int64_t nt, int64_t row_stride,
                               int P, int K, int m, ClassDesc* cls, GroupDesc* groups, int64_t* slot_row,
                               int64_t* slot_nt, int* status)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0) cls[0] = C;
    for (int64_t g = tid; g < n_groups; g += stride) {
        GroupDesc G{};
        G.psi_off = g * (int64_t)C.N * kLanes;
        G.slot0 = g * kLanes;
        G.nt_max = nt;
        G.cls = 0;
        G.N = C.N;
        G.P = P;
        G.K = K;
        G.m = m;
        G.I = kLanes;
        G.w = 1;
        groups[g] = G;
    }
    for (int64_t s = tid; s < n_groups * kLanes; s += stride) {
        const bool real = s < n_inst;
        slot_row[s] = real ? s * row_stride : 0;
        slot_nt[s] = real ? nt : -1;
        status[s] = 0;
    }
}

}  // namespace

extern "C" tdse_status tdse_propagate_static(const tdse_instance* inst_host, int64_t n_inst, double dt,
                                             const tdse_absorber* absorber, int64_t n_steps, int64_t row_stride,
                                             double* psi_dev, const double* E_dev, double* d_dev, double* a_dev,
                                             int64_t sample_base, int64_t step_begin, int64_t step_end,
                                             void* stream)
{
    if (!inst_host || !psi_dev || !E_dev || !d_dev || !a_dev) return err(TDSE_ERR_ARG, "tdse_propagate_static: NULL argument");
    const tdse_instance I = *inst_host;
    if (I.N < 16 || I.N > (1 << 20) || !(I.dx > 0.0) || !std::isfinite(I.dx) || !(I.softening > 0.0) ||
        !std::isfinite(I.softening) || !std::isfinite(I.charge))
        return err(TDSE_ERR_ARG, "tdse_propagate_static: bad instance parameters");
    if (n_inst < 1 || n_inst > (int64_t(1) << 31)) return err(TDSE_ERR_ARG, "tdse_propagate_static: n_inst out of range");
    if (!std::isfinite(dt) || dt == 0.0) return err(TDSE_ERR_ARG, "tdse_propagate_static: dt must be finite and non-zero");
    if (n_steps < 0 || step_begin < 0 || step_end < step_begin || sample_base < 0 || sample_base > step_begin)
        return err(TDSE_ERR_ARG, "tdse_propagate_static: bad step range");
    if (absorber && (!std::isfinite(absorber->width) || !std::isfinite(absorber->exponent) || absorber->exponent < 0.0))
        return err(TDSE_ERR_ARG, "tdse_propagate_static: bad absorber");
    const int64_t n_end = std::min(step_end, n_steps);
    const int64_t top = n_end > step_begin ? n_end : (step_begin == 0 ? 0 : -1);
    if (top >= 0 && top - sample_base >= row_stride)
        return err(TDSE_ERR_ARG, "tdse_propagate_static: row_stride too small for the step range");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return err(TDSE_ERR_CUDA, "tdse_propagate_static: no current device");
    void* base = nullptr;
    tdse_status st = static_scratch(dev, &base);
    if (st != TDSE_OK) return st;

    // plan: the same halo rule and segment limit as the allocating path
    ClassDesc C{};
    C.N = I.N;
    C.dx = I.dx;
    C.a = I.softening;
    C.Z = I.charge;
    C.beta = dt / (4.0 * I.dx * I.dx);
    C.one = 1.0;
    C.nzero = -0.0;
    C.tab_off = 0;
    const int mask_on = absorber && absorber->width > 0.0;
    C.jm_lo = 0;
    C.jm_hi = I.N - 1;
    if (mask_on) {
        const double xb = 0.5 * I.N * I.dx - absorber->width;
        int lo = I.N, hi = -1;
        for (int j = 0; j < I.N; ++j) {
            const double x = (j - 0.5 * (I.N - 1)) * I.dx;
            if (!(std::fabs(x) > xb)) {
                lo = std::min(lo, j);
                hi = std::max(hi, j);
            }
        }
        C.jm_lo = lo;
        C.jm_hi = hi;
    }
    const int warps = 8;
    int K = halo_for_beta(C.beta);
    const int P = class_segments(C.N, K, warps);
    if (P == 1) K = 0;
    const int m = (C.N + P - 1) / P;
    const int rows = std::min(C.N, m + 2 * K);
    const int64_t n_groups = (n_inst + kLanes - 1) / kLanes;

    // carve the static array (every block 256-byte aligned)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_cls = take(sizeof(ClassDesc));
    const size_t o_groups = take(sizeof(GroupDesc) * (size_t)n_groups);
    const size_t o_row = take(sizeof(int64_t) * (size_t)n_groups * kLanes);
    const size_t o_nt = take(sizeof(int64_t) * (size_t)n_groups * kLanes);
    const size_t o_busy = take(sizeof(int) * (size_t)n_groups);
    const size_t o_prog = take(sizeof(int) * (size_t)n_groups);
    const size_t o_status = take(sizeof(int) * (size_t)n_groups * kLanes);
    const size_t o_tab = take(sizeof(double) * (size_t)tab_doubles(C.N));
    const size_t o_scratch = off;
    const size_t per_cta = sizeof(double2) * (size_t)warps * rows * 2 * kLanes;
    if (o_scratch >= kStaticBytes || (kStaticBytes - o_scratch) / per_cta < 1) {
        static thread_local char msg[256];
        std::snprintf(msg, sizeof msg,
                      "tdse_propagate_static: N = %d with %lld instances needs more than the %zu MiB static scratch; "
                      "use tdse_batch_create/tdse_propagate",
                      C.N, (long long)n_inst, kStaticBytes >> 20);
        return err(TDSE_ERR_ARG, msg);
    }
    int sm_count = 0;
    if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return err(TDSE_ERR_CUDA, "tdse_propagate_static: cudaDeviceGetAttribute failed");
    const int64_t fit = (int64_t)((kStaticBytes - o_scratch) / per_cta);
    const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>({n_groups, (int64_t)sm_count, fit}));

    unsigned char* p = static_cast<unsigned char*>(base);
    ClassDesc* d_cls = reinterpret_cast<ClassDesc*>(p + o_cls);
    GroupDesc* d_groups = reinterpret_cast<GroupDesc*>(p + o_groups);
    int64_t* d_row = reinterpret_cast<int64_t*>(p + o_row);
    int64_t* d_nt = reinterpret_cast<int64_t*>(p + o_nt);
    int* d_busy = reinterpret_cast<int*>(p + o_busy);
    int* d_prog = reinterpret_cast<int*>(p + o_prog);
    int* d_status = reinterpret_cast<int*>(p + o_status);
    double* d_tab = reinterpret_cast<double*>(p + o_tab);
    void* d_scratch = p + o_scratch;

    cudaStream_t s = (cudaStream_t)stream;
    const int setup_blocks = (int)std::min<int64_t>(1024, (n_groups * kLanes + 255) / 256);
    k_static_setup<<<setup_blocks, 256, 0, s>>>(C, n_inst, n_groups, n_steps, row_stride, P, K, m, d_cls, d_groups,
                                                d_row, d_nt, d_status);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_build_tables(d_cls, 1, C.N, dt, mask_on ? absorber->width : 0.0, mask_on ? absorber->exponent : 0.0,
                                mask_on, d_tab, s);
    if (e == cudaSuccess)
        e = launch_propagate_full_cn(0, d_groups, n_groups, warps, ctas, d_cls, d_tab, d_row, d_nt, psi_dev, d_scratch,
                                     rows, E_dev, d_dev, a_dev, sample_base, step_begin, step_end, 16, mask_on, d_busy,
                                     d_prog, d_status, 2 /* bulk-copy ring: MIXED only */, 1u << 22, s);
    if (e != cudaSuccess) {
        static thread_local char msg[256];
        std::snprintf(msg, sizeof msg, "tdse_propagate_static: %s", cudaGetErrorString(e));
        return err(TDSE_ERR_CUDA, msg);
    }
    return TDSE_OK;
}
