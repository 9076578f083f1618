// Helpers shared by the persistent propagation kernels of libtdse (sm_103a): precision traits,
// the observable reduction and the dynamic group scheduler.
#pragma once

#include "tdse_device.cuh"
#include "tdse_internal.h"

namespace tdse {

// MIXED back substitution streams its rows through a per-warp ring of shared-memory slots, each
// holding kSlotRows rows (512-byte float2 gamma|D scratch rows, then 256-byte float2 psi rows):
// as many slots per warp (2 to 4) as fit when `per_sm` CTAs share an SM's 220 KB.  Several CTAs per
// SM let the FP64-heavy forward sweep of one group overlap the float back substitution of another
// (each CTA synchronises only its own warps).
constexpr int kSlotRows = 8;
// Points per block of the observable sums kept on the FP32 pipe before a block is added in double
// (FP64 path: float-pair sums; MIXED: float sums of the float state).
constexpr int kObsBlock = 16;
constexpr int kSlotBytes = kSlotRows * 768;
constexpr int kMaxRing = 4;
constexpr int kMinRing = 2;
// Polls of an mbarrier before a bulk-copy wait gives up (a copy of a few hundred bytes lands in
// microseconds; 2^22 polls is far beyond that), and the same bound for draining copies in flight
// after a wait gave up.
constexpr uint32_t kWaitPolls = 1u << 22;
constexpr uint32_t kDrainPolls = 1u << 22;

inline int full_cn_ring_slots(int P, int per_sm)
{
    const long red = (long)P * 3 * 32 * 8;
    const long r = (220L * 1024 / (per_sm < 1 ? 1 : per_sm) - red) / ((long)P * (kSlotBytes + 8));
    return r < kMinRing ? kMinRing : (r > kMaxRing ? kMaxRing : (int)r);
}

__host__ __device__ inline size_t full_cn_smem_bytes(int mixed, int P, int ring)
{
    size_t b = (size_t)P * 3 * 32 * sizeof(double);
    if (mixed) b += (size_t)P * ring * (sizeof(uint64_t) + kSlotBytes);
    return b;
}

// Largest dynamic shared memory the MIXED kernel asks for (over 1..16 warps, one CTA per SM).
inline size_t full_cn_smem_max_bytes()
{
    size_t m = 0;
    for (int P = 1; P <= 16; ++P) {
        const size_t b = full_cn_smem_bytes(1, P, full_cn_ring_slots(P, 1));
        m = b > m ? b : m;
    }
    return m;
}

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

// double -> float on the integer pipe: on GB300 a hardware conversion costs as much as an FP64
// multiply-add.  The 52-bit mantissa is rounded to 23 bits to nearest (ties away from zero; a carry
// into the exponent is the correct result), so the rounding is unbiased -- truncation would perturb
// every step's elimination coefficients in the same direction and the error would grow linearly
// with the number of steps.  Magnitudes below float's normal range flush to a signed zero and
// magnitudes above it saturate to float's largest finite value: the coefficients converted here
// satisfy |gamma| <= beta < 1 and |gamma| >= beta/|q|, far inside the range.  No FP64 instruction.
__device__ __forceinline__ float d2f(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
    unsigned bits = sign | ((e - 896u) << 23) | (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
    bits += (lo >> 28) & 1u;
    bits = e < 897u ? sign : bits;
    bits = e > 1149u ? (sign | 0x7f7fffffu) : bits;
    return __uint_as_float(bits);
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

// Warp 0 picks and claims the free group with the most remaining work (slices x the group's step
// cost w: the longest groups of an uneven batch start first, so they do not finish last); ties go
// to the group closest after this CTA's index (cyclically), so that CTAs starting together claim
// different groups instead of all racing for the same one.  Returns the group (its slice index in *k_out) or
// -1 when no free unfinished group is left.  Every failed claim means another CTA claimed a group,
// so the retries are bounded by the total number of claims.
__device__ __forceinline__ int pick_group(const GroupDesc* groups, int64_t n_groups, int* busy, int* progress, int64_t step_begin,
                          int64_t step_end, int slice, int* k_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t me = (int64_t)blockIdx.x % n_groups;
    for (int64_t attempt = 0; attempt < 4 * n_groups + 64; ++attempt) {
        int64_t best_rem = 0, best_d = n_groups, best_g = -1;
        for (int64_t g = lane; g < n_groups; g += 32) {
            const int64_t rem = (group_slices(groups[g], step_begin, step_end, slice) -
                                 *(volatile int*)(progress + g)) * groups[g].w;
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


}  // namespace tdse
