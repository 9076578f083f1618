// Device helpers shared by the kernels of libtdse (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tdse {

// 1/n for finite normal n > 0 (far from the overflow edge): hardware seed (rcp.approx.ftz.f64)
// refined by one third-order step of the Newton-Raphson family, y = y0 (1 + e + e^2) with
// e = 1 - n y0, which leaves a relative error of e^3 (seed error ~2^-20 gives ~2^-60, below
// double rounding).
__device__ __forceinline__ double rcp_pos(double n)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(n));
    const double e = fma(-n, y, 1.0);
    const double t = fma(e, e, e);
    return fma(y, t, y);
}

// 1/n to ~2^-40 relative (one second-order Newton-Raphson step from the hardware seed,
// y = y0 (1 + e), e = 1 - n y0, error e^2): for coefficients that are rounded to float right after.
__device__ __forceinline__ double rcp_pos_2nd(double n)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(n));
    const double e = fma(-n, y, 1.0);
    return fma(y, e, y);
}

// FP64 add, subtract and multiply issued as fused multiply-adds.  On this GPU a DADD or DMUL
// warp instruction occupies the FP64 pipe about 19 % longer than a DFMA (tdse_probe_pipes:
// dadd_fma_slots, dmul_fma_slots), while fma(x, 1, y) = x + y, fma(y, -1, x) = x - y and
// fma(x, y, -0) = x y hold exactly (one rounding of the exact result, signed zeros included).
// The 1 and -0 are read from memory (the class descriptor) so that the compiler cannot fold the
// FMAs back into adds and multiplies.  Float overloads keep the native FP32 operations.
struct Fma64 {
    double one, nzero;
    __device__ __forceinline__ double add(double x, double y) const { return fma(x, one, y); }
    __device__ __forceinline__ double sub(double x, double y) const { return fma(y, -one, x); }
    __device__ __forceinline__ double mul(double x, double y) const { return fma(x, y, nzero); }
    __device__ __forceinline__ float add(float x, float y) const { return x + y; }
    __device__ __forceinline__ float sub(float x, float y) const { return x - y; }
    __device__ __forceinline__ float mul(float x, float y) const { return x * y; }
};

// ---- float pairs on the FP32 pipe (no FP64 instruction; GB300 runs FP32 at 64x its FP64 rate) ----

// v >= 0 (a squared modulus) as h + l with h, l floats: h its leading 24 significant bits, l the rest
// rounded to 24 bits, so |h + l - v| <= 2^-48 v + 2^-126 (parts below float's normal range flush
// to zero).  Integer operations on the double's two words only.  Infinity and NaN map to a float infinity or NaN; values beyond float's range to infinity,
// so a non-finite state still shows in the sums.
__device__ __forceinline__ void split_ff(double v, float& h, float& l)
{
    const int hi = __double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
    unsigned hb = ((e - 896u) << 23) | (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
    hb = e < 897u ? 0u : hb;
    const bool special = e > 1150u;   // beyond float's range, infinity or NaN
    const bool nan = e == 2047u && ((((unsigned)hi & 0xfffffu) | lo) != 0u);
    hb = special ? (nan ? 0x7fc00000u : 0x7f800000u) : hb;
    h = __uint_as_float(hb);
    const unsigned m29 = lo & 0x1fffffffu;
    const int lz = __clz(m29);
    const unsigned long long t = ((unsigned long long)m29 << (lz + 1)) & 0xffffffffull;
    const int fe = (int)e - 917 - lz;
    unsigned lb = ((unsigned)fe << 23) | (unsigned)(t >> 9);
    lb += (unsigned)(t >> 8) & 1u;   // l rounded to nearest (a carry into the exponent is exact)
    lb = (m29 == 0u || fe <= 0 || e < 897u || special) ? 0u : lb;
    l = __uint_as_float(lb);
}

// Any finite v as h + l with h, l floats of v's sign: the split of |v| above (|h + l - v| <= 2^-48 |v|
// + 2^-126), the sign bit copied onto both.  Integer operations only.
__device__ __forceinline__ void split_sf(double v, float& h, float& l)
{
    const int hi = __double2hiint(v);
    const unsigned sign = (unsigned)hi & 0x80000000u;
    split_ff(__hiloint2double(hi & 0x7fffffff, __double2loint(v)), h, l);   // |v| by clearing the sign bit
    h = __uint_as_float(__float_as_uint(h) | sign);
    l = __uint_as_float(__float_as_uint(l) | sign);
}

// |x|^2 = xr^2 + xi^2 as a float pair (rh, rl), within 2^-44 relative (plus 2^-124 absolute: squares
// below float's normal range flush), on the FP32 pipe: xr and xi are
// split into float pairs by integer operations, the squares of the leading parts are exact with
// their FMA residuals, and the rest, (2h + l) l, is added in float.
__device__ __forceinline__ void sq_mod_ff(double xr, double xi, float& rh, float& rl)
{
    float ah, al, bh, bl;
    split_sf(xr, ah, al);
    split_sf(xi, bh, bl);
    const float p1 = __fmul_rn(ah, ah), p2 = __fmul_rn(bh, bh);
    const float e1 = fmaf(ah, ah, -p1), e2 = fmaf(bh, bh, -p2);
    const float s = __fadd_rn(p1, p2);
    const float bp = __fsub_rn(s, p1);
    const float t = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bp)), __fsub_rn(p2, bp));
    const float c = fmaf(2.0f * ah + al, al, __fmul_rn(2.0f * bh + bl, bl));   // (2h + l) l
    const float lo = __fadd_rn(__fadd_rn(t, __fadd_rn(e1, e2)), c);
    rh = __fadd_rn(s, lo);
    rl = __fsub_rn(lo, __fsub_rn(rh, s));
}

// float -> double by integer operations (exact for normal floats and infinities/NaN; zero and
// subnormals give a signed zero)
__device__ __forceinline__ double f2d_int(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned sign = b & 0x80000000u;
    unsigned h = sign | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    h = e == 255u ? (sign | 0x7ff00000u | ((b & 0x7fffffu) >> 3) | ((b & 0x7fffffu) ? 0x80000u : 0u)) : h;
    const unsigned l = e == 255u ? 0u : b << 29;
    return e == 0u ? __hiloint2double((int)sign, 0) : __hiloint2double((int)h, (int)l);
}

// (sh, sl) += (ah, al): exact two-sum of the leading parts, rounding errors and low parts into sl,
// then the pair renormalised (fast two-sum, |sl| <= half an ulp of sh) so that sl's own rounding
// stays at 2^-48 of the sum instead of growing with the number of terms.  The _rn intrinsics keep
// the compiler from contracting the two-sums into FMAs, which would break their exactness.
__device__ __forceinline__ void ff_acc(float& sh, float& sl, float ah, float al)
{
    const float t = __fadd_rn(sh, ah);
    const float bp = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(ah, bp));
    const float lo = __fadd_rn(sl, __fadd_rn(err, al));
    sh = __fadd_rn(t, lo);
    sl = __fsub_rn(lo, __fsub_rn(sh, t));
}

// (sh, sl) += (xh + xl)(rh + rl): the leading product exact by an FMA, the cross terms in float
// (the xl rl term, ~2^-48 of the product, is dropped)
__device__ __forceinline__ void ff_fma_acc(float& sh, float& sl, float xh, float xl, float rh, float rl)
{
    const float p = __fmul_rn(xh, rh);
    const float e = fmaf(xh, rh, -p);
    ff_acc(sh, sl, p, fmaf(xh, rl, fmaf(xl, rh, e)));
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// L2-only loads (ld.global.cg): data written by another SM in an earlier scheduling slice must not
// be served from a stale L1 line.
__device__ __forceinline__ double2 ld_cg(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_cg(const float2* p) { return __ldcg(p); }

// ---- bulk asynchronous copies (TMA, cp.async.bulk) into shared memory, completed on an mbarrier ----

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make mbarrier initialisation visible to the async proxy before any copy uses the barrier.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// 1D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing
// `bytes` of transaction count on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Wait until the barrier's phase with the given parity completes; gives up after `limit` polls and
// returns false (the caller records the timeout instead of hanging).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Order this thread's generic-proxy accesses before later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

}  // namespace tdse
