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

}  // namespace tdse
