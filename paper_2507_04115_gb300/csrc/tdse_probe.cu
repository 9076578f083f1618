// tdse_probe_pipes: throughput probes of the arithmetic pipes this engine is bound by (the
// roofline denominators that a copy/GEMM peak table does not give): FP64 and FP32 fused
// multiply-add, FP64 with one active lane per warp, FP64 with 1/2/4 warps per SM, and the cost of
// double<->float conversions.  Bounded loops only; one short launch per figure.
#include "tdse.h"
#include "tdse_internal.h"

#include <cstdio>

namespace {

template <int CH>
__global__ void k_fma64(double* out, int iters, int lanes, double a, double b)
{
    double acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = threadIdx.x * 1e-3 + c;
    if ((int)(threadIdx.x & 31) < lanes) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < CH; ++c) acc[c] = fma(acc[c], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += acc[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void k_fma32(float* out, int iters, float a, float b)
{
    float acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) acc[c] = fmaf(acc[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += acc[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 8 independent chains of (double -> float -> double) conversions: two conversions per element.
__global__ void k_cvt(double* out, int iters, double a)
{
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 1.0 + threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = (double)__double2float_rn(acc[c]) + a;
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 8 independent chains of one FP64 operation (0: fma, 1: add, 2: mul) per element.
template <int kOp>
__global__ void k_op64(double* out, int iters, double a, double b, double one, double nzero)
{
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 1.0 + threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if constexpr (kOp == 0) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(acc[c]) : "d"(a), "d"(b));
            else if constexpr (kOp == 1) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(acc[c]) : "d"(b));
            else if constexpr (kOp == 2) asm volatile("mul.rn.f64 %0, %0, %1;" : "+d"(acc[c]) : "d"(a));
            else if constexpr (kOp == 3) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(acc[c]) : "d"(one), "d"(b));
            else asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(acc[c]) : "d"(a), "d"(nzero));
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// A reciprocal seed without the double approximation: 1/n from the float approximation
// (rcp.approx.ftz.f32, XU pipe) of n truncated to 20 mantissa bits, narrowed and widened by
// integer arithmetic on the exponent field (double bias 1023 -> float bias 127: a shift of 896);
// relative error < 2^-20 + 2^-23 inside float's normal range.  Probed as an alternative to
// rcp.approx.ftz.f64 (the two measure the same cost, so the kernels keep the hardware seed).
__device__ __forceinline__ double rcp_seed_f32(double n)
{
    const int hi = __double2hiint(n);
    const float f = __int_as_float((hi - (896 << 20)) << 3);
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(f));
    const int yb = __float_as_int(yf);
    return __hiloint2double((yb >> 3) + (896 << 20), yb << 29);
}

// 8 independent FMA chains; with kSeed > 0 every FMA result also feeds a reciprocal seed
// (1: rcp.approx.ftz.f64, 2: rcp_seed_f32) summed into a second accumulator
// by an FMA, so that the loop's extra time over kSeed = 0 is one seed plus one FMA per element.
template <int kSeed>
__global__ void k_seed(double* out, int iters, double a, double b)
{
    double acc[8], sum[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        acc[c] = 1.0 + threadIdx.x * 1e-3 + c;
        sum[c] = 0.0;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            acc[c] = fma(acc[c], a, b);
            if constexpr (kSeed == 1) {
                double y;
                asm volatile("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(acc[c]));
                sum[c] = fma(y, a, sum[c]);
            } else if constexpr (kSeed == 2) {
                sum[c] = fma(rcp_seed_f32(acc[c]), a, sum[c]);
            }
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[c] + sum[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" tdse_status tdse_probe_pipes(int device, tdse_pipe_rates* out)
{
    if (!out) return tdse::set_error_message("tdse_probe_pipes: NULL output"), TDSE_ERR_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        tdse::set_error_message("tdse_probe_pipes: cudaSetDevice failed");
        return TDSE_ERR_ARG;
    }
    int sms = 0, clk_khz = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, device);
    const int blocks = sms * 8, threads = 256;
    double* buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tdse_status st = TDSE_OK;
    if (cudaMalloc(&buf, sizeof(double) * (size_t)blocks * threads) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        tdse::set_error_message("tdse_probe_pipes: allocation failed");
        st = TDSE_ERR_NOMEM;
    }
    auto timed = [&](auto launch) -> double {   // milliseconds of the second of two launches
        launch();
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    if (st == TDSE_OK) {
        const int it64 = 2048, it32 = 32768, itc = 512;
        double ms = timed([&] { k_fma64<8><<<blocks, threads>>>(buf, it64, 32, 0.999, 1e-3); });
        out->fp64_fma_tflops = 2.0 * 8 * it64 * (double)blocks * threads / (ms * 1e-3) / 1e12;
        ms = timed([&] { k_fma64<8><<<blocks, threads>>>(buf, it64, 1, 0.999, 1e-3); });
        out->fp64_one_lane_warp_instr_per_s = 8.0 * it64 * (double)blocks * (threads / 32) / (ms * 1e-3);
        out->fp64_warp_instr_per_s = out->fp64_fma_tflops * 1e12 / 64.0;
        ms = timed([&] { k_fma32<8><<<blocks, threads>>>(reinterpret_cast<float*>(buf), it32, 0.999f, 1e-3f); });
        out->fp32_fma_tflops = 2.0 * 8 * it32 * (double)blocks * threads / (ms * 1e-3) / 1e12;
        for (int k = 0; k < 3; ++k) {
            const int W = 1 << k;   // 1, 2, 4 warps per SM
            ms = timed([&] { k_fma64<8><<<sms, 32 * W>>>(buf, it64, 32, 0.999, 1e-3); });
            out->fp64_tflops_warps_per_sm[k] = 2.0 * 8 * it64 * (double)sms * 32 * W / (ms * 1e-3) / 1e12;
        }
        ms = timed([&] { k_cvt<<<blocks, threads>>>(buf, itc, 1e-9); });
        // per element: one double->float, one float->double, one double add
        out->cvt_pairs_per_s = 8.0 * itc * (double)blocks * threads / (ms * 1e-3);
        {
            // acc stays near b / (1 - a) = 1 (a = 0.999, b = 1e-3): inside every seed's range
            const int its = 1024;
            const double t0 = timed([&] { k_seed<0><<<blocks, threads>>>(buf, its, 0.999, 1e-3); });
            const double t1 = timed([&] { k_seed<1><<<blocks, threads>>>(buf, its, 0.999, 1e-3); });
            const double t2 = timed([&] { k_seed<2><<<blocks, threads>>>(buf, its, 0.999, 1e-3); });
            // t0 = one FMA per element; the extra FMA of the seeded loops is subtracted
            out->rcp_f64_approx_fma_slots = (t1 - t0) / t0 - 1.0;
            out->rcp_seed_fma_slots = (t2 - t0) / t0 - 1.0;
        }
        {
            const int its = 2048;
            const double tf = timed([&] { k_op64<0><<<blocks, threads>>>(buf, its, 0.999, 1e-3, 1.0, -0.0); });
            const double ta = timed([&] { k_op64<1><<<blocks, threads>>>(buf, its, 0.999, 1e-3, 1.0, -0.0); });
            const double tm = timed([&] { k_op64<2><<<blocks, threads>>>(buf, its, 0.999, 1e-3, 1.0, -0.0); });
            out->dadd_fma_slots = ta / tf;
            out->dmul_fma_slots = tm / tf;
            const double ta2 = timed([&] { k_op64<3><<<blocks, threads>>>(buf, its, 0.999, 1e-3, 1.0, -0.0); });
            const double tm2 = timed([&] { k_op64<4><<<blocks, threads>>>(buf, its, 0.999, 1e-3, 1.0, -0.0); });
            out->add_as_fma_slots = ta2 / tf;
            out->mul_as_fma_slots = tm2 / tf;
            const double tf2 = timed([&] { k_op64<0><<<blocks, threads>>>(buf, its, 0.999, 1e-3, 1.0, -0.0); });
            out->fma_repeat_slots = tf2 / tf;
        }
        out->sm_count = sms;
        out->sm_clock_mhz = clk_khz / 1000.0;
        if (cudaGetLastError() != cudaSuccess) {
            tdse::set_error_message("tdse_probe_pipes: a probe launch failed");
            st = TDSE_ERR_CUDA;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}
