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
