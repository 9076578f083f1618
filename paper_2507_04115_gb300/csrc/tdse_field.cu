// Field ingestion (Sec. 4.2): coarsely sampled driving fields are moved to the time origin and
// interpolated to the propagation step by zero-padding their DFT.  For a row of M samples
// E_c[m] = E(t_min + m dt_c) the interpolant at t (measured from the first sample) is
//     E(t) = (1/M) sum_{k=-floor(M/2)}^{floor(M/2)} w_k Ehat_k exp(2 pi i k t / T),  T = M dt_c,
// w_k = 1/2 for |k| = M/2 when M is even, else 1.  The samples are real, so Ehat_{-k} = conj(Ehat_k)
// and E(t) = sum_{k=0}^{floor(M/2)} Re(c_k exp(2 pi i k t / T)) with c_0 = Ehat_0 / M,
// c_k = 2 Ehat_k / M for 0 < k < M/2 and c_{M/2} = Ehat_{M/2} / M (even M).
//
//   k_field_coeffs  one CTA per row: the row staged in shared memory, one thread per k computing
//                   the DFT by a complex rotation re-seeded with sincospi every 64 samples;
//   k_field_synth   one thread per output sample: the sum over k by a rotation in k re-seeded
//                   every 64 terms, coefficients staged in shared memory per row.
// Work: O(M^2) per row for the coefficients and O(M n_fine) for the synthesis, all in FP64 (the
// direct form of the zero-padded inverse transform at the requested samples).
#include "tdse_device.cuh"
#include "tdse_internal.h"

namespace tdse {

namespace {

__global__ void k_field_coeffs(const double* __restrict__ coarse, int64_t n_rows, int M, double2* __restrict__ coef)
{
    extern __shared__ double row[];
    const int64_t r = blockIdx.x;
    if (r >= n_rows) return;
    for (int m = threadIdx.x; m < M; m += blockDim.x) row[m] = coarse[r * M + m];
    __syncthreads();
    const int K = M / 2;
    for (int k = threadIdx.x; k <= K; k += blockDim.x) {
        // Ehat_k = sum_m E_c[m] exp(-2 pi i k m / M); the phase step is exp(-2 pi i k / M)
        double sr = 0.0, si = 0.0, zr = 1.0, zi = 0.0, wr, wi;
        sincospi(-2.0 * k / M, &wi, &wr);
        for (int m = 0; m < M; ++m) {
            if ((m & 63) == 0) sincospi(-2.0 * (double)((int64_t)k * m % M) / M, &zi, &zr);
            sr = fma(row[m], zr, sr);
            si = fma(row[m], zi, si);
            const double nr = fma(zr, wr, -zi * wi);
            zi = fma(zr, wi, zi * wr);
            zr = nr;
        }
        const double f = (k == 0 || 2 * k == M) ? 1.0 / M : 2.0 / M;
        coef[r * (K + 1) + k] = make_double2(f * sr, f * si);
    }
}

__global__ void k_field_synth(const double2* __restrict__ coef, int64_t n_rows, int M, double dt_c, double dt_f,
                              int64_t n_fine, int64_t out_stride, double* __restrict__ out)
{
    extern __shared__ double2 c[];
    const int64_t r = blockIdx.y;
    if (r >= n_rows) return;
    const int K = M / 2;
    for (int k = threadIdx.x; k <= K; k += blockDim.x) c[k] = coef[r * (K + 1) + k];
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_fine) return;
    // theta = 2 pi t / T with t = n dt_f, reduced to one period: u = (t / T) mod 1, exp(2 pi i k u)
    const double T = M * dt_c;
    double u = (n * dt_f) / T;
    u -= floor(u);
    double wr, wi;
    sincospi(2.0 * u, &wi, &wr);
    double s = 0.0, zr = 1.0, zi = 0.0;
    for (int k = 0; k <= K; ++k) {
        if ((k & 63) == 0) {
            double ku = k * u;
            ku -= floor(ku);
            sincospi(2.0 * ku, &zi, &zr);
        }
        s = fma(c[k].x, zr, fma(-c[k].y, zi, s));   // Re(c_k z^k)
        const double nr = fma(zr, wr, -zi * wi);
        zi = fma(zr, wi, zi * wr);
        zr = nr;
    }
    out[r * out_stride + n] = s;
}

}  // namespace

cudaError_t launch_resample_field(const double* coarse, int64_t n_rows, int M, double dt_c, double dt_f,
                                  int64_t n_fine, int64_t out_stride, double* out, void* d_coef, cudaStream_t st)
{
    if (n_rows == 0 || n_fine == 0) return cudaSuccess;
    const int K = M / 2;
    static std::atomic<bool> attr_set[kMaxAttrDevices];   // rows up to 8192 samples: 64 KB of shared memory per CTA
    int dev = 0;
    if (attr_needed(attr_set, &dev)) {
        cudaError_t e = cudaFuncSetAttribute(k_field_coeffs, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_field_synth, cudaFuncAttributeMaxDynamicSharedMemorySize, 4097 * 16);
        if (e != cudaSuccess) return e;
        attr_done(attr_set, dev);
    }
    double2* coef = static_cast<double2*>(d_coef);
    for (int64_t r0 = 0; r0 < n_rows; r0 += 65535) {
        const int64_t nr = n_rows - r0 < 65535 ? n_rows - r0 : 65535;
        k_field_coeffs<<<(unsigned)nr, 256, sizeof(double) * M, st>>>(coarse + r0 * M, nr, M, coef + r0 * (K + 1));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((n_fine + 255) / 256), (unsigned)nr);
        k_field_synth<<<grid, 256, sizeof(double2) * (K + 1), st>>>(coef + r0 * (K + 1), nr, M, dt_c, dt_f, n_fine,
                                                                   out_stride, out + r0 * out_stride);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace tdse
