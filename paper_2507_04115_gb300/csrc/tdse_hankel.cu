// Output side of the hot path (sm_103a): the macroscopic source spectrum and the far field of a
// homogeneous generating medium.
//
//   tdse_dipole_spectrum  S_r(w) = weight_r dt / sqrt(2 pi) sum_n a_r,n exp(i w n dt): the temporal
//                         Fourier transform of every dipole-acceleration row in the paper's
//                         convention (Sec. 2), times the gas density of the row's point (the
//                         macroscopic source is the density times the microscopic one, Sec. 3.2).
//   tdse_hankel           Eq. "Hankel long homogeneous" (Sec. 3.2) by direct grid integration over
//                         the source points (Sec. 4.3), trapezoidal weights in rho' and z'.
//
// Kernel design.  The far field is a contraction over the source points (rho'_j, z'_i) for every
// frequency w and observation radius rho_o,
//     E[w][o] = C e^{i k z} sum_i e^{i k rho_o^2/(2 D_i)} sum_j J0(k rho_o rho'_j / D_i) T[w][i][j],
//     T[w][i][j] = wz_i wr_j rho'_j e^{i k (rho'_j^2/(2 D_i) - z'_i)} S[j][i][w] / D_i,  D_i = z - z'_i,
// whose matrix J0(k rho_o rho'_j / D_i) changes with every (w, i): there is no operand reuse, so the
// work is the generation of the Bessel values (one J0 per term), not multiply-adds, and tensor cores
// do not apply; the phases k z' reach 1e6 rad, so the arithmetic stays in FP64.  One CTA per
// (frequency, 128 observation radii); T is staged in shared memory by z' tiles (all threads read the
// same element: broadcast), each thread owns one observation radius and sums over the tile.
#include "tdse.h"
#include "tdse_internal.h"

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace tdse {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kMu0Over4Pi = 1.25663706212e-6 / (4.0 * 3.14159265358979323846);   // mu0 / (4 pi), SI
constexpr int kHankelThreads = 128;   // observation radii per CTA
constexpr int kHankelTile = 2048;     // complex source terms per shared-memory tile (32 KB)

// One thread per (row, frequency): the row streams through shared memory in 512-sample tiles; the
// twiddle e^{i w n dt} advances by complex rotation and is re-seeded with sincos every 64 samples.
__global__ void k_dipole_spectrum(const double* __restrict__ a, const int64_t* __restrict__ offs, int64_t row0,
                                  double dt, const double* __restrict__ omega, int n_w,
                                  const double* __restrict__ weight, double2* __restrict__ out)
{
    __shared__ double tile[512];
    const int64_t row = row0 + blockIdx.y;
    const int64_t base = offs[row];
    const int64_t L = offs[row + 1] - base;
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = w < n_w;
    const double om = live ? omega[w] : 0.0;
    double sr, cr;
    sincos(om * dt, &sr, &cr);
    double ar = 0.0, ai = 0.0, zr = 1.0, zi = 0.0;
    for (int64_t t0 = 0; t0 < L; t0 += 512) {
        const int cnt = (int)(L - t0 < 512 ? L - t0 : 512);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) tile[i] = a[base + t0 + i];
        __syncthreads();
        for (int i = 0; i < cnt; ++i) {
            const int64_t n = t0 + i;
            if ((n & 63) == 0) sincos(om * ((double)n * dt), &zi, &zr);
            const double v = tile[i];
            ar = fma(v, zr, ar);
            ai = fma(v, zi, ai);
            const double nr = fma(zr, cr, -zi * sr);
            const double ni = fma(zr, sr, zi * cr);
            zr = nr;
            zi = ni;
        }
    }
    if (live) {
        const double wt = (weight ? weight[row] : 1.0) * dt * (1.0 / sqrt(kTwoPi));
        out[row * (int64_t)n_w + w] = make_double2(wt * ar, wt * ai);
    }
}

// Grids packed in one device buffer: rho'[n_rho], wr[n_rho], z'[n_z], wz[n_z], k[n_w], rho_obs[n_obs].
__global__ void __launch_bounds__(kHankelThreads)
k_hankel(const double2* __restrict__ S, const double* __restrict__ grids, int n_rho, int n_z, int n_w, int n_obs,
         double z_obs, double2* __restrict__ E)
{
    __shared__ double2 T[kHankelTile];
    const double* rho = grids;
    const double* wr = rho + n_rho;
    const double* zs = wr + n_rho;
    const double* wz = zs + n_z;
    const double* kk = wz + n_z;
    const double* ro_all = kk + n_w;
    const int w = blockIdx.y;
    const double k = kk[w];
    const int o = blockIdx.x * kHankelThreads + threadIdx.x;
    const bool live = o < n_obs;
    const double ro = live ? ro_all[o] : 0.0;
    const int rows_per_tile = max(1, kHankelTile / n_rho);
    double er = 0.0, ei = 0.0;
    for (int i0 = 0; i0 < n_z; i0 += rows_per_tile) {
        const int nrow = min(rows_per_tile, n_z - i0);
        __syncthreads();   // the previous tile is consumed
        for (int p = threadIdx.x; p < nrow * n_rho; p += kHankelThreads) {
            const int ii = p / n_rho, j = p - ii * n_rho;
            const int i = i0 + ii;
            const double D = z_obs - zs[i];
            const double r = rho[j];
            double s, c;
            sincos(k * (r * r / (2.0 * D) - zs[i]), &s, &c);
            const double2 src = S[((int64_t)j * n_z + i) * n_w + w];
            const double wt = wz[i] * wr[j] * r / D;
            T[p] = make_double2(wt * fma(src.x, c, -src.y * s), wt * fma(src.x, s, src.y * c));
        }
        __syncthreads();
        for (int ii = 0; ii < nrow; ++ii) {
            const double D = z_obs - zs[i0 + ii];
            const double kap = k * ro / D;
            const double2* Tr = T + ii * n_rho;
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < n_rho; ++j) {
                const double b = j0(kap * rho[j]);
                const double2 t = Tr[j];
                sr = fma(b, t.x, sr);
                si = fma(b, t.y, si);
            }
            double s, c;
            sincos(k * ro * ro / (2.0 * D), &s, &c);
            er += fma(c, sr, -s * si);
            ei += fma(s, sr, c * si);
        }
    }
    if (live) {
        double s, c;
        sincos(k * z_obs, &s, &c);
        E[(int64_t)w * n_obs + o] = make_double2(-kMu0Over4Pi * fma(c, er, -s * ei), -kMu0Over4Pi * fma(s, er, c * ei));
    }
}

tdse_status arg_error(const std::string& msg)
{
    set_error_message(msg.c_str());
    return TDSE_ERR_ARG;
}

tdse_status cuda_error(cudaError_t e, const char* what)
{
    set_error_message((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
    return TDSE_ERR_CUDA;
}

bool ascending(const double* x, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(x[i]) || (i > 0 && !(x[i] > x[i - 1]))) return false;
    return true;
}

void trapezoid(const double* x, int n, double* w)
{
    if (n == 1) {
        w[0] = 1.0;
        return;
    }
    w[0] = 0.5 * (x[1] - x[0]);
    w[n - 1] = 0.5 * (x[n - 1] - x[n - 2]);
    for (int i = 1; i < n - 1; ++i) w[i] = 0.5 * (x[i + 1] - x[i - 1]);
}

}  // namespace
}  // namespace tdse

using namespace tdse;

extern "C" tdse_status tdse_dipole_spectrum(const double* a_dev, const int64_t* offsets_host, int64_t n_rows, double dt,
                                            const double* omega_host, int32_t n_omega, const double* weight_dev,
                                            double* out_dev, void* stream)
{
    if (!a_dev || !offsets_host || !omega_host || !out_dev) return arg_error("tdse_dipole_spectrum: NULL argument");
    if (n_rows < 1 || n_rows > (int64_t(1) << 31)) return arg_error("tdse_dipole_spectrum: n_rows out of range");
    if (n_omega < 1 || n_omega > (1 << 24)) return arg_error("tdse_dipole_spectrum: n_omega out of [1, 2^24]");
    if (!std::isfinite(dt) || !(dt > 0.0)) return arg_error("tdse_dipole_spectrum: dt must be finite and > 0");
    for (int64_t r = 0; r < n_rows; ++r)
        if (offsets_host[r] < 0 || offsets_host[r + 1] < offsets_host[r])
            return arg_error("tdse_dipole_spectrum: offsets must be non-decreasing and >= 0");
    for (int w = 0; w < n_omega; ++w)
        if (!std::isfinite(omega_host[w]) || std::fabs(omega_host[w]) > 1e6)
            return arg_error("tdse_dipole_spectrum: frequency " + std::to_string(w) + " not finite or beyond 1e6");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t* d_off = nullptr;
    double* d_om = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_off), sizeof(int64_t) * (n_rows + 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&d_om), sizeof(double) * n_omega, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, offsets_host, sizeof(int64_t) * (n_rows + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_om, omega_host, sizeof(double) * n_omega, cudaMemcpyHostToDevice, st);
    for (int64_t r0 = 0; e == cudaSuccess && r0 < n_rows; r0 += 65535) {
        const int64_t nr = std::min<int64_t>(65535, n_rows - r0);
        dim3 grid((unsigned)((n_omega + 127) / 128), (unsigned)nr);
        k_dipole_spectrum<<<grid, 128, 0, st>>>(a_dev, d_off, r0, dt, d_om, n_omega, weight_dev,
                                                reinterpret_cast<double2*>(out_dev));
        e = cudaGetLastError();
    }
    const cudaError_t f1 = d_off ? cudaFreeAsync(d_off, st) : cudaSuccess;
    const cudaError_t f2 = d_om ? cudaFreeAsync(d_om, st) : cudaSuccess;
    if (e != cudaSuccess) return cuda_error(e, "tdse_dipole_spectrum");
    if (f1 != cudaSuccess || f2 != cudaSuccess) return cuda_error(f1 != cudaSuccess ? f1 : f2, "tdse_dipole_spectrum free");
    return TDSE_OK;
}

extern "C" tdse_status tdse_hankel(const double* S_dev, const double* rho_src_host, int32_t n_rho, const double* z_src_host,
                                   int32_t n_z, const double* k_host, int32_t n_omega, double z_obs,
                                   const double* rho_obs_host, int32_t n_obs, double* E_dev, int device, void* stream)
{
    if (!S_dev || !rho_src_host || !z_src_host || !k_host || !rho_obs_host || !E_dev)
        return arg_error("tdse_hankel: NULL argument");
    if (n_rho < 1 || n_rho > kHankelTile) return arg_error("tdse_hankel: n_rho out of [1, 2048]");
    if (n_z < 1 || n_z > (1 << 20)) return arg_error("tdse_hankel: n_z out of [1, 2^20]");
    if (n_omega < 1 || n_omega > 65535) return arg_error("tdse_hankel: n_omega out of [1, 65535]");
    if (n_obs < 1 || n_obs > (1 << 24)) return arg_error("tdse_hankel: n_obs out of [1, 2^24]");
    if (!ascending(rho_src_host, n_rho) || rho_src_host[0] < 0.0)
        return arg_error("tdse_hankel: source radii must be finite, >= 0 and strictly ascending");
    if (!ascending(z_src_host, n_z)) return arg_error("tdse_hankel: source planes must be finite and strictly ascending");
    if (!std::isfinite(z_obs) || !(z_obs > z_src_host[n_z - 1]))
        return arg_error("tdse_hankel: the observation plane must lie beyond the last source plane");
    for (int w = 0; w < n_omega; ++w)
        if (!std::isfinite(k_host[w]) || !(k_host[w] > 0.0)) return arg_error("tdse_hankel: wave numbers must be finite and > 0");
    for (int o = 0; o < n_obs; ++o)
        if (!std::isfinite(rho_obs_host[o]) || rho_obs_host[o] < 0.0)
            return arg_error("tdse_hankel: observation radii must be finite and >= 0");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return arg_error("tdse_hankel: no such CUDA device");
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return cuda_error(cudaGetLastError(), "tdse_hankel: cudaSetDevice");
    std::vector<double> g((size_t)2 * n_rho + 2 * n_z + n_omega + n_obs);
    double* p = g.data();
    std::copy(rho_src_host, rho_src_host + n_rho, p);
    trapezoid(rho_src_host, n_rho, p + n_rho);
    p += 2 * n_rho;
    std::copy(z_src_host, z_src_host + n_z, p);
    trapezoid(z_src_host, n_z, p + n_z);
    p += 2 * n_z;
    std::copy(k_host, k_host + n_omega, p);
    std::copy(rho_obs_host, rho_obs_host + n_obs, p + n_omega);
    cudaStream_t st = (cudaStream_t)stream;
    double* d_g = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_g), sizeof(double) * g.size(), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_g, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        dim3 grid((unsigned)((n_obs + kHankelThreads - 1) / kHankelThreads), (unsigned)n_omega);
        k_hankel<<<grid, kHankelThreads, 0, st>>>(reinterpret_cast<const double2*>(S_dev), d_g, n_rho, n_z, n_omega, n_obs,
                                                   z_obs, reinterpret_cast<double2*>(E_dev));
        e = cudaGetLastError();
    }
    // (a copy from pageable host memory has consumed the host buffer when cudaMemcpyAsync returns)
    const cudaError_t f = d_g ? cudaFreeAsync(d_g, st) : cudaSuccess;
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_error(e, "tdse_hankel");
    if (f != cudaSuccess) return cuda_error(f, "tdse_hankel free");
    return TDSE_OK;
}
