// hcacf.cu -- md_hcacf: heat-current autocorrelation and running Green-Kubo thermal
// conductivity from the per-step heat current that md_run records (Eq. 30 summed over
// atoms).
//
//   C_a(m)     = 1/(T-m) sum_{t<T-m} J_a(t) J_a(t+m)        (every time origin)
//   kappa_a(m) = 1/(k_B T^2 V) * trapezoid integral of C_a from lag 0 to lag m
//
// Three kernels: gather the strided J columns into three contiguous fp64 arrays; the
// correlation, where a block takes kLagsPerBlock consecutive lags and each thread walks
// the time origins t = tid, tid + 256, ... so that J(t) is loaded once for all of the
// block's lags and the J(t+m) loads are coalesced across the warp; a fixed-order tree in
// shared memory per lag (deterministic); and the running trapezoid sum, one thread per
// component in lag order.
#include <algorithm>
#include <cmath>

#include "md.h"
#include "md_internal.cuh"

namespace {

constexpr int kAcfThreads = 256;
constexpr int kLagsPerBlock = 8;
constexpr double kBoltzmann = 8.617333262e-5;                       // eV / K
constexpr double kToWattPerMeterKelvin = 1.602176634e-19 / 1e-25;   // eV/(fs A K) -> W/(m K)

__global__ void k_pack_j(const double *j, int64_t T, int64_t stride, double *jc)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        jc[t] = j[t * stride];
        jc[T + t] = j[t * stride + 1];
        jc[2 * T + t] = j[t * stride + 2];
    }
}

__global__ void __launch_bounds__(kAcfThreads) k_acf(const double *jc, int64_t T, int64_t n_lags, double *c)
{
    __shared__ double red[3 * kLagsPerBlock][kAcfThreads];
    const int tid = threadIdx.x;
    for (int64_t m0 = (int64_t)blockIdx.x * kLagsPerBlock; m0 < n_lags; m0 += (int64_t)gridDim.x * kLagsPerBlock) {
        double s[3][kLagsPerBlock];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int l = 0; l < kLagsPerBlock; ++l) s[a][l] = 0.0;
        const int64_t n0 = T - m0;   // origins of the block's first lag
        for (int64_t t = tid; t < n0; t += kAcfThreads) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double *col = jc + a * T;
                const double x = col[t];
#pragma unroll
                for (int l = 0; l < kLagsPerBlock; ++l) {
                    const int64_t m = m0 + l;
                    if (m < n_lags && t + m < T) s[a][l] = fma(x, col[t + m], s[a][l]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int l = 0; l < kLagsPerBlock; ++l) red[a * kLagsPerBlock + l][tid] = s[a][l];
        __syncthreads();
        for (int o = kAcfThreads / 2; o > 0; o >>= 1) {
            if (tid < o)
                for (int r = 0; r < 3 * kLagsPerBlock; ++r) red[r][tid] += red[r][tid + o];
            __syncthreads();
        }
        if (tid < 3 * kLagsPerBlock) {
            const int a = tid / kLagsPerBlock, l = tid % kLagsPerBlock;
            const int64_t m = m0 + l;
            if (m < n_lags) c[m * 3 + a] = red[tid][0] / (double)(T - m);
        }
        __syncthreads();
    }
}

__global__ void k_running_kappa(const double *c, int64_t n_lags, double half_dt_pref, double *kappa)
{
    const int a = threadIdx.x;
    if (a >= 3) return;
    double k = 0.0;
    kappa[a] = 0.0;
    for (int64_t m = 1; m < n_lags; ++m) {
        k += (c[(m - 1) * 3 + a] + c[m * 3 + a]);
        kappa[m * 3 + a] = k * half_dt_pref;
    }
}

}  // namespace

extern "C" md_status md_hcacf(const double *j, int64_t n_rows, int64_t row_stride, int64_t n_lags, double dt_fs,
                              double volume, double temperature, double *acf, double *kappa, int io,
                              void *cuda_stream)
{
    if (!j || !acf || n_rows < 1 || n_lags < 1 || n_lags > n_rows || row_stride < 3) return MD_ERR_ARG;
    if (io != MD_IO_HOST && io != MD_IO_DEVICE) return MD_ERR_ARG;
    if (kappa && !(dt_fs > 0 && volume > 0 && temperature > 0 && std::isfinite(dt_fs) && std::isfinite(volume) &&
                   std::isfinite(temperature)))
        return MD_ERR_ARG;
    if (n_rows > (int64_t(1) << 40) / row_stride) return MD_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const bool host = io == MD_IO_HOST;
    const size_t in_bytes = sizeof(double) * (size_t)((n_rows - 1) * row_stride + 3);
    const size_t out_bytes = sizeof(double) * 3 * (size_t)n_lags;
    const double *dj = j;
    double *dc = acf, *dk = kappa, *jc = nullptr, *dj_owned = nullptr;
    bool ok = true;
    auto mal = [&](double **p, size_t b) {
        if (ok && cudaMallocAsync(reinterpret_cast<void **>(p), b, s) != cudaSuccess) ok = false;
    };
    mal(&jc, sizeof(double) * 3 * (size_t)n_rows);
    if (host) {
        mal(&dj_owned, in_bytes);
        mal(&dc, out_bytes);
        if (kappa) mal(&dk, out_bytes);
        if (ok && cudaMemcpyAsync(dj_owned, j, in_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) ok = false;
        dj = dj_owned;
    }
    if (ok) {
        const unsigned pack_blocks = (unsigned)std::min<int64_t>((n_rows + 255) / 256, 1024);
        k_pack_j<<<pack_blocks, 256, 0, s>>>(dj, n_rows, row_stride, jc);
        const unsigned acf_blocks = (unsigned)std::min<int64_t>((n_lags + kLagsPerBlock - 1) / kLagsPerBlock, 8192);
        k_acf<<<acf_blocks, kAcfThreads, 0, s>>>(jc, n_rows, n_lags, dc);
        if (kappa) {
            const double pref = kToWattPerMeterKelvin / (kBoltzmann * temperature * temperature * volume);
            k_running_kappa<<<1, 32, 0, s>>>(dc, n_lags, 0.5 * dt_fs * pref, dk);
        }
        if (cudaGetLastError() != cudaSuccess) ok = false;
    }
    if (ok && host) {
        if (cudaMemcpyAsync(acf, dc, out_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) ok = false;
        if (ok && kappa && cudaMemcpyAsync(kappa, dk, out_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            ok = false;
    }
    if (jc) cudaFreeAsync(jc, s);
    if (host) {
        if (dj_owned) cudaFreeAsync(dj_owned, s);
        if (dc && dc != acf) cudaFreeAsync(dc, s);
        if (dk && dk != kappa) cudaFreeAsync(dk, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) ok = false;
    if (!ok) {
        cudaGetLastError();
        return MD_ERR_CUDA;
    }
    return MD_OK;
}
