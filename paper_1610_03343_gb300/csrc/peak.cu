// peak.cu -- measured fused multiply-add peaks of the current GPU (diagnostics).
//
// The pair passes are bound by the FP64 pipe (fp64 path) or by instruction issue and the
// FP32 pipe (mixed path), so their rooflines need the rate at which this GPU retires FMAs
// in each precision.  A kernel of independent FMA chains measures it: every thread keeps
// accumulators a_k <- a_k * b + c that do not depend on one another, so a warp always has an
// FMA ready to issue (8 chains in fp64, 16 in fp32), with 8 warps per scheduler partition on
// every SM, timed with CUDA events around one launch after a warm-up launch.  2 flop per
// FMA.  The result goes to out[] only so that the chains are not removed as dead code.
#include <cstdint>

#include <cuda_runtime.h>

#include "md.h"

namespace {

constexpr int kChains64 = 8;    // any count from 4 to 16 gave the same fp64 rate
constexpr int kChains32 = 16;   // fp32: 16 chains keep every scheduler's FMA pipe fed
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;   // 1024 threads = 32 warps per SM

template <typename T, int kChains>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int64_t iters, T b, T c, T *out)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k);
    // unrolled so that the loop's integer instructions take few issue slots beside the FMAs
#pragma unroll 16
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[(int64_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename T>
int run_peak(int64_t iters, int repeats, double *tflops, double *ms_out)
{
    constexpr int kChains = sizeof(T) == 8 ? kChains64 : kChains32;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) {
        cudaGetLastError();
        return MD_ERR_CUDA;
    }
    const unsigned blocks = (unsigned)(n_sm * kBlocksPerSm);
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * kThreads) != cudaSuccess) {
        cudaGetLastError();
        return MD_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 0.0, best_ms = 0.0;
    // b slightly below 1 and c small keep every chain finite and normal for any length
    const T b = T(0.999999), c = T(1e-3);
    if (e == cudaSuccess) {
        k_fma_chains<T, kChains><<<blocks, kThreads>>>(iters / 8 + 1, b, c, out);   // warm-up
        for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
            cudaEventRecord(e0);
            k_fma_chains<T, kChains><<<blocks, kThreads>>>(iters, b, c, out);
            cudaEventRecord(e1);
            e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms > 0.f) {
                const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
                const double tf = flops / (ms * 1e-3) / 1e12;
                if (tf > best) {
                    best = tf;
                    best_ms = ms;
                }
            }
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MD_ERR_CUDA;
    }
    *tflops = best;
    if (ms_out) *ms_out = best_ms;
    return MD_OK;
}

}  // namespace

extern "C" int md_peak_flops(int precision, int64_t iters, int repeats, double *tflops, double *ms)
{
    if (!tflops || iters < 1 || repeats < 1 || (precision != MD_FP64 && precision != MD_MIXED)) return MD_ERR_ARG;
    return precision == MD_FP64 ? run_peak<double>(iters, repeats, tflops, ms)
                                : run_peak<float>(iters, repeats, tflops, ms);
}
