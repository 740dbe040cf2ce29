// acf.cu -- autocorrelation function A(k) and exponential autocorrelation time tau_exp
// (Sec. 4), the measure the HMC tuning is judged by.
//
// A(k) is the lagged covariance over the variance, both about the series mean (the
// centred estimator: for expectations it equals the paper's <O_t O_{t+k}> - <O>^2 over
// <O^2> - <O>^2, and unlike the uncentred sums it stays exact for an energy trace whose
// mean is hundreds of times its spread).  One block per (lag, series) makes two passes
// over the series: the mean, then the centred square and lagged-product sums, each in
// FP64 with a fixed reduction order, so every block derives the same mean and variance
// and the result is deterministic.  The fit of ln A(k) is a serial scan by one thread
// per series (a few hundred lags).
#include <math.h>

#include "common.cuh"

namespace nb {

constexpr int kAcfThreads = 256;

__device__ __forceinline__ double acf_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum in a fixed order; the result is returned to every thread.
__device__ __forceinline__ double acf_block_sum(double v, double* sm) {
    constexpr int kW = kAcfThreads / 32;
    v = acf_warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < kW; ++q) t += sm[q];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kAcfThreads) k_acf(const double* __restrict__ series, int n, int max_lag,
                                                      double* __restrict__ acf) {
    __shared__ double sm[kAcfThreads / 32];
    const int k = blockIdx.x, s = blockIdx.y;
    const double* o = series + (size_t)s * n;
    double m = 0.0;
    for (int t = threadIdx.x; t < n; t += kAcfThreads) m += o[t];
    const double mean = acf_block_sum(m, sm) / n;
    double v = 0.0, c = 0.0;
    for (int t = threadIdx.x; t < n; t += kAcfThreads) {
        const double d = o[t] - mean;
        v += d * d;
        if (t < n - k) c += d * (o[t + k] - mean);
    }
    v = acf_block_sum(v, sm);
    c = acf_block_sum(c, sm);
    if (threadIdx.x == 0) acf[(size_t)s * (max_lag + 1) + k] = (c / (n - k)) / (v / n);
}

__global__ void k_tau(const double* __restrict__ acf, int n_series, int max_lag, double a_hi, double a_lo,
                      double* __restrict__ tau) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_series) return;
    const double* a = acf + (size_t)s * (max_lag + 1);
    double sk = 0.0, sy = 0.0, skk = 0.0, sky = 0.0;
    int cnt = 0;
    bool started = false;
    for (int k = 1; k <= max_lag; ++k) {
        const double v = a[k];
        if (!(v >= a_lo)) break;  // below the noise floor (or NaN): the decay region ends
        if (!started && v <= a_hi) started = true;
        if (started) {
            const double y = log(v);
            sk += k;
            sy += y;
            skk += (double)k * k;
            sky += k * y;
            ++cnt;
        }
    }
    if (cnt < 2) {
        tau[s] = __longlong_as_double(0x7ff8000000000000ll);  // NaN
        return;
    }
    const double slope = (cnt * sky - sk * sy) / (cnt * skk - sk * sk);
    tau[s] = -1.0 / slope;
}

}  // namespace nb

extern "C" nb_status autocorrelation(const double* series, int32_t n_series, int32_t n, int32_t max_lag, double a_hi,
                                     double a_lo, double* acf, double* tau, void* stream) {
    if (!series || !acf || n_series < 1 || n < 2 || max_lag < 1 || max_lag >= n || !(a_lo > 0.0) ||
        !(a_hi > a_lo) || !(a_hi <= 1.0) || n_series > 65535)
        return NB_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    nb::k_acf<<<dim3(max_lag + 1, n_series), nb::kAcfThreads, 0, st>>>(series, n, max_lag, acf);
    if (tau) nb::k_tau<<<nb::cdiv(n_series, 64), 64, 0, st>>>(acf, n_series, max_lag, a_hi, a_lo, tau);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}
