// The likelihood distribution of the accuracy criterion (Sec. 5.2.2): for K
// noise realisations of data that the model describes up to uncorrelated
// Gaussian noise of amplitude sigma_noise, the residual D - M is the noise
// itself, so eq. likelihood (Sec. 2.3.1) gives
//
//   L_noise[k] = -1/2 [ n ln(2 pi sigma_n^2) + (sigma_noise / sigma_n)^2 sum_cells z[k,cell]^2 ]
//
// and q_i = P(L_noise <= L_bar_i) for a fitted likelihood L_bar_i.
//
// The draws z follow one counter-based definition: cells in pairs (2j, 2j+1),
// pair j of realisation k from Philox4x32-10 (Salmon et al. 2011) with counter
// (j, k mod 2^32, k / 2^32, 0) and key (seed mod 2^32, seed / 2^32), uniforms
// u = (x + 1) / 2^32 of its first two words and the Box-Muller transform
// z_2j = r cos(2 pi u2), z_2j+1 = r sin(2 pi u2), r^2 = -2 ln u1.  The sum of
// squares of a whole pair is r^2 exactly (cos^2 + sin^2 = 1), so a pair costs
// one Philox block and one logarithm; only an odd last cell needs its cosine.
//
// One 256-thread block per realisation; each thread sums its pairs with a
// compensated FP32 sum, the block combines the threads in a fixed order in
// FP64, so every L_noise[k] is reproducible bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "fg21_internal.h"

namespace fg21 {
namespace {

constexpr int NOISE_THREADS = 256;

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t &o0, uint32_t &o1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    o0 = c0;
    o1 = c1;
}

// uniform (x + 1) / 2^32 in (0, 1] (rounded to FP32)
__device__ __forceinline__ float unif(uint32_t x) { return ((float)x + 1.0f) * 2.3283064365386963e-10f; }

__global__ void __launch_bounds__(NOISE_THREADS) noise_loglike_kernel(int64_t n_cells, double lnorm, double ratio2,
                                                                     uint64_t seed, double *__restrict__ out) {
    __shared__ double part[NOISE_THREADS];
    const int64_t k = blockIdx.x;
    const int64_t n_pairs = n_cells / 2;
    const uint32_t klo = (uint32_t)k, khi = (uint32_t)((uint64_t)k >> 32);
    const uint32_t s0 = (uint32_t)seed, s1 = (uint32_t)(seed >> 32);
    float s = 0.0f, c = 0.0f;   // compensated sum of r^2 over this thread's pairs
    for (int64_t j = threadIdx.x; j < n_pairs; j += NOISE_THREADS) {
        uint32_t x0, x1;
        philox4x32_10((uint32_t)j, klo, khi, 0u, s0, s1, x0, x1);
        const float r2 = -2.0f * logf(unif(x0));
        const float y = r2 - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    double v = (double)s - (double)c;
    if (threadIdx.x == 0 && (n_cells & 1)) {
        // odd last cell: only the cosine member of pair n_pairs
        uint32_t x0, x1;
        philox4x32_10((uint32_t)n_pairs, klo, khi, 0u, s0, s1, x0, x1);
        const double r2 = -2.0 * (double)logf(unif(x0));
        const double cs = cospi(2.0 * (double)unif(x1));
        v += r2 * cs * cs;
    }
    part[threadIdx.x] = v;
    __syncthreads();
    // fixed-order tree over the block
    for (int w = NOISE_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = -0.5 * ((double)n_cells * lnorm + ratio2 * part[0]);
}

// q_i = (number of k with L_noise[k] <= L_bar_i) / K: one block per L_bar_i.
__global__ void __launch_bounds__(NOISE_THREADS) noise_q_kernel(const double *__restrict__ L, int64_t K,
                                                               const double *__restrict__ L_bar,
                                                               unsigned long long *__restrict__ count) {
    __shared__ unsigned long long part[NOISE_THREADS];
    const double b = L_bar[blockIdx.x];
    unsigned long long n = 0;
    for (int64_t k = threadIdx.x; k < K; k += NOISE_THREADS) n += L[k] <= b;
    part[threadIdx.x] = n;
    __syncthreads();
    for (int w = NOISE_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) count[blockIdx.x] = part[0];
}

}  // namespace
}  // namespace fg21

using namespace fg21;

extern "C" int fg21_noise_loglike(int64_t n_cells, double sigma_noise, double sigma_n, int64_t K, uint64_t seed,
                                  double *d_L_noise, void *stream) {
    if (n_cells < 1 || K < 0 || (K > 0 && !d_L_noise)) return set_error(FG21_E_ARG, "bad noise_loglike arguments");
    if (!(sigma_n > 0.0) || !std::isfinite(sigma_n) || !(sigma_noise >= 0.0) || !std::isfinite(sigma_noise))
        return set_error(FG21_E_ARG, "sigma_n must be > 0 and sigma_noise >= 0, both finite");
    if (n_cells / 2 >= ((int64_t)1 << 32) || K > (int64_t)INT32_MAX)
        return set_error(FG21_E_RANGE, "n_cells below 2^33 and K below 2^31 only");
    if (K == 0) return FG21_OK;
    const double lnorm = std::log(2.0 * 3.14159265358979323846 * sigma_n * sigma_n);
    const double ratio2 = (sigma_noise / sigma_n) * (sigma_noise / sigma_n);
    noise_loglike_kernel<<<(unsigned)K, NOISE_THREADS, 0, (cudaStream_t)stream>>>(n_cells, lnorm, ratio2, seed,
                                                                                  d_L_noise);
    FG21_CUDA_TRY(cudaGetLastError());
    return FG21_OK;
}

extern "C" int fg21_noise_q(const double *d_L_noise, int64_t K, const double *L_bar, int64_t n_bar, double *q,
                            void *stream) {
    if (K < 1 || !d_L_noise || n_bar < 0 || (n_bar > 0 && (!L_bar || !q)))
        return set_error(FG21_E_ARG, "bad noise_q arguments");
    if (n_bar == 0) return FG21_OK;
    if (n_bar > (int64_t)INT32_MAX) return set_error(FG21_E_RANGE, "too many L_bar values");
    cudaStream_t s = (cudaStream_t)stream;
    double *d_bar = nullptr;
    unsigned long long *d_cnt = nullptr;
    FG21_CUDA_TRY(cudaMallocAsync((void **)&d_bar, sizeof(double) * n_bar, s));
    cudaError_t e = cudaMallocAsync((void **)&d_cnt, sizeof(unsigned long long) * n_bar, s);
    std::vector<unsigned long long> cnt;
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_bar, L_bar, sizeof(double) * n_bar, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        noise_q_kernel<<<(unsigned)n_bar, NOISE_THREADS, 0, s>>>(d_L_noise, K, d_bar, d_cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        cnt.resize(n_bar);
        e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(unsigned long long) * n_bar, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d_bar, s);
    cudaFreeAsync(d_cnt, s);
    if (e != cudaSuccess) return cuda_error(e, "noise_q");
    for (int64_t i = 0; i < n_bar; ++i) q[i] = (double)cnt[i] / (double)K;
    return FG21_OK;
}
