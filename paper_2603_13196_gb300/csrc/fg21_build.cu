// Region building on the GPU: the per-pixel importance weights (Sec. 4.2,
// eq. w_beam_dynamic and its sky / horizon / uniform variants) and the
// chromatic response functions of the partition (Sec. 2.2, eq.
// chromatic_function), the O(Npix F T) parts of fg21_build_regions.  The
// partition itself (sorting by the field and Algorithms 1 / 2) stays on the
// host: it is O(Npix log Npix).
//
// The arithmetic is the host's, in FP64: ln c = ln(z_t . v) per (pixel, LST),
// the beam D = 2(p+1) exp(p ln c) above the horizon, T_sky of eq.
// skyapproximation.  Only the summation order differs (fixed-order block
// trees over pixels, then over channels), so the results agree with the host
// to FP64 rounding; every sum is deterministic.
//
//   pass 1, one block per (f, t):   den[f,t] = sum_q num(q,f,t),  Bsum[f,t] = sum_q D(q,f,t)
//   pass 2, one thread per (q, f):  pw[f,q]  = sum_t num(q,f,t) / den[f,t];
//           one thread per q:       w[q]     = (1/(F T)) sum_f pw[f,q]
//   pass 3, one block per (f, t):   A[c,f,t] = (1/Npix) sum_{q in component c} (T230_q - T_CMB) D(q,f,t)
//           over the pixels sorted by component (contiguous segments).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fg21_internal.h"

namespace fg21 {
namespace {

constexpr int BUILD_THREADS = 256;

struct DevObs {
    const double *lognu;   // [F] ln(nu_f / nu0)
    const double *beam_p;  // [F]
    const double *logcT;   // [T][npix] ln(z_t . v_q), -inf below the horizon
    const double *tskyT;   // [F][npix] T_sky(q, f) (sky and beam weightings)
    int64_t npix;
    int F, T;
    double t_cmb;
};

__device__ __forceinline__ double beam_d(double lc, double p) {
    if (lc == -INFINITY) return 0.0;
    return 2.0 * (p + 1.0) * (p == 0.0 ? 1.0 : exp(p * lc));
}

__device__ __forceinline__ double importance_num(const DevObs &o, int weighting, int64_t q, int f, double lc,
                                                 double d) {
    switch (weighting) {
        case FG21_WEIGHT_BEAM: return o.tskyT[(size_t)f * o.npix + q] * d;
        case FG21_WEIGHT_SKY: return lc == -INFINITY ? 0.0 : o.tskyT[(size_t)f * o.npix + q];
        case FG21_WEIGHT_HORIZON: return lc == -INFINITY ? 0.0 : 1.0;
        default: return 1.0;
    }
}

// fixed-order tree over the block (BUILD_THREADS doubles in shared memory)
__device__ __forceinline__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = BUILD_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void logc_kernel(const double *__restrict__ dirs, const double *__restrict__ zen, int64_t npix, int T,
                            double *__restrict__ logcT) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix * T) return;
    const int t = (int)(i / npix);
    const int64_t q = i - (int64_t)t * npix;
    const double *v = dirs + 3 * q, *z = zen + 3 * t;
    const double c = v[0] * z[0] + v[1] * z[1] + v[2] * z[2];
    logcT[i] = c > 0.0 ? log(c) : -INFINITY;
}

__global__ void tsky_kernel(const double *__restrict__ t230, const double *__restrict__ beta,
                            const double *__restrict__ lognu, double t_cmb, int64_t npix, int F,
                            double *__restrict__ tskyT) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix * F) return;
    const int f = (int)(i / npix);
    const int64_t q = i - (int64_t)f * npix;
    tskyT[i] = (t230[q] - t_cmb) * exp(-beta[q] * lognu[f]) + t_cmb;
}

__global__ void __launch_bounds__(BUILD_THREADS) den_kernel(DevObs o, int weighting, double *__restrict__ den,
                                                            double *__restrict__ bsum) {
    __shared__ double sh[BUILD_THREADS];
    const int ft = blockIdx.x, f = ft / o.T, t = ft % o.T;
    const double p = o.beam_p[f];
    const double *lc_row = o.logcT + (size_t)t * o.npix;
    double a = 0.0, b = 0.0;
    for (int64_t q = threadIdx.x; q < o.npix; q += BUILD_THREADS) {
        const double lc = lc_row[q];
        const double d = beam_d(lc, p);
        a += importance_num(o, weighting, q, f, lc, d);
        b += d;
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) {
        den[ft] = a;
        bsum[ft] = b;
    }
}

__global__ void __launch_bounds__(BUILD_THREADS) pw_kernel(DevObs o, int weighting,
                                                           const double *__restrict__ inv_den,
                                                           double *__restrict__ pw) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int f = blockIdx.y;
    if (q >= o.npix) return;
    const double p = o.beam_p[f];
    double acc = 0.0;
    for (int t = 0; t < o.T; ++t) {
        const double lc = o.logcT[(size_t)t * o.npix + q];
        acc += importance_num(o, weighting, q, f, lc, beam_d(lc, p)) * inv_den[(size_t)f * o.T + t];
    }
    pw[(size_t)f * o.npix + q] = acc;
}

__global__ void w_kernel(const double *__restrict__ pw, int64_t npix, int F, double inv_ft, double *__restrict__ w) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npix) return;
    double acc = 0.0;
    for (int f = 0; f < F; ++f) acc += pw[(size_t)f * npix + q];
    w[q] = acc * inv_ft;
}

__global__ void __launch_bounds__(BUILD_THREADS) resp_kernel(DevObs o, const double *__restrict__ t230,
                                                             const int64_t *__restrict__ perm,
                                                             const int64_t *__restrict__ seg, int N,
                                                             double *__restrict__ A) {
    __shared__ double sh[BUILD_THREADS];
    const int ft = blockIdx.x, f = ft / o.T, t = ft % o.T;
    const double p = o.beam_p[f];
    const double *lc_row = o.logcT + (size_t)t * o.npix;
    const double inv = 1.0 / (double)o.npix;
    for (int c = 0; c < N; ++c) {
        double a = 0.0;
        for (int64_t k = seg[c] + threadIdx.x; k < seg[c + 1]; k += BUILD_THREADS) {
            const int64_t q = perm[k];
            a += (t230[q] - o.t_cmb) * beam_d(lc_row[q], p);
        }
        a = block_sum(a, sh);
        if (threadIdx.x == 0) A[((size_t)c * o.F + f) * o.T + t] = a * inv;
    }
}

// Device copies of the inputs and the geometry tables, freed on destruction.
struct DevBuild {
    double *dirs = nullptr, *t230 = nullptr, *beta = nullptr, *lognu = nullptr, *beam_p = nullptr, *zen = nullptr;
    double *logcT = nullptr, *tskyT = nullptr;
    std::vector<void *> extra;
    ~DevBuild() {
        void *ps[] = {dirs, t230, beta, lognu, beam_p, zen, logcT, tskyT};
        for (void *p : ps)
            if (p) cudaFree(p);
        for (void *p : extra) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T **p, size_t n) {
        cudaError_t e = cudaMalloc((void **)p, sizeof(T) * n);
        if (e == cudaSuccess) extra.push_back(*p);
        return e;
    }
};

cudaError_t upload(double **dst, const double *src, size_t n) {
    cudaError_t e = cudaMalloc((void **)dst, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, sizeof(double) * n, cudaMemcpyHostToDevice);
    return e;
}

// inputs, ln c per (t, q) and (when needed) T_sky per (f, q)
cudaError_t prepare(const fg21_sky *s, const fg21_obs *o, bool need_tsky, DevBuild &d, DevObs &g) {
    const int64_t npix = s->npix;
    const int F = o->F, T = o->T;
    std::vector<double> lognu(F);
    for (int f = 0; f < F; ++f) lognu[f] = std::log(o->nu[f] / o->nu0);
    cudaError_t e = upload(&d.dirs, s->dirs, 3 * (size_t)npix);
    if (e == cudaSuccess) e = upload(&d.t230, s->t230, npix);
    if (e == cudaSuccess) e = upload(&d.beta, s->beta, npix);
    if (e == cudaSuccess) e = upload(&d.lognu, lognu.data(), F);
    if (e == cudaSuccess) e = upload(&d.beam_p, o->beam_p, F);
    if (e == cudaSuccess) e = upload(&d.zen, o->zenith, 3 * (size_t)T);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.logcT, sizeof(double) * (size_t)npix * T);
    if (e != cudaSuccess) return e;
    const int th = BUILD_THREADS;
    logc_kernel<<<(unsigned)((npix * T + th - 1) / th), th>>>(d.dirs, d.zen, npix, T, d.logcT);
    e = cudaGetLastError();
    if (e == cudaSuccess && need_tsky) {
        e = cudaMalloc((void **)&d.tskyT, sizeof(double) * (size_t)npix * F);
        if (e == cudaSuccess) {
            tsky_kernel<<<(unsigned)((npix * F + th - 1) / th), th>>>(d.t230, d.beta, d.lognu, o->t_cmb, npix, F,
                                                                     d.tskyT);
            e = cudaGetLastError();
        }
    }
    g.lognu = d.lognu;
    g.beam_p = d.beam_p;
    g.logcT = d.logcT;
    g.tskyT = d.tskyT;
    g.npix = npix;
    g.F = F;
    g.T = T;
    g.t_cmb = o->t_cmb;
    return e;
}

int fail(cudaError_t e, const char *what) {
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return set_error(FG21_E_NOMEM, "%s: device allocation failed", what);
    return cuda_error(e, what);
}

}  // namespace

int device_importance(const fg21_sky *s, const fg21_obs *o, int weighting, std::vector<double> &w,
                      std::vector<double> *B) {
    DevBuild d;
    DevObs g{};
    const bool need_tsky = weighting == FG21_WEIGHT_BEAM || weighting == FG21_WEIGHT_SKY;
    cudaError_t e = prepare(s, o, need_tsky, d, g);
    if (e != cudaSuccess) return fail(e, "region building (inputs)");
    const int64_t npix = s->npix;
    const int F = o->F, T = o->T;
    double *den = nullptr, *bsum = nullptr, *pw = nullptr, *dw = nullptr;
    e = d.alloc(&den, (size_t)F * T);
    if (e == cudaSuccess) e = d.alloc(&bsum, (size_t)F * T);
    if (e == cudaSuccess) e = d.alloc(&pw, (size_t)F * npix);
    if (e == cudaSuccess) e = d.alloc(&dw, (size_t)npix);
    if (e != cudaSuccess) return fail(e, "region building (importance)");
    den_kernel<<<(unsigned)(F * T), BUILD_THREADS>>>(g, weighting, den, bsum);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "den_kernel");
    std::vector<double> h_den((size_t)F * T), h_b((size_t)F * T);
    if ((e = cudaMemcpy(h_den.data(), den, sizeof(double) * F * T, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(h_b.data(), bsum, sizeof(double) * F * T, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(e, "region building (den)");
    for (auto &x : h_den) x = x > 0.0 ? 1.0 / x : 0.0;
    if ((e = cudaMemcpy(den, h_den.data(), sizeof(double) * F * T, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "region building (1/den)");
    const int th = BUILD_THREADS;
    pw_kernel<<<dim3((unsigned)((npix + th - 1) / th), (unsigned)F), th>>>(g, weighting, den, pw);
    w_kernel<<<(unsigned)((npix + th - 1) / th), th>>>(pw, npix, F, 1.0 / ((double)F * (double)T), dw);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "w_kernel");
    w.resize(npix);
    if ((e = cudaMemcpy(w.data(), dw, sizeof(double) * npix, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(e, "region building (w)");
    if (B) {
        B->resize((size_t)F * T);
        for (size_t k = 0; k < h_b.size(); ++k) (*B)[k] = h_b[k] / (double)npix;
    }
    return FG21_OK;
}

int device_precompute(const fg21_sky *s, const fg21_obs *o, const std::vector<int32_t> &lab, int N,
                      std::vector<double> &A, std::vector<double> &B) {
    DevBuild d;
    DevObs g{};
    cudaError_t e = prepare(s, o, false, d, g);
    if (e != cudaSuccess) return fail(e, "region building (inputs)");
    const int64_t npix = s->npix;
    const int F = o->F, T = o->T;
    // pixels of each component contiguous, in index order within a component
    std::vector<int64_t> seg(N + 1, 0), perm(npix);
    for (int64_t q = 0; q < npix; ++q) seg[lab[q] + 1]++;
    for (int c = 0; c < N; ++c) seg[c + 1] += seg[c];
    {
        std::vector<int64_t> pos(seg.begin(), seg.end() - 1);
        for (int64_t q = 0; q < npix; ++q) perm[pos[lab[q]]++] = q;
    }
    int64_t *dperm = nullptr, *dseg = nullptr;
    double *dA = nullptr, *den = nullptr, *bsum = nullptr;
    e = d.alloc(&dperm, (size_t)npix);
    if (e == cudaSuccess) e = d.alloc(&dseg, (size_t)N + 1);
    if (e == cudaSuccess) e = d.alloc(&dA, (size_t)N * F * T);
    if (e == cudaSuccess) e = d.alloc(&den, (size_t)F * T);
    if (e == cudaSuccess) e = d.alloc(&bsum, (size_t)F * T);
    if (e == cudaSuccess) e = cudaMemcpy(dperm, perm.data(), sizeof(int64_t) * npix, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dseg, seg.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(e, "region building (precompute)");
    resp_kernel<<<(unsigned)(F * T), BUILD_THREADS>>>(g, d.t230, dperm, dseg, N, dA);
    // B = (1/Npix) sum_q D: the uniform weighting's pass 1 gives it without T_sky
    den_kernel<<<(unsigned)(F * T), BUILD_THREADS>>>(g, FG21_WEIGHT_UNIFORM, den, bsum);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "resp_kernel");
    A.resize((size_t)N * F * T);
    B.resize((size_t)F * T);
    if ((e = cudaMemcpy(A.data(), dA, sizeof(double) * A.size(), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(B.data(), bsum, sizeof(double) * B.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(e, "region building (A, B)");
    for (auto &x : B) x /= (double)npix;
    return FG21_OK;
}

}  // namespace fg21
