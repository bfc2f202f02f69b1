// Per-request preparation, SIMT likelihood kernels and the fixed-order
// reduction of libfg21 (sm_103a).
//
// The likelihood of eq. likelihood (Sec. 2.3.1) over the fast forward model of
// eq. fast_forward_model (Sec. 2.2) is evaluated in a reference-subtracted form:
// with a per-request reference spectral index bbar_i (the midrange of the
// request's valid points) and wbar_{i,f} = (nu_f/nu0)^-bbar_i,
//
//   D - M = dref[f,t] - sum_i (wbar_{i,f} A[i,f,t]) expm1(-(beta_{p,i} - bbar_i) L_f) - T21(nu_f)
//   dref[f,t] = D[f,t] - sum_i wbar_{i,f} A[i,f,t] - T_CMB B[f,t]          (FP64, once per request)
//
// which is an exact rearrangement of D - M.  The large foreground cancels in
// FP64 inside dref, so the per-point arithmetic only carries the (small)
// departure of each point from the reference.  The plain FP32 form
// (FG21_PREC_FP32_DIRECT) evaluates M directly and is kept as the comparator.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "fg21_internal.h"
#include "fg21_pdl.cuh"

namespace fg21 {

namespace {

constexpr int PREP_THREADS = 256;
constexpr int FIN_GROUP_SCRATCH = 512;   // floats of per-group finalise results
// Head of the prep kernels' shared memory, in doubles: bbar [NPF] FP64, the
// finalise scratch [2 NPF + 2 + 16] FP32 and the group results [FIN_GROUP_SCRATCH] FP32.
__host__ __device__ inline int prep_head_doubles(int NP) {
    return NP + (2 * NP + 2 + 16 + 1) / 2 + FIN_GROUP_SCRATCH / 2;
}
constexpr int REDUCE_THREADS = 64;
constexpr int REDUCE_SERIAL_MAX = 32;       // longest partial row summed by one thread

// A point is valid when all its parameters are finite, sigma_n > 0,
// sigma21 != 0 and every amplitude scale factor alpha_i > 0 (a gain).  Tested
// on the bit patterns (integer instructions; FP64 is a scarce pipe on this
// part).
__device__ __forceinline__ bool point_valid(const double *th, const ReqDesc &r) {
    const int NP = r.NPF;
    bool ok = true;
    for (int k = 0; k < NP + 4; ++k)
        ok &= (__double_as_longlong(th[k]) & 0x7FF0000000000000ll) != 0x7FF0000000000000ll;
    ok &= __double_as_longlong(th[NP + 3]) > 0;                                // > +0 (sign clear)
    ok &= (__double_as_longlong(th[NP + 2]) & 0x7FFFFFFFFFFFFFFFll) != 0;     // != +-0
    for (int k = r.Nb; k < NP; ++k) ok &= __double_as_longlong(th[k]) > 0;    // alpha > +0
    return ok;
}


// a1, pass 1: per block of STAT_BLOCK points (one thread each), the min and
// max of each foreground parameter (each region's beta, then each amplitude
// alpha) over valid points, the valid count and max |A21|.  The reference
// point is the midrange (min + max) / 2: the rearranged likelihood is exact for
// any reference, and the midrange minimises max |theta - reference|, the bound
// that sets the weight series.  FP32, warp reductions by redux.sync.
__device__ __forceinline__ float warp_min(float v) {
    float r;
    asm("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float warp_max(float v) {
    float r;
    asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
// Warps reduce by shuffles in a fixed tree and are combined in warp order.
// Largest s with 2^s * maxabs <= 2^15 (half the FP16 range), clamped to
// [-40, 40]; exact, from the exponent and mantissa bits (no FP64 log).
__device__ __forceinline__ int pow2_exponent_for(float maxabs) {
    if (!(maxabs > 0.0f)) return 0;
    const unsigned u = __float_as_uint(maxabs);
    const int eb = (int)((u >> 23) & 0xFFu), mant = (int)(u & 0x7FFFFFu);
    if (eb == 0) return 40;                       // subnormal: far below the range
    if (eb == 0xFF) return -40;
    // maxabs in (2^(eb-128), 2^(eb-127)] ... ceil(log2 maxabs) = eb - 127 + (mant != 0)
    const int s = 15 - (eb - 127) - (mant != 0 ? 1 : 0);
    return max(-40, min(40, s));
}

template <bool BF16>
__device__ __forceinline__ uint32_t pack_pair(float a, float b) {
    if (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}
template <bool BF16>
__device__ __forceinline__ float2 unpack_pair(uint32_t u) {
    if (BF16) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
        return __bfloat1622float2(h);
    } else {
        __half2 h = *reinterpret_cast<__half2 *>(&u);
        return __half22float2(h);
    }
}

// double -> float rounded to nearest (ties away from zero) with integer
// instructions: conversions run on the FP64 pipe, which is scarce on this
// part.  Below the normal float range the result is a signed zero, above it
// (and for NaN) a signed infinity.
__device__ __forceinline__ float f32_of_f64(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);       // mantissa bits 51..29
    return __uint_as_float((sign | ((unsigned)e << 23) | m) + ((lo >> 28) & 1u));   // a carry rounds up the exponent
}

// 8-byte asynchronous copy global -> shared (no register staging; the copies
// of a thread stay in flight until cp_async_wait_all).
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Packed FP32 pairs for the SIMT kernels' FMAs (fma.rn.f32x2: two lanes of
// round-to-nearest FMA in one instruction).
__device__ __forceinline__ uint64_t pk2f(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2f(uint64_t v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2f(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// All but the most recent committed group have completed.
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

// The block's parameter rows [np][R] (contiguous at src) into shared rows of
// Rp doubles, one 8-byte cp.async per element in the flat order of the source
// (coalesced), the (row, column) of each thread stepped without a division.
__device__ __forceinline__ void copy_rows8(double *dst, int Rp, const double *src, int R, int np) {
    int row = (int)threadIdx.x / R, col = (int)threadIdx.x - row * R;
    const int drow = (int)blockDim.x / R, dcol = (int)blockDim.x - drow * R;
    while (row < np) {
        cp_async8(dst + (size_t)row * Rp + col, src + (size_t)row * R + col);
        col += dcol;
        row += drow;
        if (col >= R) {
            col -= R;
            ++row;
        }
    }
}

// (sh, sl) += (xh, xl) in double-float arithmetic: Knuth's two-sum of the high
// parts, the low parts added to its error, then renormalised.
__device__ __forceinline__ void df_add(float &sh, float &sl, float xh, float xl) {
    const float s = sh + xh;
    const float bb = s - sh;
    const float err = ((sh - (s - bb)) + (xh - bb)) + (sl + xl);
    sh = s + err;
    sl = err - (sh - s);
}

// Parameter rows staged in shared memory are padded to an odd number of
// doubles so that a warp reading one value of 32 consecutive rows spreads over
// the banks.
__host__ __device__ __forceinline__ int padded_row(int R) { return R | 1; }

// a1, pass 2, run by every block of the second prep kernel: the reference
// point (bbar_i = midrange of the valid points' beta_i, and abar_i = midrange
// of alpha_i with amplitude regions), a bound x on the weights' expm1 argument,
// max_i |beta - bbar_i| * max_f |L_f| + max_i |ln(alpha / abar_i)| (it sets the
// weight series and the power-of-two scale sW of the weight operand), the
// valid count and max |A21|.
// The fields are minima, maxima and an exact integer count, so the order in
// which the stat blocks combine does not change a bit: G threads share each
// field (thread (g, j) takes blocks g, g+G, ..., sixteen independent loads per
// round), then thread j combines the G results.  Every block computes the same
// values bit for bit; bbar goes to shared memory (`bbar_sh`), and block 0 of the
// request publishes the results for the later kernels.
struct Fin {
    float nv, ma, x;
    int sW;
};
__device__ Fin prep_finalize(const ReqDesc &r, float *sh /* [2 NPF + 2 + 2 nwarps] */,
                             float *gpart /* [FIN_GROUP_SCRATCH] */, double *bbar_sh, bool publish) {
    const int N = r.NPF, Nb = r.Nb, nb = r.n_stat_blocks, W = 2 * N + 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int G = max(1, min((int)blockDim.x / W, FIN_GROUP_SCRATCH / W));
    for (int idx = threadIdx.x; idx < G * W; idx += blockDim.x) {
        const int g = idx / W, j = idx - g * W;
        const int kind = j < 2 * N ? 1 + (j & 1) : (j == 2 * N ? 0 : 2);   // 0 count, 1 min, 2 max
        const float *q = r.stat_part + j;
        float v = kind == 0 ? 0.0f : kind == 1 ? INFINITY : -INFINITY;
        for (int b0 = g; b0 < nb; b0 += 16 * G) {
            float x[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) x[u] = b0 + u * G < nb ? __ldg(q + (size_t)(b0 + u * G) * W) : 0.0f;
#pragma unroll
            for (int u = 0; u < 16; ++u)
                if (b0 + u * G < nb) v = kind == 0 ? v + x[u] : kind == 1 ? fminf(v, x[u]) : fmaxf(v, x[u]);
        }
        gpart[idx] = v;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        const int kind = j < 2 * N ? 1 + (j & 1) : (j == 2 * N ? 0 : 2);
        float v = gpart[j];
        for (int g = 1; g < G; ++g) {
            const float x = gpart[g * W + j];
            v = kind == 0 ? v + x : kind == 1 ? fminf(v, x) : fmaxf(v, x);
        }
        sh[j] = v;
    }
    __syncthreads();
    const float nv = sh[2 * N], ma = sh[2 * N + 1];
    float dev = 0.0f, gdev = 0.0f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float mn = sh[2 * i], mx = sh[2 * i + 1];
        const float bb = nv > 0.0f ? 0.5f * (mn + mx) : 0.0f;
        bbar_sh[i] = (double)bb;
        if (publish) r.beta_bar[i] = (double)bb;
        if (nv > 0.0f) {
            if (i < Nb) dev = fmaxf(dev, fmaxf(mx - bb, bb - mn));
            else gdev = fmaxf(gdev, fmaxf(logf(mx / bb), logf(bb / mn)));   // alpha > 0
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
        gdev = fmaxf(gdev, __shfl_xor_sync(0xffffffffu, gdev, o));
    }
    float *wred = sh + W;
    if (lane == 0) {
        wred[warp] = dev;
        wred[nw + warp] = gdev;
    }
    __syncthreads();
    float dmax = 0.0f, gmax = 0.0f;
    for (int w = 0; w < nw; ++w) {
        dmax = fmaxf(dmax, wred[w]);
        gmax = fmaxf(gmax, wred[nw + w]);
    }
    Fin f;
    // a small margin on x covers the FP32 statistics
    f.x = (dmax * (float)r.Lmax + gmax) * 1.0001f;
    f.nv = nv;
    f.ma = ma;
    f.sW = pow2_exponent_for(fmaxf(fmaxf(expm1f(f.x), ma), 1.0f));
    if (publish && threadIdx.x == 0) {
        r.req_stats[0] = nv;
        r.req_stats[1] = f.x;
        r.req_stats[2] = ma;
        *r.scaleW = f.sW;
    }
    __syncthreads();
    return f;
}

__global__ void __launch_bounds__(STAT_BLOCK) prep_stats_kernel(const ReqDesc *__restrict__ reqs, int staged) {
    // shared: [STAT_BLOCK / 32][2 NPF + 2] FP32 warp partials, then (staged) the
    // block's parameter rows [STAT_BLOCK][padded_row(NPF + 4)] FP64
    extern __shared__ double sh_stats_d[];     // [STAT_BLOCK / 32][2 NPF + 2] partials, then the rows
    const ReqDesc &r = reqs[blockIdx.y];
    if ((int)blockIdx.x >= r.n_stat_blocks) return;
    const int N = r.NPF, W = 2 * N + 2, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    float *sh_stats = reinterpret_cast<float *>(sh_stats_d);
    const int64_t p0 = (int64_t)blockIdx.x * STAT_BLOCK, p = p0 + threadIdx.x;
    const int np = (int)min((int64_t)STAT_BLOCK, r.P - p0);
    const double *th;
    if (staged) {
        // coalesced copies of the block's rows, all in flight at once
        const int R = N + 4, Rp = padded_row(R);
        double *slab = sh_stats_d + (nw * W + 1) / 2;
        const double *src = r.params + p0 * R;
        copy_rows8(slab, Rp, src, R, np);
        cp_async_wait_all();
        __syncthreads();
        th = slab + (size_t)(p < r.P ? threadIdx.x : 0) * Rp;
    } else {
        th = r.params + (p < r.P ? p : 0) * (N + 4);
    }
    const bool valid = p < r.P && point_valid(th, r);
    if (p < r.P) r.pvalid[p] = valid;
    float *mine = sh_stats + warp * W;
    for (int i = 0; i < N; ++i) {
        const float b = valid ? f32_of_f64(th[i]) : 0.0f;
        const float mn = warp_min(valid ? b : INFINITY), mx = warp_max(valid ? b : -INFINITY);
        if (lane == 0) {
            mine[2 * i] = mn;
            mine[2 * i + 1] = mx;
        }
    }
    const float nv = (float)__popc(__ballot_sync(0xffffffffu, valid));
    const float ma = warp_max(valid ? fabsf(f32_of_f64(th[N])) : 0.0f);
    if (lane == 0) {
        mine[2 * N] = nv;
        mine[2 * N + 1] = ma;
    }
    __syncthreads();
    float *out = r.stat_part + (size_t)blockIdx.x * W;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        const int kind = j < 2 * N ? 1 + (j & 1) : (j == 2 * N ? 0 : 2);   // 0 sum, 1 min, 2 max
        float v = sh_stats[j];
        for (int w = 1; w < nw; ++w) {
            const float x = sh_stats[w * W + j];
            v = kind == 0 ? v + x : kind == 1 ? fminf(v, x) : fmaxf(v, x);
        }
        out[j] = v;
    }
}

// a1, pass 3: one block per (channel, t-chunk) builds that channel's
// reference: wbar_c = (nu_f/nu0)^-bbar_j (times abar_i with amplitude regions)
// for each component c = (i, j), wbar_c A[c,f,t] and
// dref = D - sum_c wbar_c A_c - T_CMB B (FP64), then writes either the FP32
// arrays of the SIMT delta form or the split-precision operand tile of the
// tensor-core form.  With amplitude regions the weights of a point are
// expm1(-(beta_j - bbar_j) L_f + ln(alpha_i / abar_i)), the same exact
// rearrangement with alpha_i (nu/nu0)^-beta_j = abar_i wbar_j exp(that argument).
//
// Operand tile layout (one per channel and t-chunk, 2 x Kp x Tc_pad 16-bit
// values): [split s in {hi, mid}][k-chunk kc = k/8][t][8 values k%8], i.e. the
// K-major core-matrix layout (8 rows of 16 bytes) the tensor cores read; row k
// < N holds wbar_k A[k,f,t] 2^sB, row Kp-2 holds 2^sB (multiplies the trough
// column of the weights), row Kp-1 holds dref 2^sB (multiplies -1), other rows
// and columns t >= Tc are zero.
//
// Blocks beyond the tiles (tensor path only) write the per-point operands of
// the weight generators, one block per 128-point tile, point-minor so that a
// thread per point reads them coalesced: rows k < Kp-2 hold beta_{p,j} - bbar_j
// of component k's spectral index j in FP32 (zero for k >= N), then A21, nu21
// and 1/(2 sigma21^2); with amplitude regions, rows Kp+4.. hold
// ln(alpha_{p,i} / abar_i) of each component's amplitude i, two components per
// 8-byte pair ([Kp/2][128][2]) so a generator thread loads a pair at once.  The
// last Kp rows hold, in the same pair layout, the low part of each deviation
// (beta - bbar less its FP32 rounding): a deviation rounded to FP32 shifts the
// point by up to 2^-25 of it in every cell of the observation at once, which
// near the posterior of a large observation moves logL by more than 1e-2
// nats, so the generators add its first-order effect to each weight.
// Two threads per point (`half` 0 and 1 of the block): the deviation rows
// alternate between them; half 0 also writes the trough rows and the sigma_n
// terms, half 1 the amplitude rows.  `th` is the point's parameter row (staged
// in shared memory).
__device__ __forceinline__ void prep_points(const ReqDesc &r, int tile, const double *bbar, const double *th) {
    const int pidx = threadIdx.x % TILE_M, half = threadIdx.x / TILE_M;
    if (half > 1) return;
    const int64_t p = (int64_t)tile * TILE_M + pidx;
    const int N = r.N, Nb = r.Nb, NP = r.NPF, Kp = r.Kp;
    float *out = r.pts32 + (size_t)tile * r.pts_rows * TILE_M + pidx;
    // the deviations' low parts: pair-interleaved rows after the other operands
    float *lo_out = out - pidx + (size_t)(Kp + 4 + (r.Na ? Kp : 0)) * TILE_M + 2 * pidx;
    const bool in = p < r.P;
    for (int k = half; k < Kp - 2; k += 2) {
        float v = 0.0f, vlo = 0.0f;
        if (in && k < N) {
            const int j = Nb == N ? k : k % Nb;
            const double dv = th[j] - bbar[j];
            v = f32_of_f64(dv);
            vlo = f32_of_f64(dv - (double)v);
        }
        out[(size_t)k * TILE_M] = v;
        lo_out[(size_t)(k >> 1) * 2 * TILE_M + (k & 1)] = vlo;
    }
    lo_out[(size_t)((Kp - 2) >> 1) * 2 * TILE_M + half] = 0.0f;     // the (trough, -1) pair
    if (half == 0) {
        out[(size_t)(Kp - 2) * TILE_M] = in ? f32_of_f64(th[NP]) : 0.0f;
        out[(size_t)(Kp - 1) * TILE_M] = in ? f32_of_f64(th[NP + 1]) : 0.0f;
        const float s21 = in ? f32_of_f64(th[NP + 2]) : 1.0f;
        out[(size_t)Kp * TILE_M] = 1.0f / (2.0f * s21 * s21);
        // the sigma_n terms of eq. likelihood for the reduction (FP64, once per point)
        if (in && r.pvalid[p]) {
            const double sig = th[NP + 3];
            r.pnorm[p] = make_double2((double)r.F * (double)r.T * log(2.0 * 3.141592653589793 * sig * sig),
                                      1.0 / (sig * sig));
        }
        return;
    }
    if (r.Na) {
        float2 *g2 = reinterpret_cast<float2 *>(out - pidx + (size_t)(Kp + 4) * TILE_M) + pidx;
        int icur = -1;
        float gcur = 0.0f;
        for (int q = 0; q < Kp / 2; ++q) {
            float gv[2];
            for (int e = 0; e < 2; ++e) {
                const int c = 2 * q + e;
                float v = 0.0f;
                if (in && c < N) {
                    const int ia = c / Nb;
                    if (ia != icur) {
                        icur = ia;
                        const double ab = bbar[Nb + ia];
                        gcur = log1pf(f32_of_f64(th[Nb + ia] - ab) / f32_of_f64(ab));   // ln(alpha / abar)
                    }
                    v = gcur;
                }
                gv[e] = v;
            }
            g2[(size_t)q * TILE_M] = make_float2(gv[0], gv[1]);
        }
    }
}

// a1 for the SIMT forms, pass 3: one block per (channel, t-chunk) builds that
// channel's reference -- wbar_c (FP64), dref[t] = D - sum_c wbar_c A_c - T_CMB B
// summed in ascending c (FP64: the foreground cancels here) -- and writes the
// FP32 arrays of the delta form (wbar_c A_c and dref); the direct form only
// needs the per-channel tables.  The blocks after them write the FP32 parameter
// rows of one 128-point tile each (pts32): the spectral indices (direct form)
// or their deviations beta - bbar (delta form), then the amplitudes (direct) or
// ln(alpha / abar) (delta).
template <int MODE>  // 2 = SIMT delta, 3 = SIMT direct
__global__ void __launch_bounds__(PREP_THREADS) prep_tiles_kernel(const ReqDesc *__restrict__ reqs) {
    extern __shared__ double smem_d[];
    pdl_wait();
    const ReqDesc &r = reqs[blockIdx.y];
    const int nfc = r.F * r.n_tchunks;
    const int N = r.N, NP = r.NPF, Nb = r.Nb, T = r.T;
    if ((int)blockIdx.x >= nfc + r.n_tiles) return;
    // shared memory: the head (bbar, finalise scratch and group results), then wbar [N] FP64
    double *bbar = smem_d;
    float *fin_sh = reinterpret_cast<float *>(bbar + NP);
    float *gpart = reinterpret_cast<float *>(bbar + NP + (2 * NP + 2 + 16 + 1) / 2);
    double *wbar = bbar + prep_head_doubles(NP);
    prep_finalize(r, fin_sh, gpart, bbar, blockIdx.x == 0);
    if ((int)blockIdx.x >= nfc) {
        const int tile = blockIdx.x - nfc, Na = r.Na;
        float *rows = r.pts32 + (size_t)tile * r.pts_rows * TILE_M;
        for (int q = threadIdx.x; q < (Nb + Na) * TILE_M; q += blockDim.x) {
            const int j = q / TILE_M, m = q - j * TILE_M;
            const int64_t pt = (int64_t)tile * TILE_M + m;
            float v = 0.0f;
            if (pt < r.P) {
                const double th = r.params[pt * (NP + 4) + j];
                if (j < Nb) v = MODE == 3 ? (float)th : (float)(th - bbar[j]);
                else v = MODE == 3 ? (float)th : log1pf((float)(th - bbar[j]) / (float)bbar[j]);
            }
            rows[q] = v;
        }
        return;
    }
    const int fc = blockIdx.x;
    const int f = fc / r.n_tchunks, c = fc % r.n_tchunks;
    const int t0 = c * r.Tc, tn = min(r.Tc, T - t0);
    const double L = r.L[f];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double w = exp(-bbar[i % Nb] * L);
        if (r.Na) w *= bbar[Nb + i / Nb];
        wbar[i] = w;
    }
    if (c == 0 && threadIdx.x == 0) {
        r.nL32[f] = (float)(-L);
        r.nu32[f] = (float)r.nu[f];
    }
    __syncthreads();
    if (MODE != 2) return;
    const size_t istride = (size_t)r.F * T;
    for (int t = threadIdx.x; t < tn; t += blockDim.x) {
        const size_t ft = (size_t)f * T + t0 + t;
        double s = 0.0;
        for (int i0 = 0; i0 < N; i0 += 8) {
            double a[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = i0 + j < N ? r.A[(size_t)(i0 + j) * istride + ft] : 0.0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (i0 + j < N) {
                    const double bw = wbar[i0 + j] * a[j];
                    s += bw;
                    r.Bp32[(size_t)(i0 + j) * istride + ft] = (float)bw;
                }
            }
        }
        r.dref32[ft] = (float)(r.data[ft] - s - r.t_cmb * r.B[ft]);
    }
}

// a1 on the tensor path, pass 3 (one launch): blocks [0, F * n_tchunks) build
// the operand tile of one (channel, t-chunk), the blocks after them the
// per-point operands of one 128-point tile.  Each block first issues
// asynchronous copies of everything it reads (the channel's A slab, D and B;
// or the tile's parameter rows) into shared memory and finalises the request
// statistics while they land, so the DRAM latency of its inputs hides behind
// the statistics.  Then, for a channel block: wbar_c (FP64, split into an FP32
// pair), the products wbar_c A[c,f,t] in place and dref[t] = D - T_CMB B -
// sum_c wbar_c A_c summed in ascending c, both in double-float arithmetic (the
// foreground cancels in dref), the tile scale 2^sB, and the split-precision
// tile from the products rounded to FP32.
//
// Operand tile layout (one per channel and t-chunk, 2 x Kp x Tc_pad 16-bit
// values): [split s in {hi, mid}][k-chunk kc = k/8][t][8 values k%8], i.e. the
// K-major core-matrix layout (8 rows of 16 bytes) the tensor cores read; row k
// < N holds wbar_k A[k,f,t] 2^sB, row Kp-2 holds 2^sB (multiplies the trough
// column of the weights), row Kp-1 holds dref 2^sB (multiplies -1), other rows
// and columns t >= Tc are zero.
//
// Shared memory: bbar [NPF], finalise scratch and group results, then the block's slab --
// channel: the products' hi and lo parts [N][Tc_pad] each, E hi / lo and dref
// [Tc_pad], wbar hi / lo [N] (FP32); points: parameter rows
// [128][padded_row(NPF+4)] FP64.
template <bool BF16>
__global__ void __launch_bounds__(PREP_THREADS) prep_tc_kernel(const ReqDesc *__restrict__ reqs) {
    extern __shared__ double smem_d[];
    __shared__ float sh_red[PREP_THREADS / 32];
    __shared__ int s_scaleB;
    pdl_wait();
    const ReqDesc &r = reqs[blockIdx.y];
    const int nfc = r.F * r.n_tchunks;
    if ((int)blockIdx.x >= nfc + r.n_tiles) return;
    const int N = r.N, NP = r.NPF, Nb = r.Nb, T = r.T;
    double *bbar = smem_d;
    float *fin_sh = reinterpret_cast<float *>(bbar + NP);
    float *gpart = reinterpret_cast<float *>(bbar + NP + (2 * NP + 2 + 16 + 1) / 2);
    double *slab = bbar + prep_head_doubles(NP);
    if ((int)blockIdx.x >= nfc) {
        // ---- per-point operands of one 128-point tile
        const int tile = blockIdx.x - nfc;
        const int64_t p0 = (int64_t)tile * TILE_M;
        const int np = (int)min((int64_t)TILE_M, r.P - p0);
        const int R = NP + 4, Rp = padded_row(R);
        const double *src = r.params + p0 * R;
        copy_rows8(slab, Rp, src, R, np);
        prep_finalize(r, fin_sh, gpart, bbar, false);
        cp_async_wait_all();
        __syncthreads();
        const int pidx = threadIdx.x % TILE_M;
        prep_points(r, tile, bbar, slab + (size_t)(pidx < np ? pidx : 0) * Rp);
        return;
    }
    // ---- operand tile of one (channel, t-chunk), in double-float arithmetic
    // (FP32 pairs; the FP64 pipe of this part is scarce): A = A32 + A_lo and
    // E = D - T_CMB B = E_hi + E_lo come from the model; p_c = wbar_c A_c by an
    // FMA two-product, dref = E - sum_c p_c by two-sums in ascending c (about
    // 2^-47 relative to the foreground, 1e-9 K at 1e4 K).
    const int fc = blockIdx.x;
    const int f = fc / r.n_tchunks, c = fc % r.n_tchunks;
    const int t0 = c * r.Tc, tn = min(r.Tc, T - t0), Tcp = r.Tc_pad;
    float *ph = reinterpret_cast<float *>(slab);   // [N][Tcp] A hi, then the products' hi parts
    float *pl = ph + (size_t)N * Tcp;              // [N][Tcp] A lo, then the products' lo parts
    float *eh = pl + (size_t)N * Tcp;              // [Tcp]
    float *el = eh + Tcp;                          // [Tcp]
    float *dref = el + Tcp;                        // [Tcp] dref rounded to FP32
    float *whi = dref + Tcp;                       // [N]
    float *wlo = whi + N;                          // [N]
    const size_t istride = (size_t)r.F * T, ft0 = (size_t)f * T + t0;
    for (int k = threadIdx.x; k < N * tn; k += blockDim.x) {
        const int i = k / tn, t = k - i * tn;
        cp_async4(ph + (size_t)i * Tcp + t, r.A32 + i * istride + ft0 + t);
        cp_async4(pl + (size_t)i * Tcp + t, r.A_lo + i * istride + ft0 + t);
    }
    for (int t = threadIdx.x; t < tn; t += blockDim.x) {
        cp_async4(eh + t, r.E_hi + ft0 + t);
        cp_async4(el + t, r.E_lo + ft0 + t);
    }
    const Fin fin = prep_finalize(r, fin_sh, gpart, bbar, fc == 0);
    const double L = r.L[f];
    if (c == 0 && threadIdx.x == 32) {
        // the generators' series coefficients for this channel (the same FP32
        // operations, in the same order, as a generator would do them)
        const SeriesPlan sp = series_plan((double)fin.x);
        const float ys = ldexpf(1.0f, -sp.s), sW = ldexpf(1.0f, fin.sW);
        const float y1 = (float)(-L) * ys;
        float pw = sp.s ? 1.0f : sW, fact = 1.0f;
#pragma unroll
        for (int j = 1; j < 9; ++j) {
            pw *= y1;
            fact *= (float)j;
            const float e = pw * (1.0f / fact);
            r.coef2[(size_t)f * 8 + j - 1] =
                ((unsigned long long)__float_as_uint(e) << 32) | (unsigned long long)__float_as_uint(e);
        }
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double w = exp(-bbar[i % Nb] * L);
        if (r.Na) w *= bbar[Nb + i / Nb];
        const float h = f32_of_f64(w);
        whi[i] = h;
        wlo[i] = f32_of_f64(w - (double)h);
    }
    if (c == 0 && threadIdx.x == 0) {
        r.nL32[f] = (float)(-L);
        r.nu32[f] = (float)r.nu[f];
    }
    cp_async_wait_all();
    __syncthreads();
    float vmax = 1.0f;
    for (int k = threadIdx.x; k < N * tn; k += blockDim.x) {
        const int i = k / tn, t = k - i * tn;
        const size_t o = (size_t)i * Tcp + t;
        const float ah = ph[o], al = pl[o], wh = whi[i], wl = wlo[i];
        const float hi = wh * ah;
        const float lo = fmaf(wh, al, fmaf(wl, ah, fmaf(wh, ah, -hi)));   // two-product + cross terms
        const float sh = hi + lo;
        ph[o] = sh;                                 // normalised pair: sh is the product rounded to FP32
        pl[o] = lo - (sh - hi);
        vmax = fmaxf(vmax, fabsf(sh));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tn; t += blockDim.x) {
        float sh = 0.0f, sl = 0.0f;
        for (int i = 0; i < N; ++i) {
            const size_t o = (size_t)i * Tcp + t;
            df_add(sh, sl, ph[o], pl[o]);
        }
        df_add(sh, sl, -eh[t], -el[t]);              // sum_c p_c - E = -dref
        dref[t] = -sh;
        vmax = fmaxf(vmax, fabsf(sh));
    }
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0) sh_red[threadIdx.x >> 5] = vmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = sh_red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, sh_red[w]);
        s_scaleB = pow2_exponent_for(v);
        r.scaleB[fc] = s_scaleB;
    }
    __syncthreads();
    const float sB = ldexpf(1.0f, s_scaleB);
    // one 16-byte chunk (8 values of k) per (split, kc, t); sB is a power of
    // two, so (float)(wbar A) * sB is the FP64 product rounded once
    const int Kp = r.Kp, nkc = Kp / 8;
    uint4 *tile = reinterpret_cast<uint4 *>(r.tiles + (size_t)fc * r.tile_rows * 128);
    for (int j = threadIdx.x; j < nkc * Tcp; j += blockDim.x) {
        const int kc = j / Tcp, t = j % Tcp;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = kc * 8 + e;
            float x = 0.0f;
            if (t < tn) {
                if (k < N) x = ph[(size_t)k * Tcp + t] * sB;              // sB = 2^s: exact
                else if (k == Kp - 2) x = sB;
                else if (k == Kp - 1) x = dref[t] * sB;
            }
            v[e] = x;
        }
        uint32_t H[4], M[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            H[e / 2] = pack_pair<BF16>(v[e], v[e + 1]);
            const float2 h = unpack_pair<BF16>(H[e / 2]);
            M[e / 2] = pack_pair<BF16>(v[e] - h.x, v[e + 1] - h.y);
        }
        tile[(size_t)kc * Tcp + t] = make_uint4(H[0], H[1], H[2], H[3]);                 // split 0 (hi)
        tile[(size_t)(nkc + kc) * Tcp + t] = make_uint4(M[0], M[1], M[2], M[3]);         // split 1 (mid)
    }
}

// ------------------------------------------------------------- SIMT paths
// One block = 128 points of one request x one channel group (an item).  The
// block walks its stages (channel, t-chunk of at most SIMT_TC columns) with
// the next stage's model slab ([N][SIMT_TC]: A for the plain form, wbar A for
// the reference-subtracted form) and data columns copied into the other half
// of a double buffer by cp.async while the current one is used.  Per channel
// the weights of the block's 128 points ([N][128]) and their troughs are
// formed in shared memory.  Each thread computes register tiles of 4 points x
// 8 columns: 32 accumulators, each an FMA chain over the regions in ascending
// order, with the next region's operands (one 16-byte load of weights, two of
// the slab row, addresses stepped by pointer) loaded while the current
// region's FMAs issue, two columns per packed FP32x2 FMA; it squares the
// residuals into its points' sums (packed too: even and odd columns in two
// chains).  Past the first round, the column blocks that do not fill a round
// of the four column slots are shared out by point instead (thread i: point i
// x 8 columns), so every warp carries the same work into the stage's barrier.  The per-point
// sums of a channel are combined in a fixed order and folded over the channels
// into a compensated (hi, lo) FP32 pair.
constexpr int SIMT_THREADS = 128;
constexpr int SIMT_TC = 128;                      // widest t-chunk staged per round (= SIMT_THREADS)
constexpr int SIMT_PT = 4, SIMT_CT = 8;           // register tile: points x columns
constexpr int SIMT_PG = TILE_M / SIMT_PT;         // 32 point groups
constexpr int SIMT_CS = SIMT_THREADS / SIMT_PG;   // 4 column slots
static_assert(SIMT_PT % 4 == 0 && SIMT_CT == 8, "weights load as float4, slab rows as two float4");
static_assert(SIMT_TC == SIMT_THREADS, "the slab is staged one column per thread");
static_assert(SIMT_TC % SIMT_CT == 0, "column blocks tile the t-chunk");

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

__device__ __forceinline__ int find_req_by_item(const ReqDesc *__restrict__ reqs, int n_reqs, int64_t item) {
    int lo = 0, hi = n_reqs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (reqs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_req_by_point(const ReqDesc *__restrict__ reqs, int n_reqs, int64_t pt) {
    int lo = 0, hi = n_reqs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (reqs[mid].pt_begin <= pt) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Shared-memory floats of a SIMT block with N components staging tc columns
// per round: weights [N+1][128] and two slabs [N+1][tc] (one spare row each,
// read ahead by the last region's load and never used), two sets of data
// columns [2][2][128], troughs and per-slot sums.  The points' parameters are
// read from their FP32 rows in global memory (pts32) when a channel's weights
// are formed, which keeps a block small enough for five to share an SM.
__host__ __device__ inline size_t simt_smem_floats(int N, int tc) {
    return (size_t)(N + 1) * TILE_M + 2 * (size_t)(N + 1) * tc + 2 * 2 * SIMT_TC + TILE_M +
           (size_t)(SIMT_CS + 1) * TILE_M;
}
constexpr size_t SIMT_SMEM_MAX = 226 * 1024;      // bytes a block may take (227 KB less the driver's share)

template <bool DIRECT>
__global__ void __launch_bounds__(SIMT_THREADS) simt_kernel(const ReqDesc *__restrict__ reqs, int n_reqs) {
    extern __shared__ __align__(16) float smem_f[];
    pdl_wait();
    const int64_t item = blockIdx.x;
    const ReqDesc &r = reqs[find_req_by_item(reqs, n_reqs, item)];
    const int64_t lid = item - r.item_begin;
    const int tile = (int)(lid / r.G), g = (int)(lid % r.G);
    const int N = r.N, Nb = r.Nb, Na = r.Na, NP = r.NPF, F = r.F, T = r.T;
    const int f0 = g * r.ch_per_group, f1 = min(F, f0 + r.ch_per_group);
    const size_t slab = (size_t)(N + 1) * r.simt_tc;
    float *Wsh = smem_f;                              // [N+1][128] weights
    float *As = Wsh + (size_t)(N + 1) * TILE_M;       // [2][N+1][tc] model slabs
    float *dcol = As + 2 * slab;                      // [2][2][SIMT_TC]: data (or dref), B
    float *s21s = dcol + 4 * SIMT_TC;                 // [128] trough of each point
    float *qp = s21s + TILE_M;                        // [SIMT_CS + 1][128] per-slot point sums
    const int tid = threadIdx.x;
    // this point's parameter rows: [Nb] beta (plain) or beta - bbar, then [Na] alpha or ln(alpha/abar)
    const float *__restrict__ prow = r.pts32 + (size_t)tile * r.pts_rows * TILE_M + tid;
    const int64_t p = (int64_t)tile * TILE_M + tid;   // the point whose weights and sums this thread owns
    const bool inb = p < r.P;
    const int TCr = r.simt_tc;
    const int nck = (T + TCr - 1) / TCr, S = (f1 - f0) * nck;
    const float *src = DIRECT ? r.A32 : r.Bp32;
    const size_t istride = (size_t)F * T;

    // stage st's slab and data columns into buffer st & 1 (column tid of each row)
    auto prefetch = [&](int st) {
        const int f = f0 + st / nck, t0 = (st % nck) * TCr;
        const int tn = min(TCr, T - t0);
        float *a = As + (size_t)(st & 1) * slab;
        float *d = dcol + (size_t)(st & 1) * 2 * SIMT_TC;
        const size_t ft = (size_t)f * T + t0 + tid;
        if (tid < tn) {
            for (int i = 0; i < N; ++i) cp_async4(a + (size_t)i * TCr + tid, src + (size_t)i * istride + ft);
            cp_async4(d + tid, DIRECT ? r.data32 + ft : r.dref32 + ft);
            if (DIRECT) cp_async4(d + SIMT_TC + tid, r.B32 + ft);
        } else if (tid < TCr) {
            for (int i = 0; i < N; ++i) a[(size_t)i * TCr + tid] = 0.0f;
            d[tid] = 0.0f;
            d[SIMT_TC + tid] = 0.0f;
        }
        cp_async_commit();
    };
    if (S > 0) prefetch(0);

    const double *th = r.params + (inb ? p : 0) * (NP + 4);
    const float a21 = (float)th[NP], nu21 = (float)th[NP + 1];
    const float inv2s2 = (float)(1.0 / (2.0 * th[NP + 2] * th[NP + 2]));
    Wsh[(size_t)N * TILE_M + tid] = 0.0f;
    // this thread's register tiles: points 4 pg .. 4 pg + 3, column blocks cs, cs + 4, ...
    // (a warp holds all 32 point groups of one column slot: broadcast slab loads)
    const int pg = tid % SIMT_PG, cs = tid / SIMT_PG;
    float qs = 0.0f, qc = 0.0f;
    float q4[SIMT_PT];                // masked (partial-block) sums of this thread's tile points
    uint64_t q2[SIMT_PT];             // packed sums: even and odd columns of full blocks
    float qr = 0.0f;                  // point tid's sum over the shared-out blocks
#pragma unroll
    for (int a = 0; a < SIMT_PT; ++a) {
        q4[a] = 0.0f;
        q2[a] = 0ull;
    }
    const uint64_t m1 = pk2f(-1.0f, -1.0f);
    for (int st = 0; st < S; ++st) {
        const int f = f0 + st / nck, ck = st % nck, t0 = ck * TCr;
        const int tn = min(TCr, T - t0);
        if (ck == 0) {
            // the channel's weights and troughs (the previous stage's readers
            // passed the barrier that ended it)
            const float nuf = (float)r.nu[f];
            const float dnu = nuf - nu21;
            s21s[tid] = a21 * expf(-dnu * dnu * inv2s2);
            if (DIRECT) {
                const float l2 = (float)(r.L[f] * 1.4426950408889634);   // log2(nu/nu0)
                for (int i = 0; i < N; ++i) {
                    const float w = exp2f(-__ldg(prow + (i % Nb) * TILE_M) * l2);
                    Wsh[i * TILE_M + tid] = Na ? __ldg(prow + (Nb + i / Nb) * TILE_M) * w : w;
                }
            } else {
                const float nL = (float)(-r.L[f]);
                for (int i = 0; i < N; ++i) {
                    float y = __ldg(prow + (i % Nb) * TILE_M) * nL;
                    if (Na) y += __ldg(prow + (Nb + i / Nb) * TILE_M);
                    Wsh[i * TILE_M + tid] = expm1f(y);
                }
            }
        }
        if (st + 1 < S) {
            prefetch(st + 1);           // buffer (st + 1) & 1 was last read by stage st - 1
            cp_async_wait_group1();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const float *a_st = As + (size_t)(st & 1) * slab;
        const float *d_st = dcol + (size_t)(st & 1) * 2 * SIMT_TC;
        const float tcmb = (float)r.t_cmb;
        const int ncb = (tn + SIMT_CT - 1) / SIMT_CT;
        // blocks taken as 4 x 8 tiles, one per column slot per round; fewer
        // blocks than slots go as whole tiles too (one round, some warps idle),
        // which beats sharing them out point by point there
        const int nfull = ncb - (ncb >= SIMT_CS ? ncb % SIMT_CS : 0);
        for (int cb = cs; cb < nfull; cb += SIMT_CS) {
            // accumulator pairs (columns 2k, 2k+1 of one point): packed FP32x2
            // FMAs, each lane the same round-to-nearest FMA as a scalar one
            uint64_t acc2[SIMT_PT][SIMT_CT / 2];
#pragma unroll
            for (int a = 0; a < SIMT_PT; ++a)
#pragma unroll
                for (int c = 0; c < SIMT_CT / 2; ++c) acc2[a][c] = 0ull;
            const float4 *wp = reinterpret_cast<const float4 *>(Wsh + SIMT_PT * pg);
            const float4 *ap = reinterpret_cast<const float4 *>(a_st + SIMT_CT * cb);
            const int wstep = TILE_M / 4, astep = TCr / 4;      // one region, in float4
            float4 wq[SIMT_PT / 4];
#pragma unroll
            for (int k = 0; k < SIMT_PT / 4; ++k) wq[k] = wp[k];
            float4 a0 = ap[0], a1 = ap[1];
            for (int i = 0; i < N; ++i) {
                // region i + 1's operands (row N is a spare row) while region i's FMAs issue
                wp += wstep;
                ap += astep;
                float4 wn[SIMT_PT / 4];
#pragma unroll
                for (int k = 0; k < SIMT_PT / 4; ++k) wn[k] = wp[k];
                const float4 a0n = ap[0], a1n = ap[1];
                const uint64_t av[SIMT_CT / 2] = {pk2f(a0.x, a0.y), pk2f(a0.z, a0.w), pk2f(a1.x, a1.y),
                                                  pk2f(a1.z, a1.w)};
#pragma unroll
                for (int a = 0; a < SIMT_PT; ++a) {
                    const float4 &q = wq[a / 4];
                    const float wa = (a & 3) == 0 ? q.x : (a & 3) == 1 ? q.y : (a & 3) == 2 ? q.z : q.w;
                    const uint64_t ww = pk2f(wa, wa);
#pragma unroll
                    for (int c = 0; c < SIMT_CT / 2; ++c) acc2[a][c] = fma2f(av[c], ww, acc2[a][c]);
                }
#pragma unroll
                for (int k = 0; k < SIMT_PT / 4; ++k) wq[k] = wn[k];
                a0 = a0n;
                a1 = a1n;
            }
            if (SIMT_CT * cb + SIMT_CT <= tn) {
                // a full block: r = (dv - s21) - acc and r^2 summed in packed FP32x2,
                // the same roundings per column as the scalar form below
                uint64_t dv2[SIMT_CT / 2];
#pragma unroll
                for (int c = 0; c < SIMT_CT / 2; ++c) {
                    const int t = SIMT_CT * cb + 2 * c;
                    dv2[c] = DIRECT ? fma2f(pk2f(-tcmb, -tcmb), pk2f(d_st[SIMT_TC + t], d_st[SIMT_TC + t + 1]),
                                            pk2f(d_st[t], d_st[t + 1]))
                                    : pk2f(d_st[t], d_st[t + 1]);
                }
#pragma unroll
                for (int a = 0; a < SIMT_PT; ++a) {
                    const float sa = s21s[SIMT_PT * pg + a];
                    const uint64_t s2 = pk2f(sa, sa);
#pragma unroll
                    for (int c = 0; c < SIMT_CT / 2; ++c) {
                        const uint64_t rr2 = fma2f(acc2[a][c], m1, fma2f(s2, m1, dv2[c]));
                        q2[a] = fma2f(rr2, rr2, q2[a]);
                    }
                }
            } else {
                float acc[SIMT_PT][SIMT_CT];
#pragma unroll
                for (int a = 0; a < SIMT_PT; ++a)
#pragma unroll
                    for (int c = 0; c < SIMT_CT / 2; ++c) upk2f(acc2[a][c], acc[a][2 * c], acc[a][2 * c + 1]);
#pragma unroll
                for (int c = 0; c < SIMT_CT; ++c) {
                    const int t = SIMT_CT * cb + c;
                    if (t < tn) {
                        const float dv = DIRECT ? d_st[t] - tcmb * d_st[SIMT_TC + t] : d_st[t];
#pragma unroll
                        for (int a = 0; a < SIMT_PT; ++a) {
                            const float rr = (dv - s21s[SIMT_PT * pg + a]) - acc[a][c];
                            q4[a] = fmaf(rr, rr, q4[a]);
                        }
                    }
                }
            }
        }
        // the blocks left over from the rounds: thread tid takes point tid x 8 columns
        for (int cb = nfull; cb < ncb; ++cb) {
            uint64_t acc2[SIMT_CT / 2] = {0ull, 0ull, 0ull, 0ull};
            const float *wp = Wsh + tid;
            const float4 *ap = reinterpret_cast<const float4 *>(a_st + SIMT_CT * cb);
            const int astep = TCr / 4;
            float wa = wp[0];
            float4 a0 = ap[0], a1 = ap[1];
            for (int i = 0; i < N; ++i) {
                wp += TILE_M;
                ap += astep;
                const float wn = wp[0];
                const float4 a0n = ap[0], a1n = ap[1];
                const uint64_t ww = pk2f(wa, wa);
                acc2[0] = fma2f(pk2f(a0.x, a0.y), ww, acc2[0]);
                acc2[1] = fma2f(pk2f(a0.z, a0.w), ww, acc2[1]);
                acc2[2] = fma2f(pk2f(a1.x, a1.y), ww, acc2[2]);
                acc2[3] = fma2f(pk2f(a1.z, a1.w), ww, acc2[3]);
                wa = wn;
                a0 = a0n;
                a1 = a1n;
            }
            float acc[SIMT_CT];
#pragma unroll
            for (int c = 0; c < SIMT_CT / 2; ++c) upk2f(acc2[c], acc[2 * c], acc[2 * c + 1]);
            const float st21 = s21s[tid];
#pragma unroll
            for (int c = 0; c < SIMT_CT; ++c) {
                const int t = SIMT_CT * cb + c;
                if (t < tn) {
                    const float dv = DIRECT ? d_st[t] - tcmb * d_st[SIMT_TC + t] : d_st[t];
                    const float rr = (dv - st21) - acc[c];
                    qr = fmaf(rr, rr, qr);
                }
            }
        }
        if (ck == nck - 1) {
            // the channel is complete: its per-point sums, combined in slot order
#pragma unroll
            for (int a = 0; a < SIMT_PT; ++a) {
                float lo, hi;
                upk2f(q2[a], lo, hi);
                qp[cs * TILE_M + SIMT_PT * pg + a] = (lo + hi) + q4[a];
                q4[a] = 0.0f;
                q2[a] = 0ull;
            }
            qp[SIMT_CS * TILE_M + tid] = qr;
            qr = 0.0f;
            __syncthreads();
            float qf = qp[tid];
#pragma unroll
            for (int k = 1; k <= SIMT_CS; ++k) qf += qp[k * TILE_M + tid];
            kahan_add(qs, qc, qf);
        }
        __syncthreads();                // every read of this stage's buffers is done
    }
    if (inb) r.partials[(size_t)p * r.n_part + g] = make_float2(qs, -qc);
}

// a6: per point, sum the channel-group partials in fixed order and form
// lnL = -1/2 (F T ln(2 pi sigma_n^2) + chi2 / sigma_n^2) (eq. likelihood).  The
// partials (compensated FP32 pairs) are summed in double-float arithmetic
// (Knuth's two-sum on FP32 pairs, about 48 bits) and converted once: FP64 is a
// scarce pipe on this part.
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}
// Each request's rows are summed in a form fixed by the row length alone, so a
// request's logL does not depend on what it is batched with:
//  - rows of at most REDUCE_SERIAL_MAX partials (the usual case): one thread per
//    point sums its row in ascending order (double-float);
//  - longer rows (one channel per group at small P): one warp per point, lane l
//    summing partials l, l+32, ... in ascending order, the lanes' sums combined
//    in a fixed butterfly.
// WARP selects the form a launch serves; requests of the other form are skipped.
// When the launch's status word is set (a bounded wait ran out, so some
// partials were never written), every logL of the launch is NaN.
template <bool WARP>
__global__ void __launch_bounds__(REDUCE_THREADS) reduce_kernel(const ReqDesc *__restrict__ reqs, int n_reqs) {
    pdl_wait();
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gid = WARP ? tid >> 5 : tid;
    const int lane = WARP ? (int)(threadIdx.x & 31) : 0;
    const ReqDesc &r = reqs[find_req_by_point(reqs, n_reqs, gid)];
    const int64_t p = gid - r.pt_begin;
    if (p < 0 || p >= r.P) return;       // uniform over a warp in WARP mode
    if ((r.n_part > REDUCE_SERIAL_MAX) != WARP) return;
    if (*r.status) {         // a kernel of this launch stopped early: its partials are incomplete
        if (lane == 0) r.logL[p] = __longlong_as_double(0x7FF8000000000000ll);
        return;
    }
    if (!r.pvalid[p]) {      // the statistics pass tested the point (point_valid)
        if (lane == 0) {
            r.logL[p] = -INFINITY;
            atomicAdd(r.invalid, 1ull);
        }
        return;
    }
    float sh = 0.0f, sl = 0.0f;
    const float2 *__restrict__ part = r.partials + (size_t)p * r.n_part;
    if (WARP) {
        for (int g = lane; g < r.n_part; g += 32) {
            const float2 v = part[g];
            two_sum_acc(sh, sl, v.x);
            two_sum_acc(sh, sl, v.y);
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
            df_add(sh, sl, oh, ol);
        }
        if (lane != 0) return;
    } else {
#pragma unroll 4
        for (int g = 0; g < r.n_part; ++g) {
            const float2 v = part[g];
            two_sum_acc(sh, sl, v.x);
            two_sum_acc(sh, sl, v.y);
        }
    }
    const double chi2 = ((double)sh + (double)sl) * r.chi2_scale;
    if (r.pnorm) {           // sigma_n terms from prep (tensor path)
        const double2 nm = r.pnorm[p];
        r.logL[p] = -0.5 * (nm.x + chi2 * nm.y);
    } else {
        const double sig = r.params[p * (r.NPF + 4) + r.NPF + 3];
        const double n = (double)r.F * (double)r.T;
        r.logL[p] = -0.5 * (n * log(2.0 * 3.141592653589793 * sig * sig) + chi2 / (sig * sig));
    }
}

// Validation helper: T_model[p,f,t] with the arithmetic of the SIMT forms.
template <bool DIRECT>
__global__ void model_eval_simt_kernel(const ReqDesc *__restrict__ req, double *__restrict__ out) {
    const ReqDesc &r = *req;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = r.P * r.F * r.T;
    if (gid >= total) return;
    const int64_t p = gid / ((int64_t)r.F * r.T);
    const int f = (int)((gid / r.T) % r.F), t = (int)(gid % r.T);
    const int N = r.N, Nb = r.Nb, Na = r.Na, NP = r.NPF;
    const double *th = r.params + p * (NP + 4);
    const size_t ft = (size_t)f * r.T + t;
    const float nuf = (float)r.nu[f], dnu = nuf - (float)th[NP + 1];
    const float s21 = (float)th[NP] * expf(-dnu * dnu * (float)(1.0 / (2.0 * th[NP + 2] * th[NP + 2])));
    if (DIRECT) {
        const float l2 = (float)(r.L[f] * 1.4426950408889634);
        float acc = 0.0f;
        for (int i = 0; i < N; ++i) {
            float w = exp2f(-(float)th[i % Nb] * l2);
            if (Na) w *= (float)th[Nb + i / Nb];
            acc = fmaf(r.A32[(size_t)i * r.F * r.T + ft], w, acc);
        }
        out[gid] = (double)(acc + (float)r.t_cmb * r.B32[ft] + s21);
    } else {
        const float nL = (float)(-r.L[f]);
        float acc = 0.0f;
        for (int i = 0; i < N; ++i) {
            const int j = i % Nb;
            float y = (float)(th[j] - r.beta_bar[j]) * nL;
            if (Na) {
                const double ab = r.beta_bar[Nb + i / Nb];
                y += log1pf((float)(th[Nb + i / Nb] - ab) / (float)ab);
            }
            acc = fmaf(r.Bp32[(size_t)i * r.F * r.T + ft], expm1f(y), acc);
        }
        const float rr = (r.dref32[ft] - s21) - acc;
        out[gid] = r.data[ft] - (double)rr;
    }
}

__global__ void resid_to_model_kernel(const ReqDesc *__restrict__ req, const float *__restrict__ resid,
                                      double *__restrict__ out) {
    const ReqDesc &r = *req;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = r.P * r.F * r.T;
    if (gid >= total) return;
    const size_t ft = (size_t)(gid % ((int64_t)r.F * r.T));
    out[gid] = r.data[ft] - (double)resid[gid];
}

}  // namespace

// Raise a kernel's dynamic shared-memory limit to `need` bytes when a launch
// asks for more than the default 48 KB (or the last limit set); the largest
// size a block may hold is checked by the runtime at the launch.
template <typename K>
cudaError_t opt_in_smem(K kernel, size_t need, size_t &current) {
    if (need <= current) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e == cudaSuccess) current = need;
    return e;
}

cudaError_t launch_prep(const ReqDesc *h_reqs, const ReqDesc *d_reqs, int n_reqs, int precision,
                        int max_stat_blocks, int max_F_chunks, int max_tiles, cudaStream_t stream) {
    int maxNP = 0;
    for (int k = 0; k < n_reqs; ++k) maxNP = maxNP > h_reqs[k].NPF ? maxNP : h_reqs[k].NPF;
    // the finalise keeps one row of statistics per thread group in FIN_GROUP_SCRATCH
    // floats (2 NPF + 2 <= 256 within the documented region limits)
    if (2 * maxNP + 2 > FIN_GROUP_SCRATCH) return cudaErrorInvalidValue;
    dim3 g1(max_stat_blocks, n_reqs);
    // warp partials, then the staged parameter rows when they fit comfortably
    const size_t part = sizeof(double) * (((size_t)(STAT_BLOCK / 32) * (2 * maxNP + 2) + 1) / 2);
    const size_t slab1 = sizeof(double) * (size_t)STAT_BLOCK * padded_row(maxNP + 4);
    const int staged = slab1 <= 96 * 1024;
    const size_t sm1 = part + (staged ? slab1 : 0);
    static size_t stats_opt_in = 48 * 1024;
    cudaError_t e = opt_in_smem(prep_stats_kernel, sm1, stats_opt_in);
    if (e != cudaSuccess) return e;
    prep_stats_kernel<<<g1, STAT_BLOCK, sm1, stream>>>(d_reqs, staged);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const bool tc = precision == FG21_PREC_FP16X3 || precision == FG21_PREC_BF16X3;
    size_t sm = 0;
    for (int k = 0; k < n_reqs; ++k) {
        const ReqDesc &r = h_reqs[k];
        const size_t head = sizeof(double) * (size_t)prep_head_doubles(r.NPF);
        size_t need;
        if (tc) {
            const size_t chan = sizeof(float) * (2 * (size_t)r.N * r.Tc_pad + 3 * (size_t)r.Tc_pad + 2 * (size_t)r.N);
            const size_t pts = sizeof(double) * (size_t)TILE_M * padded_row(r.NPF + 4);
            need = head + (chan > pts ? chan : pts);
        } else {
            need = head + sizeof(double) * (size_t)r.N;
        }
        sm = sm > need ? sm : need;
    }
    dim3 g2(max_F_chunks + max_tiles, n_reqs);
    static size_t tc_opt_in[2] = {48 * 1024, 48 * 1024};
    if (precision == FG21_PREC_FP16X3) e = opt_in_smem(prep_tc_kernel<false>, sm, tc_opt_in[0]);
    if (precision == FG21_PREC_BF16X3) e = opt_in_smem(prep_tc_kernel<true>, sm, tc_opt_in[1]);
    if (e != cudaSuccess) return e;
    switch (precision) {
        case FG21_PREC_FP16X3: e = launch_dependent(prep_tc_kernel<false>, g2, PREP_THREADS, sm, stream, d_reqs); break;
        case FG21_PREC_BF16X3: e = launch_dependent(prep_tc_kernel<true>, g2, PREP_THREADS, sm, stream, d_reqs); break;
        case FG21_PREC_FP32_DELTA:
            e = launch_dependent(prep_tiles_kernel<2>, g2, PREP_THREADS, sm, stream, d_reqs);
            break;
        default: e = launch_dependent(prep_tiles_kernel<3>, g2, PREP_THREADS, sm, stream, d_reqs); break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// The SIMT kernels may use up to the largest dynamic shared memory a block can
// hold; set once per process (the occupancy query and the launches both use
// the limit).
static cudaError_t simt_smem_limit() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(simt_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(simt_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    return err;
}

int simt_chunk_width(int N, int T) {
    // columns staged per round: the widest power of two that fits shared
    // memory, but no wider than T rounded up to a column block (128 columns
    // fit for every N up to 146, beyond the region cap of 126; the narrower
    // widths guard the shared-memory limit should that cap grow)
    const int t8 = (T + SIMT_CT - 1) / SIMT_CT * SIMT_CT;
    for (int tc = SIMT_TC; tc > 32; tc >>= 1)
        if (sizeof(float) * simt_smem_floats(N, std::min(tc, t8)) <= SIMT_SMEM_MAX) return std::min(tc, t8);
    return std::min(32, t8);
}

int simt_blocks_per_sm(int N, int tc, int precision) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const bool direct = precision == FG21_PREC_FP32_DIRECT;
    const auto key = std::make_tuple(dev, N, tc, (int)direct);
    std::lock_guard<std::mutex> lk(mu);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const size_t sm = sizeof(float) * simt_smem_floats(N, tc);
    int n = 0;
    cudaError_t e = simt_smem_limit();
    if (e == cudaSuccess)
        e = direct ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, simt_kernel<true>, SIMT_THREADS, sm)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, simt_kernel<false>, SIMT_THREADS, sm);
    if (e != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    cache[key] = n;
    return n;
}

cudaError_t launch_simt(const ReqDesc *h_reqs, const ReqDesc *d_reqs, int n_reqs, int precision,
                        cudaStream_t stream) {
    int64_t items = 0;
    size_t sm = 0;
    for (int k = 0; k < n_reqs; ++k) {
        const ReqDesc &r = h_reqs[k];
        items += (int64_t)r.n_tiles * r.G;
        const size_t need = sizeof(float) * simt_smem_floats(r.N, r.simt_tc);
        sm = sm > need ? sm : need;
    }
    if (items == 0) return cudaSuccess;
    for (int k = 0; k < n_reqs; ++k)
        if (h_reqs[k].P > 0 && (h_reqs[k].simt_tc < SIMT_CT || h_reqs[k].simt_tc > SIMT_TC ||
                                h_reqs[k].simt_tc % SIMT_CT || h_reqs[k].pts32 == nullptr))
            return cudaErrorInvalidValue;
    if (sm > SIMT_SMEM_MAX) return cudaErrorInvalidValue;
    cudaError_t e = simt_smem_limit();
    if (e != cudaSuccess) return e;
    e = precision == FG21_PREC_FP32_DIRECT
            ? launch_dependent(simt_kernel<true>, dim3((unsigned)items), SIMT_THREADS, sm, stream, d_reqs, n_reqs)
            : launch_dependent(simt_kernel<false>, dim3((unsigned)items), SIMT_THREADS, sm, stream, d_reqs, n_reqs);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_reduce(const ReqDesc *h_reqs, const ReqDesc *d_reqs, int n_reqs, cudaStream_t stream) {
    int64_t pts = 0;
    for (int k = 0; k < n_reqs; ++k) pts += h_reqs[k].P;
    if (pts == 0) return cudaSuccess;
    bool serial = false, warp = false;
    for (int k = 0; k < n_reqs; ++k) {
        if (h_reqs[k].P == 0) continue;
        (h_reqs[k].n_part > REDUCE_SERIAL_MAX ? warp : serial) = true;
    }
    const int th = REDUCE_THREADS;
    cudaError_t e = cudaSuccess;
    if (serial) e = launch_dependent(reduce_kernel<false>, dim3((unsigned)((pts + th - 1) / th)), th, 0, stream, d_reqs,
                                     n_reqs);
    if (e != cudaSuccess) return e;
    const int64_t per_block = th / 32;
    if (warp) {
        const dim3 g((unsigned)((pts + per_block - 1) / per_block));
        if (serial) reduce_kernel<true><<<g, th, 0, stream>>>(d_reqs, n_reqs);   // after the first reduction
        else e = launch_dependent(reduce_kernel<true>, g, th, 0, stream, d_reqs, n_reqs);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_model_eval(const ReqDesc *h_req, const ReqDesc *d_req, int precision, double *d_out,
                              cudaStream_t stream) {
    const int64_t total = h_req->P * h_req->F * h_req->T;
    const int th = 256;
    const unsigned blocks = (unsigned)((total + th - 1) / th);
    if (precision == FG21_PREC_FP32_DIRECT) {
        model_eval_simt_kernel<true><<<blocks, th, 0, stream>>>(d_req, d_out);
        return cudaGetLastError();
    }
    if (precision == FG21_PREC_FP32_DELTA) {
        model_eval_simt_kernel<false><<<blocks, th, 0, stream>>>(d_req, d_out);
        return cudaGetLastError();
    }
    // tensor-core forms: rerun the tensor kernel writing its residuals, then D - r
    float *resid = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&resid, sizeof(float) * total, stream);
    if (e != cudaSuccess) return e;
    e = launch_tc_residuals(h_req, d_req, precision, resid, stream);
    if (e == cudaSuccess) {
        resid_to_model_kernel<<<blocks, th, 0, stream>>>(d_req, resid, d_out);
        e = cudaGetLastError();
    }
    cudaFreeAsync(resid, stream);
    return e;
}

}  // namespace fg21
