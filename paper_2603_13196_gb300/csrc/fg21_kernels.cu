// Per-request preparation, SIMT likelihood kernels and the fixed-order
// reduction of libfg21 (sm_103a).
//
// The likelihood of eq. likelihood (Sec. 2.3.1) over the fast forward model of
// eq. fast_forward_model (Sec. 2.2) is evaluated in a reference-subtracted form:
// with a per-request reference spectral index bbar_i (mean over the request's
// valid points) and wbar_{i,f} = (nu_f/nu0)^-bbar_i,
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

#include "fg21_internal.h"

namespace fg21 {

namespace {

constexpr int PREP_THREADS = 256;
constexpr int REDUCE_THREADS = 64;

// A point is valid when all its parameters are finite, sigma_n > 0 and
// sigma21 != 0.  Tested on the bit patterns (integer instructions; FP64 is a
// scarce pipe on this part).
__device__ __forceinline__ bool point_valid(const double *th, int N) {
    bool ok = true;
    for (int k = 0; k < N + 4; ++k)
        ok &= (__double_as_longlong(th[k]) & 0x7FF0000000000000ll) != 0x7FF0000000000000ll;
    ok &= __double_as_longlong(th[N + 3]) > 0;                                 // > +0 (sign clear)
    ok &= (__double_as_longlong(th[N + 2]) & 0x7FFFFFFFFFFFFFFFll) != 0;      // != +-0
    return ok;
}

// Deterministic block reductions (fixed shuffle tree, then warps in order).
template <typename Op>
__device__ double block_reduce(double v, Op op, double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = sh[0];
    for (int w = 1; w < nw; ++w) r = op(r, sh[w]);
    __syncthreads();
    return r;
}

struct OpSum { __device__ double operator()(double a, double b) const { return a + b; } };
struct OpMin { __device__ double operator()(double a, double b) const { return fmin(a, b); } };
struct OpMax { __device__ double operator()(double a, double b) const { return fmax(a, b); } };

// a1, pass 1: per block of STAT_BLOCK points (one thread each), the sum / min
// / max of each region's beta over valid points (FP32: the reference point
// only has to be a deterministic value near the points; the rearranged
// likelihood is exact for any reference), the valid count and max |A21|.
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

// a1, pass 2, run by every block of the second prep kernel: the reference
// point bbar_i = mean of the valid points' beta_i, the largest weight argument
// x = max_i |beta - bbar_i| * max_f |L_f| (which sets the weight series and the
// power-of-two scale sW of the weight operand), the valid count and max |A21|.
// Thread j combines field j of every stat block in block order (one round of
// independent loads per 16 blocks), so every block computes the same values
// bit for bit; bbar goes to shared memory (`bbar_sh`), and block 0 of the
// request publishes the results for the later kernels.
struct Fin {
    float nv, ma, x;
    int sW;
};
__device__ Fin prep_finalize(const ReqDesc &r, float *sh /* [3N + 2 + nwarps] */, double *bbar_sh, bool publish) {
    const int N = r.N, nb = r.n_stat_blocks, W = 3 * N + 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        const int kind = j < 3 * N ? j % 3 : (j == 3 * N ? 0 : 2);   // 0 sum, 1 min, 2 max
        const float *q = r.stat_part + j;
        float v = kind == 0 ? 0.0f : kind == 1 ? INFINITY : -INFINITY;
        // 16 independent loads in flight per round, combined in block order
        for (int b0 = 0; b0 < nb; b0 += 16) {
            float x[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) x[u] = b0 + u < nb ? __ldg(q + (size_t)(b0 + u) * W) : 0.0f;
#pragma unroll
            for (int u = 0; u < 16; ++u)
                if (b0 + u < nb) v = kind == 0 ? v + x[u] : kind == 1 ? fminf(v, x[u]) : fmaxf(v, x[u]);
        }
        sh[j] = v;
    }
    __syncthreads();
    const float nv = sh[3 * N], ma = sh[3 * N + 1];
    float dev = 0.0f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float bb = nv > 0.0f ? sh[3 * i] / nv : 0.0f;
        bbar_sh[i] = (double)bb;
        if (publish) r.beta_bar[i] = (double)bb;
        if (nv > 0.0f) dev = fmaxf(dev, fmaxf(sh[3 * i + 2] - bb, bb - sh[3 * i + 1]));
    }
    for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    float *wred = sh + W;
    if (lane == 0) wred[warp] = dev;
    __syncthreads();
    float dmax = 0.0f;
    for (int w = 0; w < nw; ++w) dmax = fmaxf(dmax, wred[w]);
    Fin f;
    // a small margin on x covers the FP32 statistics
    f.x = dmax * (float)r.Lmax * 1.0001f;
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

__global__ void __launch_bounds__(STAT_BLOCK) prep_stats_kernel(const ReqDesc *__restrict__ reqs) {
    extern __shared__ float sh_stats[];        // [STAT_BLOCK / 32][3N + 2]
    const ReqDesc &r = reqs[blockIdx.y];
    if ((int)blockIdx.x >= r.n_stat_blocks) return;
    const int N = r.N, W = 3 * N + 2, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * STAT_BLOCK + threadIdx.x;
    const double *th = r.params + (p < r.P ? p : 0) * (N + 4);
    const bool valid = p < r.P && point_valid(th, N);
    float *mine = sh_stats + warp * W;
    for (int i = 0; i < N; ++i) {
        const float b = valid ? (float)th[i] : 0.0f;
        float s = b, mn = valid ? b : INFINITY, mx = valid ? b : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            mine[3 * i] = s;
            mine[3 * i + 1] = mn;
            mine[3 * i + 2] = mx;
        }
    }
    float nv = valid ? 1.0f : 0.0f, ma = valid ? fabsf((float)th[N]) : 0.0f;
    for (int o = 16; o > 0; o >>= 1) {
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
        ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    }
    if (lane == 0) {
        mine[3 * N] = nv;
        mine[3 * N + 1] = ma;
    }
    __syncthreads();
    float *out = r.stat_part + (size_t)blockIdx.x * W;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        const int kind = j < 3 * N ? j % 3 : (j == 3 * N ? 0 : 2);   // 0 sum, 1 min, 2 max
        float v = sh_stats[j];
        for (int w = 1; w < nw; ++w) {
            const float x = sh_stats[w * W + j];
            v = kind == 0 ? v + x : kind == 1 ? fminf(v, x) : fmaxf(v, x);
        }
        out[j] = v;
    }
}

// a1, pass 3: one block per (channel, t-chunk) builds that channel's
// reference: wbar_i = (nu_f/nu0)^-bbar_i, wbar_i A[i,f,t] and
// dref = D - sum_i wbar_i A_i - T_CMB B (FP64), then writes either the FP32
// arrays of the SIMT delta form or the split-precision operand tile of the
// tensor-core form.
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
// thread per point reads them coalesced: rows k < Kp-2 hold beta_{p,k} - bbar_k
// in FP32 (zero for k >= N), then A21, nu21 and 1/(2 sigma21^2).
template <int MODE>
__device__ __forceinline__ void prep_points(const ReqDesc &r, int tile, const double *bbar) {
    const int64_t p = (int64_t)tile * TILE_M + threadIdx.x;
    if (threadIdx.x >= TILE_M) return;
    const int N = r.N, R = r.Kp + 4;
    float *out = r.pts32 + (size_t)tile * R * TILE_M + threadIdx.x;
    const bool in = p < r.P;
    const double *th = r.params + (in ? p : 0) * (N + 4);
    for (int k = 0; k < r.Kp - 2; ++k)
        out[(size_t)k * TILE_M] = (in && k < N) ? (float)(th[k] - bbar[k]) : 0.0f;
    out[(size_t)(r.Kp - 2) * TILE_M] = in ? (float)th[N] : 0.0f;
    out[(size_t)(r.Kp - 1) * TILE_M] = in ? (float)th[N + 1] : 0.0f;
    const float s21 = in ? (float)th[N + 2] : 1.0f;
    out[(size_t)r.Kp * TILE_M] = 1.0f / (2.0f * s21 * s21);
}

template <int MODE>  // 0 = tensor FP16, 1 = tensor BF16, 2 = SIMT delta, 3 = SIMT direct
__global__ void __launch_bounds__(PREP_THREADS) prep_tiles_kernel(const ReqDesc *__restrict__ reqs) {
    extern __shared__ double smem_d[];
    __shared__ double sh[32];
    __shared__ int s_scaleB;
    const ReqDesc &r = reqs[blockIdx.y];
    const int nfc = r.F * r.n_tchunks;
    const int N = r.N, T = r.T;
    if ((int)blockIdx.x >= nfc + (MODE <= 1 ? r.n_tiles : 0)) return;
    // shared memory: bbar [N] FP64, finalise scratch [3N + 2 + 8] FP32 (rounded to
    // doubles), wbar [N] FP64, dref [Tc_pad] FP64, wbar32 [N] FP32
    double *bbar = smem_d;
    float *fin_sh = reinterpret_cast<float *>(bbar + N);
    double *wbar = bbar + N + (3 * N + 2 + 8 + 1) / 2;
    double *dref = wbar + N;
    float *wbar32 = reinterpret_cast<float *>(dref + r.Tc_pad);
    prep_finalize(r, fin_sh, bbar, blockIdx.x == 0);
    if (MODE <= 1 && (int)blockIdx.x >= nfc) {
        prep_points<MODE>(r, blockIdx.x - nfc, bbar);
        return;
    }
    const int fc = blockIdx.x;
    const int f = fc / r.n_tchunks, c = fc % r.n_tchunks;
    const int t0 = c * r.Tc, tn = min(r.Tc, T - t0);
    const double L = r.L[f];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        wbar[i] = exp(-bbar[i] * L);
        wbar32[i] = (float)wbar[i];
    }
    if (c == 0 && threadIdx.x == 0) {
        r.nL32[f] = (float)(-L);
        r.nu32[f] = (float)r.nu[f];
    }
    __syncthreads();
    // --- reference residual dref[t] = D - sum_i wbar_i A_i - T_CMB B (FP64: the
    // foreground cancels here) ---
    float vmax = 1.0f;
    const size_t istride = (size_t)r.F * T;
    for (int t = threadIdx.x; t < tn; t += blockDim.x) {
        const size_t ft = (size_t)f * T + t0 + t;
        double s = 0.0;
        for (int i0 = 0; i0 < N; i0 += 8) {
            double a[8];
            float a32[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                a[j] = i0 + j < N ? r.A[(size_t)(i0 + j) * istride + ft] : 0.0;
                a32[j] = i0 + j < N ? r.A32[(size_t)(i0 + j) * istride + ft] : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (i0 + j < N) {
                    const double bw = wbar[i0 + j] * a[j];
                    s += bw;
                    // the scale only needs the magnitude: FP32 product (FP64 is a scarce pipe)
                    vmax = fmaxf(vmax, fabsf(wbar32[i0 + j] * a32[j]));
                    if (MODE == 2) r.Bp32[(size_t)(i0 + j) * istride + ft] = (float)bw;
                }
            }
        }
        const double d = r.data[ft] - s - r.t_cmb * r.B[ft];
        dref[t] = d;
        vmax = fmaxf(vmax, fabsf((float)d));
        if (MODE == 2) r.dref32[ft] = (float)d;
    }
    if (MODE >= 2) return;
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = vmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = sh[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, (float)sh[w]);
        s_scaleB = pow2_exponent_for(v);
        r.scaleB[fc] = s_scaleB;
    }
    __syncthreads();
    const float sB = ldexpf(1.0f, s_scaleB);
    // --- operand tile: one 16-byte chunk (8 values of k) per (split, kc, t).
    // Region rows in FP32 (wbar_k A[k,f,t] to 24 bits, finer than the 22-bit
    // split), the dref row from its FP64 value. ---
    const int Kp = r.Kp, Tcp = r.Tc_pad, nkc = Kp / 8;
    uint4 *tile = reinterpret_cast<uint4 *>(r.tiles + (size_t)fc * r.tile_rows * 128);
    for (int j = threadIdx.x; j < nkc * Tcp; j += blockDim.x) {
        const int kc = j / Tcp, t = j % Tcp;
        float v[8];
        for (int e = 0; e < 8; ++e) {
            const int k = kc * 8 + e;
            float x = 0.0f;
            if (t < tn) {
                if (k < N) x = wbar32[k] * r.A32[(size_t)k * r.F * T + (size_t)f * T + t0 + t] * sB;
                else if (k == Kp - 2) x = sB;
                else if (k == Kp - 1) x = (float)(dref[t] * (double)sB);
            }
            v[e] = x;
        }
        uint32_t H[4], M[4];
        for (int e = 0; e < 8; e += 2) {
            H[e / 2] = pack_pair<MODE == 1>(v[e], v[e + 1]);
            const float2 h = unpack_pair<MODE == 1>(H[e / 2]);
            M[e / 2] = pack_pair<MODE == 1>(v[e] - h.x, v[e + 1] - h.y);
        }
        tile[(size_t)kc * Tcp + t] = make_uint4(H[0], H[1], H[2], H[3]);                 // split 0 (hi)
        tile[(size_t)(nkc + kc) * Tcp + t] = make_uint4(M[0], M[1], M[2], M[3]);         // split 1 (mid)
    }
}

// ------------------------------------------------------------- SIMT paths
// One block = 128 points of one request x one channel group.  Each thread owns
// a point: its weights for the channel go to a private shared-memory column,
// the channel's model slice is staged in shared memory (broadcast reads), and
// the residual of each (f, t) is squared and summed in FP32 per channel, the
// channels folded into a compensated (hi, lo) FP32 pair.
constexpr int SIMT_THREADS = 128;
constexpr int SIMT_TCH = 64;

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

template <int TCH, bool DIRECT>
__device__ __forceinline__ float simt_chunk(const float *__restrict__ As, const float *__restrict__ ds,
                                            const float *__restrict__ wcol, int N, int nvalid, float s21) {
    float acc[TCH];
#pragma unroll
    for (int j = 0; j < TCH; ++j) acc[j] = 0.0f;
    for (int i = 0; i < N; ++i) {
        const float w = wcol[i * SIMT_THREADS];
        const float4 *a4 = reinterpret_cast<const float4 *>(As + i * SIMT_TCH);
#pragma unroll
        for (int j = 0; j < TCH / 4; ++j) {
            float4 a = a4[j];
            acc[4 * j] = fmaf(a.x, w, acc[4 * j]);
            acc[4 * j + 1] = fmaf(a.y, w, acc[4 * j + 1]);
            acc[4 * j + 2] = fmaf(a.z, w, acc[4 * j + 2]);
            acc[4 * j + 3] = fmaf(a.w, w, acc[4 * j + 3]);
        }
    }
    float q = 0.0f;
#pragma unroll
    for (int j = 0; j < TCH; ++j) {
        if (j < nvalid) {
            float rr = (ds[j] - s21) - acc[j];
            q = fmaf(rr, rr, q);
        }
    }
    return q;
}

template <bool DIRECT>
__global__ void __launch_bounds__(SIMT_THREADS) simt_kernel(const ReqDesc *__restrict__ reqs, int n_reqs) {
    extern __shared__ float smem_f[];
    const int64_t item = blockIdx.x;
    const ReqDesc &r = reqs[find_req_by_item(reqs, n_reqs, item)];
    const int64_t lid = item - r.item_begin;
    const int tile = (int)(lid / r.G), g = (int)(lid % r.G);
    const int N = r.N, F = r.F, T = r.T;
    const int f0 = g * r.ch_per_group, f1 = min(F, f0 + r.ch_per_group);
    float *wcol_all = smem_f;                          // [N][128]
    float *As = smem_f + N * SIMT_THREADS;             // [N][64]
    float *ds = As + N * SIMT_TCH;                     // [64]
    const int64_t p = (int64_t)tile * TILE_M + threadIdx.x;
    const bool inb = p < r.P;
    const double *th = r.params + (inb ? p : 0) * (N + 4);
    const float a21 = (float)th[N], nu21 = (float)th[N + 1];
    const float inv2s2 = (float)(1.0 / (2.0 * th[N + 2] * th[N + 2]));
    float qs = 0.0f, qc = 0.0f;
    float *wcol = wcol_all + threadIdx.x;
    for (int f = f0; f < f1; ++f) {
        const float nuf = (float)r.nu[f];
        const float dnu = nuf - nu21;
        const float s21 = a21 * expf(-dnu * dnu * inv2s2);
        if (DIRECT) {
            const float l2 = (float)(r.L[f] * 1.4426950408889634);   // log2(nu/nu0)
            for (int i = 0; i < N; ++i) wcol[i * SIMT_THREADS] = exp2f(-(float)th[i] * l2);
        } else {
            const float nL = (float)(-r.L[f]);
            for (int i = 0; i < N; ++i)
                wcol[i * SIMT_THREADS] = expm1f((float)(th[i] - r.beta_bar[i]) * nL);
        }
        float qf = 0.0f;
        for (int tb = 0; tb < T; tb += SIMT_TCH) {
            const int nvalid = min(SIMT_TCH, T - tb);
            __syncthreads();
            for (int k = threadIdx.x; k < N * SIMT_TCH; k += SIMT_THREADS) {
                const int i = k / SIMT_TCH, j = k % SIMT_TCH;
                float v = 0.0f;
                if (j < nvalid) {
                    const size_t idx = ((size_t)i * F + f) * T + tb + j;
                    v = DIRECT ? r.A32[idx] : r.Bp32[idx];
                }
                As[k] = v;
            }
            for (int j = threadIdx.x; j < SIMT_TCH; j += SIMT_THREADS) {
                float v = 0.0f;
                if (j < nvalid) {
                    const size_t ft = (size_t)f * T + tb + j;
                    v = DIRECT ? r.data32[ft] - (float)r.t_cmb * r.B32[ft] : r.dref32[ft];
                }
                ds[j] = v;
            }
            __syncthreads();
            if (nvalid > 32)
                qf += simt_chunk<64, DIRECT>(As, ds, wcol, N, nvalid, s21);
            else if (nvalid > 16)
                qf += simt_chunk<32, DIRECT>(As, ds, wcol, N, nvalid, s21);
            else
                qf += simt_chunk<16, DIRECT>(As, ds, wcol, N, nvalid, s21);
        }
        kahan_add(qs, qc, qf);
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
__global__ void __launch_bounds__(REDUCE_THREADS) reduce_kernel(const ReqDesc *__restrict__ reqs, int n_reqs) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const ReqDesc &r = reqs[find_req_by_point(reqs, n_reqs, gid)];
    const int64_t p = gid - r.pt_begin;
    if (p < 0 || p >= r.P) return;
    const int N = r.N;
    const double *th = r.params + p * (N + 4);
    if (!point_valid(th, N)) {
        r.logL[p] = -INFINITY;
        atomicAdd(r.invalid, 1ull);
        return;
    }
    float sh = 0.0f, sl = 0.0f;
    const float2 *__restrict__ part = r.partials + (size_t)p * r.n_part;
    for (int g = 0; g < r.n_part; ++g) {
        const float2 v = part[g];
        two_sum_acc(sh, sl, v.x);
        two_sum_acc(sh, sl, v.y);
    }
    const double chi2 = (double)sh + (double)sl;
    const double sig = th[N + 3];
    const double n = (double)r.F * (double)r.T;
    r.logL[p] = -0.5 * (n * log(2.0 * 3.141592653589793 * sig * sig) + chi2 / (sig * sig));
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
    const int N = r.N;
    const double *th = r.params + p * (N + 4);
    const size_t ft = (size_t)f * r.T + t;
    const float nuf = (float)r.nu[f], dnu = nuf - (float)th[N + 1];
    const float s21 = (float)th[N] * expf(-dnu * dnu * (float)(1.0 / (2.0 * th[N + 2] * th[N + 2])));
    if (DIRECT) {
        const float l2 = (float)(r.L[f] * 1.4426950408889634);
        float acc = 0.0f;
        for (int i = 0; i < N; ++i) acc = fmaf(r.A32[(size_t)i * r.F * r.T + ft], exp2f(-(float)th[i] * l2), acc);
        out[gid] = (double)(acc + (float)r.t_cmb * r.B32[ft] + s21);
    } else {
        const float nL = (float)(-r.L[f]);
        float acc = 0.0f;
        for (int i = 0; i < N; ++i)
            acc = fmaf(r.Bp32[(size_t)i * r.F * r.T + ft], expm1f((float)(th[i] - r.beta_bar[i]) * nL), acc);
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

cudaError_t launch_prep(const ReqDesc *h_reqs, const ReqDesc *d_reqs, int n_reqs, int precision,
                        int max_stat_blocks, int max_F_chunks, int max_tiles, cudaStream_t stream) {
    int maxN0 = 0;
    for (int k = 0; k < n_reqs; ++k) maxN0 = maxN0 > h_reqs[k].N ? maxN0 : h_reqs[k].N;
    dim3 g1(max_stat_blocks, n_reqs);
    const size_t sm1 = sizeof(float) * (STAT_BLOCK / 32) * (3 * (size_t)maxN0 + 2);
    prep_stats_kernel<<<g1, STAT_BLOCK, sm1, stream>>>(d_reqs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int maxN = 0, maxTcp = 0;
    for (int k = 0; k < n_reqs; ++k) {
        maxN = maxN > h_reqs[k].N ? maxN : h_reqs[k].N;
        maxTcp = maxTcp > h_reqs[k].Tc_pad ? maxTcp : h_reqs[k].Tc_pad;
    }
    const size_t sm = sizeof(double) * (2 * (size_t)maxN + (3 * (size_t)maxN + 2 + 8 + 1) / 2 + maxTcp) +
                      sizeof(float) * (size_t)maxN;
    const bool tc = precision == FG21_PREC_FP16X3 || precision == FG21_PREC_BF16X3;
    dim3 g2(max_F_chunks + (tc ? max_tiles : 0), n_reqs);
    switch (precision) {
        case FG21_PREC_FP16X3: prep_tiles_kernel<0><<<g2, PREP_THREADS, sm, stream>>>(d_reqs); break;
        case FG21_PREC_BF16X3: prep_tiles_kernel<1><<<g2, PREP_THREADS, sm, stream>>>(d_reqs); break;
        case FG21_PREC_FP32_DELTA: prep_tiles_kernel<2><<<g2, PREP_THREADS, sm, stream>>>(d_reqs); break;
        default: prep_tiles_kernel<3><<<g2, PREP_THREADS, sm, stream>>>(d_reqs); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_simt(const ReqDesc *h_reqs, const ReqDesc *d_reqs, int n_reqs, int precision,
                        cudaStream_t stream) {
    int64_t items = 0;
    int maxN = 0;
    for (int k = 0; k < n_reqs; ++k) {
        items += (int64_t)h_reqs[k].n_tiles * h_reqs[k].G;
        maxN = maxN > h_reqs[k].N ? maxN : h_reqs[k].N;
    }
    if (items == 0) return cudaSuccess;
    const size_t sm = sizeof(float) * ((size_t)maxN * (SIMT_THREADS + SIMT_TCH) + SIMT_TCH);
    static bool attr_done[2] = {false, false};
    const bool direct = precision == FG21_PREC_FP32_DIRECT;
    if (!attr_done[direct]) {
        cudaError_t e = direct ? cudaFuncSetAttribute(simt_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)
                               : cudaFuncSetAttribute(simt_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_done[direct] = true;
    }
    if (direct)
        simt_kernel<true><<<(unsigned)items, SIMT_THREADS, sm, stream>>>(d_reqs, n_reqs);
    else
        simt_kernel<false><<<(unsigned)items, SIMT_THREADS, sm, stream>>>(d_reqs, n_reqs);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const ReqDesc *h_reqs, const ReqDesc *d_reqs, int n_reqs, cudaStream_t stream) {
    int64_t pts = 0;
    for (int k = 0; k < n_reqs; ++k) pts += h_reqs[k].P;
    if (pts == 0) return cudaSuccess;
    const int th = REDUCE_THREADS;
    reduce_kernel<<<(unsigned)((pts + th - 1) / th), th, 0, stream>>>(d_reqs, n_reqs);
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
