// Tensor-core (tcgen05) likelihood kernel of libfg21 for sm_103a.
//
// Per channel f the reference-subtracted residual of every point is one small
// GEMM (Sec. 2.2 eq. fast_forward_model, rearranged about a per-request
// reference; see fg21_kernels.cu):
//
//   acc[p, t] = sum_k W[p, k] Bop[k, t],  k = 0..N+1
//     W[p, i]   = 2^sW expm1(-(beta_{p,i} - bbar_i) L_f)   (i < N)
//     W[p, N]   = 2^sW T21(nu_f; theta_p)                    (eq. t21model)
//     W[p, N+1] = -2^sW
//     Bop[i, t] = 2^sB wbar_{i,f} A[i,f,t],  Bop[N, t] = 2^sB,  Bop[N+1, t] = 2^sB dref[f,t]
//   so acc = -2^(sW+sB) (D - M)  and  chi2_p += sum_t acc^2 2^-2(sW+sB)   (eq. likelihood)
//
// The product runs as split precision on the tensor cores: both operands are
// split into hi + mid 16-bit values (FP16 or BF16) and three MMAs
// (hi*hi + hi*mid + mid*hi) accumulate in FP32 in tensor memory.
//
// One persistent CTA per SM walks a static list of work items (request, tile
// of 128 points, group of channels); a stage is one channel (one t-chunk) of
// the tile.  Warp roles (18 warps):
//   warps 0-7    weight generators: warp w serves the points of tensor-memory
//                lane quadrant w%4 and half w/4 of the weight columns; each
//                thread evaluates its point's weights for the channel in
//                registers, splits them into hi + mid and writes them straight
//                into tensor memory (tcgen05.st), where the MMA reads its A
//                operand;
//   warps 8-15   epilogue: tcgen05.ld of the accumulator rows of quadrant w%4,
//                half (w-8)/4 of the t-columns; square-and-sum over t, unscale,
//                compensated sum over channels, one partial chi2 per (point,
//                item, half);
//   warp 16      TMA producer: cp.async.bulk.tensor loads of the channel's
//                operand tile Bop (prepared per request in global memory);
//   warp 17      MMA issuer (one elected thread) and tensor-memory owner.
// Shared memory carries only the operand tiles (the B side), so the tensor
// cores' shared-memory reads are one operand per MMA.  RING (2-4) stage slots
// each hold an operand tile in shared memory and an accumulator plus a weight
// block in tensor memory.  Each slot has two mbarriers: `full` completes when
// the 8 generator warps have stored the weights, the TMA bytes have landed and
// the 8 epilogue warps have released the slot's accumulator (17 arrivals +
// transaction bytes); `done` receives the single tcgen05.commit of the stage's
// MMAs and tells the producers the slot is free and the epilogue the
// accumulator is ready.
// Every wait is bounded (a few seconds of %globaltimer); on expiry the kernel
// sets a status bit, the roles stop, in-flight MMAs are drained with bounded
// waits and tensor memory is released before the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "fg21_internal.h"
#include "fg21_pdl.cuh"

namespace fg21 {

namespace {

constexpr int NUM_THREADS = 576;
constexpr int MAX_RING = 4;       // stage slots (the launch picks 2-4 by tensor-memory room)
constexpr int FULL_ARRIVALS = 17; // 8 generator warps + 1 TMA producer + 8 epilogue warps
constexpr int WARP_TMA = 16, WARP_MMA = 17;
constexpr int EPI_NB = 4;         // accumulator blocks an epilogue warp loads per wait
// TMA boxes are 64 x box_rows 16-bit values (128-byte rows); box_rows divides
// every request's tile height (a multiple of 8, at most 256)
constexpr uint64_t WAIT_LIMIT_NS = 4000000000ull;
// suspend-time hint of try_wait: a waiting thread sleeps (up to this long, or
// until the phase completes) instead of re-polling, leaving issue slots to the
// warps that compute
constexpr uint32_t TRY_WAIT_HINT_NS = 10000000u;

struct __align__(8) Barriers {
    uint64_t full[MAX_RING];
    uint64_t done[MAX_RING];
    uint64_t drain;
    uint32_t tmem_base;
    volatile uint32_t abort_flag;
};

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// One arrival for the whole (converged) warp, made by an elected lane under a
// predicate rather than a branch.
__device__ __forceinline__ void mbar_arrive_warp(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "@p mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(TRY_WAIT_HINT_NS)
        : "memory");
    return ok != 0;
}
// Non-blocking test of a phase.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: true when the phase completed; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, Barriers *S, unsigned *status,
                                          unsigned code, uint64_t limit_ns = WAIT_LIMIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (S->abort_flag) return false;
        if (globaltimer() - t0 > limit_ns) {
            atomicOr(status, code);
            S->abort_flag = 1;
            return false;
        }
    }
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of 8 rows
// x 16 bytes; lbo = byte distance between the two 8-element K chunks of an MMA
// step, sbo = byte distance between consecutive 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of tcgen05
    return d;                 // base offset 0, relative LBO, swizzle none
}
// Instruction descriptor of kind::f16: D = F32, A = B = F16 (0) or BF16 (1),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t instr_desc(int M, int N, bool bf16) {
    const uint32_t fmt = bf16 ? 1u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D (+)= A B with A in tensor memory (128 lanes = rows, K packed two 16-bit
// values per 32-bit column) and B in shared memory.
__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                           uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// This thread's lane, N consecutive 32-bit columns from taddr.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 2^e for integer e in the normal range (exact; the scale exponents here are
// clamped to +-40 each, so their sums stay within +-80).
__device__ __forceinline__ float exp2i(int e) {
    return __int_as_float((min(max(e, -126), 127) + 127) << 23);
}
__device__ __forceinline__ void kahan_add_dev(float &s, float &c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// ---------------------------------------------------------- work items
struct Item {
    int req, tile, g, f0, f1;
};
__device__ __forceinline__ int find_req(const ReqDesc *__restrict__ reqs, int n, int64_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (reqs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ Item decode_item(const ReqDesc *__restrict__ reqs, int n, int64_t item) {
    Item it;
    it.req = find_req(reqs, n, item);
    const ReqDesc &r = reqs[it.req];
    const int64_t lid = item - r.item_begin;
    it.tile = (int)(lid / r.G);
    it.g = (int)(lid % r.G);
    it.f0 = it.g * r.ch_per_group;
    it.f1 = min(r.F, it.f0 + r.ch_per_group);
    return it;
}

// ----------------------------------------------------- weight generation
// Packed FP32 pairs (fma/mul/sub .f32x2): one instruction for two lanes' worth
// of the Horner chains and splits.
__device__ __forceinline__ uint64_t pk2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// expm1 by its Taylor series on y = x / 2^s (|y| <= 0.55) and s squarings
// (1 + e)^2 - 1 = e (e + 2):  with y = d * nL / 2^s,
//   expm1(y) = sum_{j=1..D} e_j d^j,   e_j = (nL / 2^s)^j / j!,
// evaluated by Horner's rule in d (the per-point deviation) with the channel's
// coefficients e_j (2^sW folded into them when s = 0), on two arguments at
// once.  Relative truncation error |y|^D / (D+1)!: D = 3 for |y| <= 0.01,
// 5 for |y| <= 0.1, 8 for |y| <= 0.55; each squaring adds about two roundings.
// LO: the deviation is d + dlo (dlo2, its part below FP32); the last Horner
// step adds e_1 dlo, the first-order effect of dlo (its next term is about
// |y| times smaller and below FP32 resolution).
template <int D, int CH, bool LO>
__device__ __forceinline__ void em1_series2(uint64_t (&w)[CH], const uint64_t *d2, const uint64_t *e2,
                                            const uint64_t *dlo2) {
#pragma unroll
    for (int i = 0; i < CH; ++i) w[i] = fma2(e2[D], d2[i], e2[D - 1]);
#pragma unroll
    for (int j = D - 2; j >= 1; --j)
#pragma unroll
        for (int i = 0; i < CH; ++i) w[i] = fma2(w[i], d2[i], e2[j]);
#pragma unroll
    for (int i = 0; i < CH; ++i) w[i] = LO ? fma2(w[i], d2[i], mul2(e2[1], dlo2[i])) : mul2(w[i], d2[i]);
}

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}
template <bool BF16>
__device__ __forceinline__ float2 unpack2(uint32_t u) {
    if (BF16) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
        return __bfloat1622float2(h);
    } else {
        __half2 h = *reinterpret_cast<__half2 *>(&u);
        return __half22float2(h);
    }
}
// split a pair into hi (rounded) and mid (rounded remainder)
template <bool BF16>
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &mid) {
    hi = pack2<BF16>(a, b);
    const float2 h = unpack2<BF16>(hi);
    float ra, rb;
    upk2(sub2(pk2(a, b), pk2(h.x, h.y)), ra, rb);
    mid = pack2<BF16>(ra, rb);
}

// One channel's weights of this thread's point for its half of the request's
// Kr columns (nph = Kr/4 pairs, at most NPHMAX; FULL: nph = NPHMAX), written
// to tensor memory: hi at columns t_hi.., mid at t_mid.. (one 32-bit column
// per pair: the lower K index in the low half).  Pair i holds deviations d2[i]
// (zero beyond N -> zero weight); on the last half the final pair is
// (trough, -1) instead (columns Kr-2, Kr-1).  A chunk whose pairs all lie
// beyond N (pair index >= nz) is stored as zeros without evaluation.  The
// Horner chains of a chunk of CH pairs advance together.
// ALPHA (amplitude regions): the series runs on y = d nL + g with g =
// ln(alpha / abar) of each component (pairs at gp[i * 128]) and the channel's
// nL in nL2; e2 then holds the constant coefficients 2^(-s j) / j!.  DF: the
// series degree fixed at compile time (3, 5 or 8; 0 = the request's sp.D at
// run time); the lean kernel dispatches on it once per work item.
template <int NPHMAX, bool BF16, bool FULL, bool ALPHA, int DF = 0>
__device__ __forceinline__ void gen_half(uint32_t t_hi, uint32_t t_mid, const uint64_t *d2,
                                         const float2 *__restrict__ lop, const uint64_t *e2, SeriesPlan sp,
                                         uint64_t sW2, int nph_rt, int nz, bool last, float s21, float sW,
                                         const float2 *__restrict__ gp, uint64_t nL2) {
    constexpr int CH = 4;
    const int nph = FULL ? NPHMAX : nph_rt;
#pragma unroll
    for (int c0 = 0; c0 < NPHMAX; c0 += CH) {
        if (!FULL && c0 >= nph) break;
        uint64_t w[CH];
        if (c0 < nz) {
            const uint64_t *x2 = d2 + c0;
            uint64_t y2[CH];
            if (ALPHA) {
                // nph is a multiple of CH, so every pair of a chunk below nz is below nph
#pragma unroll
                for (int i = 0; i < CH; ++i) {
                    const float2 g = __ldg(gp + (size_t)(c0 + i) * 128);
                    y2[i] = fma2(d2[c0 + i], nL2, pk2(g.x, g.y));
                }
                x2 = y2;
            }
            if (DF == 3 || (DF == 0 && sp.D == 3)) {
                // short series (a batch spread below ~0.007 in beta, as near a
                // posterior): the deviations' low parts enter the weights
                uint64_t l2[CH];
#pragma unroll
                for (int i = 0; i < CH; ++i) {
                    const float2 v = ALPHA ? make_float2(0.0f, 0.0f) : __ldg(lop + (size_t)(c0 + i) * 128);
                    l2[i] = pk2(v.x, v.y);
                }
                em1_series2<3, CH, !ALPHA>(w, x2, e2, l2);
            } else if (DF == 5 || (DF == 0 && sp.D == 5)) {
                em1_series2<5, CH, false>(w, x2, e2, nullptr);
            } else {
                em1_series2<8, CH, false>(w, x2, e2, nullptr);
            }
            if (DF != 3 && DF != 5 && sp.s > 0) {
                const uint64_t two2 = pk2(2.0f, 2.0f);
                for (int q = 0; q < sp.s; ++q)
#pragma unroll
                    for (int i = 0; i < CH; ++i) w[i] = mul2(w[i], add2(w[i], two2));
#pragma unroll
                for (int i = 0; i < CH; ++i) w[i] = mul2(w[i], sW2);
            }
        } else {
#pragma unroll
            for (int i = 0; i < CH; ++i) w[i] = 0;
        }
        uint32_t H[CH], M[CH];
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            float a, b;
            upk2(w[i], a, b);
            const bool tr = FULL ? (c0 + i == NPHMAX - 1) : (c0 + i == nph - 1);
            if (last && tr) {
                a = s21;
                b = -sW;
            }
            split2<BF16>(a, b, H[i], M[i]);
        }
        tmem_st4(t_hi + c0, H);
        tmem_st4(t_mid + c0, M);
    }
}

struct Params {
    const ReqDesc *reqs;
    int n_reqs;
    int64_t n_items;
    int b_stage_bytes;     // bytes of one operand-tile stage
    int acc_cols;          // tensor-memory columns of one accumulator slot
    int ring;              // stage slots (2..MAX_RING)
    uint32_t tmem_cols;    // allocated tensor-memory columns
    unsigned *status;
    float *resid;          // validation mode: residuals [P][F][T] of request 0, else null
    int box_rows;          // rows per TMA box
};

// Stage counter of a role: slot = stage mod ring, phase parity flips each lap.
struct Ring {
    uint32_t slot = 0, ph = 0;
    __device__ __forceinline__ void next(int ring) {
        if (++slot == (uint32_t)ring) {
            slot = 0;
            ph ^= 1u;
        }
    }
};

// ------------------------------------------------------------ generators
// Generator state of one item: this thread's deviations for its half of the
// columns, and the request constants.
template <int NPHMAX>
struct GenItem {
    uint64_t d2[NPHMAX];
    const float2 *lop;     // this thread's first low-part pair of its half (spectral-index-only models)
    float a21, nu21, inv2s2, sW;
    int Kr, nz;            // nz: pairs of this half from index nz on carry no region
    SeriesPlan sp;
    const float2 *gp;      // amplitude regions: this thread's ln(alpha/abar) pairs of its half, else null
};
template <int NPHMAX>
__device__ __forceinline__ void gen_item_load(GenItem<NPHMAX> &g, const ReqDesc &r, const Item &it, int half,
                                              int m) {
    const int Kr = r.Kp, nph = Kr / 4;
    const float *__restrict__ pts = r.pts32 + (size_t)it.tile * r.pts_rows * 128 + m;
    // this half's pairs [half*nph, half*nph + nph): regions 2*pair, 2*pair+1 (zero beyond N)
#pragma unroll
    for (int i = 0; i < NPHMAX; ++i) {
        const int k = 2 * (half * nph + i);
        const float a = (i < nph && k < Kr - 2) ? pts[(size_t)k * 128] : 0.0f;
        const float b = (i < nph && k + 1 < Kr - 2) ? pts[(size_t)(k + 1) * 128] : 0.0f;
        g.d2[i] = pk2(a, b);
    }
    // low parts: pair-interleaved rows after the other operands (pairs beyond N hold zeros)
    g.lop = reinterpret_cast<const float2 *>(pts - m + (size_t)(Kr + 4 + (r.Na ? Kr : 0)) * 128) +
            (size_t)half * nph * 128 + m;
    g.a21 = half ? pts[(size_t)(Kr - 2) * 128] : 0.0f;
    g.nu21 = half ? pts[(size_t)(Kr - 1) * 128] : 0.0f;
    g.inv2s2 = half ? pts[(size_t)Kr * 128] : 0.0f;
    g.sW = exp2i(*r.scaleW);
    g.sp = series_plan(r.req_stats[1]);
    g.Kr = Kr;
    g.nz = min(nph, max(0, (r.N + 1) / 2 - half * nph));
    g.gp = r.Na ? reinterpret_cast<const float2 *>(pts - m + (size_t)(Kr + 4) * 128) + (size_t)half * nph * 128 + m
                : nullptr;
}

// The weights of every stage of one item by one generator warp (FULL: the
// request's Kr equals the kernel's KP).  Per stage: wait until the weight slot
// is free (the MMAs of stage - ring are done), evaluate and store the weights,
// then one arrival on full[slot].  Returns false on a wait timeout.
template <int KP, bool BF16, bool FULL, bool ALPHA, int DF = 0>
__device__ __forceinline__ bool gen_item(const Params &prm, Barriers *S, Ring &rg, const ReqDesc &r, const Item &it,
                                         const GenItem<KP / 4> &gi, uint32_t w_lane, int half) {
    constexpr int NPHMAX = KP / 4;
    const int lane = threadIdx.x & 31, nch = r.n_tchunks;
    const int nph = gi.Kr / 4;
    const float *__restrict__ nLp = r.nL32;
    const float *__restrict__ nup = r.nu32;
    const float ys = exp2i(-gi.sp.s);
    const uint64_t sW2 = pk2(gi.sW, gi.sW);
    float nL_n = __ldg(nLp + it.f0), nu_n = __ldg(nup + it.f0);
    for (int f = it.f0; f < it.f1; ++f) {
        const float nL = nL_n, nuf = nu_n;
        const int fn = min(f + 1, it.f1 - 1);            // next channel's constants, one ahead
        nL_n = __ldg(nLp + fn);
        nu_n = __ldg(nup + fn);
        // e_j = (nL / 2^s)^j / j! (ALPHA: 2^(-s j) / j!, the series being in y), times 2^sW when s = 0
        uint64_t e2[9];
        e2[0] = 0;
        if (ALPHA) {
            // constant coefficients 2^(-s j) / j! (the series runs in y)
            float pw = gi.sp.s ? 1.0f : gi.sW, fact = 1.0f;
#pragma unroll
            for (int j = 1; j < 9; ++j) {
                pw *= ys;
                fact *= (float)j;
                const float e = pw * (1.0f / fact);
                e2[j] = pk2(e, e);
            }
        } else {
            // the channel's coefficients, written by prep as packed pairs
            const ulonglong2 *cf = reinterpret_cast<const ulonglong2 *>(r.coef2 + (size_t)f * 8);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const ulonglong2 v = __ldg(cf + j);
                e2[2 * j + 1] = v.x;
                e2[2 * j + 2] = v.y;
            }
        }
        float s21 = 0.0f;
        if (half) {
            const float dnu = nuf - gi.nu21;
            s21 = gi.sW * gi.a21 * __expf(-dnu * dnu * gi.inv2s2);
        }
        for (int c = 0; c < nch; ++c) {
            if (!mbar_wait(&S->done[rg.slot], rg.ph ^ 1, S, prm.status, STATUS_TIMEOUT_GEN)) return false;
            tc_fence_after();
            const uint32_t wb = w_lane + rg.slot * KP;
            if (FULL)
                gen_half<NPHMAX, BF16, true, ALPHA, DF>(wb + half * NPHMAX, wb + KP / 2 + half * NPHMAX, gi.d2, gi.lop,
                                                    e2, gi.sp, sW2, NPHMAX, gi.nz, half != 0, s21, gi.sW, gi.gp,
                                                    pk2(nL, nL));
            else
                gen_half<NPHMAX, BF16, false, ALPHA, DF>(wb + half * nph, wb + gi.Kr / 2 + half * nph, gi.d2, gi.lop,
                                                     e2, gi.sp, sW2, nph, gi.nz, half != 0, s21, gi.sW, gi.gp,
                                                     pk2(nL, nL));
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            mbar_arrive_warp(&S->full[rg.slot]);
            rg.next(prm.ring);
        }
    }
    return true;
}

// ------------------------------------------------------------- epilogue
// tcgen05.ld of up to NB 16-column blocks of this thread's accumulator row.
template <int NB>
__device__ __forceinline__ void acc_issue(uint32_t taddr, int b0, int nb, float (&v)[NB][16]) {
    tmem_ld16(taddr + b0 * 16, v[0]);
#pragma unroll
    for (int i = 1; i < NB; ++i)
        if (nb > i) tmem_ld16(taddr + (b0 + i) * 16, v[i]);
}
// Sum of squares of NB 16-column blocks with packed FP32x2 FMAs: accumulator
// pair k sums columns 2k, 2k+8 (low half) and 2k+1, 2k+9 (high half) of every
// block, i.e. eight independent scalar chains in a fixed order, combined by a
// fixed tree (half the instructions of scalar FMAs).
template <int NB>
__device__ __forceinline__ float acc_sumsq(const float (&v)[NB][16], int nb) {
    uint64_t q[4] = {0, 0, 0, 0};
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
        if (bb < nb) {
#pragma unroll
            for (int jj = 0; jj < 16; jj += 2) {
                const uint64_t x = pk2(v[bb][jj], v[bb][jj + 1]);
                q[(jj >> 1) & 3] = fma2(x, x, q[(jj >> 1) & 3]);
            }
        }
    }
    float a[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) upk2(q[k], a[2 * k], a[2 * k + 1]);
    return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

// The epilogue of every stage of one item by one epilogue warp: per stage wait
// for the MMAs (the accumulator), read and reduce this warp's half of the
// t-blocks, release the accumulator slot; per item one compensated partial.
template <bool RESID>
__device__ __forceinline__ bool epi_item(const Params &prm, Barriers *S, Ring &rg, const ReqDesc &r, const Item &it,
                                         uint32_t lane_addr, int half, int m) {
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)it.tile * 128 + m;
    const bool in = p < r.P;
    const int sWexp = *r.scaleW;
    const int nch = r.n_tchunks, Tc = r.Tc, T = r.T, F = r.F;
    const int nblk = r.Tc_pad / 16, hb = (nblk + 1) / 2;
    const int b_lo = half * hb, b_hi = min(nblk, b_lo + hb);
    const int *__restrict__ scaleB = r.scaleB;
    float qs = 0.0f, qc = 0.0f;
    int sb_n = __ldg(scaleB + it.f0 * nch);
    for (int f = it.f0; f < it.f1; ++f) {
        float qf = 0.0f;
        for (int c = 0; c < nch; ++c) {
            const int sb = sb_n;
            sb_n = __ldg(scaleB + min(f * nch + c + 1, it.f1 * nch - 1));   // next stage's scale, one ahead
            if (!mbar_wait(&S->done[rg.slot], rg.ph, S, prm.status, STATUS_TIMEOUT_EPI)) return false;
            tc_fence_after();
            const float unscale = exp2i(-(sWexp + sb));
            const uint32_t taddr = lane_addr + rg.slot * prm.acc_cols;
            float q = 0.0f;
            for (int b0 = b_lo; b0 < b_hi; b0 += EPI_NB) {
                const int nb = min(EPI_NB, b_hi - b0);
                float v[EPI_NB][16];
                acc_issue<EPI_NB>(taddr, b0, nb, v);
                tmem_ld_wait();
                if (RESID) {
                    if (in) {
                        const int t0 = c * Tc, tn = min(Tc, T - t0);
                        for (int bb = 0; bb < nb; ++bb)
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) {
                                const int t = (b0 + bb) * 16 + jj;
                                if (t < tn) prm.resid[((size_t)p * F + f) * T + t0 + t] = -v[bb][jj] * unscale;
                            }
                    }
                } else {
                    q += acc_sumsq<EPI_NB>(v, nb);
                }
            }
            tc_fence_before();
            __syncwarp();
            mbar_arrive_warp(&S->full[rg.slot]);                 // accumulator free for stage + ring
            rg.next(prm.ring);
            qf += q * unscale * unscale;
        }
        kahan_add_dev(qs, qc, qf);
    }
    if (!RESID && in) r.partials[(size_t)p * r.n_part + 2 * it.g + half] = make_float2(qs, -qc);
    return true;
}

// The MMA issuer's walk over its stages (items, channels, t-chunks) with the
// per-item operand geometry.
struct MmaStage {
    int64_t item;
    int f, c, f1, nch, ksteps, Kr, tc_pad;
    uint32_t b_lbo, b_split;
    Ring rg;
    bool valid;
    __device__ __forceinline__ void load_item(const Params &prm) {
        valid = item < prm.n_items;
        if (!valid) return;
        const Item it = decode_item(prm.reqs, prm.n_reqs, item);
        const ReqDesc &r = prm.reqs[it.req];
        f = it.f0;
        f1 = it.f1;
        c = 0;
        nch = r.n_tchunks;
        Kr = r.Kp;
        ksteps = Kr / 16;
        b_lbo = (uint32_t)r.Tc_pad * 16;
        b_split = (uint32_t)(Kr / 8) * b_lbo;
        tc_pad = r.Tc_pad;
    }
    __device__ __forceinline__ void init(const Params &prm) {
        item = blockIdx.x;
        rg = Ring();
        load_item(prm);
    }
    __device__ __forceinline__ void next(const Params &prm, int ring) {
        rg.next(ring);
        if (++c < nch) return;
        c = 0;
        if (++f < f1) return;
        item += gridDim.x;
        load_item(prm);
    }
};

// The stage's MMAs as straight-line code for KS k steps: the issuing thread
// shares its scheduler with ALU warps, and loop control between the MMAs
// measurably delays them.
//
// Each MMA rounds its sum toward zero in FP32 (measured on this part: the
// accumulator and the 16 products are aligned to the largest exponent E,
// truncated at 2^(E-25), added, and the sum truncated to FP32), so every MMA
// whose result is as large as the residual biases |D - M| low by about half an
// ulp.  The small correction products (hi*mid, mid*hi) of every k step go
// first, while the accumulator is still small, then the hi*hi products, last k
// step first: only the last MMA ends at the size of the residual, and the
// reduction adds back its expected half-ulp (chi2_scale).
template <int KS>
__device__ __forceinline__ void issue_mmas(uint32_t d_tmem, uint32_t w_hi, uint32_t w_mid, uint32_t b_addr,
                                           uint32_t b_lbo, uint32_t b_split, uint32_t idesc) {
#pragma unroll
    // one descriptor for the stage's tile; each MMA adds its offset (16-byte
    // units) to the start-address field, which shared-memory addresses below
    // 256 KB never carry out of (the issuing thread is busy about half the
    // kernel's time in this sequence: building every descriptor afresh cost 3%)
    const uint64_t d0 = smem_desc(b_addr, b_lbo, 128);
    const uint32_t step = (2 * b_lbo) >> 4, split = b_split >> 4;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        mma_f16_ts(d_tmem, w_hi + ks * 8, d0 + split + ks * step, idesc, ks > 0 ? 1u : 0u);
        mma_f16_ts(d_tmem, w_mid + ks * 8, d0 + ks * step, idesc, 1u);
    }
#pragma unroll
    for (int ks = KS - 1; ks >= 0; --ks)
        mma_f16_ts(d_tmem, w_hi + ks * 8, d0 + ks * step, idesc, 1u);
}

template <int KP, bool BF16>
__device__ __forceinline__ void issue_stage(const MmaStage &st, uint32_t tmem, uint32_t w_col0, char *b_slots,
                                            const Params &prm) {
    const uint32_t idesc = instr_desc(128, st.tc_pad, BF16);
    const uint32_t w_hi = tmem + w_col0 + st.rg.slot * KP, w_mid = w_hi + st.Kr / 2;
    const uint32_t b_addr = smem_u32(b_slots + st.rg.slot * prm.b_stage_bytes);
    const uint32_t d_tmem = tmem + st.rg.slot * prm.acc_cols;
    if (KP == 16 || st.ksteps == 1) issue_mmas<1>(d_tmem, w_hi, w_mid, b_addr, st.b_lbo, st.b_split, idesc);
    else if (KP == 32 || st.ksteps == 2) issue_mmas<2>(d_tmem, w_hi, w_mid, b_addr, st.b_lbo, st.b_split, idesc);
    else if (st.ksteps == 3) issue_mmas<3>(d_tmem, w_hi, w_mid, b_addr, st.b_lbo, st.b_split, idesc);
    else issue_mmas<4>(d_tmem, w_hi, w_mid, b_addr, st.b_lbo, st.b_split, idesc);
}

// Tensor-memory columns: accumulator of slot s at s * acc_cols; weights of
// slot s at ring * acc_cols + s * KP (hi: Kr/2 columns, then mid: Kr/2).
// RESID: validation mode (residuals of request 0 to prm.resid instead of the
// chi2 partials); a separate instantiation keeps that code out of the
// production kernel.  LEAN: every request of the launch has spectral-index
// regions only (1: and K = KP, 2: K of any size), so the generators carry the
// variants of their loop those requests need instead of all of them, each with
// the series degree fixed per work item (smaller code: 5-9% faster).
template <int KP, bool BF16, bool RESID, int LEAN>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    tc_loglike_kernel(const __grid_constant__ CUtensorMap tmap, const Params prm) {
    extern __shared__ __align__(1024) char smem_raw[];
    char *smem = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int ring = prm.ring;
    char *b_slots = smem;                                             // [ring] x b_stage_bytes
    Barriers *S = reinterpret_cast<Barriers *>(b_slots + ring * prm.b_stage_bytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ring; ++s) {
            mbar_init(&S->full[s], FULL_ARRIVALS);
            mbar_init(&S->done[s], 1);
        }
        mbar_init(&S->drain, 1);
        S->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == WARP_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem_base)),
                     "r"(prm.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    // the set-up above touches only this CTA's shared and tensor memory; from
    // here on the kernel reads what the operand pass wrote
    pdl_wait();
    const uint32_t tmem = S->tmem_base;
    const uint32_t w_col0 = (uint32_t)(ring * prm.acc_cols);
    const ReqDesc *__restrict__ reqs = prm.reqs;

    if (warp < 8) {
        // ================================================ weight generators
        const int quad = warp & 3, half = warp >> 2;
        const int m = quad * 32 + lane;
        const uint32_t w_lane = tmem + ((uint32_t)(quad * 32) << 16) + w_col0;
        Ring rg;
        bool ok = true;
        GenItem<KP / 4> gi;
        for (int64_t item = blockIdx.x; item < prm.n_items && ok; item += gridDim.x) {
            const Item it = decode_item(reqs, prm.n_reqs, item);
            const ReqDesc &r = reqs[it.req];
            gen_item_load(gi, r, it, half, m);
            // a request's Kr fixes the column count of each half; it must match its operand tiles
            if (LEAN == 1 || (LEAN == 2 && gi.Kr == KP))
                ok = gi.sp.D == 3 ? gen_item<KP, BF16, true, false, 3>(prm, S, rg, r, it, gi, w_lane, half)
                   : gi.sp.D == 5 ? gen_item<KP, BF16, true, false, 5>(prm, S, rg, r, it, gi, w_lane, half)
                                  : gen_item<KP, BF16, true, false, 8>(prm, S, rg, r, it, gi, w_lane, half);
            else if (LEAN == 2)
                ok = gi.sp.D == 3 ? gen_item<KP, BF16, false, false, 3>(prm, S, rg, r, it, gi, w_lane, half)
                   : gi.sp.D == 5 ? gen_item<KP, BF16, false, false, 5>(prm, S, rg, r, it, gi, w_lane, half)
                                  : gen_item<KP, BF16, false, false, 8>(prm, S, rg, r, it, gi, w_lane, half);
            else if (r.Na) ok = gi.Kr == KP ? gen_item<KP, BF16, true, true>(prm, S, rg, r, it, gi, w_lane, half)
                                            : gen_item<KP, BF16, false, true>(prm, S, rg, r, it, gi, w_lane, half);
            else if (gi.Kr == KP) ok = gen_item<KP, BF16, true, false>(prm, S, rg, r, it, gi, w_lane, half);
            else ok = gen_item<KP, BF16, false, false>(prm, S, rg, r, it, gi, w_lane, half);
        }
    } else if (warp < 16) {
        // ========================================================= epilogue
        const int quad = warp & 3, half = (warp - 8) >> 2;
        const int m = quad * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16);
        // the accumulators of every slot start free: count their first release
        if (lane == 0)
            for (int sl = 0; sl < ring; ++sl) mbar_arrive(&S->full[sl]);
        Ring rg;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < prm.n_items && ok; item += gridDim.x) {
            const Item it = decode_item(reqs, prm.n_reqs, item);
            ok = epi_item<RESID>(prm, S, rg, reqs[it.req], it, lane_addr, half, m);
        }
    } else if (warp == WARP_TMA) {
        // ====================================================== TMA producer
        bool ok = true;
        Ring rg;
        if (lane == 0) {
            for (int64_t item = blockIdx.x; item < prm.n_items && ok; item += gridDim.x) {
                const Item it = decode_item(reqs, prm.n_reqs, item);
                const ReqDesc &r = reqs[it.req];
                const int rows = (int)r.tile_rows, nch = r.n_tchunks;
                const int64_t tile_row0 = r.tile_row0;
                for (int f = it.f0; f < it.f1 && ok; ++f) {
                    for (int c = 0; c < nch; ++c) {
                        // the operand slot is free once the MMAs of stage - ring are done
                        if (!mbar_wait(&S->done[rg.slot], rg.ph ^ 1, S, prm.status, STATUS_TIMEOUT_TMA)) { ok = false; break; }
                        mbar_arrive_expect_tx(&S->full[rg.slot], (uint32_t)(rows * 128));
                        const int64_t row0 = tile_row0 + (int64_t)(f * nch + c) * rows;
                        char *dst = b_slots + rg.slot * prm.b_stage_bytes;
                        for (int jr = 0; jr < rows; jr += prm.box_rows)
                            tma_load_2d(dst + jr * 128, &tmap, 0, (int)(row0 + jr), &S->full[rg.slot]);
                        rg.next(ring);
                    }
                }
            }
            if (!ok) {
                // copies already issued land within microseconds; give them time
                // before the CTA (and its shared memory) goes away
                const uint64_t t0 = globaltimer();
                while (globaltimer() - t0 < 200000ull) {
                }
            }
        }
        __syncwarp();
    } else {
        // ========================================================= MMA issuer
        // Stages are issued in pairs when the next one is already complete: a
        // barrier operation right after a burst of MMAs stalls the issuing thread
        // until they drain, so two stages' MMAs and commits go out back to back
        // with the next stage's barrier tested (non-blocking) before the first.
        bool ok = true;
        if (lane == 0) {
            MmaStage cur;
            cur.init(prm);
            while (cur.valid && ok) {
                if (!mbar_wait(&S->full[cur.rg.slot], cur.rg.ph, S, prm.status, STATUS_TIMEOUT_MMA)) { ok = false; break; }
                MmaStage nxt = cur;
                nxt.next(prm, ring);
                const bool pair = nxt.valid && mbar_test(&S->full[nxt.rg.slot], nxt.rg.ph);
                tc_fence_after();
                issue_stage<KP, BF16>(cur, tmem, w_col0, b_slots, prm);
                mma_commit(&S->done[cur.rg.slot]);
                if (pair) {
                    issue_stage<KP, BF16>(nxt, tmem, w_col0, b_slots, prm);
                    mma_commit(&S->done[nxt.rg.slot]);
                    nxt.next(prm, ring);
                }
                cur = nxt;
            }
            // drain: every MMA issued so far completes before tensor memory is freed
            mma_commit(&S->drain);
            uint64_t t0 = globaltimer();
            while (!mbar_try_wait(&S->drain, 0)) {
                if (globaltimer() - t0 > WAIT_LIMIT_NS) {
                    atomicOr(prm.status, STATUS_TIMEOUT_DRAIN);
                    break;
                }
            }
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == WARP_MMA) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(prm.tmem_cols)
                     : "memory");
    }
}

// ------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::once_flag g_encode_once;
int g_encode_rc = FG21_OK;

size_t smem_bytes(int ring, int b_stage_bytes) {
    return 1024 + (size_t)ring * b_stage_bytes + sizeof(Barriers) + 64;
}

template <int KP, bool BF16, bool RESID, int LEAN>
cudaError_t launch_kpr(const CUtensorMap &map, const Params &prm, int grid, size_t sm, cudaStream_t stream) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc_loglike_kernel<KP, BF16, RESID, LEAN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaError_t e = launch_dependent(tc_loglike_kernel<KP, BF16, RESID, LEAN>, dim3(grid), dim3(NUM_THREADS), sm,
                                     stream, map, prm);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int KP, bool BF16>
cudaError_t launch_kp(const CUtensorMap &map, const Params &prm, int grid, size_t sm, int lean,
                      cudaStream_t stream) {
    if (prm.resid) return launch_kpr<KP, BF16, true, 0>(map, prm, grid, sm, stream);
    if (lean == 1) return launch_kpr<KP, BF16, false, 1>(map, prm, grid, sm, stream);
    if (lean == 2 && KP > 16) return launch_kpr<KP, BF16, false, 2>(map, prm, grid, sm, stream);
    return launch_kpr<KP, BF16, false, 0>(map, prm, grid, sm, stream);
}

cudaError_t launch_common(const ReqDesc *d_reqs, int n_reqs, int64_t n_items, int kp_max, int tc_pad_max,
                          int precision, void *arena, int64_t arena_rows, unsigned *status, float *resid,
                          int box_rows, int num_sms, int lean, cudaStream_t stream) {
    if (n_items == 0) return cudaSuccess;
    if (tc_map_init() != FG21_OK) return cudaErrorNotSupported;
    CUtensorMap map;
    cuuint64_t gdim[2] = {64, (cuuint64_t)arena_rows};
    cuuint64_t gstride[1] = {128};
    if (box_rows < 8 || box_rows > 256 || box_rows % 8) return cudaErrorInvalidValue;
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estride[2] = {1, 1};
    CUresult cr = g_encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, arena, gdim, gstride, box, estride,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int kp = tc_launch_kp(kp_max);
    if (tc_pad_max < 16 || tc_pad_max > TC_MAX || tc_pad_max % 16) return cudaErrorInvalidValue;
    Params prm;
    prm.reqs = d_reqs;
    prm.n_reqs = n_reqs;
    prm.n_items = n_items;
    prm.b_stage_bytes = ((4 * kp_max * tc_pad_max) + 1023) & ~1023;
    prm.acc_cols = tc_pad_max;
    // as many stage slots (accumulator + weights in tensor memory) as fit, 2..4
    const int per_slot = tc_pad_max + kp;
    int ring = 512 / per_slot;
    if (ring > MAX_RING) ring = MAX_RING;
    if (ring < 2) return cudaErrorInvalidValue;
    // ... and as fit shared memory next to the barriers
    while (ring > 2 && smem_bytes(ring, prm.b_stage_bytes) > 227 * 1024) --ring;
    prm.ring = ring;
    uint32_t cols = 32;
    while (cols < (uint32_t)(ring * per_slot)) cols *= 2;
    if (cols > 512) return cudaErrorInvalidValue;
    prm.tmem_cols = cols;
    prm.status = status;
    prm.resid = resid;
    prm.box_rows = box_rows;
    // at least ~120 KB so that a single CTA (and its tensor memory) owns each SM
    size_t sm = smem_bytes(ring, prm.b_stage_bytes);
    if (sm < 120 * 1024) sm = 120 * 1024;
    if (sm > 227 * 1024) return cudaErrorInvalidValue;
    const int grid = (int)(n_items < num_sms ? n_items : num_sms);
    const bool bf16 = precision == FG21_PREC_BF16X3;
    if (kp == 16)
        return bf16 ? launch_kp<16, true>(map, prm, grid, sm, lean, stream)
                    : launch_kp<16, false>(map, prm, grid, sm, lean, stream);
    if (kp == 32)
        return bf16 ? launch_kp<32, true>(map, prm, grid, sm, lean, stream)
                    : launch_kp<32, false>(map, prm, grid, sm, lean, stream);
    return bf16 ? launch_kp<64, true>(map, prm, grid, sm, lean, stream)
                : launch_kp<64, false>(map, prm, grid, sm, lean, stream);
}

// Self-test of the bounded waits, on barriers that nothing ever arrives on.
// Warp 0 waits with the kernel's limit: it gives up first, sets
// STATUS_TIMEOUT_TMA and raises the abort flag.  Warps 1-3 wait with twice
// that limit and must come back through the abort flag, as the other roles of
// a stalled likelihood launch do, without a status bit of their own.
// elapsed[w] = nanoseconds warp w waited (all ones if its barrier completed).
__global__ void __launch_bounds__(128) wait_selftest_kernel(unsigned *status, unsigned long long *elapsed) {
    __shared__ Barriers S;
    if (threadIdx.x == 0) {
        mbar_init(&S.full[0], 1);
        mbar_init(&S.full[1], 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const uint64_t t0 = globaltimer();
    const bool ok = warp == 0 ? mbar_wait(&S.full[0], 0, &S, status, STATUS_TIMEOUT_TMA)
                              : mbar_wait(&S.full[1], 0, &S, status, STATUS_TIMEOUT_GEN, 2 * WAIT_LIMIT_NS);
    const uint64_t dt = globaltimer() - t0;
    if ((threadIdx.x & 31) == 0) elapsed[warp] = ok ? ~0ull : dt;
}

// One MMA exactly as the likelihood kernel issues it (kind::f16, F16
// operands, F32 accumulator, M = 128, N = 16, K = 16, A in tensor memory, B
// from shared memory by descriptor): d = c + a b for caller-given operands, so
// that a host can check the accumulator's rounding.  a [128][16] and b
// [16 n][16 k] are F16 bit patterns, c and d [128][16] FP32.  One CTA of 128
// threads; the completion wait is bounded (status bit STATUS_TIMEOUT_MMA).
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(const uint16_t *__restrict__ a,
                                                            const uint16_t *__restrict__ b,
                                                            const float *__restrict__ c, float *__restrict__ d,
                                                            unsigned *status) {
    __shared__ __align__(1024) uint16_t sb[2][16][8];      // [k chunk][n][8 values of k]
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                     "r"(32)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < 256; i += 128) sb[(i & 15) >> 3][i >> 4][i & 7] = b[i];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tbase, lane_base = tm + ((uint32_t)(warp * 32) << 16);
    uint32_t v[16];
#pragma unroll
    for (int n = 0; n < 16; ++n) v[n] = __float_as_uint(c[tid * 16 + n]);
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            lane_base),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = (uint32_t)a[tid * 16 + 2 * j] | ((uint32_t)a[tid * 16 + 2 * j + 1] << 16);
    tmem_st4(lane_base + 16, w);
    tmem_st4(lane_base + 20, w + 4);
    tmem_st_wait();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        mma_f16_ts(tm, tm + 16, smem_desc(smem_u32(&sb[0][0][0]), 16 * 16, 128), instr_desc(128, 16, false), 1u);
        mma_commit(&bar);
    }
    const uint64_t t0 = globaltimer();
    bool ok = true;
    while (!mbar_try_wait(&bar, 0)) {
        if (globaltimer() - t0 > WAIT_LIMIT_NS) {
            if (tid == 0) atomicOr(status, STATUS_TIMEOUT_MMA);
            ok = false;
            break;
        }
    }
    tc_fence_after();
    float r[16];
    tmem_ld16(lane_base, r);
    tmem_ld_wait();
#pragma unroll
    for (int n = 0; n < 16; ++n) d[tid * 16 + n] = ok ? r[n] : __int_as_float(0x7FC00000);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(32) : "memory");
    }
}

}  // namespace

cudaError_t launch_mma_probe(const uint16_t *a, const uint16_t *b, const float *c, float *d, unsigned *status,
                             cudaStream_t stream) {
    mma_probe_kernel<<<1, 128, 0, stream>>>(a, b, c, d, status);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned *status, unsigned long long *elapsed, cudaStream_t stream) {
    wait_selftest_kernel<<<1, 128, 0, stream>>>(status, elapsed);
    return cudaGetLastError();
}

int tc_map_init() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            g_encode_rc = set_error(FG21_E_CUDA, "cuTensorMapEncodeTiled is not available");
            return;
        }
        g_encode = (EncodeTiledFn)fn;
    });
    return g_encode_rc;
}

int tc_box_rows(const int64_t *tile_rows, int n) {
    int64_t g = 0;
    for (int k = 0; k < n; ++k) {
        int64_t a = tile_rows[k], b = g;
        while (b) {
            int64_t t = a % b;
            a = b;
            b = t;
        }
        g = a;
    }
    int64_t box = 8;
    for (int64_t c = 256; c >= 8; c -= 8)
        if (g % c == 0) {
            box = c;
            break;
        }
    return (int)box;
}

cudaError_t launch_tc(const TcLaunch &L, int num_sms, cudaStream_t stream) {
    return launch_common(L.d_reqs, L.n_reqs, L.n_items, L.kp_max, L.tc_pad_max, L.precision, L.arena,
                         L.arena_rows, L.status, nullptr, L.box_rows, num_sms, L.lean, stream);
}

cudaError_t launch_tc_residuals(const ReqDesc *h_req, const ReqDesc *d_req, int precision, float *resid,
                                cudaStream_t stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int sms = 1;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    char *arena = h_req->tiles - h_req->tile_row0 * 128;
    const int64_t rows = h_req->tile_row0 + (int64_t)h_req->F * h_req->n_tchunks * h_req->tile_rows;
    const int64_t items = (int64_t)h_req->n_tiles * h_req->G;
    return launch_common(d_req, 1, items, h_req->Kp, h_req->Tc_pad, precision, arena, rows, h_req->status, resid,
                         tc_box_rows(&h_req->tile_rows, 1), sms, 0, stream);
}

}  // namespace fg21
