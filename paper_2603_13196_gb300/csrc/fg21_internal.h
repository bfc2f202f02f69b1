// Internal declarations shared by the host code and the CUDA kernels of libfg21.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fg21.h"

namespace fg21 {

// ------------------------------------------------------------------ errors
int set_error(int code, const char *fmt, ...);
void set_invalid_count(int64_t n);
int cuda_error(cudaError_t e, const char *what);
#define FG21_CUDA_TRY(expr)                                            \
    do {                                                               \
        cudaError_t e__ = (expr);                                      \
        if (e__ != cudaSuccess) return ::fg21::cuda_error(e__, #expr); \
    } while (0)

// Device status word bits (written by kernels with atomicOr).
enum : unsigned {
    STATUS_TIMEOUT_TMA = 1u,
    STATUS_TIMEOUT_MMA = 2u,
    STATUS_TIMEOUT_GEN = 4u,
    STATUS_TIMEOUT_EPI = 8u,
    STATUS_TIMEOUT_DRAIN = 16u,
    STATUS_BAD_SHAPE = 32u,
};

constexpr int TILE_M = 128;         // points per MMA tile (tcgen05 M)
constexpr int TC_MAX = 192;         // max t-columns per MMA (tcgen05 N): two stage slots of
                                    // accumulators (<= 192 columns) plus weights (<= 64 columns)
                                    // fit the 512 tensor-memory columns of an SM
constexpr int STAT_BLOCK = 128;     // points (threads) per statistics block of the per-request prep
constexpr int KP_MAX = 64;          // max padded K on the tensor path
static_assert(STAT_BLOCK % TILE_M == 0, "a statistics block covers whole 128-point tiles");

// Series parameters of the weights' expm1 (tensor path) for |argument| <= xmax:
// s halvings of the argument (undone by squarings) until it is at most 0.55,
// then the Taylor degree D: 3 for |y| <= 0.01, 5 for |y| <= 0.1, else 8.  Prep
// (the per-channel coefficients) and the generators derive it from the same x.
struct SeriesPlan {
    int D, s;
};
__host__ __device__ inline SeriesPlan series_plan(double xmax) {
    SeriesPlan sp{8, 0};
    while (xmax > 0.55 && sp.s < 12) {
        xmax *= 0.5;
        ++sp.s;
    }
    sp.D = xmax <= 0.01 ? 3 : xmax <= 0.1 ? 5 : 8;
    return sp;
}

// Per-request descriptor, laid out identically on host and device.
struct ReqDesc {
    // model arrays (device)
    const double *A;       // [N][F][T]
    const double *B;       // [F][T]
    const double *data;    // [F][T]
    const double *L;       // [F] ln(nu_f / nu0)
    const double *nu;      // [F] MHz
    const float *A32;      // [N][F][T]   (direct FP32 form)
    const float *B32;      // [F][T]
    const float *data32;   // [F][T]
    const float *A_lo;     // [N][F][T]   A - (float)A: with A32 a double-float copy of A (tensor-path prep)
    const float *E_hi;     // [F][T]      E = D - T_CMB B as a double-float pair (hi, lo)
    const float *E_lo;     // [F][T]
    // request I/O (device)
    const double *params;  // [P][NPF+4]
    double *logL;          // [P]
    double t_cmb;
    double Lmax;           // max_f |ln(nu_f / nu0)|
    int64_t P;
    int N, F, T;           // N: components (rows of A, weight columns) = max(Na, 1) * Nb
    int Nb;                // spectral-index regions; component c has beta index c % Nb
    int Na;                // amplitude parameters (0: none, alpha = 1); component c has alpha index c / Nb
    int NPF;               // foreground parameters Nb + Na: a parameter row is [beta.., alpha.., A21, nu21,
                           // sigma21, sigma_n] of NPF + 4 values
    int Kp;                // K = N + 2 padded to a multiple of 16 (tensor path)
    int pts_rows;          // rows of 128 floats per point tile of pts32
    int Tc, Tc_pad, n_tchunks;   // t-chunks: Tc columns each (last may be shorter), padded to 16
    int G, ch_per_group;         // channel groups per 128-point tile
    int cpg_hint;                // channels per group chosen by the autotuner for this size (0 = model)
    int n_part;                  // partial sums per point (G on the SIMT forms, 2G on the tensor path)
    int simt_tc;                 // SIMT forms: t-columns staged per round (128, or 64 / 32 where the
                                 // double-buffered slabs of a large N would not fit shared memory;
                                 // never more than T rounded up to a multiple of 8)
    int n_tiles;                 // ceil(P / 128)
    int n_stat_blocks;           // ceil(P / STAT_BLOCK)
    int64_t item_begin;          // first global work-item id of this request
    int64_t tile_row0;           // first 128-byte row of this request's operand tiles in the arena
    int64_t tile_rows;           // rows per (channel, t-chunk) tile
    int64_t pt_begin;            // first global point index of this request (reduction)
    char *tiles;                 // this request's operand tiles (arena + tile_row0 * 128)
    // workspace (device)
    float *stat_part;      // [n_stat_blocks][2 NPF + 2]: min, max per foreground parameter, n_valid,
                           // max|A21|
    double *beta_bar;      // [NPF] reference point: midrange of each foreground parameter (beta_bar, alpha_bar)
    double *req_stats;     // [4]: n_valid, bound x on |expm1 argument|, max|A21|, reserved
    float *nL32;           // [F] -ln(nu_f/nu0)
    unsigned long long *coef2;   // [F][8] the weight series' coefficients e_j = (nL_f 2^-s)^j / j! (times
                                 // 2^sW when s = 0), j = 1..8, each as a packed FP32 pair (tensor path)
    float *nu32;           // [F]
    int *scaleB;           // [F * n_tchunks] power-of-two exponent of each operand tile
    int *scaleW;           // [1] power-of-two exponent of the weight operand
    float *Bp32;           // [N][F][T] wbar_i A (FP32, SIMT delta form)
    float *dref32;         // [F][T]    reference residual (FP32, SIMT delta form)
    float2 *partials;      // [P][n_part] compensated partial chi^2 (hi, lo)
    unsigned char *pvalid; // [P] 1 if the point is valid (written by the statistics pass)
    double2 *pnorm;        // [P] (F T ln(2 pi sigma_n^2), 1 / sigma_n^2) of each valid point (tensor path: written
                           // by prep's point blocks; null on the SIMT paths, whose reduction forms them itself)
    float *pts32;          // [n_tiles][pts_rows][128] per point: beta - bbar of each component's
                           // spectral index (rows < Kp-2, zero beyond N), then A21, nu21,
                           // 1/(2 sigma21^2) (rows Kp-2..Kp); with amplitude parameters, rows
                           // Kp+4.. hold ln(alpha / alpha_bar) of each component, pair-interleaved
                           // ([Kp/2 pairs][128 points][2]); the last Kp rows hold the low parts
                           // of the deviations (beta - bbar minus its FP32 rounding), pair-
                           // interleaved the same way; tensor path.  SIMT forms: [n_tiles]
                           // [Nb + Na][128] beta (direct) or beta - bbar (delta) of each spectral
                           // index, then alpha (direct) or ln(alpha / abar) (delta)
    double chi2_scale;     // the reduction multiplies chi2 by this: 1 + (2/3) 2^-23 on the tensor
                           // path (the expected half-ulp that the accumulator's final rounding
                           // toward zero drops, relative to chi2), 1 on the SIMT paths
    unsigned *status;      // device status word (shared by a launch)
    unsigned long long *invalid;  // invalid-point counter
};

// Sizes of one request's workspace pieces (bytes, each 256-aligned).
struct ReqLayout {
    size_t stat_part, beta_bar, req_stats, nL32, nu32, coef2, scaleB, scaleW, Bp32, dref32, partials, pvalid, pnorm,
        pts32, tiles;
    size_t total() const {
        return stat_part + beta_bar + req_stats + nL32 + nu32 + coef2 + scaleB + scaleW + Bp32 + dref32 +
               partials + pvalid + pnorm + pts32 + tiles;
    }
};

// Shape decisions for one request (autotuned channel grouping).
void plan_request(ReqDesc &r, int precision, int num_sms, int64_t total_tiles_in_launch);
ReqLayout request_layout(const ReqDesc &r, int precision);

// ------------------------------------------------------- kernel launchers
// All enqueue on `stream` and return cudaError_t of the launch.
cudaError_t launch_prep(const ReqDesc *h_reqs, const ReqDesc *d_reqs, int n_reqs, int precision,
                        int max_stat_blocks, int max_F_chunks, int max_tiles, cudaStream_t stream);
cudaError_t launch_simt(const ReqDesc *h_reqs, const ReqDesc *d_reqs, int n_reqs, int precision,
                        cudaStream_t stream);
// Blocks of the SIMT kernel of `precision` that one SM holds at once for a
// request shape (the CUDA occupancy calculator, cached per device and shape),
// and the t-chunk width that shape stages (the widest of 128, 64, 32 whose
// shared memory fits a block).
int simt_blocks_per_sm(int N, int tc, int precision);
int simt_chunk_width(int N, int T);
cudaError_t launch_reduce(const ReqDesc *h_reqs, const ReqDesc *d_reqs, int n_reqs,
                          cudaStream_t stream);
cudaError_t launch_model_eval(const ReqDesc *h_req, const ReqDesc *d_req, int precision,
                              double *d_out, cudaStream_t stream);
// Tensor kernel in validation mode: writes the residual D - M of every (p, f, t)
// of one request to resid [P][F][T] instead of reducing it.
cudaError_t launch_tc_residuals(const ReqDesc *h_req, const ReqDesc *d_req, int precision, float *resid,
                                cudaStream_t stream);

// Tensor-core path: one persistent launch over all requests' work items.
struct TcLaunch {
    const ReqDesc *d_reqs;
    int n_reqs;
    int64_t n_items;
    int kp_max;              // max padded K over requests
    int tc_pad_max;          // max padded t-chunk over requests
    int precision;           // FG21_PREC_FP16X3 / BF16X3
    int box_rows;            // TMA box height (divides every request's tile height)
    void *arena;             // operand tile arena (device), 128-byte rows
    int64_t arena_rows;
    unsigned *status;
    int lean;                // 1: every request has no amplitude regions and Kp equal to the launch's padded
                             // K; 2: no amplitude regions, Kp of any size; 0: otherwise
};
// The padded K of a tensor-core launch whose largest request K is kp_max.
inline int tc_launch_kp(int kp_max) { return kp_max <= 16 ? 16 : kp_max <= 32 ? 32 : 64; }
cudaError_t launch_tc(const TcLaunch &L, int num_sms, cudaStream_t stream);
// One CTA whose waits expire by design (status + 4 per-warp waiting times).
cudaError_t launch_wait_selftest(unsigned *status, unsigned long long *elapsed, cudaStream_t stream);
constexpr int WAIT_SELFTEST_WARPS = 4;
// One tcgen05.mma (kind::f16, M = 128, N = 16, K = 16) on device buffers:
// d = c + a b (a [128][16], b [16][16] F16 bits, c, d [128][16] FP32).
cudaError_t launch_mma_probe(const uint16_t *a, const uint16_t *b, const float *c, float *d, unsigned *status,
                             cudaStream_t stream);
// Largest multiple of 8 (<= 256 rows of 128 bytes) dividing every tile height.
int tc_box_rows(const int64_t *tile_rows, int n);
int tc_map_init();  // resolves cuTensorMapEncodeTiled; FG21_OK or error

// Region building on the current device (fg21_build.cu): the importance
// weights w[npix] of `weighting` (Sec. 4.2) and, optionally, B[F][T]; the
// response functions A[N][F][T] of the components `lab` (Sec. 2.2 eq.
// chromatic_function) and B.  Same FP64 arithmetic as the host code, other
// summation order.  FG21_OK or an error code (message set).
int device_importance(const fg21_sky *s, const fg21_obs *o, int weighting, std::vector<double> &w,
                      std::vector<double> *B);
int device_precompute(const fg21_sky *s, const fg21_obs *o, const std::vector<int32_t> &lab, int N,
                      std::vector<double> &A, std::vector<double> &B);

}  // namespace fg21
