/*
 * fg21.h -- C ABI of the GB300 library for the batched likelihood of the
 * region-partitioned global-21cm foreground model (arXiv 2603.13196).
 *
 * Conventions for every call below:
 *  - All functions are `extern "C"`, never throw, and return an int status:
 *    FG21_OK (0) or a negative FG21_E_* code.  fg21_last_error() returns a
 *    thread-local message describing the last failure of the calling thread.
 *  - Arrays are row-major (C order) FP64 in HOST memory unless a name says
 *    `d_` (device memory of the current CUDA device).
 *  - Parameter rows follow the paper's parameter vector (Sec. 2.3, eq.
 *    likelihood and the table of priors):
 *        theta_p = [beta_1 .. beta_N, A21 (K), nu21 (MHz), sigma21 (MHz), sigma_n (K)]
 *    with regions in ascending spectral-index order, so params is P x (N+4).
 *    Models with amplitude regions (fg21_build_regions_ab, Sec. 2.2 eqs.
 *    forward_model / fast_forward_model with N_alpha > 1) insert the scale
 *    factors after the spectral indices:
 *        theta_p = [beta_1 .. beta_Nb, alpha_1 .. alpha_Na, A21, nu21, sigma21, sigma_n]
 *    (P x (Nb+Na+4); fg21_model_shape gives the row length of any model).
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.
 *  - The library owns the device memory of a model; handles are not
 *    thread-safe: one call at a time per model (the serving loop, below, is the
 *    concurrent interface).
 *  - There is no CPU fallback: without a usable CUDA device every compute call
 *    returns FG21_E_CUDA.
 */
#ifndef FG21_H
#define FG21_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define FG21_OK            0
#define FG21_E_ARG        -1   /* invalid argument (NULL, size out of range, bad enum, non-unit vector) */
#define FG21_E_NOMEM      -2   /* host or device allocation failed */
#define FG21_E_CUDA       -3   /* CUDA runtime / driver error, or no usable device */
#define FG21_E_TIMEOUT    -4   /* a wait ran past its limit (serving tickets) */
#define FG21_E_BUSY       -5   /* admission deferred: not enough memory budget yet */
#define FG21_E_STATE      -6   /* call not valid in the object's current state */
#define FG21_E_NOTFOUND   -7   /* unknown run id or ticket */
#define FG21_E_CANCELLED  -8   /* the request was cancelled before it ran */
#define FG21_E_DEVICE     -9   /* a kernel reported an internal failure (bounded wait expired) */
#define FG21_E_RANGE     -10   /* problem size above a documented limit */

/* ------------------------------------------------------------------ enums */
/* Partition schemes (Sec. 4.1 and Sec. 4.3). */
#define FG21_SCHEME_RECURSIVE     0  /* Algorithm 2: bisect the largest-mass region at its beta midpoint */
#define FG21_SCHEME_HIERARCHICAL  1  /* Algorithm 1: 2^floor(log2 N) equal-mass regions, then bisect
                                        the widest unsplit base region at its importance midpoint */
#define FG21_SCHEME_LINEAR        2  /* equal-width beta intervals (Sec. 4.1 (i), not nested) */
#define FG21_SCHEME_PERCENTILE    3  /* equal pixel-count intervals (Sec. 4.1 (ii), not nested) */

/* Importance weightings (Sec. 4.2). */
#define FG21_WEIGHT_BEAM     0  /* T_sky D H / integral (eq. w_beam_dynamic), the default */
#define FG21_WEIGHT_SKY      1  /* T_sky H / integral */
#define FG21_WEIGHT_HORIZON  2  /* H / integral */
#define FG21_WEIGHT_UNIFORM  3  /* 1/Npix (observation independent) */

/* Arithmetic of the likelihood kernels (all produce FP64 logL). */
#define FG21_PREC_FP16X3      0  /* tcgen05, reference-subtracted contraction in split FP16 (hi*hi + hi*mid +
                                    mid*hi), FP32 accumulation in tensor memory; the default */
#define FG21_PREC_BF16X3      1  /* as FP16X3 with BF16 operands (wider range, 8-bit significands) */
#define FG21_PREC_FP32_DELTA  2  /* SIMT FP32, reference-subtracted */
#define FG21_PREC_FP32_DIRECT 3  /* SIMT FP32, the plain eq. fast_forward_model in FP32 (comparator) */
/* Accuracy of the reference-subtracted forms: each residual carries a relative
 * error of about u (2^-22 split FP16, 2^-16 split BF16, 2^-24 FP32) of the
 * batch's departure from its reference point, sum_i |A_i| |w(beta_p,i) - w(bbar_i)|,
 * so the logL error grows with the spread of the batch in beta and with the
 * number of cells F T.  Measured with split FP16 at F T = 30100: 3e-3 nats for a
 * batch within 1e-6 of one point, 0.03 nats within 1e-5.  The plain FP32 form
 * carries u of the whole foreground instead. */

/* Limits. */
#define FG21_MAX_REGIONS_TC  62      /* N <= 62 on the tensor-core path (K = N + 2 padded to <= 64) */
#define FG21_MAX_REGIONS    126      /* N limit of region building and of the SIMT paths */

/* ------------------------------------------------------------------ types */
typedef struct fg21_model fg21_model;     /* opaque: resident A, B, data of one observation + partition */
typedef struct fg21_server fg21_server;   /* opaque: serving loop */
typedef struct fg21_graph fg21_graph;     /* opaque: a captured evaluation of a fixed batch */

/* Pixelised sky (Sec. 2.1).  dirs: unit vectors in the frame of `zenith`;
 * t230: the 230 MHz template [K]; beta: per-pixel spectral index. */
typedef struct {
    int64_t npix;
    const double *dirs;   /* [npix][3] */
    const double *t230;   /* [npix] */
    const double *beta;   /* [npix] */
} fg21_sky;

/* Observation: channels, LST bins and the chromatic beam of eq. simantenna.
 * The beam is D = 2(p_f + 1) max(0, z_t . v)^p_f, zero below the horizon, which
 * integrates to 4 pi over the sphere (a directivity). */
typedef struct {
    int32_t F;               /* channels */
    const double *nu;        /* [F] MHz, > 0 */
    double nu0;              /* reference frequency of the template, MHz (230 in the paper, Sec. 2.1) */
    int32_t T;               /* LST bins */
    const double *zenith;    /* [T][3] unit zenith vectors */
    const double *beam_p;    /* [F] beam exponent p(nu) >= 0 */
    double t_cmb;            /* K */
} fg21_obs;

typedef struct {
    int32_t n_regions;       /* N >= 1 */
    int32_t scheme;          /* FG21_SCHEME_* */
    int32_t weighting;       /* FG21_WEIGHT_* */
} fg21_partition_opts;

/* Amplitude regions of the joint model (Sec. 2.2: masks M_alpha,i with one
 * scale factor alpha_i each, besides the spectral-index masks M_beta,j).  The
 * paper leaves their construction open, noting that the partition Algorithms
 * apply to them unchanged; here they partition a per-pixel `field` chosen by
 * the caller (e.g. ln T230, so that regions of similar template brightness
 * share one gain) with the same schemes, conventions and importance
 * weightings as the spectral-index regions (field values in place of beta). */
typedef struct {
    int32_t n_regions;       /* N_alpha >= 1 */
    int32_t scheme;          /* FG21_SCHEME_* */
    int32_t weighting;       /* FG21_WEIGHT_* */
    const double *field;     /* [npix] finite values to partition */
} fg21_amplitude_opts;

/* --------------------------------------------------------------- errors */
/* Message of the calling thread's last failure ("" if none).  The pointer stays
 * valid until the thread's next fg21 call. */
const char *fg21_last_error(void);

/* Number of points the calling thread's last likelihood call marked invalid
 * (non-finite parameter, sigma_n <= 0, sigma21 == 0 or an amplitude scale
 * factor alpha_i <= 0; their logL is -inf). */
int64_t fg21_last_invalid_count(void);

/* Library version string. */
const char *fg21_version(void);

/* Number of CUDA devices visible (0 on a machine without a GPU; never fails). */
int fg21_device_count(void);

/* ---------------------------------------------------------------- build */
/* Partition the sky into nested regions by importance-weighted spectral index
 * and precompute the chromatic response functions, for one observation.
 *   Sec. 4.2 (importance maps, eq. w_beam_dynamic; CDF eq. weighted_cdf),
 *   Sec. 4.3 (Algorithms 1 and 2), Sec. 2.2 (eq. chromatic_function):
 *     w[pix]   = (1/(F T)) sum_{f,t} W(pix,f,t),  W = num / sum_pix num
 *     A[i,f,t] = (1/Npix) sum_{pix in region i} (T230 - T_CMB) D(pix,f,t)
 *     B[f,t]   = (1/Npix) sum_pix D(pix,f,t)       (multiplies T_CMB)
 * Regions are (edge_i, edge_{i+1}], the lowest closed below, in ascending
 * beta; labels are assigned by comparing beta with the edges.  Empty regions
 * are allowed (their A rows are zero) and counted by fg21_model_info.
 * On success *out is a new model owned by the caller (fg21_model_destroy);
 * its data vector is zero until fg21_model_set_data.  labels_out [npix] and
 * edges_out [N+1] are optional (may be NULL).  The library copies what it
 * needs; inputs may be freed on return.
 * Errors: FG21_E_ARG (NULL input, N < 1 or N > npix or N > FG21_MAX_REGIONS,
 * F, T, npix <= 0, nu <= 0, beam_p < 0, |v| or |z| not within 1e-6 of 1,
 * unknown scheme/weighting), FG21_E_NOMEM, FG21_E_CUDA. */
int fg21_build_regions(const fg21_sky *sky, const fg21_obs *obs, const fg21_partition_opts *opt,
                       fg21_model **out, int32_t *labels_out, double *edges_out);

/* The host half of fg21_build_regions without any device work: the same
 * partition and precompute, written to caller buffers labels_out [npix],
 * edges_out [N+1], A_out [N][F][T], B_out [F][T] (each may be NULL).  For
 * machines without a GPU and for checking the host logic. */
int fg21_build_regions_host(const fg21_sky *sky, const fg21_obs *obs, const fg21_partition_opts *opt,
                            int32_t *labels_out, double *edges_out, double *A_out, double *B_out);

/* The joint amplitude / spectral-index model (Sec. 2.2, eqs. forward_model,
 * chromatic_function, fast_forward_model):
 *   K[i,j,f,t] = (1/Npix) sum_pix M_alpha,i M_beta,j (T230 - T_CMB) D(pix,f,t)
 *   M[p,f,t]   = sum_i sum_j alpha_{p,i} K[i,j,f,t] (nu_f/nu0)^-beta_{p,j} + T_CMB B[f,t] + T21
 * Spectral-index regions as fg21_build_regions with beta_opt; amplitude
 * regions partition alpha_opt->field with alpha_opt's scheme and weighting.
 * The model's components are the Na x Nb intersections, component c = i Nb + j
 * (its A row is K[i,j]; fg21_model_get_arrays returns K flattened that way and
 * fg21_model_info reports N = Na Nb); its parameter rows are
 * [beta_1..beta_Nb, alpha_1..alpha_Na, A21, nu21, sigma21, sigma_n].  Every
 * likelihood call accepts it (tensor-core precisions need Na Nb <=
 * FG21_MAX_REGIONS_TC).  A point with an alpha_i <= 0 is invalid (logL =
 * -inf, counted): the scale factors are gains.  Optional outputs:
 * beta_labels [npix], beta_edges [Nb+1], alpha_labels [npix], alpha_edges
 * [Na+1].  Errors: as fg21_build_regions, plus FG21_E_ARG for a NULL or
 * non-finite field, Na < 1, Na > npix or Na Nb > FG21_MAX_REGIONS. */
int fg21_build_regions_ab(const fg21_sky *sky, const fg21_obs *obs, const fg21_partition_opts *beta_opt,
                          const fg21_amplitude_opts *alpha_opt, fg21_model **out, int32_t *beta_labels,
                          double *beta_edges, int32_t *alpha_labels, double *alpha_edges);

/* The host half of fg21_build_regions_ab (no device work): labels, edges,
 * K_out [Na][Nb][F][T] and B_out [F][T] to caller buffers (each may be NULL). */
int fg21_build_regions_ab_host(const fg21_sky *sky, const fg21_obs *obs, const fg21_partition_opts *beta_opt,
                               const fg21_amplitude_opts *alpha_opt, int32_t *beta_labels, double *beta_edges,
                               int32_t *alpha_labels, double *alpha_edges, double *K_out, double *B_out);

/* Parameter layout of a model: spectral-index regions, amplitude parameters
 * (0 for models of fg21_build_regions) and values per parameter row
 * (n_beta + n_alpha + 4).  Any output may be NULL. */
int fg21_model_shape(const fg21_model *m, int32_t *n_beta, int32_t *n_alpha, int32_t *n_params);

/* Release a model and its device memory (NULL is allowed). */
int fg21_model_destroy(fg21_model *m);

/* Replace the model's data vector D(nu_f, t_l) (eq. likelihood), [F][T] host
 * FP64, copied to the device; e.g. a signal-free validation set (Sec. 5.2.1). */
int fg21_model_set_data(fg21_model *m, const double *data);

/* Copy the model's FP64 arrays to host memory: A [N][F][T], B [F][T]
 * (either may be NULL).  For parity checks against an independent oracle. */
int fg21_model_get_arrays(const fg21_model *m, double *A, double *B);

/* Sizes of a model; any output pointer may be NULL.  device_bytes counts the
 * model's resident device memory (A, B, data and tables; the bytes the
 * serving loop budgets for a run); the per-call workspace comes on top. */
int fg21_model_info(const fg21_model *m, int32_t *N, int32_t *F, int32_t *T, int32_t *n_empty,
                    size_t *device_bytes);

/* Simulated antenna temperature of eq. simantenna (Sec. 2.1), per pixel with the
 * sky's own spectral index:
 *   data[f,t] = (1/Npix) sum_pix D(pix,f,t) T_sky(pix,f) + T21(nu_f; t21)
 *               + sigma_noise * noise[f,t]
 * with T_sky of eq. skyapproximation and T21 of eq. t21model.  t21 = {A21, nu21,
 * sigma21}; noise [F][T] standard-normal draws or NULL (noise-free).
 * data_out [F][T] is written.  Host FP64 computation; no device needed. */
int fg21_simulate_data(const fg21_sky *sky, const fg21_obs *obs, const double *t21,
                       double sigma_noise, const double *noise, double *data_out);

/* ----------------------------------------------------------- likelihood */
/* Batched Gaussian log-likelihood of the fast forward model (Sec. 2.2 eq.
 * fast_forward_model plus the trough of eq. t21model; Sec. 2.3.1 eq.
 * likelihood):
 *   M[p,f,t] = sum_i A[i,f,t] (nu_f/nu0)^-beta_{p,i} + T_CMB B[f,t] + T21(nu_f; theta_p)
 *   logL[p]  = -1/2 sum_{f,t} [ ln(2 pi sigma_n^2) + (D[f,t] - M[p,f,t])^2 / sigma_n^2 ]
 * params [P][N+4] and logL [P] are HOST buffers; the call copies params to the
 * device, evaluates on `stream`, copies logL back and returns when done.
 * Buffers in page-locked memory (cudaMallocHost, cudaHostAlloc,
 * cudaHostRegister) are copied by DMA directly; pageable ones pass through a
 * page-locked staging buffer the model keeps.  When a call repeats the previous
 * call's P and precision, the model captures the evaluation as a CUDA graph and
 * replays it on later calls of that size (one graph kept per model; the
 * results are the same bit for bit as the direct launches).
 * precision: FG21_PREC_*.  Points with a non-finite parameter, sigma_n <= 0 or
 * sigma21 == 0 get logL = -inf and are counted (fg21_last_invalid_count); the
 * call still succeeds.  Prior bounds are not enforced.  P = 0 is a no-op.
 * Errors: FG21_E_ARG, FG21_E_RANGE (N above the precision's limit),
 * FG21_E_NOMEM, FG21_E_CUDA, FG21_E_DEVICE. */
int fg21_loglike_batch(fg21_model *m, const double *params, int64_t P, double *logL,
                       int precision, void *stream);

/* As fg21_loglike_batch with DEVICE buffers d_params [P][N+4] and d_logL [P],
 * enqueued asynchronously on `stream` (nothing is copied to or from the host;
 * the call returns before the kernels finish).  The model's workspace is
 * reused by the next call on the same model, which must be ordered after this
 * one (same stream, or synchronised).  The device-side invalid count and any
 * kernel failure are read by fg21_model_sync_status. */
int fg21_loglike_batch_device(fg21_model *m, const double *d_params, int64_t P, double *d_logL,
                              int precision, void *stream);

/* Size of the scratch array of fg21_loglike_batch_device_noalloc (per GPU). */
#define FG21_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The paper has no counterpart to this call.  It serves callers that cannot
 * allocate GPU memory while they evaluate the likelihood: a host application
 * that gives the library a fixed device-memory budget at start-up and forbids
 * growth afterwards, or a runtime that owns the GPU's memory pool and refuses
 * allocations from plug-ins once it is running.  Same arguments and results as
 * fg21_loglike_batch_device, for the tensor-core precisions (FG21_PREC_FP16X3,
 * FG21_PREC_BF16X3), but it calls no cudaMalloc / cudaFree and allocates
 * nothing: all per-call scratch, the request descriptor included, comes from
 * one static device array of FG21_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU
 * which loads the library keeps until the process exits.  The model itself
 * must already exist (fg21_build_regions allocates it); the call takes the
 * model's lock and makes the model's device current, as the regular calls do.
 * A request whose scratch would not fit returns FG21_E_RANGE (the limit is
 * about 73,000 points at N = 24, F = 301, T = 100; split larger batches).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture on that device.  All calls share the array and
 * leave its contents behind (the status word is cleared at the start of each
 * call, everything else is rewritten): calls that overlap on the GPU race, so
 * order them, e.g. on one stream.  Invalid points get logL = -inf as in the
 * other calls; the invalid count is not reported by this call, and a kernel's
 * internal failure (a bounded wait that ran out) shows as logL = NaN for every
 * point of the call. */
int fg21_loglike_batch_device_noalloc(fg21_model *m, const double *d_params, int64_t P, double *d_logL,
                                      int precision, void *stream);

/* Wait for the model's outstanding work on `stream`, then report the invalid
 * count of its last device call (may be NULL) and FG21_E_DEVICE if a kernel
 * reported an internal failure (the logL of that call are then NaN). */
int fg21_model_sync_status(fg21_model *m, void *stream, int64_t *invalid_count);

/* The paper has no counterpart to this call: it checks the library's failure
 * detection without a GPU fault.  Every wait inside the tensor-core
 * likelihood kernel is bounded (4 s); when a wait runs out the kernel sets a
 * bit of its device status word, tells its other warps to stop, and returns,
 * and the next status read reports FG21_E_DEVICE.  This call runs one block of
 * four warps whose waits use that same primitive on barriers that nothing
 * ever completes, on `stream`, and waits for it (about 4 s): warp 0 times out
 * with the kernel's limit, and warps 1-3, whose own limit is twice as long,
 * must stop through the abort signal.  Outputs: *status_word = the device
 * status word (bit 0 set when warp 0 timed out); elapsed_s[4] = the seconds
 * each warp waited, from the GPU's global timer (negative if its barrier
 * unexpectedly completed).  Returns FG21_E_DEVICE when the status word is
 * non-zero (the expected outcome, the same code a stalled likelihood launch
 * gives), FG21_OK when no wait expired, FG21_E_ARG for a NULL output,
 * FG21_E_CUDA or FG21_E_NOMEM on a CUDA failure.  The CUDA context stays usable. */
int fg21_selftest_bounded_wait(uint32_t *status_word, double *elapsed_s, void *stream);

/* The paper has no counterpart to this call: it exposes the tensor cores'
 * accumulation, which the library's split-precision likelihood relies on.  It
 * issues one tcgen05.mma exactly as the likelihood kernel does (kind::f16,
 * FP16 operands, FP32 accumulator, M = 128, N = 16, K = 16, A in tensor memory,
 * B in shared memory) and returns d = c + a b: a [128][16] row-major and b
 * [16][16] stored as b[n][k], both FP16 bit patterns; c and d [128][16] FP32;
 * all four in HOST memory, owned by the caller (the call allocates and frees
 * its own device copies and waits for the result on `stream`).  On the parts
 * this library targets the result follows one rule: the accumulator and the 16
 * products are aligned to the largest exponent E (exponent sums for products),
 * each is truncated toward zero at 2^(E-25), they are added exactly, and the
 * sum is truncated toward zero to FP32; the likelihood's reduction adds back the
 * expected half-ulp that the last such truncation removes.  FG21_E_ARG for a
 * NULL pointer, FG21_E_NOMEM, FG21_E_CUDA, FG21_E_DEVICE if the MMA did not
 * complete within the bounded wait. */
int fg21_selftest_mma_rounding(const uint16_t *a, const uint16_t *b, const float *c, float *d, void *stream);

/* Measured choice of the work split of requests of P points of model m at
 * `precision` (the number of channels per work item of the batched
 * evaluation of eq. likelihood over eq. fast_forward_model): runs one
 * evaluation per candidate split (every distinct channels-per-item value that
 * cuts the F channels into 1..32 groups) five times on the caller's DEVICE
 * buffers d_params [P][N+4] / d_logL [P] (d_logL is overwritten with valid
 * results), times the last four with CUDA events on `stream`, keeps the split
 * with the smallest median in the model and returns it (and its time in ms).
 * Every later plan of model m at `precision` for the same number of 128-point
 * tiles (alone, batched, served or captured in a graph) uses it, so a
 * request's results still depend only on its own model and size.  Blocks
 * until the timings are done.  Errors as fg21_loglike_batch_device. */
int fg21_autotune(fg21_model *m, const double *d_params, int64_t P, double *d_logL, int precision, void *stream,
                  int32_t *best_cpg, double *best_ms);

/* Kernel timing of a model's calls: with enable != 0 (which also clears the
 * record), every later likelihood call on m records CUDA events on its launch
 * stream around the per-request preparation (a1), the main likelihood kernel
 * (a2-a5) and the reduction (a6), for up to the last 8192 calls.
 * fg21_model_timing_totals waits for the last recorded call and returns the
 * number of calls recorded and the summed durations in milliseconds (any
 * pointer may be NULL); FG21_E_STATE if timing is off or nothing was recorded. */
int fg21_model_timing(fg21_model *m, int enable);
int fg21_model_timing_totals(fg21_model *m, int64_t *calls, double *prep_ms, double *main_ms, double *reduce_ms);

/* Model temperatures for a batch (the quantity compared per channel against
 * the oracle): T_model[p][f][t] = M[p,f,t] above, written to HOST memory,
 * evaluated with the same arithmetic as `precision` uses inside the likelihood
 * (the reference-subtracted forms return D - r with r their residual).
 * Meant for validation at small P (P*F*T*8 bytes of output). */
int fg21_model_eval(fg21_model *m, const double *params, int64_t P, double *T_model,
                    int precision, void *stream);

/* Uneven batch: several models (different N, T, P and data) evaluated in ONE
 * persistent kernel launch.  params[k] [P[k]][N_k+4] and logL[k] [P[k]] are host
 * buffers.  precision as above (FP16X3 or BF16X3 run as one tensor-core launch;
 * the SIMT precisions run per model).  Same invalid-point rules. */
int fg21_loglike_multi(fg21_model *const *models, const double *const *params, const int64_t *P,
                       double *const *logL, int n_models, int precision, void *stream);

/* CUDA-graph evaluation of a fixed batch (eq. likelihood, Sec. 2.3.1, over
 * eq. fast_forward_model, Sec. 2.2, for the points a nested sampler proposes,
 * Sec. 3).  fg21_graph_create_multi plans the batch of n_models requests
 * (model k, P[k] points, DEVICE buffers d_params[k] [P[k]][N_k+4] and
 * d_logL[k] [P[k]] on the current device), sizes a workspace owned by the
 * graph, uploads the request descriptors and captures one evaluation (status
 * clear, prep, tensor-core or SIMT kernel, reduction) into a CUDA graph.
 * fg21_graph_launch replays it on `stream`; each replay reads the parameter
 * buffers as they are when it runs and writes the logL buffers, with the same
 * arithmetic (and the same results, bit for bit) as fg21_loglike_multi /
 * fg21_loglike_batch_device on that batch.  The models and the buffers must
 * outlive the graph; replays of one graph must be ordered (one stream, or
 * events) since they share its workspace.  fg21_graph_sync_status waits for
 * `stream` and returns the status and invalid-point count of the last replay.
 * Errors: FG21_E_ARG (bad arguments, wrong device, no points), FG21_E_RANGE
 * (N above the tensor-core limit for FP16X3 / BF16X3), FG21_E_NOMEM,
 * FG21_E_CUDA (capture failed); FG21_E_DEVICE from sync_status as for the
 * other calls. */
int fg21_graph_create(fg21_model *m, const double *d_params, int64_t P, double *d_logL, int precision,
                      fg21_graph **out);
int fg21_graph_create_multi(fg21_model *const *models, const double *const *d_params, const int64_t *P,
                            double *const *d_logL, int n_models, int precision, fg21_graph **out);
int fg21_graph_launch(fg21_graph *g, void *stream);
int fg21_graph_sync_status(fg21_graph *g, void *stream, int64_t *invalid_count);
int fg21_graph_destroy(fg21_graph *g);

/* ------------------------------------------------- accuracy criterion (q_i) */
/* The likelihood distribution of the accuracy criterion (Sec. 5.2.2): K
 * realisations of data that the model describes perfectly up to uncorrelated
 * Gaussian noise of amplitude sigma_noise, evaluated with eq. likelihood at
 * noise level sigma_n over n_cells = F*T cells.  The residual D - M of
 * realisation k is the noise itself, so
 *   L_noise[k] = -1/2 sum_cells [ ln(2 pi sigma_n^2) + (sigma_noise z[k,cell])^2 / sigma_n^2 ]
 * with standard-normal z from Philox4x32-10 (Salmon et al. 2011): cell pair
 * (2j, 2j+1) of realisation k uses counter (j, k mod 2^32, k / 2^32, 0), key
 * (seed mod 2^32, seed / 2^32), uniforms u = (x + 1) / 2^32 of the first two
 * output words and the Box-Muller transform (z_2j = sqrt(-2 ln u1) cos 2 pi u2,
 * z_2j+1 = sqrt(-2 ln u1) sin 2 pi u2).  d_L_noise [K] is DEVICE memory,
 * written asynchronously on `stream`; results are reproducible bit for bit.
 * Errors: FG21_E_ARG (n_cells < 1, K < 0, sigma_n <= 0, sigma_noise < 0),
 * FG21_E_RANGE (K >= 2^31 or n_cells >= 2^33), FG21_E_CUDA. */
int fg21_noise_loglike(int64_t n_cells, double sigma_noise, double sigma_n, int64_t K, uint64_t seed,
                       double *d_L_noise, void *stream);

/* q_i = P(L_noise <= L_bar_i), the lower-tail probability of each fitted
 * likelihood L_bar_i (HOST [n_bar]) under the K values of d_L_noise (DEVICE):
 * the fraction counted on the device, written to q (HOST [n_bar]); the call
 * waits for `stream`.  A fit is consistent with noise when q_i >= 0.01 (the
 * paper's threshold). */
int fg21_noise_q(const double *d_L_noise, int64_t K, const double *L_bar, int64_t n_bar, double *q, void *stream);

/* ---------------------------------------------------------------- serving */
/* Continuous-batching likelihood server for many concurrent nested-sampling
 * runs (Sec. 3: batched replacement of live points, many independent runs).
 * Runs are registered with a model (device-resident A, B, data), admitted
 * while their resident bytes fit `mem_budget_bytes`, and submit requests of P
 * points; a batcher thread packs pending requests into persistent launches
 * on up to `max_inflight` streams, so new requests are admitted while earlier
 * batches run.  Each request's result is independent of what it was batched
 * with (per-request reference, fixed-order reductions). */
typedef struct {
    size_t mem_budget_bytes;   /* admission budget over registered runs' resident bytes */
    int64_t max_batch_points;  /* points per launch (>= the largest single request) */
    int32_t max_wait_us;       /* how long the batcher may wait to fill a launch while earlier launches
                                  are still running; with every slot idle, pending work goes at once */
    int32_t max_inflight;      /* launches in flight (1..8) */
    int32_t precision;         /* FG21_PREC_FP16X3 or FG21_PREC_BF16X3 */
    int32_t device;            /* CUDA device ordinal */
} fg21_serve_opts;

typedef struct {
    double p50_ms, p99_ms, mean_ms;   /* submit -> completion latency of finished requests */
    double evals_per_s;               /* points evaluated / wall time since create */
    double macs_per_s;                /* algorithmic N*F*T multiply-adds per second */
    int64_t requests_done, points_done, launches;
    int64_t queue_depth;              /* requests waiting for a launch */
    size_t admitted_bytes;            /* resident bytes of admitted runs */
    int32_t runs_admitted, runs_waiting;
} fg21_stats;

typedef int64_t fg21_ticket;

int fg21_serve_create(const fg21_serve_opts *opts, fg21_server **out);
/* Stop the batcher after in-flight launches finish; pending tickets complete
 * with FG21_E_CANCELLED.  NULL is allowed. */
int fg21_serve_destroy(fg21_server *s);
/* Register a run that evaluates against `m` (not owned; must outlive the run).
 * Returns FG21_OK if admitted now, FG21_E_BUSY if queued for admission (it is
 * admitted in order once budget frees up; submits to it wait for admission).
 * A run whose bytes exceed the whole budget is rejected with FG21_E_RANGE. */
int fg21_serve_register_run(fg21_server *s, fg21_model *m, int32_t *run_id);
/* Remove a run; its pending requests complete with FG21_E_CANCELLED. */
int fg21_serve_unregister_run(fg21_server *s, int32_t run_id);
/* Queue P points (params copied now).  logL_out [P] must stay valid until the
 * ticket completes or is cancelled. */
int fg21_serve_submit(fg21_server *s, int32_t run_id, const double *params, int64_t P,
                      double *logL_out, fg21_ticket *ticket);
/* Wait up to timeout_ms (< 0: no limit) for a ticket; returns the request's
 * status (FG21_OK, FG21_E_CANCELLED, FG21_E_DEVICE ...) or FG21_E_TIMEOUT.
 * A completed ticket is released by the first wait/poll that reports it. */
int fg21_serve_wait(fg21_server *s, fg21_ticket t, int32_t timeout_ms);
/* Non-blocking: FG21_E_BUSY while pending, else as fg21_serve_wait. */
int fg21_serve_poll(fg21_server *s, fg21_ticket t);
/* Cancel a pending ticket (no effect once its launch started). */
int fg21_serve_cancel(fg21_server *s, fg21_ticket t);
int fg21_serve_stats(fg21_server *s, fg21_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* FG21_H */
