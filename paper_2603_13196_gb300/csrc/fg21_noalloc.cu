// fg21_loglike_batch_device_noalloc: the device-buffer likelihood call for
// callers that must not allocate GPU memory during a call.
//
// Some callers cannot call cudaMalloc at the point where they evaluate the
// likelihood: a host application that hands the library a fixed device-memory
// budget at start-up and forbids growth afterwards, or a runtime that owns the
// GPU's memory pool and rejects allocations from plug-ins once it is running.
// The regular entry points grow a per-model workspace with cudaMalloc on
// first use; this one instead takes all of its per-call scratch (request
// statistics, reference data, operand tiles, point operands, partial sums, the
// request descriptor and the status word) from one file-scope device array of
// FG21_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
// until the process exits.  It runs the same kernels (prep, tensor-core
// likelihood, reduction) as fg21_loglike_batch_device.
//
// The request descriptor reaches the array through the arguments of a
// one-thread kernel (kernel arguments are copied when the launch is enqueued),
// so no host buffer has to outlive the call.
//
// Every call shares the array and leaves its contents behind: the status word
// and invalid counter are cleared at the start of each call, everything else
// is fully rewritten.  Calls that overlap on the GPU (two streams, or two host
// threads) race on the array; callers must order them.  If a kernel reports an
// internal failure (a bounded wait that ran out), the reduction writes NaN to
// every logL of the call instead of a value built from stale partial sums.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "fg21_internal.h"
#include "fg21_model.h"

namespace fg21 {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FG21_NOALLOC_SCRATCH_BYTES];

// Device address of the array, looked up once per device with that device
// current (host code may not use the symbol's name as a device address).
std::mutex g_na_mu;
std::vector<void *> g_na_ptr;

int noalloc_base(int device, char **base) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if ((int)g_na_ptr.size() <= device) g_na_ptr.resize(device + 1, nullptr);
    if (!g_na_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(FG21_E_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
        }
        g_na_ptr[device] = p;
    }
    *base = static_cast<char *>(g_na_ptr[device]);
    return FG21_OK;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Stores the request descriptor, passed by value, into the scratch array.
static_assert(sizeof(ReqDesc) <= 4096, "the request descriptor travels as a kernel argument");
__global__ void store_desc_kernel(const ReqDesc r, ReqDesc *dst) { *dst = r; }

}  // namespace
}  // namespace fg21

using namespace fg21;

extern "C" int fg21_loglike_batch_device_noalloc(fg21_model *m, const double *d_params, int64_t P,
                                                 double *d_logL, int precision, void *stream) {
    if (!m) return set_error(FG21_E_ARG, "NULL model");
    if (P < 0 || (P > 0 && (!d_params || !d_logL))) return set_error(FG21_E_ARG, "bad params/logL/P");
    if (precision != FG21_PREC_FP16X3 && precision != FG21_PREC_BF16X3)
        return set_error(FG21_E_ARG, "the no-allocation call runs the tensor-core forms (FP16X3 / BF16X3)");
    if (m->N > FG21_MAX_REGIONS_TC) return set_error(FG21_E_RANGE, "N = %d above the tensor-core limit", m->N);
    if (P == 0) return FG21_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // the model's lock keeps its device arrays fixed while the request reads
    // them; the model's device is made current, as the regular calls do
    std::lock_guard<std::mutex> lk(m->mu);
    const int dev = m->device;
    int cur = -1;
    FG21_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != dev) FG21_CUDA_TRY(cudaSetDevice(dev));
    char *base = nullptr;
    int rc = noalloc_base(dev, &base);
    if (rc) return rc;

    // plan and lay out exactly as the regular call does, then carve the array
    ReqDesc r = model_request(m, d_params, P, d_logL, precision);
    plan_request(r, precision, num_sms_of(dev), (P + TILE_M - 1) / TILE_M);
    const ReqLayout L = request_layout(r, precision);
    const size_t head = a256(status_bytes(1)) + a256(sizeof(ReqDesc));      // status block + descriptor
    const size_t need = head + (L.total() - L.tiles) + a256(L.tiles);
    if (need > FG21_NOALLOC_SCRATCH_BYTES)
        return set_error(FG21_E_RANGE,
                         "request needs %zu scratch bytes, above the %zu-byte limit of the no-allocation call "
                         "(fewer points per call)",
                         need, (size_t)FG21_NOALLOC_SCRATCH_BYTES);
    unsigned *status = reinterpret_cast<unsigned *>(base);
    ReqDesc *d_req = reinterpret_cast<ReqDesc *>(base + a256(status_bytes(1)));
    char *p = base + head;
    r.stat_part = (float *)p; p += L.stat_part;
    r.beta_bar = (double *)p; p += L.beta_bar;
    r.req_stats = (double *)p; p += L.req_stats;
    r.nL32 = (float *)p; p += L.nL32;
    r.nu32 = (float *)p; p += L.nu32;
    r.coef2 = (unsigned long long *)p; p += L.coef2;
    r.scaleB = (int *)p; p += L.scaleB;
    r.scaleW = (int *)p; p += L.scaleW;
    r.Bp32 = nullptr; p += L.Bp32;
    r.dref32 = nullptr; p += L.dref32;
    r.partials = (float2 *)p; p += L.partials;
    r.pvalid = (unsigned char *)p; p += L.pvalid;
    r.pnorm = (double2 *)p; p += L.pnorm;
    r.pts32 = (float *)p; p += L.pts32;
    char *arena = p;
    r.item_begin = 0;
    r.pt_begin = 0;
    r.tile_row0 = 0;
    r.tiles = arena;
    r.status = status;
    r.invalid = reinterpret_cast<unsigned long long *>(base + 16);

    // the status word and invalid counter start at zero; the rest is rewritten
    FG21_CUDA_TRY(cudaMemsetAsync(status, 0, status_bytes(1), s));
    store_desc_kernel<<<1, 1, 0, s>>>(r, d_req);
    FG21_CUDA_TRY(cudaGetLastError());
    FG21_CUDA_TRY(launch_prep(&r, d_req, 1, precision, r.n_stat_blocks, r.F * r.n_tchunks, r.n_tiles, s));
    TcLaunch T;
    T.d_reqs = d_req;
    T.n_reqs = 1;
    T.n_items = (int64_t)r.n_tiles * r.G;
    T.kp_max = r.Kp;
    T.tc_pad_max = r.Tc_pad;
    T.precision = precision;
    T.box_rows = tc_box_rows(&r.tile_rows, 1);
    T.arena = arena;
    T.arena_rows = (int64_t)(L.tiles / 128);
    T.status = status;
    T.lean = r.Na != 0 ? 0 : r.Kp == tc_launch_kp(r.Kp) ? 1 : 2;
    cudaError_t e = launch_tc(T, num_sms_of(dev), s);
    if (e != cudaSuccess) return cuda_error(e, "tensor-core likelihood launch");
    FG21_CUDA_TRY(launch_reduce(&r, d_req, 1, s));
    return FG21_OK;
}
