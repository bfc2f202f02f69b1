// Model handles, device workspaces, shape planning and the likelihood entry
// points of fg21.h.  Every likelihood is evaluated by the kernels in
// fg21_kernels.cu (prep, SIMT, reduce) and fg21_tc.cu (tensor cores).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "fg21_internal.h"
#include "fg21_model.h"

namespace fg21 {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static int round16(int x) { return (x + 15) & ~15; }

int num_sms_of(int device) {
    static std::mutex mu;
    static std::vector<int> cache;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= device) cache.resize(device + 1, 0);
    if (!cache[device]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            cudaGetLastError();
            n = 1;
        }
        cache[device] = n;
    }
    return cache[device];
}

// ------------------------------------------------------------- workspace
int Workspace::ensure(size_t dev_need, size_t arena_need, size_t pinned_need, int n_reqs) {
    if (device < 0) FG21_CUDA_TRY(cudaGetDevice(&device));
    if (!done) FG21_CUDA_TRY(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    // staging and scratch may still be in use by the previous call on this workspace
    FG21_CUDA_TRY(cudaEventSynchronize(done));
    if (!d_status) {
        void *p = nullptr;
        FG21_CUDA_TRY(cudaMalloc(&p, 256));
        d_status = (unsigned *)p;
        d_invalid = (unsigned long long *)((char *)p + 16);
    }
    if (dev_need > dev_bytes) {
        if (dev) cudaFree(dev);
        dev = nullptr;
        dev_bytes = 0;
        size_t want = std::max(dev_need, dev_need + dev_need / 4);
        if (cudaMalloc((void **)&dev, want) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FG21_E_NOMEM, "cudaMalloc of %zu workspace bytes failed", want);
        }
        dev_bytes = want;
    }
    if (arena_need > arena_bytes) {
        if (arena) cudaFree(arena);
        arena = nullptr;
        arena_bytes = 0;
        size_t want = std::max(arena_need, arena_need + arena_need / 4);
        if (cudaMalloc((void **)&arena, want) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FG21_E_NOMEM, "cudaMalloc of %zu operand-tile bytes failed", want);
        }
        arena_bytes = want;
    }
    if (pinned_need > pinned_bytes) {
        if (pinned) cudaFreeHost(pinned);
        pinned = nullptr;
        pinned_bytes = 0;
        size_t want = std::max(pinned_need, (size_t)4096);
        if (cudaMallocHost((void **)&pinned, want) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FG21_E_NOMEM, "cudaMallocHost of %zu bytes failed", want);
        }
        pinned_bytes = want;
    }
    if (n_reqs > reqs_cap) {
        if (d_reqs) cudaFree(d_reqs);
        d_reqs = nullptr;
        reqs_cap = 0;
        int want = std::max(n_reqs, 8);
        FG21_CUDA_TRY(cudaMalloc((void **)&d_reqs, sizeof(ReqDesc) * want));
        reqs_cap = want;
    }
    return FG21_OK;
}

// The timing events are created when timing is switched on, never inside a
// timed call (creating thousands of events takes milliseconds).
int Workspace::timing_prepare() {
    if (!tev.empty()) return FG21_OK;
    tev.assign((size_t)TIMING_CAP * 4, nullptr);
    for (auto &e : tev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            for (auto &x : tev)
                if (x) cudaEventDestroy(x);
            tev.clear();
            return set_error(FG21_E_CUDA, "cudaEventCreate of the timing events failed");
        }
    return FG21_OK;
}

cudaEvent_t *Workspace::timing_slot() {
    if (!timing || tev.empty()) return nullptr;
    cudaEvent_t *slot = &tev[(size_t)(tcalls % TIMING_CAP) * 4];
    ++tcalls;
    return slot;
}

void Workspace::release() {
    if (done) cudaEventSynchronize(done);
    if (dev) cudaFree(dev);
    if (arena) cudaFree(arena);
    if (pinned) cudaFreeHost(pinned);
    if (d_reqs) cudaFree(d_reqs);
    if (d_status) cudaFree(d_status);
    if (done) cudaEventDestroy(done);
    for (auto &e : tev)
        if (e) cudaEventDestroy(e);
    tev.clear();
    tcalls = 0;
    dev = arena = pinned = nullptr;
    d_reqs = nullptr;
    d_status = nullptr;
    d_invalid = nullptr;
    done = nullptr;
    dev_bytes = arena_bytes = pinned_bytes = 0;
    reqs_cap = 0;
}

// --------------------------------------------------------------- planning
static int g_cpg_override() {
    static int v = [] {
        const char *e = std::getenv("FG21_CHANNELS_PER_GROUP");
        return e ? std::atoi(e) : 0;
    }();
    return v;
}

// Channels per work item: minimise (waves of items over the `slots` items
// the GPU runs at once) x (channels per item + a per-item overhead of about
// one channel), with at most max_groups groups.
static int choose_channels_per_group(int64_t total_tiles, int F, int slots, int max_groups = 1 << 30) {
    if (g_cpg_override() > 0) return std::min(F, g_cpg_override());
    double best = 1e300;
    int best_cpg = F;
    for (int cpg = 1; cpg <= F; ++cpg) {
        int G = (F + cpg - 1) / cpg;
        if (G > max_groups) continue;
        double waves = std::ceil((double)total_tiles * G / slots);
        double cost = waves * (cpg + 1.0);
        if (cost < best - 1e-9) {
            best = cost;
            best_cpg = cpg;
        }
    }
    return best_cpg;
}

void plan_request(ReqDesc &r, int precision, int num_sms, int64_t total_tiles) {
    r.Kp = round16(r.N + 2);
    r.pts_rows = precision == FG21_PREC_FP16X3 || precision == FG21_PREC_BF16X3 ? r.Kp + 4 + (r.Na ? r.Kp : 0) + r.Kp
                                                                             : r.Nb + r.Na;
    // t-chunks of at most TC_MAX columns: the same cap for every K keeps the
    // plan of a request independent of what it is batched with
    r.n_tchunks = (r.T + TC_MAX - 1) / TC_MAX;
    r.Tc = (r.T + r.n_tchunks - 1) / r.n_tchunks;
    r.Tc_pad = round16(r.Tc);
    r.n_tiles = (int)((r.P + TILE_M - 1) / TILE_M);
    r.n_stat_blocks = (int)((r.P + STAT_BLOCK - 1) / STAT_BLOCK);
    const bool tc = precision == FG21_PREC_FP16X3 || precision == FG21_PREC_BF16X3;
    r.simt_tc = tc ? 0 : simt_chunk_width(r.N, r.T);
    int cpg;
    if (r.cpg_hint > 0) {
        cpg = std::min(r.F, r.cpg_hint);
    } else if (tc) {
        cpg = choose_channels_per_group(total_tiles, r.F, num_sms);
    } else {
        // SIMT blocks are not persistent: the waves are counted in the blocks
        // the GPU holds at once (at most 32 groups, the reduction's serial row)
        const int slots = num_sms * simt_blocks_per_sm(r.N, r.simt_tc, precision);
        cpg = choose_channels_per_group(total_tiles, r.F, slots, 32);
    }
    r.G = (r.F + cpg - 1) / cpg;
    r.ch_per_group = (r.F + r.G - 1) / r.G;
    r.n_part = tc ? 2 * r.G : r.G;      // the tensor path splits each point's t-columns over two warps
    r.chi2_scale = tc ? 1.0 + (2.0 / 3.0) * std::ldexp(1.0, -23) : 1.0;
    r.tile_rows = (int64_t)r.Kp * r.Tc_pad / 32;   // 2 splits x Kp x Tc_pad x 2 bytes / 128
}

ReqLayout request_layout(const ReqDesc &r, int precision) {
    ReqLayout L{};
    const bool tc = precision == FG21_PREC_FP16X3 || precision == FG21_PREC_BF16X3;
    L.stat_part = align256(sizeof(float) * (size_t)r.n_stat_blocks * (2 * r.NPF + 2));
    L.beta_bar = align256(sizeof(double) * r.NPF);
    L.req_stats = align256(sizeof(double) * 4);
    L.nL32 = align256(sizeof(float) * r.F);
    L.nu32 = align256(sizeof(float) * r.F);
    L.coef2 = tc ? align256(sizeof(unsigned long long) * 8 * (size_t)r.F) : 0;
    L.scaleB = align256(sizeof(int) * (size_t)r.F * r.n_tchunks);
    L.scaleW = align256(sizeof(int));
    const bool delta = precision == FG21_PREC_FP32_DELTA;
    L.Bp32 = delta ? align256(sizeof(float) * (size_t)r.N * r.F * r.T) : 0;
    L.dref32 = delta ? align256(sizeof(float) * (size_t)r.F * r.T) : 0;
    L.partials = align256(sizeof(float2) * (size_t)r.P * r.n_part);
    L.pvalid = align256((size_t)r.P);
    L.pnorm = tc ? align256(sizeof(double2) * (size_t)r.P) : 0;
    L.pts32 = align256(sizeof(float) * (size_t)r.n_tiles * r.pts_rows * TILE_M);
    L.tiles = tc ? (size_t)r.F * r.n_tchunks * r.tile_rows * 128 : 0;
    return L;
}

int prepare_requests(Workspace &ws, std::vector<ReqDesc> &reqs, int precision, Prepared &pp) {
    const int n = (int)reqs.size();
    pp = Prepared{};
    pp.n = n;
    pp.precision = precision;
    if (n == 0) return FG21_OK;
    const bool tc = precision == FG21_PREC_FP16X3 || precision == FG21_PREC_BF16X3;
    int dev = 0;
    FG21_CUDA_TRY(cudaGetDevice(&dev));
    pp.num_sms = num_sms_of(dev);
    size_t dev_need = 0, arena_need = 0;
    std::vector<ReqLayout> lay(n);
    for (int k = 0; k < n; ++k) {
        // each request is planned as if alone, so its work split (and with it
        // every rounding) does not depend on what it is batched with
        plan_request(reqs[k], precision, pp.num_sms, (reqs[k].P + TILE_M - 1) / TILE_M);
        lay[k] = request_layout(reqs[k], precision);
        arena_need += lay[k].tiles;
        dev_need += lay[k].total() - lay[k].tiles;
    }
    int rc = ws.ensure(dev_need, arena_need, sizeof(ReqDesc) * n, n);
    if (rc) return rc;
    char *p = ws.dev;
    int64_t item = 0, row = 0, pts = 0;
    int kp_max = 16, tc_max = 16;
    pp.max_blocks = pp.max_fchunks = pp.max_tiles = 1;
    for (int k = 0; k < n; ++k) {
        ReqDesc &r = reqs[k];
        const ReqLayout &L = lay[k];
        r.stat_part = (float *)p; p += L.stat_part;
        r.beta_bar = (double *)p; p += L.beta_bar;
        r.req_stats = (double *)p; p += L.req_stats;
        r.nL32 = (float *)p; p += L.nL32;
        r.nu32 = (float *)p; p += L.nu32;
        r.coef2 = L.coef2 ? (unsigned long long *)p : nullptr; p += L.coef2;
        r.scaleB = (int *)p; p += L.scaleB;
        r.scaleW = (int *)p; p += L.scaleW;
        r.Bp32 = L.Bp32 ? (float *)p : nullptr; p += L.Bp32;
        r.dref32 = L.dref32 ? (float *)p : nullptr; p += L.dref32;
        r.partials = (float2 *)p; p += L.partials;
        r.pvalid = (unsigned char *)p; p += L.pvalid;
        r.pnorm = L.pnorm ? (double2 *)p : nullptr; p += L.pnorm;
        r.pts32 = L.pts32 ? (float *)p : nullptr; p += L.pts32;
        r.item_begin = item;
        item += (int64_t)r.n_tiles * r.G;
        r.pt_begin = pts;
        pts += r.P;
        r.tile_row0 = row;
        r.tiles = ws.arena + row * 128;
        row += (int64_t)(L.tiles / 128);
        r.status = ws.d_status;
        r.invalid = ws.d_invalid;
        kp_max = std::max(kp_max, r.Kp);
        tc_max = std::max(tc_max, r.Tc_pad);
        pp.max_blocks = std::max(pp.max_blocks, r.n_stat_blocks);
        pp.max_fchunks = std::max(pp.max_fchunks, r.F * r.n_tchunks);
        pp.max_tiles = std::max(pp.max_tiles, r.n_tiles);
    }
    if (tc && kp_max > KP_MAX)
        return set_error(FG21_E_RANGE, "N = %d regions exceeds the tensor-core limit %d", kp_max - 2,
                         FG21_MAX_REGIONS_TC);
    pp.tc = tc;
    if (tc) {
        TcLaunch &L = pp.tcl;
        L.d_reqs = ws.d_reqs;
        L.n_reqs = n;
        L.n_items = item;
        L.kp_max = kp_max;
        L.tc_pad_max = tc_max;
        L.precision = precision;
        std::vector<int64_t> rows_of(n);
        for (int k = 0; k < n; ++k) rows_of[k] = reqs[k].tile_rows;
        L.box_rows = tc_box_rows(rows_of.data(), n);
        L.arena = ws.arena;
        L.arena_rows = row;
        L.status = ws.d_status;
        bool no_alpha = true, full = true;
        for (int k = 0; k < n; ++k) {
            no_alpha = no_alpha && reqs[k].Na == 0;
            full = full && reqs[k].Kp == tc_launch_kp(kp_max);
        }
        L.lean = !no_alpha ? 0 : full ? 1 : 2;
    }
    std::memcpy(ws.pinned, reqs.data(), sizeof(ReqDesc) * n);
    return FG21_OK;
}

int launch_requests(Workspace &ws, const std::vector<ReqDesc> &reqs, const Prepared &pp, cudaStream_t stream,
                    bool upload, bool timing) {
    const int n = pp.n;
    if (n == 0) return FG21_OK;
    FG21_CUDA_TRY(cudaMemsetAsync(ws.d_status, 0, status_bytes(n), stream));   // status word, invalid counter
    if (upload)
        FG21_CUDA_TRY(cudaMemcpyAsync(ws.d_reqs, ws.pinned, sizeof(ReqDesc) * n, cudaMemcpyHostToDevice, stream));
    cudaEvent_t *ev = timing ? ws.timing_slot() : nullptr;
    if (ev) FG21_CUDA_TRY(cudaEventRecord(ev[0], stream));
    FG21_CUDA_TRY(launch_prep(reqs.data(), ws.d_reqs, n, pp.precision, pp.max_blocks, pp.max_fchunks, pp.max_tiles,
                              stream));
    if (ev) FG21_CUDA_TRY(cudaEventRecord(ev[1], stream));
    if (pp.tc) {
        cudaError_t e = launch_tc(pp.tcl, pp.num_sms, stream);
        if (e != cudaSuccess) return cuda_error(e, "tensor-core likelihood launch");
    } else {
        FG21_CUDA_TRY(launch_simt(reqs.data(), ws.d_reqs, n, pp.precision, stream));
    }
    if (ev) FG21_CUDA_TRY(cudaEventRecord(ev[2], stream));
    FG21_CUDA_TRY(launch_reduce(reqs.data(), ws.d_reqs, n, stream));
    if (ev) FG21_CUDA_TRY(cudaEventRecord(ev[3], stream));
    return FG21_OK;
}

int enqueue_requests(Workspace &ws, std::vector<ReqDesc> &reqs, int precision, cudaStream_t stream) {
    Prepared pp;
    int rc = prepare_requests(ws, reqs, precision, pp);
    if (rc || pp.n == 0) return rc;
    rc = launch_requests(ws, reqs, pp, stream, true, true);
    if (rc) return rc;
    FG21_CUDA_TRY(cudaEventRecord(ws.done, stream));
    return FG21_OK;
}

// ------------------------------------------------------------------ model
// E = D - T_CMB B (FP64) as a double-float pair: hi = (float)E, lo = (float)(E - hi).
// data may be NULL (a zero data vector).
void split_data_term(const fg21_model *m, const double *data, std::vector<float> &hi, std::vector<float> &lo) {
    const size_t FT = (size_t)m->F * m->T;
    hi.resize(FT);
    lo.resize(FT);
    for (size_t k = 0; k < FT; ++k) {
        const double e = (data ? data[k] : 0.0) - m->t_cmb * m->B[k];
        hi[k] = (float)e;
        lo[k] = (float)(e - (double)hi[k]);
    }
}

int model_upload(fg21_model *m) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return set_error(FG21_E_CUDA, "no usable CUDA device");
    }
    m->device = dev;
    const size_t NFT = (size_t)m->N * m->F * m->T, FT = (size_t)m->F * m->T;
    std::vector<double> L(m->F);
    m->Lmax = 0.0;
    for (int f = 0; f < m->F; ++f) {
        L[f] = std::log(m->nu[f] / m->nu0);
        m->Lmax = std::max(m->Lmax, std::fabs(L[f]));
    }
    std::vector<float> A32(NFT), Alo(NFT), B32(FT), zero32(FT, 0.0f), Ehi(FT), Elo(FT);
    for (size_t k = 0; k < NFT; ++k) {
        A32[k] = (float)m->A[k];
        Alo[k] = (float)(m->A[k] - (double)A32[k]);
    }
    for (size_t k = 0; k < FT; ++k) B32[k] = (float)m->B[k];
    split_data_term(m, nullptr, Ehi, Elo);
    struct Item { void **dst; const void *src; size_t bytes; };
    std::vector<double> zero(FT, 0.0);
    Item items[] = {
        {(void **)&m->d_A, m->A.data(), sizeof(double) * NFT},
        {(void **)&m->d_B, m->B.data(), sizeof(double) * FT},
        {(void **)&m->d_data, zero.data(), sizeof(double) * FT},
        {(void **)&m->d_L, L.data(), sizeof(double) * m->F},
        {(void **)&m->d_nu, m->nu.data(), sizeof(double) * m->F},
        {(void **)&m->d_A32, A32.data(), sizeof(float) * NFT},
        {(void **)&m->d_B32, B32.data(), sizeof(float) * FT},
        {(void **)&m->d_data32, zero32.data(), sizeof(float) * FT},
        {(void **)&m->d_Alo, Alo.data(), sizeof(float) * NFT},
        {(void **)&m->d_Ehi, Ehi.data(), sizeof(float) * FT},
        {(void **)&m->d_Elo, Elo.data(), sizeof(float) * FT},
    };
    m->resident_bytes = 0;
    for (auto &it : items) {
        if (cudaMalloc(it.dst, it.bytes) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FG21_E_NOMEM, "cudaMalloc of %zu model bytes failed", it.bytes);
        }
        FG21_CUDA_TRY(cudaMemcpy(*it.dst, it.src, it.bytes, cudaMemcpyHostToDevice));
        m->resident_bytes += it.bytes;
    }
    return FG21_OK;
}

ReqDesc model_request(fg21_model *m, const double *d_params, int64_t P, double *d_logL, int precision) {
    ReqDesc r;
    std::memset(&r, 0, sizeof r);
    {
        std::lock_guard<std::mutex> lk(m->tune_mu);
        const auto it = m->tuned_cpg.find({precision, (int)((P + TILE_M - 1) / TILE_M)});
        r.cpg_hint = it == m->tuned_cpg.end() ? 0 : it->second;
    }
    r.A = m->d_A;
    r.B = m->d_B;
    r.data = m->d_data;
    r.L = m->d_L;
    r.nu = m->d_nu;
    r.A32 = m->d_A32;
    r.B32 = m->d_B32;
    r.data32 = m->d_data32;
    r.A_lo = m->d_Alo;
    r.E_hi = m->d_Ehi;
    r.E_lo = m->d_Elo;
    r.params = d_params;
    r.logL = d_logL;
    r.t_cmb = m->t_cmb;
    r.Lmax = m->Lmax;
    r.P = P;
    r.N = m->N;
    r.Nb = m->n_beta;
    r.Na = m->n_alpha;
    r.NPF = m->n_beta + m->n_alpha;
    r.F = m->F;
    r.T = m->T;
    return r;
}

static int check_precision(const fg21_model *m, int precision) {
    if (precision < 0 || precision > 3) return set_error(FG21_E_ARG, "unknown precision %d", precision);
    if ((precision == FG21_PREC_FP16X3 || precision == FG21_PREC_BF16X3) && m->N > FG21_MAX_REGIONS_TC)
        return set_error(FG21_E_RANGE, "N = %d exceeds the tensor-core limit %d (use FG21_PREC_FP32_DELTA)",
                         m->N, FG21_MAX_REGIONS_TC);
    return FG21_OK;
}

static int device_guard(const fg21_model *m) {
    int cur = -1;
    FG21_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != m->device) FG21_CUDA_TRY(cudaSetDevice(m->device));
    return FG21_OK;
}

// Host-buffer evaluation: params are staged through the model's pinned I/O
// buffers, evaluated on the device, and logL copied back.
// True for host memory the CUDA runtime has page-locked (cudaMallocHost,
// cudaHostAlloc, cudaHostRegister): a DMA can read or write it directly.
static bool host_pinned(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

static int run_host(fg21_model *m, const double *params, int64_t P, double *logL, int precision,
                    cudaStream_t stream) {
    const size_t pbytes = sizeof(double) * (size_t)P * m->n_params(), lbytes = sizeof(double) * (size_t)P;
    const size_t need = align256(pbytes) + align256(lbytes) + 64;
    if (m->io_cap < need) {
        if (m->ws.done) FG21_CUDA_TRY(cudaEventSynchronize(m->ws.done));
        if (m->host_graph) {
            fg21_graph_destroy(m->host_graph);
            m->host_graph = nullptr;
        }
        if (m->io_d) cudaFree(m->io_d);
        if (m->io_h) cudaFreeHost(m->io_h);
        m->io_d = nullptr;
        m->io_h = nullptr;
        m->io_cap = 0;
        if (cudaMalloc((void **)&m->io_d, need) != cudaSuccess ||
            cudaMallocHost((void **)&m->io_h, need) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FG21_E_NOMEM, "I/O buffers of %zu bytes", need);
        }
        m->io_cap = need;
    }
    struct { double *d_params, *d_logL; char *h; } iob{(double *)m->io_d, (double *)(m->io_d + align256(pbytes)), m->io_h};
    auto *io = &iob;
    // caller buffers in page-locked memory are copied from and to directly;
    // pageable ones go through the model's page-locked staging buffer
    const bool pin_in = host_pinned(params), pin_out = host_pinned(logL);
    if (!pin_in) std::memcpy(io->h, params, pbytes);
    FG21_CUDA_TRY(cudaMemcpyAsync(io->d_params, pin_in ? (const void *)params : (const void *)io->h, pbytes,
                                  cudaMemcpyHostToDevice, stream));
    std::vector<ReqDesc> reqs{model_request(m, io->d_params, P, io->d_logL, precision)};
    const unsigned *d_status = nullptr;
    const int cpg = reqs[0].cpg_hint;
    const bool kept = m->host_graph && m->hg_P == P && m->hg_prec == precision && m->hg_cpg == cpg;
    const bool repeat = m->last_P == P && m->last_prec == precision && m->last_cpg == cpg;
    m->last_P = P;
    m->last_prec = precision;
    m->last_cpg = cpg;
    if (!m->ws.timing && (kept || repeat)) {
        // repeated calls of one size replay a graph of the status clear and the
        // kernels on the staging buffers, captured when a size, precision and
        // tuned work split come twice in a row (a size that changes every call
        // never pays for a capture)
        if (!kept) {
            if (m->host_graph) {
                fg21_graph_destroy(m->host_graph);
                m->host_graph = nullptr;
            }
            fg21_graph *g = nullptr;
            int rc = fg21_graph_create(m, io->d_params, P, io->d_logL, precision, &g);
            if (rc) return rc;
            m->host_graph = g;
            m->hg_P = P;
            m->hg_prec = precision;
            m->hg_cpg = cpg;
        }
        int rc = fg21_graph_launch(m->host_graph, stream);
        if (rc) return rc;
        d_status = graph_status(m->host_graph);
    } else {
        // first calls of a size, and timed calls (fg21_model_timing, so that each
        // kernel is bracketed), launch directly
        int rc = enqueue_requests(m->ws, reqs, precision, stream);
        if (rc) return rc;
        d_status = m->ws.d_status;
    }
    char *h_log = io->h + align256(pbytes);
    FG21_CUDA_TRY(cudaMemcpyAsync(pin_out ? (void *)logL : (void *)h_log, io->d_logL, lbytes, cudaMemcpyDeviceToHost,
                                  stream));
    FG21_CUDA_TRY(cudaMemcpyAsync(h_log + align256(lbytes), d_status, 32, cudaMemcpyDeviceToHost, stream));
    FG21_CUDA_TRY(cudaStreamSynchronize(stream));
    if (!pin_out) std::memcpy(logL, h_log, lbytes);
    const unsigned *st = (const unsigned *)(h_log + align256(lbytes));
    unsigned long long inv = 0;
    std::memcpy(&inv, st + 4, sizeof inv);
    set_invalid_count((int64_t)inv);
    if (st[0]) return set_error(FG21_E_DEVICE, "likelihood kernel reported status 0x%x", st[0]);
    return FG21_OK;
}

}  // namespace fg21

using namespace fg21;

extern "C" {

int fg21_model_destroy(fg21_model *m) {
    if (!m) return FG21_OK;
    {
        std::lock_guard<std::mutex> lk(m->mu);
        if (m->host_graph) fg21_graph_destroy(m->host_graph);
        m->host_graph = nullptr;
        m->ws.release();
        void *ptrs[] = {m->d_A, m->d_B, m->d_data, m->d_L, m->d_nu, m->d_A32, m->d_B32, m->d_data32, m->d_Alo,
                        m->d_Ehi, m->d_Elo, m->io_d};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        if (m->io_h) cudaFreeHost(m->io_h);
    }
    delete m;
    return FG21_OK;
}

int fg21_model_set_data(fg21_model *m, const double *data) {
    if (!m || !data) return set_error(FG21_E_ARG, "NULL model/data");
    std::lock_guard<std::mutex> lk(m->mu);
    int rc = device_guard(m);
    if (rc) return rc;
    const size_t FT = (size_t)m->F * m->T;
    std::vector<float> d32(FT);
    for (size_t k = 0; k < FT; ++k) {
        if (!std::isfinite(data[k])) return set_error(FG21_E_ARG, "non-finite data[%zu]", k);
        d32[k] = (float)data[k];
    }
    std::vector<float> ehi, elo;
    split_data_term(m, data, ehi, elo);
    if (m->ws.done) FG21_CUDA_TRY(cudaEventSynchronize(m->ws.done));
    FG21_CUDA_TRY(cudaMemcpy(m->d_data, data, sizeof(double) * FT, cudaMemcpyHostToDevice));
    FG21_CUDA_TRY(cudaMemcpy(m->d_data32, d32.data(), sizeof(float) * FT, cudaMemcpyHostToDevice));
    FG21_CUDA_TRY(cudaMemcpy(m->d_Ehi, ehi.data(), sizeof(float) * FT, cudaMemcpyHostToDevice));
    FG21_CUDA_TRY(cudaMemcpy(m->d_Elo, elo.data(), sizeof(float) * FT, cudaMemcpyHostToDevice));
    return FG21_OK;
}

int fg21_model_get_arrays(const fg21_model *m, double *A, double *B) {
    if (!m) return set_error(FG21_E_ARG, "NULL model");
    if (A) std::memcpy(A, m->A.data(), sizeof(double) * m->A.size());
    if (B) std::memcpy(B, m->B.data(), sizeof(double) * m->B.size());
    return FG21_OK;
}

int fg21_model_info(const fg21_model *m, int32_t *N, int32_t *F, int32_t *T, int32_t *n_empty,
                    size_t *device_bytes) {
    if (!m) return set_error(FG21_E_ARG, "NULL model");
    if (N) *N = m->N;
    if (F) *F = m->F;
    if (T) *T = m->T;
    if (n_empty) *n_empty = m->n_empty;
    if (device_bytes) *device_bytes = m->resident_bytes;
    return FG21_OK;
}

int fg21_model_shape(const fg21_model *m, int32_t *n_beta, int32_t *n_alpha, int32_t *n_params) {
    if (!m) return set_error(FG21_E_ARG, "NULL model");
    if (n_beta) *n_beta = m->n_beta;
    if (n_alpha) *n_alpha = m->n_alpha;
    if (n_params) *n_params = m->n_params();
    return FG21_OK;
}

int fg21_loglike_batch(fg21_model *m, const double *params, int64_t P, double *logL, int precision,
                       void *stream) {
    if (!m) return set_error(FG21_E_ARG, "NULL model");
    if (P < 0 || (P > 0 && (!params || !logL))) return set_error(FG21_E_ARG, "bad params/logL/P");
    int rc = check_precision(m, precision);
    if (rc) return rc;
    set_invalid_count(0);
    if (P == 0) return FG21_OK;
    std::lock_guard<std::mutex> lk(m->mu);
    rc = device_guard(m);
    if (rc) return rc;
    return run_host(m, params, P, logL, precision, (cudaStream_t)stream);
}

int fg21_loglike_batch_device(fg21_model *m, const double *d_params, int64_t P, double *d_logL,
                              int precision, void *stream) {
    if (!m) return set_error(FG21_E_ARG, "NULL model");
    if (P < 0 || (P > 0 && (!d_params || !d_logL))) return set_error(FG21_E_ARG, "bad params/logL/P");
    int rc = check_precision(m, precision);
    if (rc) return rc;
    if (P == 0) return FG21_OK;
    std::lock_guard<std::mutex> lk(m->mu);
    rc = device_guard(m);
    if (rc) return rc;
    std::vector<ReqDesc> reqs{model_request(m, d_params, P, d_logL, precision)};
    return enqueue_requests(m->ws, reqs, precision, (cudaStream_t)stream);
}

int fg21_autotune(fg21_model *m, const double *d_params, int64_t P, double *d_logL, int precision, void *stream,
                  int32_t *best_cpg, double *best_ms) {
    if (!m) return set_error(FG21_E_ARG, "NULL model");
    if (P <= 0 || !d_params || !d_logL) return set_error(FG21_E_ARG, "bad params/logL/P");
    int rc = check_precision(m, precision);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(m->mu);
    rc = device_guard(m);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // candidates: every distinct channels-per-group value that splits the
    // channels into 1..32 groups, plus the planner's model choice
    std::vector<int> cand;
    for (int G = 1; G <= std::min(m->F, 32); ++G) {
        const int cpg = (m->F + G - 1) / G;
        if (std::find(cand.begin(), cand.end(), cpg) == cand.end()) cand.push_back(cpg);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FG21_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_error(cudaGetLastError(), "cudaEventCreate");
    }
    const bool was_timing = m->ws.timing;
    m->ws.timing = false;
    int best = 0;
    double best_t = 1e300;
    for (int cpg : cand) {
        float ms[4];
        for (int rep = 0; rep < 5 && rc == FG21_OK; ++rep) {
            std::vector<ReqDesc> reqs{model_request(m, d_params, P, d_logL, precision)};
            reqs[0].cpg_hint = cpg;
            if (rep > 0 && cudaEventRecord(e0, s) != cudaSuccess) rc = cuda_error(cudaGetLastError(), "event");
            if (rc == FG21_OK) rc = enqueue_requests(m->ws, reqs, precision, s);
            if (rc == FG21_OK && rep > 0) {
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms[rep - 1], e0, e1) != cudaSuccess)
                    rc = cuda_error(cudaGetLastError(), "autotune timing");
            }
        }
        if (rc) break;
        std::sort(ms, ms + 4);
        const double t = 0.5 * (ms[1] + ms[2]);      // median of 4 (one warm-up run discarded)
        if (t < best_t) {
            best_t = t;
            best = cpg;
        }
    }
    m->ws.timing = was_timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> tl(m->tune_mu);
        m->tuned_cpg[{precision, (int)((P + TILE_M - 1) / TILE_M)}] = best;
    }
    if (best_cpg) *best_cpg = best;
    if (best_ms) *best_ms = best_t;
    return FG21_OK;
}

int fg21_model_sync_status(fg21_model *m, void *stream, int64_t *invalid_count) {
    if (!m) return set_error(FG21_E_ARG, "NULL model");
    std::lock_guard<std::mutex> lk(m->mu);
    FG21_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (!m->ws.d_status) {
        if (invalid_count) *invalid_count = 0;
        return FG21_OK;
    }
    unsigned st[8];
    FG21_CUDA_TRY(cudaMemcpy(st, m->ws.d_status, 32, cudaMemcpyDeviceToHost));
    unsigned long long inv = 0;
    std::memcpy(&inv, st + 4, sizeof inv);
    if (invalid_count) *invalid_count = (int64_t)inv;
    set_invalid_count((int64_t)inv);
    if (st[0]) return set_error(FG21_E_DEVICE, "likelihood kernel reported status 0x%x", st[0]);
    return FG21_OK;
}

int fg21_selftest_bounded_wait(uint32_t *status_word, double *elapsed_s, void *stream) {
    if (!status_word || !elapsed_s) return set_error(FG21_E_ARG, "NULL output");
    cudaStream_t s = (cudaStream_t)stream;
    void *p = nullptr;
    if (cudaMalloc(&p, 64) != cudaSuccess) {
        cudaGetLastError();
        return set_error(FG21_E_NOMEM, "cudaMalloc of 64 bytes failed");
    }
    // [0, 4): status word; [32, 64): one waiting time per warp
    unsigned *d_status = (unsigned *)p;
    unsigned long long *d_elapsed = (unsigned long long *)((char *)p + 32);
    unsigned char h[64];
    cudaError_t e = cudaMemsetAsync(p, 0, 64, s);
    if (e == cudaSuccess) e = launch_wait_selftest(d_status, d_elapsed, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, p, 64, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(p);
    if (e != cudaSuccess) return cuda_error(e, "bounded-wait self-test");
    std::memcpy(status_word, h, sizeof(uint32_t));
    for (int w = 0; w < WAIT_SELFTEST_WARPS; ++w) {
        unsigned long long ns;
        std::memcpy(&ns, h + 32 + 8 * w, sizeof ns);
        elapsed_s[w] = ns == ~0ull ? -1.0 : 1e-9 * (double)ns;
    }
    if (*status_word) return set_error(FG21_E_DEVICE, "self-test kernel reported status 0x%x", *status_word);
    return FG21_OK;
}

int fg21_selftest_mma_rounding(const uint16_t *a, const uint16_t *b, const float *c, float *d, void *stream) {
    if (!a || !b || !c || !d) return set_error(FG21_E_ARG, "NULL operand");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t na = 128 * 16 * 2, nb = 16 * 16 * 2, nc = 128 * 16 * 4;
    char *p = nullptr;
    if (cudaMalloc((void **)&p, 256 + na + nb + 2 * nc) != cudaSuccess) {
        cudaGetLastError();
        return set_error(FG21_E_NOMEM, "cudaMalloc of the probe buffers failed");
    }
    unsigned *d_status = (unsigned *)p;
    uint16_t *d_a = (uint16_t *)(p + 256);
    uint16_t *d_b = (uint16_t *)(p + 256 + na);
    float *d_c = (float *)(p + 256 + na + nb);
    float *d_d = d_c + 128 * 16;
    unsigned st = 0;
    cudaError_t e = cudaMemsetAsync(d_status, 0, 4, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_a, a, na, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_b, b, nb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_c, c, nc, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_mma_probe(d_a, d_b, d_c, d_d, d_status, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, d_d, nc, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, d_status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(p);
    if (e != cudaSuccess) return cuda_error(e, "MMA rounding self-test");
    if (st) return set_error(FG21_E_DEVICE, "MMA probe reported status 0x%x", st);
    return FG21_OK;
}

int fg21_model_timing(fg21_model *m, int enable) {
    if (!m) return set_error(FG21_E_ARG, "NULL model");
    std::lock_guard<std::mutex> lk(m->mu);
    if (m->ws.done) FG21_CUDA_TRY(cudaEventSynchronize(m->ws.done));
    if (enable) {
        int rc = m->ws.timing_prepare();
        if (rc) return rc;
    }
    m->ws.timing = enable != 0;
    m->ws.tcalls = 0;
    return FG21_OK;
}

int fg21_model_timing_totals(fg21_model *m, int64_t *calls, double *prep_ms, double *main_ms, double *reduce_ms) {
    if (!m) return set_error(FG21_E_ARG, "NULL model");
    std::lock_guard<std::mutex> lk(m->mu);
    Workspace &ws = m->ws;
    if (!ws.timing || ws.tcalls == 0) return set_error(FG21_E_STATE, "timing not enabled or no call recorded");
    const int64_t n = ws.tcalls < Workspace::TIMING_CAP ? ws.tcalls : Workspace::TIMING_CAP;
    const int64_t last = (ws.tcalls - 1) % Workspace::TIMING_CAP;
    FG21_CUDA_TRY(cudaEventSynchronize(ws.tev[(size_t)last * 4 + 3]));
    double a = 0, b = 0, c = 0;
    for (int64_t k = 0; k < n; ++k) {
        cudaEvent_t *e = &ws.tev[(size_t)k * 4];
        float x = 0, y = 0, z = 0;
        FG21_CUDA_TRY(cudaEventElapsedTime(&x, e[0], e[1]));
        FG21_CUDA_TRY(cudaEventElapsedTime(&y, e[1], e[2]));
        FG21_CUDA_TRY(cudaEventElapsedTime(&z, e[2], e[3]));
        a += x;
        b += y;
        c += z;
    }
    if (calls) *calls = n;
    if (prep_ms) *prep_ms = a;
    if (main_ms) *main_ms = b;
    if (reduce_ms) *reduce_ms = c;
    return FG21_OK;
}

int fg21_model_eval(fg21_model *m, const double *params, int64_t P, double *T_model, int precision,
                    void *stream) {
    if (!m || !params || !T_model || P <= 0) return set_error(FG21_E_ARG, "bad model_eval arguments");
    int rc = check_precision(m, precision);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(m->mu);
    rc = device_guard(m);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t pbytes = sizeof(double) * (size_t)P * m->n_params();
    const size_t obytes = sizeof(double) * (size_t)P * m->F * m->T;
    double *d_params = nullptr, *d_out = nullptr, *d_logL = nullptr;
    if (cudaMalloc((void **)&d_params, pbytes) != cudaSuccess || cudaMalloc((void **)&d_out, obytes) != cudaSuccess ||
        cudaMalloc((void **)&d_logL, sizeof(double) * P) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_params);
        cudaFree(d_out);
        return set_error(FG21_E_NOMEM, "model_eval buffers");
    }
    int out = FG21_OK;
    do {
        if (cudaMemcpyAsync(d_params, params, pbytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            out = cuda_error(cudaGetLastError(), "model_eval H2D");
            break;
        }
        std::vector<ReqDesc> reqs{model_request(m, d_params, P, d_logL, precision)};
        out = enqueue_requests(m->ws, reqs, precision, s);
        if (out) break;
        cudaError_t e = launch_model_eval(&reqs[0], m->ws.d_reqs, precision, d_out, s);
        if (e != cudaSuccess) {
            out = cuda_error(e, "model_eval launch");
            break;
        }
        if (cudaMemcpyAsync(T_model, d_out, obytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            out = cuda_error(cudaGetLastError(), "model_eval D2H");
            break;
        }
    } while (0);
    cudaStreamSynchronize(s);
    cudaFree(d_params);
    cudaFree(d_out);
    cudaFree(d_logL);
    return out;
}

int fg21_loglike_multi(fg21_model *const *models, const double *const *params, const int64_t *P,
                       double *const *logL, int n_models, int precision, void *stream) {
    if (n_models < 0 || (n_models > 0 && (!models || !params || !P || !logL)))
        return set_error(FG21_E_ARG, "bad multi arguments");
    set_invalid_count(0);
    if (n_models == 0) return FG21_OK;
    if (precision < 0 || precision > 3) return set_error(FG21_E_ARG, "unknown precision %d", precision);
    for (int k = 0; k < n_models; ++k) {
        if (!models[k] || P[k] < 0 || (P[k] > 0 && (!params[k] || !logL[k])))
            return set_error(FG21_E_ARG, "bad request %d", k);
        int rc = check_precision(models[k], precision);
        if (rc) return rc;
    }
    static std::mutex mu;
    static Workspace ws;
    static double *d_io = nullptr;
    static char *h_io = nullptr;
    static size_t io_cap = 0;
    std::lock_guard<std::mutex> lk(mu);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<size_t> poff(n_models), loff(n_models);
    size_t total = 0;
    for (int k = 0; k < n_models; ++k) {
        poff[k] = total;
        total += align256(sizeof(double) * (size_t)P[k] * models[k]->n_params());
        loff[k] = total;
        total += align256(sizeof(double) * (size_t)P[k]);
    }
    total += 64;
    if (ws.done) FG21_CUDA_TRY(cudaEventSynchronize(ws.done));
    if (total > io_cap) {
        if (d_io) cudaFree(d_io);
        if (h_io) cudaFreeHost(h_io);
        d_io = nullptr;
        h_io = nullptr;
        io_cap = 0;
        if (cudaMalloc((void **)&d_io, total) != cudaSuccess || cudaMallocHost((void **)&h_io, total) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FG21_E_NOMEM, "multi I/O buffers");
        }
        io_cap = total;
    }
    std::vector<ReqDesc> reqs;
    std::vector<int> map;
    for (int k = 0; k < n_models; ++k) {
        if (P[k] == 0) continue;
        const size_t pb = sizeof(double) * (size_t)P[k] * models[k]->n_params();
        std::memcpy(h_io + poff[k], params[k], pb);
        reqs.push_back(model_request(models[k], (const double *)((char *)d_io + poff[k]), P[k],
                                     (double *)((char *)d_io + loff[k]), precision));
        map.push_back(k);
    }
    if (reqs.empty()) return FG21_OK;
    FG21_CUDA_TRY(cudaMemcpyAsync(d_io, h_io, loff[n_models - 1] + align256(sizeof(double) * P[n_models - 1]),
                                  cudaMemcpyHostToDevice, s));
    int rc = enqueue_requests(ws, reqs, precision, s);
    if (rc) return rc;
    FG21_CUDA_TRY(cudaMemcpyAsync(h_io, d_io, total - 64, cudaMemcpyDeviceToHost, s));
    unsigned st[8];
    FG21_CUDA_TRY(cudaMemcpyAsync(st, ws.d_status, 32, cudaMemcpyDeviceToHost, s));
    FG21_CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t j = 0; j < map.size(); ++j) {
        int k = map[j];
        std::memcpy(logL[k], h_io + loff[k], sizeof(double) * P[k]);
    }
    unsigned long long inv = 0;
    std::memcpy(&inv, st + 4, sizeof inv);
    set_invalid_count((int64_t)inv);
    if (st[0]) return set_error(FG21_E_DEVICE, "likelihood kernel reported status 0x%x", st[0]);
    return FG21_OK;
}

}  // extern "C"
