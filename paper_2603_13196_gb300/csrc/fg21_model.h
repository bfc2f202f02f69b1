// Model handle and device workspace of libfg21 (internal).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <vector>

#include "fg21_internal.h"

namespace fg21 {

// Device scratch for one launch (request workspaces, operand-tile arena, the
// request descriptors, status word) plus pinned host staging.  Grow-only.
struct Workspace {
    int device = -1;
    char *dev = nullptr;
    size_t dev_bytes = 0;
    char *arena = nullptr;          // operand tiles, addressed by the TMA tensor map
    size_t arena_bytes = 0;
    char *pinned = nullptr;         // host staging (params, logL, descriptors)
    size_t pinned_bytes = 0;
    ReqDesc *d_reqs = nullptr;
    int reqs_cap = 0;
    unsigned *d_status = nullptr;   // bytes 0..3 status word, 16..23 invalid counter
    unsigned long long *d_invalid = nullptr;
    cudaEvent_t done = nullptr;     // recorded after the last launch of a call
    bool timing = false;            // record events around prep / main / reduce of every call
    static constexpr int TIMING_CAP = 8192;
    std::vector<cudaEvent_t> tev;   // [TIMING_CAP][4], created on first use
    int64_t tcalls = 0;             // calls recorded since timing was enabled
    int timing_prepare();           // creates the timing events (when timing is switched on)
    cudaEvent_t *timing_slot();     // the 4 events of the next call (nullptr if timing off)

    int ensure(size_t dev_need, size_t arena_need, size_t pinned_need, int n_reqs);
    void release();
    size_t bytes() const { return dev_bytes + arena_bytes; }
};

// Bytes of the status block cleared per call: status word and invalid counter.
inline size_t status_bytes(int) { return 32; }

// Launch a set of requests whose params/logL device pointers are filled in.
// Plans shapes, carves request workspaces out of `ws`, and enqueues prep,
// main and reduce kernels on `stream`.  The status word and invalid counter
// are cleared first.  Returns FG21_OK or an error code.
int enqueue_requests(Workspace &ws, std::vector<ReqDesc> &reqs, int precision, cudaStream_t stream);

// The two halves of enqueue_requests: plan, size the workspace, carve and fill
// the descriptors (staged in ws.pinned) ...
struct Prepared {
    int n = 0, precision = 0, num_sms = 1;
    int max_blocks = 1, max_fchunks = 1, max_tiles = 1;
    bool tc = false;
    TcLaunch tcl{};
};
int prepare_requests(Workspace &ws, std::vector<ReqDesc> &reqs, int precision, Prepared &pp);
// ... and enqueue the status clear, the descriptor upload (if `upload`) and
// the kernels.  Nothing here allocates or synchronises, so it can be captured
// into a CUDA graph.
int launch_requests(Workspace &ws, const std::vector<ReqDesc> &reqs, const Prepared &pp, cudaStream_t stream,
                    bool upload, bool timing);

int num_sms_of(int device);

}  // namespace fg21

struct fg21_model {
    int N = 0, F = 0, T = 0;        // N: components (rows of A) = max(n_alpha, 1) * n_beta
    int n_beta = 0;                 // spectral-index regions
    int n_alpha = 0;                // amplitude regions with a free scale factor (0: none, alpha = 1)
    int n_params() const { return n_beta + n_alpha + 4; }   // values per parameter row
    int64_t npix = 0;
    int n_empty = 0;
    double nu0 = 0, t_cmb = 0, Lmax = 0;
    std::vector<double> nu, edges, edges_alpha, A, B;
    int device = 0;
    double *d_A = nullptr, *d_B = nullptr, *d_data = nullptr, *d_L = nullptr, *d_nu = nullptr;
    float *d_A32 = nullptr, *d_B32 = nullptr, *d_data32 = nullptr;
    float *d_Alo = nullptr, *d_Ehi = nullptr, *d_Elo = nullptr;   // double-float parts of A and D - T_CMB B
    size_t resident_bytes = 0;      // A, B, data, tables (not the workspace)
    char *io_d = nullptr, *io_h = nullptr;   // params/logL staging of the host-buffer calls
    size_t io_cap = 0;
    // the host-buffer call's evaluation captured as a CUDA graph on io_d, replayed
    // while the point count, precision, staging buffers and work split stay the same
    fg21_graph *host_graph = nullptr;
    int64_t hg_P = 0;
    int hg_prec = -1, hg_cpg = -1;
    int64_t last_P = -1;            // the previous host-buffer call's size, precision and split:
    int last_prec = -1, last_cpg = -1;   // a graph is captured when a call repeats them
    fg21::Workspace ws;
    std::map<std::pair<int, int>, int> tuned_cpg;   // (precision, 128-point tiles) -> channels per group
    std::mutex tune_mu;                              // guards tuned_cpg
    std::mutex mu;
};

namespace fg21 {
int model_upload(fg21_model *m);
// A request descriptor of model m for `precision` (carrying the autotuned work
// split for its size, if any).
ReqDesc model_request(fg21_model *m, const double *d_params, int64_t P, double *d_logL, int precision);
// The device status word (and invalid count) of a graph's workspace.
unsigned *graph_status(fg21_graph *g);
}  // namespace fg21
