// CUDA-graph evaluation of a fixed batch: fg21_graph_create / _create_multi
// capture one likelihood evaluation of a fixed set of requests (models, point
// counts, device parameter and output buffers) into a CUDA graph once, and
// fg21_graph_launch replays it.  The plan, workspace and request descriptors
// are made and uploaded at creation; a replay is the status clear, the prep,
// tensor-core (or SIMT) and reduction kernels, and reads whatever the
// parameter buffers hold when it runs.  This is the batched evaluation of
// eq. likelihood (Sec. 2.3.1) over eq. fast_forward_model (Sec. 2.2) for the
// points a nested sampler proposes (Sec. 3), with the per-call host work and
// launch latency taken out of the loop.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "fg21_internal.h"
#include "fg21_model.h"

struct fg21_graph {
    int device = 0;
    fg21::Workspace ws;
    std::vector<fg21::ReqDesc> reqs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace fg21;

namespace {

void graph_free(fg21_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->ws.release();
    delete g;
}

}  // namespace

unsigned *fg21::graph_status(fg21_graph *g) { return g->ws.d_status; }

extern "C" {

int fg21_graph_create_multi(fg21_model *const *models, const double *const *d_params, const int64_t *P,
                            double *const *d_logL, int n_models, int precision, fg21_graph **out) {
    if (!out) return set_error(FG21_E_ARG, "NULL output");
    *out = nullptr;
    if (n_models <= 0 || !models || !d_params || !P || !d_logL) return set_error(FG21_E_ARG, "bad graph arguments");
    if (precision < 0 || precision > 3) return set_error(FG21_E_ARG, "unknown precision %d", precision);
    int dev = 0;
    FG21_CUDA_TRY(cudaGetDevice(&dev));
    fg21_graph *g = new fg21_graph;
    g->device = dev;
    for (int k = 0; k < n_models; ++k) {
        fg21_model *m = models[k];
        if (!m || P[k] < 0 || (P[k] > 0 && (!d_params[k] || !d_logL[k]))) {
            graph_free(g);
            return set_error(FG21_E_ARG, "bad request %d", k);
        }
        if (m->device != dev) {
            graph_free(g);
            return set_error(FG21_E_ARG, "model %d lives on device %d, current device is %d", k, m->device, dev);
        }
        if ((precision == FG21_PREC_FP16X3 || precision == FG21_PREC_BF16X3) && m->N > FG21_MAX_REGIONS_TC) {
            graph_free(g);
            return set_error(FG21_E_RANGE, "model %d: N = %d above the tensor-core limit", k, m->N);
        }
        if (P[k] > 0) g->reqs.push_back(model_request(m, d_params[k], P[k], d_logL[k], precision));
    }
    if (g->reqs.empty()) {
        graph_free(g);
        return set_error(FG21_E_ARG, "no points in the batch");
    }
    Prepared pp;
    int rc = prepare_requests(g->ws, g->reqs, precision, pp);
    if (rc) {
        graph_free(g);
        return rc;
    }
    // descriptors once, outside the graph
    cudaError_t e = cudaMemcpy(g->ws.d_reqs, g->ws.pinned, sizeof(ReqDesc) * g->reqs.size(), cudaMemcpyHostToDevice);
    cudaStream_t s = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        if (s) cudaStreamDestroy(s);
        graph_free(g);
        return cuda_error(e, "graph capture setup");
    }
    rc = launch_requests(g->ws, g->reqs, pp, s, false, false);
    e = cudaStreamEndCapture(s, &g->graph);
    if (rc == FG21_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    cudaStreamDestroy(s);
    if (rc) {
        graph_free(g);
        return rc;
    }
    if (e != cudaSuccess) {
        graph_free(g);
        return cuda_error(e, "graph capture");
    }
    *out = g;
    return FG21_OK;
}

int fg21_graph_create(fg21_model *m, const double *d_params, int64_t P, double *d_logL, int precision,
                      fg21_graph **out) {
    return fg21_graph_create_multi(&m, &d_params, &P, &d_logL, 1, precision, out);
}

int fg21_graph_launch(fg21_graph *g, void *stream) {
    if (!g || !g->exec) return set_error(FG21_E_ARG, "NULL graph");
    int dev = 0;
    FG21_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != g->device) return set_error(FG21_E_ARG, "graph lives on device %d, current device is %d", g->device, dev);
    FG21_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return FG21_OK;
}

int fg21_graph_sync_status(fg21_graph *g, void *stream, int64_t *invalid_count) {
    if (!g) return set_error(FG21_E_ARG, "NULL graph");
    FG21_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned st[8];
    FG21_CUDA_TRY(cudaMemcpy(st, g->ws.d_status, 32, cudaMemcpyDeviceToHost));
    unsigned long long inv = 0;
    std::memcpy(&inv, st + 4, sizeof inv);
    if (invalid_count) *invalid_count = (int64_t)inv;
    set_invalid_count((int64_t)inv);
    if (st[0]) return set_error(FG21_E_DEVICE, "likelihood kernel reported status 0x%x", st[0]);
    return FG21_OK;
}

int fg21_graph_destroy(fg21_graph *g) {
    if (!g) return FG21_OK;
    cudaDeviceSynchronize();
    graph_free(g);
    return FG21_OK;
}

}  // extern "C"
