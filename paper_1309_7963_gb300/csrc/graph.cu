// CUDA-graph launch plans (host code): one batch launch (count reset, queue-head reset,
// event kernel) captured once for fixed buffers and replayed with one cudaGraphLaunch.
// Each plan owns its queue head, so replays of different plans may overlap.
#include "api_internal.h"

using namespace pnuc;

struct pnuc_graph {
    pnuc_ctx *ctx = nullptr;
    pnuc_precision precision = PNUC_FP32;
    pnuc_method method = PNUC_PERSISTENT;
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long *head = nullptr;
};

namespace {

pnuc_status capture(pnuc_graph *g, const pnuc_batch *b, const pnuc_output *o, cudaGraph_t *out)
{
    pnuc_ctx *ctx = g->ctx;
    CU(ctx, cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal));
    pnuc_status st = launch_batch(ctx, g->precision, g->method, b, o, g->capture, ctx->tuning[tuning_slot(g->precision)],
                                    g->head);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->capture, &graph);
    if (st != PNUC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(ctx, PNUC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    *out = graph;
    return PNUC_OK;
}

}  // namespace

extern "C" {

pnuc_status pnuc_graph_destroy(pnuc_graph *g)
{
    if (!g) return PNUC_OK;
    if (g->ctx) cudaSetDevice(g->ctx->cfg.device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->capture) cudaStreamDestroy(g->capture);
    cudaFree(g->head);
    delete g;
    return PNUC_OK;
}

pnuc_status pnuc_graph_create(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method, const pnuc_batch *batch,
                              const pnuc_output *out, pnuc_graph **graph)
{
    if (!graph) return fail(ctx, PNUC_ERR_ARG, "null graph pointer");
    *graph = nullptr;
    pnuc_status st = check_batch(ctx, precision, method, batch, out);
    if (st != PNUC_OK) return st;
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    pnuc_graph *g = new pnuc_graph();
    g->ctx = ctx;
    g->precision = precision;
    g->method = method;
    if (cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&g->head, 128) != cudaSuccess) {
        pnuc_graph_destroy(g);
        return fail(ctx, PNUC_ERR_CUDA, "graph set-up failed");
    }
    st = capture(g, batch, out, &g->graph);
    if (st == PNUC_OK) {
        cudaError_t e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) st = fail(ctx, PNUC_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    if (st != PNUC_OK) {
        pnuc_graph_destroy(g);
        return st;
    }
    *graph = g;
    return PNUC_OK;
}

pnuc_status pnuc_graph_update(pnuc_graph *g, const pnuc_batch *batch, const pnuc_output *out)
{
    if (!g) return PNUC_ERR_ARG;
    pnuc_ctx *ctx = g->ctx;
    pnuc_status st = check_batch(ctx, g->precision, g->method, batch, out);
    if (st != PNUC_OK) return st;
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    cudaGraph_t ng = nullptr;
    st = capture(g, batch, out, &ng);
    if (st != PNUC_OK) return st;
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(g->exec, ng, &info) != cudaSuccess) {
        cudaGetLastError();  // clear the update failure, then instantiate afresh
        cudaGraphExec_t ne = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ne, ng, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(ng);
            return fail(ctx, PNUC_ERR_CUDA, "graph re-instantiate failed: %s", cudaGetErrorString(e));
        }
        cudaGraphExecDestroy(g->exec);
        g->exec = ne;
    }
    cudaGraphDestroy(g->graph);
    g->graph = ng;
    return PNUC_OK;
}

pnuc_status pnuc_graph_launch(pnuc_graph *g, void *stream)
{
    if (!g) return PNUC_ERR_ARG;
    CU(g->ctx, cudaSetDevice(g->ctx->cfg.device));
    CU(g->ctx, cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return PNUC_OK;
}

}  // extern "C"
