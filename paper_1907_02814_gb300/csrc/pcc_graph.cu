// The multi-step collision loop captured as one CUDA graph.
//
// A step is what a PIC code runs between two pushes: the collision kernels
// of the three projectile groups (electron-ion, positron-ion, photon-ion,
// Sec. III.A, in that order) followed by the commit of the secondaries of
// the three species.  n such steps are captured once into a graph, so that
// a launch costs one host call instead of about twenty per step.  The step
// index of each captured step is fixed at capture time (it keys the random
// streams and the secondary identifiers), so a graph stands for the steps
// [step0, step0 + n); capture again to continue past them.
#include <cuda_runtime.h>

#include "pcc_internal.h"

using namespace pcc;

void pcc_free_graph(pcc_ctx* ctx)
{
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
    for (cudaEvent_t e : ctx->graph_events) cudaEventDestroy(e);
    ctx->graph_events.clear();
    ctx->graph_steps = 0;
    ctx->graph_kernels = 0;
}

static int record(pcc_ctx* ctx, int idx, cudaStream_t cs)
{
    if (ctx->graph_events.empty()) return PCC_OK;
    const cudaError_t e = cudaEventRecordWithFlags(ctx->graph_events[idx], cs, cudaEventRecordExternal);
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_steps_capture: event record");
}

struct GroupEvents {
    pcc_ctx* ctx;
    int base;
    cudaStream_t cs;
};

static int after_group(void* user, int g)
{
    const GroupEvents* r = static_cast<const GroupEvents*>(user);
    return record(r->ctx, r->base + 1 + g, r->cs);
}

// One step on the capture stream: the groups of the mask one by one (the
// batched path's class sort of all groups comes first, inside the first
// part), then the three commits, with an event before and after each part.
static int capture_step(pcc_ctx* ctx, const pcc_step_desc* d, uint64_t step, int s, cudaStream_t cs)
{
    GroupEvents ev{ctx, 5 * s, cs};
    int rc = record(ctx, 5 * s, cs);
    if (rc == PCC_OK)
        rc = collide_groups(ctx, d->cells, d->em, d->ep, d->ph, d->ion, d->dt, d->seed, step, d->mask, d->precision,
                            d->ledger, cs, after_group, &ev);
    if (rc == PCC_OK) rc = pcc_append_secondaries(ctx, d->cells->n_cells, d->em, cs);
    if (rc == PCC_OK) rc = pcc_append_secondaries(ctx, d->cells->n_cells, d->ep, cs);
    if (rc == PCC_OK) rc = pcc_append_secondaries(ctx, d->cells->n_cells, d->ph, cs);
    if (rc == PCC_OK) rc = record(ctx, 5 * s + 4, cs);
    return rc;
}

extern "C" int pcc_steps_capture(pcc_ctx* ctx, const pcc_step_desc* d, uint64_t step0, int n_steps, int timing,
                                 void* stream)
{
    if (!ctx || !d || !d->cells || !d->em || !d->ep || !d->ph || !d->ion || n_steps < 1 || n_steps > 100000) {
        set_error("pcc_steps_capture: invalid argument");
        return PCC_E_INVALID;
    }
    pcc_free_graph(ctx);
    // every allocation and occupancy query of the step happens here, outside the capture
    int rc = collide_prepare(ctx, d->cells, d->em, d->ep, d->ph, d->ion, d->mask, d->precision);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (!ctx->capture_stream) e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "pcc_steps_capture: stream");
    if (timing) {
        ctx->graph_events.resize((size_t)5 * n_steps, nullptr);
        for (auto& ev : ctx->graph_events) {
            e = cudaEventCreate(&ev);
            if (e != cudaSuccess) { pcc_free_graph(ctx); return cuda_fail(e, "pcc_steps_capture: events"); }
        }
    }
    cudaStream_t cs = ctx->capture_stream;
    const unsigned long long before = launches_so_far();
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { pcc_free_graph(ctx); return cuda_fail(e, "pcc_steps_capture: begin"); }
    for (int s = 0; s < n_steps && rc == PCC_OK; ++s) rc = capture_step(ctx, d, step0 + (uint64_t)s, s, cs);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    const unsigned long long captured = launches_so_far() - before;
    note_launches(0ull - captured);   // captured, not launched
    if (rc != PCC_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        pcc_free_graph(ctx);
        return rc != PCC_OK ? rc : cuda_fail(e, "pcc_steps_capture: end");
    }
    e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e == cudaSuccess) e = cudaGraphUpload(ctx->graph_exec, (cudaStream_t)stream);
    if (e != cudaSuccess) { pcc_free_graph(ctx); return cuda_fail(e, "pcc_steps_capture: instantiate"); }
    ctx->graph_steps = n_steps;
    ctx->graph_kernels = captured;
    return PCC_OK;
}

extern "C" int pcc_steps_launch(pcc_ctx* ctx, void* stream)
{
    if (!ctx || !ctx->graph_exec) { set_error("pcc_steps_launch: nothing captured"); return PCC_E_INVALID; }
    const cudaError_t e = cudaGraphLaunch(ctx->graph_exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "pcc_steps_launch");
    note_launches(ctx->graph_kernels);
    return PCC_OK;
}

extern "C" int pcc_steps_timing(pcc_ctx* ctx, float* ms_out)
{
    if (!ctx || !ms_out || ctx->graph_events.empty()) {
        set_error("pcc_steps_timing: no graph captured with timing");
        return PCC_E_INVALID;
    }
    cudaError_t e = cudaEventSynchronize(ctx->graph_events.back());
    for (int s = 0; s < ctx->graph_steps && e == cudaSuccess; ++s)
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            e = cudaEventElapsedTime(&ms_out[4 * s + k], ctx->graph_events[5 * s + k], ctx->graph_events[5 * s + k + 1]);
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_steps_timing");
}
