// Context lifetime, status readback and error reporting of the C ABI.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>

#include "pcc_internal.h"

namespace pcc {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void note_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return PCC_E_CUDA;
}

int ensure_scratch(pcc_ctx* ctx, size_t bytes)
{
    if (bytes <= ctx->scratch_bytes) return PCC_OK;
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->scratch, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
    ctx->scratch_bytes = bytes;
    return PCC_OK;
}

}  // namespace pcc

using namespace pcc;

void pcc_free_tables(pcc_ctx* ctx);

extern "C" const char* pcc_version(void) { return "pcc 0.1 (sm_103a)"; }

extern "C" const char* pcc_last_error(void) { return g_last_error.c_str(); }

extern "C" unsigned long long pcc_launch_count(void) { return launches_so_far(); }

extern "C" const char* pcc_status_string(int code)
{
    switch (code) {
    case PCC_OK: return "PCC_OK: success";
    case PCC_E_INVALID: return "PCC_E_INVALID: bad argument";
    case PCC_E_CUDA: return "PCC_E_CUDA: a CUDA runtime call failed";
    case PCC_E_CAPACITY: return "PCC_E_CAPACITY: a buffer or supported size is too small";
    case PCC_E_NO_TABLES: return "PCC_E_NO_TABLES: tables not built on this context";
    default: return "unknown return code";
    }
}

extern "C" const char* pcc_status_bit_string(unsigned bit)
{
    switch (bit) {
    case PCC_ST_TABLE_RANGE: return "PCC_ST_TABLE_RANGE";
    case PCC_ST_PROB_LARGE: return "PCC_ST_PROB_LARGE";
    case PCC_ST_CAPACITY: return "PCC_ST_CAPACITY";
    case PCC_ST_NONFINITE: return "PCC_ST_NONFINITE";
    case PCC_ST_ID_RANGE: return "PCC_ST_ID_RANGE";
    case PCC_ST_TIMEOUT: return "PCC_ST_TIMEOUT";
    case PCC_ST_BOUND_RANGE: return "PCC_ST_BOUND_RANGE";
    default: return "unknown status bit";
    }
}

extern "C" int pcc_create(pcc_ctx** out, int device)
{
    if (!out) { set_error("pcc_create: null output"); return PCC_E_INVALID; }
    *out = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "pcc_create: cudaSetDevice");
    pcc_ctx* ctx = new pcc_ctx();
    ctx->device = device;
    e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->stats, sizeof(DevStats));
    if (e == cudaSuccess) e = cudaMemset(ctx->stats, 0, sizeof(DevStats));
    if (e != cudaSuccess) {
        if (ctx->stats) cudaFree(ctx->stats);
        delete ctx;
        return cuda_fail(e, "pcc_create");
    }
    *out = ctx;
    return PCC_OK;
}

extern "C" void pcc_destroy(pcc_ctx* ctx)
{
    if (!ctx) return;
    pcc_free_graph(ctx);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    pcc_free_tables(ctx);
    if (ctx->stats) cudaFree(ctx->stats);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->lists) cudaFree(ctx->lists);
    if (ctx->queue_a) cudaFree(ctx->queue_a);
    if (ctx->queue_b) cudaFree(ctx->queue_b);
    delete ctx;
}

extern "C" int pcc_read_status(pcc_ctx* ctx, unsigned* status_out, pcc_stats* stats_out, void* stream)
{
    if (!ctx) { set_error("pcc_read_status: null context"); return PCC_E_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    DevStats h;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->stats, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->stats, 0, sizeof(DevStats), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "pcc_read_status");
    if (status_out) *status_out = h.status;
    if (stats_out) {
        for (int i = 0; i < 3; ++i) stats_out->pairs[i] = h.pairs[i];
        for (int i = 0; i < 5; ++i) {
            stats_out->accepted[i] = h.accepted[i];
            stats_out->created[i] = h.created[i];
        }
        stats_out->energy_change = h.energy_change;
        stats_out->charge_change = h.charge_change;
        for (int i = 0; i < 3; ++i) stats_out->candidates[i] = h.candidates[i];
    }
    return PCC_OK;
}
