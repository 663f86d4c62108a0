// Allocation-free variant of pcc_totals.
//
// Some callers cannot allocate device memory while they run: a simulation
// code that sizes every device buffer once at start-up and forbids
// allocation inside its time loop, or a host application whose own
// allocator owns the whole device and would see a library allocation as a
// leak or a fragmentation hazard.  pcc_totals obtains its scratch (the
// per-block partial sums) from the context, which may allocate; this variant
// uses a fixed array in the library's own device memory instead.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its 96 KiB until the process exits.  Host code cannot use
// its name as a device address, so the address is looked up with
// cudaGetSymbolAddress, with the device current, on the first call in each
// CUDA context, and passed to the kernels.  The lookup is cached per context
// (keyed by the driver's context identifier, which is never reused), so a
// context created anew after cudaDeviceReset, or a second context on the
// same device, gets its own address instead of a stale one.  All calls
// share the array: calls whose kernels overlap on the GPU (different
// streams without ordering) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "pcc_internal.h"

namespace {

constexpr int kCellsPerBlock = 1024;
constexpr int kMaxBlocks = 4096;                       // at most 4,194,304 cells
constexpr long long kMaxCells = (long long)kCellsPerBlock * kMaxBlocks;

// Per-block partial sums {sum W, sum W E, sum W |u|}; every block of a call
// writes its own three entries before the reduction reads them, so nothing
// has to start at zero.
static __device__ __align__(256) double g_partial[3 * kMaxBlocks];

std::mutex g_mutex;

// Scratch addresses already looked up, by CUDA context identifier.
struct CachedAddress { unsigned long long ctx_id; double* ptr; };
constexpr int kMaxContexts = 64;
CachedAddress g_cache[kMaxContexts] = {};
int g_cache_next = 0;

// Block b sums the live particles of cells [b * 1024, (b + 1) * 1024), one warp
// per cell at a time, lanes over particles; fixed-order reduction.
__global__ void totals_block_kernel(const pcc_species sp, int n_cells, int is_photon, double* __restrict__ partial)
{
    __shared__ double acc[3][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c_begin = blockIdx.x * kCellsPerBlock;
    const int c_end = min(c_begin + kCellsPerBlock, n_cells);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int c = c_begin + wid; c < c_end; c += nw) {
        const int b = sp.cell_start[c], n = sp.cell_count[c];
        for (int k = lane; k < n; k += 32) {
            const double ux = sp.ux[b + k], uy = sp.uy[b + k], uz = sp.uz[b + k], w = sp.w[b + k];
            const double u = sqrt(ux * ux + uy * uy + uz * uz);
            s0 += w;
            s1 += w * (is_photon ? u : sqrt(1.0 + u * u));
            s2 += w * u;
        }
    }
    s0 = pcc::warp_sum(s0);
    s1 = pcc::warp_sum(s1);
    s2 = pcc::warp_sum(s2);
    if (lane == 0) { acc[0][wid] = s0; acc[1][wid] = s1; acc[2][wid] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < nw; ++k) { t0 += acc[0][k]; t1 += acc[1][k]; t2 += acc[2][k]; }
        partial[3 * blockIdx.x + 0] = t0;
        partial[3 * blockIdx.x + 1] = t1;
        partial[3 * blockIdx.x + 2] = t2;
    }
}

__global__ void totals_sum_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    for (int b = 0; b < nb; ++b) { t0 += partial[3 * b]; t1 += partial[3 * b + 1]; t2 += partial[3 * b + 2]; }
    out[0] = t0;
    out[1] = t1;
    out[2] = t2;
}

// Identifier of the CUDA context current on this thread (cuCtxGetId; unique
// within the process and never reused).  The two driver calls are resolved
// through the runtime, so the library does not link the driver library.
// *id = 0 when no context is current yet.
int current_context_id(unsigned long long* id)
{
    using GetCurrentFn = CUresult (*)(CUcontext*);
    using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    *id = 0;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return pcc::cuda_fail(e, "pcc_totals_noalloc: cudaGetDriverEntryPointByVersion");
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            pcc::set_error("pcc_totals_noalloc: the driver does not provide cuCtxGetCurrent/cuCtxGetId");
            return PCC_E_CUDA;
        }
        get_current = reinterpret_cast<GetCurrentFn>(f1);
        get_id = reinterpret_cast<GetIdFn>(f2);
    }
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS) {
        pcc::set_error("pcc_totals_noalloc: cuCtxGetCurrent failed");
        return PCC_E_CUDA;
    }
    if (c && get_id(c, id) != CUDA_SUCCESS) {
        pcc::set_error("pcc_totals_noalloc: cuCtxGetId failed");
        return PCC_E_CUDA;
    }
    return PCC_OK;
}

// Device address of g_partial in the current context: looked up with
// cudaGetSymbolAddress on the first call in each context, then cached.
int partial_address(double** out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    unsigned long long id = 0;
    int rc = current_context_id(&id);
    if (rc != PCC_OK) return rc;
    if (id != 0) {
        for (const CachedAddress& c : g_cache)
            if (c.ctx_id == id) { *out = c.ptr; return PCC_OK; }
    }
    // first call in this context (cudaGetSymbolAddress also creates the
    // device's primary context when none is current yet)
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_partial);
    if (e != cudaSuccess) return pcc::cuda_fail(e, "pcc_totals_noalloc: cudaGetSymbolAddress");
    rc = current_context_id(&id);
    if (rc != PCC_OK) return rc;
    if (id != 0) {
        g_cache[g_cache_next] = {id, static_cast<double*>(p)};
        g_cache_next = (g_cache_next + 1) % kMaxContexts;
    }
    *out = static_cast<double*>(p);
    return PCC_OK;
}

}  // namespace

extern "C" int pcc_totals_noalloc(int n_cells, const pcc_species* sp, int is_photon, double* out, void* stream)
{
    if (!sp || !out || !sp->ux || !sp->uy || !sp->uz || !sp->w || !sp->cell_start || !sp->cell_count || n_cells < 1) {
        pcc::set_error("pcc_totals_noalloc: invalid argument");
        return PCC_E_INVALID;
    }
    if ((long long)n_cells > kMaxCells) {
        pcc::set_error("pcc_totals_noalloc: " + std::to_string(n_cells) + " cells exceed the fixed scratch limit of " +
                       std::to_string(kMaxCells) + " cells; use pcc_totals");
        return PCC_E_CAPACITY;
    }
    double* partial = nullptr;
    const int rc = partial_address(&partial);
    if (rc != PCC_OK) return rc;
    const int nb = (n_cells + kCellsPerBlock - 1) / kCellsPerBlock;
    cudaStream_t st = (cudaStream_t)stream;
    totals_block_kernel<<<nb, 256, 0, st>>>(*sp, n_cells, is_photon, partial);
    totals_sum_kernel<<<1, 32, 0, st>>>(partial, nb, out);
    pcc::note_launches(2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCC_OK : pcc::cuda_fail(e, "pcc_totals_noalloc: launch");
}
