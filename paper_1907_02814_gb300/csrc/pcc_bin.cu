// Binning by cell (counting sort into cell regions, each cell in pid order),
// the per-step commit of appended secondaries, and FP64 totals.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pcc_internal.h"

namespace pcc {

constexpr int kMaxCellSort = 16384;
constexpr int kScanBlock = 1024;

// ---- histogram: warp-aggregated atomics (one atomic per distinct cell per warp)
__global__ void bin_count_kernel(const int* __restrict__ cell, int n, int n_cells, int* __restrict__ counts,
                                 DevStats* st)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = i < n;
    int c = in ? cell[i] : -1;
    if (in && (c < 0 || c >= n_cells)) {
        raise_status(st, PCC_ST_NONFINITE);
        c = -1;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(peers) - 1;
    if (c >= 0 && (threadIdx.x & 31) == leader) atomicAdd(&counts[c], __popc(peers));
}

// ---- three-pass exclusive scan of region sizes
__device__ __forceinline__ long long region_of(int count, int slack_abs, double slack_rel)
{
    const long long extra = (long long)ceil(slack_rel * (double)count);
    return (long long)count + (extra > slack_abs ? extra : slack_abs);
}

__global__ void scan_local_kernel(const int* __restrict__ counts, int n, int slack_abs, double slack_rel,
                                  long long* __restrict__ out, long long* __restrict__ block_sums)
{
    __shared__ long long s[kScanBlock];
    const int base = blockIdx.x * kScanBlock;
    for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x) {
        const int i = base + k;
        s[k] = i < n ? region_of(counts[i], slack_abs, slack_rel) : 0;
    }
    __syncthreads();
    // Hillis-Steele inclusive scan in shared memory
    for (int off = 1; off < kScanBlock; off <<= 1) {
        long long v[kScanBlock / 256];
        for (int k = threadIdx.x, q = 0; k < kScanBlock; k += blockDim.x, ++q) v[q] = k >= off ? s[k - off] : 0;
        __syncthreads();
        for (int k = threadIdx.x, q = 0; k < kScanBlock; k += blockDim.x, ++q) s[k] += v[q];
        __syncthreads();
    }
    for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x) {
        const int i = base + k;
        if (i < n) out[i] = s[k];   // inclusive
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = s[kScanBlock - 1];
}

__global__ void scan_blocks_kernel(long long* block_sums, int nb)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        long long acc = 0;
        for (int b = 0; b < nb; ++b) {
            const long long v = block_sums[b];
            block_sums[b] = acc;   // exclusive
            acc += v;
        }
    }
}

__global__ void scan_finish_kernel(const long long* __restrict__ incl, const long long* __restrict__ block_off,
                                   const int* __restrict__ counts, int n, int* __restrict__ cell_start,
                                   int* __restrict__ cell_count, int* __restrict__ cell_added,
                                   long long* __restrict__ total_and_max)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long end = incl[i] + block_off[i / kScanBlock];
    if (end <= 0x7fffffffLL) cell_start[i + 1] = (int)end;
    if (i == 0) cell_start[0] = 0;
    cell_count[i] = counts[i];
    cell_added[i] = 0;
    if (i == n - 1) atomicMax((unsigned long long*)&total_and_max[0], (unsigned long long)end);
    atomicMax((unsigned long long*)&total_and_max[1], (unsigned long long)counts[i]);
}

// ---- scatter into the temporary region layout
struct Rec {
    const float *ux, *uy, *uz, *w, *x;
    const uint64_t* pid;
};
struct MRec {
    float *ux, *uy, *uz, *w, *x;
    uint64_t* pid;
};

__global__ void bin_scatter_kernel(Rec in, const int* __restrict__ cell, int n, int n_cells,
                                   const int* __restrict__ cell_start, int* __restrict__ cursor, MRec tmp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < n;
    int c = act ? cell[i] : -1;
    if (c >= n_cells) c = -1;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (c >= 0 && lane == leader) base = atomicAdd(&cursor[c], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    if (c < 0) return;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int dst = cell_start[c] + base + rank;
    tmp.ux[dst] = in.ux[i];
    tmp.uy[dst] = in.uy[i];
    tmp.uz[dst] = in.uz[i];
    tmp.w[dst] = in.w[i];
    if (in.x) tmp.x[dst] = in.x[i];
    tmp.pid[dst] = in.pid[i];
}

// ---- per-cell bitonic sort by pid (one block per cell), then gather
__global__ void cell_sort_kernel(const int* __restrict__ cell_start, const int* __restrict__ cell_count, int n_pow2,
                                 Rec tmp, MRec out)
{
    extern __shared__ unsigned char smem[];
    uint64_t* key = (uint64_t*)smem;
    int* idx = (int*)(key + n_pow2);
    const int c = blockIdx.x;
    const int n = cell_count[c], s0 = cell_start[c];
    if (n == 0) return;
    int m = 1;
    while (m < n) m <<= 1;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        key[k] = k < n ? tmp.pid[s0 + k] : ~0ull;
        idx[k] = k;
    }
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = threadIdx.x; k < m; k += blockDim.x) {
                const int p = k ^ stride;
                if (p > k) {
                    const bool up = (k & size) == 0;
                    const uint64_t a = key[k], b = key[p];
                    if ((a > b) == up) {
                        key[k] = b; key[p] = a;
                        const int t = idx[k]; idx[k] = idx[p]; idx[p] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int src = s0 + idx[k], dst = s0 + k;
        out.ux[dst] = tmp.ux[src];
        out.uy[dst] = tmp.uy[src];
        out.uz[dst] = tmp.uz[src];
        out.w[dst] = tmp.w[src];
        if (out.x) out.x[dst] = tmp.x[src];
        out.pid[dst] = key[k];
    }
}

// ---- commit of appended secondaries: order by pid, then make live
__global__ void commit_kernel(MRec sp, const int* __restrict__ cell_start, int* __restrict__ cell_count,
                              int* __restrict__ cell_added, int n_cells)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int a = cell_added[c];
    if (a == 0) return;
    const int b = cell_start[c] + cell_count[c];
    for (int i = 1; i < a; ++i) {   // insertion sort of the (few) appended records
        const uint64_t kp = sp.pid[b + i];
        const float vx = sp.ux[b + i], vy = sp.uy[b + i], vz = sp.uz[b + i], vw = sp.w[b + i];
        const float vxx = sp.x ? sp.x[b + i] : 0.f;
        int j = i - 1;
        while (j >= 0 && sp.pid[b + j] > kp) {
            sp.pid[b + j + 1] = sp.pid[b + j];
            sp.ux[b + j + 1] = sp.ux[b + j];
            sp.uy[b + j + 1] = sp.uy[b + j];
            sp.uz[b + j + 1] = sp.uz[b + j];
            sp.w[b + j + 1] = sp.w[b + j];
            if (sp.x) sp.x[b + j + 1] = sp.x[b + j];
            --j;
        }
        sp.pid[b + j + 1] = kp;
        sp.ux[b + j + 1] = vx; sp.uy[b + j + 1] = vy; sp.uz[b + j + 1] = vz; sp.w[b + j + 1] = vw;
        if (sp.x) sp.x[b + j + 1] = vxx;
    }
    cell_count[c] += a;
    cell_added[c] = 0;
}

// ---- FP64 totals: one warp per cell, fixed-order partials per block
__global__ void totals_kernel(const pcc_species sp, int n_cells, int is_photon, double* __restrict__ partial)
{
    __shared__ double acc[3][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int c = blockIdx.x * nw + wid; c < n_cells; c += gridDim.x * nw) {
        const int b = sp.cell_start[c], n = sp.cell_count[c];
        for (int k = lane; k < n; k += 32) {
            const double ux = sp.ux[b + k], uy = sp.uy[b + k], uz = sp.uz[b + k], w = sp.w[b + k];
            const double u = sqrt(ux * ux + uy * uy + uz * uz);
            const double E = is_photon ? u : sqrt(1.0 + u * u);
            s0 += w;
            s1 += w * E;
            s2 += w * u;
        }
    }
    s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2);
    if (lane == 0) { acc[0][wid] = s0; acc[1][wid] = s1; acc[2][wid] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0, t1 = 0, t2 = 0;
        for (int k = 0; k < nw; ++k) { t0 += acc[0][k]; t1 += acc[1][k]; t2 += acc[2][k]; }
        partial[3 * blockIdx.x + 0] = t0;
        partial[3 * blockIdx.x + 1] = t1;
        partial[3 * blockIdx.x + 2] = t2;
    }
}

__global__ void totals_final_kernel(const double* partial, int nb, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t0 = 0, t1 = 0, t2 = 0;
        for (int b = 0; b < nb; ++b) { t0 += partial[3 * b]; t1 += partial[3 * b + 1]; t2 += partial[3 * b + 2]; }
        out[0] = t0; out[1] = t1; out[2] = t2;
    }
}

}  // namespace pcc

using namespace pcc;

extern "C" int pcc_bin(pcc_ctx* ctx, const pcc_particles* in, int n_cells, pcc_species* out, int slack_abs,
                       double slack_rel, void* stream)
{
    if (!ctx || !in || !out) { set_error("pcc_bin: null argument"); return PCC_E_INVALID; }
    if (n_cells < 1 || in->n < 0 || slack_abs < 0 || !(slack_rel >= 0.0) || out->capacity < 0) {
        set_error("pcc_bin: invalid sizes");
        return PCC_E_INVALID;
    }
    if (in->n > 0 && (!in->ux || !in->uy || !in->uz || !in->w || !in->pid || !in->cell)) {
        set_error("pcc_bin: null input array");
        return PCC_E_INVALID;
    }
    if (!out->ux || !out->uy || !out->uz || !out->w || !out->pid || !out->cell_start || !out->cell_count ||
        !out->cell_added || ((in->x == nullptr) != (out->x == nullptr) && in->x != nullptr)) {
        set_error("pcc_bin: null output array (x must be given on both sides or only on the output)");
        return PCC_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (n_cells + kScanBlock - 1) / kScanBlock;
    const size_t cap = (size_t)out->capacity;
    // scratch: counts, cursor, inclusive scan, block sums, total/max, temp records
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_counts = take(n_cells * sizeof(int));
    const size_t o_cursor = take(n_cells * sizeof(int));
    const size_t o_incl = take(n_cells * sizeof(long long));
    const size_t o_bsum = take(nb * sizeof(long long));
    const size_t o_tm = take(2 * sizeof(long long));
    const size_t o_f = take(cap * 5 * sizeof(float));
    const size_t o_pid = take(cap * sizeof(uint64_t));
    int rc = ensure_scratch(ctx, off);
    if (rc) return rc;
    char* base = (char*)ctx->scratch;
    int* counts = (int*)(base + o_counts);
    int* cursor = (int*)(base + o_cursor);
    long long* incl = (long long*)(base + o_incl);
    long long* bsum = (long long*)(base + o_bsum);
    long long* tm = (long long*)(base + o_tm);
    float* tf = (float*)(base + o_f);
    MRec tmp{tf, tf + cap, tf + 2 * cap, tf + 3 * cap, out->x ? tf + 4 * cap : nullptr, (uint64_t*)(base + o_pid)};

    cudaError_t e = cudaMemsetAsync(counts, 0, n_cells * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, n_cells * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tm, 0, 2 * sizeof(long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "pcc_bin: memset");
    if (in->n > 0) {
        bin_count_kernel<<<(in->n + 255) / 256, 256, 0, st>>>(in->cell, in->n, n_cells, counts, ctx->stats);
        note_launches(1);
    }
    scan_local_kernel<<<nb, 256, 0, st>>>(counts, n_cells, slack_abs, slack_rel, incl, bsum);
    scan_blocks_kernel<<<1, 32, 0, st>>>(bsum, nb);
    scan_finish_kernel<<<(n_cells + 255) / 256, 256, 0, st>>>(incl, bsum, counts, n_cells, out->cell_start,
                                                             out->cell_count, out->cell_added, tm);
    note_launches(3);
    long long h_tm[2] = {0, 0};
    e = cudaMemcpyAsync(h_tm, tm, sizeof(h_tm), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "pcc_bin: count/scan");
    if (h_tm[0] > (long long)cap) {
        set_error("pcc_bin: regions need " + std::to_string(h_tm[0]) + " slots, capacity " + std::to_string(cap));
        return PCC_E_CAPACITY;
    }
    if (h_tm[1] > kMaxCellSort) {
        set_error("pcc_bin: a cell holds " + std::to_string(h_tm[1]) + " particles (max 16384)");
        return PCC_E_CAPACITY;
    }
    if (in->n > 0) {
        Rec rin{in->ux, in->uy, in->uz, in->w, out->x ? in->x : nullptr, in->pid};
        bin_scatter_kernel<<<(in->n + 255) / 256, 256, 0, st>>>(rin, in->cell, in->n, n_cells, out->cell_start,
                                                                 cursor, tmp);
        int m = 1;
        while (m < h_tm[1]) m <<= 1;
        const size_t smem = (size_t)m * (sizeof(uint64_t) + sizeof(int));
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(cell_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        Rec rt{tmp.ux, tmp.uy, tmp.uz, tmp.w, tmp.x, tmp.pid};
        MRec ro{out->ux, out->uy, out->uz, out->w, out->x, out->pid};
        cell_sort_kernel<<<n_cells, 256, smem, st>>>(out->cell_start, out->cell_count, m, rt, ro);
        note_launches(2);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_bin: kernels");
}

extern "C" int pcc_append_secondaries(pcc_ctx* ctx, int n_cells, pcc_species* sp, void* stream)
{
    if (!ctx || !sp || n_cells < 1 || !sp->cell_start || !sp->cell_count || !sp->cell_added || !sp->pid) {
        set_error("pcc_append_secondaries: invalid argument");
        return PCC_E_INVALID;
    }
    MRec r{sp->ux, sp->uy, sp->uz, sp->w, sp->x, sp->pid};
    commit_kernel<<<(n_cells + 255) / 256, 256, 0, (cudaStream_t)stream>>>(r, sp->cell_start, sp->cell_count,
                                                                            sp->cell_added, n_cells);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_append_secondaries");
}

extern "C" int pcc_totals(pcc_ctx* ctx, int n_cells, const pcc_species* sp, int is_photon, double* out,
                          void* stream)
{
    if (!ctx || !sp || !out || n_cells < 1) { set_error("pcc_totals: invalid argument"); return PCC_E_INVALID; }
    const int blocks = 2 * std::max(ctx->num_sms, 1);
    int rc = ensure_scratch(ctx, (size_t)blocks * 3 * sizeof(double));
    if (rc) return rc;
    double* partial = (double*)ctx->scratch;
    cudaStream_t st = (cudaStream_t)stream;
    totals_kernel<<<blocks, 256, 0, st>>>(*sp, n_cells, is_photon, partial);
    totals_final_kernel<<<1, 32, 0, st>>>(partial, blocks, out);
    note_launches(2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_totals");
}
