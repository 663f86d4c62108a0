// Library-internal context and launcher declarations (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/pcc.h"
#include "pcc_device.cuh"

struct pcc_ctx {
    int device = 0;
    int num_sms = 0;
    // tables (device)
    int n_mat = 0;
    pcc_table_spec spec{};
    double* screen = nullptr;         // [n_mat][8]
    double* brems_sigma = nullptr;    // [n_mat][R]
    double* brems_cdf = nullptr;      // [n_mat][R][C]
    double* bh_sigma = nullptr;
    double* bh_cdf = nullptr;
    double* tri_gp_cdf = nullptr;     // [R][C]
    double* tri_split_cdf = nullptr;
    float* f_brems_lnsig = nullptr;   // FP32 copies: ln sigma and CDFs
    float* f_brems_cdf = nullptr;
    float* f_bh_lnsig = nullptr;
    float* f_bh_cdf = nullptr;
    float* f_tri_gp_cdf = nullptr;
    float* f_tri_split_cdf = nullptr;
    float* f_Z = nullptr;             // [n_mat] nuclear charge as float
    float* f_bound = nullptr;         // [n_mat][3] acceptance bounds: Brems, Trident, BH
    // status and counters
    pcc::DevStats* stats = nullptr;
    // scratch
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // cell work lists of the batched collision kernels (3 groups + class counters)
    int* lists = nullptr;
    int lists_cells = 0;
    // launch schedule of the batched kernels (set by pcc_tune or defaults)
    void* queue_a = nullptr;       // candidate queue over projectile slots
    size_t queue_a_cap = 0;
    void* queue_b = nullptr;       // candidate queue over target slots (N_p < N_t cells)
    size_t queue_b_cap = 0;
    int minb = 4;                  // register budget: minimum resident blocks per SM
    // lane groups of the batched scan per group (e-, e+, photons): size
    // classes (two per octave of N_pair) from which a cell takes a whole
    // warp, 16, 8 or 4 lanes (below: 2).  Chosen by timing on the 2^20-cell
    // batched Cu workload; the autotuner may replace them.
    int scan_thr[3][4] = {{20, 20, 15, 2}, {12, 12, 6, 0}, {17, 17, 15, 13}};
    int blocks_per_sm = 0;         // persistent grid cap (0: as many as fit)
    bool class_smem_ready = false; // large shared memory enabled for the class-sort offsets
    int wait_polls = 1 << 22;      // bounded waits give up after this many polls (fault injection: 0)
    // resident blocks per SM of the persistent kernels, by (kernel, dynamic smem)
    struct Occ { const void* fn; int smem; int per_sm; };
    std::vector<Occ> occ;
    // captured multi-step graph
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    std::vector<cudaEvent_t> graph_events;   // per step: 5 events (see pcc_steps_capture)
    int graph_steps = 0;
    unsigned long long graph_kernels = 0;    // kernel nodes per launch of the graph
};

namespace pcc {

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
int ensure_scratch(pcc_ctx* ctx, size_t bytes);
// Count kernel launches enqueued by the library (read by pcc_launch_count).
void note_launches(unsigned long long n);
unsigned long long launches_so_far();

// Table geometry passed to kernels by value.
struct TableGeom {
    int n_rows, n_cols;
    double T_min, T_max;   // row variable range
    double ln_T_min, inv_dln_row;
    double ln_x_min;       // Brems column floor (log)
    double ln_tri_min;     // Trident pair column floor (log)
    float f_ln_T_min, f_inv_dln_row, f_ln_x_min, f_ln_tri_min;
};
TableGeom make_geom(const pcc_table_spec& s);

}  // namespace pcc

// Buffers and launch geometry of a pcc_collide call with these arguments,
// set up ahead (allocations, occupancy queries) so the call itself can be
// captured into a graph.
int collide_prepare(pcc_ctx* ctx, const pcc_cells* cells, const pcc_species* em, const pcc_species* ep,
                    const pcc_species* ph, const pcc_species* ion, unsigned mask, int precision);
// The work of pcc_collide on stream st.  After the kernels of group g
// (0 e-, 1 e+, 2 photons) are enqueued, whether or not the group runs,
// after_group(user, g) is called if given, so that a caller can record
// events between the groups; a non-zero return ends the call with it.  The
// batched path sorts the cells of every group that runs by size class
// before the first group.
int collide_groups(pcc_ctx* ctx, const pcc_cells* cells, pcc_species* em, pcc_species* ep, pcc_species* ph,
                   const pcc_species* ion, double dt, uint64_t seed, uint64_t step, unsigned mask, int precision,
                   float* ledger, cudaStream_t st, int (*after_group)(void* user, int group), void* user);
void pcc_free_graph(pcc_ctx* ctx);
