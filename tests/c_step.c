/*
 * A full collision step driven from plain C through include/pcc.h, checked
 * against the FP64 oracle linked into the same program.  It shows the
 * boundary is usable without Python: the caller owns the device arrays
 * (cudaMalloc), bins each species, builds the tables, runs three steps on
 * the FP64 plain path (every process, then Trident alone and Bethe-Heitler
 * alone with longer steps), commits the secondaries after each and reads
 * the status.  The oracle steps the same host particles; the status, the
 * step counters and the identifiers and weights of every live particle
 * must agree exactly (the plain path takes the oracle's decisions), the
 * momenta to float32 storage.
 *
 * Test infrastructure: built and run by tests/test_gpu_c_step.py on a GPU.
 * Exit status 0 on agreement, 1 on a mismatch, 2 when a call fails.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "pcc.h"
#include "pcc_oracle.h"

enum { NCELL = 16, NSPEC = 4 };

static uint64_t sm_state = 0x243F6A8885A308D3ull;
static uint64_t sm_next(void)   /* SplitMix64 (Steele et al., 2014) */
{
    uint64_t z = (sm_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double sm_u01(void) { return ((double)(sm_next() >> 11) + 0.5) * 0x1.0p-53; }

#define CALL(x)                                                                            \
    do {                                                                                   \
        int rc_ = (x);                                                                     \
        if (rc_ != 0) {                                                                    \
            fprintf(stderr, "%s:%d: %s -> %d (%s)\n", __FILE__, __LINE__, #x, rc_, pcc_last_error()); \
            exit(2);                                                                       \
        }                                                                                  \
    } while (0)
#define CU(x)                                                                              \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) {                                                           \
            fprintf(stderr, "%s:%d: %s -> %s\n", __FILE__, __LINE__, #x, cudaGetErrorString(e_)); \
            exit(2);                                                                       \
        }                                                                                  \
    } while (0)

/* Host particles of one species. */
typedef struct {
    int n, cap;
    float *ux, *uy, *uz, *w;
    uint64_t *pid;
    int32_t *cell;
} host_sp;

static void *xmalloc(size_t n)
{
    void *p = calloc(n ? n : 1, 1);
    if (!p) exit(2);
    return p;
}

static void hs_alloc(host_sp *s, int cap)
{
    s->n = 0;
    s->cap = cap;
    s->ux = xmalloc(sizeof(float) * (size_t)cap);
    s->uy = xmalloc(sizeof(float) * (size_t)cap);
    s->uz = xmalloc(sizeof(float) * (size_t)cap);
    s->w = xmalloc(sizeof(float) * (size_t)cap);
    s->pid = xmalloc(sizeof(uint64_t) * (size_t)cap);
    s->cell = xmalloc(sizeof(int32_t) * (size_t)cap);
}

static void hs_push(host_sp *s, int cell, double umag, double w, uint64_t pid)
{
    double c = 2.0 * sm_u01() - 1.0, ph = 6.283185307179586 * sm_u01(), sn = sqrt(1.0 - c * c);
    int i = s->n++;
    s->ux[i] = (float)(umag * sn * cos(ph));
    s->uy[i] = (float)(umag * sn * sin(ph));
    s->uz[i] = (float)(umag * c);
    s->w[i] = (float)w;
    s->pid[i] = pid;
    s->cell[i] = cell;
}

static void *dcopy(const void *h, size_t bytes)
{
    void *d = NULL;
    CU(cudaMalloc(&d, bytes ? bytes : 16));
    if (bytes) CU(cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice));
    return d;
}

static void *dzero(size_t bytes)
{
    void *d = NULL;
    CU(cudaMalloc(&d, bytes ? bytes : 16));
    CU(cudaMemset(d, 0, bytes ? bytes : 16));
    return d;
}

/* Bin one host species into a device species of `cap` slots. */
static void bin_species(pcc_ctx *ctx, const host_sp *h, pcc_species *d, int cap)
{
    size_t n = (size_t)h->n;
    pcc_particles in;
    memset(&in, 0, sizeof in);
    in.n = h->n;
    in.ux = dcopy(h->ux, 4 * n);
    in.uy = dcopy(h->uy, 4 * n);
    in.uz = dcopy(h->uz, 4 * n);
    in.w = dcopy(h->w, 4 * n);
    in.pid = dcopy(h->pid, 8 * n);
    in.cell = dcopy(h->cell, 4 * n);
    memset(d, 0, sizeof *d);
    d->capacity = cap;
    d->ux = dzero(4 * (size_t)cap);
    d->uy = dzero(4 * (size_t)cap);
    d->uz = dzero(4 * (size_t)cap);
    d->w = dzero(4 * (size_t)cap);
    d->pid = dzero(8 * (size_t)cap);
    d->cell_start = dzero(4 * (NCELL + 1));
    d->cell_count = dzero(4 * NCELL);
    d->cell_added = dzero(4 * NCELL);
    CALL(pcc_bin(ctx, &in, NCELL, d, 64, 1.0, NULL));
    cudaFree((void *)in.ux); cudaFree((void *)in.uy); cudaFree((void *)in.uz); cudaFree((void *)in.w);
    cudaFree((void *)in.pid); cudaFree((void *)in.cell);
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

/* Live particles of a device species, sorted by pid: pid, |u|, w. */
typedef struct { uint64_t pid; float u2, w; } rec;
static int cmp_rec(const void *a, const void *b) { return cmp_u64(&((const rec *)a)->pid, &((const rec *)b)->pid); }

static int live_device(const pcc_species *d, rec **out)
{
    int start[NCELL + 1], count[NCELL];
    CU(cudaMemcpy(start, d->cell_start, sizeof start, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(count, d->cell_count, sizeof count, cudaMemcpyDeviceToHost));
    size_t cap = (size_t)d->capacity;
    float *ux = xmalloc(4 * cap), *uy = xmalloc(4 * cap), *uz = xmalloc(4 * cap), *w = xmalloc(4 * cap);
    uint64_t *pid = xmalloc(8 * cap);
    CU(cudaMemcpy(ux, d->ux, 4 * cap, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(uy, d->uy, 4 * cap, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(uz, d->uz, 4 * cap, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(w, d->w, 4 * cap, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(pid, d->pid, 8 * cap, cudaMemcpyDeviceToHost));
    int n = 0;
    for (int c = 0; c < NCELL; ++c) n += count[c];
    rec *r = xmalloc(sizeof(rec) * (size_t)(n + 1));
    int k = 0;
    for (int c = 0; c < NCELL; ++c)
        for (int i = start[c]; i < start[c] + count[c]; ++i) {
            r[k].pid = pid[i];
            r[k].u2 = ux[i] * ux[i] + uy[i] * uy[i] + uz[i] * uz[i];
            r[k].w = w[i];
            ++k;
        }
    qsort(r, (size_t)n, sizeof(rec), cmp_rec);
    free(ux); free(uy); free(uz); free(w); free(pid);
    *out = r;
    return n;
}

static int live_oracle(const orc_species *s, rec **out)
{
    rec *r = xmalloc(sizeof(rec) * (size_t)(s->n + 1));
    for (int i = 0; i < s->n; ++i) {
        r[i].pid = s->pid[i];
        r[i].u2 = s->ux[i] * s->ux[i] + s->uy[i] * s->uy[i] + s->uz[i] * s->uz[i];
        r[i].w = s->w[i];
    }
    qsort(r, (size_t)s->n, sizeof(rec), cmp_rec);
    *out = r;
    return s->n;
}

int main(void)
{
    /* ---- synthetic input: solid Cu, ragged cells, e-, photons, ions ---- */
    const double n_i = 8.5e28;
    host_sp h[NSPEC];   /* em, ep, ph, ion */
    for (int k = 0; k < NSPEC; ++k) hs_alloc(&h[k], 4096);
    uint64_t pid = 1;
    for (int c = 0; c < NCELL; ++c) {
        int ne = 8 + 5 * c, ng = c % 5 == 0 ? 0 : 3 + c, ni = 4 + (c * 7) % 13;
        for (int i = 0; i < ne; ++i) {
            double T = -20.0 * log(sm_u01()) + 0.5;   /* exponential, mean ~10 MeV */
            hs_push(&h[0], c, sqrt(T * (T + 2.0)), n_i / 48.0 * (0.5 + sm_u01()), pid++);
        }
        for (int i = 0; i < ng; ++i) hs_push(&h[2], c, 3.0 + 60.0 * sm_u01(), n_i / 48.0, pid++);
        for (int i = 0; i < ni; ++i) hs_push(&h[3], c, 0.0, n_i / ni, pid++);
    }
    const double dt = 300e-15, ion_mass = 115800.0;
    const uint64_t seed = 0xC0FFEEull, step = 7;
    int32_t mat[NCELL];
    for (int c = 0; c < NCELL; ++c) mat[c] = 0;

    /* ---- GPU through the C ABI ---- */
    pcc_ctx *ctx = NULL;
    CALL(pcc_create(&ctx, 0));
    pcc_material m = {29, 5.0, n_i, 100.0, 1.0, 1.0};
    pcc_table_spec spec = {64, 64, 8, 1.002, 2000.0, 7, 1e-5, 0, PCC_SCREEN_REDUCED};
    CALL(pcc_tables_build(ctx, &m, 1, &spec, NULL));
    pcc_species d[NSPEC];
    for (int k = 0; k < NSPEC; ++k) bin_species(ctx, &h[k], &d[k], h[k].n + 64 * NCELL + 2 * h[k].n);
    pcc_cells cells = {NCELL, dcopy(mat, sizeof mat), ion_mass};

    /* ---- the oracle's tables ---- */
    orc_material om = {29, 5.0, n_i, 100.0, 1.0, 1.0};
    orc_tables t;
    memset(&t, 0, sizeof t);
    orc_table_spec osp = {64, 64, 8, 1.002 - 1.0, 2000.0 - 1.0, 1e-7, 1e-5, ORC_NR_EXACT, ORC_SCREEN_REDUCED};
    t.spec = osp;
    t.n_mat = 1;
    orc_screening scr;
    orc_screening_prep(&om, &scr);
    t.scr = &scr;
    t.brems_sigma = xmalloc(8 * 64); t.brems_cdf = xmalloc(8 * 64 * 64);
    t.bh_sigma = xmalloc(8 * 64); t.bh_cdf = xmalloc(8 * 64 * 64);
    t.tri_gp_cdf = xmalloc(8 * 64 * 64); t.tri_split_cdf = xmalloc(8 * 64 * 64);
    if (orc_tables_build(&t) != 0) return 2;
    orc_species os[NSPEC];
    for (int k = 0; k < NSPEC; ++k) {
        os[k].n = h[k].n; os[k].cap = h[k].cap;
        os[k].ux = h[k].ux; os[k].uy = h[k].uy; os[k].uz = h[k].uz; os[k].w = h[k].w;
        os[k].x = NULL; os[k].pid = h[k].pid; os[k].cell = h[k].cell;
    }
    double ledger[2 * NCELL];
    memset(ledger, 0, sizeof ledger);

    /* ---- three steps on both sides: every process, then Trident alone and
     * BH alone with steps long enough for their rarer events ---- */
    const unsigned masks[3] = {PCC_BREMS | PCC_TRIDENT | PCC_BH, PCC_TRIDENT, PCC_BH};
    const unsigned omasks[3] = {ORC_PROC_BREMS | ORC_PROC_TRIDENT | ORC_PROC_BH, ORC_PROC_TRIDENT, ORC_PROC_BH};
    const double dts[3] = {dt, 1e-9, 3e-11};
    int bad = 0;
    double created[5] = {0, 0, 0, 0, 0};
    for (int s = 0; s < 3; ++s) {
        CALL(pcc_collide(ctx, &cells, &d[0], &d[1], &d[2], &d[3], dts[s], seed, step + (uint64_t)s, masks[s],
                         PCC_FP64_PLAIN, NULL, NULL));
        for (int k = 0; k < 3; ++k) CALL(pcc_append_secondaries(ctx, NCELL, &d[k], NULL));
        unsigned status = 0;
        pcc_stats gs;
        CALL(pcc_read_status(ctx, &status, &gs, NULL));
        orc_stats ost;
        memset(&ost, 0, sizeof ost);
        if (orc_step(&t, NCELL, mat, &os[0], &os[1], &os[2], &os[3], ion_mass, dts[s], seed, step + (uint64_t)s,
                     omasks[s], ledger, &ost) != 0) return 2;
        if (status != ost.status) { fprintf(stderr, "step %d: status %u vs oracle %u\n", s, status, ost.status); ++bad; }
        for (int g = 0; g < 3; ++g)
            if ((double)gs.pairs[g] != ost.pairs[g]) { fprintf(stderr, "step %d: pairs[%d]\n", s, g); ++bad; }
        for (int c = 0; c < 5; ++c) {
            created[c] += ost.created[c];
            if ((double)gs.accepted[c] != ost.accepted[c] || (double)gs.created[c] != ost.created[c]) {
                fprintf(stderr, "step %d channel %d: accepted %llu/%g created %llu/%g\n", s, c, gs.accepted[c],
                        ost.accepted[c], gs.created[c], ost.created[c]);
                ++bad;
            }
        }
    }

    /* ---- the live particles after the three steps ---- */
    for (int k = 0; k < 3; ++k) {
        rec *a, *b;
        int na = live_device(&d[k], &a), nb = live_oracle(&os[k], &b);
        if (na != nb) { fprintf(stderr, "species %d: %d live vs oracle %d\n", k, na, nb); ++bad; }
        for (int i = 0; i < na && i < nb; ++i) {
            if (a[i].pid != b[i].pid || a[i].w != b[i].w ||
                fabs((double)a[i].u2 - (double)b[i].u2) > 5e-6 * ((double)b[i].u2 + 1.0)) {
                fprintf(stderr, "species %d particle %d differs\n", k, i);
                ++bad;
                break;
            }
        }
        free(a); free(b);
    }
    printf("created: Brems %g + %g, Trident %g + %g, BH %g\n", created[0], created[1], created[2], created[3],
           created[4]);
    if (created[0] < 20 || created[2] < 5 || created[4] < 5) { fprintf(stderr, "too few events to compare\n"); ++bad; }
    pcc_destroy(ctx);
    if (bad) return 1;
    printf("C step matches the oracle\n");
    return 0;
}
