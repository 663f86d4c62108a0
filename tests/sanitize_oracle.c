/*
 * Native driver for the FP64 oracle, compiled by the CPU test suite with
 * AddressSanitizer and UndefinedBehaviorSanitizer.  It runs every entry
 * point of the oracle over small inputs that reach its edges: both
 * screening modes, both nonrelativistic momentum-transfer bounds, a
 * two-material table set, empty cells, a single-particle cell, ragged
 * counts, cells without ions, energies above the table, photons, and
 * several steps with appended secondaries.  Any out-of-bounds access,
 * use of freed memory, leak, signed overflow, misaligned access or
 * undefined shift aborts with a sanitizer report and a non-zero status.
 *
 * Test infrastructure only: it links the oracle and nothing else.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "pcc_oracle.h"

/* SplitMix64: this program's own input generator (Steele et al., 2014). */
static uint64_t sm_state = 0x9E3779B97F4A7C15ull;
static uint64_t sm_next(void)
{
    uint64_t z = (sm_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double sm_u01(void) { return ((double)(sm_next() >> 11) + 0.5) * 0x1.0p-53; }

static int failures = 0;
#define CHECK(cond, ...)                                                   \
    do {                                                                   \
        if (!(cond)) {                                                     \
            fprintf(stderr, "check failed (%s:%d): ", __FILE__, __LINE__); \
            fprintf(stderr, __VA_ARGS__);                                  \
            fputc('\n', stderr);                                           \
            ++failures;                                                    \
        }                                                                  \
    } while (0)

static void *xcalloc(size_t n, size_t sz)
{
    void *p = calloc(n ? n : 1, sz);
    if (!p) {
        fprintf(stderr, "out of memory\n");
        exit(3);
    }
    return p;
}

static void species_alloc(orc_species *s, int cap, int with_x)
{
    memset(s, 0, sizeof *s);
    s->cap = cap;
    s->ux = xcalloc((size_t)cap, sizeof(float));
    s->uy = xcalloc((size_t)cap, sizeof(float));
    s->uz = xcalloc((size_t)cap, sizeof(float));
    s->w = xcalloc((size_t)cap, sizeof(float));
    s->x = with_x ? xcalloc((size_t)cap, sizeof(float)) : NULL;
    s->pid = xcalloc((size_t)cap, sizeof(uint64_t));
    s->cell = xcalloc((size_t)cap, sizeof(int32_t));
}

static void species_free(orc_species *s)
{
    free(s->ux); free(s->uy); free(s->uz); free(s->w); free(s->x); free(s->pid); free(s->cell);
    memset(s, 0, sizeof *s);
}

/* Appends one particle with an isotropic momentum of magnitude |u|. */
static void push(orc_species *s, int cell, double umag, double w, uint64_t pid)
{
    if (s->n >= s->cap) return;
    double c = 2.0 * sm_u01() - 1.0, ph = 6.283185307179586 * sm_u01();
    double sn = sqrt(1.0 - c * c);
    int i = s->n++;
    s->ux[i] = (float)(umag * sn * cos(ph));
    s->uy[i] = (float)(umag * sn * sin(ph));
    s->uz[i] = (float)(umag * c);
    s->w[i] = (float)w;
    if (s->x) s->x[i] = (float)sm_u01();
    s->pid[i] = pid;
    s->cell[i] = cell;
}

static int tables_alloc_build(orc_tables *t, const orc_material *mats, int n_mat, orc_table_spec sp)
{
    size_t R = (size_t)sp.n_rows, Cn = (size_t)sp.n_cols;
    memset(t, 0, sizeof *t);
    t->spec = sp;
    t->n_mat = n_mat;
    t->scr = xcalloc((size_t)n_mat, sizeof(orc_screening));
    for (int m = 0; m < n_mat; ++m) orc_screening_prep(&mats[m], &t->scr[m]);
    t->brems_sigma = xcalloc((size_t)n_mat * R, sizeof(double));
    t->brems_cdf = xcalloc((size_t)n_mat * R * Cn, sizeof(double));
    t->bh_sigma = xcalloc((size_t)n_mat * R, sizeof(double));
    t->bh_cdf = xcalloc((size_t)n_mat * R * Cn, sizeof(double));
    t->tri_gp_cdf = xcalloc(R * Cn, sizeof(double));
    t->tri_split_cdf = xcalloc(R * Cn, sizeof(double));
    return orc_tables_build(t);
}

static void tables_free(orc_tables *t)
{
    free(t->scr); free(t->brems_sigma); free(t->brems_cdf); free(t->bh_sigma); free(t->bh_cdf);
    free(t->tri_gp_cdf); free(t->tri_split_cdf);
    memset(t, 0, sizeof *t);
}

static int all_finite(const double *a, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!isfinite(a[i])) return 0;
    return 1;
}

static orc_table_spec make_spec(int rows, int cols, int nr_qbounds, int screening)
{
    orc_table_spec sp;
    memset(&sp, 0, sizeof sp);
    sp.n_rows = rows;
    sp.n_cols = cols;
    sp.quad_nodes = 8;
    sp.T_min = 0.002;
    sp.T_max = 1999.0;
    sp.x_min = 1e-7;
    sp.tri_y_min = 1e-5;
    sp.nr_qbounds = nr_qbounds;
    sp.screening = screening;
    return sp;
}

/* One multi-step run on a small ragged population; returns the number of
 * secondaries created.  The middle step is so long that every pair collides
 * (ORC_ST_PROB_LARGE); a small photon capacity makes the appends overflow
 * (ORC_ST_CAPACITY), which the step reports as an error. */
static double run_steps(const orc_tables *t, int with_x, int ph_cap, uint64_t seed)
{
    enum { NCELL = 7, STEPS = 3 };
    /* per-cell counts: an empty cell, a single electron, ragged counts, a
     * cell without ions, and a cell of fast electrons above the table */
    static const int n_em[NCELL] = {0, 1, 5, 9, 4, 6, 3};
    static const int n_ep[NCELL] = {2, 0, 3, 1, 0, 2, 1};
    static const int n_ph[NCELL] = {1, 0, 4, 0, 3, 2, 2};
    static const int n_io[NCELL] = {3, 2, 4, 0, 1, 2, 3};
    int32_t mat[NCELL];
    orc_species em, ep, ph, ion;
    const int cap = 4096;
    species_alloc(&em, cap, with_x);
    species_alloc(&ep, cap, with_x);
    species_alloc(&ph, ph_cap, with_x);
    species_alloc(&ion, 64, with_x);
    uint64_t pid = 1;
    for (int c = 0; c < NCELL; ++c) {
        mat[c] = c % t->n_mat;
        double fast = (c == 6) ? 5000.0 : 1.0;
        /* weights are densities [m^-3]; unequal, so that the weight
         * correction both keeps and drops events */
        for (int i = 0; i < n_em[c]; ++i) push(&em, c, fast * (1.0 + 40.0 * sm_u01()), 1e27 * (0.2 + sm_u01()), pid++);
        for (int i = 0; i < n_ep[c]; ++i) push(&ep, c, 1.0 + 40.0 * sm_u01(), 1e27 * (0.2 + sm_u01()), pid++);
        for (int i = 0; i < n_ph[c]; ++i) push(&ph, c, 5.0 + 200.0 * sm_u01(), 1e27 * (0.2 + sm_u01()), pid++);
        for (int i = 0; i < n_io[c]; ++i) push(&ion, c, 1e-4 * sm_u01(), 2e28 * (0.2 + sm_u01()), pid++);
    }
    double ledger[2 * NCELL];
    memset(ledger, 0, sizeof ledger);
    double created = 0.0;
    unsigned status = 0;
    for (uint64_t s = 0; s < STEPS; ++s) {
        orc_stats st;
        memset(&st, 0, sizeof st);
        double dt = s == 1 ? 1e-9 : 1e-13;
        int rc = orc_step(t, NCELL, mat, &em, &ep, &ph, &ion, 115800.0, dt, seed, s, 7u, ledger, &st);
        CHECK((rc == 0) == !(st.status & ORC_ST_CAPACITY), "orc_step returned %d with status %u", rc, st.status);
        status |= st.status;
        for (int k = 0; k < 5; ++k) {
            CHECK(st.created[k] <= st.accepted[k], "created > accepted");
            created += st.created[k];
        }
        CHECK(em.n <= em.cap && ep.n <= ep.cap && ph.n <= ph.cap, "population above capacity");
    }
    CHECK(status & ORC_ST_PROB_LARGE, "the long step must set ORC_ST_PROB_LARGE");
    CHECK(status & ORC_ST_TABLE_RANGE, "electrons above the table must set ORC_ST_TABLE_RANGE");
    CHECK(((status & ORC_ST_CAPACITY) != 0) == (ph_cap < 256), "capacity status (cap %d)", ph_cap);
    CHECK(all_finite(ledger, 2 * NCELL), "ledger not finite");
    for (int i = 0; i < em.n; ++i) CHECK(em.cell[i] >= 0 && em.cell[i] < NCELL, "electron cell out of range");
    for (int i = 0; i < ph.n; ++i) CHECK(isfinite(ph.ux[i]) && isfinite(ph.w[i]), "photon not finite");
    species_free(&em);
    species_free(&ep);
    species_free(&ph);
    species_free(&ion);
    return created;
}

int main(void)
{
    orc_material mats[2] = {
        {29, 5.0, 8.5e28, 100.0, 1.0, 1.0},   /* solid Cu, warm */
        {79, 0.0, 5.9e28, 0.0, 1.0, 1.0},     /* neutral cold Au: no Debye term */
    };

    /* the scalar physics entry points, at and near their edges */
    CHECK(isnan(orc_lambert_w0(-1.0)), "W0 below -1/e must be NaN");
    CHECK(orc_lambert_w0(0.0) == 0.0, "W0(0)");
    CHECK(fabs(orc_lambert_w0(1e300) - 684.71) < 1.0, "W0 of a large argument");
    CHECK(fabs(orc_lambert_w0(-0.3678) + 0.9802) < 1e-3, "W0 near the branch point");
    for (int Z = 1; Z <= 92; Z += 13) CHECK(isfinite(orc_fC(Z)), "fC(%d)", Z);
    for (int m = 0; m < 2; ++m) {
        orc_screening s;
        orc_screening_prep(&mats[m], &s);
        CHECK(s.LTF > 0.0 && s.LR > 0.0 && isfinite(s.ITFD), "screening of material %d", m);
        for (int q = 0; q < 2; ++q) {
            s.tfd_quad = q;
            for (double g = 1.001; g < 3000.0; g *= 3.7) {
                double k = 0.3 * (g - 1.0);
                CHECK(isfinite(orc_dsdk_brems(&s, g, k, ORC_NR_EXACT)), "brems");
                CHECK(isfinite(orc_dsdk_brems(&s, g, k, ORC_NR_PRINTED)), "brems printed");
                if (g > 3.0) CHECK(isfinite(orc_dsdg_bh(&s, 2.0 * g, g)), "bh");
                CHECK(isfinite(orc_sigma_trident(mats[m].Z, g + 3.0)), "trident");
            }
            double I1, I2;
            orc_I12_tfd_quad(&s, 1e-3, &I1, &I2);
            CHECK(isfinite(I1) && isfinite(I2), "I12");
        }
        /* equal Thomas-Fermi and Debye lengths: the midpoint limits */
        s.tfd_quad = 0;
        s.LD = s.LTF;
        CHECK(isfinite(orc_I_tfd(s.etaTF, s.LTF, s.etaD, s.LD)), "I_TFD at L_D = L_TF");
        CHECK(isfinite(orc_dsdk_brems_nr(&s, 1.01, 0.004, ORC_NR_EXACT)), "NR brems at L_D = L_TF");
    }
    CHECK(orc_split_shape(0.5, 1.0) >= 0.0, "split shape");
    double gx[64], gw[64];
    for (int n = 1; n <= 64; n *= 2) {
        orc_gauss_legendre(n, gx, gw);
        double sum = 0.0;
        for (int i = 0; i < n; ++i) sum += gw[i];
        CHECK(fabs(sum - 2.0) < 1e-12, "GL(%d) weights sum", n);
    }

    /* random numbers, the exact accept decision and the pairing permutation */
    uint32_t ctr[4] = {1u, 2u, 3u, 4u}, key[2] = {5u, 6u}, out[4];
    orc_philox4x32_10(ctr, key, out);
    CHECK(orc_u01(0u) > 0.0 && orc_u01(0xFFFFFFFFu) < 1.0, "u01 range");
    static const double ps[] = {0.0, 1.0, 2.0, 1e-300, 0x1.0p-32, 1.0 - 0x1.0p-40, 0.5};
    for (size_t i = 0; i < sizeof ps / sizeof ps[0]; ++i) {
        double p = ps[i] > 1.0 ? 1.0 : ps[i];
        uint32_t tie = p >= 1.0 ? 0xFFFFu : (uint32_t)floor(p * 65536.0);
        for (uint32_t c0 = 0; c0 < 4; ++c0) {
            orc_accept(tie, ps[i], 7u + c0, 11u, 99u, 6u << 4, 0xABCDEFull);
            orc_accept((uint32_t)sm_next() & 0xFFFFu, ps[i], 7u + c0, 11u, 99u, 6u << 4, 0xABCDEFull);
        }
    }
    CHECK(orc_accept(0u, 0.0, 0, 0, 0, 0, 0) == 0, "p = 0 accepts");
    CHECK(orc_accept(0xFFFFu, 1.0, 0, 0, 0, 0, 0) == 1, "p = 1 rejects");
    for (uint32_t n = 1; n <= 70; n += 23) {
        uint32_t rk[4] = {(uint32_t)sm_next(), (uint32_t)sm_next(), (uint32_t)sm_next(), (uint32_t)sm_next()};
        for (uint32_t j = 0; j < n; ++j)
            CHECK(orc_perm_pos(orc_perm_elem(j, n, rk), n, rk) == j, "permutation inverse (n=%u)", n);
    }
    double ui[3] = {0.3, -0.2, 0.1}, in4[4] = {2.0, 0.5, 1.0, -1.2}, o4[4], back[4];
    orc_boost(ui, in4, o4, 0);
    orc_boost(ui, o4, back, 1);
    for (int k = 0; k < 4; ++k) CHECK(fabs(back[k] - in4[k]) < 1e-12, "boost round trip");

    /* tables in every mode, the lookups, and multi-step runs */
    for (int mode = 0; mode < 4; ++mode) {
        orc_tables t;
        orc_table_spec sp = make_spec(12 + 5 * mode, 9 + 4 * mode, mode & 1 ? ORC_NR_PRINTED : ORC_NR_EXACT,
                                      mode & 2 ? ORC_SCREEN_TFD_QUAD : ORC_SCREEN_REDUCED);
        int rc = tables_alloc_build(&t, mats, 2, sp);
        CHECK(rc == 0, "tables build (mode %d) returned %d", mode, rc);
        size_t R = (size_t)sp.n_rows, Cn = (size_t)sp.n_cols;
        CHECK(all_finite(t.brems_sigma, 2 * R) && all_finite(t.bh_sigma, 2 * R), "sigma rows");
        CHECK(all_finite(t.brems_cdf, 2 * R * Cn) && all_finite(t.tri_split_cdf, R * Cn), "cdf rows");
        for (int r = 0; r < sp.n_rows; ++r) (void)orc_row_value(&sp, r);
        for (int tb = 0; tb < 4; ++tb)
            for (int c = 0; c < sp.n_cols; ++c) (void)orc_col_value(&sp, tb, c);
        unsigned st = 0;
        for (int i = 0; i < 200; ++i) {
            double r = exp(log(1e-4) + (log(1e5) - log(1e-4)) * sm_u01());   /* below, inside, above */
            (void)orc_sigma_lookup(&sp, t.brems_sigma, r, &st);
            (void)orc_sigma_lookup(&sp, t.bh_sigma + R, r, &st);
            double u1 = i < 2 ? (i ? 1.0 - 1e-16 : 0.0) : sm_u01();
            (void)orc_sample(&sp, 0, t.brems_cdf, r, sm_u01(), u1);
            (void)orc_sample(&sp, 1, t.bh_cdf + R * Cn, r, sm_u01(), u1);
            (void)orc_sample(&sp, 2, t.tri_gp_cdf, r, u1, sm_u01());
            (void)orc_sample(&sp, 3, t.tri_split_cdf, r, sm_u01(), u1);
        }
        CHECK(st != 0, "out-of-table lookups must set a status bit");
        double created = run_steps(&t, mode & 1, mode == 3 ? 16 : 4096, 0x1234ull + (uint64_t)mode);
        CHECK(created > 0.0, "no secondaries in mode %d", mode);
        tables_free(&t);
    }

    /* an invalid spec is refused without touching the arrays */
    {
        orc_tables t;
        orc_table_spec sp = make_spec(1, 1, ORC_NR_EXACT, 7);
        int rc = tables_alloc_build(&t, mats, 1, sp);
        CHECK(rc != 0, "invalid spec accepted");
        tables_free(&t);
    }

    /* the expected-emission operator and its gradient */
    {
        enum { NS = 33 };
        double g[NS], w[NS], o3[3], g3[3] = {1.0, -0.5, 0.25}, grad[5];
        for (int i = 0; i < NS; ++i) {
            g[i] = 1.0 + 100.0 * sm_u01();
            w[i] = sm_u01();
        }
        g[0] = 1.0;   /* at rest: no emission */
        orc_expected_emission(&mats[0], NS, g, w, 16, o3);
        CHECK(all_finite(o3, 3) && o3[0] > 0.0, "expected emission");
        orc_expected_emission(&mats[1], 0, g, w, 200, o3);   /* empty input; n_quad clamped */
        CHECK(o3[0] == 0.0 && o3[1] == 0.0 && o3[2] == 0.0, "empty expected emission");
        orc_expected_emission_grad(&mats[0], NS, g, w, 12, g3, grad);
        CHECK(all_finite(grad, 5), "expected emission gradient");
    }

    if (failures) {
        fprintf(stderr, "%d checks failed\n", failures);
        return 1;
    }
    printf("oracle sanitizer driver: all checks passed\n");
    return 0;
}
