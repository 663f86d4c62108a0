/*
 * FP64 CPU oracle for the pairwise Coulomb-process collision step of
 * Martinez et al., "High-Energy Radiation and Pair Production by Coulomb
 * Processes in Particle-In-Cell Simulations" (arXiv:1907.02814).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares no source,
 * header, helper or constant generator with the CUDA library; the two are
 * written independently from the paper and compared value by value.
 *
 * Everything here is plain, slow C in double precision, single-threaded
 * unless orc_set_threads asks for OpenMP threads over the cells of a group
 * (for timing the CPU baseline; cells are independent, so the result is the
 * same).
 * Particle state is held in the same storage format as the product
 * (float32 momenta and weights, uint64 ids); all arithmetic is FP64.
 *
 * Parity pins: every formula function is pinned by the CPU tests against
 * quadrature of its integral definition, a textbook limit, a closed-form
 * invariant or a value printed in the paper.  The Trident shapes (Sec. II.D)
 * are pinned by limits: the pair-energy spectrum integrates to the
 * Landau-Lifshitz leading-logarithm total at large gamma_1 and rises as the
 * low-energy Bhabha form E_p^3 at threshold; the split CDF equals its exact
 * antiderivative.
 */
#ifndef PCC_ORACLE_H
#define PCC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Plasma state of one material (Sec. II.A): nuclear charge Z, ionization
 * degree Z*, ion density n_i [m^-3], temperature T [eV], and scale factors
 * s_TF, s_D applied to the Thomas-Fermi and Debye lengths (1 = as printed). */
typedef struct {
    int Z;
    double Zstar, n_i, T_e, s_TF, s_D;
} orc_material;

/* Derived screening quantities (lengths normalised by the reduced Compton
 * wavelength r_C = hbar/(m_e c)). */
typedef struct {
    int Z;
    double Zstar;
    double LTF, LD;        /* Eq. (LTF), Eq. (LDH) with the r_i lower bound  */
    double etaTF, etaD;    /* q_TF/q = 1 - Zs/Z and q_D/q = Zs/Z, Zs = Z^* (Eq. V_TFD) */
    double ITFD;           /* Eq. (ITFD)                                     */
    double LR;             /* Eq. (lambert-W)                                */
    double fC;             /* Coulomb correction (Sec. II.B.3)               */
    double lambdaD, ri;    /* unclamped Debye length and ion-sphere radius [m] */
    int tfd_quad;          /* 1: relativistic Brems and BH use I1, I2 of the full
                              TFD potential by quadrature; 0: the reduced L_R  */
} orc_screening;

enum { ORC_NR_EXACT = 0, ORC_NR_PRINTED = 1 };
enum { ORC_SCREEN_REDUCED = 0, ORC_SCREEN_TFD_QUAD = 1 };

typedef struct {
    int n_rows, n_cols, quad_nodes;
    double T_min, T_max;   /* row grid: log-spaced row variable on [T_min, T_max] */
    double x_min;          /* Brems cut-off k/(gamma-1) >= x_min (Sec. III.A)      */
    double tri_y_min;      /* Trident pair-energy column floor                     */
    int nr_qbounds;        /* ORC_NR_EXACT or ORC_NR_PRINTED                       */
    int screening;         /* ORC_SCREEN_REDUCED or ORC_SCREEN_TFD_QUAD            */
} orc_table_spec;

/* Tables; all arrays owned by the caller.
 * brems_sigma[m][r], brems_cdf[m][r][c], bh_sigma[m][r], bh_cdf[m][r][c],
 * tri_gp_cdf[r][c], tri_split_cdf[r][c]. */
typedef struct {
    orc_table_spec spec;
    int n_mat;
    orc_screening *scr;
    double *brems_sigma, *brems_cdf;
    double *bh_sigma, *bh_cdf;
    double *tri_gp_cdf, *tri_split_cdf;
} orc_tables;

/* Mutable particle population (float32 storage, canonical order not assumed). */
typedef struct {
    int n, cap;
    float *ux, *uy, *uz, *w;   /* u = p/(m c); photons: k * direction */
    float *x;                  /* optional 1D position (may be NULL)   */
    uint64_t *pid;
    int32_t *cell;
} orc_species;

typedef struct {
    double pairs[3];        /* macro-collisions per group: e-, e+, gamma      */
    double accepted[5];     /* U1 < P per channel (Brems e-, Brems e+, Tri e-, Tri e+, BH) */
    double created[5];      /* events that passed the weight correction       */
    unsigned status;        /* ORC_ST_* bits                                  */
} orc_stats;

enum { ORC_ST_TABLE_RANGE = 1u, ORC_ST_PROB_LARGE = 2u, ORC_ST_CAPACITY = 4u };
enum { ORC_PROC_BREMS = 1u, ORC_PROC_TRIDENT = 2u, ORC_PROC_BH = 4u };

/* ---- physics (Sec. II) ---- */
void   orc_screening_prep(const orc_material *m, orc_screening *out);
double orc_lambert_w0(double z);
double orc_fC(int Z);
double orc_I1_yukawa(double delta, double L);
double orc_I2_yukawa(double delta, double L);
double orc_I_tfd(double etaTF, double LTF, double etaD, double LD);
void   orc_I12_tfd_quad(const orc_screening *s, double delta, double *I1, double *I2);
double orc_dsdk_brems(const orc_screening *s, double gamma1, double k, int nr_qbounds);
double orc_dsdk_brems_nr(const orc_screening *s, double gamma1, double k, int nr_qbounds);
double orc_dsdk_brems_rel(const orc_screening *s, double gamma1, double k, double fc);
double orc_dsdg_bh(const orc_screening *s, double k, double gplus);
double orc_sigma_trident(int Z, double gamma1);
double orc_dsdgp_trident(int Z, double gamma1, double gp);
double orc_split_shape(double gp, double gplus);

/* ---- quadrature and tables ---- */
void   orc_gauss_legendre(int n, double *x, double *w);
double orc_row_value(const orc_table_spec *sp, int r);
double orc_col_value(const orc_table_spec *sp, int table, int c);
int    orc_tables_build(orc_tables *t);

/* ---- random numbers and pairing ---- */
void     orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double   orc_u01(uint32_t r);
/* U < p for U = (2^48 a + e + 1/2) 2^-64: a the 16-bit first digit, e the
 * 48-bit rest from words 0, 1 of the draw (c0, cell, step, tag), read only
 * on a tie a = floor(2^16 p). */
int      orc_accept(uint32_t a, double p, uint32_t c0, uint32_t cell, uint64_t step, uint32_t tag, uint64_t seed);
uint32_t orc_perm_pos(uint32_t s, uint32_t n, const uint32_t rk[4]);   /* P^-1(s) */
uint32_t orc_perm_elem(uint32_t j, uint32_t n, const uint32_t rk[4]);  /* P(j)    */

/* ---- table lookups (used by the step) ---- */
double orc_sigma_lookup(const orc_table_spec *sp, const double *sigma_row, double r, unsigned *status);
double orc_sample(const orc_table_spec *sp, int table, const double *cdf, double r,
                  double u_row, double u_col);

/* ---- Lorentz transform to/from an ion rest frame (Sec. III.A) ---- */
void orc_boost(const double ui[3], const double in[4], double out[4], int inverse);

/* ---- the collision step (Sec. III.A) ---- */
/* Threads over the cells of a group (OpenMP builds only; timing only, the
 * result does not depend on it).  Default 1. */
void orc_set_threads(int n);
int  orc_get_threads(void);
int orc_step(const orc_tables *t, int n_cells, const int32_t *material_of_cell,
             orc_species *em, orc_species *ep, orc_species *ph, const orc_species *ion,
             double ion_mass, double dt, uint64_t seed, uint64_t step, unsigned mask,
             double *ledger /* [n_cells][2] accumulated */, orc_stats *st);

/* ---- expected-emission operator (Eq. N_br_theo1/2 rate form) ---- */
void orc_expected_emission(const orc_material *m, int n_samples, const double *gamma,
                           const double *w, int n_quad, double *out3);
void orc_expected_emission_grad(const orc_material *m, int n_samples, const double *gamma,
                                const double *w, int n_quad, const double *g_out, double *grad5);
/* The same gradient by the chain rule written out by hand: d/dL of the
 * reduced screening functions, the partials of I_TFD and of the NR cross
 * term, the implicit Lambert-W derivative dL_R/da, and the Jacobian of
 * (L_TF, L_D, eta_D, L_R) with respect to theta.  At Z* = 0 the Z*
 * derivative is the limit from Z* > 0 (lambda_D -> infinity). */
void orc_expected_emission_grad_analytic(const orc_material *m, int n_samples, const double *gamma,
                                         const double *w, int n_quad, const double *g_out, double *grad5);
void orc_dI12_dL(double delta, double L, double *dI1, double *dI2);
void orc_dsdk_brems_grad(const orc_material *m, double gamma1, double k, double out4[4]);
void orc_screening_jacobian(const orc_material *m, double jac20[20]);

#ifdef __cplusplus
}
#endif
#endif
