/*
 * pcc.h -- C ABI of the GB300 (sm_103a) pairwise Coulomb-process collision
 * library: the per-cell, per-step Monte Carlo Bremsstrahlung, Bethe-Heitler
 * and Coulomb-Trident step for weighted PIC macro-particles of
 * B. Martinez et al., arXiv:1907.02814.
 *
 * Conventions
 *   - Momenta are proper velocities u = p/(m c) in float32 (photons store
 *     k * direction with k in m_e c^2); weights W are densities in m^-3, so
 *     that the density of a species in a cell is the sum of its weights
 *     (Sec. III.A); times in seconds; lengths in metres.
 *   - Every pointer inside a struct or argument marked "device" is CUDA
 *     device memory owned by the caller; the library never frees it.
 *   - Every entry point returns a pcc_status code synchronously for argument
 *     and launch errors.  Conditions found on the device (capacity, table
 *     range, non-finite values, a wait that gave up) set bits of a sticky
 *     device status word read by pcc_read_status().
 *   - Work is enqueued on the given CUDA stream (cudaStream_t passed as
 *     void*, NULL = default stream); calls are asynchronous unless stated.
 */
#ifndef PCC_H
#define PCC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcc_ctx pcc_ctx;

typedef enum {
    PCC_OK = 0,
    PCC_E_INVALID = 1,      /* bad argument (message in pcc_last_error)        */
    PCC_E_CUDA = 2,         /* a CUDA runtime call failed                       */
    PCC_E_CAPACITY = 3,     /* a buffer or supported size is too small          */
    PCC_E_NO_TABLES = 4     /* pcc_collide before pcc_tables_build              */
} pcc_status;

/* Bits of the device status word (pcc_read_status). */
#define PCC_ST_TABLE_RANGE 0x1u   /* an energy above the table; the last row was used   */
#define PCC_ST_PROB_LARGE  0x2u   /* a pair had n sigma v dt > 1 (time step too long)   */
#define PCC_ST_CAPACITY    0x4u   /* a cell region overflowed; the secondary was dropped */
#define PCC_ST_NONFINITE   0x8u   /* a non-finite momentum, or a cell or material index
                                     out of range, was met; that item was skipped       */
#define PCC_ST_ID_RANGE    0x10u  /* cell >= 2^24, step >= 2^19 or > 65536 pairs per cell:
                                     secondary identifiers are no longer unique          */
#define PCC_ST_TIMEOUT     0x20u  /* a bounded wait (bulk copy barrier) gave up          */
#define PCC_ST_BOUND_RANGE 0x40u  /* batched path only: an evaluated pair had an ion-frame
                                     Lorentz factor above 1e7, where the Trident bound of
                                     the quick reject is no longer proven, so pairs of that
                                     energy may have been rejected without evaluation     */

typedef enum { PCC_FP64_PLAIN = 0, PCC_FP32_BATCHED = 1 } pcc_precision;

/* Process mask bits for pcc_collide.  The group bits restrict a call to
 * the electron-ion, positron-ion or photon-ion pairs; when none of them is
 * set, every group runs. */
#define PCC_BREMS    0x1u
#define PCC_TRIDENT  0x2u
#define PCC_BH       0x4u
#define PCC_GROUP_EM 0x100u
#define PCC_GROUP_EP 0x200u
#define PCC_GROUP_PH 0x400u

/* Plasma state of one material (Sec. II.A): nuclear charge Z, ionization
 * degree Zstar (an input: the paper's More fit is not given), ion density
 * n_i [m^-3], temperature T_e [eV], and factors s_TF, s_D multiplying the
 * Thomas-Fermi (Eq. LTF) and Debye (Eq. LDH, lower bound r_i) lengths
 * (1 for the paper's model). */
typedef struct {
    int Z;
    double Zstar, n_i, T_e, s_TF, s_D;
} pcc_material;

/* Table layout (Sec. III.A: tabulated cross sections, inverse CDF).
 * Rows: the row variable (Brems gamma-1, BH k-2, Trident gamma_1-3,
 * Trident split gamma_p-2) log-spaced on [gamma_min-1, gamma_max-1].
 * Columns: Brems x = k/(gamma-1) log-spaced on [10^-cutoff_exp, 1]; BH and
 * split y linear on [0, 1]; Trident pair energy y = (gamma_p-2)/(gamma_1-3)
 * log-spaced on [tri_y_min, 1].  quad_nodes Gauss-Legendre points per
 * column interval.  nr_qbounds 0: momentum-transfer bounds p1 +/- p2;
 * 1: the printed 2 p1 - k and k (Sec. II.B.1).  screening: the screening
 * functions I1, I2 (Eqs. defphi1, defphi2) of the relativistic Brems
 * regimes (Eqs. csre, csur) and of Bethe-Heitler (Eq. dsdkbh);
 * PCC_SCREEN_REDUCED takes the closed forms (Eqs. deriv_I1, deriv_I2) of the
 * reduced single-Yukawa potential at L_R (Eq. lambert-W), as the paper's
 * code does; PCC_SCREEN_TFD_QUAD integrates them numerically with the form
 * factor (Eq. defF) of the full Thomas-Fermi-Debye potential (Eq. V_TFD),
 * the reference the paper compares the reduced formula with (Sec. II.B.2-3,
 * Sec. II.C).  The non-relativistic regime uses the full potential in both. */
enum { PCC_SCREEN_REDUCED = 0, PCC_SCREEN_TFD_QUAD = 1 };
typedef struct {
    int n_rows, n_cols, quad_nodes;
    double gamma_min, gamma_max;
    int cutoff_exp;
    double tri_y_min;
    int nr_qbounds;
    int screening;          /* PCC_SCREEN_REDUCED or PCC_SCREEN_TFD_QUAD */
} pcc_table_spec;

/* One species in cell-region layout (all device memory, caller-owned).
 * Cell c owns slots [cell_start[c], cell_start[c+1]); its live particles
 * are the first cell_count[c] slots, in ascending pid order.  Secondaries
 * created during a step are appended after them (cell_added[c]) and become
 * live at pcc_append_secondaries.  x may be NULL.  capacity = total slots. */
typedef struct {
    float *ux, *uy, *uz, *w;
    float *x;
    uint64_t *pid;
    int *cell_start;      /* [n_cells + 1] */
    int *cell_count;      /* [n_cells]     */
    int *cell_added;      /* [n_cells]     */
    int capacity;
} pcc_species;

/* Unsorted input particles for pcc_bin (device memory, caller-owned). */
typedef struct {
    int n;
    const float *ux, *uy, *uz, *w;
    const float *x;       /* may be NULL */
    const uint64_t *pid;  /* unique within the species, < 2^63 */
    const int *cell;      /* cell index in [0, n_cells) */
} pcc_particles;

/* Cells: count, material index per cell (device, [n_cells]) and the ion
 * mass in electron masses. */
typedef struct {
    int n_cells;
    const int *material_of_cell;
    double ion_mass;
} pcc_cells;

/* Step counters read back by pcc_read_status (host struct). */
typedef struct {
    unsigned long long pairs[3];     /* macro-collisions: e-, e+, photon groups        */
    unsigned long long accepted[5];  /* U1 < P per channel: Brems e-, Brems e+,
                                        Trident e-, Trident e+, Bethe-Heitler          */
    unsigned long long created[5];   /* events kept by the weight correction          */
    double energy_change;            /* sum over events of W (E_out - E_in), m_e c^2 m^-3 */
    double charge_change;            /* sum over events of W (q_out - q_in), e m^-3        */
    unsigned long long candidates[3];/* batched path: pairs whose accept digit fell below
                                        the per-material bound, evaluated in full        */
} pcc_stats;

/* Library version string and the message of the last synchronous error
 * (thread-local; empty when none). */
const char *pcc_version(void);
const char *pcc_last_error(void);

/* Name and one-line meaning of a return code ("PCC_E_CAPACITY: ...");
 * "unknown return code" for any value outside pcc_status.  Static storage,
 * never NULL, needs no device. */
const char *pcc_status_string(int code);

/* Name of one bit of the device status word ("PCC_ST_TIMEOUT");
 * "unknown status bit" unless exactly one PCC_ST_* bit is set.  Static
 * storage, never NULL, needs no device. */
const char *pcc_status_bit_string(unsigned bit);

/* Create a context on CUDA device `device`; it owns the tables, the device
 * status word, step counters and scratch buffers.  Returns PCC_E_CUDA when
 * the device is unusable.  Destroy with pcc_destroy (NULL is accepted). */
int  pcc_create(pcc_ctx **out, int device);
void pcc_destroy(pcc_ctx *ctx);

/* Material preparation and table build, in FP64 on the GPU (Sec. II):
 * screening lengths (Eq. LTF, LDH with r_i), weights (Eq. V_TFD), I_TFD
 * (Eq. ITFD), the reduced length (Eq. reduit, lambert-W), f_C (Sec. II.B.3),
 * then per material the Brems cross section sigma_B and its inverse-CDF
 * table (Eq. cs_br_nr with the Elwert factor, Eq. csre, Eq. csur with the
 * reduced I1, I2 of Eq. deriv_I1/I2) and the Bethe-Heitler sigma_BH and
 * CDF (Eq. dsdkbh); the Trident pair-energy and split CDFs (Sec. II.D) are
 * shared by all materials.  FP32 copies are made for the batched path.
 * mats: host array of n_mats (1..4096).  Replaces earlier tables.
 * Synchronises the stream.  PCC_E_INVALID on a bad spec or material. */
int pcc_tables_build(pcc_ctx *ctx, const pcc_material *mats, int n_mats,
                     const pcc_table_spec *spec, void *stream);

/* Copy the FP64 tables to host arrays (any pointer may be NULL):
 * brems_sigma[n_mats][n_rows], brems_cdf[n_mats][n_rows][n_cols], bh_sigma,
 * bh_cdf (same shapes), tri_gp_cdf[n_rows][n_cols], tri_split_cdf, and
 * screening[n_mats][8] = {L_TF, L_D, eta_TF, eta_D, I_TFD, L_R, f_C, Z}
 * (lengths in units of hbar/(m_e c)).  Synchronous. */
int pcc_tables_read(pcc_ctx *ctx, double *brems_sigma, double *brems_cdf, double *bh_sigma,
                    double *bh_cdf, double *tri_gp_cdf, double *tri_split_cdf, double *screening);

/* Bin by cell (Sec. III.A: "in a given mesh cell"): counting sort of `in`
 * into the cell-region layout of `out`, each cell's particles in ascending
 * pid order.  Region of cell c: count_c + max(slack_abs, ceil(slack_rel *
 * count_c)) slots.  out->cell_start/cell_count/cell_added are written;
 * cell_added is zeroed.  Synchronises the stream (it reads back the
 * largest cell); PCC_E_CAPACITY if the regions do not fit out->capacity or
 * a cell holds more than 16384 particles. */
int pcc_bin(pcc_ctx *ctx, const pcc_particles *in, int n_cells, pcc_species *out,
            int slack_abs, double slack_rel, void *stream);

/* One collision step (Sec. III.A, Eq. proba1-proba3) over all cells:
 * electron-ion pairs (Brems then Trident on each pair), positron-ion pairs,
 * photon-ion pairs (Bethe-Heitler); N_pair = max(N_p, N_t) random pairs per
 * cell, acceptance 1 - exp(-(n_p n_t / n_pt) sigma' p' c dt / (gamma gamma_i))
 * then the weight correction W_t / max(W_p, W_t); inverse-CDF sampling of
 * the secondary energy; secondaries appended to the cell regions (photons
 * from Brems, e-/e+ from Trident and BH); absorbed photons removed.  ion may
 * not be NULL; em, ep, ph may have zero live particles but not be NULL.
 * A pair collides if U < p, p = 1 - exp(-x), for the uniform
 * U = (2^48 a + e + 1/2) 2^-64 compared digit by digit: the pair's 16-bit
 * accept digit a settles it unless a = floor(2^16 p), and only then is the
 * 48-bit rest e drawn, so even per-pair probabilities far below 1e-7 (small
 * time steps, rare processes) are honoured (see pcc_accept_check).
 * precision PCC_FP64_PLAIN: one thread block per cell, FP64 arithmetic;
 * PCC_FP32_BATCHED: persistent kernel, FP32 arithmetic, and a pair whose
 * accept digit exceeds floor(2^16 b) for a per-material bound b of its
 * acceptance probability is rejected without being evaluated (exact, since
 * 1 - exp(-x) <= x <= b; the Trident bound assumes ion-frame Lorentz factors
 * below 1e7).  ledger: optional device float[n_cells][4], per cell {radiated
 * photon energy, compensation, created weight, compensation} accumulated
 * with Kahan summation.  Random numbers: Philox4x32-10 keyed by `seed`,
 * counters (slot or pair, cell, step, stream tag).  Asynchronous. */
int pcc_collide(pcc_ctx *ctx, const pcc_cells *cells, pcc_species *em, pcc_species *ep,
                pcc_species *ph, const pcc_species *ion, double dt, uint64_t seed, uint64_t step,
                unsigned process_mask, int precision, float *ledger, void *stream);

/* Launch schedule of the batched FP32 collision kernels (no counterpart in
 * the paper; a performance setting that never changes results).  Cells are
 * scanned largest size class first, a warp for each large cell and a group
 * of 16 to 2 lanes for each smaller one; min_blocks_per_sm
 * (2 to 6) selects the register budget of the kernel (a minimum of that
 * many resident 256-thread blocks per SM) and blocks_per_sm caps the
 * persistent grid (0 = as many as fit).  Applies to later pcc_collide calls
 * on this context.  PCC_E_INVALID outside these ranges. */
int pcc_set_schedule(pcc_ctx *ctx, int min_blocks_per_sm, int blocks_per_sm);

/* Lane groups of the batched scan (no counterpart in the paper; a
 * performance setting).  The random streams do not depend on it; it changes
 * only the order of the FP32 sums of a cell's weights, hence at most the
 * last bit of the pair coefficient and with it, rarely, a decision within
 * float rounding of its threshold.  Cells are sorted into
 * size classes, two per octave of N_pair = max(N_p, N_t): class 0 is
 * N_pair = 1, and with b the bit length of N_pair, class 2(b-1) holds
 * [2^(b-1), 1.5 2^(b-1)) and class 2(b-1)+1 holds [1.5 2^(b-1), 2^b); 34
 * classes.  For group (0 e-, 1 e+, 2 photons), thresholds[4] = {warp, g16,
 * g8, g4}: cells of class >= warp take a whole warp, [g16, warp) 16 lanes,
 * [g8, g16) 8 lanes, [g4, g8) 4 lanes and the smaller ones 2 lanes.
 * Requires 0 <= g4 <= g8 <= g16 <= warp <= 34 (PCC_E_INVALID otherwise).
 * Applies to later pcc_collide calls on this context.  pcc_get_scan_classes
 * reads the current setting (host int[4]). */
int pcc_set_scan_classes(pcc_ctx *ctx, int group, const int *thresholds);
int pcc_get_scan_classes(const pcc_ctx *ctx, int group, int *thresholds);

/* Fault injection (no counterpart in the paper): the bounded waits of the
 * batched kernels (the mbarrier of the bulk copy that stages the ln sigma
 * rows in shared memory) give up after `polls` polls instead of 4194304,
 * set PCC_ST_TIMEOUT and fall back to the global rows (same values), after
 * a second bounded wait that lets the copy land.  polls = 0 makes every
 * staged launch time out, to test the status path without a hang or a
 * fault.  Applies to later pcc_collide calls on this context; PCC_E_INVALID
 * for polls < 0. */
int pcc_set_wait_limit(pcc_ctx *ctx, int polls);

/* Make the secondaries of the last step live (Sec. III.A: created
 * macro-particles join the simulation): per cell, order the appended
 * particles by pid, then cell_count += cell_added, cell_added = 0.
 * Asynchronous. */
int pcc_append_secondaries(pcc_ctx *ctx, int n_cells, pcc_species *sp, void *stream);

/* Diagnostic: the accept decision of the collision kernels (Eq. proba3: a
 * pair collides if U < p, p = 1 - exp(-x)) for n given 16-bit accept digits
 * r[i] (in [0, 2^16); a larger value is never accepted unless p >= 1) and
 * probabilities p[i].  U = (2^48 r + e + 1/2) 2^-64 is compared with p
 * digit by digit: r settles it unless r = floor(2^16 p); only then is the
 * 48-bit rest e = 2^16 w0 + (w1 >> 16) drawn, from words w0, w1 of the
 * Philox4x32-10 draw with counter (c0[i], cell[i], step, tag[i]) and key
 * seed.  out64[i]: the decision with p in FP64 (the plain path); out32[i]:
 * with p rounded to FP32 (the batched path).  Device arrays of n entries
 * (outputs 0 or 1).  PCC_E_INVALID for n < 0 or a null array.
 * Asynchronous. */
int pcc_accept_check(int n, const uint32_t *r, const double *p, const uint32_t *c0, const uint32_t *cell,
                     const uint32_t *tag, uint64_t step, uint64_t seed, int *out32, int *out64, void *stream);

/* Diagnostic: the pairing of Sec. III.A for one projectile species against
 * the targets.  For live projectile slot s of cell c (written at index
 * cell_start[c] + s): out_j = its first pair index j, out_t = that pair's
 * target slot.  group 0 = electrons, 1 = positrons, 2 = photons.
 * Asynchronous. */
int pcc_pairing(pcc_ctx *ctx, int n_cells, const pcc_species *proj, const pcc_species *targ,
                int group, uint64_t seed, uint64_t step, int *out_j, int *out_t, void *stream);

/* FP64 totals over the live particles of a species (Sec. III.A energy
 * bookkeeping): out[0] = sum W, out[1] = sum W E (E = gamma for leptons,
 * k for photons, in m_e c^2), out[2] = sum W |u|.  out: device double[3].
 * Deterministic for a given layout.  Asynchronous. */
int pcc_totals(pcc_ctx *ctx, int n_cells, const pcc_species *sp, int is_photon, double *out,
               void *stream);

/* Allocation-free variant of pcc_totals (no counterpart in the paper; a
 * service for callers that may not allocate device memory while they run,
 * such as a simulation that sizes all its buffers at start-up and forbids
 * allocation in its time loop, or an application whose own allocator owns
 * the whole device).  Same result as pcc_totals up to the order of the FP64
 * sums; needs no context.  Its scratch is a fixed 96 KiB array in the
 * library's device memory (held by every GPU that loads the library until
 * the process exits), so n_cells is limited to 4,194,304: larger counts
 * return PCC_E_CAPACITY without launching anything.  The first call in a
 * CUDA context (normally once per device, with that device current) looks
 * up the array's device address with cudaGetSymbolAddress and caches it per
 * context; make that first call before any stream capture.  A context
 * created anew (after cudaDeviceReset, or a second context on the device)
 * gets its own lookup on its first call.  Calls share the array and it
 * keeps the last call's partial sums (each call overwrites the entries it
 * reads, so nothing needs clearing); two calls whose kernels can run at the
 * same time (unordered streams) race.  Allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.
 * out: device double[3].  Asynchronous after the first call. */
int pcc_totals_noalloc(int n_cells, const pcc_species *sp, int is_photon, double *out, void *stream);

/* The multi-step collision loop as one CUDA graph (the batching pattern
 * around Sec. III.A's per-step procedure).  One captured step is:
 * the work of one pcc_collide call with the descriptor's mask (groups in
 * the order e-, e+, photons), then pcc_append_secondaries for e-, e+ and
 * photons.  pcc_steps_capture records
 * n_steps such steps, for step indices step0 .. step0 + n_steps - 1, into a
 * graph owned by the context (replacing any earlier one); every allocation
 * the steps need happens before the capture, which runs on a stream of the
 * context's own, so the caller's stream is not captured.  All pointers in
 * the descriptor must stay valid and unchanged while the graph is used.
 * timing != 0 adds five timing events per step (before the e- group, after
 * each group, after the commits), read by pcc_steps_timing; on the batched
 * path the size-class sort of all groups runs before the e- group's kernels
 * and is timed with them.
 * pcc_steps_launch enqueues the whole graph on the stream.  A launch
 * repeats the same step indices: capture again to go on. */
typedef struct {
    const pcc_cells *cells;
    pcc_species *em, *ep, *ph;
    const pcc_species *ion;
    double dt;
    uint64_t seed;
    unsigned mask;          /* PCC_BREMS | PCC_TRIDENT | PCC_BH [| group bits] */
    int precision;          /* pcc_precision */
    float *ledger;          /* device [n_cells][4] or NULL, as for pcc_collide */
} pcc_step_desc;

int pcc_steps_capture(pcc_ctx *ctx, const pcc_step_desc *desc, uint64_t step0, int n_steps, int timing,
                      void *stream);
int pcc_steps_launch(pcc_ctx *ctx, void *stream);
/* After a launch: ms_out[n_steps][4] = e- group, e+ group, photon group,
 * commits, in milliseconds (waits for the launch to finish). */
int pcc_steps_timing(pcc_ctx *ctx, float *ms_out);

/* Number of kernels the library has enqueued in this process (a graph
 * launch counts each kernel node of the graph; capturing counts nothing). */
unsigned long long pcc_launch_count(void);

/* Read and clear the device status word and step counters.  Synchronises
 * the stream.  status_out: PCC_ST_* bits; stats_out may be NULL. */
int pcc_read_status(pcc_ctx *ctx, unsigned *status_out, pcc_stats *stats_out, void *stream);

/* Expected-emission operator (rate form of Eq. N_br_theo1/2, radiative
 * stopping power of Sec. III.B) per cell c for electrons at rest ions:
 *   out[c][0] = n_i sum_s w_s v_s sigma_B(gamma_s)
 *   out[c][1] = n_i sum_s w_s v_s sigma_T(gamma_s)
 *   out[c][2] = n_i sum_s w_s v_s int k dsigma_B/dk dk
 * with sigma_B = int_{1e-7}^{1} dsigma/dk (gamma-1) dx by a fixed n_quad
 * point Gauss-Legendre rule in ln x, for parameters params[c][5] =
 * {n_i, T_e, Zstar, s_TF, s_D} of element Z.  gamma, w: [n_cells][n_samples].
 * All device float32.  n_quad <= 128.  Asynchronous. */
int pcc_expected_emission_fwd(pcc_ctx *ctx, int n_cells, int n_samples, int Z, int n_quad,
                              const float *params, const float *gamma, const float *w, float *out,
                              void *stream);

/* Adjoint of pcc_expected_emission_fwd: grad_params[c][k] = sum_j
 * grad_out[c][j] d out[c][j] / d params[c][k].  The Debye-length lower bound
 * max(lambda_D, r_i) takes the derivative of the active branch (r_i on a
 * tie).  All device float32.  Asynchronous. */
int pcc_expected_emission_bwd(pcc_ctx *ctx, int n_cells, int n_samples, int Z, int n_quad,
                              const float *params, const float *gamma, const float *w,
                              const float *grad_out, float *grad_params, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PCC_H */
