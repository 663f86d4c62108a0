// The pairwise collision step of Sec. III.A for electron-ion (Bremsstrahlung
// then Trident on each pair), positron-ion and photon-ion (Bethe-Heitler)
// pairs.  One routine per cell, templated on the arithmetic type and on the
// thread group that owns the cell:
//   plain   (FP64): one thread block per cell, grid = cells;
//   batched (FP32): persistent grid, one warp per cell, cells strided over
//                   warps, ln sigma rows staged in shared memory by a bulk
//                   copy (cp.async.bulk + mbarrier).
#include <algorithm>

#include "pcc_internal.h"
#include "pcc_physics.cuh"

namespace pcc {

struct SpeciesView {
    float *ux, *uy, *uz, *w, *x;
    uint64_t* pid;
    const int* start;
    int* count;
    int* added;
};

__host__ __device__ inline SpeciesView view_of(const pcc_species& s)
{
    return SpeciesView{s.ux, s.uy, s.uz, s.w, s.x, s.pid, s.cell_start, s.cell_count, s.cell_added};
}

struct StepArgs {
    int n_cells;
    const int* mat_of_cell;
    SpeciesView em, ep, ph, ion;
    double dt;
    uint64_t seed, step;
    unsigned mask;
    float* ledger;           // [n_cells][4] or null
    TableGeom g;
    int n_mat;
    // FP64 tables
    const double *brems_sigma, *brems_cdf, *bh_sigma, *bh_cdf, *tri_gp, *tri_split, *screen;
    // FP32 tables
    const float *f_brems_lnsig, *f_brems_cdf, *f_bh_lnsig, *f_bh_cdf, *f_tri_gp, *f_tri_split, *f_Z;
    const float* f_bound;    // [n_mat][3] acceptance bounds (Brems, Trident, BH)
    DevStats* st;
    PhiloxKeys keys;         // round keys of the seed
    float f_cdt;             // c dt in float
    int wait_polls;          // bounded waits give up after this many polls
};

// ---- per-thread accumulators ---------------------------------------------
struct Acc {
    unsigned long long pairs[3];
    unsigned accepted[5], created[5];
    unsigned candidates[3];
    double dE, dQ;
    unsigned status;
    __device__ void zero()
    {
        for (int i = 0; i < 3; ++i) pairs[i] = 0, candidates[i] = 0;
        for (int i = 0; i < 5; ++i) accepted[i] = created[i] = 0;
        dE = dQ = 0.0;
        status = 0;
    }
};

// ---- thread groups ---------------------------------------------------------
struct WarpGroup {
    int* scratch;   // 64 ints per warp
    __device__ int rank() const { return threadIdx.x & 31; }
    __device__ int size() const { return 32; }
    __device__ void sync() const { __syncwarp(); }
    template <typename T> __device__ T sum(T v) const { return warp_sum(v); }
    __device__ float fmin(float v) const
    {
        for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
    __device__ float fmax(float v) const
    {
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
    __device__ bool any(bool p) const { return __any_sync(0xffffffffu, p); }
};

struct CtaGroup {
    int* scratch;       // 64 ints
    double* red;        // blockDim/32 doubles
    __device__ int rank() const { return threadIdx.x; }
    __device__ int size() const { return blockDim.x; }
    __device__ void sync() const { __syncthreads(); }
    template <typename T> __device__ T sum(T v) const
    {
        v = warp_sum(v);
        const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[w] = (double)v;
        __syncthreads();
        T t = 0;
        for (int k = 0; k < nw; ++k) t += (T)red[k];
        return t;
    }
    __device__ float fmin(float v) const { return -fmax(-v); }
    __device__ float fmax(float v) const
    {
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[w] = (double)v;
        __syncthreads();
        float t = (float)red[0];
        for (int k = 1; k < nw; ++k) t = fmaxf(t, (float)red[k]);
        return t;
    }
    __device__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
};

// ---- table access ----------------------------------------------------------
template <typename Real> struct Tab;

template <> struct Tab<double> {
    const double *bsig, *bcdf, *hsig, *hcdf, *tgp, *tsp;
    __device__ double ln_sigma(const double* s, int i) const { return log(s[i]); }
};
template <> struct Tab<float> {
    const float *bsig, *bcdf, *hsig, *hcdf, *tgp, *tsp;   // bsig/hsig hold ln sigma
    __device__ float ln_sigma(const float* s, int i) const { return s[i]; }
};

// Arithmetic of the two paths: FP64 plain uses correctly rounded library
// functions; the FP32 batched path uses the hardware approximations (a few
// ulp), which changes an accept decision only for pairs within ~1e-6 of the
// threshold.
__device__ __forceinline__ double q_div(double a, double b) { return a / b; }
__device__ __forceinline__ float q_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double q_log(double a) { return log(a); }
__device__ __forceinline__ float q_log(float a) { return __logf(a); }
__device__ __forceinline__ double q_exp(double a) { return exp(a); }
__device__ __forceinline__ float q_exp(float a) { return __expf(a); }
__device__ __forceinline__ double q_sqrt1(double a) { return sqrt(a); }            // a >= 1
__device__ __forceinline__ float q_sqrt1(float a) { return a * rsqrtf(a); }        // a >= 1
__device__ __forceinline__ double q_sqrt0(double a) { return sqrt(a); }            // a >= 0
__device__ __forceinline__ float q_sqrt0(float a) { return a > 0.f ? a * rsqrtf(a) : 0.f; }

template <typename Real>
__device__ __forceinline__ Real row_ln0(const TableGeom& g);
template <> __device__ __forceinline__ double row_ln0<double>(const TableGeom& g) { return g.ln_T_min; }
template <> __device__ __forceinline__ float row_ln0<float>(const TableGeom& g) { return g.f_ln_T_min; }
template <typename Real>
__device__ __forceinline__ Real row_inv(const TableGeom& g);
template <> __device__ __forceinline__ double row_inv<double>(const TableGeom& g) { return g.inv_dln_row; }
template <> __device__ __forceinline__ float row_inv<float>(const TableGeom& g) { return g.f_inv_dln_row; }

// Total cross section at row variable r: log-log interpolation, 0 below
// the table, last row (and TABLE_RANGE) above it.
template <typename Real>
__device__ __forceinline__ Real sigma_at(const Tab<Real>& tb, const Real* row_tab, const TableGeom& g, Real r,
                                         unsigned& status)
{
    if (!(r >= (Real)g.T_min)) return (Real)0;
    const Real t = (q_log(r) - row_ln0<Real>(g)) * row_inv<Real>(g);
    if (t > (Real)(g.n_rows - 1)) {
        status |= PCC_ST_TABLE_RANGE;
        return q_exp(tb.ln_sigma(row_tab, g.n_rows - 1));
    }
    int j = (int)t;
    if (j > g.n_rows - 2) j = g.n_rows - 2;
    const Real f = t - (Real)j;
    const Real l0 = tb.ln_sigma(row_tab, j), l1 = tb.ln_sigma(row_tab, j + 1);
    return q_exp(l0 + f * (l1 - l0));
}

// Inverse-CDF sample of the column variable: stochastic row pick, binary
// search in the row, linear interpolation in ln y (log grid) or y.
template <typename Real>
__device__ Real sample_col(const Real* cdf, const TableGeom& g, Real r, Real u_row, Real u_col, bool log_grid,
                           double ln_ymin)
{
    Real t = (log(r) - row_ln0<Real>(g)) * row_inv<Real>(g);
    if (!(t > (Real)0)) t = (Real)0;
    if (t > (Real)(g.n_rows - 1)) t = (Real)(g.n_rows - 1);
    int j = (int)t;
    if (j > g.n_rows - 2) j = g.n_rows - 2;
    const Real f = t - (Real)j;
    const int row = j + (u_row < f ? 1 : 0);
    const Real* F = cdf + (size_t)row * g.n_cols;
    int lo = 0, hi = g.n_cols - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (F[mid] <= u_col) lo = mid; else hi = mid;
    }
    const Real frac = (u_col - F[lo]) / (F[lo + 1] - F[lo]);
    if (log_grid) {
        const Real ly = (Real)ln_ymin;
        return exp(ly + ((Real)lo + frac) * (-ly / (Real)(g.n_cols - 1)));
    }
    return ((Real)lo + frac) / (Real)(g.n_cols - 1);
}

// ---- kinematics --------------------------------------------------------------
template <typename Real>
struct Frame {
    Real ui[3], gi;     // ion proper velocity and Lorentz factor
    Real gl;            // projectile energy in the simulation frame
    Real pp, Tp;        // momentum and kinetic energy in the ion frame
    Real n[3];          // ion-frame momentum; a unit direction after normalize()
    __device__ __forceinline__ void normalize()
    {
        const Real inv = pp > (Real)0 ? (Real)1 / pp : (Real)0;
        n[0] *= inv; n[1] *= inv; n[2] *= inv;
    }
};

// E' = gi E - ui.p ; p' = p + ((ui.p)/(gi+1) - E) ui  (Sec. III.A transform)
template <typename Real>
__device__ __forceinline__ void to_ion_frame(Frame<Real>& f, const Real u[3])
{
    f.gl = q_sqrt1((Real)1 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const Real d = f.ui[0] * u[0] + f.ui[1] * u[1] + f.ui[2] * u[2];
    const Real fac = q_div(d, f.gi + (Real)1) - f.gl;
    f.n[0] = u[0] + fac * f.ui[0];
    f.n[1] = u[1] + fac * f.ui[1];
    f.n[2] = u[2] + fac * f.ui[2];
    const Real p2 = f.n[0] * f.n[0] + f.n[1] * f.n[1] + f.n[2] * f.n[2];
    f.pp = q_sqrt0(p2);
    f.Tp = q_div(p2, (Real)1 + q_sqrt1((Real)1 + p2));
}

// (E', p') in the ion frame back to the simulation frame.
template <typename Real>
__device__ __forceinline__ void from_ion_frame(const Frame<Real>& f, Real E, const Real p[3], Real& Eo, Real po[3])
{
    const Real d = f.ui[0] * p[0] + f.ui[1] * p[1] + f.ui[2] * p[2];
    Eo = f.gi * E + d;
    const Real fac = d / (f.gi + (Real)1) + E;
    po[0] = p[0] + fac * f.ui[0];
    po[1] = p[1] + fac * f.ui[1];
    po[2] = p[2] + fac * f.ui[2];
}

// Lepton of kinetic energy T along the ion-frame direction n, in the lab.
template <typename Real>
__device__ __forceinline__ Real lepton_to_lab(const Frame<Real>& f, Real T, Real out[3])
{
    const Real p = sqrt(T * (T + (Real)2));
    const Real pv[3] = {p * f.n[0], p * f.n[1], p * f.n[2]};
    Real E;
    from_ion_frame(f, (Real)1 + T, pv, E, out);
    return E;
}

// ---- appending a secondary into a cell region -------------------------------
__device__ __forceinline__ bool append_particle(const SpeciesView& sp, int cell, const float u[3], float w, float x,
                                                bool has_x, uint64_t pid, unsigned& status)
{
    const int base = sp.start[cell], lim = sp.start[cell + 1];
    const int live = sp.count[cell];
    const int k = atomicAdd(&sp.added[cell], 1);
    const int slot = base + live + k;
    if (slot >= lim) {
        atomicSub(&sp.added[cell], 1);
        status |= PCC_ST_CAPACITY;
        return false;
    }
    sp.ux[slot] = u[0]; sp.uy[slot] = u[1]; sp.uz[slot] = u[2]; sp.w[slot] = w;
    if (has_x && sp.x) sp.x[slot] = x;
    sp.pid[slot] = pid;
    return true;
}

// ---- the permutation of the larger list (n <= 32 uses the group's smem) ------
struct Pairing {
    PermKeys rk;
    uint32_t Np, Nt;
    bool caseA;       // Np >= Nt: permute projectiles
    bool small;       // larger list <= 32
    const int* pos;   // small: P^-1 table
    const int* elem;  // small: P table
    // projectile slot s: first pair index (case A) / target of pair j (case B)
    __device__ __forceinline__ uint32_t pair_of_slot(uint32_t s) const
    {
        return small ? (uint32_t)pos[s] : perm_pos_large(s, Np, rk);
    }
    __device__ __forceinline__ uint32_t target_of_pair(uint32_t j) const
    {
        return small ? (uint32_t)elem[j] : perm_elem_large(j, Nt, rk);
    }
};

template <class G>
__device__ __forceinline__ Pairing make_pairing(const G& grp, uint32_t Np, uint32_t Nt, uint32_t cell,
                                                uint32_t group, const StepArgs& a)
{
    Pairing P;
    const Philox4 k = draw(0, cell, a.step, stream_tag(group, kPerm, 0), a.seed);
    P.rk.k[0] = k.v[0]; P.rk.k[1] = k.v[1]; P.rk.k[2] = k.v[2]; P.rk.k[3] = k.v[3];
    P.Np = Np; P.Nt = Nt;
    P.caseA = Np >= Nt;
    const uint32_t NL = P.caseA ? Np : Nt;
    P.small = NL <= 32;
    P.pos = grp.scratch;
    P.elem = grp.scratch + 32;
    if (P.small) {
        grp.sync();
        for (int s = grp.rank(); s < (int)NL; s += grp.size()) {
            const uint32_t r = perm_pos_small((uint32_t)s, NL, P.rk);
            grp.scratch[s] = (int)r;
            grp.scratch[32 + r] = s;
        }
        grp.sync();
    }
    return P;
}

// ---- rare event paths (out of line: they run on about 1e-4 of the pairs) -----
struct EventResult {
    float u[3];        // projectile after the event (lab frame)
    double dE;         // W (E_out - E_in)
    float rad, wc;     // radiated photon energy W k, created weight
    unsigned status;
    int created;       // 1 when the weight correction kept the event
};

// Brems event on pair j (Sec. III.A): weight correction, inverse-CDF photon
// energy, photon parallel to the electron in the ion frame, recoil.
template <typename Real>
__device__ __noinline__ EventResult brems_event(const StepArgs* ap, Tab<Real> tb, int group, int cell, int mat,
                                                uint32_t j, float wp, float wt, float xpos, Frame<Real> f)
{
    const StepArgs& a = *ap;
    EventResult r{};
    f.normalize();
    const int ch = group == kGroupEm ? kChBremsEm : kChBremsEp;
    const Philox4 ev = draw(j, cell, a.step, stream_tag(group, kEvtBrems, 0), a.seed);
    if ((wt < wp) && !(u01<Real>(ev.v[0]) < (Real)wt / (Real)wp)) return r;
    r.created = 1;
    const Real* cdf = tb.bcdf + (size_t)mat * a.g.n_rows * a.g.n_cols;
    const Real xk = sample_col<Real>(cdf, a.g, f.Tp, u01<Real>(ev.v[1]), u01<Real>(ev.v[2]), true, a.g.ln_x_min);
    const Real kp = xk * f.Tp;
    Real ue[3], kg[3], Ek;
    const Real Ee = lepton_to_lab(f, f.Tp * ((Real)1 - xk), ue);
    const Real pk[3] = {kp * f.n[0], kp * f.n[1], kp * f.n[2]};
    from_ion_frame(f, kp, pk, Ek, kg);
    const float gk[3] = {(float)kg[0], (float)kg[1], (float)kg[2]};
    r.u[0] = (float)ue[0]; r.u[1] = (float)ue[1]; r.u[2] = (float)ue[2];
    if (append_particle(a.ph, cell, gk, wp, xpos, a.em.x != nullptr, secondary_pid(a.step, ch, cell, j, 0),
                        r.status)) {
        r.dE = (double)wp * ((double)Ee + (double)Ek - (double)f.gl);
        r.rad = wp * (float)Ek;
        r.wc = wp;
    }
    return r;
}

// Trident event on pair j (Sec. II.D): pair energy from its CDF, positron
// share from the split CDF, both leptons along the electron in the ion frame.
template <typename Real>
__device__ __noinline__ EventResult trident_event(const StepArgs* ap, Tab<Real> tb, int group, int cell, uint32_t j,
                                                  float wp, float wt, float xpos, Frame<Real> f)
{
    const StepArgs& a = *ap;
    EventResult r{};
    f.normalize();
    const int ch = group == kGroupEm ? kChTriEm : kChTriEp;
    const Philox4 e1 = draw(j, cell, a.step, stream_tag(group, kEvtTri1, 0), a.seed);
    if ((wt < wp) && !(u01<Real>(e1.v[0]) < (Real)wt / (Real)wp)) return r;
    r.created = 1;
    const Philox4 e2 = draw(j, cell, a.step, stream_tag(group, kEvtTri2, 0), a.seed);
    const Real y = sample_col<Real>(tb.tgp, a.g, f.Tp - (Real)2, u01<Real>(e1.v[1]), u01<Real>(e1.v[2]), true,
                                    a.g.ln_tri_min);
    const Real gpair = (Real)2 + y * (f.Tp - (Real)2);
    const Real y2 = sample_col<Real>(tb.tsp, a.g, gpair - (Real)2, u01<Real>(e1.v[3]), u01<Real>(e2.v[0]), false,
                                     0.0);
    Real uf[3], up[3], um[3];
    const Real Ef = lepton_to_lab(f, (f.Tp - (Real)2) * ((Real)1 - y), uf);
    const Real Ep = lepton_to_lab(f, y2 * (gpair - (Real)2), up);
    const Real Em = lepton_to_lab(f, (gpair - (Real)2) * ((Real)1 - y2), um);
    const float fm[3] = {(float)um[0], (float)um[1], (float)um[2]};
    const float fp[3] = {(float)up[0], (float)up[1], (float)up[2]};
    const bool hx = a.em.x != nullptr;
    const bool ok1 = append_particle(a.em, cell, fm, wp, xpos, hx, secondary_pid(a.step, ch, cell, j, 0), r.status);
    const bool ok2 = append_particle(a.ep, cell, fp, wp, xpos, hx, secondary_pid(a.step, ch, cell, j, 1), r.status);
    if (ok1 && ok2) {
        r.dE = (double)wp * ((double)Ef + (double)Ep + (double)Em - (double)f.gl);
        r.wc = 2.f * wp;
    }
    r.u[0] = (float)uf[0]; r.u[1] = (float)uf[1]; r.u[2] = (float)uf[2];
    return r;
}

// Bethe-Heitler event on pair j (Sec. III.A): e+ e- along the photon in the
// ion frame, energies from the BH CDF; the photon is absorbed.
template <typename Real>
__device__ __noinline__ EventResult bh_event(const StepArgs* ap, Tab<Real> tb, int cell, int mat, uint32_t j, float wp,
                                             float wt, float xpos, Frame<Real> f, Real kp, Real k)
{
    const StepArgs& a = *ap;
    EventResult r{};
    const Philox4 ev = draw(j, cell, a.step, stream_tag(kGroupPh, kEvtBH, 0), a.seed);
    if ((wt < wp) && !(u01<Real>(ev.v[0]) < (Real)wt / (Real)wp)) return r;
    r.created = 1;
    const Real* cdf = tb.hcdf + (size_t)mat * a.g.n_rows * a.g.n_cols;
    const Real y = sample_col<Real>(cdf, a.g, kp - (Real)2, u01<Real>(ev.v[1]), u01<Real>(ev.v[2]), false, 0.0);
    Real up[3], um[3];
    const Real Ep = lepton_to_lab(f, y * (kp - (Real)2), up);
    const Real Em = lepton_to_lab(f, (kp - (Real)2) * ((Real)1 - y), um);
    const float fm[3] = {(float)um[0], (float)um[1], (float)um[2]};
    const float fp[3] = {(float)up[0], (float)up[1], (float)up[2]};
    const bool hx = a.ph.x != nullptr;
    const bool ok1 = append_particle(a.em, cell, fm, wp, xpos, hx, secondary_pid(a.step, kChBH, cell, j, 0), r.status);
    const bool ok2 = append_particle(a.ep, cell, fp, wp, xpos, hx, secondary_pid(a.step, kChBH, cell, j, 1), r.status);
    if (ok1 && ok2) {
        r.dE = (double)wp * ((double)Ep + (double)Em - (double)k);
        r.wc = 2.f * wp;
    }
    return r;
}

// ---- one electron/positron - ion pair: Brems then Trident -------------------
// The weights (projectile *wp, target ion.w) are read only for accepted
// pairs; no event writes a live particle's weight.  rB, rT: the pair's
// accept digits for Brems and Trident; src names the extension draw of the
// Brems uniform (the Trident one has the next counter).
template <typename Real>
__device__ __forceinline__ void ei_pair(const StepArgs* ap, const Tab<Real>& tb, int group, int cell, int mat, Real Zf,
                                        Real coef, float u[3], const float* wp, float xpos, int t_slot, uint32_t j,
                                        uint32_t rB, uint32_t rT, const AcceptSrc& src, Acc& acc, float& rad,
                                        float& wcre, bool& had)
{
    const StepArgs& a = *ap;
    const SpeciesView& ion = a.ion;
    Frame<Real> f;
    f.ui[0] = ion.ux[t_slot]; f.ui[1] = ion.uy[t_slot]; f.ui[2] = ion.uz[t_slot];
    f.gi = q_sqrt1((Real)1 + f.ui[0] * f.ui[0] + f.ui[1] * f.ui[1] + f.ui[2] * f.ui[2]);
    const Real uu[3] = {(Real)u[0], (Real)u[1], (Real)u[2]};
    to_ion_frame(f, uu);
    if (!isfinite(f.gl)) { acc.status |= PCC_ST_NONFINITE; return; }
    // the batched path's Trident quick-reject bound is proven up to gamma' = 1e7
    if (sizeof(Real) == 4 && (a.mask & PCC_TRIDENT) && f.Tp > (Real)(1e7 - 1.0)) acc.status |= PCC_ST_BOUND_RANGE;
    if (a.mask & PCC_BREMS) {
        const Real sig = sigma_at<Real>(tb, tb.bsig + (size_t)mat * a.g.n_rows, a.g, f.Tp, acc.status);
        const Real x = q_div(coef * sig * f.pp, f.gl * f.gi);
        if (x > (Real)1) acc.status |= PCC_ST_PROB_LARGE;
        if (sig > (Real)0 && accept_u<Real>(rB, -expm1(-x), src, a.step, a.seed)) {
            const int ch = group == kGroupEm ? kChBremsEm : kChBremsEp;
            acc.accepted[ch]++;
            const EventResult r = brems_event<Real>(ap, tb, group, cell, mat, j, *wp, ion.w[t_slot], xpos, f);
            if (r.created) {
                acc.created[ch]++;
                acc.dE += r.dE;
                acc.status |= r.status;
                rad += r.rad;
                wcre += r.wc;
                had = true;   // the projectile changed
                u[0] = r.u[0]; u[1] = r.u[1]; u[2] = r.u[2];
                const Real nu[3] = {(Real)u[0], (Real)u[1], (Real)u[2]};
                to_ion_frame(f, nu);
            }
        }
    }
    if ((a.mask & PCC_TRIDENT) && f.Tp >= (Real)2) {
        // Gryaznykh fit (Sec. II.D) above the threshold gamma = 3
        const Real l = q_log(q_div(f.Tp + (Real)5.5, (Real)6.89));
        const Real sig = (Real)5.22e-34 * Zf * Zf * l * l * l;
        const Real x = q_div(coef * sig * f.pp, f.gl * f.gi);
        if (x > (Real)1) acc.status |= PCC_ST_PROB_LARGE;
        AcceptSrc srcT = src;
        srcT.c0 += 1;   // the Trident digit follows the Brems digit
        if (sig > (Real)0 && accept_u<Real>(rT, -expm1(-x), srcT, a.step, a.seed)) {
            const int ch = group == kGroupEm ? kChTriEm : kChTriEp;
            acc.accepted[ch]++;
            const EventResult r = trident_event<Real>(ap, tb, group, cell, j, *wp, ion.w[t_slot], xpos, f);
            if (r.created) {
                acc.created[ch]++;
                acc.dE += r.dE;
                acc.status |= r.status;
                wcre += r.wc;
                had = true;
                u[0] = r.u[0]; u[1] = r.u[1]; u[2] = r.u[2];
            }
        }
    }
}

// Cell sums of Sec. III.A: n_p = sum W_p, n_t = sum W_t and
// n_pt = sum over pairs of min(W_p, W_t).  One pass over both lists; when
// every target of the cell has the same weight, a projectile's pairs all
// contribute min(W_p, W_t), so n_pt needs no permutation.
template <typename Real, class G>
__device__ __forceinline__ void cell_sums(const G& grp, const SpeciesView& P, const SpeciesView& I, int p0, int t0,
                                          uint32_t Np, uint32_t Nt, const Pairing& pr, Real& n_p, Real& n_t,
                                          Real& n_pt)
{
    const float w0 = I.w[t0];
    Real sp = 0, st = 0, sf = 0;
    float wmin = w0, wmax = w0;
    const uint32_t N = Np > Nt ? Np : Nt;
#pragma unroll 4
    for (uint32_t s = grp.rank(); s < N; s += grp.size()) {
        if (s < Nt) {
            const float wt = I.w[t0 + s];
            st += (Real)wt;
            wmin = fminf(wmin, wt);
            wmax = fmaxf(wmax, wt);
        }
        if (s < Np) {
            const float wp = P.w[p0 + s];
            sp += (Real)wp;
            const uint32_t npairs = pr.caseA ? 1u : (Nt - s + Np - 1) / Np;
            sf += (Real)fminf(wp, w0) * (Real)npairs;
        }
    }
    n_p = grp.sum(sp);
    n_t = grp.sum(st);
    const float lo = grp.fmin(wmin), hi = grp.fmax(wmax);
    if (lo == hi) {
        n_pt = grp.sum(sf);
        return;
    }
    Real spt = 0;
    for (uint32_t s = grp.rank(); s < Np; s += grp.size()) {
        const float wp = P.w[p0 + s];
        if (pr.caseA) {
            spt += (Real)fminf(wp, I.w[t0 + pr.pair_of_slot(s) % Nt]);
        } else {
            for (uint32_t j = s; j < Nt; j += Np) spt += (Real)fminf(wp, I.w[t0 + pr.target_of_pair(j)]);
        }
    }
    n_pt = grp.sum(spt);
}

// ---- one cell of electron (or positron) - ion pairs ---------------------------
template <typename Real, class G>
__device__ void ei_cell(const G& grp, const StepArgs* ap, const Tab<Real>& tb, int group, int cell, Acc& acc)
{
    const StepArgs& a = *ap;
    const SpeciesView& P = group == kGroupEm ? a.em : a.ep;
    const SpeciesView& I = a.ion;
    const uint32_t Np = P.count[cell], Nt = I.count[cell];
    if (Np == 0 || Nt == 0) return;
    const int p0 = P.start[cell], t0 = I.start[cell];
    const int mat = a.mat_of_cell[cell];
    if ((unsigned)mat >= (unsigned)a.n_mat) {
        acc.status |= PCC_ST_NONFINITE;
        return;
    }
    const Pairing pr = make_pairing(grp, Np, Nt, cell, group, a);
    Real n_p, n_t, n_pt;
    cell_sums<Real>(grp, P, I, p0, t0, Np, Nt, pr, n_p, n_t, n_pt);
    const Real coef = (n_p / n_pt) * n_t * (Real)(kC * a.dt);
    const uint32_t Npair = Np > Nt ? Np : Nt;
    if (grp.rank() == 0) acc.pairs[group] += Npair;
    if (Npair > 65536u || (uint32_t)cell > 0xFFFFFFu || a.step > 0x7FFFFull) acc.status |= PCC_ST_ID_RANGE;
    const Real Zf = sizeof(Real) == 8 ? (Real)a.screen[(size_t)mat * kScreenFields + 7] : (Real)a.f_Z[mat];
    // the FP32 path rejects from the accept digits alone above the bounds
    const bool quick = sizeof(Real) == 4;
    const uint32_t kB = quick && (a.mask & PCC_BREMS) ? accept_threshold((float)(coef * (Real)a.f_bound[3 * mat])) : 0u;
    const uint32_t kT =
        quick && (a.mask & PCC_TRIDENT) ? accept_threshold((float)(coef * (Real)a.f_bound[3 * mat + 1])) : 0u;
    float rad = 0.f, wcre = 0.f;
    bool had = false;
    const bool has_x = P.x != nullptr;
    // two 16-bit accept digits per pair (Brems, Trident): slots 4q .. 4q + 3
    // share the draw of counter q, slot 4q + h its digits 2h and 2h + 1.  A
    // thread per slot (each takes its own copy of the draw), so that small
    // cells keep their threads busy.
    for (uint32_t s = grp.rank(); s < Np; s += grp.size()) {
        const uint32_t q = s >> 2, h = s & 3u;
        {
            const int sl = p0 + (int)s;
            float u[3] = {P.ux[sl], P.uy[sl], P.uz[sl]};
            const float w = P.w[sl];
            const float xp = has_x ? P.x[sl] : 0.f;
            bool dirty = false;
            if (pr.caseA) {
                const uint32_t j = pr.pair_of_slot(s);
                const Philox4 ac = draw(q, cell, a.step, stream_tag(group, kAccept, 0), a.seed);
                const uint32_t rB = accept_digit(ac, 2 * h), rT = accept_digit(ac, 2 * h + 1);
                if (!quick || rB <= kB || rT <= kT) {
                    if (quick) acc.candidates[group]++;
                    const AcceptSrc src{8 * q + 2 * h, (uint32_t)cell, stream_tag(group, kAcceptExt, 0)};
                    ei_pair<Real>(ap, tb, group, cell, mat, Zf, coef, u, &w, xp, t0 + (int)(j % Nt), j, rB, rT, src,
                                  acc, rad, wcre, dirty);
                }
            } else {
                for (uint32_t m = 0, j = s; j < Nt; ++m, j += Np) {
                    const Philox4 am = draw(q, cell, a.step, stream_tag(group, kAccept, m), a.seed);
                    const uint32_t rB = accept_digit(am, 2 * h), rT = accept_digit(am, 2 * h + 1);
                    if (quick && !(rB <= kB || rT <= kT)) continue;
                    acc.candidates[group]++;
                    const AcceptSrc src{8 * q + 2 * h, (uint32_t)cell, stream_tag(group, kAcceptExt, m)};
                    ei_pair<Real>(ap, tb, group, cell, mat, Zf, coef, u, &w, xp, t0 + (int)pr.target_of_pair(j), j,
                                  rB, rT, src, acc, rad, wcre, dirty);
                }
            }
            if (dirty) {
                P.ux[sl] = u[0]; P.uy[sl] = u[1]; P.uz[sl] = u[2];
                had = true;
            }
        }
    }
    if (a.ledger && grp.any(had)) {
        const float r = grp.sum(rad), wc = grp.sum(wcre);
        if (grp.rank() == 0) {
            float4* L = reinterpret_cast<float4*>(a.ledger) + cell;
            float4 v = *L;
            Kahan k1{v.x, v.y}, k2{v.z, v.w};
            k1.add(r);
            k2.add(wc);
            *L = make_float4(k1.s, k1.c, k2.s, k2.c);
        }
    }
}

// ---- one cell of photon - ion pairs (Bethe-Heitler) ---------------------------
template <typename Real, class G>
__device__ void bh_cell(const G& grp, const StepArgs* ap, const Tab<Real>& tb, int cell, Acc& acc)
{
    const StepArgs& a = *ap;
    const SpeciesView& P = a.ph;
    const SpeciesView& I = a.ion;
    const uint32_t Np = P.count[cell], Nt = I.count[cell];
    if (Np == 0 || Nt == 0) return;
    const int p0 = P.start[cell], t0 = I.start[cell];
    const int mat = a.mat_of_cell[cell];
    if ((unsigned)mat >= (unsigned)a.n_mat) {
        acc.status |= PCC_ST_NONFINITE;
        return;
    }
    const Pairing pr = make_pairing(grp, Np, Nt, cell, kGroupPh, a);
    Real n_p, n_t, n_pt;
    cell_sums<Real>(grp, P, I, p0, t0, Np, Nt, pr, n_p, n_t, n_pt);
    const Real coef = (n_p / n_pt) * n_t * (Real)(kC * a.dt);
    const uint32_t Npair = Np > Nt ? Np : Nt;
    if (grp.rank() == 0) acc.pairs[kGroupPh] += Npair;
    if (Npair > 65536u || (uint32_t)cell > 0xFFFFFFu || a.step > 0x7FFFFull) acc.status |= PCC_ST_ID_RANGE;
    float wcre = 0.f;
    bool absorbed_any = false;
    const bool has_x = P.x != nullptr;
    const bool quick = sizeof(Real) == 4;
    const uint32_t kBH = quick ? accept_threshold((float)(coef * (Real)a.f_bound[3 * mat + 2])) : 0u;
    // one 16-bit accept digit per pair (BH): slots 8q .. 8q + 7 share the
    // draw of counter q, slot 8q + h its digit h; a thread per slot
    for (uint32_t s = grp.rank(); s < Np; s += grp.size()) {
        const uint32_t q = s >> 3, h = s & 7u;
        {
            const int sl = p0 + (int)s;
            const uint32_t npass = pr.caseA ? 1u : (Nt - s + Np - 1) / Np;
            bool loaded = false;
            Real uk[3] = {0, 0, 0}, k = 0;
            for (uint32_t m = 0; m < npass; ++m) {
                uint32_t j, tau;
                const uint32_t rw =
                    accept_digit(draw(q, cell, a.step, stream_tag(kGroupPh, kAccept, m), a.seed), h);
                if (quick && !(rw <= kBH)) continue;   // exact quick reject
                if (pr.caseA) {
                    j = pr.pair_of_slot(s);
                    tau = j % Nt;
                } else {
                    j = s + m * Np;
                    tau = pr.target_of_pair(j);
                }
                if (quick) acc.candidates[kGroupPh]++;
                if (!loaded) {
                    uk[0] = (Real)P.ux[sl]; uk[1] = (Real)P.uy[sl]; uk[2] = (Real)P.uz[sl];
                    k = sqrt(uk[0] * uk[0] + uk[1] * uk[1] + uk[2] * uk[2]);
                    loaded = true;
                }
                if (!isfinite(k)) { acc.status |= PCC_ST_NONFINITE; break; }
                const int ts = t0 + (int)tau;
                Frame<Real> f;
                f.ui[0] = I.ux[ts]; f.ui[1] = I.uy[ts]; f.ui[2] = I.uz[ts];
                f.gi = sqrt((Real)1 + f.ui[0] * f.ui[0] + f.ui[1] * f.ui[1] + f.ui[2] * f.ui[2]);
                const Real d = f.ui[0] * uk[0] + f.ui[1] * uk[1] + f.ui[2] * uk[2];
                const Real kp = f.gi * k - d;
                const Real sig = sigma_at<Real>(tb, tb.hsig + (size_t)mat * a.g.n_rows, a.g, kp - (Real)2, acc.status);
                if (!(sig > (Real)0)) continue;
                const Real x = coef * sig * kp / (k * f.gi);
                if (x > (Real)1) acc.status |= PCC_ST_PROB_LARGE;
                const AcceptSrc src{8 * q + h, (uint32_t)cell, stream_tag(kGroupPh, kAcceptExt, m)};
                if (!accept_u<Real>(rw, -expm1(-x), src, a.step, a.seed)) continue;
                acc.accepted[kChBH]++;
                const Real fac = d / (f.gi + (Real)1) - k;
                const Real pv[3] = {uk[0] + fac * f.ui[0], uk[1] + fac * f.ui[1], uk[2] + fac * f.ui[2]};
                const Real pm = sqrt(pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]);
                f.n[0] = pv[0] / pm; f.n[1] = pv[1] / pm; f.n[2] = pv[2] / pm;
                const float xpos = has_x ? P.x[sl] : 0.f;
                const EventResult r = bh_event<Real>(ap, tb, cell, mat, j, P.w[sl], I.w[ts], xpos, f, kp, k);
                if (!r.created) continue;
                acc.created[kChBH]++;
                acc.dE += r.dE;
                acc.status |= r.status;
                wcre += r.wc;
                P.w[sl] = 0.f;   // removal marker, compacted below; skips the photon's later pairs
                absorbed_any = true;
                break;
            }
        }
    }
    if (grp.any(absorbed_any)) {
        grp.sync();
        if (a.ledger) {
            const float wc = grp.sum(wcre);
            if (grp.rank() == 0) {
                float4* L = reinterpret_cast<float4*>(a.ledger) + cell;
                float4 v = *L;
                Kahan k2{v.z, v.w};
                k2.add(wc);
                *L = make_float4(v.x, v.y, k2.s, k2.c);
            }
        }
        if (grp.rank() == 0) {   // stable compaction of the region (rare path)
            const int n_all = (int)Np + P.added[cell];
            int wr = 0, removed = 0;
            for (int i = 0; i < n_all; ++i) {
                const int src = p0 + i;
                if (i < (int)Np && P.w[src] == 0.f) { ++removed; continue; }
                if (wr != i) {
                    const int dst = p0 + wr;
                    P.ux[dst] = P.ux[src]; P.uy[dst] = P.uy[src]; P.uz[dst] = P.uz[src]; P.w[dst] = P.w[src];
                    if (has_x) P.x[dst] = P.x[src];
                    P.pid[dst] = P.pid[src];
                }
                ++wr;
            }
            P.count[cell] = (int)Np - removed;
        }
        grp.sync();
    }
}

// ---- kernels --------------------------------------------------------------------
__device__ void flush_acc(Acc& acc, DevStats* st, bool lane_reduce)
{
    unsigned long long pv[3];
    unsigned av[5], cv[5], kv[3];
    double dE = acc.dE, dQ = acc.dQ;
    unsigned status = acc.status;
    for (int i = 0; i < 3; ++i) pv[i] = acc.pairs[i], kv[i] = acc.candidates[i];
    for (int i = 0; i < 5; ++i) { av[i] = acc.accepted[i]; cv[i] = acc.created[i]; }
    if (lane_reduce) {
        for (int i = 0; i < 3; ++i) pv[i] = warp_sum(pv[i]), kv[i] = warp_sum(kv[i]);
        for (int i = 0; i < 5; ++i) { av[i] = warp_sum(av[i]); cv[i] = warp_sum(cv[i]); }
        dE = warp_sum(dE);
        dQ = warp_sum(dQ);
        status = __reduce_or_sync(0xffffffffu, status);
        if ((threadIdx.x & 31) != 0) return;
    }
    for (int i = 0; i < 3; ++i) {
        if (pv[i]) atomicAdd(&st->pairs[i], pv[i]);
        if (kv[i]) atomicAdd(&st->candidates[i], (unsigned long long)kv[i]);
    }
    for (int i = 0; i < 5; ++i) {
        if (av[i]) atomicAdd(&st->accepted[i], (unsigned long long)av[i]);
        if (cv[i]) atomicAdd(&st->created[i], (unsigned long long)cv[i]);
    }
    if (dE != 0.0) atomicAdd(&st->energy_change, dE);
    if (dQ != 0.0) atomicAdd(&st->charge_change, dQ);
    if (status) atomicOr(&st->status, status);
}

// Plain FP64: one block per cell.
template <int GROUP>
__global__ void __launch_bounds__(128) collide_plain_kernel(const __grid_constant__ StepArgs a)
{
    __shared__ int scratch[64];
    __shared__ double red[4];
    CtaGroup grp{scratch, red};
    Tab<double> tb{a.brems_sigma, a.brems_cdf, a.bh_sigma, a.bh_cdf, a.tri_gp, a.tri_split};
    Acc acc;
    acc.zero();
    const int cell = blockIdx.x;
    if (GROUP == kGroupPh) bh_cell<double>(grp, &a, tb, cell, acc);
    else ei_cell<double>(grp, &a, tb, GROUP, cell, acc);
    flush_acc(acc, a.st, true);
}

// Batched FP32 -----------------------------------------------------------------
// Every cell with both lists non-empty is scanned by one warp, or by a lane
// group of one when it is small.  Cells are listed by decreasing size class
// (bit length of N_pair) and dealt to the warps of a persistent grid
// round-robin, so each warp receives a similar share of large and small
// cells.
constexpr int kBatchedThreads = 256;
// Size classes of the cells, two per octave of N_pair = max(N_p, N_t)
// (see size_class).
constexpr int kClasses = 34;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

struct CellList {
    int* list;       // [n_cells], cells by decreasing size class
    int* hist;       // [kClasses] cells per class
    int* cursor;     // [kClasses] (unused)
    int* bh;         // [kClasses][nblk] per-block class counts, then their offsets
    int nblk;        // blocks of kClassBlock cells
    int thr[4];      // scan lane groups: classes >= thr[0] a whole warp, [thr[1], thr[0]) 16 lanes,
                     // [thr[2], thr[1]) 8, [thr[3], thr[2]) 4, below 2 (pcc_set_scan_classes)
};

constexpr int kClassBlock = 1024;                 // cells per class-sort block
constexpr int kClassSmemMax = 200 * 1024;         // offsets scanned in shared memory up to this size

// Class of a cell with N_pair = max(N_p, N_t) pairs: with b the bit length
// of N_pair, class 2(b - 1) for N_pair in [2^(b-1), 1.5 2^(b-1)) and
// 2(b - 1) + 1 for [1.5 2^(b-1), 2^b); N_pair = 1 is class 0.
__device__ __forceinline__ int size_class(int np, int nt)
{
    const int n = np > nt ? np : nt;
    const int b = 32 - __clz(n);
    const int k = b >= 2 ? 2 * (b - 1) + ((n >> (b - 2)) & 1) : 0;
    return k < kClasses ? k : kClasses - 1;
}

// The class sorts of the three groups {e-, e+, photon} against the ions,
// done together: the counts do not change during a collide call (secondaries
// are committed after it), so one pass reads the ion counts once.
struct ClassSort {
    CellList L[3];
    const int* cnt_p[3];   // projectile counts per group
    const int* cnt_t;      // ion counts
    int n_cells;
    unsigned run;          // bit g: group g is sorted
    unsigned* serial;      // collide calls so far (stamps the per-cell ion summaries)
};

// Counting sort of the cells with both species by decreasing size class,
// in three passes without global atomics: per-block class counts, their
// exclusive scan (classes from the largest, blocks in order), and the
// scatter with ranks from shared-memory counters.  The order within one
// block's cells of one class follows the shared atomics and may differ from
// run to run; no result depends on it, since every cell is processed
// independently of where it sits in the list.
__global__ void class_hist_kernel(const __grid_constant__ ClassSort S)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *S.serial += 1u;   // a new call: earlier summaries go stale
    __shared__ int h[3][kClasses];
    for (int i = threadIdx.x; i < 3 * kClasses; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < S.n_cells) {
        const int nt = S.cnt_t[c];
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            if (!(S.run >> g & 1u) || nt <= 0) continue;
            const int np = S.cnt_p[g][c];
            if (np > 0) atomicAdd(&h[g][size_class(np, nt)], 1);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * kClasses; i += blockDim.x) {
        const int g = i / kClasses, k = i - g * kClasses;
        if (S.run >> g & 1u) S.L[g].bh[k * S.L[g].nblk + blockIdx.x] = h[g][k];
    }
}

// One block per group: bh[k][b] -> offset of block b's cells of class k in
// the list; hist[k] -> cells of class k.  The counts are staged in shared
// memory when they fit (SMEM = true), else scanned in place in global memory.
template <bool SMEM>
__global__ void __launch_bounds__(1024) class_offsets_kernel(const __grid_constant__ ClassSort S)
{
    extern __shared__ int sm[];
    __shared__ int part[32];
    if (!(S.run >> blockIdx.x & 1u)) return;
    const CellList& L = S.L[blockIdx.x];
    const int n = kClasses * L.nblk;
    int* v = SMEM ? sm : L.bh;
    if (SMEM)
        for (int i = threadIdx.x; i < n; i += blockDim.x) sm[i] = L.bh[i];
    __syncthreads();
    // scan order: classes from the largest, blocks in order; thread t takes
    // a contiguous chunk [i0, i1) of that order, entry (class k, block b)
    // stepped without divisions
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int i0 = min((int)threadIdx.x * per, n), i1 = min(i0 + per, n);
    const int k0 = kClasses - 1 - i0 / L.nblk, b0 = i0 - (kClasses - 1 - k0) * L.nblk;
    int sum = 0;
    for (int e = i0, k = k0, b = b0; e < i1; ++e) {
        sum += v[k * L.nblk + b];
        if (++b == L.nblk) { b = 0; --k; }
    }
    // exclusive scan of the thread sums: within each warp by shuffles, then
    // over the warp totals
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) part[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int x = lane < nw ? part[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        part[lane] = x;
    }
    __syncthreads();
    int run = (wid ? part[wid - 1] : 0) + incl - sum;
    for (int e = i0, k = k0, b = b0; e < i1; ++e) {
        int& x = v[k * L.nblk + b];
        const int c = x;
        x = run;
        run += c;
        if (++b == L.nblk) { b = 0; --k; }
    }
    __syncthreads();
    // class k occupies [offset of its block 0, offset of block 0 of class
    // k - 1) of the list; class 0 ends at the total
    if (threadIdx.x < kClasses) {
        const int k = threadIdx.x;
        const int end = k == 0 ? part[nw - 1] : v[(k - 1) * L.nblk];
        L.hist[k] = end - v[k * L.nblk];
    }
    if (SMEM)
        for (int i = threadIdx.x; i < n; i += blockDim.x) L.bh[i] = sm[i];
}

__global__ void class_scatter_kernel(const __grid_constant__ ClassSort S)
{
    __shared__ int rank[3][kClasses];
    for (int i = threadIdx.x; i < 3 * kClasses; i += blockDim.x) (&rank[0][0])[i] = 0;
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < S.n_cells) {
        const int nt = S.cnt_t[c];
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            if (!(S.run >> g & 1u) || nt <= 0) continue;
            const int np = S.cnt_p[g][c];
            if (np > 0) {
                const int cls = size_class(np, nt);
                const CellList& L = S.L[g];
                L.list[L.bh[cls * L.nblk + blockIdx.x] + atomicAdd(&rank[g][cls], 1)] = c;
            }
        }
    }
}

// Poll the mbarrier at smem address b for phase 0, at most `polls` times;
// true once the phase has completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t b, int polls)
{
    uint32_t done = 0;
    for (int it = 0; it < polls && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(b)
            : "memory");
    }
    return done != 0;
}

// Stage the ln sigma rows (n_mat x n_rows floats) in shared memory with one
// bulk copy; returns the shared copy, or the global one if the wait gives up
// after `polls` polls (status PCC_ST_TIMEOUT).  A block that gave up still
// waits, bounded again, for its copy to land before going on, so that no
// copy into its shared memory is left in flight; the global rows hold the
// same values, so only the status differs.
__device__ const float* stage_table(const float* src, int bytes, unsigned char* dyn, unsigned long long* bar,
                                    int polls, unsigned& status)
{
    if (bytes <= 0) return src;
    const uint32_t b = smem_u32(bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(dyn)),
                     "l"(src), "r"(bytes), "r"(b)
                     : "memory");
    }
    const bool done = mbar_wait_bounded(b, polls);
    const int all = __syncthreads_and((int)done);
    if (!all) {
        status |= PCC_ST_TIMEOUT;
        mbar_wait_bounded(b, 1 << 22);   // let this block's copy land
        __syncthreads();
        return src;
    }
    return reinterpret_cast<const float*>(dyn);
}

template <int GROUP>
__device__ __forceinline__ Tab<float> batched_tab(const StepArgs& a, const float* staged)
{
    return Tab<float>{GROUP == kGroupPh ? a.f_brems_lnsig : staged, a.f_brems_cdf,
                      GROUP == kGroupPh ? staged : a.f_bh_lnsig, a.f_bh_cdf, a.f_tri_gp, a.f_tri_split};
}

// j mod n for j < 2^24 via a float reciprocal (exact after the correction).
__device__ __forceinline__ uint32_t fast_mod(uint32_t j, uint32_t n, float inv_n)
{
    uint32_t q = __float2uint_rz((float)j * inv_n);
    int r = (int)j - (int)(q * n);
    if (r < 0) r += (int)n;
    if (r >= (int)n) r -= (int)n;
    return (uint32_t)r;
}

// i = quot n + rem for n >= 1 by a float reciprocal (inv_n = 1/n), exact: the
// estimate is off by at most one below 2^24, and larger i divide exactly.
__device__ __forceinline__ void div_small(uint32_t i, uint32_t n, float inv_n, uint32_t& quot, uint32_t& rem)
{
    if (i >= (1u << 24)) {
        quot = i / n;
        rem = i - quot * n;
        return;
    }
    uint32_t qq = __float2uint_rz((float)i * inv_n);
    int r = (int)i - (int)(qq * n);
    if (r < 0) { r += (int)n; --qq; }
    if (r >= (int)n) { r -= (int)n; ++qq; }
    quot = qq;
    rem = (uint32_t)r;
}

// Per-cell summary of the ions written by the electron scan, which reads
// every ion of its cells anyway, for the positron and photon scans of the
// same call: x = n_t (the electron scan's FP32 sum), y = w0 (first ion
// weight), z = 1 + max |beta_i| rounded up (negative when the ion weights are
// not all w0), w = the call's serial (bits).  A scan whose cell carries
// another serial (no electrons there, or the electron group did not run in
// this call) reads the ion weights itself.
struct IonCache {
    float4* sum;            // [n_cells]
    const unsigned* serial; // incremented by the class sort at the start of each call
};

// Per-cell metadata, loaded one cell ahead by the persistent loop.
struct CellMeta {
    int cell, p0, t0, mat;
    uint32_t Np, Nt;
};

__device__ __forceinline__ CellMeta load_meta(const StepArgs& a, const SpeciesView& P, int cell)
{
    CellMeta m;
    m.cell = cell;
    // a list entry outside [0, n_cells) is skipped (never read through)
    if (cell < 0 || cell >= a.n_cells) { m.Np = m.Nt = 0; m.p0 = m.t0 = m.mat = 0; return m; }
    m.Np = P.count[cell];
    m.Nt = a.ion.count[cell];
    m.p0 = P.start[cell];
    m.t0 = a.ion.start[cell];
    m.mat = a.mat_of_cell[cell];
    return m;
}

// Per-block counters of the batched kernels, updated with shared atomics and
// added to the context's counters once per block.
struct BlockAcc {
    unsigned long long pairs[3], accepted[5], created[5], candidates[3];
    double dE;
    unsigned status;
};

__device__ __forceinline__ void block_acc_init(BlockAcc& b)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < 3; ++i) b.pairs[i] = b.candidates[i] = 0;
        for (int i = 0; i < 5; ++i) b.accepted[i] = b.created[i] = 0;
        b.dE = 0.0;
        b.status = 0;
    }
}

__device__ __forceinline__ void block_acc_flush(const BlockAcc& b, DevStats* st)
{
    if (threadIdx.x != 0) return;
    for (int i = 0; i < 3; ++i) {
        if (b.pairs[i]) atomicAdd(&st->pairs[i], b.pairs[i]);
        if (b.candidates[i]) atomicAdd(&st->candidates[i], b.candidates[i]);
    }
    for (int i = 0; i < 5; ++i) {
        if (b.accepted[i]) atomicAdd(&st->accepted[i], b.accepted[i]);
        if (b.created[i]) atomicAdd(&st->created[i], b.created[i]);
    }
    if (b.dE != 0.0) atomicAdd(&st->energy_change, b.dE);
    if (b.status) atomicOr(&st->status, b.status);
}

// Candidate queues and per-call cell state of the batched path.
struct Queue {
    uint2* flat;          // [cap_flat] (cell, projectile slot) of candidates in cells with N_p >= N_t
    int* flat_count;      // [1]
    uint32_t cap_flat;
    uint32_t* qb;         // [target capacity] pair indices of candidates in cells with N_p < N_t,
                          // written into the cell's target region in increasing pair order per projectile
    int* cand;            // [n_cells] such candidates of the cell
    int* caseb;           // [n_cells] cells with N_p < N_t and candidates
    int* caseb_count;     // [1]
    int* flagged;         // [n_cells] cells with an event in this call
    int* flagged_count;   // [1]
    int* flag;            // [n_cells] 1 once listed (cleared by the finalize kernel)
    float2* evacc;        // [n_cells] this call's ledger contributions (radiated energy, created weight)
    int4* rec;            // [2 n_cells] per cell with candidates: {p0, t0, N_p, N_t}, {mat, coef bits, 0, 0}
};

// The scan leaves the cell data the candidate kernels need in one 32-byte
// record (a single sector) instead of five metadata arrays and the
// coefficient.
struct CellRec {
    int p0, t0;
    uint32_t Np, Nt;
    int mat;
    float coef;
};

__device__ __forceinline__ CellRec load_rec(const Queue& Q, int cell)
{
    const int4 r0 = Q.rec[2 * (size_t)cell], r1 = Q.rec[2 * (size_t)cell + 1];
    CellRec c;
    c.p0 = r0.x; c.t0 = r0.y; c.Np = (uint32_t)r0.z; c.Nt = (uint32_t)r0.w;
    c.mat = r1.x; c.coef = __int_as_float(r1.y);
    return c;
}

__device__ __forceinline__ void flag_cell(const Queue& Q, int cell)
{
    if (atomicCAS(&Q.flag[cell], 0, 1) == 0) Q.flagged[atomicAdd(Q.flagged_count, 1)] = cell;
}

// Acceptance bounds of the group at this coefficient, as thresholds on the
// 16-bit accept digits: a pair can be accepted only if a <= floor(2^16 b).  The
// per-material bounds carry the ion-motion factor 1 + |beta_i| at its
// largest value 2; for the electrons the scan passes coef times
// (1 + max |beta_i|)/2 of the cell, which halves their candidates where the
// ions are slow.
template <int GROUP>
__device__ __forceinline__ void bound_thresholds(const StepArgs& a, int mat, float coef, uint32_t& k1, uint32_t& k2)
{
    float b1, b2;
    if (GROUP == kGroupPh) {
        b1 = coef * a.f_bound[3 * mat + 2];
        b2 = 0.f;
    } else {
        b1 = (a.mask & PCC_BREMS) ? coef * a.f_bound[3 * mat] : 0.f;
        b2 = (a.mask & PCC_TRIDENT) ? coef * a.f_bound[3 * mat + 1] : 0.f;
    }
    k1 = accept_threshold(b1);
    k2 = accept_threshold(b2);
}

// One photon-ion candidate pair (Bethe-Heitler); returns true when the photon
// is absorbed (its weight is then set to 0 for the compaction).
__device__ __forceinline__ bool bh_candidate(const StepArgs& a, const Tab<float>& tb, int cell, int mat, float coef,
                                             int sl, int ts, uint32_t j, uint32_t rw, const AcceptSrc& src, Acc& acc,
                                             float& wcre)
{
    const SpeciesView& P = a.ph;
    const SpeciesView& I = a.ion;
    const float uk[3] = {P.ux[sl], P.uy[sl], P.uz[sl]};
    const float k = sqrtf(uk[0] * uk[0] + uk[1] * uk[1] + uk[2] * uk[2]);
    if (!isfinite(k)) {
        acc.status |= PCC_ST_NONFINITE;
        return false;
    }
    Frame<float> f;
    f.ui[0] = I.ux[ts]; f.ui[1] = I.uy[ts]; f.ui[2] = I.uz[ts];
    f.gi = q_sqrt1(1.f + f.ui[0] * f.ui[0] + f.ui[1] * f.ui[1] + f.ui[2] * f.ui[2]);
    const float d = f.ui[0] * uk[0] + f.ui[1] * uk[1] + f.ui[2] * uk[2];
    const float kp = f.gi * k - d;
    const float sig = sigma_at<float>(tb, tb.hsig + (size_t)mat * a.g.n_rows, a.g, kp - 2.f, acc.status);
    if (!(sig > 0.f)) return false;
    const float x = q_div(coef * sig * kp, k * f.gi);
    if (x > 1.f) acc.status |= PCC_ST_PROB_LARGE;
    if (!accept_u<float>(rw, -expm1f(-x), src, a.step, a.seed)) return false;
    acc.accepted[kChBH]++;
    const float fac = q_div(d, f.gi + 1.f) - k;
    const float pv[3] = {uk[0] + fac * f.ui[0], uk[1] + fac * f.ui[1], uk[2] + fac * f.ui[2]};
    const float pm = sqrtf(pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]);
    f.n[0] = pv[0] / pm; f.n[1] = pv[1] / pm; f.n[2] = pv[2] / pm;
    const float xpos = P.x ? P.x[sl] : 0.f;
    const EventResult r = bh_event<float>(&a, tb, cell, mat, j, P.w[sl], I.w[ts], xpos, f, kp, k);
    if (!r.created) return false;
    acc.created[kChBH]++;
    acc.dE += r.dE;
    acc.status |= r.status;
    wcre += r.wc;
    P.w[sl] = 0.f;   // removal marker
    return true;
}

// The accept digits of projectile slot s (random-stream layout; a draw holds
// eight 16-bit digits, see accept_digit): an e+- pair takes digits 2(s&3)
// (Brems) and 2(s&3)+1 (Trident) of counter s>>2, a photon pair, which has
// one (BH), digit s&7 of counter s>>3.  The extension draw of digit d of
// counter q has counter 8q + d: 2s (Brems), 2s + 1 (Trident), s (BH).
template <int GROUP>
struct AcceptSlots {
    static constexpr uint32_t kPerDraw = GROUP == kGroupPh ? 8u : 4u;
    static __device__ __forceinline__ uint32_t ctr(uint32_t s) { return GROUP == kGroupPh ? s >> 3 : s >> 2; }
    static __device__ __forceinline__ uint32_t digit(uint32_t s) { return GROUP == kGroupPh ? (s & 7u) : 2u * (s & 3u); }
    static __device__ __forceinline__ uint32_t ext(uint32_t s) { return GROUP == kGroupPh ? s : 2u * s; }
    // slot kPerDraw q + h of a draw: may the pair be accepted under the digit
    // thresholds k1 (Brems or BH), k2 (Trident)?  A high half is tested on
    // the whole word (w >> 16 <= k iff w <= 2^16 k + 0xFFFF).
    static __device__ __forceinline__ bool hit(const Philox4& d, int h, uint32_t k1, uint32_t k2)
    {
        const uint32_t hi1 = (k1 << 16) | 0xFFFFu;
        if (GROUP == kGroupPh) return (h & 1) ? (d.v[h >> 1] & 0xFFFFu) <= k1 : d.v[h >> 1] <= hi1;
        return d.v[h] <= hi1 || (d.v[h] & 0xFFFFu) <= k2;
    }
};

// Philox4x32-10 on counters (x, c1, c2, c3) with only x varying: the first
// round's product of c2 and the second round's product of the first word do
// not depend on x, so they are taken once (PhiloxFixed) and each draw
// multiplies 18 times instead of 20.  The result equals draw_k(x, c1, c2, c3).
struct PhiloxFixed { uint32_t t0, b1, c1k, d1; };
__device__ __forceinline__ PhiloxFixed philox_fixed(uint32_t c1, uint32_t c2, uint32_t c3, const PhiloxKeys& K)
{
    const uint64_t m1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t a = (uint32_t)(m1 >> 32) ^ c1 ^ K.k0[0];   // word 0 after round 1
    const uint64_t m0 = (uint64_t)0xD2511F53u * a;             // its round-2 product
    PhiloxFixed f;
    f.t0 = c3 ^ K.k1[0];
    f.b1 = (uint32_t)m1 ^ K.k0[1];
    f.c1k = (uint32_t)(m0 >> 32) ^ K.k1[1];
    f.d1 = (uint32_t)m0;
    return f;
}
__device__ __forceinline__ Philox4 draw_fixed(uint32_t x, const PhiloxFixed& f, const PhiloxKeys& K)
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * x;                 // round 1
    const uint32_t w2 = (uint32_t)(p0 >> 32) ^ f.t0, w3 = (uint32_t)p0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * w2;                // round 2
    uint32_t c0 = (uint32_t)(p1 >> 32) ^ f.b1, c1 = (uint32_t)p1, c2 = f.c1k ^ w3, c3 = f.d1;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint64_t m0 = (uint64_t)0xD2511F53u * c0, m1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(m1 >> 32) ^ c1 ^ K.k0[r], n2 = (uint32_t)(m0 >> 32) ^ c3 ^ K.k1[r];
        c1 = (uint32_t)m1; c3 = (uint32_t)m0; c0 = n0; c2 = n2;
    }
    Philox4 o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// Sum over the G consecutive lanes of an aligned lane group (G a power of two).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int G>
__device__ __forceinline__ float group_max(float v)
{
#pragma unroll
    for (int o = G >> 1; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// n_pt of one cell summed over its actual pairs, for cells whose target
// weights are not all equal.  All 32 lanes take part; the result is
// warp-uniform.  Lists of at most 32 entries are permuted by rank keys
// staged in tab (64 ints), longer ones by the Feistel walk.
template <int GROUP>
__device__ __forceinline__ float npt_over_pairs(const StepArgs& a, const SpeciesView& P, int cell, int p0, int t0,
                                                uint32_t Np, uint32_t Nt, int* tab, int lane)
{
    const SpeciesView& I = a.ion;
    const bool caseA = Np >= Nt;
    const Philox4 kp = draw_k(0, (uint32_t)cell, (uint32_t)a.step, stream_tag(GROUP, kPerm, 0), a.keys);
    PermKeys rk;
    rk.k[0] = kp.v[0]; rk.k[1] = kp.v[1]; rk.k[2] = kp.v[2]; rk.k[3] = kp.v[3];
    const uint32_t NL = caseA ? Np : Nt;
    if (NL <= 32) {
        __syncwarp();
        if (lane < (int)NL) {
            const uint32_t r = perm_pos_small(lane, NL, rk);
            tab[r] = lane;    // P table
            tab[32 + lane] = r;
        }
        __syncwarp();
    }
    float spt = 0.f;
    const float inv_nt = 1.0f / (float)Nt;
    if (caseA) {
        for (uint32_t s = lane; s < Np; s += 32) {
            const uint32_t j = NL <= 32 ? (uint32_t)tab[32 + s] : perm_pos_large(s, Np, rk);
            spt += fminf(P.w[p0 + s], I.w[t0 + fast_mod(j, Nt, inv_nt)]);
        }
    } else {   // lanes over the pairs: projectile j mod N_p, target P(j)
        for (uint32_t j = lane; j < Nt; j += 32) {
            const uint32_t t = NL <= 32 ? (uint32_t)tab[j] : perm_elem_large(j, Nt, rk);
            spt += fminf(P.w[p0 + j % Np], I.w[t0 + t]);
        }
    }
    return warp_sum(spt);
}

constexpr int kWarpBuf = 256;   // per-warp staging of candidates before the flat queue

// Scan state of one warp, carried from one size-class segment to the next.
struct ScanWarp {
    int nb;                              // candidates staged in the warp buffer (warp-uniform)
    unsigned long long npairs, ncands;   // counts of the cells this lane leads
};

__device__ __forceinline__ void flush_staged(const Queue& Q, const uint2* wb, int nb, BlockAcc& bacc, int lane)
{
    __syncwarp();
    int base_q = 0;
    if (lane == 0) base_q = atomicAdd(Q.flat_count, nb);
    base_q = __shfl_sync(0xffffffffu, base_q, 0);
    for (int i = lane; i < nb; i += 32)
        if ((uint32_t)(base_q + i) < Q.cap_flat) Q.flat[base_q + i] = wb[i];
    if (lane == 0 && (uint32_t)(base_q + nb) > Q.cap_flat) atomicOr(&bacc.status, PCC_ST_CAPACITY);
    __syncwarp();
}

// Stage the candidates a lane marked in cmask (bit (it - it0) S + h: slot
// S (it G + gl) + h of its cell, iteration it of the accept loop) in the
// warp's buffer, after a warp-wide prefix of the counts; a buffer that would
// overflow goes to the flat queue first, and a batch larger than the buffer
// (every pair a candidate) straight to it.  All 32 lanes call it.
template <int G, uint32_t S>
__device__ __forceinline__ void emit_candidates(const Queue& Q, uint2* wb, ScanWarp& sw, int cell, uint32_t cmask,
                                                uint32_t it0, int gl, int lane, BlockAcc& bacc)
{
    const uint32_t n = __popc(cmask);
    uint32_t incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = (int)__shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    if (sw.nb + total > kWarpBuf) {
        flush_staged(Q, wb, sw.nb, bacc, lane);
        sw.nb = 0;
    }
    const bool direct = total > kWarpBuf;
    uint32_t base = (uint32_t)sw.nb;
    if (direct) {
        if (lane == 0) base = (uint32_t)atomicAdd(Q.flat_count, total);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane == 0 && base + (uint32_t)total > Q.cap_flat) atomicOr(&bacc.status, PCC_ST_CAPACITY);
    }
    uint32_t k = base + incl - n;
    while (cmask) {
        const uint32_t b = (uint32_t)(__ffs(cmask) - 1);
        cmask &= cmask - 1u;
        const uint2 e = make_uint2((uint32_t)cell, ((it0 + b / S) * G + (uint32_t)gl) * S + b % S);
        if (!direct) wb[k] = e;
        else if (k < Q.cap_flat) Q.flat[k] = e;
        ++k;
    }
    if (!direct) sw.nb += total;
}

// The cells of list entries [e0, e1), taken C = 32 / G at a time by a warp:
// lane group g (lanes gG .. gG + G - 1) owns one cell, its lane l owns the
// S slots base + S l .. base + S l + S - 1 per pass, whose accept digits are
// those of the lane's Philox draw (S = 4 for e+-, 8 for photons; the counter
// depends on the slot, not on the lane, so the random stream does not depend
// on G).  Tuples of C
// entries are dealt to the warps round-robin starting at tuple t_first.
// Loops that hold ballots run to the largest trip count of the warp's
// groups, so every collective is reached by all 32 lanes.
template <int GROUP, int G>
__device__ __forceinline__ void scan_segment(const StepArgs& a, const CellList& L, const Queue& Q, const IonCache& IC,
                                             int e0, int e1, int t_first, int nwarps, int* tab,
                                             uint2* wb, ScanWarp& sw, BlockAcc& bacc)
{
    constexpr int C = 32 / G;
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, gi = lane / G, gl = lane % G;
    const unsigned gmask = G == 32 ? kFull : ((1u << G) - 1u) << (gi * G);
    const unsigned below = (1u << lane) - 1u;
    const SpeciesView& P = GROUP == kGroupEm ? a.em : (GROUP == kGroupEp ? a.ep : a.ph);
    const SpeciesView& I = a.ion;
    const uint32_t step32 = (uint32_t)a.step;
    const int ntup = (e1 - e0 + C - 1) / C;
    const int e_lane = e0 + gi;   // entry of tuple t for this lane: e_lane + t C
    // Two-stage prefetch: the metadata of the tuple after next, and (electron
    // scan) the first G ion weights of the next tuple, load while a tuple is
    // scanned.
    constexpr bool kWriter = GROUP == kGroupEm;   // the electron scan writes the ion summaries
    const auto first_ion = [&](const CellMeta& m) -> float {
        return (uint32_t)gl < m.Nt ? I.w[m.t0 + gl] : 0.f;
    };
    const auto ion_sum = [&](const CellMeta& m) -> float4 {
        return (m.cell >= 0 && m.cell < a.n_cells) ? IC.sum[m.cell] : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    int t = t_first;
    CellMeta next = load_meta(a, P, t < ntup && e_lane + t * C < e1 ? L.list[e_lane + t * C] : -1);
    float next_tw = kWriter ? first_ion(next) : 0.f;
    float4 next_is = kWriter ? make_float4(0.f, 0.f, 0.f, 0.f) : ion_sum(next);
    int t2 = t + nwarps;
    CellMeta next2 = load_meta(a, P, t2 < ntup && e_lane + t2 * C < e1 ? L.list[e_lane + t2 * C] : -1);
    while (t < ntup) {
        const CellMeta cm = next;
        float tw0 = next_tw;
        const float4 is = next_is;   // its ion summary (readers)
        t += nwarps;
        next = next2;
        if constexpr (kWriter) next_tw = first_ion(next);
        else next_is = ion_sum(next);
        t2 = t + nwarps;
        next2 = load_meta(a, P, t2 < ntup && e_lane + t2 * C < e1 ? L.list[e_lane + t2 * C] : -1);
        uint32_t Np = cm.Np, Nt = cm.Nt;
        const int cell = cm.cell, p0 = cm.p0, t0 = cm.t0, mat = cm.mat;
        bool active = Np != 0 && Nt != 0;
        if (active && (unsigned)mat >= (unsigned)a.n_mat) {
            if (gl == 0) atomicOr(&bacc.status, PCC_ST_NONFINITE);
            active = false;
        }
        if constexpr (G == 32) {   // one cell per warp: warp-uniform
            if (!active) continue;
        } else {
            if (!active) Np = Nt = 0;
            if (!__any_sync(kFull, active)) continue;
        }
        const bool caseA = Np >= Nt;
        // ---- sums (the first G weights of each list were prefetched).  The
        // electron scan sums the ion weights and takes the largest ion speed
        // of the cell for the bound (beta^2 = u^2/(1 + u^2); non-finite
        // momenta give beta = 1); the other scans take both from the
        // electron scan's summary when it is from this call, else sum the ion
        // weights themselves and keep the bound's factor at 2.
        const bool have = !kWriter && __float_as_uint(is.w) == *IC.serial;
        if (!kWriter && !have) tw0 = first_ion(cm);
        // (every collective below runs on all 32 lanes; `have` only selects)
        const float w0s = __shfl_sync(kFull, tw0, 0, G);
        const float w0 = have ? is.y : w0s;
        float sp = 0.f, st = 0.f, sf = 0.f, b2 = 0.f;
        bool uni = have ? is.z > 0.f : true;
        if (!have) {
            // beta^2 = u^2 / (1 + u^2) is increasing in u^2: the lane keeps
            // the largest u^2, and the sum of them only to see whether any
            // was non-finite (then beta = 1)
            float u2m = 0.f, u2s = 0.f;
#pragma unroll 4
            for (uint32_t s = gl; s < Nt; s += G) {
                const float wt = s < (uint32_t)G ? tw0 : I.w[t0 + s];
                st += wt;
                uni &= (wt == w0);
                if constexpr (kWriter) {
                    const float ux = I.ux[t0 + s], uy = I.uy[t0 + s], uz = I.uz[t0 + s];
                    const float u2 = ux * ux + uy * uy + uz * uz;
                    u2m = fmaxf(u2m, u2);
                    u2s += u2;
                }
            }
            // (u^2 >= 1e30 gives beta^2 = 1 to float precision)
            if constexpr (kWriter) b2 = isfinite(u2s) && u2m < 1e30f ? __fdividef(u2m, 1.f + u2m) : 1.f;
            else b2 = (uint32_t)gl < Nt ? 1.f : 0.f;
        }
        const float st_sum = group_sum<G>(st);
        const float n_t = have ? is.x : st_sum;
        // 1 + max |beta_i| of the cell, rounded up past the few ulps of its
        // float evaluation (2 without the summary in the other scans)
        const float bmax = group_max<G>(b2);
        float bfac;
        if (have) {
            bfac = fabsf(is.z);
        } else {   // sqrt as b rsqrt(b): its few-ulp error is far inside the 2^-20 margin
            const float bm = fminf(bmax, 1.f);
            bfac = fminf((1.f + (bm > 0.f ? bm * rsqrtf(bm) : 0.f)) * (1.f + 0x1p-20f), 2.f);
        }
        if constexpr (kWriter) {
            if (active && gl == 0)
                IC.sum[cell] = make_float4(n_t, w0, uni ? bfac : -bfac, __uint_as_float(*IC.serial));
        }
        if (caseA) {
            // the weights as float4 from the region's first 16-byte boundary
            // (its start rounded up), the ragged head and tail (at most 3 + 3
            // weights) one by one
            const uint32_t al = (uint32_t)((reinterpret_cast<uintptr_t>(P.w + p0) >> 2) & 3u);
            const uint32_t hd = min((4u - al) & 3u, Np), nb = (Np - hd) >> 2, tl = Np - hd - 4 * nb;
            const float4* W4 = reinterpret_cast<const float4*>(P.w + p0 + hd);
#pragma unroll 2
            for (uint32_t v = gl; v < nb; v += G) {
                const float4 q = W4[v];
                sp += (q.x + q.y) + (q.z + q.w);
                sf += (fminf(q.x, w0) + fminf(q.y, w0)) + (fminf(q.z, w0) + fminf(q.w, w0));
            }
            for (uint32_t i = gl; i < hd + tl; i += G) {
                const float wp = P.w[p0 + (i < hd ? i : 4 * nb + i)];
                sp += wp;
                sf += fminf(wp, w0);
            }
        } else {   // projectile s takes part in ceil((N_t - s) / N_p) = q0 + [s < r0] pairs, N_t = q0 N_p + r0
            const uint32_t q0 = Nt / Np, r0 = Nt - q0 * Np;
            for (uint32_t s = gl; s < Np; s += G) {
                const float wp = P.w[p0 + s];
                sp += wp;
                sf += fminf(wp, w0) * (float)(q0 + (s < r0 ? 1u : 0u));
            }
        }
        const float n_p = group_sum<G>(sp);
        float n_pt;
        if constexpr (G == 32) {
            n_pt = __all_sync(kFull, uni) ? warp_sum(sf) : npt_over_pairs<GROUP>(a, P, cell, p0, t0, Np, Nt, tab, lane);
        } else {
            n_pt = group_sum<G>(sf);
            // unequal target weights: n_pt over the actual pairs, one such
            // cell at a time with the whole warp
            unsigned odd = __ballot_sync(kFull, !uni);
            odd = __ballot_sync(kFull, active && gl == 0 && (odd & gmask) != 0u);
            while (odd) {
                const int src = __ffs(odd) - 1;
                odd &= odd - 1u;
                const float v = npt_over_pairs<GROUP>(a, P, __shfl_sync(kFull, cell, src),
                                                      __shfl_sync(kFull, p0, src), __shfl_sync(kFull, t0, src),
                                                      __shfl_sync(kFull, Np, src), __shfl_sync(kFull, Nt, src), tab,
                                                      lane);
                if (gi == src / G) n_pt = v;
            }
        }
        const float coef = __fdividef(n_p, n_pt) * n_t * a.f_cdt;
        uint32_t k1 = 0, k2 = 0;
        if (active) bound_thresholds<GROUP>(a, mat, coef * (0.5f * bfac), k1, k2);
        uint32_t ncand = 0;   // candidates of this lane's cell (uniform over its group)
        // ---- cells with N_p >= N_t: one pair per projectile slot; a lane
        // takes the S slots of one draw per iteration (S = 2 for e+-, 4 for
        // photons)
        using AS = AcceptSlots<GROUP>;
        constexpr uint32_t S = AS::kPerDraw;
        const uint32_t itA = active && caseA ? (Np + S * G - 1) / (S * G) : 0u;
        const uint32_t nitA = G == 32 ? itA : __reduce_max_sync(kFull, itA);
        const PhiloxFixed pf = philox_fixed((uint32_t)cell, step32, stream_tag(GROUP, kAccept, 0), a.keys);
        uint32_t mine = 0;   // candidates of this lane
        if constexpr (GROUP != kGroupPh) {
            // e+-: candidates are marked in a per-lane mask, 32 / S
            // iterations per mask, and staged when it is full or the loop ends
            constexpr uint32_t kIt = 32 / S;
            uint32_t cmask = 0, it0 = 0;
            for (uint32_t it = 0; it < nitA; ++it) {
                const Philox4 ph = draw_fixed(it * G + gl, pf, a.keys);
                const uint32_t s0 = (it * G + gl) * S;
                const uint32_t lim = (G == 32 || it < itA) && s0 < Np ? Np - s0 : 0u;   // live slots of the draw
#pragma unroll
                for (int h = 0; h < (int)S; ++h)
                    if ((uint32_t)h < lim && AS::hit(ph, h, k1, k2)) cmask |= 1u << ((it - it0) * S + h);
                if (it - it0 == kIt - 1 || it + 1 == nitA) {   // warp-uniform
                    mine += __popc(cmask);
                    emit_candidates<G, S>(Q, wb, sw, cell, cmask, it0, gl, lane, bacc);
                    cmask = 0;
                    it0 = it + 1;
                }
            }
        } else {
            // photons (rarer candidates, eight slots a draw): a vote per
            // iteration, ballots only when some lane has a candidate
            for (uint32_t it = 0; it < nitA; ++it) {
                const Philox4 ph = draw_fixed(it * G + gl, pf, a.keys);
                const bool live = G == 32 || it < itA;
                const uint32_t s0 = (it * G + gl) * S;
                bool c[S];
                uint32_t nc = 0;
#pragma unroll
                for (int h = 0; h < (int)S; ++h) {
                    c[h] = live && s0 + h < Np && AS::hit(ph, h, k1, k2);
                    nc += (uint32_t)c[h];
                }
                if (__any_sync(kFull, nc != 0)) {
                    if (sw.nb + (int)__reduce_add_sync(kFull, nc) > kWarpBuf) {   // room for this iteration's candidates
                        flush_staged(Q, wb, sw.nb, bacc, lane);
                        sw.nb = 0;
                    }
#pragma unroll
                    for (int h = 0; h < (int)S; ++h) {
                        const unsigned m = __ballot_sync(kFull, c[h]);
                        if (c[h]) wb[sw.nb + __popc(m & below)] = make_uint2((uint32_t)cell, s0 + h);
                        sw.nb += __popc(m);
                        mine += (uint32_t)c[h];
                    }
                }
            }
        }
        ncand = group_sum<G>(mine);
        // ---- cells with N_p < N_t.  Draw units (pass m, draw q): unit
        // i = m Qn + q covers slots S q .. S q + S - 1 of pass m, i.e. pairs
        // j = s + m N_p.  A group's lanes take consecutive units, so each
        // projectile's pairs are queued in increasing j.
        uint32_t cnt = 0;
        if (__any_sync(kFull, active && !caseA)) {   // most warps hold no such cell
            const uint32_t Qn = (Np + S - 1) / S, passes = Np ? (Nt + Np - 1) / Np : 0u, units = Qn * passes;
            const uint32_t itB = active && !caseA ? (units + G - 1) / G : 0u;
            const uint32_t nitB = G == 32 ? itB : __reduce_max_sync(kFull, itB);
            const float inv_qn = Qn ? 1.0f / (float)Qn : 0.f;
            for (uint32_t it = 0; it < nitB; ++it) {
                const uint32_t i = it * G + gl;
                const bool valid = (G == 32 || it < itB) && i < units;
                uint32_t mp = 0u, q = 0u;
                if (valid) div_small(i, Qn, inv_qn, mp, q);
                const Philox4 ph = draw_k(q, (uint32_t)cell, step32, stream_tag(GROUP, kAccept, mp), a.keys);
                bool c[S], anyc = false;
#pragma unroll
                for (int h = 0; h < (int)S; ++h) {
                    const uint32_t s = S * q + h;
                    c[h] = valid && s < Np && s + mp * Np < Nt && AS::hit(ph, h, k1, k2);
                    anyc |= c[h];
                }
                if (!__any_sync(kFull, anyc)) continue;   // the common case: no candidate in the warp
#pragma unroll
                for (int h = 0; h < (int)S; ++h) {
                    const unsigned m = __ballot_sync(kFull, c[h]);
                    if (c[h]) Q.qb[t0 + cnt + __popc(m & gmask & below)] = S * q + h + mp * Np;
                    cnt += __popc(m & gmask);
                }
            }
        }
        if (!caseA) ncand = cnt;
        if (gl == 0 && active) {
            if (!caseA) {
                Q.cand[cell] = (int)cnt;
                if (cnt) Q.caseb[atomicAdd(Q.caseb_count, 1)] = cell;
            }
            if (ncand) {
                Q.rec[2 * (size_t)cell] = make_int4(p0, t0, (int)Np, (int)Nt);
                Q.rec[2 * (size_t)cell + 1] = make_int4(mat, __float_as_int(coef), 0, 0);
            }
            sw.npairs += caseA ? Np : Nt;
            sw.ncands += ncand;
            if ((caseA ? Np : Nt) > 65536u || (uint32_t)cell > 0xFFFFFFu || a.step > 0x7FFFFull)
                atomicOr(&bacc.status, PCC_ST_ID_RANGE);
        }
    }
}

// Scan: for each cell, the sums n_p, n_t, n_pt of Sec. III.A, the
// coefficient, and the accept uniforms of every pair against the
// per-material bounds.  Pairs at or above the bounds are rejected here,
// exactly (U >= bound >= x >= 1 - exp(-x)), without reading the particle
// records; the others are queued.  The list holds the size classes from the
// largest (class k: N_pair in [2^(k-1), 2^k)); the largest cells take a
// whole warp, smaller ones a group of 16, 8, 4 or 2 lanes (ScanClass), so
// that the per-cell work (metadata, sums, coefficient, record) is shared by
// up to 16 cells per warp instruction.  Contains no calls, so its loop state
// stays in registers.
template <int GROUP, int MINB>
__global__ void __launch_bounds__(kBatchedThreads, MINB) scan_kernel(const __grid_constant__ StepArgs a, CellList L,
                                                                     Queue Q, IonCache IC)
{
    __shared__ int scratch[kBatchedThreads / 32][64];
    __shared__ uint2 buf[kBatchedThreads / 32][kWarpBuf];
    __shared__ BlockAcc bacc;
    block_acc_init(bacc);
    __syncthreads();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* tab = scratch[wid];
    uint2* wb = buf[wid];
    // segment ends: whole warps, then 16-, 8-, 4- and 2-lane groups
    int e32 = 0, e16 = 0, e8 = 0, e4 = 0, e2 = 0;
    for (int k = kClasses - 1; k >= 0; --k) {
        const int h = L.hist[k];
        if (k >= L.thr[0]) e32 += h;
        else if (k >= L.thr[1]) e16 += h;
        else if (k >= L.thr[2]) e8 += h;
        else if (k >= L.thr[3]) e4 += h;
        else e2 += h;
    }
    e16 += e32;
    e8 += e16;
    e4 += e8;
    e2 += e4;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + wid;
    ScanWarp sw{0, 0ull, 0ull};
    // the round-robin continues across segments: a segment's first tuple
    // goes to the warp after the one that took the previous segment's last
    int d = 0;
    scan_segment<GROUP, 32>(a, L, Q, IC, 0, e32, gw, nwarps, tab, wb, sw, bacc);
    d = (d + e32) % nwarps;
    scan_segment<GROUP, 16>(a, L, Q, IC, e32, e16, (gw - d + nwarps) % nwarps, nwarps, tab, wb, sw,
                             bacc);
    d = (d + (e16 - e32 + 1) / 2) % nwarps;
    scan_segment<GROUP, 8>(a, L, Q, IC, e16, e8, (gw - d + nwarps) % nwarps, nwarps, tab, wb, sw,
                             bacc);
    d = (d + (e8 - e16 + 3) / 4) % nwarps;
    scan_segment<GROUP, 4>(a, L, Q, IC, e8, e4, (gw - d + nwarps) % nwarps, nwarps, tab, wb, sw,
                             bacc);
    d = (d + (e4 - e8 + 7) / 8) % nwarps;
    scan_segment<GROUP, 2>(a, L, Q, IC, e4, e2, (gw - d + nwarps) % nwarps, nwarps, tab, wb, sw,
                             bacc);
    if (sw.nb > 0) flush_staged(Q, wb, sw.nb, bacc, lane);   // final flush
    if (sw.npairs) atomicAdd(&bacc.pairs[GROUP], sw.npairs);
    if (sw.ncands) atomicAdd(&bacc.candidates[GROUP], sw.ncands);
    __syncthreads();
    block_acc_flush(bacc, a.st);
}

// Fold the per-thread counters of a batched kernel into the block, then the context.
__device__ __forceinline__ void fold_acc(Acc& acc, BlockAcc& bacc, DevStats* st)
{
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < 5; ++i) {
        const unsigned av = warp_sum(acc.accepted[i]), cv = warp_sum(acc.created[i]);
        if (lane == 0) {
            if (av) atomicAdd(&bacc.accepted[i], (unsigned long long)av);
            if (cv) atomicAdd(&bacc.created[i], (unsigned long long)cv);
        }
    }
    const double dE = warp_sum(acc.dE);
    const unsigned stt = __reduce_or_sync(0xffffffffu, acc.status);
    if (lane == 0) {
        if (dE != 0.0) atomicAdd(&bacc.dE, dE);
        if (stt) atomicOr(&bacc.status, stt);
    }
    __syncthreads();
    block_acc_flush(bacc, st);
}

// Candidates of cells with N_p >= N_t (one pair per projectile), one thread
// each: pairing, ion frame, cross section, acceptance, events.  Event
// contributions to the cell ledger are gathered per cell (float atomics) and
// the cell is listed for the finalize kernel.
template <int GROUP>
__global__ void __launch_bounds__(kBatchedThreads, 4) flat_cand_kernel(const __grid_constant__ StepArgs a, Queue Q,
                                                                       int stage_bytes)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ BlockAcc bacc;
    __shared__ __align__(8) unsigned long long bar;
    block_acc_init(bacc);
    unsigned st0 = 0;
    const float* ls = stage_table(GROUP == kGroupPh ? a.f_bh_lnsig : a.f_brems_lnsig, stage_bytes, dyn, &bar, a.wait_polls, st0);
    if (st0 && threadIdx.x == 0) bacc.status |= st0;
    __syncthreads();
    const Tab<float> tb = batched_tab<GROUP>(a, ls);
    const SpeciesView& P = GROUP == kGroupEm ? a.em : (GROUP == kGroupEp ? a.ep : a.ph);
    const uint32_t step32 = (uint32_t)a.step;
    const int total = min(*Q.flat_count, (int)Q.cap_flat);
    Acc acc;
    acc.zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint2 e = Q.flat[i];
        const int cell = (int)e.x;
        const uint32_t s = e.y;
        if (cell < 0 || cell >= a.n_cells) continue;
        const CellRec cm = load_rec(Q, cell);
        const uint32_t Np = cm.Np, Nt = cm.Nt;
        const float coef = cm.coef;
        const Philox4 kp = draw_k(0, (uint32_t)cell, step32, stream_tag(GROUP, kPerm, 0), a.keys);
        PermKeys rk;
        rk.k[0] = kp.v[0]; rk.k[1] = kp.v[1]; rk.k[2] = kp.v[2]; rk.k[3] = kp.v[3];
        const uint32_t j = Np <= 32 ? perm_pos_small(s, Np, rk) : perm_pos_large(s, Np, rk);
        const int ts = cm.t0 + (int)fast_mod(j, Nt, 1.0f / (float)Nt);
        using AS = AcceptSlots<GROUP>;
        const uint32_t dg = AS::digit(s);
        const Philox4 ph = draw_k(AS::ctr(s), (uint32_t)cell, step32, stream_tag(GROUP, kAccept, 0), a.keys);
        const uint32_t r1 = accept_digit(ph, dg), r2 = GROUP == kGroupPh ? 0u : accept_digit(ph, dg + 1);
        const AcceptSrc src{AS::ext(s), (uint32_t)cell, stream_tag(GROUP, kAcceptExt, 0)};
        const int sl = cm.p0 + (int)s;
        float rad = 0.f, wcre = 0.f;
        bool event = false;
        if (GROUP == kGroupPh) {
            event = bh_candidate(a, tb, cell, cm.mat, coef, sl, ts, j, r1, src, acc, wcre);
        } else {
            float u[3] = {P.ux[sl], P.uy[sl], P.uz[sl]};
            const float xp = P.x ? P.x[sl] : 0.f;
            ei_pair<float>(&a, tb, GROUP, cell, cm.mat, a.f_Z[cm.mat], coef, u, P.w + sl, xp, ts, j, r1, r2, src, acc,
                           rad, wcre, event);
            if (event) {
                P.ux[sl] = u[0]; P.uy[sl] = u[1]; P.uz[sl] = u[2];
            }
        }
        if (event) {
            if (rad != 0.f) atomicAdd(&Q.evacc[cell].x, rad);
            if (wcre != 0.f) atomicAdd(&Q.evacc[cell].y, wcre);
            flag_cell(Q, cell);
        }
    }
    fold_acc(acc, bacc, a.st);
}

// Candidates of cells with N_p < N_t, one warp per cell, in queue order on
// one lane (a projectile's pairs in increasing pair index; a photon absorbed
// on an earlier pair skips its later ones).
template <int GROUP>
__global__ void __launch_bounds__(kBatchedThreads, 2) caseb_cand_kernel(const __grid_constant__ StepArgs a, Queue Q,
                                                                        int stage_bytes)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ int scratch[kBatchedThreads / 32][64];
    __shared__ BlockAcc bacc;
    __shared__ __align__(8) unsigned long long bar;
    block_acc_init(bacc);
    unsigned st0 = 0;
    const float* ls = stage_table(GROUP == kGroupPh ? a.f_bh_lnsig : a.f_brems_lnsig, stage_bytes, dyn, &bar, a.wait_polls, st0);
    if (st0 && threadIdx.x == 0) bacc.status |= st0;
    __syncthreads();
    const Tab<float> tb = batched_tab<GROUP>(a, ls);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* tab = scratch[wid];
    const int n = *Q.caseb_count;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const SpeciesView& P = GROUP == kGroupEm ? a.em : (GROUP == kGroupEp ? a.ep : a.ph);
    const uint32_t step32 = (uint32_t)a.step;
    Acc acc;
    acc.zero();
    for (int kk = blockIdx.x * (blockDim.x >> 5) + wid; kk < n; kk += nwarps) {
        const int cell = Q.caseb[kk];
        if (cell < 0 || cell >= a.n_cells) continue;
        const CellRec cm = load_rec(Q, cell);
        const uint32_t Np = cm.Np, Nt = cm.Nt;
        const int cnt = Q.cand[cell];
        const float coef = cm.coef;
        const Philox4 kp = draw_k(0, (uint32_t)cell, step32, stream_tag(GROUP, kPerm, 0), a.keys);
        PermKeys rk;
        rk.k[0] = kp.v[0]; rk.k[1] = kp.v[1]; rk.k[2] = kp.v[2]; rk.k[3] = kp.v[3];
        if (Nt <= 32) {   // P table of the targets
            __syncwarp();
            if (lane < (int)Nt) tab[perm_pos_small(lane, Nt, rk)] = lane;
            __syncwarp();
        }
        if (lane == 0) {
            float rad = 0.f, wcre = 0.f;
            bool any = false;
            for (int k = 0; k < cnt; ++k) {
                const uint32_t j = Q.qb[cm.t0 + k];
                const uint32_t s = j % Np, mp = j / Np;
                using AS = AcceptSlots<GROUP>;
                const uint32_t dg = AS::digit(s);
                const Philox4 ph = draw_k(AS::ctr(s), (uint32_t)cell, step32, stream_tag(GROUP, kAccept, mp), a.keys);
                const uint32_t r1 = accept_digit(ph, dg), r2 = GROUP == kGroupPh ? 0u : accept_digit(ph, dg + 1);
                const AcceptSrc src{AS::ext(s), (uint32_t)cell, stream_tag(GROUP, kAcceptExt, mp)};
                const uint32_t t = Nt <= 32 ? (uint32_t)tab[j] : perm_elem_large(j, Nt, rk);
                const int ts = cm.t0 + (int)t, sl = cm.p0 + (int)s;
                bool event = false;
                if (GROUP == kGroupPh) {
                    if (P.w[sl] == 0.f) continue;   // absorbed earlier in this step
                    event = bh_candidate(a, tb, cell, cm.mat, coef, sl, ts, j, r1, src, acc, wcre);
                } else {
                    float u[3] = {P.ux[sl], P.uy[sl], P.uz[sl]};
                    const float xp = P.x ? P.x[sl] : 0.f;
                    ei_pair<float>(&a, tb, GROUP, cell, cm.mat, a.f_Z[cm.mat], coef, u, P.w + sl, xp, ts, j, r1, r2,
                                   src, acc, rad, wcre, event);
                    if (event) {
                        P.ux[sl] = u[0]; P.uy[sl] = u[1]; P.uz[sl] = u[2];
                    }
                }
                any |= event;
            }
            if (any) {
                if (rad != 0.f) atomicAdd(&Q.evacc[cell].x, rad);
                if (wcre != 0.f) atomicAdd(&Q.evacc[cell].y, wcre);
                flag_cell(Q, cell);
            }
        }
        __syncwarp();
    }
    fold_acc(acc, bacc, a.st);
}

// Stable removal of the absorbed photons (weight 0) from the first Np slots
// of a cell region, keeping the order of the rest (including the Np..n_all
// secondaries appended in this step), one warp.  The records before the
// first removed one are not touched; from there each batch of 4 x 32
// records is read into registers before any of it is written, and
// destinations never pass sources.
__device__ void compact_region_warp(const SpeciesView& P, int cell)
{
    constexpr unsigned kFull = 0xffffffffu;
    constexpr int kU = 4;   // 32-record chunks loaded before any of them is stored
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int p0 = P.start[cell], Np = P.count[cell];
    const int n_all = Np + P.added[cell];
    const bool has_x = P.x != nullptr;
    // the records before the first removed one stay where they are
    int c0 = 0;
    for (; c0 < Np; c0 += 32 * kU) {
        bool hole = false;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = c0 + 32 * u + lane;
            if (i < Np) hole |= P.w[p0 + i] == 0.f;
        }
        if (__any_sync(kFull, hole)) break;
    }
    if (c0 >= Np) return;   // nothing removed
    int wr = c0;            // warp-uniform write position
    for (int b = c0; b < n_all; b += 32 * kU) {
        float ux[kU], uy[kU], uz[kU], w[kU], x[kU];
        uint64_t pid[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = b + 32 * u + lane;
            ux[u] = uy[u] = uz[u] = w[u] = x[u] = 0.f;
            pid[u] = 0;
            if (i < n_all) {
                const int src = p0 + i;
                ux[u] = P.ux[src]; uy[u] = P.uy[src]; uz[u] = P.uz[src]; w[u] = P.w[src];
                if (has_x) x[u] = P.x[src];
                pid[u] = P.pid[src];
            }
        }
        __syncwarp();   // every record of the batch is read before any is overwritten
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = b + 32 * u + lane;
            const bool keep = i < n_all && !(i < Np && w[u] == 0.f);
            const unsigned m = __ballot_sync(kFull, keep);
            if (keep) {
                const int dst = p0 + wr + __popc(m & below);
                if (dst != p0 + i) {
                    P.ux[dst] = ux[u]; P.uy[dst] = uy[u]; P.uz[dst] = uz[u]; P.w[dst] = w[u];
                    if (has_x) P.x[dst] = x[u];
                    P.pid[dst] = pid[u];
                }
            }
            wr += __popc(m);
        }
        __syncwarp();
    }
    if (lane == 0) P.count[cell] = wr - P.added[cell];
}

// Cells with an event in this call: the Kahan update of the cell ledger
// from the gathered contributions, and (photons) the compaction that removes
// absorbed photons.  Photon cells take a warp each (the compaction is
// warp-wide); the other groups' cells take one thread each.
__device__ __forceinline__ void finalize_ledger(const StepArgs& a, const Queue& Q, int cell)
{
    const float2 ev = Q.evacc[cell];
    if (a.ledger) {
        float4* Lg = reinterpret_cast<float4*>(a.ledger) + cell;
        float4 v = *Lg;
        Kahan ka{v.x, v.y}, kb{v.z, v.w};
        ka.add(ev.x);
        kb.add(ev.y);
        *Lg = make_float4(ka.s, ka.c, kb.s, kb.c);
    }
    Q.evacc[cell] = make_float2(0.f, 0.f);
}

template <int GROUP>
__global__ void finalize_kernel(const __grid_constant__ StepArgs a, Queue Q)
{
    const int n = *Q.flagged_count;
    if (GROUP != kGroupPh) {
        for (int kk = blockIdx.x * blockDim.x + threadIdx.x; kk < n; kk += gridDim.x * blockDim.x) {
            const int cell = Q.flagged[kk];
            if (cell < 0 || cell >= a.n_cells) continue;
            finalize_ledger(a, Q, cell);
            Q.flag[cell] = 0;
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int kk = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); kk < n; kk += nwarps) {
        const int cell = Q.flagged[kk];
        if (cell < 0 || cell >= a.n_cells) continue;
        if (lane == 0) finalize_ledger(a, Q, cell);
        compact_region_warp(a.ph, cell);
        __syncwarp();
        if (lane == 0) Q.flag[cell] = 0;
    }
}

// Pairing diagnostic: one warp per cell.
__global__ void pairing_kernel(StepArgs a, SpeciesView P, SpeciesView I, int group, int* out_j, int* out_t)
{
    __shared__ int scratch[8][64];
    const int wid = threadIdx.x >> 5;
    WarpGroup grp{scratch[wid]};
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int cell = blockIdx.x * (blockDim.x >> 5) + wid; cell < a.n_cells; cell += nwarps) {
        const uint32_t Np = P.count[cell], Nt = I.count[cell];
        if (Np == 0 || Nt == 0) continue;
        const Pairing pr = make_pairing(grp, Np, Nt, cell, group, a);
        for (int s = grp.rank(); s < (int)Np; s += 32) {
            uint32_t j, t;
            if (pr.caseA) {
                j = pr.pair_of_slot(s);
                t = j % Nt;
            } else {
                j = s;
                t = pr.target_of_pair(j);
            }
            out_j[P.start[cell] + s] = (int)j;
            out_t[P.start[cell] + s] = (int)t;
        }
    }
}

}  // namespace pcc

using namespace pcc;

static bool species_ok(const pcc_species* s)
{
    return s && s->ux && s->uy && s->uz && s->w && s->pid && s->cell_start && s->cell_count && s->cell_added;
}

static StepArgs make_args(pcc_ctx* ctx, const pcc_cells* cells, pcc_species* em, pcc_species* ep, pcc_species* ph,
                          const pcc_species* ion, double dt, uint64_t seed, uint64_t step, unsigned mask,
                          float* ledger)
{
    StepArgs a;
    a.n_cells = cells->n_cells;
    a.mat_of_cell = cells->material_of_cell;
    a.em = view_of(*em);
    a.ep = view_of(*ep);
    a.ph = view_of(*ph);
    a.ion = view_of(*ion);
    a.dt = dt;
    a.seed = seed;
    a.step = step;
    a.mask = mask;
    a.ledger = ledger;
    a.g = make_geom(ctx->spec);
    a.n_mat = ctx->n_mat;
    a.brems_sigma = ctx->brems_sigma; a.brems_cdf = ctx->brems_cdf;
    a.bh_sigma = ctx->bh_sigma; a.bh_cdf = ctx->bh_cdf;
    a.tri_gp = ctx->tri_gp_cdf; a.tri_split = ctx->tri_split_cdf; a.screen = ctx->screen;
    a.f_brems_lnsig = ctx->f_brems_lnsig; a.f_brems_cdf = ctx->f_brems_cdf;
    a.f_bh_lnsig = ctx->f_bh_lnsig; a.f_bh_cdf = ctx->f_bh_cdf;
    a.f_tri_gp = ctx->f_tri_gp_cdf; a.f_tri_split = ctx->f_tri_split_cdf; a.f_Z = ctx->f_Z;
    a.f_bound = ctx->f_bound;
    a.keys = philox_keys(seed);
    a.f_cdt = (float)(kC * dt);
    a.wait_polls = ctx->wait_polls;
    a.st = ctx->stats;
    return a;
}

// Blocks of a persistent kernel: resident blocks per SM (or the tuned count) x SMs.
static int persistent_grid(pcc_ctx* ctx, const void* fn, int smem, int want_per_sm)
{
    int per_sm = 0;
    for (const auto& o : ctx->occ)
        if (o.fn == fn && o.smem == smem) per_sm = o.per_sm;
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchedThreads, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        ctx->occ.push_back({fn, smem, per_sm});
    }
    if (want_per_sm > 0 && want_per_sm < per_sm) per_sm = want_per_sm;
    return per_sm * std::max(ctx->num_sms, 1);
}

// Per-call cell state of the batched path, one int buffer of n = n_cells:
//   [0, 3n) cell lists of the three groups   [3n) candidates (N_p < N_t cells)
//   [4n) unused                              [5n) cells with N_p < N_t candidates
//   [6n) cells with events                   [7n) listed flags
//   [8n, 10n) ledger contributions (float2)  [R, R + 8n) cell records (int4 pairs,
//   R = 10n rounded up to 4 ints)           [R + 8n) class histograms and cursors,
//   then three counters (flat queue, N_p < N_t cells, cells with events), then
//   the per-block class counts of the three groups.
// Flags and contributions start at zero and are cleared by the finalize kernel.
static size_t rec_off(size_t n) { return (10 * n + 3) & ~(size_t)3; }
static size_t hist_off(size_t n) { return rec_off(n) + 8 * n; }
// then, 16-byte aligned, the per-cell ion summaries (float4, see IonCache)
static size_t ionsum_off(size_t n)
{
    const size_t nblk = (n + kClassBlock - 1) / kClassBlock;
    return (hist_off(n) + 6 * kClasses + 8 + 3 * kClasses * nblk + 3) & ~(size_t)3;
}

static int ensure_lists(pcc_ctx* ctx, int n_cells)
{
    if (ctx->lists && ctx->lists_cells >= n_cells) return PCC_OK;
    if (ctx->lists) cudaFree(ctx->lists);
    ctx->lists = nullptr;
    ctx->lists_cells = 0;
    const size_t bytes = (ionsum_off(n_cells) + 4 * (size_t)n_cells) * sizeof(int);
    cudaError_t e = cudaMalloc(&ctx->lists, bytes);
    if (e == cudaSuccess) e = cudaMemset(ctx->lists, 0, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "pcc_collide: cell lists");
    ctx->lists_cells = n_cells;
    return PCC_OK;
}

static int ensure_queue(pcc_ctx* ctx, size_t cap_a, size_t cap_b)
{
    if (cap_a > ctx->queue_a_cap) {
        if (ctx->queue_a) cudaFree(ctx->queue_a);
        ctx->queue_a = nullptr;
        ctx->queue_a_cap = 0;
        cudaError_t e = cudaMalloc(&ctx->queue_a, cap_a * sizeof(uint2));
        if (e != cudaSuccess) return cuda_fail(e, "pcc_collide: candidate queue");
        ctx->queue_a_cap = cap_a;
    }
    if (cap_b > ctx->queue_b_cap) {
        if (ctx->queue_b) cudaFree(ctx->queue_b);
        ctx->queue_b = nullptr;
        ctx->queue_b_cap = 0;
        cudaError_t e = cudaMalloc(&ctx->queue_b, cap_b * sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_fail(e, "pcc_collide: candidate queue");
        ctx->queue_b_cap = cap_b;
    }
    return PCC_OK;
}

static CellList list_of(pcc_ctx* ctx, int group)
{
    const size_t n = ctx->lists_cells;
    CellList L;
    L.list = ctx->lists + (size_t)group * n;
    L.hist = ctx->lists + hist_off(n) + (size_t)(2 * group) * kClasses;
    L.cursor = L.hist + kClasses;
    L.nblk = (int)((n + kClassBlock - 1) / kClassBlock);
    L.bh = ctx->lists + hist_off(n) + 6 * kClasses + 8 + (size_t)group * kClasses * L.nblk;
    for (int i = 0; i < 4; ++i) L.thr[i] = ctx->scan_thr[group][i];
    return L;
}

static int* counters_of(pcc_ctx* ctx) { return ctx->lists + hist_off(ctx->lists_cells) + 6 * kClasses; }

// counters: [0..2] cleared per group; [4] the call serial (never cleared)
static IonCache ion_cache_of(pcc_ctx* ctx)
{
    IonCache C;
    C.sum = reinterpret_cast<float4*>(ctx->lists + ionsum_off(ctx->lists_cells));
    C.serial = reinterpret_cast<const unsigned*>(counters_of(ctx) + 4);
    return C;
}

static Queue queue_of(pcc_ctx* ctx)
{
    const size_t n = ctx->lists_cells;
    int* c = counters_of(ctx);
    Queue Q;
    Q.flat = (uint2*)ctx->queue_a;
    Q.cap_flat = (uint32_t)std::min<size_t>(ctx->queue_a_cap, 0xFFFFFFFFu);
    Q.flat_count = c;
    Q.qb = (uint32_t*)ctx->queue_b;
    Q.cand = ctx->lists + 3 * n;
    Q.caseb = ctx->lists + 5 * n;
    Q.caseb_count = c + 1;
    Q.flagged = ctx->lists + 6 * n;
    Q.flagged_count = c + 2;
    Q.flag = ctx->lists + 7 * n;
    Q.evacc = reinterpret_cast<float2*>(ctx->lists + 8 * n);
    Q.rec = reinterpret_cast<int4*>(ctx->lists + rec_off(n));
    return Q;
}

template <int GROUP, int MINB>
static void launch_scan(pcc_ctx* ctx, const StepArgs& a, const CellList& L, const Queue& Q, cudaStream_t st)
{
    const int g = persistent_grid(ctx, (const void*)scan_kernel<GROUP, MINB>, 0, ctx->blocks_per_sm);
    scan_kernel<GROUP, MINB><<<g, kBatchedThreads, 0, st>>>(a, L, Q, ion_cache_of(ctx));
}

// Per group, after the class sort of all groups: counters, scan (register
// budget chosen by the schedule: 2 to 6 resident blocks per SM),
// candidates, finalize.
template <int GROUP>
static cudaError_t launch_batched(pcc_ctx* ctx, const StepArgs& a, int stage, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counters_of(ctx), 0, 3 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    const CellList L = list_of(ctx, GROUP);
    const Queue Q = queue_of(ctx);
    switch (ctx->minb) {
    case 2: launch_scan<GROUP, 2>(ctx, a, L, Q, st); break;
    case 3: launch_scan<GROUP, 3>(ctx, a, L, Q, st); break;
    case 5: launch_scan<GROUP, 5>(ctx, a, L, Q, st); break;
    case 6: launch_scan<GROUP, 6>(ctx, a, L, Q, st); break;
    default: launch_scan<GROUP, 4>(ctx, a, L, Q, st); break;
    }
    const int gf = persistent_grid(ctx, (const void*)flat_cand_kernel<GROUP>, stage, 0);
    flat_cand_kernel<GROUP><<<gf, kBatchedThreads, stage, st>>>(a, Q, stage);
    const int gb = persistent_grid(ctx, (const void*)caseb_cand_kernel<GROUP>, stage, 0);
    caseb_cand_kernel<GROUP><<<gb, kBatchedThreads, stage, st>>>(a, Q, stage);
    finalize_kernel<GROUP><<<2 * std::max(ctx->num_sms, 1), 256, 0, st>>>(a, Q);
    note_launches(4);
    return cudaSuccess;
}

// The size-class lists of the groups that run, in three launches.
static void launch_class_sort(pcc_ctx* ctx, const StepArgs& a, unsigned run, cudaStream_t st)
{
    ClassSort S;
    for (int g = 0; g < 3; ++g) S.L[g] = list_of(ctx, g);
    S.cnt_p[0] = a.em.count;
    S.cnt_p[1] = a.ep.count;
    S.cnt_p[2] = a.ph.count;
    S.cnt_t = a.ion.count;
    S.n_cells = a.n_cells;
    S.run = run;
    S.serial = reinterpret_cast<unsigned*>(counters_of(ctx) + 4);
    const int nblk = S.L[0].nblk;
    class_hist_kernel<<<nblk, kClassBlock, 0, st>>>(S);
    const size_t off_smem = (size_t)kClasses * nblk * sizeof(int);
    if (off_smem <= (size_t)kClassSmemMax) class_offsets_kernel<true><<<3, 1024, off_smem, st>>>(S);
    else class_offsets_kernel<false><<<3, 1024, 0, st>>>(S);
    class_scatter_kernel<<<nblk, kClassBlock, 0, st>>>(S);
    note_launches(3);
}

static int table_stage_bytes(const pcc_ctx* ctx)
{
    const size_t tab_bytes = (size_t)ctx->n_mat * ctx->spec.n_rows * sizeof(float);
    return (tab_bytes % 16 == 0 && tab_bytes <= 48 * 1024) ? (int)tab_bytes : 0;
}

template <int GROUP>
static void warm_occupancy(pcc_ctx* ctx, int stage)
{
    switch (ctx->minb) {
    case 2: persistent_grid(ctx, (const void*)scan_kernel<GROUP, 2>, 0, 0); break;
    case 3: persistent_grid(ctx, (const void*)scan_kernel<GROUP, 3>, 0, 0); break;
    case 5: persistent_grid(ctx, (const void*)scan_kernel<GROUP, 5>, 0, 0); break;
    case 6: persistent_grid(ctx, (const void*)scan_kernel<GROUP, 6>, 0, 0); break;
    default: persistent_grid(ctx, (const void*)scan_kernel<GROUP, 4>, 0, 0); break;
    }
    persistent_grid(ctx, (const void*)flat_cand_kernel<GROUP>, stage, 0);
    persistent_grid(ctx, (const void*)caseb_cand_kernel<GROUP>, stage, 0);
}

int collide_prepare(pcc_ctx* ctx, const pcc_cells* cells, const pcc_species* em, const pcc_species* ep,
                    const pcc_species* ph, const pcc_species* ion, unsigned mask, int precision)
{
    if (!ctx || !cells || !em || !ep || !ph || !ion || cells->n_cells < 1) {
        set_error("pcc_collide: invalid argument");
        return PCC_E_INVALID;
    }
    if (!ctx->class_smem_ready) {   // per device, before any capture
        if (cudaFuncSetAttribute(class_offsets_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kClassSmemMax) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "pcc_collide: class sort shared memory");
        ctx->class_smem_ready = true;
    }
    if (precision != PCC_FP32_BATCHED) return PCC_OK;
    const unsigned groups = (mask & 0x700u) ? (mask & 0x700u) : 0x700u;
    const bool ei = (mask & (PCC_BREMS | PCC_TRIDENT)) != 0, bh = (mask & PCC_BH) != 0;
    const bool run_em = ei && (groups & PCC_GROUP_EM), run_ep = ei && (groups & PCC_GROUP_EP);
    const bool run_ph = bh && (groups & PCC_GROUP_PH);
    int rc = ensure_lists(ctx, cells->n_cells);
    if (rc) return rc;
    size_t cap_a = 0;
    if (run_em) cap_a = std::max(cap_a, (size_t)em->capacity);
    if (run_ep) cap_a = std::max(cap_a, (size_t)ep->capacity);
    if (run_ph) cap_a = std::max(cap_a, (size_t)ph->capacity);
    rc = ensure_queue(ctx, std::max<size_t>(cap_a, 1), std::max<size_t>((size_t)ion->capacity, 1));
    if (rc) return rc;
    const int stage = table_stage_bytes(ctx);
    if (run_em) warm_occupancy<kGroupEm>(ctx, stage);
    if (run_ep) warm_occupancy<kGroupEp>(ctx, stage);
    if (run_ph) warm_occupancy<kGroupPh>(ctx, stage);
    return PCC_OK;
}

extern "C" int pcc_set_wait_limit(pcc_ctx* ctx, int polls)
{
    if (!ctx || polls < 0) {
        set_error("pcc_set_wait_limit: invalid argument");
        return PCC_E_INVALID;
    }
    ctx->wait_polls = polls;
    return PCC_OK;
}

extern "C" int pcc_set_scan_classes(pcc_ctx* ctx, int group, const int* thresholds)
{
    if (!ctx || group < 0 || group > 2 || !thresholds) {
        set_error("pcc_set_scan_classes: invalid argument");
        return PCC_E_INVALID;
    }
    const int* t = thresholds;
    if (!(0 <= t[3] && t[3] <= t[2] && t[2] <= t[1] && t[1] <= t[0] && t[0] <= kClasses)) {
        set_error("pcc_set_scan_classes: thresholds must satisfy 0 <= g4 <= g8 <= g16 <= warp <= " +
                  std::to_string(kClasses));
        return PCC_E_INVALID;
    }
    for (int i = 0; i < 4; ++i) ctx->scan_thr[group][i] = t[i];
    return PCC_OK;
}

extern "C" int pcc_get_scan_classes(const pcc_ctx* ctx, int group, int* thresholds)
{
    if (!ctx || group < 0 || group > 2 || !thresholds) {
        set_error("pcc_get_scan_classes: invalid argument");
        return PCC_E_INVALID;
    }
    for (int i = 0; i < 4; ++i) thresholds[i] = ctx->scan_thr[group][i];
    return PCC_OK;
}

extern "C" int pcc_set_schedule(pcc_ctx* ctx, int min_blocks_per_sm, int blocks_per_sm)
{
    if (!ctx || min_blocks_per_sm < 2 || min_blocks_per_sm > 6 || blocks_per_sm < 0) {
        set_error("pcc_set_schedule: invalid schedule");
        return PCC_E_INVALID;
    }
    ctx->minb = min_blocks_per_sm;
    ctx->blocks_per_sm = blocks_per_sm;
    return PCC_OK;
}

int collide_groups(pcc_ctx* ctx, const pcc_cells* cells, pcc_species* em, pcc_species* ep, pcc_species* ph,
                   const pcc_species* ion, double dt, uint64_t seed, uint64_t step, unsigned mask, int precision,
                   float* ledger, cudaStream_t st, int (*after_group)(void* user, int group), void* user)
{
    if (!ctx || !cells || !cells->material_of_cell || cells->n_cells < 1) {
        set_error("pcc_collide: invalid cells");
        return PCC_E_INVALID;
    }
    if (!species_ok(em) || !species_ok(ep) || !species_ok(ph) || !species_ok(ion)) {
        set_error("pcc_collide: every species needs ux, uy, uz, w, pid and the three cell arrays");
        return PCC_E_INVALID;
    }
    if ((em->x == nullptr) != (ep->x == nullptr) || (em->x == nullptr) != (ph->x == nullptr)) {
        set_error("pcc_collide: x must be given for all of e-, e+ and photons or for none");
        return PCC_E_INVALID;
    }
    if (!(dt > 0.0) || (mask & ~0x707u) || (precision != PCC_FP64_PLAIN && precision != PCC_FP32_BATCHED)) {
        set_error("pcc_collide: invalid dt, process mask or precision");
        return PCC_E_INVALID;
    }
    if (ctx->n_mat == 0) { set_error("pcc_collide: tables not built"); return PCC_E_NO_TABLES; }
    StepArgs a = make_args(ctx, cells, em, ep, ph, ion, dt, seed, step, mask, ledger);
    const unsigned groups = (mask & 0x700u) ? (mask & 0x700u) : 0x700u;
    const bool ei = (mask & (PCC_BREMS | PCC_TRIDENT)) != 0, bh = (mask & PCC_BH) != 0;
    const bool run_em = ei && (groups & PCC_GROUP_EM), run_ep = ei && (groups & PCC_GROUP_EP);
    const bool run_ph = bh && (groups & PCC_GROUP_PH);
    a.mask = mask & 7u;
    const bool run[3] = {run_em, run_ep, run_ph};
    int stage = 0;
    if (precision == PCC_FP32_BATCHED) {
        int rc = collide_prepare(ctx, cells, em, ep, ph, ion, mask, precision);
        if (rc) return rc;
        launch_class_sort(ctx, a, (run_em ? 1u : 0u) | (run_ep ? 2u : 0u) | (run_ph ? 4u : 0u), st);
        stage = table_stage_bytes(ctx);
    }
    for (int g = 0; g < 3; ++g) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "pcc_collide: launch");
        if (run[g]) {
            if (precision == PCC_FP64_PLAIN) {
                if (g == kGroupEm) collide_plain_kernel<kGroupEm><<<cells->n_cells, 128, 0, st>>>(a);
                else if (g == kGroupEp) collide_plain_kernel<kGroupEp><<<cells->n_cells, 128, 0, st>>>(a);
                else collide_plain_kernel<kGroupPh><<<cells->n_cells, 128, 0, st>>>(a);
                note_launches(1);
            } else {
                if (g == kGroupEm) e = launch_batched<kGroupEm>(ctx, a, stage, st);
                else if (g == kGroupEp) e = launch_batched<kGroupEp>(ctx, a, stage, st);
                else e = launch_batched<kGroupPh>(ctx, a, stage, st);
                if (e != cudaSuccess) return cuda_fail(e, "pcc_collide: batched launch");
            }
        }
        if (after_group) {
            const int rc = after_group(user, g);
            if (rc) return rc;
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_collide: launch");
}

extern "C" int pcc_collide(pcc_ctx* ctx, const pcc_cells* cells, pcc_species* em, pcc_species* ep, pcc_species* ph,
                           const pcc_species* ion, double dt, uint64_t seed, uint64_t step, unsigned mask,
                           int precision, float* ledger, void* stream)
{
    return collide_groups(ctx, cells, em, ep, ph, ion, dt, seed, step, mask, precision, ledger, (cudaStream_t)stream,
                          nullptr, nullptr);
}

extern "C" int pcc_pairing(pcc_ctx* ctx, int n_cells, const pcc_species* proj, const pcc_species* targ, int group,
                           uint64_t seed, uint64_t step, int* out_j, int* out_t, void* stream)
{
    if (!ctx || !species_ok(proj) || !species_ok(targ) || !out_j || !out_t || n_cells < 1 || group < 0 || group > 2) {
        set_error("pcc_pairing: invalid argument");
        return PCC_E_INVALID;
    }
    StepArgs a{};
    a.n_cells = n_cells;
    a.seed = seed;
    a.step = step;
    pairing_kernel<<<std::max(1, std::min((n_cells + 7) / 8, 65535)), 256, 0, (cudaStream_t)stream>>>(
        a, view_of(*proj), view_of(*targ), group, out_j, out_t);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_pairing");
}
