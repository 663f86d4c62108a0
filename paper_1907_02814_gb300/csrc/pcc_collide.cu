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
    DevStats* st;
};

// ---- per-thread accumulators ---------------------------------------------
struct Acc {
    unsigned long long pairs[3];
    unsigned accepted[5], created[5];
    double dE, dQ;
    unsigned status;
    __device__ void zero()
    {
        for (int i = 0; i < 3; ++i) pairs[i] = 0;
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
    const Real t = (log(r) - row_ln0<Real>(g)) * row_inv<Real>(g);
    if (t > (Real)(g.n_rows - 1)) {
        status |= PCC_ST_TABLE_RANGE;
        return exp(tb.ln_sigma(row_tab, g.n_rows - 1));
    }
    int j = (int)t;
    if (j > g.n_rows - 2) j = g.n_rows - 2;
    const Real f = t - (Real)j;
    return exp(((Real)1 - f) * tb.ln_sigma(row_tab, j) + f * tb.ln_sigma(row_tab, j + 1));
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
    Real n[3];          // direction in the ion frame
};

// E' = gi E - ui.p ; p' = p + ((ui.p)/(gi+1) - E) ui  (Sec. III.A transform)
template <typename Real>
__device__ __forceinline__ void to_ion_frame(Frame<Real>& f, const Real u[3])
{
    f.gl = sqrt((Real)1 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const Real d = f.ui[0] * u[0] + f.ui[1] * u[1] + f.ui[2] * u[2];
    const Real fac = d / (f.gi + (Real)1) - f.gl;
    const Real px = u[0] + fac * f.ui[0], py = u[1] + fac * f.ui[1], pz = u[2] + fac * f.ui[2];
    const Real p2 = px * px + py * py + pz * pz;
    f.pp = sqrt(p2);
    f.Tp = p2 / ((Real)1 + sqrt((Real)1 + p2));
    const Real inv = f.pp > (Real)0 ? (Real)1 / f.pp : (Real)0;
    f.n[0] = px * inv; f.n[1] = py * inv; f.n[2] = pz * inv;
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

// ---- one electron/positron - ion pair: Brems then Trident -------------------
template <typename Real>
__device__ void ei_pair(const StepArgs& a, const Tab<Real>& tb, int group, int cell, int mat, Real Zf, Real coef,
                        float u[3], float wp, float xpos, const SpeciesView& ion, int t_slot, uint32_t j, Real UB,
                        Real UT, Acc& acc, Kahan& rad, Kahan& wcre, bool& had)
{
    Frame<Real> f;
    f.ui[0] = ion.ux[t_slot]; f.ui[1] = ion.uy[t_slot]; f.ui[2] = ion.uz[t_slot];
    const float wt = ion.w[t_slot];
    f.gi = sqrt((Real)1 + f.ui[0] * f.ui[0] + f.ui[1] * f.ui[1] + f.ui[2] * f.ui[2]);
    Real uu[3] = {(Real)u[0], (Real)u[1], (Real)u[2]};
    to_ion_frame(f, uu);
    if (!isfinite(f.gl)) { acc.status |= PCC_ST_NONFINITE; return; }
    const SpeciesView& ph = a.ph;
    const bool has_x = a.em.x != nullptr;
    if (a.mask & PCC_BREMS) {
        const Real* row_tab = tb.bsig + (size_t)mat * a.g.n_rows;
        const Real sig = sigma_at<Real>(tb, row_tab, a.g, f.Tp, acc.status);
        if (sig > (Real)0) {
            const Real x = coef * sig * f.pp / (f.gl * f.gi);
            if (x > (Real)1) acc.status |= PCC_ST_PROB_LARGE;
            if (UB < x && UB < -expm1(-x)) {
                const int ch = group == kGroupEm ? kChBremsEm : kChBremsEp;
                acc.accepted[ch]++;
                const Philox4 ev = draw(j, cell, a.step, stream_tag(group, kEvtBrems, 0), a.seed);
                if (!(wt < wp) || u01<Real>(ev.v[0]) < (Real)wt / (Real)wp) {
                    acc.created[ch]++;
                    const Real* cdf = tb.bcdf + (size_t)mat * a.g.n_rows * a.g.n_cols;
                    const Real xk = sample_col<Real>(cdf, a.g, f.Tp, u01<Real>(ev.v[1]), u01<Real>(ev.v[2]), true,
                                                     a.g.ln_x_min);
                    const Real kp = xk * f.Tp;
                    Real ue[3], kg[3], Ee, Ek;
                    Ee = lepton_to_lab(f, f.Tp * ((Real)1 - xk), ue);
                    const Real pk[3] = {kp * f.n[0], kp * f.n[1], kp * f.n[2]};
                    from_ion_frame(f, kp, pk, Ek, kg);
                    const float nu[3] = {(float)ue[0], (float)ue[1], (float)ue[2]};
                    const float gk[3] = {(float)kg[0], (float)kg[1], (float)kg[2]};
                    if (append_particle(ph, cell, gk, wp, xpos, has_x, secondary_pid(a.step, ch, cell, j, 0),
                                        acc.status)) {
                        acc.dE += (double)wp * ((double)Ee + (double)Ek - (double)f.gl);
                        rad.add(wp * (float)Ek);
                        wcre.add(wp);
                        had = true;
                    }
                    u[0] = nu[0]; u[1] = nu[1]; u[2] = nu[2];
                    uu[0] = nu[0]; uu[1] = nu[1]; uu[2] = nu[2];
                    to_ion_frame(f, uu);
                }
            }
        }
    }
    if (a.mask & PCC_TRIDENT) {
        const Real g1 = (Real)1 + f.Tp;
        const Real sig = sigma_trident<Real>(Zf, g1);
        if (sig > (Real)0) {
            const Real x = coef * sig * f.pp / (f.gl * f.gi);
            if (x > (Real)1) acc.status |= PCC_ST_PROB_LARGE;
            if (UT < x && UT < -expm1(-x)) {
                const int ch = group == kGroupEm ? kChTriEm : kChTriEp;
                acc.accepted[ch]++;
                const Philox4 e1 = draw(j, cell, a.step, stream_tag(group, kEvtTri1, 0), a.seed);
                if (!(wt < wp) || u01<Real>(e1.v[0]) < (Real)wt / (Real)wp) {
                    acc.created[ch]++;
                    const Philox4 e2 = draw(j, cell, a.step, stream_tag(group, kEvtTri2, 0), a.seed);
                    const Real y = sample_col<Real>(tb.tgp, a.g, f.Tp - (Real)2, u01<Real>(e1.v[1]),
                                                    u01<Real>(e1.v[2]), true, a.g.ln_tri_min);
                    const Real gpair = (Real)2 + y * (f.Tp - (Real)2);
                    const Real y2 = sample_col<Real>(tb.tsp, a.g, gpair - (Real)2, u01<Real>(e1.v[3]),
                                                     u01<Real>(e2.v[0]), false, 0.0);
                    Real uf[3], up[3], um[3];
                    const Real Ef = lepton_to_lab(f, (f.Tp - (Real)2) * ((Real)1 - y), uf);
                    const Real Ep = lepton_to_lab(f, y2 * (gpair - (Real)2), up);
                    const Real Em = lepton_to_lab(f, (gpair - (Real)2) * ((Real)1 - y2), um);
                    const float fm[3] = {(float)um[0], (float)um[1], (float)um[2]};
                    const float fp[3] = {(float)up[0], (float)up[1], (float)up[2]};
                    const bool ok1 = append_particle(a.em, cell, fm, wp, xpos, has_x,
                                                     secondary_pid(a.step, ch, cell, j, 0), acc.status);
                    const bool ok2 = append_particle(a.ep, cell, fp, wp, xpos, has_x,
                                                     secondary_pid(a.step, ch, cell, j, 1), acc.status);
                    if (ok1 && ok2) {
                        acc.dE += (double)wp * ((double)Ef + (double)Ep + (double)Em - (double)f.gl);
                        wcre.add(2.f * wp);
                        had = true;
                    }
                    u[0] = (float)uf[0]; u[1] = (float)uf[1]; u[2] = (float)uf[2];
                }
            }
        }
    }
}

// ---- one cell of electron (or positron) - ion pairs ---------------------------
template <typename Real, class G>
__device__ void ei_cell(const G& grp, const StepArgs& a, const Tab<Real>& tb, int group, int cell, Acc& acc)
{
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
    Real sp = 0, st = 0;
    for (int s = grp.rank(); s < (int)Np; s += grp.size()) sp += (Real)P.w[p0 + s];
    for (int s = grp.rank(); s < (int)Nt; s += grp.size()) st += (Real)I.w[t0 + s];
    const Real n_p = grp.sum(sp), n_t = grp.sum(st);
    const Pairing pr = make_pairing(grp, Np, Nt, cell, group, a);
    Real spt = 0;
    for (int s = grp.rank(); s < (int)Np; s += grp.size()) {
        const float wp = P.w[p0 + s];
        if (pr.caseA) {
            const uint32_t j = pr.pair_of_slot(s);
            spt += (Real)fminf(wp, I.w[t0 + j % Nt]);
        } else {
            for (uint32_t j = s; j < Nt; j += Np) spt += (Real)fminf(wp, I.w[t0 + pr.target_of_pair(j)]);
        }
    }
    const Real n_pt = grp.sum(spt);
    const Real coef = (n_p / n_pt) * n_t * (Real)(kC * a.dt);
    const uint32_t Npair = Np > Nt ? Np : Nt;
    if (grp.rank() == 0) acc.pairs[group] += Npair;
    if (Npair > 65536u || (uint32_t)cell > 0xFFFFFFu || a.step > 0x7FFFFull) acc.status |= PCC_ST_ID_RANGE;
    const Real Zf = sizeof(Real) == 8 ? (Real)a.screen[(size_t)mat * kScreenFields + 7] : (Real)a.f_Z[mat];
    Kahan rad, wcre;
    bool had = false;
    const bool has_x = P.x != nullptr;
    for (uint32_t q = grp.rank(); 2 * q < Np; q += grp.size()) {
        const int nh = (2 * q + 1 < Np) ? 2 : 1;
        float u[2][3], w[2], xp[2];
        bool dirty[2] = {false, false};
        for (int h = 0; h < nh; ++h) {
            const int sl = p0 + 2 * q + h;
            u[h][0] = P.ux[sl]; u[h][1] = P.uy[sl]; u[h][2] = P.uz[sl];
            w[h] = P.w[sl];
            xp[h] = has_x ? P.x[sl] : 0.f;
        }
        uint32_t jfirst[2] = {0, 0};
        if (pr.caseA)
            for (int h = 0; h < nh; ++h) jfirst[h] = pr.pair_of_slot(2 * q + h);
        for (uint32_t m = 0;; ++m) {
            bool any = false;
            const Philox4 ac = draw(q, cell, a.step, stream_tag(group, kAccept, m), a.seed);
            for (int h = 0; h < nh; ++h) {
                const uint32_t s = 2 * q + h;
                uint32_t j, tau;
                if (pr.caseA) {
                    if (m > 0) continue;
                    j = jfirst[h];
                    tau = j % Nt;
                } else {
                    j = s + m * Np;
                    if (j >= Nt) continue;
                    tau = pr.target_of_pair(j);
                }
                any = true;
                const float before[3] = {u[h][0], u[h][1], u[h][2]};
                ei_pair<Real>(a, tb, group, cell, mat, Zf, coef, u[h], w[h], xp[h], I, t0 + (int)tau, j,
                              u01<Real>(ac.v[2 * h]), u01<Real>(ac.v[2 * h + 1]), acc, rad, wcre, had);
                dirty[h] |= (before[0] != u[h][0]) | (before[1] != u[h][1]) | (before[2] != u[h][2]);
            }
            if (!any || pr.caseA) break;
        }
        for (int h = 0; h < nh; ++h)
            if (dirty[h]) {
                const int sl = p0 + 2 * q + h;
                P.ux[sl] = u[h][0]; P.uy[sl] = u[h][1]; P.uz[sl] = u[h][2];
            }
    }
    if (a.ledger && grp.any(had)) {
        const float r = grp.sum(rad.s + (-rad.c)), wc = grp.sum(wcre.s + (-wcre.c));
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
__device__ void bh_cell(const G& grp, const StepArgs& a, const Tab<Real>& tb, int cell, Acc& acc)
{
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
    Real sp = 0, st = 0;
    for (int s = grp.rank(); s < (int)Np; s += grp.size()) sp += (Real)P.w[p0 + s];
    for (int s = grp.rank(); s < (int)Nt; s += grp.size()) st += (Real)I.w[t0 + s];
    const Real n_p = grp.sum(sp), n_t = grp.sum(st);
    const Pairing pr = make_pairing(grp, Np, Nt, cell, kGroupPh, a);
    Real spt = 0;
    for (int s = grp.rank(); s < (int)Np; s += grp.size()) {
        const float wp = P.w[p0 + s];
        if (pr.caseA) {
            spt += (Real)fminf(wp, I.w[t0 + pr.pair_of_slot(s) % Nt]);
        } else {
            for (uint32_t j = s; j < Nt; j += Np) spt += (Real)fminf(wp, I.w[t0 + pr.target_of_pair(j)]);
        }
    }
    const Real n_pt = grp.sum(spt);
    const Real coef = (n_p / n_pt) * n_t * (Real)(kC * a.dt);
    const uint32_t Npair = Np > Nt ? Np : Nt;
    if (grp.rank() == 0) acc.pairs[kGroupPh] += Npair;
    if (Npair > 65536u || (uint32_t)cell > 0xFFFFFFu || a.step > 0x7FFFFull) acc.status |= PCC_ST_ID_RANGE;
    Kahan wcre;
    bool absorbed_any = false;
    const bool has_x = P.x != nullptr;
    for (uint32_t q = grp.rank(); 2 * q < Np; q += grp.size()) {
        const int nh = (2 * q + 1 < Np) ? 2 : 1;
        bool dead[2] = {false, false};
        uint32_t jfirst[2] = {0, 0};
        if (pr.caseA)
            for (int h = 0; h < nh; ++h) jfirst[h] = pr.pair_of_slot(2 * q + h);
        for (uint32_t m = 0;; ++m) {
            bool any = false;
            const Philox4 ac = draw(q, cell, a.step, stream_tag(kGroupPh, kAccept, m), a.seed);
            for (int h = 0; h < nh; ++h) {
                const uint32_t s = 2 * q + h;
                uint32_t j, tau;
                if (pr.caseA) {
                    if (m > 0) continue;
                    j = jfirst[h];
                    tau = j % Nt;
                } else {
                    j = s + m * Np;
                    if (j >= Nt) continue;
                    tau = pr.target_of_pair(j);
                }
                any = true;
                if (dead[h]) continue;
                const int sl = p0 + (int)s, ts = t0 + (int)tau;
                const Real uk[3] = {(Real)P.ux[sl], (Real)P.uy[sl], (Real)P.uz[sl]};
                const float wp = P.w[sl], wt = I.w[ts];
                Frame<Real> f;
                f.ui[0] = I.ux[ts]; f.ui[1] = I.uy[ts]; f.ui[2] = I.uz[ts];
                f.gi = sqrt((Real)1 + f.ui[0] * f.ui[0] + f.ui[1] * f.ui[1] + f.ui[2] * f.ui[2]);
                const Real k = sqrt(uk[0] * uk[0] + uk[1] * uk[1] + uk[2] * uk[2]);
                const Real d = f.ui[0] * uk[0] + f.ui[1] * uk[1] + f.ui[2] * uk[2];
                const Real kp = f.gi * k - d;
                const Real fac = d / (f.gi + (Real)1) - k;
                const Real pv[3] = {uk[0] + fac * f.ui[0], uk[1] + fac * f.ui[1], uk[2] + fac * f.ui[2]};
                const Real pm = sqrt(pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]);
                if (!isfinite(k)) { acc.status |= PCC_ST_NONFINITE; continue; }
                const Real* row_tab = tb.hsig + (size_t)mat * a.g.n_rows;
                const Real sig = sigma_at<Real>(tb, row_tab, a.g, kp - (Real)2, acc.status);
                if (!(sig > (Real)0)) continue;
                const Real x = coef * sig * kp / (k * f.gi);
                if (x > (Real)1) acc.status |= PCC_ST_PROB_LARGE;
                const Real U = u01<Real>(ac.v[2 * h]);
                if (!(U < x && U < -expm1(-x))) continue;
                acc.accepted[kChBH]++;
                const Philox4 ev = draw(j, cell, a.step, stream_tag(kGroupPh, kEvtBH, 0), a.seed);
                if ((wt < wp) && !(u01<Real>(ev.v[0]) < (Real)wt / (Real)wp)) continue;
                acc.created[kChBH]++;
                const Real* cdf = tb.hcdf + (size_t)mat * a.g.n_rows * a.g.n_cols;
                const Real y = sample_col<Real>(cdf, a.g, kp - (Real)2, u01<Real>(ev.v[1]), u01<Real>(ev.v[2]), false,
                                                0.0);
                f.n[0] = pv[0] / pm; f.n[1] = pv[1] / pm; f.n[2] = pv[2] / pm;
                Real up[3], um[3];
                const Real Ep = lepton_to_lab(f, y * (kp - (Real)2), up);
                const Real Em = lepton_to_lab(f, (kp - (Real)2) * ((Real)1 - y), um);
                const float fm[3] = {(float)um[0], (float)um[1], (float)um[2]};
                const float fp[3] = {(float)up[0], (float)up[1], (float)up[2]};
                const float xpos = has_x ? P.x[sl] : 0.f;
                const bool ok1 = append_particle(a.em, cell, fm, wp, xpos, has_x,
                                                 secondary_pid(a.step, kChBH, cell, j, 0), acc.status);
                const bool ok2 = append_particle(a.ep, cell, fp, wp, xpos, has_x,
                                                 secondary_pid(a.step, kChBH, cell, j, 1), acc.status);
                if (ok1 && ok2) {
                    acc.dE += (double)wp * ((double)Ep + (double)Em - (double)k);
                    wcre.add(2.f * wp);
                }
                dead[h] = true;
                P.w[sl] = 0.f;   // removal marker, compacted below
                absorbed_any = true;
            }
            if (!any || pr.caseA) break;
        }
    }
    const bool anyd = grp.any(absorbed_any);
    if (anyd) {
        grp.sync();
        if (a.ledger) {
            const float wc = grp.sum(wcre.s + (-wcre.c));
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
    unsigned av[5], cv[5];
    double dE = acc.dE, dQ = acc.dQ;
    unsigned status = acc.status;
    for (int i = 0; i < 3; ++i) pv[i] = acc.pairs[i];
    for (int i = 0; i < 5; ++i) { av[i] = acc.accepted[i]; cv[i] = acc.created[i]; }
    if (lane_reduce) {
        for (int i = 0; i < 3; ++i) pv[i] = warp_sum(pv[i]);
        for (int i = 0; i < 5; ++i) { av[i] = warp_sum(av[i]); cv[i] = warp_sum(cv[i]); }
        dE = warp_sum(dE);
        dQ = warp_sum(dQ);
        status = __reduce_or_sync(0xffffffffu, status);
        if ((threadIdx.x & 31) != 0) return;
    }
    for (int i = 0; i < 3; ++i)
        if (pv[i]) atomicAdd(&st->pairs[i], pv[i]);
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
__global__ void __launch_bounds__(128) collide_plain_kernel(StepArgs a)
{
    __shared__ int scratch[64];
    __shared__ double red[4];
    CtaGroup grp{scratch, red};
    Tab<double> tb{a.brems_sigma, a.brems_cdf, a.bh_sigma, a.bh_cdf, a.tri_gp, a.tri_split};
    Acc acc;
    acc.zero();
    const int cell = blockIdx.x;
    if (GROUP == kGroupPh) bh_cell<double>(grp, a, tb, cell, acc);
    else ei_cell<double>(grp, a, tb, GROUP, cell, acc);
    flush_acc(acc, a.st, true);
}

// Batched FP32: persistent grid, one warp per cell.
constexpr int kBatchedThreads = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int GROUP>
__global__ void __launch_bounds__(kBatchedThreads) collide_batched_kernel(StepArgs a, int stage_bytes)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ int scratch[kBatchedThreads / 32][64];
    __shared__ __align__(8) unsigned long long bar;
    const int wid = threadIdx.x >> 5;
    WarpGroup grp{scratch[wid]};
    const float* lnsig_src = GROUP == kGroupPh ? a.f_bh_lnsig : a.f_brems_lnsig;
    const float* lnsig = lnsig_src;
    Acc acc;
    acc.zero();
    if (stage_bytes > 0) {
        // Bulk copy of the ln sigma rows of every material into shared memory.
        const uint32_t b = smem_u32(&bar);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(stage_bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(dyn)),
                "l"(lnsig_src), "r"(stage_bytes), "r"(b)
                : "memory");
        }
        uint32_t done = 0;
        for (int it = 0; it < (1 << 22) && !done; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(done)
                : "r"(b)
                : "memory");
        }
        if (done) lnsig = reinterpret_cast<const float*>(dyn);
        else acc.status |= PCC_ST_TIMEOUT;   // keep reading the global copy
        __syncthreads();
    }
    Tab<float> tb{GROUP == kGroupPh ? a.f_brems_lnsig : lnsig, a.f_brems_cdf, GROUP == kGroupPh ? lnsig : a.f_bh_lnsig,
                  a.f_bh_cdf, a.f_tri_gp, a.f_tri_split};
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int cell = blockIdx.x * (blockDim.x >> 5) + wid; cell < a.n_cells; cell += nwarps) {
        if (GROUP == kGroupPh) bh_cell<float>(grp, a, tb, cell, acc);
        else ei_cell<float>(grp, a, tb, GROUP, cell, acc);
    }
    flush_acc(acc, a.st, true);
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
    a.st = ctx->stats;
    return a;
}

// Blocks of the persistent batched kernel: resident blocks per SM x SMs.
static int batched_grid(pcc_ctx* ctx, const void* fn, int smem)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchedThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * std::max(ctx->num_sms, 1);
}

extern "C" int pcc_collide(pcc_ctx* ctx, const pcc_cells* cells, pcc_species* em, pcc_species* ep, pcc_species* ph,
                           const pcc_species* ion, double dt, uint64_t seed, uint64_t step, unsigned mask,
                           int precision, float* ledger, void* stream)
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
    cudaStream_t st = (cudaStream_t)stream;
    StepArgs a = make_args(ctx, cells, em, ep, ph, ion, dt, seed, step, mask, ledger);
    const unsigned groups = (mask & 0x700u) ? (mask & 0x700u) : 0x700u;
    const bool ei = (mask & (PCC_BREMS | PCC_TRIDENT)) != 0, bh = (mask & PCC_BH) != 0;
    const bool run_em = ei && (groups & PCC_GROUP_EM), run_ep = ei && (groups & PCC_GROUP_EP);
    const bool run_ph = bh && (groups & PCC_GROUP_PH);
    a.mask = mask & 7u;
    if (precision == PCC_FP64_PLAIN) {
        if (run_em) collide_plain_kernel<kGroupEm><<<cells->n_cells, 128, 0, st>>>(a);
        if (run_ep) collide_plain_kernel<kGroupEp><<<cells->n_cells, 128, 0, st>>>(a);
        if (run_ph) collide_plain_kernel<kGroupPh><<<cells->n_cells, 128, 0, st>>>(a);
    } else {
        const size_t tab_bytes = (size_t)ctx->n_mat * ctx->spec.n_rows * sizeof(float);
        const int stage = (tab_bytes % 16 == 0 && tab_bytes <= 48 * 1024) ? (int)tab_bytes : 0;
        if (run_em || run_ep) {
            const int g = batched_grid(ctx, (const void*)collide_batched_kernel<kGroupEm>, stage);
            if (run_em) collide_batched_kernel<kGroupEm><<<g, kBatchedThreads, stage, st>>>(a, stage);
            if (run_ep) collide_batched_kernel<kGroupEp><<<g, kBatchedThreads, stage, st>>>(a, stage);
        }
        if (run_ph) {
            const int g = batched_grid(ctx, (const void*)collide_batched_kernel<kGroupPh>, stage);
            collide_batched_kernel<kGroupPh><<<g, kBatchedThreads, stage, st>>>(a, stage);
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_collide: launch");
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
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_pairing");
}
