// Material preparation and table build (Sec. II, Sec. III.A) in FP64, plus
// the FP32 copies used by the batched collision kernel.
#include <cmath>
#include <cstring>
#include <vector>

#include "pcc_internal.h"
#include "pcc_physics.cuh"

namespace pcc {

TableGeom make_geom(const pcc_table_spec& s)
{
    TableGeom g;
    g.n_rows = s.n_rows;
    g.n_cols = s.n_cols;
    g.T_min = s.gamma_min - 1.0;
    g.T_max = s.gamma_max - 1.0;
    g.ln_T_min = std::log(g.T_min);
    g.inv_dln_row = (s.n_rows - 1) / std::log(g.T_max / g.T_min);
    g.ln_x_min = -s.cutoff_exp * std::log(10.0);
    g.ln_tri_min = std::log(s.tri_y_min);
    g.f_ln_T_min = (float)g.ln_T_min;
    g.f_inv_dln_row = (float)g.inv_dln_row;
    g.f_ln_x_min = (float)g.ln_x_min;
    g.f_ln_tri_min = (float)g.ln_tri_min;
    return g;
}

enum TableKind { kBrems = 0, kBH = 1, kTriPair = 2, kTriSplit = 3 };
constexpr int kEdgePanels = 12;   // graded sub-panels (ratio 1/4) on the outer column intervals
constexpr int kMaxQuad = 32;

__global__ void material_prep_kernel(const pcc_material* mats, int n, double* screen)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Screen s = screen_from_material(mats[i]);
    double* o = screen + (size_t)i * kScreenFields;
    o[0] = s.LTF; o[1] = s.LD; o[2] = s.etaTF; o[3] = s.etaD;
    o[4] = s.ITFD; o[5] = s.LR; o[6] = s.fC; o[7] = s.Z;
}

// Gauss-Legendre nodes/weights on [-1, 1] (Newton on the Legendre recurrence).
__device__ void legendre_nodes(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double a = 1.0, b = z;
            for (int l = 2; l <= n; ++l) {
                const double c = ((2.0 * l - 1.0) * z * b - (l - 1.0) * a) / l;
                a = b;
                b = c;
            }
            dp = n * (z * b - a) / (z * z - 1.0);
            const double dz = b / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Flags of the table kernels: the printed non-relativistic momentum-transfer
// bounds, and the TFD-quadrature screening mode.
constexpr int kFlagPrinted = 1, kFlagTfdQuad = 2;
constexpr int kTfdNodes = 12;

// Eqs. (defphi1) and (defphi2) for the full Thomas-Fermi-Debye potential,
// whose form factor (Eq. defF, Eq. V_TFD) is
//   1 - F(u) = eta_TF a^2 / (1 + a^2) + eta_D b^2 / (1 + b^2),  a = L_TF u, b = L_D u,
// by quadrature in t = ln u on unit panels from t = 0 down to ln delta (the
// last one shorter), kTfdNodes-point Gauss-Legendre each (nodes gx, gw on
// [-1, 1]).  With r = u/delta the integrands in t are (1 - 1/r)^2 (1 - F)^2
// and (1 + (3 - 6 ln r)/r^2 - 4/r^3) (1 - F)^2.  Zero for delta >= 1.
__device__ void tfd_I12(const Screen& s, double d, const double* gx, const double* gw, double& I1, double& I2)
{
    I1 = 0.0;
    I2 = 0.0;
    if (!(d > 0.0 && d < 1.0)) return;
    const double t0 = log(d);
    for (double hi = 0.0; hi > t0; hi -= 1.0) {
        const double lo = fmax(hi - 1.0, t0);
        const double h = 0.5 * (hi - lo), m = 0.5 * (hi + lo);
        double p1 = 0.0, p2 = 0.0;
        for (int q = 0; q < kTfdNodes; ++q) {
            const double t = m + h * gx[q];
            const double lr = t - t0, ir = exp(-lr);
            const double u = exp(t);
            const double a2 = s.LTF * s.LTF * u * u, b2 = s.LD * s.LD * u * u;
            const double f = s.etaTF * a2 / (1.0 + a2) + s.etaD * b2 / (1.0 + b2);
            const double f2 = f * f;
            const double om = -expm1(-lr);
            p1 += gw[q] * om * om * f2;
            p2 += gw[q] * (1.0 + (3.0 - 6.0 * lr) * ir * ir - 4.0 * ir * ir * ir) * f2;
        }
        I1 += h * p1;
        I2 += h * p2;
    }
}

template <int KIND>
__device__ __forceinline__ double integrand(const Screen& s, double rowv, double v, int flags, const double* tx,
                                            const double* tw)
{
    if (KIND == kBrems) {
        const double x = exp(v);
        const double g1 = 1.0 + rowv, k = x * rowv;
        if ((flags & kFlagTfdQuad) && g1 > 2.0) {
            if (!(k > 0.0 && k < g1 - 1.0)) return 0.0;
            double I1, I2;
            tfd_I12(s, brems_delta(g1, k), tx, tw, I1, I2);
            return dsdk_relativistic_I(s, g1, k, g1 <= 100.0 ? 0.0 : s.fC, I1, I2) * rowv * x;
        }
        return dsdk_brems(s, g1, k, flags & kFlagPrinted) * rowv * x;
    } else if (KIND == kBH) {
        const double k = 2.0 + rowv, gp = 1.0 + v * rowv;
        if (flags & kFlagTfdQuad) {
            const double gm = k - gp;
            if (!(gp > 1.0 && gm > 1.0)) return 0.0;
            double I1, I2;
            tfd_I12(s, k / (2.0 * gp * gm), tx, tw, I1, I2);
            return dsdg_bethe_heitler_I(s, k, gp, I1, I2) * rowv;
        }
        return dsdg_bethe_heitler(s, k, gp) * rowv;
    } else if (KIND == kTriPair) {
        const double y = exp(v);
        return trident_pair_shape(3.0 + rowv, 2.0 + y * rowv) * rowv * y;
    } else {
        return trident_split_shape(2.0 + rowv, 1.0 + v * rowv) * rowv;
    }
}

template <int KIND>
__device__ double panel(const Screen& s, double rowv, double a, double b, int Q, const double* gx, const double* gw,
                        int flags, const double* tx, const double* tw)
{
    const double h = 0.5 * (b - a), m = 0.5 * (a + b);
    double acc = 0.0;
    for (int q = 0; q < Q; ++q) acc += gw[q] * integrand<KIND>(s, rowv, m + h * gx[q], flags, tx, tw);
    return h * acc;
}

// One block per (row, material): integrals over every column interval, then
// the cumulative sum in column order, normalisation and the total.
template <int KIND>
__global__ void table_rows_kernel(const double* screen, TableGeom g, int Q, int flags, double* sigma_out,
                                  double* cdf_out)
{
    extern __shared__ double part[];   // [n_cols]
    __shared__ double gx[kMaxQuad], gw[kMaxQuad], tx[kTfdNodes], tw[kTfdNodes];
    __shared__ double total;
    const int r = blockIdx.x, mat = blockIdx.y, nc = g.n_cols;
    if (threadIdx.x == 0) legendre_nodes(Q, gx, gw);
    if (threadIdx.x == 32 && (flags & kFlagTfdQuad)) legendre_nodes(kTfdNodes, tx, tw);
    Screen s{};
    if (KIND == kBrems || KIND == kBH) s = load_screen(screen + (size_t)mat * kScreenFields);
    const double rowv = g.T_min * pow(g.T_max / g.T_min, (double)r / (g.n_rows - 1));
    const bool logcol = (KIND == kBrems || KIND == kTriPair);
    const double ly = (KIND == kBrems) ? g.ln_x_min : g.ln_tri_min;
    __syncthreads();
    for (int c = threadIdx.x; c < nc - 1; c += blockDim.x) {
        double a, b;
        if (logcol) {
            a = ly * (1.0 - (double)c / (nc - 1));
            b = ly * (1.0 - (double)(c + 1) / (nc - 1));
        } else {
            a = (double)c / (nc - 1);
            b = (double)(c + 1) / (nc - 1);
        }
        const bool right = (c == nc - 2);
        const bool left = (c == 0) && !logcol;
        double v = 0.0;
        if (right) {
            double lo = a, f = 1.0;
            for (int i = 0; i < kEdgePanels; ++i) {
                f *= 0.25;
                const double hi = b - (b - a) * f;
                v += panel<KIND>(s, rowv, lo, hi, Q, gx, gw, flags, tx, tw);
                lo = hi;
            }
            v += panel<KIND>(s, rowv, lo, b, Q, gx, gw, flags, tx, tw);
        } else if (left) {
            double hi = b, f = 1.0;
            for (int i = 0; i < kEdgePanels; ++i) {
                f *= 0.25;
                const double lo = a + (b - a) * f;
                v += panel<KIND>(s, rowv, lo, hi, Q, gx, gw, flags, tx, tw);
                hi = lo;
            }
            v += panel<KIND>(s, rowv, a, hi, Q, gx, gw, flags, tx, tw);
        } else {
            v = panel<KIND>(s, rowv, a, b, Q, gx, gw, flags, tx, tw);
        }
        part[c + 1] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double cum = 0.0;
        part[0] = 0.0;
        for (int c = 1; c < nc; ++c) {
            cum += part[c];
            part[c] = cum;
        }
        total = cum;
    }
    __syncthreads();
    double* row = cdf_out + ((size_t)mat * g.n_rows + r) * nc;
    const double tot = total;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        double v;
        if (tot > 0.0) v = (c == nc - 1) ? 1.0 : part[c] / tot;
        else v = (double)c / (nc - 1);   // zero shape: uniform in the column variable
        row[c] = v;
    }
    if (threadIdx.x == 0 && sigma_out) sigma_out[(size_t)mat * g.n_rows + r] = tot;
}

__global__ void to_float_kernel(const double* in, float* out, size_t n, int take_log)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = take_log ? (float)log(in[i]) : (float)in[i];
}

__global__ void z_to_float_kernel(const double* screen, float* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)screen[(size_t)i * kScreenFields + 7];
}

// Per-material upper bounds B with x <= coef * B for every pair (coef =
// (n_p n_t / n_pt) c dt), used to reject a pair from its uniform alone:
//   Brems:   x = coef sigma(T') p'/(g_e g_i) <= coef sigma(T') beta' (1 + |beta_i|),
//            and the log-log interpolated sigma between rows j, j+1 is at most
//            max(sigma_j, sigma_j+1) while beta' <= beta(T_j+1); the last row
//            covers energies above the table.
//   Trident: sigma_T is increasing in gamma; the bound holds for gamma' <= 1e7.
//   BH:      x = coef sigma(k') k'/(k g_i) <= coef sigma(k') (1 + |beta_i|).
// The factor 2 covers 1 + |beta_i|; 1e-3 more covers float rounding of x.
__global__ void bounds_kernel(const double* screen, const double* brems_sigma, const double* bh_sigma, TableGeom g,
                              int n_mat, float* bound)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_mat) return;
    const double* sb = brems_sigma + (size_t)m * g.n_rows;
    const double* sh = bh_sigma + (size_t)m * g.n_rows;
    double bb = sb[g.n_rows - 1], bh = 0.0;
    for (int j = 0; j + 1 < g.n_rows; ++j) {
        const double T = g.T_min * pow(g.T_max / g.T_min, (double)(j + 1) / (g.n_rows - 1));
        const double beta = sqrt(T * (T + 2.0)) / (1.0 + T);
        bb = fmax(bb, fmax(sb[j], sb[j + 1]) * beta);
    }
    for (int j = 0; j < g.n_rows; ++j) bh = fmax(bh, sh[j]);
    const double Z = screen[(size_t)m * kScreenFields + 7];
    const double l = log((1e7 + 4.5) / 6.89);
    const double bt = 5.22e-34 * Z * Z * l * l * l;
    const double margin = 2.0 * 1.001;
    bound[3 * m + 0] = (float)(margin * bb);
    bound[3 * m + 1] = (float)(margin * bt);
    bound[3 * m + 2] = (float)(margin * bh);
}

}  // namespace pcc

using namespace pcc;

static void free_tables(pcc_ctx* ctx)
{
    void* ptrs[] = {ctx->screen, ctx->brems_sigma, ctx->brems_cdf, ctx->bh_sigma, ctx->bh_cdf, ctx->tri_gp_cdf,
                    ctx->tri_split_cdf, ctx->f_brems_lnsig, ctx->f_brems_cdf, ctx->f_bh_lnsig, ctx->f_bh_cdf,
                    ctx->f_tri_gp_cdf, ctx->f_tri_split_cdf, ctx->f_Z, ctx->f_bound};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    ctx->screen = ctx->brems_sigma = ctx->brems_cdf = ctx->bh_sigma = ctx->bh_cdf = nullptr;
    ctx->tri_gp_cdf = ctx->tri_split_cdf = nullptr;
    ctx->f_brems_lnsig = ctx->f_brems_cdf = ctx->f_bh_lnsig = ctx->f_bh_cdf = nullptr;
    ctx->f_tri_gp_cdf = ctx->f_tri_split_cdf = ctx->f_Z = ctx->f_bound = nullptr;
    ctx->n_mat = 0;
}

void pcc_free_tables(pcc_ctx* ctx) { free_tables(ctx); }

extern "C" int pcc_tables_build(pcc_ctx* ctx, const pcc_material* mats, int n_mats, const pcc_table_spec* spec,
                                void* stream)
{
    if (!ctx || !mats || !spec) { set_error("pcc_tables_build: null argument"); return PCC_E_INVALID; }
    const pcc_table_spec& s = *spec;
    if (n_mats < 1 || n_mats > 4096 || s.n_rows < 2 || s.n_rows > 4096 || s.n_cols < 3 || s.n_cols > 4096 ||
        s.quad_nodes < 1 || s.quad_nodes > kMaxQuad || !(s.gamma_min > 1.0) || !(s.gamma_max > s.gamma_min) ||
        s.cutoff_exp < 1 || s.cutoff_exp > 30 || !(s.tri_y_min > 0.0 && s.tri_y_min < 1.0) ||
        (s.nr_qbounds != 0 && s.nr_qbounds != 1) ||
        (s.screening != PCC_SCREEN_REDUCED && s.screening != PCC_SCREEN_TFD_QUAD)) {
        set_error("pcc_tables_build: invalid table spec");
        return PCC_E_INVALID;
    }
    for (int i = 0; i < n_mats; ++i) {
        const pcc_material& m = mats[i];
        if (m.Z < 1 || m.Z > 120 || !(m.Zstar >= 0.0 && m.Zstar <= m.Z) || !(m.n_i > 0.0) || !(m.T_e >= 0.0) ||
            !(m.s_TF > 0.0) || !(m.s_D > 0.0) || (m.Zstar > 0.0 && !(m.T_e > 0.0))) {
            set_error("pcc_tables_build: invalid material " + std::to_string(i));
            return PCC_E_INVALID;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    free_tables(ctx);
    const size_t R = s.n_rows, C = s.n_cols, M = n_mats;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    A((void**)&ctx->screen, M * kScreenFields * sizeof(double));
    A((void**)&ctx->brems_sigma, M * R * sizeof(double));
    A((void**)&ctx->brems_cdf, M * R * C * sizeof(double));
    A((void**)&ctx->bh_sigma, M * R * sizeof(double));
    A((void**)&ctx->bh_cdf, M * R * C * sizeof(double));
    A((void**)&ctx->tri_gp_cdf, R * C * sizeof(double));
    A((void**)&ctx->tri_split_cdf, R * C * sizeof(double));
    A((void**)&ctx->f_brems_lnsig, M * R * sizeof(float));
    A((void**)&ctx->f_brems_cdf, M * R * C * sizeof(float));
    A((void**)&ctx->f_bh_lnsig, M * R * sizeof(float));
    A((void**)&ctx->f_bh_cdf, M * R * C * sizeof(float));
    A((void**)&ctx->f_tri_gp_cdf, R * C * sizeof(float));
    A((void**)&ctx->f_tri_split_cdf, R * C * sizeof(float));
    A((void**)&ctx->f_Z, M * sizeof(float));
    A((void**)&ctx->f_bound, 3 * M * sizeof(float));
    if (e != cudaSuccess) { free_tables(ctx); return cuda_fail(e, "pcc_tables_build: cudaMalloc"); }

    pcc_material* dmats = nullptr;
    e = cudaMalloc(&dmats, M * sizeof(pcc_material));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dmats, mats, M * sizeof(pcc_material), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { free_tables(ctx); if (dmats) cudaFree(dmats); return cuda_fail(e, "pcc_tables_build: upload"); }
    material_prep_kernel<<<(n_mats + 63) / 64, 64, 0, st>>>(dmats, n_mats, ctx->screen);

    const TableGeom g = make_geom(s);
    const int flags = (s.nr_qbounds ? kFlagPrinted : 0) | (s.screening == PCC_SCREEN_TFD_QUAD ? kFlagTfdQuad : 0);
    const size_t smem = C * sizeof(double);
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(table_rows_kernel<kBrems>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(table_rows_kernel<kBH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(table_rows_kernel<kTriPair>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(table_rows_kernel<kTriSplit>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    table_rows_kernel<kBrems><<<dim3(s.n_rows, n_mats), 128, smem, st>>>(ctx->screen, g, s.quad_nodes, flags,
                                                                         ctx->brems_sigma, ctx->brems_cdf);
    table_rows_kernel<kBH><<<dim3(s.n_rows, n_mats), 128, smem, st>>>(ctx->screen, g, s.quad_nodes, flags,
                                                                      ctx->bh_sigma, ctx->bh_cdf);
    table_rows_kernel<kTriPair><<<dim3(s.n_rows, 1), 128, smem, st>>>(ctx->screen, g, s.quad_nodes, flags,
                                                                      nullptr, ctx->tri_gp_cdf);
    table_rows_kernel<kTriSplit><<<dim3(s.n_rows, 1), 128, smem, st>>>(ctx->screen, g, s.quad_nodes, flags,
                                                                       nullptr, ctx->tri_split_cdf);
    auto conv = [&](const double* in, float* out, size_t n, int lg) {
        to_float_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n, lg);
    };
    conv(ctx->brems_sigma, ctx->f_brems_lnsig, M * R, 1);
    conv(ctx->brems_cdf, ctx->f_brems_cdf, M * R * C, 0);
    conv(ctx->bh_sigma, ctx->f_bh_lnsig, M * R, 1);
    conv(ctx->bh_cdf, ctx->f_bh_cdf, M * R * C, 0);
    conv(ctx->tri_gp_cdf, ctx->f_tri_gp_cdf, R * C, 0);
    conv(ctx->tri_split_cdf, ctx->f_tri_split_cdf, R * C, 0);
    z_to_float_kernel<<<(n_mats + 63) / 64, 64, 0, st>>>(ctx->screen, ctx->f_Z, n_mats);
    bounds_kernel<<<(n_mats + 63) / 64, 64, 0, st>>>(ctx->screen, ctx->brems_sigma, ctx->bh_sigma, g, n_mats,
                                                     ctx->f_bound);
    note_launches(13);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dmats);
    if (e != cudaSuccess) { free_tables(ctx); return cuda_fail(e, "pcc_tables_build: kernels"); }
    ctx->n_mat = n_mats;
    ctx->spec = s;
    return PCC_OK;
}

extern "C" int pcc_tables_read(pcc_ctx* ctx, double* brems_sigma, double* brems_cdf, double* bh_sigma,
                               double* bh_cdf, double* tri_gp_cdf, double* tri_split_cdf, double* screening)
{
    if (!ctx) { set_error("pcc_tables_read: null context"); return PCC_E_INVALID; }
    if (ctx->n_mat == 0) { set_error("pcc_tables_read: no tables"); return PCC_E_NO_TABLES; }
    const size_t R = ctx->spec.n_rows, C = ctx->spec.n_cols, M = ctx->n_mat;
    cudaError_t e = cudaSuccess;
    auto cp = [&](double* dst, const double* src, size_t n) {
        if (dst && e == cudaSuccess) e = cudaMemcpy(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost);
    };
    cp(brems_sigma, ctx->brems_sigma, M * R);
    cp(brems_cdf, ctx->brems_cdf, M * R * C);
    cp(bh_sigma, ctx->bh_sigma, M * R);
    cp(bh_cdf, ctx->bh_cdf, M * R * C);
    cp(tri_gp_cdf, ctx->tri_gp_cdf, R * C);
    cp(tri_split_cdf, ctx->tri_split_cdf, R * C);
    cp(screening, ctx->screen, M * kScreenFields);
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, "pcc_tables_read");
}
