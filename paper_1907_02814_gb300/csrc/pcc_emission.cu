// Expected-emission operator and its adjoint (see pcc.h).
//
// Per cell c with plasma parameters theta = (n_i, T_e, Z*, s_TF, s_D) and
// electron samples (gamma_s, w_s), for ions at rest:
//   R_gamma = n_i sum_s w_s v_s sigma_B(gamma_s)          (rate form of Eq. N_br_theo1)
//   R_pair  = n_i sum_s w_s v_s sigma_T(gamma_s)          (Sec. II.D fit)
//   P_rad   = n_i sum_s w_s v_s int k dsigma_B/dk dk      (radiative stopping power, Sec. III.B)
// where the k-integrals run over x = k/(gamma-1) in [1e-7, 1] by one n-point
// Gauss-Legendre panel in ln x.  dsigma/dk is Eq. (cs_br_nr) with the Elwert
// factor for gamma <= 2, Eq. (csre) for 2 < gamma <= 100 and Eq. (csur)
// above, with the screening of Sec. II.A.
//
// Precision.  Relativistic nodes run in FP32.  The printed closed form of
// I2 (Eq. deriv_I2) cancels terms of size (L delta)^2 ln L down to O(1),
// which destroys FP32 once L delta >> 1 (L_R is 45 to 10^4 here).  For
// L delta > 1 it is evaluated in a rearranged form with no such cancellation:
// with u = L delta, rho = L^2/(1+L^2), z = L(1-delta)/(1+L u), g(z) = z - atan z,
//   2 I2 = -2 ln d - 6 u^2 ln d/(1+L^2) + (1+3u^2)(log1p(L^-2) - log1p(u^-2))
//          + 4 u^3 g(z) + 4 u^2 (1-d)/(1+u L) - 4 u^2 (1-d)/(1+L^2) + rho (d^2-1),
// (the same function; g by its odd series for z < 1/4), and atan L - atan u
// as atan(L(1-d)/(1+L u)).  Non-relativistic nodes (gamma <= 2, a small
// share of samples, warp-uniform because a warp takes one sample) run in
// FP32 in a rearranged form (nr_sample32), or in FP64 in cells where L_D is
// within 5 % of L_TF, where the cross term's divided difference cancels.  Sums over nodes and samples use compensated FP32 per lane and FP64
// across lanes and warps.
//
// Adjoint.  The parameters enter only through the screening quantities
// (L_R for gamma > 2; L_TF, L_D and eta_D = Z*/Z = 1 - eta_TF for gamma <= 2)
// and the n_i prefactor.  The adjoint kernel carries forward tangents of the
// node integrands with respect to those four quantities (dual numbers),
// reduces them per cell, and contracts them with grad_out through the
// analytic Jacobian of the screening quantities:
//   L_TF = s_TF Z^(-1/3)/alpha,  L_D = s_D max(lambda_D, r_i)/r_C,
//   a = I_TFD, h(x) = ln(1+x) - x/(1+x), h(L_R^2) = 2a  =>  dL_R/da = (1+L_R^2)^2/L_R^3.
#include <cmath>
#include <vector>

#include "pcc_internal.h"
#include "pcc_physics.cuh"

namespace {

using namespace pcc;

constexpr int kMaxQuad = 128;
constexpr int kEmThreads = 256;
constexpr int kEmWarps = kEmThreads / 32;

// ---------------------------------------------------------------- duals ---
template <typename T, int N>
struct Dual {
    T v;
    T d[N];
};

template <typename T> __device__ __forceinline__ T val(T x) { return x; }
template <typename T, int N> __device__ __forceinline__ T val(const Dual<T, N>& x) { return x.v; }

template <typename T, int N>
__device__ __forceinline__ Dual<T, N> mk(T v)
{
    Dual<T, N> r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = T(0);
    return r;
}

#define DUAL_BIN(OP, DV)                                                                                  \
    template <typename T, int N>                                                                          \
    __device__ __forceinline__ Dual<T, N> operator OP(const Dual<T, N>& a, const Dual<T, N>& b)           \
    {                                                                                                     \
        Dual<T, N> r;                                                                                     \
        r.v = a.v OP b.v;                                                                                 \
        _Pragma("unroll") for (int i = 0; i < N; ++i) r.d[i] = DV;                                        \
        return r;                                                                                         \
    }
DUAL_BIN(+, a.d[i] + b.d[i])
DUAL_BIN(-, a.d[i] - b.d[i])
DUAL_BIN(*, a.d[i] * b.v + a.v * b.d[i])
#undef DUAL_BIN

template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b)
{
    Dual<T, N> r;
    const T ib = T(1) / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}

template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a)
{
    Dual<T, N> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}

// mixed with a plain scalar
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const Dual<T, N>& a, T b) { Dual<T, N> r = a; r.v += b; return r; }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator+(T b, const Dual<T, N>& a) { return a + b; }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a, T b) { Dual<T, N> r = a; r.v -= b; return r; }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(T b, const Dual<T, N>& a) { return -a + b; }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N>& a, T b)
{
    Dual<T, N> r;
    r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
    return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(T b, const Dual<T, N>& a) { return a * b; }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator/(T a, const Dual<T, N>& b)
{
    Dual<T, N> r;
    const T ib = T(1) / b.v;
    r.v = a * ib;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -r.v * b.d[i] * ib;
    return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator/(const Dual<T, N>& a, T b) { return a * (T(1) / b); }

// chain rule for a scalar function with value f and derivative df at a.v
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> chain(const Dual<T, N>& a, T f, T df)
{
    Dual<T, N> r;
    r.v = f;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * df;
    return r;
}

__device__ __forceinline__ float f_atan(float x) { return atanf(x); }
__device__ __forceinline__ float f_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double f_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float f_log(float x) { return logf(x); }
__device__ __forceinline__ double f_log(double x) { return log(x); }

template <typename T, int N>
__device__ __forceinline__ Dual<T, N> f_atan(const Dual<T, N>& a) { return chain(a, f_atan(a.v), T(1) / (T(1) + a.v * a.v)); }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> f_log1p(const Dual<T, N>& a) { return chain(a, f_log1p(a.v), T(1) / (T(1) + a.v)); }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> f_log(const Dual<T, N>& a) { return chain(a, f_log(a.v), T(1) / a.v); }

// ------------------------------------------------------ Yukawa I1, I2 -----
// z - atan z: odd series below 1/4, direct above.
template <typename R>
__device__ __forceinline__ R z_minus_atan(R z)
{
    using S = decltype(val(z));
    if (val(z) < S(0.25)) {
        const R z2 = z * z;
        // z^3 (1/3 - z^2/5 + z^4/7 - ... ) to z^15
        R s = S(1.0 / 15.0) - z2 * S(1.0 / 17.0);
        s = S(1.0 / 13.0) - z2 * s;
        s = S(1.0 / 11.0) - z2 * s;
        s = S(1.0 / 9.0) - z2 * s;
        s = S(1.0 / 7.0) - z2 * s;
        s = S(1.0 / 5.0) - z2 * s;
        s = S(1.0 / 3.0) - z2 * s;
        return s * z2 * z;
    }
    return z - f_atan(z);
}

// I1(d, L) and I2(d, L) of Eqs. (deriv_I1), (deriv_I2); L may carry tangents.
template <typename R, typename S>
__device__ __forceinline__ void yukawa_I12(R L, S d, R& I1, R& I2)
{
    const S one = S(1), omd = one - d;
    const R u = L * d;
    const R L2 = L * L, u2 = u * u;
    const R A = f_atan(L * omd / (one + L * u));                 // atan L - atan u
    const R lnr = f_log1p(L2 * (one - d * d) / (one + u2));      // ln((1+L^2)/(1+u^2))
    const R rho = L2 / (one + L2);
    I1 = -(u * A) - S(0.5) * rho * (omd * omd) + S(0.5) * lnr;
    const S lnd = f_log(d);
    R t;
    if (val(u) <= one) {
        t = S(-4) * u2 * u * A + (one + S(3) * u2) * lnr + S(6) * lnd * u2 * rho + rho * (d * d - one) +
            S(4) * omd * u2 * rho;
    } else {
        const R z = L * omd / (one + L * u);
        t = S(-2) * lnd - S(6) * lnd * u2 / (one + L2) +
            (one + S(3) * u2) * (f_log1p(one / L2) - f_log1p(one / u2)) + S(4) * u2 * u * z_minus_atan(z) +
            S(4) * omd * u2 / (one + u * L) - S(4) * omd * u2 / (one + L2) + rho * (d * d - one);
    }
    I2 = S(0.5) * t;
}

// -------------------------------------------- non-relativistic (FP64) ----
// g of Eq. (cs_br_nr).
template <typename R>
__device__ __forceinline__ R nr_g_t(double qp, double qm, R eta, R L)
{
    const R L2 = L * L;
    const R Dp = 1.0 + (qp * qp) * L2, Dm = 1.0 + (qm * qm) * L2;
    return 0.5 * (eta * eta) * (f_log1p(((qp * qp - qm * qm) * L2) / Dm) + 1.0 / Dp - 1.0 / Dm);
}

// Gamma_c of Eq. (cs_br_nr), midpoint limit when L_D ~ L_TF.
template <typename R>
__device__ __forceinline__ R nr_cross_t(double qp, double qm, R eTF, R LTF, R eD, R LD)
{
    const R A = LTF * LTF, B = LD * LD;
    const R d = B - A;
    if (fabs(val(d)) <= 1e-6 * fmax(val(A), val(B))) {
        const R M = 0.5 * (A + B);
        const R Mp = 1.0 + (qp * qp) * M, Mm = 1.0 + (qm * qm) * M;
        return eTF * eD * (f_log(Mp / Mm) + 1.0 / Mp - 1.0 / Mm);
    }
    const R Tp = 1.0 + (qp * qp) * A, Tm = 1.0 + (qm * qm) * A;
    const R Dp = 1.0 + (qp * qp) * B, Dm = 1.0 + (qm * qm) * B;
    return eTF * eD / d * (A * f_log(Dm / Dp) + B * f_log(Tp / Tm));
}

// ---------------------------------------------------------------- cells ---
struct CellScreen {
    double LTF, LD, etaTF, etaD, a, LR;
    double n_i, T_e, Zs, sTF, sD;
    bool debye;   // lambda_D > r_i (the Debye branch of L_D is active)
    bool nr32;    // L_D and L_TF far enough apart for the FP32 non-relativistic branch
    bool ok;
};

__device__ CellScreen cell_screen(const float* p, int Z)
{
    CellScreen c;
    c.n_i = p[0]; c.T_e = p[1]; c.Zs = p[2]; c.sTF = p[3]; c.sD = p[4];
    c.ok = c.n_i > 0.0 && c.T_e >= 0.0 && c.Zs >= 0.0 && c.Zs <= Z && c.sTF > 0.0 && c.sD > 0.0 &&
           isfinite(c.n_i) && isfinite(c.T_e);
    if (!c.ok) return c;
    c.LTF = c.sTF * exp(-log((double)Z) / 3.0) / kAlpha;
    const double ri = cbrt(3.0 / (4.0 * kPi * c.n_i));
    if (c.Zs > 0.0) {
        const double lam = sqrt(kEps0 * c.T_e / (kQe * c.n_i * c.Zs * (c.Zs + 1.0)));
        c.debye = lam > ri;
        c.LD = c.sD * fmax(lam, ri) / kRc;
    } else {
        // Z* = 0: Eq. LDH gives lambda_D = infinity.  Nothing depends on L_D
        // then (eta_D = 0), and the derivative with respect to Z* is the limit
        // from Z* > 0, in which the cross terms take their L_D -> infinity
        // values.  A finite stand-in 1e5 L_TF gives those limits to ~1e-9
        // and keeps every FP32 product of the non-relativistic duals finite.
        c.debye = false;
        c.LD = 1e5 * c.LTF;
    }
    c.etaD = c.Zs / Z;
    c.etaTF = 1.0 - c.etaD;
    c.a = i_tfd(c.etaTF, c.LTF, c.etaD, c.LD);
    const double w = lambert_w0_neg(-exp(-1.0 - 2.0 * c.a));
    c.LR = sqrt(expm1(w + 1.0 + 2.0 * c.a));
    const double A = c.LTF * c.LTF, B = c.LD * c.LD;
    c.nr32 = fabs(B - A) > 0.05 * fmax(A, B);
    return c;
}

// Screening quantities of every cell, one thread per cell (FP64).
__global__ void screen_kernel(const float* __restrict__ params, int n_cells, int Z, CellScreen* __restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_cells) out[c] = cell_screen(params + 5 * (size_t)c, Z);
}

struct EmArgs {
    int n_cells, n_samples, Z, n_quad;
    double fC;          // Coulomb correction f_C(Z)
    const float* params;
    const float* gamma;
    const float* w;
    const float* grad_out;
    float* out;
    DevStats* st;
    const CellScreen* screen;   // per-cell screening, computed by screen_kernel
    float lx[kMaxQuad]; // ln x at the nodes
    float hw[kMaxQuad]; // half-width times weight
};

// Per-lane accumulators: value sums of sigma and k sigma, and their
// tangents with respect to L_R (relativistic) and (L_TF, L_D, eta_D) (NR).
struct Acc {
    Kahan r, p;
    Kahan r_LR, p_LR;
    double r_nr[3], p_nr[3];
};

template <bool GRAD>
__device__ __forceinline__ void rel_sample(const EmArgs& a, float g, float bw, float LR, float fc, int lane, Acc& acc)
{
    const float T = g - 1.0f, ig = 1.0f / g;
    float sr = 0.f, sp = 0.f, dr = 0.f, dp = 0.f;
    for (int q = lane; q < a.n_quad; q += 32) {
        const float l = a.lx[q];
        const float x = expf(l), omx = -expm1f(l);
        const float k = x * T;
        const float gk = 1.0f + T * omx;              // gamma - k
        const float eps = gk * ig;
        const float d = k / (2.0f * g * gk);
        const float c1 = 1.0f + eps * eps, c2 = (2.0f / 3.0f) * eps;
        float f, df = 0.f;
        if (GRAD) {
            Dual<float, 1> L = mk<float, 1>(LR), I1, I2;
            L.d[0] = 1.0f;
            yukawa_I12(L, d, I1, I2);
            f = c1 * (I1.v + 1.0f - fc) - c2 * (I2.v + 5.0f / 6.0f - fc);
            df = c1 * I1.d[0] - c2 * I2.d[0];
        } else {
            float I1, I2;
            yukawa_I12(LR, d, I1, I2);
            f = c1 * (I1 + 1.0f - fc) - c2 * (I2 + 5.0f / 6.0f - fc);
        }
        if (!(f > 0.0f)) { f = 0.0f; df = 0.0f; }
        const float h = a.hw[q];
        sr += h * f;
        sp += h * f * k;
        if (GRAD) { dr += h * df; dp += h * df * k; }
    }
    acc.r.add(bw * sr);
    acc.p.add(bw * sp);
    if (GRAD) { acc.r_LR.add(bw * dr); acc.p_LR.add(bw * dp); }
}

// FP32 form of Eq. (cs_br_nr) with the Elwert factor, used when L_D and L_TF
// differ by more than 5 %.  With P = q+^2 - q-^2 = 4 p1 p2 exactly, the
// Yukawa terms are log1p(P L^2 / D-) - P L^2 / (D+ D-) and the cross term is
// (B log1p(P A / T-) - A log1p(P B / D-)) / (B - A), A = L_TF^2, B = L_D^2:
// no difference of nearly equal numbers is formed.
template <typename R>
__device__ __forceinline__ R nr_g32(float P, float qp, float qm, R eta, R L)
{
    const R L2 = L * L;
    const R Dp = 1.0f + (qp * qp) * L2, Dm = 1.0f + (qm * qm) * L2;
    return 0.5f * (eta * eta) * (f_log1p((P * L2) / Dm) - (P * L2) / (Dp * Dm));
}

template <typename R>
__device__ __forceinline__ R nr_cross32(float P, float qm, R eTF, R LTF, R eD, R LD)
{
    const R A = LTF * LTF, B = LD * LD;
    const R Tm = 1.0f + (qm * qm) * A, Dm = 1.0f + (qm * qm) * B;
    return eTF * eD / (B - A) * (B * f_log1p((P * A) / Tm) - A * f_log1p((P * B) / Dm));
}

template <bool GRAD>
__device__ __forceinline__ void nr_sample32(const EmArgs& a, float g, float bw, const CellScreen& cs, int lane,
                                            Acc& acc)
{
    const float T1 = g - 1.0f, p1 = sqrtf(T1 * (T1 + 2.0f)), b1 = p1 / g;
    const float az = 2.0f * (float)kPi * (float)a.Z * (float)kAlpha;
    const float ex1 = -expm1f(-az / b1);
    float sr = 0.f, sp = 0.f, dr[3] = {0.f, 0.f, 0.f}, dp[3] = {0.f, 0.f, 0.f};
    for (int q = lane; q < a.n_quad; q += 32) {
        const float l = a.lx[q];
        const float x = expf(l), k = x * T1;
        const float T2 = T1 * (-expm1f(l));
        if (!(k > 0.f && T2 > 0.f)) continue;
        const float p2 = sqrtf(T2 * (T2 + 2.0f));
        const float qp = p1 + p2, qm = k * (T1 + T2 + 2.0f) / qp;
        const float b2 = p2 / (1.0f + T2);
        const float fE = (b1 / b2) * ex1 / (-expm1f(-az / b2));
        const float pre = 4.0f / (3.0f * p1 * p1) * fE;
        const float P = 4.0f * p1 * p2;
        float fv, fd[3] = {0.f, 0.f, 0.f};
        if (GRAD) {
            Dual<float, 3> LTF = mk<float, 3>((float)cs.LTF), LD = mk<float, 3>((float)cs.LD);
            Dual<float, 3> eD = mk<float, 3>((float)cs.etaD), eTF = mk<float, 3>((float)cs.etaTF);
            LTF.d[0] = 1.0f; LD.d[1] = 1.0f; eD.d[2] = 1.0f; eTF.d[2] = -1.0f;
            const Dual<float, 3> br = nr_g32(P, qp, qm, eTF, LTF) + nr_g32(P, qp, qm, eD, LD) +
                                      nr_cross32(P, qm, eTF, LTF, eD, LD);
            fv = pre * br.v;
            for (int i = 0; i < 3; ++i) fd[i] = pre * br.d[i];
        } else {
            const float LTF = (float)cs.LTF, LD = (float)cs.LD, eTF = (float)cs.etaTF, eD = (float)cs.etaD;
            fv = pre * (nr_g32(P, qp, qm, eTF, LTF) + nr_g32(P, qp, qm, eD, LD) + nr_cross32(P, qm, eTF, LTF, eD, LD));
        }
        if (!(fv > 0.f)) { fv = 0.f; fd[0] = fd[1] = fd[2] = 0.f; }
        const float h = a.hw[q];
        sr += h * fv;
        sp += h * fv * k;
        if (GRAD)
            for (int i = 0; i < 3; ++i) { dr[i] += h * fd[i]; dp[i] += h * fd[i] * k; }
    }
    acc.r.add(bw * sr);
    acc.p.add(bw * sp);
    if (GRAD)
        for (int i = 0; i < 3; ++i) { acc.r_nr[i] += (double)(bw * dr[i]); acc.p_nr[i] += (double)(bw * dp[i]); }
}

template <bool GRAD>
__device__ __forceinline__ void nr_sample(const EmArgs& a, double g, double bw, const CellScreen& cs, int lane,
                                          Acc& acc)
{
    const double T1 = g - 1.0, p1 = sqrt(T1 * (T1 + 2.0)), b1 = p1 / g;
    const double Z = a.Z, az = 2.0 * kPi * Z * kAlpha;
    double sr = 0.0, sp = 0.0, dr[3] = {0, 0, 0}, dp[3] = {0, 0, 0};
    for (int q = lane; q < a.n_quad; q += 32) {
        const double l = a.lx[q];
        const double x = exp(l), k = x * T1;
        const double T2 = T1 * (-expm1(l));
        if (!(k > 0.0 && T2 > 0.0)) continue;
        const double p2 = sqrt(T2 * (T2 + 2.0));
        const double qp = p1 + p2, qm = k * (T1 + T2 + 2.0) / (p1 + p2);
        const double b2 = p2 / (1.0 + T2);
        const double fE = (b1 / b2) * (-expm1(-az / b1)) / (-expm1(-az / b2));
        // f / (4 Z^2 r_e^2 alpha) = 4/(3 p1^2) * bracket * f_E
        const double pre = 4.0 / (3.0 * p1 * p1) * fE;
        double fv;
        double fd[3] = {0, 0, 0};
        if (GRAD) {
            Dual<double, 3> LTF = mk<double, 3>(cs.LTF), LD = mk<double, 3>(cs.LD);
            Dual<double, 3> eD = mk<double, 3>(cs.etaD), eTF = mk<double, 3>(cs.etaTF);
            LTF.d[0] = 1.0; LD.d[1] = 1.0; eD.d[2] = 1.0; eTF.d[2] = -1.0;
            const Dual<double, 3> br = nr_g_t(qp, qm, eTF, LTF) + nr_g_t(qp, qm, eD, LD) +
                                       nr_cross_t(qp, qm, eTF, LTF, eD, LD);
            fv = pre * br.v;
            for (int i = 0; i < 3; ++i) fd[i] = pre * br.d[i];
        } else {
            const double br = nr_g_t(qp, qm, cs.etaTF, cs.LTF) + nr_g_t(qp, qm, cs.etaD, cs.LD) +
                              nr_cross_t(qp, qm, cs.etaTF, cs.LTF, cs.etaD, cs.LD);
            fv = pre * br;
        }
        if (!(fv > 0.0)) { fv = 0.0; fd[0] = fd[1] = fd[2] = 0.0; }
        const double h = a.hw[q];
        sr += h * fv;
        sp += h * fv * k;
        if (GRAD)
            for (int i = 0; i < 3; ++i) { dr[i] += h * fd[i]; dp[i] += h * fd[i] * k; }
    }
    acc.r.add((float)(bw * sr));
    acc.p.add((float)(bw * sp));
    if (GRAD)
        for (int i = 0; i < 3; ++i) { acc.r_nr[i] += bw * dr[i]; acc.p_nr[i] += bw * dp[i]; }
}

// Sums per cell, in units of 4 Z^2 r_e^2 alpha c (rates) and m_e c^2 (power):
// [0] sum w beta sigma, [1] sum w beta k-sigma, [2] sum w v sigma_T (SI),
// [3] d[0]/dL_R, [4] d[1]/dL_R, [5..7] d[0]/d(L_TF, L_D, eta_D), [8..10] d[1]/d(...)
constexpr int kSums = 11;

template <bool GRAD>
__global__ void __launch_bounds__(kEmThreads, GRAD ? 2 : 4) emission_kernel(const __grid_constant__ EmArgs a)
{
    __shared__ double part[kEmWarps][kSums];
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const CellScreen cs = a.screen[c];
    if (!cs.ok) {
        if (threadIdx.x == 0) {
            raise_status(a.st, PCC_ST_NONFINITE);
            const float nan = __int_as_float(0x7fc00000);
            if (GRAD) for (int k = 0; k < 5; ++k) a.out[5 * (size_t)c + k] = nan;
            else for (int k = 0; k < 3; ++k) a.out[3 * (size_t)c + k] = nan;
        }
        return;
    }
    Acc acc;
    for (int i = 0; i < 3; ++i) acc.r_nr[i] = acc.p_nr[i] = 0.0;
    Kahan pair;
    const float LR = (float)cs.LR;
    const float* gs = a.gamma + (size_t)c * a.n_samples;
    const float* ws = a.w + (size_t)c * a.n_samples;
    for (int s = wid; s < a.n_samples; s += kEmWarps) {
        const float g = gs[s], wt = ws[s];
        if (!(g > 1.0f) || !(wt != 0.0f)) continue;               // at rest or no weight: no emission
        const float T = g - 1.0f;
        const float bw = wt * (sqrtf(T * (T + 2.0f)) / g);    // w beta, FP32 (the FP64 units are scarce)
        if (g <= 2.0f) {
            if (cs.nr32) nr_sample32<GRAD>(a, g, bw, cs, lane, acc);
            else nr_sample<GRAD>(a, (double)g, (double)bw, cs, lane, acc);
        }
        else rel_sample<GRAD>(a, g, bw, LR, g > 100.0f ? (float)a.fC : 0.0f, lane, acc);
        if (lane == 0) pair.add(bw * sigma_trident<float>((float)a.Z, g));
    }
    double v[kSums];
    v[0] = (double)acc.r.s - acc.r.c;
    v[1] = (double)acc.p.s - acc.p.c;
    v[2] = (double)pair.s - pair.c;
    v[3] = (double)acc.r_LR.s - acc.r_LR.c;
    v[4] = (double)acc.p_LR.s - acc.p_LR.c;
    for (int i = 0; i < 3; ++i) { v[5 + i] = acc.r_nr[i]; v[8 + i] = acc.p_nr[i]; }
    for (int i = 0; i < kSums; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0)
        for (int i = 0; i < kSums; ++i) part[wid][i] = v[i];
    __syncthreads();
    if (threadIdx.x != 0) return;
    double S[kSums];
    for (int i = 0; i < kSums; ++i) {
        S[i] = 0.0;
        for (int k = 0; k < kEmWarps; ++k) S[i] += part[k][i];
    }
    const double C0 = 4.0 * a.Z * a.Z * kRe * kRe * kAlpha * kC;   // rate unit
    const double R = cs.n_i * C0 * S[0], P = cs.n_i * C0 * S[1], Rp = cs.n_i * kC * S[2];
    if (!GRAD) {
        a.out[3 * (size_t)c + 0] = (float)R;
        a.out[3 * (size_t)c + 1] = (float)Rp;
        a.out[3 * (size_t)c + 2] = (float)P;
        return;
    }
    // ---- adjoint: d out / d theta through the screening quantities
    const double g0 = a.grad_out[3 * (size_t)c + 0], g1 = a.grad_out[3 * (size_t)c + 1],
                 g2 = a.grad_out[3 * (size_t)c + 2];
    // d(g0 R + g2 P)/dS for S = L_R, L_TF, L_D, eta_D (without the n_i C0 factor)
    const double dLR = g0 * S[3] + g2 * S[4];
    const double dLTF = g0 * S[5] + g2 * S[8];
    const double dLD = g0 * S[6] + g2 * S[9];
    const double deD = g0 * S[7] + g2 * S[10];
    // a = I_TFD(eta_TF, L_TF, eta_D, L_D) and its partials
    const double A = cs.LTF * cs.LTF, B = cs.LD * cs.LD;
    const double hA = log1p(A) - A / (1.0 + A), hB = log1p(B) - B / (1.0 + B);
    const double hpA = A / ((1.0 + A) * (1.0 + A)), hpB = B / ((1.0 + B) * (1.0 + B));
    double X, XA, XB;
    const double D = B - A;
    if (fabs(D) <= 1e-4 * fmax(A, B)) {
        const double M = 0.5 * (A + B);
        X = log1p(M) - M / (1.0 + M);
        XA = XB = 0.5 * M / ((1.0 + M) * (1.0 + M));
    } else {
        const double N = B * log1p(A) - A * log1p(B);
        X = N / D;
        XA = ((B / (1.0 + A) - log1p(B)) * D + N) / (D * D);
        XB = ((log1p(A) - A / (1.0 + B)) * D - N) / (D * D);
    }
    const double eT = cs.etaTF, eDv = cs.etaD;
    const double da_deD = -eT * hA + eDv * hB + (eT - eDv) * X;
    const double da_dLTF = (0.5 * eT * eT * hpA + eT * eDv * XA) * 2.0 * cs.LTF;
    const double da_dLD = (0.5 * eDv * eDv * hpB + eT * eDv * XB) * 2.0 * cs.LD;
    const double x = cs.LR * cs.LR;
    const double dLR_da = (1.0 + x) * (1.0 + x) / (x * cs.LR);
    // totals with respect to L_TF, L_D, eta_D (direct NR part + through L_R)
    const double tLTF = dLTF + dLR * dLR_da * da_dLTF;
    const double tLD = dLD + dLR * dLR_da * da_dLD;
    const double teD = deD + dLR * dLR_da * da_deD;
    // d(L_TF, L_D, eta_D)/d theta
    double dLD_dth[5] = {0, 0, 0, 0, 0};
    if (cs.Zs == 0.0) {
        // no path through L_D (see cell_screen)
    } else if (cs.debye) {
        dLD_dth[0] = -0.5 * cs.LD / cs.n_i;
        dLD_dth[1] = 0.5 * cs.LD / cs.T_e;
        dLD_dth[2] = -0.5 * cs.LD * (2.0 * cs.Zs + 1.0) / (cs.Zs * (cs.Zs + 1.0));
    } else {
        dLD_dth[0] = -cs.LD / (3.0 * cs.n_i);
    }
    if (cs.Zs != 0.0) dLD_dth[4] = cs.LD / cs.sD;
    const double dLTF_dsTF = cs.LTF / cs.sTF;
    const double deD_dZs = 1.0 / a.Z;
    const double scale = cs.n_i * C0;
    double gp[5];
    gp[0] = scale * tLD * dLD_dth[0] + (g0 * R + g1 * Rp + g2 * P) / cs.n_i;
    gp[1] = scale * tLD * dLD_dth[1];
    gp[2] = scale * (tLD * dLD_dth[2] + teD * deD_dZs);
    gp[3] = scale * tLTF * dLTF_dsTF;
    gp[4] = scale * tLD * dLD_dth[4];
    for (int k = 0; k < 5; ++k) a.out[5 * (size_t)c + k] = (float)gp[k];
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= n; ++l) {
                const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

int launch(pcc_ctx* ctx, bool grad, int n_cells, int n_samples, int Z, int n_quad, const float* params,
           const float* gamma, const float* w, const float* grad_out, float* out, void* stream, const char* name)
{
    if (!ctx || n_cells < 1 || n_samples < 0 || Z < 1 || Z > 100 || n_quad < 2 || n_quad > kMaxQuad || !params ||
        !out || (n_samples > 0 && (!gamma || !w)) || (grad && !grad_out)) {
        set_error(std::string(name) + ": invalid argument");
        return PCC_E_INVALID;
    }
    EmArgs a{};
    a.n_cells = n_cells;
    a.n_samples = n_samples;
    a.Z = Z;
    a.n_quad = n_quad;
    a.fC = coulomb_fc(Z);
    a.params = params;
    a.gamma = gamma;
    a.w = w;
    a.grad_out = grad_out;
    a.out = out;
    a.st = ctx->stats;
    std::vector<double> gx, gw;
    gauss_legendre(n_quad, gx, gw);
    const double lo = std::log(1e-7), hi = 0.0, mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
    for (int q = 0; q < n_quad; ++q) {
        a.lx[q] = (float)(mid + half * gx[q]);
        a.hw[q] = (float)(half * gw[q]);
    }
    const int rc = ensure_scratch(ctx, (size_t)n_cells * sizeof(CellScreen));
    if (rc) return rc;
    CellScreen* screen = static_cast<CellScreen*>(ctx->scratch);
    a.screen = screen;
    cudaStream_t st = (cudaStream_t)stream;
    screen_kernel<<<(n_cells + 127) / 128, 128, 0, st>>>(params, n_cells, Z, screen);
    if (grad) emission_kernel<true><<<n_cells, kEmThreads, 0, st>>>(a);
    else emission_kernel<false><<<n_cells, kEmThreads, 0, st>>>(a);
    note_launches(2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCC_OK : cuda_fail(e, name);
}

}  // namespace

extern "C" int pcc_expected_emission_fwd(pcc_ctx* ctx, int n_cells, int n_samples, int Z, int n_quad,
                                         const float* params, const float* gamma, const float* w, float* out,
                                         void* stream)
{
    return launch(ctx, false, n_cells, n_samples, Z, n_quad, params, gamma, w, nullptr, out, stream,
                  "pcc_expected_emission_fwd");
}

extern "C" int pcc_expected_emission_bwd(pcc_ctx* ctx, int n_cells, int n_samples, int Z, int n_quad,
                                         const float* params, const float* gamma, const float* w,
                                         const float* grad_out, float* grad_params, void* stream)
{
    return launch(ctx, true, n_cells, n_samples, Z, n_quad, params, gamma, w, grad_out, grad_params, stream,
                  "pcc_expected_emission_bwd");
}
