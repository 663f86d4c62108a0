// Cross sections of Sec. II evaluated on the device (FP64 for the table
// build; sigma_T also in the collision precision).
#pragma once

#include "pcc_device.cuh"

namespace pcc {

// Screening of one material (lengths in units of hbar/(m_e c)).
struct Screen {
    double LTF, LD, etaTF, etaD, ITFD, LR, fC, Z;
};
constexpr int kScreenFields = 8;

__device__ __forceinline__ Screen load_screen(const double* p)
{
    Screen s;
    s.LTF = p[0]; s.LD = p[1]; s.etaTF = p[2]; s.etaD = p[3];
    s.ITFD = p[4]; s.LR = p[5]; s.fC = p[6]; s.Z = p[7];
    return s;
}

// ---- Sec. II.A -------------------------------------------------------------

// Lambert W on the principal branch for z in [-1/e, 0): Halley iteration from
// the branch-point expansion (p = sqrt(2(e z + 1))) or from z(1 - z).
__device__ inline double lambert_w0_neg(double z)
{
    const double e = 2.718281828459045;
    const double p2 = 2.0 * (e * z + 1.0);
    double w;
    if (p2 < 1.0) {
        const double p = sqrt(fmax(p2, 0.0));
        w = -1.0 + p * (1.0 + p * (-1.0 / 3.0 + p * (11.0 / 72.0)));
    } else {
        w = z - z * z;
    }
    for (int i = 0; i < 64; ++i) {
        const double ew = exp(w);
        const double f = w * ew - z;
        const double w1 = w + 1.0;
        if (w1 == 0.0) break;
        const double step = f / (ew * w1 - 0.5 * (w + 2.0) * f / w1);
        w -= step;
        if (fabs(step) <= 1e-16 * (1.0 + fabs(w))) break;
    }
    return w;
}

// sum_{n>=2} n^-s, summed downward to n = 2000 plus the Euler-Maclaurin tail.
__host__ __device__ inline double zeta_tail(double s)
{
    double acc = 0.0;
    for (int n = 2000; n >= 2; --n) acc += exp(-s * log((double)n));
    const double N = 2000.0;
    return acc + exp((1.0 - s) * log(N)) / (s - 1.0) - 0.5 * exp(-s * log(N)) + s / 12.0 * exp((-s - 1.0) * log(N));
}

// Coulomb correction: a^2 [1/(1+a^2) + sum_{n=0}^{3} (-a^2)^n (zeta(2n+3) - 1)].
__host__ __device__ inline double coulomb_fc(int Z)
{
    const double a2 = (kAlpha * Z) * (kAlpha * Z);
    double s = 0.0, p = 1.0;
    for (int n = 0; n < 4; ++n) {
        s += p * zeta_tail(2.0 * n + 3.0);
        p *= -a2;
    }
    return a2 * (1.0 / (1.0 + a2) + s);
}

// (B ln(1+A) - A ln(1+B)) / (B - A), by its midpoint limit when A ~ B.
__device__ __forceinline__ double tfd_cross(double A, double B)
{
    const double d = B - A;
    if (fabs(d) <= 1e-6 * fmax(A, B)) {
        const double M = 0.5 * (A + B);
        return log1p(M) - M / (1.0 + M);
    }
    return (B * log1p(A) - A * log1p(B)) / d;
}

// Eq. (ITFD).
__device__ __forceinline__ double i_tfd(double eTF, double LTF, double eD, double LD)
{
    const double A = LTF * LTF, B = LD * LD;
    const double hA = ((1.0 + A) * log1p(A) - A) / (1.0 + A);
    const double hB = ((1.0 + B) * log1p(B) - B) / (1.0 + B);
    return 0.5 * eTF * eTF * hA + 0.5 * eD * eD * hB + eTF * eD * tfd_cross(A, B);
}

__device__ inline Screen screen_from_material(const pcc_material& m)
{
    Screen s;
    s.Z = m.Z;
    s.LTF = m.s_TF * exp(-log((double)m.Z) / 3.0) / kAlpha;
    const double ri = cbrt(3.0 / (4.0 * kPi * m.n_i));
    double lam = 0.0;
    if (m.Zstar > 0.0) lam = sqrt(kEps0 * m.T_e / (kQe * m.n_i * m.Zstar * (m.Zstar + 1.0)));
    s.LD = m.s_D * fmax(lam, ri) / kRc;
    s.etaD = m.Zstar / m.Z;
    s.etaTF = 1.0 - s.etaD;
    s.ITFD = i_tfd(s.etaTF, s.LTF, s.etaD, s.LD);
    const double w = lambert_w0_neg(-exp(-1.0 - 2.0 * s.ITFD));
    s.LR = sqrt(expm1(w + 1.0 + 2.0 * s.ITFD));
    s.fC = coulomb_fc(m.Z);
    return s;
}

// ---- Sec. II.B -------------------------------------------------------------

// Eq. (deriv_I1).
__device__ __forceinline__ double yukawa_I1(double d, double L)
{
    const double L2 = L * L;
    return L * d * (atan(L * d) - atan(L)) - 0.5 * L2 * (1.0 - d) * (1.0 - d) / (1.0 + L2) +
           0.5 * log((1.0 + L2) / (1.0 + L2 * d * d));
}

// Eq. (deriv_I2).
__device__ __forceinline__ double yukawa_I2(double d, double L)
{
    const double L2 = L * L, d2 = d * d;
    const double t = 4.0 * L2 * L * d2 * d * (atan(L * d) - atan(L)) +
                     (1.0 + 3.0 * L2 * d2) * log((1.0 + L2) / (1.0 + L2 * d2)) +
                     6.0 * L2 * L2 * d2 / (1.0 + L2) * log(d) +
                     L2 * (d - 1.0) * (d + 1.0 - 4.0 * L2 * d2) / (1.0 + L2);
    return 0.5 * t;
}

// g of Eq. (cs_br_nr).
__device__ __forceinline__ double nr_g(double qp, double qm, double eta, double L)
{
    const double L2 = L * L;
    const double Dp = 1.0 + qp * qp * L2, Dm = 1.0 + qm * qm * L2;
    return 0.5 * eta * eta * (log1p((qp * qp - qm * qm) * L2 / Dm) + 1.0 / Dp - 1.0 / Dm);
}

// Gamma_c of Eq. (cs_br_nr).
__device__ __forceinline__ double nr_coupling(double qp, double qm, const Screen& s)
{
    const double A = s.LTF * s.LTF, B = s.LD * s.LD;
    const double d = B - A;
    if (fabs(d) <= 1e-6 * fmax(A, B)) {
        const double M = 0.5 * (A + B);
        const double Mp = 1.0 + qp * qp * M, Mm = 1.0 + qm * qm * M;
        return s.etaTF * s.etaD * (log(Mp / Mm) + 1.0 / Mp - 1.0 / Mm);
    }
    const double Tp = 1.0 + qp * qp * A, Tm = 1.0 + qm * qm * A;
    const double Dp = 1.0 + qp * qp * B, Dm = 1.0 + qm * qm * B;
    return s.etaTF * s.etaD / d * (A * log(Dm / Dp) + B * log(Tp / Tm));
}

// Eq. (cs_br_nr) times f_E, 1 < gamma1 <= 2.
__device__ inline double dsdk_nonrel(const Screen& s, double g1, double k, int printed)
{
    const double T1 = g1 - 1.0;
    if (!(k > 0.0 && k < T1)) return 0.0;
    const double T2 = T1 - k;
    const double p1 = sqrt(T1 * (T1 + 2.0)), p2 = sqrt(T2 * (T2 + 2.0));
    double qp, qm;
    if (printed) {
        qp = 2.0 * p1 - k;
        qm = k;
    } else {
        qp = p1 + p2;
        qm = k * (T1 + T2 + 2.0) / (p1 + p2);
    }
    const double br = nr_g(qp, qm, s.etaTF, s.LTF) + nr_g(qp, qm, s.etaD, s.LD) + nr_coupling(qp, qm, s);
    const double born = 16.0 * kRe * kRe * s.Z * s.Z * kAlpha / (3.0 * k * p1 * p1) * br;
    const double b1 = p1 / g1, b2 = p2 / (1.0 + T2);
    const double a = 2.0 * kPi * s.Z * kAlpha;
    return born * (b1 / b2) * expm1(-a / b1) / expm1(-a / b2);
}

// delta of Eq. (csre): the minimum momentum transfer k / (2 gamma1 gamma2).
__device__ __forceinline__ double brems_delta(double g1, double k) { return k / (2.0 * g1 * (g1 - k)); }

// Eq. (csre) with fc = 0, Eq. (csur) with fc = f_C, for the screening
// functions I1, I2 at delta = brems_delta(g1, k).
__device__ inline double dsdk_relativistic_I(const Screen& s, double g1, double k, double fc, double I1, double I2)
{
    if (!(k > 0.0 && k < g1 - 1.0)) return 0.0;
    const double eps = (g1 - k) / g1;
    const double v = 4.0 * s.Z * s.Z * kRe * kRe * kAlpha / k *
                     ((1.0 + eps * eps) * (I1 + 1.0 - fc) - (2.0 / 3.0) * eps * (I2 + 5.0 / 6.0 - fc));
    return fmax(v, 0.0);
}

// The same with the reduced single-Yukawa potential at L = L_R.
__device__ inline double dsdk_relativistic(const Screen& s, double g1, double k, double fc)
{
    const double d = brems_delta(g1, k);
    return dsdk_relativistic_I(s, g1, k, fc, yukawa_I1(d, s.LR), yukawa_I2(d, s.LR));
}

__device__ __forceinline__ double dsdk_brems(const Screen& s, double g1, double k, int printed)
{
    if (g1 <= 2.0) return dsdk_nonrel(s, g1, k, printed);
    return dsdk_relativistic(s, g1, k, g1 <= 100.0 ? 0.0 : s.fC);
}

// ---- Sec. II.C-D -----------------------------------------------------------

// Eq. (dsdkbh) for the screening functions I1, I2 at delta = k / (2 gamma+ gamma-).
__device__ inline double dsdg_bethe_heitler_I(const Screen& s, double k, double gp, double I1, double I2)
{
    const double gm = k - gp;
    if (!(gp > 1.0 && gm > 1.0)) return 0.0;
    const double v = 4.0 * s.Z * s.Z * kRe * kRe * kAlpha / (k * k * k) *
                     ((gp * gp + gm * gm) * (I1 + 1.0) + (2.0 / 3.0) * gp * gm * (I2 + 5.0 / 6.0));
    return fmax(v, 0.0);
}

// The same with the reduced single-Yukawa potential at L = L_R.
__device__ inline double dsdg_bethe_heitler(const Screen& s, double k, double gp)
{
    const double d = k / (2.0 * gp * (k - gp));
    return dsdg_bethe_heitler_I(s, k, gp, yukawa_I1(d, s.LR), yukawa_I2(d, s.LR));
}

// Gryaznykh fit of the total Trident cross section, zero below gamma1 = 3.
template <typename T>
__device__ __forceinline__ T sigma_trident(T Z, T g1)
{
    if (g1 < (T)3) return (T)0;
    const T l = log((g1 + (T)4.5) / (T)6.89);
    return (T)5.22e-34 * Z * Z * l * l * l;
}

// Pair-energy shape (Z = 1): product over sum of the Bhabha NR and
// relativistic forms.
__device__ inline double trident_pair_shape(double g1, double gp)
{
    if (!(gp > 2.0 && gp < g1 - 1.0)) return 0.0;
    const double pre = (kRe * kAlpha) * (kRe * kAlpha);
    const double x2 = 1.0 / (g1 * g1);
    const double q = x2 / (1.0 - x2);
    const double L = -log(x2);
    const double x4 = x2 * x2, x6 = x4 * x2, x8 = x4 * x4;
    const double C = 4.0 * q * L - (4.0 / 3.0) * x2 + x4 / 6.0;
    const double Cz = 3.0 * q * (1.0 - q * L) - 2.6 * x2 + 1.75 * x4 - 0.9 * x6 + 0.2 * x8;
    const double Cr = -1.5 * q * (1.0 - q * L) + 0.8 * x2 - 0.125 * x4 - 0.05 * x6 + 0.025 * x8;
    const double Ek = gp - 2.0;
    const double nr = pre / 32.0 * (2.0 * log(g1) - 161.0 / 60.0 + C + Cr + Cz) * Ek * Ek * Ek;
    const double r = 56.0 / (9.0 * kPi) * pre * log(gp) * log(g1 / gp) / gp;
    if (!(nr > 0.0 && r > 0.0)) return 0.0;
    return nr * r / (nr + r);
}

// Positron-energy shape at pair energy gp, clamped at zero.
__device__ __forceinline__ double trident_split_shape(double gp, double gplus)
{
    const double gm = gp - gplus;
    if (!(gplus > 1.0 && gm > 1.0)) return 0.0;
    const double v = (gplus * gplus + gm * gm + (2.0 / 3.0) * gplus * gm) * log(gplus * gm / gp);
    return fmax(v, 0.0);
}

}  // namespace pcc
