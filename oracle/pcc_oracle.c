/*
 * FP64 CPU oracle for arXiv:1907.02814 (Martinez et al.), the pairwise
 * Monte Carlo Bremsstrahlung / Bethe-Heitler / Trident collision step.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It is written
 * from the paper, in the paper's order and notation, with no blocking,
 * fusion or reordering; see pcc_oracle.h for the pin status of each part.
 *
 * Readings of the paper where it is silent, garbled or ambiguous:
 *   R1  NR momentum-transfer bounds: exact p1 +/- p2 by default; the
 *       printed 2 p1 - k and k are selectable (Sec. II.B.1).
 *   R2  f_C: a^2 [1/(1+a^2) + sum_{n=0..3} (-a^2)^n (zeta(2n+3) - 1)],
 *       a = alpha Z (the printed series has a divergent n=0 term).
 *   R5  the Brems cut-off interval is in x = k/(gamma-1), x in [1e-7, 1].
 *   R6  regimes: NR gamma<=2, relativistic 2<gamma<=100, UR gamma>100.
 *   R7  the frame transform's last factor is the ion velocity.
 *   R8  BH probability: gamma_e -> k, gamma'_e -> k', v'_e -> c.
 *   R10 inverse-CDF sampling: stochastic row pick, binary search, linear
 *       interpolation in the column's spacing variable.
 *   R11 Trident shapes: natural logs, E_p = gamma_p - 2 in the NR form and
 *       gamma_p in the relativistic form, the split shape clamped at 0 and
 *       a uniform split where the clamped shape vanishes (gamma_p <= 4).
 *   R12 sigma_T = 0 below the pair threshold gamma_1 = 3.
 *   Pairing: only the larger list is permuted; Brems and Trident share the
 *       electron-ion pairing of the step; random numbers from Philox4x32-10
 *       with the counter layout documented at orc_step().
 */
#include "pcc_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 */
static const double ALPHA = 7.2973525693e-3;        /* fine-structure constant      */
static const double R_E = 2.8179403262e-15;          /* classical electron radius, m */
static const double R_C = 3.8615926796e-13;          /* hbar/(m_e c), m              */
static const double C_LIGHT = 299792458.0;           /* m/s                          */
static const double EPS0 = 8.8541878128e-12;         /* F/m                          */
static const double Q_E = 1.602176634e-19;           /* C                            */
static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Sec. II.A: screening lengths and the Thomas-Fermi-Debye potential         */
/* ------------------------------------------------------------------------ */

/* Principal branch W0 of the Lambert function, by Halley iteration
 * (Corless, Gonnet, Hare, Jeffrey, Knuth, Adv. Comput. Math. 5, 329 (1996)),
 * started from the branch-point series near -1/e and from z(1-z) or
 * log1p(z) elsewhere. */
double orc_lambert_w0(double z)
{
    const double inv_e = 0.36787944117144233;
    if (z < -inv_e) return NAN;
    if (z == 0.0) return 0.0;
    double w;
    double p2 = 2.0 * (2.718281828459045 * z + 1.0);
    if (z < 0.0 && p2 < 1.0) {
        double p = sqrt(p2 > 0.0 ? p2 : 0.0);
        w = -1.0 + p - p * p / 3.0 + 11.0 / 72.0 * p * p * p;
    } else if (z < 0.0) {
        w = z * (1.0 - z);
    } else {
        w = log1p(z);
    }
    for (int it = 0; it < 64; ++it) {
        double ew = exp(w);
        double f = w * ew - z;
        double wp1 = w + 1.0;
        if (wp1 == 0.0) break;
        double d = ew * wp1 - (w + 2.0) * f / (2.0 * wp1);
        double dw = f / d;
        w -= dw;
        if (fabs(dw) <= 1e-16 * (1.0 + fabs(w))) break;
    }
    return w;
}

/* Riemann zeta(s) - 1 by direct summation with an Euler-Maclaurin tail. */
static double zeta_minus_one(double s)
{
    const int N = 2000;
    double sum = 0.0;
    for (int n = N; n >= 2; --n) sum += pow((double)n, -s);
    double tail = pow((double)N, 1.0 - s) / (s - 1.0) - 0.5 * pow((double)N, -s)
                + s / 12.0 * pow((double)N, -s - 1.0);
    return sum + tail;
}

/* Coulomb correction f_C(Z) of the ultra-relativistic Brems formula
 * (Sec. II.B.3), four terms of the zeta series as the paper says.  The
 * printed series starts at zeta(1), which diverges; it is read as the
 * Davies-Bethe-Maximon form a^2 [1/(1+a^2) + sum_{n=0..3} (-a^2)^n
 * (zeta(2n+3) - 1)], a = alpha Z. */
double orc_fC(int Z)
{
    double a2 = (ALPHA * Z) * (ALPHA * Z);
    double series = 0.0, pw = 1.0;
    for (int n = 0; n < 4; ++n) {
        series += pw * zeta_minus_one(2.0 * n + 3.0);
        pw *= -a2;
    }
    return a2 * (1.0 / (1.0 + a2) + series);
}

/* (A_D ln(1+A_TF) - A_TF ln(1+A_D)) / (A_D - A_TF), the cross term of
 * Eq. (ITFD); for nearly equal arguments its limit at the midpoint,
 * ln(1+A) - A/(1+A), which it equals to second order. */
static double cross_term(double A_TF, double A_D)
{
    double d = A_D - A_TF, s = fmax(A_D, A_TF);
    if (fabs(d) <= 1e-6 * s) {
        double A = 0.5 * (A_D + A_TF);
        return log1p(A) - A / (1.0 + A);
    }
    return (A_D * log1p(A_TF) - A_TF * log1p(A_D)) / d;
}

/* Eq. (ITFD): the delta -> 0 limit of I1 and I2 for the two-Yukawa
 * potential, with eta = q/q_total weights and lengths in units of r_C. */
double orc_I_tfd(double etaTF, double LTF, double etaD, double LD)
{
    double A = LTF * LTF, B = LD * LD;
    double t1 = 0.5 * etaTF * etaTF * ((1.0 + A) * log1p(A) - A) / (1.0 + A);
    double t2 = 0.5 * etaD * etaD * ((1.0 + B) * log1p(B) - B) / (1.0 + B);
    double t3 = etaTF * etaD * cross_term(A, B);
    return t1 + t2 + t3;
}

/* Eq. (LTF), Eq. (LDH) with the lower bound r_i, Eq. (V_TFD) weights,
 * Eq. (ITFD), Eq. (reduit)/(lambert-W) and f_C. */
void orc_screening_prep(const orc_material *m, orc_screening *o)
{
    memset(o, 0, sizeof *o);
    o->Z = m->Z;
    o->Zstar = m->Zstar;
    /* L_TF = a0 Z^-1/3 with a0 = r_C / alpha */
    o->LTF = m->s_TF * pow((double)m->Z, -1.0 / 3.0) / ALPHA;
    o->ri = cbrt(3.0 / (4.0 * PI * m->n_i));
    if (m->Zstar > 0.0)
        o->lambdaD = sqrt(EPS0 * m->T_e / (Q_E * m->n_i * m->Zstar * (m->Zstar + 1.0)));
    else
        o->lambdaD = 0.0;
    o->LD = m->s_D * fmax(o->lambdaD, o->ri) / R_C;
    o->etaTF = 1.0 - m->Zstar / m->Z;
    o->etaD = m->Zstar / m->Z;
    o->ITFD = orc_I_tfd(o->etaTF, o->LTF, o->etaD, o->LD);
    double a = o->ITFD;
    double W = orc_lambert_w0(-exp(-1.0 - 2.0 * a));
    double x = expm1(W + 1.0 + 2.0 * a);
    o->LR = sqrt(x);
    o->fC = orc_fC(m->Z);
}

/* ------------------------------------------------------------------------ */
/* Sec. II.B: Bremsstrahlung cross sections                                  */
/* ------------------------------------------------------------------------ */

/* Eq. (deriv_I1): I1(delta) for a single Yukawa potential of length L. */
double orc_I1_yukawa(double d, double L)
{
    double L2 = L * L;
    return L * d * (atan(d * L) - atan(L))
         - 0.5 * L2 * (1.0 - d) * (1.0 - d) / (1.0 + L2)
         + 0.5 * log((1.0 + L2) / (1.0 + L2 * d * d));
}

/* Eq. (deriv_I2): I2(delta) for a single Yukawa potential of length L. */
double orc_I2_yukawa(double d, double L)
{
    double L2 = L * L, d2 = d * d;
    double two_I2 = 4.0 * L2 * L * d2 * d * (atan(L * d) - atan(L))
                  + (1.0 + 3.0 * L2 * d2) * log((1.0 + L2) / (1.0 + L2 * d2))
                  + 6.0 * L2 * L2 * d2 / (1.0 + L2) * log(d)
                  + L2 * (d - 1.0) * (d + 1.0 - 4.0 * L2 * d2) / (1.0 + L2);
    return 0.5 * two_I2;
}

/* Eq. (defF) for the potential of Eq. (V_TFD): the Fourier transform of each
 * Yukawa term (q_i/r) exp(-r/L_i) gives 1 - F = (L_i u)^2 / (1 + (L_i u)^2)
 * for its charge fraction, so 1 - F(u) is their sum weighted by
 * eta_i = q_i/q (u in units of m_e c, lengths in units of r_C). */
static double one_minus_F_tfd(const orc_screening *s, double u)
{
    double a = s->LTF * u, b = s->LD * u;
    return s->etaTF * a * a / (1.0 + a * a) + s->etaD * b * b / (1.0 + b * b);
}

/* Eqs. (defphi1) and (defphi2) with the form factor of the full
 * Thomas-Fermi-Debye potential, by quadrature in t = ln u over
 * [ln delta, 0]: composite 8-point Gauss-Legendre on equal panels no wider
 * than 1/2 (the form factor changes over about one unit of ln u around
 * u = 1/L_TF and u = 1/L_D).  With r = u/delta the integrands are
 *   I1: (u - delta)^2 / u^3 du = (1 - 1/r)^2 dt,
 *   I2: [u^3 - 6 delta^2 u ln(u/delta) + 3 delta^2 u - 4 delta^3] / u^4 du
 *       = (1 + (3 - 6 ln r)/r^2 - 4/r^3) dt,
 * each times (1 - F(u))^2.  Zero for delta >= 1 (empty range). */
void orc_I12_tfd_quad(const orc_screening *s, double delta, double *I1, double *I2)
{
    double gx[8], gw[8];
    orc_gauss_legendre(8, gx, gw);
    *I1 = 0.0;
    *I2 = 0.0;
    if (!(delta > 0.0 && delta < 1.0)) return;
    double t0 = log(delta);
    int n = (int)ceil(-t0 / 0.5);
    double h = -t0 / n;
    double s1 = 0.0, s2 = 0.0;
    for (int p = 0; p < n; ++p) {
        double mid = t0 + (p + 0.5) * h;
        for (int q = 0; q < 8; ++q) {
            double t = mid + 0.5 * h * gx[q];
            double lr = t - t0;                 /* ln r */
            double r = exp(lr);
            double f = one_minus_F_tfd(s, exp(t));
            double f2 = f * f;
            double a = -expm1(-lr);             /* 1 - 1/r */
            s1 += gw[q] * a * a * f2;
            s2 += gw[q] * (1.0 + (3.0 - 6.0 * lr) / (r * r) - 4.0 / (r * r * r)) * f2;
        }
    }
    *I1 = 0.5 * h * s1;
    *I2 = 0.5 * h * s2;
}

/* I1, I2 of the material's screening mode: the reduced single-Yukawa
 * potential at L_R (Sec. II.B.2), or the full TFD potential by quadrature. */
static void screening_I12(const orc_screening *s, double delta, double *I1, double *I2)
{
    if (s->tfd_quad) {
        orc_I12_tfd_quad(s, delta, I1, I2);
    } else {
        *I1 = orc_I1_yukawa(delta, s->LR);
        *I2 = orc_I2_yukawa(delta, s->LR);
    }
}

/* g(dp+, dp-, eta, L) of Eq. (cs_br_nr). */
static double g_nr(double dpp, double dpm, double eta, double L)
{
    double L2 = L * L;
    double Dp = dpp * dpp * L2 + 1.0, Dm = dpm * dpm * L2 + 1.0;
    double lr = log1p((dpp * dpp - dpm * dpm) * L2 / Dm);
    return 0.5 * eta * eta * (lr + 1.0 / Dp - 1.0 / Dm);
}

/* Gamma_c of Eq. (cs_br_nr), with the midpoint limit for L_D ~ L_TF. */
static double gamma_c_nr(double dpp, double dpm, double etaTF, double LTF, double etaD, double LD)
{
    double A = LTF * LTF, B = LD * LD;
    double Tp = dpp * dpp * A + 1.0, Tm = dpm * dpm * A + 1.0;
    double Dp = dpp * dpp * B + 1.0, Dm = dpm * dpm * B + 1.0;
    double d = B - A;
    if (fabs(d) <= 1e-6 * fmax(A, B)) {
        double M = 0.5 * (A + B);
        double Mp = dpp * dpp * M + 1.0, Mm = dpm * dpm * M + 1.0;
        return etaTF * etaD * (log(Mp / Mm) + 1.0 / Mp - 1.0 / Mm);
    }
    return etaTF * etaD / d * (A * log(Dm / Dp) + B * log(Tp / Tm));
}

/* Eq. (cs_br_nr) times the Elwert factor f_E: NR Brems, 1 < gamma1 <= 2. */
double orc_dsdk_brems_nr(const orc_screening *s, double gamma1, double k, int nr_qbounds)
{
    double T1 = gamma1 - 1.0;
    if (!(k > 0.0 && k < T1)) return 0.0;
    double T2 = T1 - k;
    double p1 = sqrt(T1 * (T1 + 2.0)), p2 = sqrt(T2 * (T2 + 2.0));
    double dpp, dpm;
    if (nr_qbounds == ORC_NR_PRINTED) {
        dpp = 2.0 * p1 - k;
        dpm = k;
    } else {
        dpp = p1 + p2;
        dpm = k * (T1 + T2 + 2.0) / (p1 + p2);   /* = p1 - p2 */
    }
    double Z = s->Z;
    double bracket = g_nr(dpp, dpm, s->etaTF, s->LTF) + g_nr(dpp, dpm, s->etaD, s->LD)
                   + gamma_c_nr(dpp, dpm, s->etaTF, s->LTF, s->etaD, s->LD);
    double born = 16.0 * R_E * R_E * Z * Z * ALPHA / (3.0 * k * p1 * p1) * bracket;
    double b1 = p1 / gamma1, b2 = p2 / (1.0 + T2);
    double a = 2.0 * PI * Z * ALPHA;
    double fE = (b1 / b2) * (-expm1(-a / b1)) / (-expm1(-a / b2));
    return born * fE;
}

/* Eq. (csre) (fc = 0) and Eq. (csur) (fc = f_C): relativistic Brems with the
 * screening functions of the material's mode (reduced single Yukawa at
 * L = L_R, or the full TFD potential by quadrature). */
double orc_dsdk_brems_rel(const orc_screening *s, double gamma1, double k, double fc)
{
    if (!(k > 0.0 && k < gamma1 - 1.0)) return 0.0;
    double eps = (gamma1 - k) / gamma1;
    double delta = k / (2.0 * gamma1 * (gamma1 - k));
    double I1, I2;
    screening_I12(s, delta, &I1, &I2);
    double Z = s->Z;
    double v = 4.0 * Z * Z * R_E * R_E * ALPHA / k
             * ((1.0 + eps * eps) * (I1 + 1.0 - fc) - 2.0 / 3.0 * eps * (I2 + 5.0 / 6.0 - fc));
    return v > 0.0 ? v : 0.0;
}

/* dsigma/dk in the ion rest frame, regime chosen by gamma1: the
 * non-relativistic form up to 2, the relativistic one up to 100, the
 * ultra-relativistic one above (the paper's ranges share their end points;
 * the jumps there are kept). */
double orc_dsdk_brems(const orc_screening *s, double gamma1, double k, int nr_qbounds)
{
    if (gamma1 <= 2.0) return orc_dsdk_brems_nr(s, gamma1, k, nr_qbounds);
    if (gamma1 <= 100.0) return orc_dsdk_brems_rel(s, gamma1, k, 0.0);
    return orc_dsdk_brems_rel(s, gamma1, k, s->fC);
}

/* ------------------------------------------------------------------------ */
/* Sec. II.C-D: pair production                                               */
/* ------------------------------------------------------------------------ */

/* Eq. (dsdkbh): Bethe-Heitler cross section differential in gamma_+. */
double orc_dsdg_bh(const orc_screening *s, double k, double gp)
{
    double gm = k - gp;
    if (!(gp > 1.0 && gm > 1.0)) return 0.0;
    double delta = k / (2.0 * gp * gm);
    double I1, I2;
    screening_I12(s, delta, &I1, &I2);
    double Z = s->Z;
    double v = 4.0 * Z * Z * R_E * R_E * ALPHA / (k * k * k)
             * ((gp * gp + gm * gm) * (I1 + 1.0) + 2.0 / 3.0 * gp * gm * (I2 + 5.0 / 6.0));
    return v > 0.0 ? v : 0.0;
}

/* Sec. II.D: Gryaznykh fit of the total Trident cross section, zero below
 * the pair threshold gamma1 = 3 (the fit itself turns negative below 2.39). */
double orc_sigma_trident(int Z, double g1)
{
    if (g1 < 3.0) return 0.0;
    double l = log((g1 + 4.50) / 6.89);
    return 5.22 * (double)Z * Z * l * l * l * 1e-34;
}

/* Sec. II.D: Bhabha low- and high-energy pair-energy spectra combined by
 * the product-over-sum interpolation.  Logs are natural; E_p is the pair's
 * kinetic energy gamma_p - 2 in the low-energy form, so that the spectrum
 * vanishes at threshold, and gamma_p in the high-energy form. */
double orc_dsdgp_trident(int Z, double g1, double gp)
{
    if (!(gp > 2.0 && gp < g1 - 1.0)) return 0.0;
    double pre = (Z * R_E * ALPHA) * (Z * R_E * ALPHA);
    double x2 = 1.0 / (g1 * g1);
    double q = x2 / (1.0 - x2);
    double L = log(1.0 / x2);
    double C = 4.0 * q * L - 4.0 / 3.0 * x2 + x2 * x2 / 6.0;
    double Cz = 3.0 * q * (1.0 - q * L) - 13.0 / 5.0 * x2 + 7.0 / 4.0 * x2 * x2
              - 9.0 / 10.0 * x2 * x2 * x2 + x2 * x2 * x2 * x2 / 5.0;
    double Cr = -1.5 * q * (1.0 - q * L) + 4.0 / 5.0 * x2 - x2 * x2 / 8.0
              - x2 * x2 * x2 / 20.0 + x2 * x2 * x2 * x2 / 40.0;
    double Ep = gp - 2.0;
    double nr = pre / 32.0 * (log(g1 * g1) - 161.0 / 60.0 + C + Cr + Cz) * Ep * Ep * Ep;
    double r = 56.0 / (9.0 * PI) * pre * log(gp) * log(g1 / gp) / gp;
    if (!(nr > 0.0 && r > 0.0)) return 0.0;
    return nr * r / (nr + r);
}

/* Sec. II.D: shape of the positron energy at fixed pair energy, clamped. */
double orc_split_shape(double gp, double gplus)
{
    double gm = gp - gplus;
    if (!(gplus > 1.0 && gm > 1.0)) return 0.0;
    double v = (gplus * gplus + gm * gm + 2.0 / 3.0 * gplus * gm) * log(gplus * gm / gp);
    return v > 0.0 ? v : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Quadrature and tables                                                     */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n. */
void orc_gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= n; ++l) {
                double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

enum { TB_BREMS = 0, TB_BH = 1, TB_TRI_GP = 2, TB_TRI_SPLIT = 3 };

/* Row grid: the row variable (Brems gamma-1, BH k-2, Trident gamma1-3,
 * split gamma_p-2) log-spaced on [T_min, T_max]. */
double orc_row_value(const orc_table_spec *sp, int r)
{
    return sp->T_min * pow(sp->T_max / sp->T_min, (double)r / (sp->n_rows - 1));
}

static int col_is_log(int table) { return table == TB_BREMS || table == TB_TRI_GP; }

static double col_ymin(const orc_table_spec *sp, int table)
{
    return table == TB_BREMS ? sp->x_min : sp->tri_y_min;
}

/* Column grid value y_c: log-spaced on [y_min, 1] or linear on [0, 1]. */
double orc_col_value(const orc_table_spec *sp, int table, int c)
{
    if (col_is_log(table)) {
        double ly = log(col_ymin(sp, table));
        return exp(ly * (1.0 - (double)c / (sp->n_cols - 1)));
    }
    return (double)c / (sp->n_cols - 1);
}

/* Integrand of the cumulative distribution in the column's spacing variable
 * (ln y or y): the differential cross section times the Jacobian. */
static double cdf_integrand(const orc_tables *t, int table, int mat, double rowv, double v)
{
    const orc_table_spec *sp = &t->spec;
    if (table == TB_BREMS) {
        double x = exp(v), T = rowv;
        return orc_dsdk_brems(&t->scr[mat], 1.0 + T, x * T, sp->nr_qbounds) * T * x;
    }
    if (table == TB_BH) {
        double k = 2.0 + rowv;
        return orc_dsdg_bh(&t->scr[mat], k, 1.0 + v * rowv) * rowv;
    }
    if (table == TB_TRI_GP) {
        double y = exp(v), g1 = 3.0 + rowv;
        return orc_dsdgp_trident(1, g1, 2.0 + y * rowv) * rowv * y;
    }
    double gp = 2.0 + rowv;
    return orc_split_shape(gp, 1.0 + v * rowv) * rowv;
}

/* Q-point Gauss-Legendre on [a, b]. */
static double gl_panel(const orc_tables *t, int table, int mat, double rowv, double a, double b,
                       const double *gx, const double *gw)
{
    double h = 0.5 * (b - a), mid = 0.5 * (a + b), part = 0.0;
    for (int q = 0; q < t->spec.quad_nodes; ++q) part += gw[q] * cdf_integrand(t, table, mat, rowv, mid + h * gx[q]);
    return h * part;
}

/* Sub-panels of the outermost column intervals, graded geometrically (ratio
 * 1/4) towards the end of the range: the cross sections change over a width
 * of order 1/gamma next to the kinematic limits. */
enum { EDGE_PANELS = 12 };

static double column_integral(const orc_tables *t, int table, int mat, double rowv, double a, double b,
                              int grade_left, int grade_right, const double *gx, const double *gw)
{
    if (!grade_left && !grade_right) return gl_panel(t, table, mat, rowv, a, b, gx, gw);
    double h = b - a, sum = 0.0;
    if (grade_right) {
        double lo = a, f = 1.0;
        for (int i = 0; i < EDGE_PANELS; ++i) {
            f *= 0.25;
            double hi = b - h * f;
            sum += gl_panel(t, table, mat, rowv, lo, hi, gx, gw);
            lo = hi;
        }
        return sum + gl_panel(t, table, mat, rowv, lo, b, gx, gw);
    }
    double hi = b, f = 1.0;
    for (int i = 0; i < EDGE_PANELS; ++i) {
        f *= 0.25;
        double lo = a + h * f;
        sum += gl_panel(t, table, mat, rowv, lo, hi, gx, gw);
        hi = lo;
    }
    return sum + gl_panel(t, table, mat, rowv, a, hi, gx, gw);
}

/* One table row: cumulative integral at every column by composite
 * Gauss-Legendre on each column interval (graded sub-panels on the two
 * outermost intervals); returns the total. */
static double build_row(const orc_tables *t, int table, int mat, int r, double *cdf_row,
                        const double *gx, const double *gw)
{
    const orc_table_spec *sp = &t->spec;
    double rowv = orc_row_value(sp, r);
    int nc = sp->n_cols;
    double cum = 0.0;
    cdf_row[0] = 0.0;
    for (int c = 0; c + 1 < nc; ++c) {
        double a, b;
        if (col_is_log(table)) {
            a = log(orc_col_value(sp, table, c));
            b = log(orc_col_value(sp, table, c + 1));
        } else {
            a = orc_col_value(sp, table, c);
            b = orc_col_value(sp, table, c + 1);
        }
        int left = (c == 0) && !col_is_log(table);
        int right = (c + 2 == nc);
        cum += column_integral(t, table, mat, rowv, a, b, left, right, gx, gw);
        cdf_row[c + 1] = cum;
    }
    if (cum > 0.0) {
        for (int c = 0; c < nc; ++c) cdf_row[c] /= cum;
        cdf_row[nc - 1] = 1.0;
    } else {
        /* zero shape (split for gamma_p <= 4): uniform in the column variable */
        for (int c = 0; c < nc; ++c) cdf_row[c] = (double)c / (nc - 1);
    }
    return cum;
}

int orc_tables_build(orc_tables *t)
{
    const orc_table_spec *sp = &t->spec;
    int Q = sp->quad_nodes;
    if (Q < 1 || Q > 64 || sp->n_rows < 2 || sp->n_cols < 2) return 1;
    if (sp->screening != ORC_SCREEN_REDUCED && sp->screening != ORC_SCREEN_TFD_QUAD) return 1;
    double gx[64], gw[64];
    orc_gauss_legendre(Q, gx, gw);
    size_t R = sp->n_rows, C = sp->n_cols;
    for (int m = 0; m < t->n_mat; ++m) t->scr[m].tfd_quad = sp->screening == ORC_SCREEN_TFD_QUAD;
    for (int m = 0; m < t->n_mat; ++m) {
        for (int r = 0; r < sp->n_rows; ++r) {
            t->brems_sigma[m * R + r] = build_row(t, TB_BREMS, m, r, t->brems_cdf + (m * R + r) * C, gx, gw);
            t->bh_sigma[m * R + r] = build_row(t, TB_BH, m, r, t->bh_cdf + (m * R + r) * C, gx, gw);
        }
    }
    for (int r = 0; r < sp->n_rows; ++r) {
        build_row(t, TB_TRI_GP, 0, r, t->tri_gp_cdf + r * C, gx, gw);
        build_row(t, TB_TRI_SPLIT, 0, r, t->tri_split_cdf + r * C, gx, gw);
    }
    return 0;
}

/* Fractional row coordinate of a row variable, clamped to the grid. */
static double row_coord(const orc_table_spec *sp, double r)
{
    double t = log(r / sp->T_min) / (log(sp->T_max / sp->T_min) / (sp->n_rows - 1));
    if (!(t > 0.0)) t = 0.0;
    if (t > sp->n_rows - 1) t = sp->n_rows - 1;
    return t;
}

/* Total cross section at row variable r: log-log interpolation; 0 below the
 * table, the last row (and a status bit) above it. */
double orc_sigma_lookup(const orc_table_spec *sp, const double *sig, double r, unsigned *status)
{
    if (!(r >= sp->T_min)) return 0.0;
    double t = log(r / sp->T_min) / (log(sp->T_max / sp->T_min) / (sp->n_rows - 1));
    if (t > sp->n_rows - 1) {
        *status |= ORC_ST_TABLE_RANGE;
        return sig[sp->n_rows - 1];
    }
    int j = (int)floor(t);
    if (j > sp->n_rows - 2) j = sp->n_rows - 2;
    double f = t - j;
    return exp((1.0 - f) * log(sig[j]) + f * log(sig[j + 1]));
}

/* Inverse-CDF sample of the column variable: between the two rows around
 * r, the upper one is taken when u_row is below r's fractional log position;
 * then a binary search of that row's CDF and linear interpolation in the
 * column's spacing variable (ln y for log-spaced columns, y otherwise). */
double orc_sample(const orc_table_spec *sp, int table, const double *cdf, double r,
                  double u_row, double u_col)
{
    double t = row_coord(sp, r);
    int j = (int)floor(t);
    if (j > sp->n_rows - 2) j = sp->n_rows - 2;
    double f = t - j;
    int row = j + (u_row < f ? 1 : 0);
    const double *F = cdf + (size_t)row * sp->n_cols;
    int lo = 0, hi = sp->n_cols - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (F[mid] <= u_col) lo = mid; else hi = mid;
    }
    double frac = (u_col - F[lo]) / (F[lo + 1] - F[lo]);
    if (col_is_log(table)) {
        double ly = log(col_ymin(sp, table));
        double step = -ly / (sp->n_cols - 1);
        return exp(ly + (lo + frac) * step);
    }
    return (lo + frac) / (sp->n_cols - 1);
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)                         */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on (0, 1): (2m + 1) 2^-24 with m the top 23 bits of r, a 24-bit
 * odd integer times a power of two, so exactly representable in float. */
double orc_u01(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

/* ------------------------------------------------------------------------ */
/* Random permutation used for the pairing                                   */
/* ------------------------------------------------------------------------ */

/* 32-bit keyed mixing function (round function and sort key). */
static uint32_t mix32(uint32_t r, uint32_t k)
{
    uint32_t t = r ^ k;
    t *= 0x9E3779B1u;
    t ^= t >> 15;
    t *= 0x85EBCA77u;
    t ^= t >> 13;
    return t;
}

/* Domains of up to 32 elements: P^-1(s) is the rank of s under the sort
 * keys mix32(mix32(s, rk0), rk1), ties broken by index. */
static uint32_t small_key(uint32_t s, const uint32_t rk[4]) { return mix32(mix32(s, rk[0]), rk[1]); }

static uint32_t small_rank(uint32_t s, uint32_t n, const uint32_t rk[4])
{
    uint32_t ks = small_key(s, rk), rank = 0;
    for (uint32_t t = 0; t < n; ++t) {
        uint32_t kt = small_key(t, rk);
        if (kt < ks || (kt == ks && t < s)) ++rank;
    }
    return rank;
}

/* Larger domains: a four-round Feistel network on b = bitlen(n-1) bits,
 * halves floor(b/2) and ceil(b/2) swapping widths each round
 * (Luby-Rackoff), restricted to [0, n) by cycle walking (Black-Rogaway). */
static uint32_t feistel_enc(uint32_t v, int b, const uint32_t rk[4])
{
    int wl = b >> 1, wr = b - wl;
    uint32_t L = v >> wr, R = v & ((1u << wr) - 1u);
    for (int i = 0; i < 4; ++i) {
        uint32_t nL = R, nR = (L ^ mix32(R, rk[i])) & ((1u << wl) - 1u);
        int t = wl; wl = wr; wr = t;
        L = nL; R = nR;
    }
    return (L << wr) | R;
}

static uint32_t feistel_dec(uint32_t v, int b, const uint32_t rk[4])
{
    int wl = b >> 1, wr = b - wl;
    uint32_t L = v >> wr, R = v & ((1u << wr) - 1u);
    for (int i = 3; i >= 0; --i) {
        uint32_t oR = L, oL = (R ^ mix32(L, rk[i])) & ((1u << wr) - 1u);
        int t = wl; wl = wr; wr = t;
        L = oL; R = oR;
    }
    return (L << wr) | R;
}

static int bitlen(uint32_t v) { int b = 0; while (v) { ++b; v >>= 1; } return b; }

uint32_t orc_perm_pos(uint32_t s, uint32_t n, const uint32_t rk[4])
{
    if (n <= 1) return 0;
    if (n <= 32) return small_rank(s, n, rk);
    int b = bitlen(n - 1);
    uint32_t y = feistel_enc(s, b, rk);
    for (uint32_t it = 0; y >= n && it < (1u << b); ++it) y = feistel_enc(y, b, rk);
    return y;
}

uint32_t orc_perm_elem(uint32_t j, uint32_t n, const uint32_t rk[4])
{
    if (n <= 1) return 0;
    if (n <= 32) {
        for (uint32_t s = 0; s < n; ++s)
            if (small_rank(s, n, rk) == j) return s;
        return 0;
    }
    int b = bitlen(n - 1);
    uint32_t y = feistel_dec(j, b, rk);
    for (uint32_t it = 0; y >= n && it < (1u << b); ++it) y = feistel_dec(y, b, rk);
    return y;
}

/* ------------------------------------------------------------------------ */
/* Sec. III.A: the pairwise collision step                                   */
/* ------------------------------------------------------------------------ */

enum { G_EM = 0, G_EP = 1, G_BH = 2 };
enum { PU_PERM = 0, PU_ACCEPT = 1, PU_EVT_B = 2, PU_EVT_T1 = 3, PU_EVT_T2 = 4, PU_EVT_BH = 5, PU_ACCEPT_EXT = 6 };
enum { CH_BREMS_EM = 0, CH_BREMS_EP = 1, CH_TRI_EM = 2, CH_TRI_EP = 3, CH_BH = 4 };

static uint32_t tag(int group, int purpose, uint32_t m) { return (uint32_t)group | ((uint32_t)purpose << 4) | (m << 8); }

static void philox_at(uint32_t c0, uint32_t cell, uint64_t step, uint32_t tg, uint64_t seed, uint32_t out[4])
{
    uint32_t ctr[4] = { c0, cell, (uint32_t)step, tg };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* Where the rest of an accept uniform comes from: the draw (c0, cell, step,
 * tag) with the ACCEPT_EXT purpose, its words 0 and 1. */
typedef struct { uint32_t c0, cell; uint64_t step; uint32_t tag; uint64_t seed; } accept_src;

/* The accept decision U < p (Eq. proba3: the pair collides with probability
 * p = 1 - exp(-x)) for the uniform U = (2^48 a + e + 1/2) 2^-64, with a
 * 16-bit first digit a and a 48-bit rest e = 2^16 w0 + (w1 >> 16) taken from
 * the extension draw (words w0, w1), compared digit by digit: a settles it
 * unless a = floor(2^16 p), and only then (probability 2^-16) is e drawn.
 * Every p in [0, 1] is honoured down to 2^-64, which per-pair probabilities
 * of rare processes at small time steps need (Trident: ~1e-10 per pair at
 * the paper's 7.4e-3 fs). */
static int accept_u(uint32_t a, double p, const accept_src *src)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return 1;
    double X = ldexp(p, 16), fl = floor(X);
    if ((double)a < fl) return 1;
    if ((double)a > fl) return 0;
    uint32_t ext[4];
    philox_at(src->c0, src->cell, src->step, src->tag, src->seed, ext);
    uint64_t e = ((uint64_t)ext[0] << 16) | (ext[1] >> 16);
    return (double)e + 0.5 < ldexp(X - fl, 48);
}

int orc_accept(uint32_t a, double p, uint32_t c0, uint32_t cell, uint64_t step, uint32_t tg, uint64_t seed)
{
    accept_src src = { c0, cell, step, tg, seed };
    return accept_u(a, p, &src);
}

/* Identifier of a secondary: marker bit, step, channel, cell, pair, slot. */
static uint64_t secondary_pid(uint64_t step, int ch, uint32_t cell, uint32_t j, int sub)
{
    return (1ull << 63) | ((step & 0x7FFFFull) << 44) | ((uint64_t)ch << 41)
         | ((uint64_t)(cell & 0xFFFFFFu) << 17) | ((uint64_t)(j & 0xFFFFu) << 1) | (uint64_t)sub;
}

typedef struct { int32_t cell; uint64_t pid; int idx; } sort_rec;

static int cmp_rec(const void *a, const void *b)
{
    const sort_rec *x = a, *y = b;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    if (x->pid != y->pid) return x->pid < y->pid ? -1 : 1;
    return 0;
}

/* Canonical order: particles of each cell sorted by id; off[c]..off[c+1]. */
static int *canonical(const orc_species *sp, int n_cells, int **off_out)
{
    int n = sp->n;
    sort_rec *r = malloc(sizeof(sort_rec) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) { r[i].cell = sp->cell[i]; r[i].pid = sp->pid[i]; r[i].idx = i; }
    qsort(r, n, sizeof(sort_rec), cmp_rec);
    int *idx = malloc(sizeof(int) * (n > 0 ? n : 1));
    int *off = calloc(n_cells + 1, sizeof(int));
    for (int i = 0; i < n; ++i) { idx[i] = r[i].idx; off[r[i].cell + 1]++; }
    for (int c = 0; c < n_cells; ++c) off[c + 1] += off[c];
    free(r);
    *off_out = off;
    return idx;
}

typedef struct { double E; double p[3]; } vec4;

/* Lorentz transform of (E, p) into the rest frame of a particle with proper
 * velocity ui (Sec. III.A; the printed last factor gamma_e beta_e is read as
 * the ion's velocity, which makes the formula a boost):  E' = g E - ui.p,
 * p' = p + [ (ui.p)/(g+1) - E ] ui,  with g = sqrt(1 + ui^2). */
static vec4 to_rest(vec4 a, const double ui[3], double gi)
{
    double d = ui[0] * a.p[0] + ui[1] * a.p[1] + ui[2] * a.p[2];
    vec4 b;
    b.E = gi * a.E - d;
    double f = d / (gi + 1.0) - a.E;
    for (int i = 0; i < 3; ++i) b.p[i] = a.p[i] + f * ui[i];
    return b;
}

/* Inverse transform, from the rest frame of ui back to the simulation frame. */
static vec4 from_rest(vec4 a, const double ui[3], double gi)
{
    double d = ui[0] * a.p[0] + ui[1] * a.p[1] + ui[2] * a.p[2];
    vec4 b;
    b.E = gi * a.E + d;
    double f = d / (gi + 1.0) + a.E;
    for (int i = 0; i < 3; ++i) b.p[i] = a.p[i] + f * ui[i];
    return b;
}

/* Exported for the tests: (E, p) to (inverse = 0) or from (inverse = 1) the
 * rest frame of a particle with proper velocity ui. */
void orc_boost(const double ui[3], const double in[4], double out[4], int inverse)
{
    double gi = sqrt(1.0 + ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]);
    vec4 a = { in[0], { in[1], in[2], in[3] } };
    vec4 b = inverse ? from_rest(a, ui, gi) : to_rest(a, ui, gi);
    out[0] = b.E; out[1] = b.p[0]; out[2] = b.p[1]; out[3] = b.p[2];
}

/* Append one particle.  Under OpenMP the slot is taken with an atomic
 * increment (cells run on several threads); a slot past the capacity is
 * refused and the count is clamped back after the group (orc_step). */
static int append(orc_species *sp, const double u[3], double w, float x, int has_x, uint64_t pid, int cell)
{
    int i;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
    i = sp->n++;
    if (i >= sp->cap) return 1;
    sp->ux[i] = (float)u[0]; sp->uy[i] = (float)u[1]; sp->uz[i] = (float)u[2];
    sp->w[i] = (float)w;
    if (sp->x && has_x) sp->x[i] = x;
    sp->pid[i] = pid;
    sp->cell[i] = cell;
    return 0;
}

typedef struct {
    const orc_tables *t;
    const orc_screening *scr;
    int mat;
    double ion_mass;
    double coef;           /* (n_p n_t / n_pt) c dt */
    uint64_t seed, step;
    uint32_t cell;
    double *ledger;
    orc_stats *st;
} pair_ctx;

/* Ion-frame kinematics of a massive projectile. */
typedef struct { double gl, gi, Tp, pp, n[3]; double ui[3]; } frame;

static void make_frame(const orc_species *P, int ip, const orc_species *I, int it, frame *f)
{
    double ue[3] = { P->ux[ip], P->uy[ip], P->uz[ip] };
    f->ui[0] = I->ux[it]; f->ui[1] = I->uy[it]; f->ui[2] = I->uz[it];
    f->gl = sqrt(1.0 + ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2]);
    f->gi = sqrt(1.0 + f->ui[0] * f->ui[0] + f->ui[1] * f->ui[1] + f->ui[2] * f->ui[2]);
    vec4 a = { f->gl, { ue[0], ue[1], ue[2] } };
    vec4 b = to_rest(a, f->ui, f->gi);
    double p2 = b.p[0] * b.p[0] + b.p[1] * b.p[1] + b.p[2] * b.p[2];
    f->pp = sqrt(p2);
    f->Tp = p2 / (1.0 + sqrt(1.0 + p2));
    for (int i = 0; i < 3; ++i) f->n[i] = f->pp > 0.0 ? b.p[i] / f->pp : 0.0;
}

/* Momentum of kinetic energy T along n in the ion frame, boosted to the lab. */
static void lepton_lab(double T, const double n[3], const frame *f, double out[3])
{
    double p = sqrt(T * (T + 2.0));
    vec4 a = { 1.0 + T, { p * n[0], p * n[1], p * n[2] } };
    vec4 b = from_rest(a, f->ui, f->gi);
    for (int i = 0; i < 3; ++i) out[i] = b.p[i];
}

/* One Bremsstrahlung trial on pair j (Eq. proba3 and Sec. III.A). */
static int brems_pair(pair_ctx *c, int group, orc_species *P, int ip, const orc_species *I, int it,
                      uint32_t j, uint32_t r1, const accept_src *src, orc_species *ph)
{
    const orc_tables *t = c->t;
    const orc_table_spec *sp = &t->spec;
    frame f;
    make_frame(P, ip, I, it, &f);
    double sigma = orc_sigma_lookup(sp, t->brems_sigma + (size_t)c->mat * sp->n_rows, f.Tp, &c->st->status);
    if (sigma <= 0.0) return 0;
    double x = c->coef * sigma * f.pp / (f.gl * f.gi);
    if (x > 1.0) c->st->status |= ORC_ST_PROB_LARGE;
    if (!accept_u(r1, -expm1(-x), src)) return 0;
    int ch = group == G_EM ? CH_BREMS_EM : CH_BREMS_EP;
    c->st->accepted[ch] += 1;
    uint32_t ev[4];
    philox_at(j, c->cell, c->step, tag(group, PU_EVT_B, 0), c->seed, ev);
    double wp = P->w[ip], wt = I->w[it];
    if (wt < wp && !(orc_u01(ev[0]) < wt / wp)) return 0;
    c->st->created[ch] += 1;
    const double *cdf = t->brems_cdf + (size_t)c->mat * sp->n_rows * sp->n_cols;
    double xk = orc_sample(sp, TB_BREMS, cdf, f.Tp, orc_u01(ev[1]), orc_u01(ev[2]));
    double kp = xk * f.Tp;
    double uf[3];
    lepton_lab(f.Tp * (1.0 - xk), f.n, &f, uf);
    vec4 g = { kp, { kp * f.n[0], kp * f.n[1], kp * f.n[2] } };
    vec4 gl = from_rest(g, f.ui, f.gi);
    P->ux[ip] = (float)uf[0]; P->uy[ip] = (float)uf[1]; P->uz[ip] = (float)uf[2];
    float xpos = P->x ? P->x[ip] : 0.0f;
    if (append(ph, gl.p, wp, xpos, P->x != NULL, secondary_pid(c->step, ch, c->cell, j, 0), (int)c->cell)) {
        c->st->status |= ORC_ST_CAPACITY;
        return 1;
    }
    c->ledger[2 * c->cell] += wp * gl.E;
    c->ledger[2 * c->cell + 1] += wp;
    return 0;
}

/* One Trident trial on pair j (Sec. II.D, "similar scheme" of Sec. III.A). */
static int trident_pair(pair_ctx *c, int group, orc_species *P, int ip, const orc_species *I, int it,
                        uint32_t j, uint32_t r1, const accept_src *src, orc_species *em, orc_species *ep)
{
    const orc_tables *t = c->t;
    const orc_table_spec *sp = &t->spec;
    frame f;
    make_frame(P, ip, I, it, &f);
    double g1 = 1.0 + f.Tp;
    double sigma = orc_sigma_trident(c->scr->Z, g1);
    if (sigma <= 0.0) return 0;
    double x = c->coef * sigma * f.pp / (f.gl * f.gi);
    if (x > 1.0) c->st->status |= ORC_ST_PROB_LARGE;
    if (!accept_u(r1, -expm1(-x), src)) return 0;
    int ch = group == G_EM ? CH_TRI_EM : CH_TRI_EP;
    c->st->accepted[ch] += 1;
    uint32_t e1[4], e2[4];
    philox_at(j, c->cell, c->step, tag(group, PU_EVT_T1, 0), c->seed, e1);
    philox_at(j, c->cell, c->step, tag(group, PU_EVT_T2, 0), c->seed, e2);
    double wp = P->w[ip], wt = I->w[it];
    if (wt < wp && !(orc_u01(e1[0]) < wt / wp)) return 0;
    c->st->created[ch] += 1;
    double y = orc_sample(sp, TB_TRI_GP, t->tri_gp_cdf, f.Tp - 2.0, orc_u01(e1[1]), orc_u01(e1[2]));
    double gpair = 2.0 + y * (f.Tp - 2.0);
    double y2 = orc_sample(sp, TB_TRI_SPLIT, t->tri_split_cdf, gpair - 2.0, orc_u01(e1[3]), orc_u01(e2[0]));
    double Tplus = y2 * (gpair - 2.0), Tminus = (gpair - 2.0) * (1.0 - y2);
    double uf[3], upl[3], umi[3];
    lepton_lab((f.Tp - 2.0) * (1.0 - y), f.n, &f, uf);
    lepton_lab(Tplus, f.n, &f, upl);
    lepton_lab(Tminus, f.n, &f, umi);
    P->ux[ip] = (float)uf[0]; P->uy[ip] = (float)uf[1]; P->uz[ip] = (float)uf[2];
    float xpos = P->x ? P->x[ip] : 0.0f;
    int bad = append(em, umi, wp, xpos, P->x != NULL, secondary_pid(c->step, ch, c->cell, j, 0), (int)c->cell);
    bad |= append(ep, upl, wp, xpos, P->x != NULL, secondary_pid(c->step, ch, c->cell, j, 1), (int)c->cell);
    if (bad) { c->st->status |= ORC_ST_CAPACITY; return 1; }
    c->ledger[2 * c->cell + 1] += 2.0 * wp;
    return 0;
}

/* One Bethe-Heitler trial on pair j; returns 1 when the photon is absorbed. */
static int bh_pair(pair_ctx *c, orc_species *ph, int ip, const orc_species *I, int it, uint32_t j,
                   uint32_t r1, const accept_src *src, orc_species *em, orc_species *ep, int *err)
{
    const orc_tables *t = c->t;
    const orc_table_spec *sp = &t->spec;
    double uk[3] = { ph->ux[ip], ph->uy[ip], ph->uz[ip] };
    double k = sqrt(uk[0] * uk[0] + uk[1] * uk[1] + uk[2] * uk[2]);
    frame f;
    f.ui[0] = I->ux[it]; f.ui[1] = I->uy[it]; f.ui[2] = I->uz[it];
    f.gi = sqrt(1.0 + f.ui[0] * f.ui[0] + f.ui[1] * f.ui[1] + f.ui[2] * f.ui[2]);
    vec4 a = { k, { uk[0], uk[1], uk[2] } };
    vec4 b = to_rest(a, f.ui, f.gi);
    double kp = b.E;
    double pm = sqrt(b.p[0] * b.p[0] + b.p[1] * b.p[1] + b.p[2] * b.p[2]);
    double sigma = orc_sigma_lookup(sp, t->bh_sigma + (size_t)c->mat * sp->n_rows, kp - 2.0, &c->st->status);
    if (sigma <= 0.0) return 0;
    double x = c->coef * sigma * kp / (k * f.gi);
    if (x > 1.0) c->st->status |= ORC_ST_PROB_LARGE;
    if (!accept_u(r1, -expm1(-x), src)) return 0;
    c->st->accepted[CH_BH] += 1;
    uint32_t ev[4];
    philox_at(j, c->cell, c->step, tag(G_BH, PU_EVT_BH, 0), c->seed, ev);
    double wp = ph->w[ip], wt = I->w[it];
    if (wt < wp && !(orc_u01(ev[0]) < wt / wp)) return 0;
    c->st->created[CH_BH] += 1;
    const double *cdf = t->bh_cdf + (size_t)c->mat * sp->n_rows * sp->n_cols;
    double y = orc_sample(sp, TB_BH, cdf, kp - 2.0, orc_u01(ev[1]), orc_u01(ev[2]));
    for (int i = 0; i < 3; ++i) f.n[i] = b.p[i] / pm;
    double upl[3], umi[3];
    lepton_lab(y * (kp - 2.0), f.n, &f, upl);
    lepton_lab((kp - 2.0) * (1.0 - y), f.n, &f, umi);
    float xpos = ph->x ? ph->x[ip] : 0.0f;
    int bad = append(em, umi, wp, xpos, ph->x != NULL, secondary_pid(c->step, CH_BH, c->cell, j, 0), (int)c->cell);
    bad |= append(ep, upl, wp, xpos, ph->x != NULL, secondary_pid(c->step, CH_BH, c->cell, j, 1), (int)c->cell);
    if (bad) { c->st->status |= ORC_ST_CAPACITY; *err = 1; }
    c->ledger[2 * c->cell + 1] += 2.0 * wp;
    return 1;
}

/* Pair j of a cell (only the larger list is permuted):
 *   N_p >= N_t: projectile P(j), target j mod N_t;
 *   N_p <  N_t: projectile j mod N_p, target P(j);
 * where P is the random permutation of the larger list. */
static void pair_of(uint32_t j, uint32_t Np, uint32_t Nt, const uint32_t rk[4], uint32_t *s, uint32_t *tau)
{
    if (Np >= Nt) { *s = orc_perm_elem(j, Np, rk); *tau = j % Nt; }
    else { *s = j % Np; *tau = orc_perm_elem(j, Nt, rk); }
}

/*
 * One collision step over all cells.
 *
 * Order: electron-ion pairs (Brems then Trident on each pair), positron-ion
 * pairs (same), photon-ion pairs (Bethe-Heitler).  Each group pairs the
 * particles present at the start of the step; secondaries join their
 * species but are not projectiles until the next step; ions are never
 * modified.  Random numbers: Philox4x32-10, key = seed, counter
 *   permutation keys:  (0,      cell, step, group | PERM<<4)
 *   accept digits:     a draw (q, cell, step, group | ACCEPT<<4 | m<<8)
 *                      holds eight 16-bit digits, digit i being the high
 *                      (i even) or low (i odd) half of word i>>1;
 *                      e+-: q = s>>2, digits 2(s&3) (Brems) and
 *                      2(s&3)+1 (Trident); photons (one digit per pair,
 *                      BH): q = s>>3, digit s&7; s = projectile slot in
 *                      id order, m = pass index;
 *                      the rest of the uniform (only when the digit is
 *                      floor(2^16 p)): the draw (8q + i, cell, step,
 *                      group | ACCEPT_EXT<<4 | m<<8), see accept_u
 *   event draws:       (j,      cell, step, group | EVT<<4)
 * with U = ((r >> 9) + 1/2) 2^-23 for the event draws.
 */
static int g_threads = 1;

/* Threads for the cells of one group in orc_step (timing only; the result
 * does not depend on it).  1 without OpenMP. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    g_threads = n < 1 ? 1 : n;
#else
    (void)n;
    g_threads = 1;
#endif
}

int orc_get_threads(void) { return g_threads; }

static void clamp_count(orc_species *sp)
{
    if (sp->n > sp->cap) sp->n = sp->cap;
}

int orc_step(const orc_tables *t, int n_cells, const int32_t *material_of_cell,
             orc_species *em, orc_species *ep, orc_species *ph, const orc_species *ion,
             double ion_mass, double dt, uint64_t seed, uint64_t step, unsigned mask,
             double *ledger, orc_stats *st)
{
    (void)ion_mass;
    int *off_i, *off_g[3];
    int *idx_i = canonical(ion, n_cells, &off_i);
    orc_species *proj[3] = { em, ep, ph };
    int *idx_g[3];
    int n0[3];
    for (int g = 0; g < 3; ++g) { idx_g[g] = canonical(proj[g], n_cells, &off_g[g]); n0[g] = proj[g]->n; }
    int err = 0;
    unsigned char *dead = calloc(ph->n > 0 ? ph->n : 1, 1);
    /* per-thread counters, merged after each group (integer-valued sums, so
     * the merge order does not matter) */
    int nth = g_threads;
    orc_stats *tst = calloc((size_t)nth, sizeof(orc_stats));

    for (int g = 0; g < 3 && !err; ++g) {
        if (g < 2 && !(mask & (ORC_PROC_BREMS | ORC_PROC_TRIDENT))) continue;
        if (g == 2 && !(mask & ORC_PROC_BH)) continue;
        orc_species *P = proj[g];
        /* cells are independent within a group: a cell touches only its own
         * projectiles, ledger entry and absorbed-photon flags, and appends
         * secondaries through atomically taken slots */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8) num_threads(nth)
#endif
        for (int cell = 0; cell < n_cells; ++cell) {
            int stop;
#ifdef _OPENMP
#pragma omp atomic read
#endif
            stop = err;
            if (stop) continue;
#ifdef _OPENMP
            orc_stats *mst = &tst[omp_get_thread_num()];
#else
            orc_stats *mst = &tst[0];
#endif
            int cerr = 0;
            uint32_t Np = off_g[g][cell + 1] - off_g[g][cell];
            uint32_t Nt = off_i[cell + 1] - off_i[cell];
            if (Np == 0 || Nt == 0) continue;
            const int *pidx = idx_g[g] + off_g[g][cell];
            const int *tidx = idx_i + off_i[cell];
            double n_p = 0.0, n_t = 0.0, n_pt = 0.0;
            for (uint32_t s = 0; s < Np; ++s) n_p += P->w[pidx[s]];
            for (uint32_t s = 0; s < Nt; ++s) n_t += ion->w[tidx[s]];
            uint32_t Npair = Np > Nt ? Np : Nt;
            uint32_t rk[4];
            philox_at(0, (uint32_t)cell, step, tag(g, PU_PERM, 0), seed, rk);
            for (uint32_t j = 0; j < Npair; ++j) {
                uint32_t s, tau;
                pair_of(j, Np, Nt, rk, &s, &tau);
                n_pt += fmin((double)P->w[pidx[s]], (double)ion->w[tidx[tau]]);
            }
            mst->pairs[g] += Npair;
            pair_ctx c;
            c.t = t;
            c.mat = material_of_cell[cell];
            c.scr = &t->scr[c.mat];
            c.ion_mass = ion_mass;
            c.coef = n_p * n_t / n_pt * C_LIGHT * dt;
            c.seed = seed; c.step = step; c.cell = (uint32_t)cell;
            c.ledger = ledger; c.st = mst;
            for (uint32_t j = 0; j < Npair && !cerr; ++j) {
                uint32_t s, tau;
                pair_of(j, Np, Nt, rk, &s, &tau);
                uint32_t m = Np >= Nt ? 0 : j / Np;
                /* eight 16-bit digits per draw: e+- pairs take two
                 * (Brems, Trident), four pairs per draw; photon pairs one
                 * (BH), eight pairs per draw */
                uint32_t q = g < 2 ? s >> 2 : s >> 3;
                uint32_t i = g < 2 ? 2 * (s & 3) : (s & 7);
                uint32_t acc[4];
                philox_at(q, (uint32_t)cell, step, tag(g, PU_ACCEPT, m), seed, acc);
                uint32_t d0 = (i & 1) ? acc[i >> 1] & 0xFFFFu : acc[i >> 1] >> 16;
                uint32_t d1 = acc[i >> 1] & 0xFFFFu;   /* digit i + 1 (e+-: i is even) */
                accept_src s1 = { 8 * q + i, (uint32_t)cell, step, tag(g, PU_ACCEPT_EXT, m), seed };
                accept_src s2 = s1;
                s2.c0 += 1;
                int ip = pidx[s], it = tidx[tau];
                if (g < 2) {
                    if (mask & ORC_PROC_BREMS)
                        cerr |= brems_pair(&c, g, P, ip, ion, it, j, d0, &s1, ph);
                    if (mask & ORC_PROC_TRIDENT)
                        cerr |= trident_pair(&c, g, P, ip, ion, it, j, d1, &s2, em, ep);
                } else {
                    if (dead[ip]) continue;
                    if (bh_pair(&c, P, ip, ion, it, j, d0, &s1, em, ep, &cerr)) dead[ip] = 1;
                }
            }
            if (cerr) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                err = 1;
            }
        }
        clamp_count(em);
        clamp_count(ep);
        clamp_count(ph);
    }
    for (int k = 0; k < nth; ++k) {
        for (int g = 0; g < 3; ++g) st->pairs[g] += tst[k].pairs[g];
        for (int ch = 0; ch < 5; ++ch) { st->accepted[ch] += tst[k].accepted[ch]; st->created[ch] += tst[k].created[ch]; }
        st->status |= tst[k].status;
    }
    free(tst);
    /* remove absorbed photons, keeping the order of the rest */
    int w = 0;
    for (int i = 0; i < ph->n; ++i) {
        if (i < n0[2] && dead[i]) continue;
        if (w != i) {
            ph->ux[w] = ph->ux[i]; ph->uy[w] = ph->uy[i]; ph->uz[w] = ph->uz[i]; ph->w[w] = ph->w[i];
            if (ph->x) ph->x[w] = ph->x[i];
            ph->pid[w] = ph->pid[i]; ph->cell[w] = ph->cell[i];
        }
        ++w;
    }
    ph->n = w;
    free(dead);
    free(idx_i); free(off_i);
    for (int g = 0; g < 3; ++g) { free(idx_g[g]); free(off_g[g]); }
    return err;
}

/* ------------------------------------------------------------------------ */
/* Expected emission operator: the rate form of Eq. (N_br_theo1/2)          */
/* ------------------------------------------------------------------------ */

/* For ions at rest and electrons of Lorentz factor gamma[s] and weight w[s]:
 *   out[0] = n_i sum_s w_s v_s sigma_B(gamma_s)             photons / (m^3 s)
 *   out[1] = n_i sum_s w_s v_s sigma_T(gamma_s)             pairs   / (m^3 s)
 *   out[2] = n_i sum_s w_s v_s int_k k dsigma_B/dk dk        m_e c^2 / (m^3 s)
 * with the k-integrals over x = k/(gamma-1) in [1e-7, 1] by one n_quad-point
 * Gauss-Legendre panel in ln x. */
void orc_expected_emission(const orc_material *m, int n_samples, const double *gamma,
                           const double *w, int n_quad, double *out3)
{
    orc_screening s;
    orc_screening_prep(m, &s);
    double gx[128], gw[128];
    if (n_quad > 128) n_quad = 128;
    orc_gauss_legendre(n_quad, gx, gw);
    double a = log(1e-7), b = 0.0, h = 0.5 * (b - a), mid = 0.5 * (a + b);
    double R = 0.0, Rp = 0.0, P = 0.0;
    for (int i = 0; i < n_samples; ++i) {
        double g = gamma[i], T = g - 1.0;
        double v = C_LIGHT * sqrt(T * (T + 2.0)) / g;
        double sig = 0.0, ksig = 0.0;
        for (int q = 0; q < n_quad; ++q) {
            double x = exp(mid + h * gx[q]);
            double f = orc_dsdk_brems(&s, g, x * T, ORC_NR_EXACT) * T * x;
            sig += h * gw[q] * f;
            ksig += h * gw[q] * f * x * T;
        }
        R += w[i] * v * sig;
        Rp += w[i] * v * orc_sigma_trident(m->Z, g);
        P += w[i] * v * ksig;
    }
    out3[0] = m->n_i * R;
    out3[1] = m->n_i * Rp;
    out3[2] = m->n_i * P;
}

/* Gradient of the expected-emission operator with respect to the plasma
 * parameters theta = (n_i, T_e, Z*, s_TF, s_D), contracted with g_out:
 *   grad[k] = sum_j g_out[j] d out[j] / d theta_k.
 * By the definition of the derivative: central differences of the FP64
 * operator with relative step h = 1e-3 theta_k, Richardson-extrapolated from
 * steps h and h/2 (error O(h^4)).  Valid away from the kink of
 * max(lambda_D, r_i). */
void orc_expected_emission_grad(const orc_material *m, int n_samples, const double *gamma,
                                const double *w, int n_quad, const double *g_out, double *grad)
{
    for (int k = 0; k < 5; ++k) {
        double D[2];
        for (int r = 0; r < 2; ++r) {
            orc_material lo = *m, hi = *m;
            double *plo[5] = { &lo.n_i, &lo.T_e, &lo.Zstar, &lo.s_TF, &lo.s_D };
            double *phi[5] = { &hi.n_i, &hi.T_e, &hi.Zstar, &hi.s_TF, &hi.s_D };
            double h = 1e-3 * fabs(*plo[k]) / (r == 0 ? 1.0 : 2.0);
            *plo[k] -= h;
            *phi[k] += h;
            double olo[3], ohi[3];
            orc_expected_emission(&lo, n_samples, gamma, w, n_quad, olo);
            orc_expected_emission(&hi, n_samples, gamma, w, n_quad, ohi);
            D[r] = 0.0;
            for (int j = 0; j < 3; ++j) D[r] += g_out[j] * (ohi[j] - olo[j]) / (2.0 * h);
        }
        grad[k] = (4.0 * D[1] - D[0]) / 3.0;
    }
}


/* ------------------------------------------------------------------------ */
/* Analytic gradient of the expected-emission operator                       */
/* ------------------------------------------------------------------------ */

/* Derivatives with respect to L of the single-Yukawa screening functions of
 * Eqs. (deriv_I1) and (deriv_I2), by differentiating each term by hand:
 *   dI1/dL = d (atan dL - atan L) + L (1-d)/(1+L^2) - L (1-d)^2/(1+L^2)^2,
 *   d(2 I2)/dL = 12 L^2 d^3 (atan dL - atan L) + 4 L^3 d^3 (d/(1+L^2 d^2) - 1/(1+L^2))
 *              + 6 L d^2 ln((1+L^2)/(1+L^2 d^2)) + (1 + 3 L^2 d^2)(2L/(1+L^2) - 2 L d^2/(1+L^2 d^2))
 *              + 12 d^2 ln d  L^3 (L^2+2)/(1+L^2)^2
 *              + (d-1)(2L(d+1) - 16 L^3 d^2 - 8 L^5 d^2)/(1+L^2)^2.
 * atan dL - atan L is formed as atan((dL - L)/(1 + d L^2)).  Where delta L > 4
 * these terms (those of d(2 I2)/dL of order L (delta L)^2) cancel down to
 * O(1/(delta^2 L^3)); there both derivatives are taken from their integral
 * definitions (dI12_dL_quad) instead. */
static void dI12_dL_quad(double d, double L, double *dI1, double *dI2);

void orc_dI12_dL(double d, double L, double *dI1, double *dI2)
{
    double L2 = L * L, d2 = d * d, u2 = L2 * d2;
    double q = 1.0 + L2;
    if (d * L > 4.0) {
        /* the terms below cancel to O(1/(d^2 L^3)) */
        dI12_dL_quad(d, L, dI1, dI2);
        return;
    }
    double dat = atan((d * L - L) / (1.0 + d * L2));
    *dI1 = d * dat + L * (1.0 - d) / q - L * (1.0 - d) * (1.0 - d) / (q * q);
    double t1 = 12.0 * L2 * d2 * d * dat + 4.0 * L2 * L * d2 * d * (d / (1.0 + u2) - 1.0 / q);
    double t2 = 6.0 * L * d2 * log(q / (1.0 + u2)) + (1.0 + 3.0 * u2) * (2.0 * L / q - 2.0 * L * d2 / (1.0 + u2));
    double t3 = 12.0 * d2 * log(d) * L2 * L * (L2 + 2.0) / (q * q);
    double t4 = (d - 1.0) * (2.0 * L * (d + 1.0) - 16.0 * L2 * L * d2 - 8.0 * L2 * L2 * L * d2) / (q * q);
    *dI2 = 0.5 * (t1 + t2 + t3 + t4);
}

/* d I1/dL and d I2/dL from the integral definitions (Eqs. defphi1, defphi2)
 * for the single-Yukawa form factor 1 - F = (L u)^2/(1 + (L u)^2) of Eq.
 * (defF): with t = ln u and r = u/delta,
 *   dI1/dL = int_{ln delta}^0 (1 - 1/r)^2 d(1-F)^2/dL dt,
 *   dI2/dL = int_{ln delta}^0 [1 + (3 - 6 ln r)/r^2 - 4/r^3] d(1-F)^2/dL dt,
 * d(1-F)^2/dL = 4 L^3 u^4/(1 + L^2 u^2)^3; composite 8-point Gauss-Legendre
 * on equal panels no wider than 1/2.  Used where delta L > 4, where the
 * closed forms lose their digits to cancellation. */
static void dI12_dL_quad(double d, double L, double *dI1, double *dI2)
{
    double gx[8], gw[8];
    orc_gauss_legendre(8, gx, gw);
    double t0 = log(d);
    int n = (int)ceil(-t0 / 0.5);
    double h = -t0 / n, s1 = 0.0, s2 = 0.0;
    for (int p = 0; p < n; ++p) {
        double mid = t0 + (p + 0.5) * h;
        for (int q = 0; q < 8; ++q) {
            double t = mid + 0.5 * h * gx[q];
            double lr = t - t0, r = exp(lr), u = exp(t), Lu2 = L * L * u * u;
            double a = -expm1(-lr);
            double k2 = 1.0 + (3.0 - 6.0 * lr) / (r * r) - 4.0 / (r * r * r);
            double dF2 = 4.0 * L * L * L * u * u * u * u / ((1.0 + Lu2) * (1.0 + Lu2) * (1.0 + Lu2));
            s1 += gw[q] * a * a * dF2;
            s2 += gw[q] * k2 * dF2;
        }
    }
    *dI1 = 0.5 * h * s1;
    *dI2 = 0.5 * h * s2;
}

/* The two functions that enter a cross term K(A, B) = (B f(A) - A f(B))/(B - A):
 * kind 0: f(t) = ln(1 + t) (Eq. ITFD); kind 1: f(t) = ln((1 + p t)/(1 + m t))
 * (Gamma_c of Eq. cs_br_nr, p = dp+^2, m = dp-^2).  Value and two derivatives. */
static void cross_f(int kind, double p, double m, double t, double *f, double *f1, double *f2)
{
    if (kind == 0) {
        *f = log1p(t);
        *f1 = 1.0 / (1.0 + t);
        *f2 = -1.0 / ((1.0 + t) * (1.0 + t));
    } else {
        double P = 1.0 + p * t, M = 1.0 + m * t;
        *f = log(P / M);
        *f1 = p / P - m / M;
        *f2 = -p * p / (P * P) + m * m / (M * M);
    }
}

/* K(A, B) = (B f(A) - A f(B))/(B - A) and its partial derivatives.  Far from
 * A = B directly: K_A = (B f'(A) - f(B) + K)/(B - A), K_B = (f(A) - A f'(B) - K)/(B - A).
 * Near A = B (|B - A| <= B/10) through the divided difference of chi(t) = f(t)/t:
 * K = -A B chi[A, B] with chi[A, B] = int_0^1 chi'(A + s(B - A)) ds, and
 * d chi[A,B]/dA = int_0^1 (1 - s) chi''(.) ds, d chi[A,B]/dB = int_0^1 s chi''(.) ds,
 * by 8-point Gauss-Legendre in s (chi is analytic on a disk much wider than
 * the interval, so the rule is exact to rounding). */
static void cross_partials(int kind, double p, double m, double A, double B, double *K, double *KA, double *KB)
{
    double D = B - A;
    if (fabs(D) > 0.1 * fmax(A, B)) {
        double fA, fA1, fA2, fB, fB1, fB2;
        cross_f(kind, p, m, A, &fA, &fA1, &fA2);
        cross_f(kind, p, m, B, &fB, &fB1, &fB2);
        *K = (B * fA - A * fB) / D;
        *KA = (B * fA1 - fB + *K) / D;
        *KB = (fA - A * fB1 - *K) / D;
        return;
    }
    double gx[8], gw[8];
    orc_gauss_legendre(8, gx, gw);
    double J0 = 0.0, JA = 0.0, JB = 0.0;
    for (int q = 0; q < 8; ++q) {
        double s = 0.5 * (gx[q] + 1.0), w = 0.5 * gw[q];
        double t = A + s * D, f, f1, f2;
        cross_f(kind, p, m, t, &f, &f1, &f2);
        double c1 = f1 / t - f / (t * t);
        double c2 = f2 / t - 2.0 * f1 / (t * t) + 2.0 * f / (t * t * t);
        J0 += w * c1;
        JA += w * (1.0 - s) * c2;
        JB += w * s * c2;
    }
    *K = -A * B * J0;
    *KA = -B * J0 - A * B * JA;
    *KB = -A * J0 - A * B * JB;
}

/* Jacobian J[i][k] = d S_i / d theta_k of the screening quantities
 * S = (L_TF, L_D, eta_D, L_R) with respect to theta = (n_i, T_e, Z*, s_TF, s_D):
 *   L_TF = s_TF Z^(-1/3)/alpha (Eq. LTF);
 *   L_D = s_D max(lambda_D, r_i)/r_C (Eq. LDH), the active branch's derivative
 *     (r_i on a tie), lambda_D^2 = eps0 T_e/(e n_i Z*(Z*+1)), r_i^3 = 3/(4 pi n_i);
 *   eta_D = Zs/Z with Zs = Z^*, eta_TF = 1 - eta_D (Eq. V_TFD);
 *   a = I_TFD (Eq. ITFD); L_R^2 = x solves h(x) = ln(1+x) - x/(1+x) = 2a
 *     (Eq. reduit), so dL_R/da = (1/(2 L_R)) 2/h'(x) = (1+x)^2/(x L_R).
 * At Z* = 0, Eq. LDH gives lambda_D = infinity: the operator does not depend
 * on L_D there (eta_D = 0), and the derivative with respect to Z* is the
 * limit from Z* > 0, in which the cross terms tend to their B -> infinity
 * values (ln(1+A) for I_TFD) and every path through L_D vanishes. */
static void screening_jacobian(const orc_material *m, const orc_screening *s, double J[4][5])
{
    memset(J, 0, sizeof(double) * 20);
    double Z = m->Z, Zs = m->Zstar;
    int inf_debye = !(Zs > 0.0);
    J[0][3] = s->LTF / m->s_TF;
    if (!inf_debye) {
        if (s->lambdaD > s->ri) {
            J[1][0] = -0.5 * s->LD / m->n_i;
            J[1][1] = 0.5 * s->LD / m->T_e;
            J[1][2] = -0.5 * s->LD * (2.0 * Zs + 1.0) / (Zs * (Zs + 1.0));
        } else {
            J[1][0] = -s->LD / (3.0 * m->n_i);
        }
        J[1][4] = s->LD / m->s_D;
    }
    J[2][2] = 1.0 / Z;
    double A = s->LTF * s->LTF, B = s->LD * s->LD;
    double eT = s->etaTF, eD = s->etaD;
    double gA = log1p(A) - A / (1.0 + A), g1A = A / ((1.0 + A) * (1.0 + A));
    double gB = log1p(B) - B / (1.0 + B), g1B = B / ((1.0 + B) * (1.0 + B));
    double C, CA, CB;
    if (inf_debye) { C = log1p(A); CA = 1.0 / (1.0 + A); CB = 0.0; gB = 0.0; g1B = 0.0; }
    else cross_partials(0, 0.0, 0.0, A, B, &C, &CA, &CB);
    double a_LTF = (0.5 * eT * eT * g1A + eT * eD * CA) * 2.0 * s->LTF;
    double a_LD = inf_debye ? 0.0 : (0.5 * eD * eD * g1B + eT * eD * CB) * 2.0 * s->LD;
    double a_eD = -eT * gA + eD * gB + (eT - eD) * C;
    double x = s->LR * s->LR;
    double LR_a = (1.0 + x) * (1.0 + x) / (x * s->LR);
    for (int k = 0; k < 5; ++k)
        J[3][k] = LR_a * (a_LTF * J[0][k] + a_LD * J[1][k] + a_eD * J[2][k]);
}

/* Partial derivatives of dsigma/dk (orc_dsdk_brems with exact NR bounds)
 * with respect to S = (L_TF, L_D, eta_D, L_R) at fixed Z and energies; zero
 * where the cross section is clamped at zero.  inf_debye: L_D = infinity
 * (Z* = 0). */
static void dsdk_brems_partials(const orc_screening *s, double gamma1, double k, int inf_debye, double out[4])
{
    out[0] = out[1] = out[2] = out[3] = 0.0;
    double T1 = gamma1 - 1.0;
    if (!(k > 0.0 && k < T1)) return;
    if (orc_dsdk_brems(s, gamma1, k, ORC_NR_EXACT) <= 0.0) return;
    double Z = s->Z;
    if (gamma1 <= 2.0) {
        double T2 = T1 - k;
        double p1 = sqrt(T1 * (T1 + 2.0)), p2 = sqrt(T2 * (T2 + 2.0));
        double dpp = p1 + p2, dpm = k * (T1 + T2 + 2.0) / (p1 + p2);
        double b1 = p1 / gamma1, b2 = p2 / (1.0 + T2), az = 2.0 * PI * Z * ALPHA;
        double fE = (b1 / b2) * (-expm1(-az / b1)) / (-expm1(-az / b2));
        double pre = 16.0 * R_E * R_E * Z * Z * ALPHA / (3.0 * k * p1 * p1) * fE;
        double pp = dpp * dpp, mm = dpm * dpm;
        /* g(eta, L) = eta^2/2 [ln(D+/D-) + 1/D+ - 1/D-], D+- = dp+-^2 L^2 + 1:
         * dg/deta = eta [..], dg/dL = eta^2 L^3 (dp+^4/D+^2 - dp-^4/D-^2) */
        double LT = s->LTF, LTa = LT * LT;
        double Dp = pp * LTa + 1.0, Dm = mm * LTa + 1.0;
        double brT = log(Dp / Dm) + 1.0 / Dp - 1.0 / Dm;
        double gT_L = s->etaTF * s->etaTF * LTa * LT * (pp * pp / (Dp * Dp) - mm * mm / (Dm * Dm));
        double gT_eta = s->etaTF * brT;
        double gD_L = 0.0, gD_eta = 0.0;
        if (!inf_debye) {
            double LD = s->LD, LDa = LD * LD;
            double Ep = pp * LDa + 1.0, Em = mm * LDa + 1.0;
            gD_L = s->etaD * s->etaD * LDa * LD * (pp * pp / (Ep * Ep) - mm * mm / (Em * Em));
            gD_eta = s->etaD * (log(Ep / Em) + 1.0 / Ep - 1.0 / Em);
        }
        /* Gamma_c = eta_TF eta_D K(A, B), K(A, B) = (B psi(A) - A psi(B))/(B - A) */
        double K, KA, KB;
        if (inf_debye) {
            double f, f1, f2;
            cross_f(1, pp, mm, LTa, &f, &f1, &f2);
            K = f; KA = f1; KB = 0.0;
        } else {
            cross_partials(1, pp, mm, LTa, s->LD * s->LD, &K, &KA, &KB);
        }
        double eT = s->etaTF, eD = s->etaD;
        out[0] = pre * (gT_L + eT * eD * KA * 2.0 * LT);
        out[1] = inf_debye ? 0.0 : pre * (gD_L + eT * eD * KB * 2.0 * s->LD);
        out[2] = pre * (-gT_eta + gD_eta + (eT - eD) * K);
        return;
    }
    /* relativistic regimes: f_C does not depend on theta */
    double eps = (gamma1 - k) / gamma1;
    double delta = k / (2.0 * gamma1 * (gamma1 - k));
    double dI1, dI2;
    orc_dI12_dL(delta, s->LR, &dI1, &dI2);
    out[3] = 4.0 * Z * Z * R_E * R_E * ALPHA / k * ((1.0 + eps * eps) * dI1 - 2.0 / 3.0 * eps * dI2);
}

/* Exported for the tests: d(dsigma/dk)/d(L_TF, L_D, eta_D, L_R) and the
 * screening Jacobian d(L_TF, L_D, eta_D, L_R)/d(n_i, T_e, Z*, s_TF, s_D). */
void orc_dsdk_brems_grad(const orc_material *m, double gamma1, double k, double out4[4])
{
    orc_screening s;
    orc_screening_prep(m, &s);
    dsdk_brems_partials(&s, gamma1, k, !(m->Zstar > 0.0), out4);
}

void orc_screening_jacobian(const orc_material *m, double jac20[20])
{
    orc_screening s;
    orc_screening_prep(m, &s);
    double J[4][5];
    screening_jacobian(m, &s, J);
    memcpy(jac20, J, sizeof J);
}

/* Gradient of the expected-emission operator, contracted with g_out, by the
 * chain rule written out by hand (no differencing):
 *   d out_j/d theta_k = [k = n_i] out_j/n_i
 *     + n_i sum_s w_s v_s sum_q h w_q T x (x T)^[j=2] sum_i d(dsigma/dk)/dS_i J[i][k]
 * for j = 0 (photons) and 2 (power); the pair rate (j = 1) depends on theta
 * through n_i only.  Same quadrature as orc_expected_emission. */
void orc_expected_emission_grad_analytic(const orc_material *m, int n_samples, const double *gamma,
                                         const double *w, int n_quad, const double *g_out, double *grad)
{
    orc_screening s;
    orc_screening_prep(m, &s);
    double J[4][5];
    screening_jacobian(m, &s, J);
    int inf_debye = !(m->Zstar > 0.0);
    double gx[128], gw[128];
    if (n_quad > 128) n_quad = 128;
    orc_gauss_legendre(n_quad, gx, gw);
    double a = log(1e-7), b = 0.0, h = 0.5 * (b - a), mid = 0.5 * (a + b);
    double dS[4] = { 0.0, 0.0, 0.0, 0.0 };   /* d(g0 R + g2 P)/dS / n_i */
    double out3[3];
    orc_expected_emission(m, n_samples, gamma, w, n_quad, out3);
    for (int i = 0; i < n_samples; ++i) {
        double g = gamma[i], T = g - 1.0;
        double v = C_LIGHT * sqrt(T * (T + 2.0)) / g;
        for (int q = 0; q < n_quad; ++q) {
            double x = exp(mid + h * gx[q]);
            double part[4];
            dsdk_brems_partials(&s, g, x * T, inf_debye, part);
            double c = w[i] * v * h * gw[q] * T * x * (g_out[0] + g_out[2] * x * T);
            for (int r = 0; r < 4; ++r) dS[r] += c * part[r];
        }
    }
    for (int k = 0; k < 5; ++k) {
        double acc = 0.0;
        for (int r = 0; r < 4; ++r) acc += dS[r] * J[r][k];
        grad[k] = m->n_i * acc;
    }
    grad[0] += (g_out[0] * out3[0] + g_out[1] * out3[1] + g_out[2] * out3[2]) / m->n_i;
}
