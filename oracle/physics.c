/*
 * Oracle, part 1: single formulas of the hybrid-PIC method in SI, FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Each function names the passage of arXiv 2107.01723 it writes out.
 * Equations are numbered as the paper's revtex source numbers them:
 * (1) a0, (4) bremsstrahlung stopping power, (5) ionisation stopping power,
 * (A1)-(A3) Ohm / Ampere-Maxwell / Faraday, (A4)-(A6) reduced Lee-More,
 * (A7) temperature rise, (A8) heat capacity, (B1) injection count,
 * (B4) Davies scatter angle.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>

/* CODATA 2018 SI values; mu0 is taken as 1/(eps0 c^2) */
#define Q_E 1.602176634e-19
#define M_E 9.1093837015e-31
#define C_L 299792458.0
#define EPS0 8.8541878128e-12
#define H_PL 6.62607015e-34
#define K_B 1.380649e-23
#define PI 3.14159265358979323846
#define HBAR (H_PL / (2.0 * PI))
#define A_BOHR 5.29177210903e-11   /* Bohr radius (m) */
#define AMU 1.66053906660e-27      /* atomic mass constant (kg) */

/* ---------------- Philox4x32-10 ----------------
 * Counter-based generator of Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64
 * multiplies on a 4-word counter, with a Weyl-sequence key schedule.  The
 * multipliers and key increments are the ones that paper publishes. */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in the open interval (0,1): the top 23 bits plus one half, over
 * 2^23.  Every value is exact in both float and double. */
double orc_uniform(uint32_t x) {
  return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* ---------------- laser ---------------- */
/* Eq. (1), Sec. II.A: a0 ~ 8.5e-6 sqrt(I0 lambda^2), I0 in W m^-2, lambda in m */
double orc_a0(double I0_Wm2, double lambda_m) {
  return 8.5e-6 * sqrt(I0_Wm2 * lambda_m * lambda_m);
}

/* ---------------- compounds ----------------
 * App. A: several elements may share every cell (a compound solid such as
 * plastic).  The paper prints the rule for the heating only: n_e = Z n_i is
 * replaced by the sum over the elements and 1/C by its n_e-weighted mean, so
 * that two overlapping solids of one material behave as the single solid.
 * For the rest the readings are the usual mixture rules: ionisation
 * stopping powers and bremsstrahlung rates (n_i sigma) add (Bragg's rule),
 * Davies scatter variances add, and the resistivity of Eqs. (A4)-(A6) takes
 * the free-electron density sum Z* n_i, the e-i collision density sum
 * Z*^2 n_i and the total ion density for the ion-sphere radius. */
static int n_solids(const orc_target *t) { return 1 + t->n_extra; }

/* element s of the target as a single-element target */
static orc_target solid(const orc_target *t, int s) {
  orc_target o = *t;
  o.n_extra = 0;
  if (s > 0) {
    o.Z = t->extra[s - 1].Z;
    o.n_i = t->extra[s - 1].n_i;
    o.I_ex = t->extra[s - 1].I_ex;
    o.Zstar = t->extra[s - 1].Zstar;
    o.A_ion = t->extra[s - 1].A_ion;
  }
  return o;
}

/* ---------------- stopping powers ---------------- */
/* Eq. (5), Sec. III.B: continuous ionisation stopping power (J/m) for an
 * electron of kinetic energy eps_k.  The bracket is held at >= 0 (it is
 * positive for every energy above the tracking cut). */
static double stop_ion_1(const orc_target *t, double eps_k) {
  double mc2 = M_E * C_L * C_L;
  double gamma = 1.0 + eps_k / mc2;
  double beta2 = 1.0 - 1.0 / (gamma * gamma);
  double v2 = beta2 * C_L * C_L;
  double pref = t->Z * t->n_i * pow(Q_E, 4) / (4.0 * PI * EPS0 * EPS0 * M_E * v2);
  double bracket = log(eps_k / t->I_ex) + 0.5 * log(gamma + 1.0) +
                   0.909 / (gamma * gamma) - 0.818 / gamma - 0.246;
  if (bracket < 0.0) bracket = 0.0;
  return pref * bracket;
}

double orc_stop_ion(const orc_target *t, double eps_k) {
  double s = stop_ion_1(t, eps_k);
  for (int q = 1; q < n_solids(t); ++q) {
    orc_target o = solid(t, q);
    s += stop_ion_1(&o, eps_k);
  }
  return s;
}

/* the screening logarithm of Eq. (4) */
static double brem_log(double Z) {
  return log(5.6 * PI * EPS0 * HBAR * C_L / (cbrt(Z) * Q_E * Q_E));
}

/* Eq. (4), Sec. III.B: bremsstrahlung stopping power over all photon
 * energies (J/m). */
static double stop_brem_1(const orc_target *t, double eps_k) {
  double gamma = 1.0 + eps_k / (M_E * C_L * C_L);
  return gamma * pow(Q_E, 6) * t->n_i * t->Z * t->Z * brem_log(t->Z) /
         (12.0 * PI * PI * PI * pow(EPS0, 3) * M_E * pow(C_L, 3) * HBAR);
}

double orc_stop_brem(const orc_target *t, double eps_k) {
  double s = stop_brem_1(t, eps_k);
  for (int q = 1; q < n_solids(t); ++q) {
    orc_target o = solid(t, q);
    s += stop_brem_1(&o, eps_k);
  }
  return s;
}

/* ---------------- bremsstrahlung cross section ----------------
 * The Seltzer-Berger tables the paper samples (App. B) are not printed, so
 * the differential cross section is the screened Bethe-Heitler shape
 *   dsigma/dk = C(eps) s(k/eps) / k,   s(u) = (4/3)(1-u) + u^2,
 * with C(eps) fixed so that n_i * integral_0^eps k dsigma/dk dk is exactly
 * the stopping power of Eq. (4).  Since integral_0^1 s(u) du = 1, that is
 * C(eps) = stop_brem(eps) / (n_i eps). */
static double brem_C(const orc_target *t, double eps_k) {
  return orc_stop_brem(t, eps_k) / (t->n_i * eps_k);
}

static double shape_s(double u) { return (4.0 / 3.0) * (1.0 - u) + u * u; }

double orc_dsigma_dk(const orc_target *t, double eps_k, double k) {
  if (k <= 0.0 || k > eps_k) return 0.0;
  return brem_C(t, eps_k) * shape_s(k / eps_k) / k;
}

/* integral of s(u)/u from u0 to u */
static double shape_G(double u0, double u) {
  return (4.0 / 3.0) * (log(u / u0) - (u - u0)) + 0.5 * (u * u - u0 * u0);
}

/* total cross section for photons k_min <= k <= eps_k (m^2, per ion of the
 * target's own element; a compound's is its emission rate over that n_i) */
double orc_sigma_tot(const orc_target *t, double k_min, double eps_k) {
  if (eps_k <= k_min) return 0.0;
  return brem_C(t, eps_k) * shape_G(k_min / eps_k, 1.0);
}

/* emission rate per unit length, the sum of n_i sigma_tot over the elements
 * (the photon spectrum's shape s(k/eps)/k is the same for every element) */
double orc_brem_rate(const orc_target *t, double k_min, double eps_k) {
  return t->n_i * orc_sigma_tot(t, k_min, eps_k);
}

/* Inverse-CDF table.  Row i is the electron energy
 * eps_i = k_min (E_max/k_min)^(i/(rows-1)); column j holds v(r_j),
 * r_j = j/(cols-1), where k = k_min (eps_i/k_min)^v is the photon energy at
 * which the cumulative emission probability reaches r_j.  Found by
 * bisection on the closed-form CDF.  Row 0 (eps = k_min) takes the limit
 * of a spectrum flat in ln k, v = r. */
void orc_brem_table(const orc_target *t, double k_min, double E_max, int rows,
                    int cols, double *v) {
  (void)t; /* the shape in v does not depend on the material */
  for (int i = 0; i < rows; ++i) {
    double eps = k_min * pow(E_max / k_min, (double)i / (double)(rows - 1));
    for (int j = 0; j < cols; ++j) {
      double r = (double)j / (double)(cols - 1);
      if (i == 0) {
        v[i * cols + j] = r;
        continue;
      }
      double u0 = k_min / eps;
      double target = r * shape_G(u0, 1.0);
      double lo = 0.0, hi = 1.0;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double u = pow(u0, 1.0 - mid);
        if (shape_G(u0, u) < target) lo = mid; else hi = mid;
        if (hi - lo < 1e-17) break;
      }
      v[i * cols + j] = 0.5 * (lo + hi);
    }
  }
}

/* Sampling rule: r -> column position (linear), ln eps -> row position
 * (linear), clamped to the table; k = k_min (eps/k_min)^v. */
double orc_brem_sample(const double *v, int rows, int cols, double k_min,
                       double E_max, double eps_k, double r) {
  double L = log(eps_k / k_min) / log(E_max / k_min) * (double)(rows - 1);
  int i = (int)floor(L);
  if (i < 0) i = 0;
  if (i > rows - 2) i = rows - 2;
  double f = L - (double)i;
  if (f < 0.0) f = 0.0;
  if (f > 1.0) f = 1.0;
  double cpos = r * (double)(cols - 1);
  int j = (int)floor(cpos);
  if (j < 0) j = 0;
  if (j > cols - 2) j = cols - 2;
  double g = cpos - (double)j;
  double va = v[i * cols + j] * (1.0 - g) + v[i * cols + j + 1] * g;
  double vb = v[(i + 1) * cols + j] * (1.0 - g) + v[(i + 1) * cols + j + 1] * g;
  double vv = va * (1.0 - f) + vb * f;
  return k_min * exp(vv * log(eps_k / k_min));
}

/* Photon polar angle about the electron direction.  The Tsai sampler of the
 * paper (App. B) is not printed; theta = t / gamma with t distributed as
 * t / (1+t^2)^2 (the leading relativistic form), truncated at theta <= pi.
 * Inverse CDF: F(t) = t^2/(1+t^2), F = u F_max. */
double orc_photon_theta(double gamma, double u) {
  double a = PI * gamma;
  double Fmax = a * a / (1.0 + a * a);
  double F = u * Fmax;
  double oneminusF = (1.0 - u) + u / (1.0 + a * a);
  return sqrt(F / oneminusF) / gamma;
}

/* ---------------- elastic scatter ---------------- */
/* Eq. (B4), App. B (Davies): rms polar deflection over dt for momentum p
 * (SI).  The logarithm is held at >= 0. */
static double davies_var_1(const orc_target *t, double p, double dt) {
  double gamma = sqrt(1.0 + (p / (M_E * C_L)) * (p / (M_E * C_L)));
  double lg = log(4.0 * EPS0 * H_PL * p / (cbrt(t->Z) * M_E * Q_E * Q_E));
  if (lg < 0.0) lg = 0.0;
  return t->Z * t->Z * pow(Q_E, 4) * t->n_i * gamma * M_E /
         (2.0 * PI * EPS0 * EPS0 * p * p * p) * lg * dt;
}

double orc_davies_sigma(const orc_target *t, double p, double dt) {
  double var = davies_var_1(t, p, dt);
  for (int q = 1; q < n_solids(t); ++q) {
    orc_target o = solid(t, q);
    var += davies_var_1(&o, p, dt);
  }
  return sqrt(var);
}

/* ---------------- background solid ---------------- */
/* Eq. (A8), App. A: heat capacity C(T'), T' = (k_B T_e / e) Z^(-4/3) */
double orc_heat_capacity(double T_K, double Z) {
  double Tp = (K_B * T_K / Q_E) * pow(Z, -4.0 / 3.0);
  return 0.3 + 1.2 * Tp * (2.2 + Tp) / ((1.1 + Tp) * (1.1 + Tp));
}

/* Eq. (A7): dT = rho / (Z n_i C k_B); a compound replaces Z n_i by the sum
 * of n_e = Z n_i over its elements and 1/C by its n_e-weighted mean */
double orc_temperature_rise(const orc_target *t, double T_K, double rho) {
  if (t->n_extra == 0) return rho / (t->Z * t->n_i * orc_heat_capacity(T_K, t->Z) * K_B);
  double ne = 0.0, inv_c = 0.0;
  for (int q = 0; q < n_solids(t); ++q) {
    orc_target o = solid(t, q);
    double n = o.Z * o.n_i;
    ne += n;
    inv_c += n / orc_heat_capacity(T_K, o.Z);
  }
  return rho * (inv_c / ne) / (ne * K_B);
}

/* Eqs. (A4)-(A6), App. A: reduced Lee-More resistivity.  tauA is the larger
 * of the hot (A5) and cold (A6) limits; the cold limit is dropped when
 * lambda1 = 0; the result is multiplied by lambda2 and capped at eta_max. */
double orc_resistivity(const orc_target *t, double T_K) {
  double kT = K_B * T_K;
  double ne = 0.0, nz2 = 0.0, ni = 0.0;  /* sum Z* n_i, sum Z*^2 n_i, sum n_i */
  for (int q = 0; q < n_solids(t); ++q) {
    orc_target o = solid(t, q);
    ne += o.Zstar * o.n_i;
    nz2 += o.Zstar * o.Zstar * o.n_i;
    ni += o.n_i;
  }
  double tau_hot = 128.0 * PI * EPS0 * EPS0 / (3.0 * pow(Q_E, 4)) *
                   sqrt(M_E / (2.0 * PI)) * pow(kT, 1.5) / (nz2 * t->lnLambda);
  double tau = tau_hot;
  if (t->lambda1 > 0.0) {
    double R0 = cbrt(3.0 / (4.0 * PI * ni));
    double vbar = sqrt(3.0 * kT / M_E);
    double tau_cold = R0 / vbar * t->lambda1;
    if (tau_cold > tau) tau = tau_cold;
  }
  double eta = t->lambda2 * M_E / (ne * Q_E * Q_E * tau);
  if (eta > t->eta_max) eta = t->eta_max;
  return eta;
}

/* App. B: ionised-screening enhancement of the bremsstrahlung cross section
 *   F_sigma = 1 + ln(lambda_D / a_s) / ln(a_s m_e c / hbar) (Zstar / Z)^2,
 * a_s = 1.4 a_B Z^(-1/3) the atomic screening length, lambda_D the Debye
 * length of the background ions, (eps0 k_B T_i / (n_i Zstar^2 e^2))^(1/2).
 * The printed denominator ln|a_s m_e c^2/hbar| is not dimensionless; it is
 * read as the log of a_s over the reduced Compton wavelength hbar/(m_e c). */
double orc_f_sigma(const orc_target *t, double Ti_K) {
  double lambda_D = sqrt(EPS0 * K_B * Ti_K / (t->n_i * t->Zstar * t->Zstar * Q_E * Q_E));
  double a_s = 1.4 * A_BOHR * pow(t->Z, -1.0 / 3.0);
  double ratio = t->Zstar / t->Z;
  return 1.0 + log(lambda_D / a_s) / log(a_s * M_E * C_L / HBAR) * ratio * ratio;
}

/* App. A: electron-ion equilibration,
 *   dT_e/dt = (T_i - T_e) Z*^2 e^4 n_i / t_c,
 *   dT_i/dt = (T_e - T_i) Z*^3 e^4 n_i / t_c,
 *   1/t_c = 2 / (3 (2 pi k_B)^(3/2)) sqrt(m_e m_i) ln(Lambda)
 *           / (eps0^2 (T_e m_i + T_i m_e)^(3/2)). */
void orc_ei_rates(const orc_target *t, double Te_K, double Ti_K, double *rate_e,
                  double *rate_i) {
  double m_i = t->A_ion * AMU;
  double inv_tc = 2.0 / (3.0 * pow(2.0 * PI * K_B, 1.5)) * sqrt(M_E * m_i) * t->lnLambda /
                  (EPS0 * EPS0 * pow(Te_K * m_i + Ti_K * M_E, 1.5));
  double base = pow(Q_E, 4) * t->n_i * inv_tc;
  *rate_e = t->Zstar * t->Zstar * base;
  *rate_i = t->Zstar * t->Zstar * t->Zstar * base;
}

/* ---------------- geometry ---------------- */
/* Rotate unit vector d by polar angle theta at azimuth phi.  The azimuth is
 * measured in the orthonormal frame (e1, e2) of Duff et al., "Building an
 * orthonormal basis, revisited" (JCGT 6(1), 2017). */
void orc_rotate(const double d[3], double theta, double phi, double out[3]) {
  double sgn = d[2] >= 0.0 ? 1.0 : -1.0;
  double a = -1.0 / (sgn + d[2]);
  double b = d[0] * d[1] * a;
  double e1[3] = {1.0 + sgn * d[0] * d[0] * a, sgn * b, -sgn * d[0]};
  double e2[3] = {b, sgn + d[1] * d[1] * a, -d[1]};
  double ct = cos(theta), st = sin(theta), cp = cos(phi), sp = sin(phi);
  for (int c = 0; c < 3; ++c)
    out[c] = d[c] * ct + (e1[c] * cp + e2[c] * sp) * st;
}

/* ---------------- relativistic push ----------------
 * The paper does not name its pusher; the relativistic Boris scheme is used:
 * half electric kick, magnetic rotation, half electric kick, for charge -e.
 * u = p/(m_e c) in and out; E in V/m, B in T. */
void orc_boris(double u[3], const double E[3], const double B[3], double dt) {
  double qe = -Q_E;
  double ke = qe * dt / (2.0 * M_E * C_L);
  double um[3] = {u[0] + ke * E[0], u[1] + ke * E[1], u[2] + ke * E[2]};
  double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  double kb = qe * dt / (2.0 * M_E * gm);
  double tv[3] = {kb * B[0], kb * B[1], kb * B[2]};
  double t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
  double sv[3] = {2.0 * tv[0] / (1.0 + t2), 2.0 * tv[1] / (1.0 + t2), 2.0 * tv[2] / (1.0 + t2)};
  double up[3] = {um[0] + (um[1] * tv[2] - um[2] * tv[1]),
                  um[1] + (um[2] * tv[0] - um[0] * tv[2]),
                  um[2] + (um[0] * tv[1] - um[1] * tv[0])};
  double uq[3] = {um[0] + (up[1] * sv[2] - up[2] * sv[1]),
                  um[1] + (up[2] * sv[0] - up[0] * sv[2]),
                  um[2] + (up[0] * sv[1] - up[1] * sv[0])};
  u[0] = uq[0] + ke * E[0];
  u[1] = uq[1] + ke * E[1];
  u[2] = uq[2] + ke * E[2];
}
