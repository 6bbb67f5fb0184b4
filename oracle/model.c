/*
 * Oracle, part 3: the paper's three-macro-electron estimate of the energy
 * loss channels (Sec. III.B, "Energy loss mechanisms"), in SI and FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Steps, in the paper's order:
 *  1. a0 from Eq. (1); mean injected kinetic energy <eps> = a0 m_e c^2 <sqrt(fg)>;
 *     injected count N_e = I0 <fg> (pi r_fwhm^2/4)(t_fwhm sqrt(ln10/ln2)) eta_le / <eps>.
 *  2. The exponential spectrum dN/d eps = N_e/<eps> exp(-eps/<eps>) is cut at
 *     the X-ray threshold eps_th and the escape energy eps_esc = kappa_esc a0 m_e c^2
 *     into a "warm" (eps < eps_th), an "emitting" (eps_th <= eps < eps_esc) and
 *     an "escaping" (eps >= eps_esc) macro-electron; each carries the count
 *     and the energy of its band, i.e. the band's mean energy per electron.
 *  3. Each macro-electron is integrated along its path x through
 *       d eps/dx = -(S_brem(eps) + S_ion(eps) + S_tnsa + S_field(x)),
 *     Eqs. (stop_brem), (stop_ion), (stop_tnsa), (stop_field); the warm and
 *     emitting ones until they have no energy left, the escaping one to
 *     x = L_x, where what remains escapes.  Photons above eps_th are counted
 *     with S_brem evaluated at eps - eps_th.
 *
 * Readings where the paper is silent:
 *  - "no more energy" is eps <= E_stop; the remainder is ionisation loss;
 *  - the integrator is classical RK4 in x, each step at most rel_step eps /
 *    S_total(eps, x) and rel_step (x + r/tan(theta_c)) long, so that neither
 *    the energy nor the field's current radius changes by more than a fraction
 *    rel_step (the escaping one's last step ends on L_x); every
 *    channel's loss over a step uses the same RK4 weights, so the channels
 *    add up to the injected energy exactly;
 *  - where eps_esc <= eps_th the escaping band starts at eps_esc, the warm
 *    band ends there and the emitting band is empty;
 *  - the ionisation bracket is floored at 0 (it turns negative below I_ex);
 *  - S_brem(eps - eps_th) jumps from 0 to S_brem(0) at the threshold, as
 *    printed; the step across the jump is only first-order accurate.
 */
#include "oracle.h"

#include <math.h>

#define Q_E 1.602176634e-19
#define M_E 9.1093837015e-31
#define C_L 299792458.0
#define EPS0 8.8541878128e-12
#define H_PL 6.62607015e-34
#define PI 3.14159265358979323846
#define HBAR (H_PL / (2.0 * PI))
#define MC2 (M_E * C_L * C_L)

typedef struct {
  const orc_model_in *m;
  double Kb;      /* S_brem = Kb gamma (J/m) */
  double Ki;      /* S_ion = Ki / beta^2 * bracket */
  double St;      /* S_tnsa (J/m) */
  double Fc;      /* S_field = Fc / (x tan(theta_c) + r)^2 */
  double r, tan_c;
} model_ctx;

/* the four channels (J/m) and the above-threshold photon rate at (eps, x) */
static void channels(const model_ctx *c, double eps, double x, double s[5]) {
  const orc_model_in *m = c->m;
  double gam = 1.0 + eps / MC2;
  s[0] = (m->mechanisms & ORC_MODEL_BREM) ? c->Kb * gam : 0.0;
  s[1] = 0.0;
  if ((m->mechanisms & ORC_MODEL_ION) && eps > 0.0) {
    double beta2 = 1.0 - 1.0 / (gam * gam);
    double br = log(eps / m->I_ex) + 0.5 * log(gam + 1.0) + 0.909 / (gam * gam) - 0.818 / gam - 0.246;
    s[1] = br > 0.0 ? c->Ki / beta2 * br : 0.0;
  }
  s[2] = (m->mechanisms & ORC_MODEL_TNSA) ? c->St : 0.0;
  if (m->mechanisms & ORC_MODEL_FIELD) {
    double rr = x * c->tan_c + c->r;
    s[3] = c->Fc / (rr * rr);
  } else {
    s[3] = 0.0;
  }
  s[4] = ((m->mechanisms & ORC_MODEL_BREM) && eps > m->eps_th)
             ? c->Kb * (1.0 + (eps - m->eps_th) / MC2) : 0.0;
}

/* one macro-electron of kinetic energy eps0 (J, per electron); adds its
 * per-electron channel losses to loss[0..3] (brem, ion, tnsa, field),
 * photons above threshold to loss[4], escaped energy to loss[5]; returns
 * the path length */
static double integrate(const model_ctx *c, double eps0, int escaping, double loss[6]) {
  const orc_model_in *m = c->m;
  double eps = eps0, x = 0.0;
  for (long it = 0; it < 10000000L; ++it) {
    if (!escaping && eps <= m->E_stop) {
      loss[1] += eps;  /* the remainder is deposited by ionisation */
      return x;
    }
    if (escaping && x >= m->Lx) {
      loss[5] += eps;
      return x;
    }
    if (eps <= 0.0) return x;
    double k1[5], k2[5], k3[5], k4[5];
    channels(c, eps, x, k1);
    double tot1 = k1[0] + k1[1] + k1[2] + k1[3];
    if (!(tot1 > 0.0)) {  /* nothing slows it down any more */
      loss[escaping ? 5 : 1] += eps;
      return escaping ? m->Lx : x;
    }
    double h = m->rel_step * eps / tot1;
    if (m->mechanisms & ORC_MODEL_FIELD) {  /* resolve the field's fall-off too */
      double hx = m->rel_step * (x + c->r / c->tan_c);
      if (hx < h) h = hx;
    }
    if (escaping && x + h > m->Lx) h = m->Lx - x;
    channels(c, eps - 0.5 * h * tot1, x + 0.5 * h, k2);
    double tot2 = k2[0] + k2[1] + k2[2] + k2[3];
    channels(c, eps - 0.5 * h * tot2, x + 0.5 * h, k3);
    double tot3 = k3[0] + k3[1] + k3[2] + k3[3];
    channels(c, eps - h * tot3, x + h, k4);
    double d[5], de = 0.0;
    for (int q = 0; q < 5; ++q) d[q] = h / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
    for (int q = 0; q < 4; ++q) de += d[q];
    if (de >= eps) {  /* the step would overshoot zero: share what is left */
      for (int q = 0; q < 4; ++q) loss[q] += eps * d[q] / de;
      loss[4] += d[4] * eps / de;
      return x + h * eps / de;
    }
    for (int q = 0; q < 5; ++q) loss[q] += d[q];
    eps -= de;
    x += h;
  }
  return x;
}

void orc_model(const orc_model_in *m, orc_model_out *out) {
  model_ctx c;
  c.m = m;
  double a0 = orc_a0(m->I0, m->lambda);
  double T = a0 * MC2 * m->mean_sqrt_fg;                   /* <eps> */
  double N_e = m->I0 * m->mean_fg * (PI * m->r_fwhm * m->r_fwhm / 4.0) *
               (m->t_fwhm * sqrt(log(10.0) / log(2.0))) * m->eta_l2e / T;
  double Lrad = log(5.6 * PI * EPS0 * HBAR * C_L / (cbrt(m->Z) * Q_E * Q_E));
  c.Kb = pow(Q_E, 6) / (12.0 * PI * PI * PI * pow(EPS0, 3) * M_E * pow(C_L, 3) * HBAR) *
         m->n_i * m->Z * m->Z * Lrad;                      /* Eq. (stop_brem) / gamma */
  c.Ki = m->Z * m->n_i * pow(Q_E, 4) / (4.0 * PI * EPS0 * EPS0 * M_E * C_L * C_L);
  c.St = 3.0 * m->kappa_tnsa * a0 * MC2 / (m->Lx + m->Ly + m->Lz);   /* Eq. (stop_tnsa) */
  c.r = 0.5 * m->r_fwhm;
  c.tan_c = tan(m->theta_c);
  c.Fc = Q_E * Q_E * m->eta_avg * m->I0 * m->mean_fg * c.r * c.r * m->eta_l2e / T;  /* (stop_field) */

  double th = m->eps_th, esc = m->kappa_esc * a0 * MC2;
  double lo[3] = {0.0, th, esc};
  double hi[3] = {th < esc ? th : esc, esc, INFINITY};
  for (int q = 0; q < 8; ++q) out->E[q] = 0.0;
  out->N_e = N_e;
  out->a0 = a0;
  for (int b = 0; b < 3; ++b) {
    out->N_band[b] = 0.0;
    out->eps_band[b] = 0.0;
    out->x_end[b] = 0.0;
    if (!(hi[b] > lo[b])) continue;
    double ea = exp(-lo[b] / T), eb = isinf(hi[b]) ? 0.0 : exp(-hi[b] / T);
    double n = N_e * (ea - eb);
    double e = N_e * ((lo[b] + T) * ea - (isinf(hi[b]) ? 0.0 : (hi[b] + T) * eb));
    if (!(n > 0.0)) continue;
    double eps = e / n, loss[6] = {0, 0, 0, 0, 0, 0};
    out->N_band[b] = n;
    out->eps_band[b] = eps;
    out->x_end[b] = integrate(&c, eps, b == 2, loss);
    out->E[ORC_MODEL_E_INJ] += e;
    for (int q = 0; q < 6; ++q) out->E[1 + q] += n * loss[q];
  }
}
