// Per-node device code of the field solve and heating (arXiv 2107.01723,
// Eqs. (A2)-(A8)), shared by the single-target and the batched kernels.
#pragma once

#include "kernels.h"

namespace hpic {

// (i, j, k) of node q; node counts stay below 2^31 (checked at creation), so
// 32-bit division suffices
__device__ __forceinline__ void node_of(long long q, int nx, int ny, int &i, int &j, int &k) {
  const unsigned uq = (unsigned)q, sy = (unsigned)nx + 1u, sz = sy * ((unsigned)ny + 1u);
  const unsigned kk = uq / sz, r = uq - kk * sz, jj = r / sy;
  k = (int)kk;
  j = (int)jj;
  i = (int)(r - jj * sy);
}

// ---------------------------------------------------------------- E, Eq. (A2)
// E on the three edges owned by node q (tangential E = 0 on the walls)
template <typename R>
__device__ __forceinline__ void efield_node(const Consts &K, const GView<R> &g, long long q) {
  const int nx = K.nx, ny = K.ny, nz = K.nz;
  const int sy = nx + 1;
  const long long sz = (long long)(nx + 1) * (ny + 1);
  const long long cy = nx, cz = (long long)nx * ny;
  const R Fc = R(K.F_curl), Fj = R(K.F_j);
  const R *Bx = g.B[0], *By = g.B[1], *Bz = g.B[2];
  int i, j, k;
  node_of(q, nx, ny, i, j, k);
  R ex = 0, ey = 0, ez = 0;
  const long long c = i + cy * j + cz * k;  // cell (i, j, k)
  if (i < nx && j >= 1 && j <= ny - 1 && k >= 1 && k <= nz - 1) {
    const R curl = (Bz[q] - Bz[q - sy]) - (By[q] - By[q - sz]);
    const R eta = R(0.25) * (g.eta_r[c - cy - cz] + g.eta_r[c - cz] + g.eta_r[c - cy] + g.eta_r[c]);
    ex = eta * (Fc * curl - Fj * g.J[0][q]);
  }
  if (j < ny && i >= 1 && i <= nx - 1 && k >= 1 && k <= nz - 1) {
    const R curl = (Bx[q] - Bx[q - sz]) - (Bz[q] - Bz[q - 1]);
    const R eta = R(0.25) * (g.eta_r[c - 1 - cz] + g.eta_r[c - cz] + g.eta_r[c - 1] + g.eta_r[c]);
    ey = eta * (Fc * curl - Fj * g.J[1][q]);
  }
  if (k < nz && i >= 1 && i <= nx - 1 && j >= 1 && j <= ny - 1) {
    const R curl = (By[q] - By[q - 1]) - (Bx[q] - Bx[q - sy]);
    const R eta = R(0.25) * (g.eta_r[c - 1 - cy] + g.eta_r[c - cy] + g.eta_r[c - 1] + g.eta_r[c]);
    ez = eta * (Fc * curl - Fj * g.J[2][q]);
  }
  g.E[0][q] = ex;
  g.E[1][q] = ey;
  g.E[2][q] = ez;
}

// T + rho / (Z n_i k_B C(T)) with the heat capacity of Eq. (A8),
// C = 0.3 + 1.2 T'(2.2 + T')/(1.1 + T')^2, T' = (k_B T/e) Z^(-4/3), brought
// over one denominator (one FP64 division per cell)
__device__ __forceinline__ double heated(const Consts &K, double T, double rho) {
  if (K.n_solids == 1) {
    const double tp = T * K.Tp_fac, D = 1.1 + tp;
    const double D2 = D * D;
    return T + rho * D2 / (K.heat_den * (0.3 * D2 + 1.2 * tp * (2.2 + tp)));
  }
  // a compound: heat_den = k_B sum Z n_i, 1/C averaged with the n_e weights
  double inv_c = 0.0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (s >= K.n_solids) break;
    const double tp = T * K.Tp_fac_s[s], D = 1.1 + tp;
    const double D2 = D * D;
    inv_c += K.ne_frac[s] * D2 / (0.3 * D2 + 1.2 * tp * (2.2 + tp));
  }
  return T + rho * inv_c / K.heat_den;
}

// The FP32-mixed path: the increment rho / (n k_B C(T)) of the same
// expression in FP32 (relative error ~1e-7 of the increment); T itself
// accumulates in FP64
__device__ __forceinline__ float heat_increment_f32(const Consts &K, double T, float rho) {
  const float Tf = (float)T;
  if (K.n_solids == 1) {
    const float tp = Tf * (float)K.Tp_fac, D = 1.1f + tp;
    const float D2 = D * D;
    return rho * D2 / ((float)K.heat_den * (0.3f * D2 + 1.2f * tp * (2.2f + tp)));
  }
  float inv_c = 0.0f;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (s >= K.n_solids) break;
    const float tp = Tf * (float)K.Tp_fac_s[s], D = 1.1f + tp;
    const float D2 = D * D;
    inv_c += (float)K.ne_frac[s] * D2 / (0.3f * D2 + 1.2f * tp * (2.2f + tp));
  }
  return rho * inv_c / (float)K.heat_den;
}

// reduced Lee-More resistivity, Eqs. (A4)-(A6), capped; inside the band
// where the cap holds, the cap itself.  eta_num / max(tau_hot, tau_cold) is
// the smaller of eta_num/(A_hot (kT)^1.5) and eta_num sqrt(kT)/B_cold, both
// formed from one reciprocal square root (no FP64 division)
__device__ __forceinline__ double resistivity(const Consts &K, double T) {
  if (T > K.eta_Tlo && T < K.eta_Thi) return K.eta_max;
  const double kT = 1.380649e-23 * T;
  const double r = rsqrt(kT);
  double eta = K.eta_hot_c * (r * r * r);
  if (K.lambda1 > 0.0) {
    const double ec = K.eta_cold_c * (kT * r);
    eta = ec < eta ? ec : eta;
  }
  return eta < K.eta_max ? eta : K.eta_max;
}

// ---------------------------------------------------------------- B, Eq. (A3), and heating
// Faraday on the faces owned by node q, then heating of cell q; returns the
// cell's Ohmic energy (J)
template <typename R>
__device__ __forceinline__ double bheat_node(const Consts &K, const GView<R> &g, long long q) {
  const int nx = K.nx, ny = K.ny, nz = K.nz;
  const int sy = nx + 1;
  const long long sz = (long long)(nx + 1) * (ny + 1);
  const R cdt = R(K.cdt_dx);
  const R *Ex = g.E[0], *Ey = g.E[1], *Ez = g.E[2];
  double e_ohm = 0.0;
  int i, j, k;
  node_of(q, nx, ny, i, j, k);
  if (K.physics & P_FARADAY) {
    if (j < ny && k < nz) g.B[0][q] -= cdt * ((Ez[q + sy] - Ez[q]) - (Ey[q + sz] - Ey[q]));
    if (i < nx && k < nz) g.B[1][q] -= cdt * ((Ex[q + sz] - Ex[q]) - (Ez[q + 1] - Ez[q]));
    if (i < nx && j < ny) g.B[2][q] -= cdt * ((Ey[q + 1] - Ey[q]) - (Ex[q + sy] - Ex[q]));
  }
  if (i < nx && j < ny && k < nz) {
    const long long c = i + (long long)nx * (j + (long long)ny * k);
    const double Hc = g.H[c];
    R jb2 = R(0);
    if (K.physics & P_FIELDS) {
      const R *Jx = g.J[0], *Jy = g.J[1], *Jz = g.J[2];
      // cell-centred mean of the edge current in the field precision
      const R jbx = R(0.25) * (Jx[q] + Jx[q + sy] + Jx[q + sz] + Jx[q + sy + sz]);
      const R jby = R(0.25) * (Jy[q] + Jy[q + 1] + Jy[q + sz] + Jy[q + 1 + sz]);
      const R jbz = R(0.25) * (Jz[q] + Jz[q + 1] + Jz[q + sy] + Jz[q + 1 + sy]);
      jb2 = jbx * jbx + jby * jby + jbz * jbz;
    }
    // a cell without drag heat or current keeps T and eta (and adds no
    // Ohmic energy) unless e-i equilibration moves it
    if (Hc == 0.0 && jb2 == R(0) && !(K.physics & P_EI)) return e_ohm;
    double Te = g.T[c];
    bool changed = false;
    if constexpr (sizeof(R) == 4) {
      const float ro = g.eta_r[c] * (float)K.F_ohm * jb2;
      const float rho = (float)(Hc * K.F_H) + ro;
      e_ohm = (double)ro * K.dx3;
      if ((K.physics & P_HEATING) && rho != 0.0f) {  // rho = 0 leaves T as it is
        Te += (double)heat_increment_f32(K, Te, rho);
        changed = true;
      }
    } else {
      double rho = Hc * K.F_H;
      const double ro = g.eta[c] * K.F_ohm * (double)jb2;
      e_ohm = ro * K.dx3;
      rho += ro;
      if ((K.physics & P_HEATING) && rho != 0.0) {  // rho = 0 leaves T as it is
        Te = heated(K, Te, rho);
        changed = true;
      }
    }
    // e-i equilibration over the step (App. A): with a = rate_e dt and
    // b = rate_i dt frozen, the gap d = T_e - T_i decays by exp(-(a + b)) and
    // b T_e + a T_i is kept
    if (K.physics & P_EI) {
      double Ti = g.Ti[c];
      const double d = Te - Ti;
      const double a = K.ei_a / pow(Te * K.ei_mi + Ti * K.ei_me, 1.5), b = K.Zstar * a;
      if (d != 0.0 && a + b > 0.0) {
        const double f = expm1(-(a + b)) / (a + b);
        Te += a * d * f;
        Ti -= b * d * f;
        g.Ti[c] = Ti;
        if (K.physics & P_FSIGMA) g.Fsig[c] = R(1.0 + K.fs_q * (0.5 * log(Ti) + K.fs_c));
        changed = true;
      }
    }
    if (changed) {  // eta(T) follows T_e
      const double e = resistivity(K, Te);
      g.T[c] = Te;
      g.eta[c] = e;
      if constexpr (sizeof(R) == 4) g.eta_r[c] = R(e);
    }
  }
  return e_ohm;
}

}  // namespace hpic
