// Host side of the C-ABI in include/hpic.h: context, device buffers, the
// folding of the paper's SI coefficients into normalised kernel constants,
// and the per-step launch sequence.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

namespace {

// CODATA 2018 SI values; mu0 taken as 1/(eps0 c^2)
constexpr double QE = 1.602176634e-19;
constexpr double ME = 9.1093837015e-31;
constexpr double CL = 299792458.0;
constexpr double EPS0 = 8.8541878128e-12;
constexpr double HPL = 6.62607015e-34;
constexpr double KB = 1.380649e-23;
constexpr double PI = 3.14159265358979323846;
constexpr double HBAR = HPL / (2.0 * PI);
constexpr double MU0 = 1.0 / (EPS0 * CL * CL);
constexpr double MC2 = ME * CL * CL;
constexpr double AMU = 1.66053906660e-27;  // atomic mass constant (kg)
constexpr double A_BOHR = 5.29177210903e-11;

thread_local std::string g_create_error;

}  // namespace

void hpic::set_global_error(const char *msg) { g_create_error = msg; }


namespace {

int fail(hpic_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg; else g_create_error = msg;
  return code;
}

int cuda_fail(hpic_ctx *c, cudaError_t e, const char *where) {
  return fail(c, HPIC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                        \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);            \
  } while (0)

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

int n_rows(const hpic_ctx *c) { return c->run.n_Ebins + 2; }
long long hist_len(const hpic_ctx *c) { return (long long)n_rows(c) * c->run.n_thbins; }

// electrons the scheduled laser will inject in all
long long injection_total(const hpic_ctx *c) {
  if (!c->have_laser) return 0;
  if (c->K.weighted) return c->K.per_cell * c->K.n_inj_cells * c->K.n_inj_steps;
  return c->K.n_macro;
}

// one resident wave of the field and heating kernels (or fewer blocks)
int field_blocks(const hpic_ctx *c, long long nodes) {
  const long long want = (nodes + 255) / 256;
  const long long cap = (long long)c->sm_count * hpic::kFieldBlocksPerSm;
  long long g = want < cap ? want : cap;
  return (int)(g < 1 ? 1 : g);
}

int grid_blocks(const hpic_ctx *c, long long work) {
  const long long want = (work + 255) / 256;
  const long long cap = (long long)c->sm_count * 8;
  long long g = want < cap ? want : cap;
  return (int)(g < 1 ? 1 : g);
}

size_t particle_bytes(const hpic_ctx *c, long long stride) {
  return (size_t)stride * (8 * c->rsz + sizeof(uint32_t));  // 7 reals, weight, id
}

int read_counters(hpic_ctx *ctx, hpic::Counters *h) {
  CK(cudaMemcpyAsync(h, ctx->cnt, sizeof(*h), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return HPIC_OK;
}

int write_counters(hpic_ctx *ctx, const hpic::Counters *h) {
  CK(cudaMemcpyAsync(ctx->cnt, h, sizeof(*h), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return HPIC_OK;
}

// grow particle storage to hold `need` slots, keeping the first n
int reserve(hpic_ctx *ctx, long long need) {
  if (need <= ctx->cap) return HPIC_OK;
  ctx->keys_step = -1;  // the key buffers are reallocated
  if (ctx->owner) return fail(ctx, HPIC_ENOMEM, "more particles than the target's slots in the batch");
  hpic::Counters h;
  int rc = read_counters(ctx, &h);
  if (rc) return rc;
  const long long cap = round_up(need < 1024 ? 1024 : need, 64);
  void *nb[2] = {nullptr, nullptr};
  uint32_t *nk = nullptr;
  for (int b = 0; b < 2; ++b) {
    if (cudaMalloc(&nb[b], particle_bytes(ctx, cap)) != cudaSuccess) {
      cudaGetLastError();
      if (nb[0]) cudaFree(nb[0]);
      return fail(ctx, HPIC_ENOMEM, "particle storage allocation failed");
    }
  }
  if (cudaMalloc(&nk, 2 * cap * sizeof(uint32_t)) != cudaSuccess) {  // sort keys, then ranks
    cudaGetLastError();
    cudaFree(nb[0]);
    cudaFree(nb[1]);
    return fail(ctx, HPIC_ENOMEM, "sort key allocation failed");
  }
  if (ctx->pbuf[ctx->cur] && h.n > 0) {
    const size_t so = (size_t)ctx->stride, sn = (size_t)cap;
    char *src = static_cast<char *>(ctx->pbuf[ctx->cur]);
    char *dst = static_cast<char *>(nb[0]);
    for (int a = 0; a < 8; ++a)
      CK(cudaMemcpyAsync(dst + a * sn * ctx->rsz, src + a * so * ctx->rsz, h.n * ctx->rsz,
                         cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dst + 8 * sn * ctx->rsz, src + 8 * so * ctx->rsz, h.n * sizeof(uint32_t),
                       cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  cudaFree(ctx->pbuf[0]);
  cudaFree(ctx->pbuf[1]);
  cudaFree(ctx->keys);
  ctx->pbuf[0] = nb[0];
  ctx->pbuf[1] = nb[1];
  ctx->keys = nk;
  ctx->cur = 0;
  ctx->cap = cap;
  ctx->stride = cap;
  return HPIC_OK;
}

}  // namespace

// fold the paper's SI coefficients of one target into normalised constants
void hpic::fold(const hpic_target_desc &t, const hpic_run_params &r, const hpic_laser_desc *laser,
                Consts &K) {
  const double dx = t.dx_m, dt = r.dt_s, Z = t.Z, ni = t.n_i_m3;
  K.weighted = 0;  // set below for the Gaussian envelope; inj_cells is kept
  K.moore = 0;
  K.per_cell = K.n_inj_cells = 0;
  K.g_c = K.t_pk = K.g_min = K.inj_unit = 0.0;
  K.nx = t.nx; K.ny = t.ny; K.nz = t.nz;
  K.nvec = (long long)(t.nx + 1) * (t.ny + 1) * (t.nz + 1);
  K.ncell = (long long)t.nx * t.ny * t.nz;
  K.nti = (t.nx + 3) / 4;
  K.ntj = (t.ny + 3) / 4;
  K.ntk = (t.nz + 3) / 4;
  K.nkeys = (long long)K.nti * K.ntj * K.ntk * 64;
  K.cdt_dx = CL * dt / dx;
  // per element s (0: the target's own, then the compound's extra ones)
  K.n_solids = 1 + t.n_extra;
  double Kb = 0.0, ne_tot = 0.0, nz1 = 0.0, nz2 = 0.0, ni_tot = 0.0;
  for (int s = 0; s < 4; ++s) {
    K.K_ion[s] = K.L_I[s] = K.K_sc[s] = K.K_lg[s] = K.ne_frac[s] = K.Tp_fac_s[s] = 0.0;
  }
  for (int s = 0; s < K.n_solids; ++s) {
    const double Zs = s ? t.extra[s - 1].Z : Z, ns = s ? t.extra[s - 1].n_i_m3 : ni;
    const double Is = s ? t.extra[s - 1].I_ex_J : t.I_ex_J, Zss = s ? t.extra[s - 1].Zstar : t.Zstar;
    // Eq. (5): S v dt = Z n_i e^4 dt / (4 pi eps0^2 m_e v) [bracket]
    K.K_ion[s] = Zs * ns * std::pow(QE, 4) * dt / (4.0 * PI * EPS0 * EPS0 * ME * CL) / MC2;
    K.L_I[s] = std::log(MC2 / Is);
    // Eq. (B4) with p = m_e c u
    K.K_sc[s] = Zs * Zs * std::pow(QE, 4) * ns * dt / (2.0 * PI * EPS0 * EPS0 * ME * ME * std::pow(CL, 3));
    K.K_lg[s] = 4.0 * EPS0 * HPL * CL / (std::cbrt(Zs) * QE * QE);
    // Eq. (4) per unit gamma; the elements' emission rates add
    const double Lrad = std::log(5.6 * PI * EPS0 * HBAR * CL / (std::cbrt(Zs) * QE * QE));
    Kb += std::pow(QE, 6) * ns * Zs * Zs * Lrad /
          (12.0 * PI * PI * PI * std::pow(EPS0, 3) * ME * std::pow(CL, 3) * HBAR);
    K.ne_frac[s] = Zs * ns;  // normalised below
    K.Tp_fac_s[s] = (KB / QE) * std::pow(Zs, -4.0 / 3.0);
    ne_tot += Zs * ns;
    nz1 += Zss * ns;
    nz2 += Zss * Zss * ns;
    ni_tot += ns;
  }
  for (int s = 0; s < K.n_solids; ++s) K.ne_frac[s] /= ne_tot;
  // sigma_tot n_i v dt = boost Kb c dt/mc2 * (u/eps) G(u0)
  K.K_tau = r.brem_boost * Kb * CL * dt / MC2;
  K.k_min = r.k_min_J / MC2;
  K.boost = r.brem_boost;
  K.inv_boost = 1.0 / r.brem_boost;
  K.E_cut = r.E_cut_J / MC2;
  K.sigma_dtheta = r.sigma_dtheta_rad;
  K.n_E = r.n_Ebins;
  K.n_th = r.n_thbins;
  K.tE_min = r.tally_Emin_J / MC2;
  K.tE_max = r.tally_Emax_J / MC2;
  K.inv_dlogE = r.n_Ebins / std::log(r.tally_Emax_J / r.tally_Emin_J);
  K.ce_thr = r.ce_threshold_J / MC2;
  K.max_history = r.max_history;
  K.t_rows = r.table_rows;
  K.t_cols = r.table_cols;
  K.t_inv_dlog = (r.table_rows - 1) / std::log(r.table_Emax_J / r.k_min_J);
  // Eqs. (A2)-(A3) in normalised fields
  K.F_curl = r.curlB_term ? 1.0 / (CL * dx * MU0) : 0.0;
  K.F_j = QE * QE * dt / (ME * dx * dx * dx);
  // Eqs. (A4)-(A8)
  K.F_ohm = std::pow(QE * CL / (dx * dx * dx), 2) * dt;
  K.F_H = MC2 / (dx * dx * dx);
  K.dx3 = dx * dx * dx;
  K.heat_den = K.n_solids == 1 ? Z * ni * KB : ne_tot * KB;
  K.Tp_fac = (KB / QE) * std::pow(Z, -4.0 / 3.0);
  // Eqs. (A4)-(A6); a compound's free-electron density sum Z* n_i, e-i
  // collision density sum Z*^2 n_i and total ion density
  K.eta_num = K.n_solids == 1 ? t.lambda2 * ME / (t.Zstar * ni * QE * QE)
                              : t.lambda2 * ME / (nz1 * QE * QE);
  K.A_hot = 128.0 * PI * EPS0 * EPS0 / (3.0 * std::pow(QE, 4)) * std::sqrt(ME / (2.0 * PI)) /
            ((K.n_solids == 1 ? t.Zstar * t.Zstar * ni : nz2) * t.lnLambda);
  K.B_cold = std::cbrt(3.0 / (4.0 * PI * (K.n_solids == 1 ? ni : ni_tot))) * t.lambda1 *
             std::sqrt(ME / 3.0);
  K.eta_max = t.eta_max_ohm_m;
  K.lambda1 = t.lambda1;
  K.eta_hot_c = K.eta_num / K.A_hot;
  K.eta_cold_c = t.lambda1 > 0.0 ? K.eta_num / K.B_cold : 0.0;
  // eta = eta_max exactly while tau <= eta_num/eta_max: tau_hot = A_hot (k T)^1.5
  // grows with T, tau_cold = B_cold/sqrt(k T) falls; the band is narrowed by a
  // relative 1e-6 so that inside it the full formula is capped with room to spare
  {
    const double X = K.eta_num / K.eta_max;
    const double T_hot = std::pow(X / K.A_hot, 2.0 / 3.0) / KB;
    const double T_cold = t.lambda1 > 0.0 ? std::pow(K.B_cold / X, 2.0) / KB : 0.0;
    K.eta_Tlo = T_cold * (1.0 + 1e-6);
    K.eta_Thi = T_hot * (1.0 - 1e-6);
  }
  // App. B: F_sigma = 1 + ln(lambda_D/a_s)/ln(a_s m_e c/hbar) (Z*/Z)^2 with
  // ln lambda_D = ln(T_i)/2 + ln(eps0 k_B/(n_i Z*^2 e^2))/2
  {
    const double a_s = 1.4 * A_BOHR * std::pow(Z, -1.0 / 3.0);
    const double q = (t.Zstar / Z) * (t.Zstar / Z);
    K.fs_q = q / std::log(a_s * ME * CL / HBAR);
    K.fs_c = 0.5 * std::log(EPS0 * KB / (ni * t.Zstar * t.Zstar * QE * QE)) - std::log(a_s);
  }
  // App. A: rate_e dt = Z*^2 e^4 n_i dt 2/(3 (2 pi k_B)^(3/2)) sqrt(m_e m_i) lnL
  // / (eps0^2 (T_e m_i + T_i m_e)^(3/2)), masses in u
  K.ei_mi = t.A_ion;
  K.ei_me = ME / AMU;
  K.Zstar = t.Zstar;
  K.ei_a = t.Zstar * t.Zstar * std::pow(QE, 4) * ni * dt * 2.0 /
           (3.0 * std::pow(2.0 * PI * KB, 1.5)) * std::sqrt(K.ei_me * t.A_ion) * t.lnLambda /
           (EPS0 * EPS0 * std::sqrt(AMU));
  K.key0 = (uint32_t)(r.seed & 0xFFFFFFFFull);
  K.key1 = (uint32_t)(r.seed >> 32);
  K.target_index = r.target_index;
  K.physics = r.physics;
  // laser-dependent terms; without a laser a0 = 0 and the weight is 1
  double a0 = 0.0, w = 1.0;
  if (laser) {
    const hpic_laser_desc &l = *laser;
    a0 = 8.5e-6 * std::sqrt(l.I0_Wm2 * l.lambda_m * l.lambda_m);  // Eq. (1)
    if (l.n_macro > 0 && a0 > 0.0) {
      const double N_real = l.eta_l2e * l.I0_Wm2 * PI * l.spot_radius_m * l.spot_radius_m *
                            l.t_inj_s / (a0 * MC2);  // Eq. (B1) summed, flat-top
      w = N_real / (double)l.n_macro;
    }
    K.spot_r = l.spot_radius_m / dx;
    K.spot_y = l.spot_y_m / dx;
    K.spot_z = l.spot_z_m / dx;
    K.omc_cone = 2.0 * std::pow(std::sin(0.5 * l.cone_half_angle_rad), 2);
    K.n_macro = l.n_macro;
    long long S = std::llround(l.t_inj_s / dt);
    K.n_inj_steps = S < 1 ? 1 : S;
    K.moore = l.moore_cap != 0;
    if (l.envelope == HPIC_ENV_GAUSS) {
      // App. B: g = exp(-4 ln2 ((s + 1/2) dt - t_pk)^2 / t_fwhm^2), g(0) = g_min
      K.weighted = 1;
      K.per_cell = l.per_cell;
      K.n_inj_cells = (long long)injection_cells(t, l).size();
      K.g_c = 4.0 * std::log(2.0) * (dt / l.t_fwhm_s) * (dt / l.t_fwhm_s);
      K.t_pk = 0.5 * l.t_fwhm_s * std::sqrt(std::log(1.0 / l.g_min) / std::log(2.0)) / dt;
      K.g_min = l.g_min;
      K.inj_unit = a0 > 0.0 ? l.I0_Wm2 * dx * dx * dt * l.eta_l2e / (a0 * MC2 * l.per_cell) : 0.0;
      long long s = 0;  // steps while g >= g_min (g rises from g_min, peaks, falls)
      while (std::exp(-K.g_c * (s + 0.5 - K.t_pk) * (s + 0.5 - K.t_pk)) >= l.g_min) ++s;
      K.n_inj_steps = s + 1;  // one more: the kernel itself decides on g
      K.n_macro = 0;
      w = 1.0;
    }
  } else {
    K.n_macro = 0;
    K.n_inj_steps = 1;
  }
  K.w = w;
  K.T_hot = a0;
  K.eps_esc = r.kappa_esc * a0;
  K.du_reflux = r.kappa_tnsa * a0;
}

const char *hpic::check_target(const hpic_target_desc &t, const hpic_run_params &r) {
  if (t.nx < 2 || t.ny < 2 || t.nz < 2) return "each dimension must be >= 2";
  if ((long long)(t.nx + 4) * (t.ny + 4) * (t.nz + 4) >= 0x7FFFFFFFll ||
      (long long)t.nx * t.ny * t.nz >= (1ll << 27) - 1)
    return "grid too large (at most 2^27 - 2 cells)";
  if (!(t.dx_m > 0) || !(r.dt_s > 0) || CL * r.dt_s >= t.dx_m) return "need dx > c dt > 0";
  if (!(t.Z > 0) || !(t.n_i_m3 > 0) || !(t.I_ex_J > 0) || !(t.Zstar > 0) ||
      !(t.lnLambda > 0) || !(t.eta_max_ohm_m > 0) || !(t.lambda2 > 0) || !(t.T0_K > 0) ||
      t.lambda1 < 0)
    return "material parameters must be positive";
  if (r.precision != HPIC_FP64 && r.precision != HPIC_FP32_MIXED) return "unknown precision";
  if ((r.physics & HPIC_EI_EQUIL) && !(t.A_ion > 0)) return "e-i equilibration needs A_ion > 0";
  if (t.n_extra < 0 || t.n_extra > 3) return "a compound has at most three further elements";
  for (int s = 0; s < t.n_extra; ++s)
    if (!(t.extra[s].Z > 0) || !(t.extra[s].n_i_m3 > 0) || !(t.extra[s].I_ex_J > 0) ||
        !(t.extra[s].Zstar > 0))
      return "compound element parameters must be positive";
  if (t.n_extra > 0 && (r.physics & (HPIC_FSIGMA | HPIC_EI_EQUIL)))
    return "F_sigma and e-i equilibration are defined for single-element targets only";
  if (!(r.brem_boost > 0) || !(r.k_min_J > 0) || !(r.E_cut_J > 0) ||
      !(r.table_Emax_J > r.k_min_J) || r.table_rows < 2 || r.table_cols < 2 ||
      r.n_Ebins < 1 || r.n_thbins < 1 || !(r.tally_Emax_J > r.tally_Emin_J) ||
      !(r.tally_Emin_J > 0) || r.max_history < 0 || r.sort_interval < 0 ||
      r.kappa_esc < 0 || r.kappa_tnsa < 0 || r.sigma_dtheta_rad < 0 ||
      (r.physics & ~(HPIC_ALL | HPIC_UNBOUNDED | HPIC_FSIGMA | HPIC_EI_EQUIL)) != 0)
    return "run parameters out of range";
  return nullptr;
}

const char *hpic::check_laser(const hpic_laser_desc &l, const hpic_target_desc &t) {
  if (!(l.I0_Wm2 >= 0) || !(l.lambda_m > 0) || !(l.eta_l2e >= 0) || !(l.spot_radius_m >= 0) ||
      !(l.t_inj_s >= 0) || l.n_macro < 0 || l.n_macro >= 0xFFFFFFFFll ||
      !(l.cone_half_angle_rad >= 0) || l.cone_half_angle_rad > PI)
    return "laser parameters out of range";
  if ((l.envelope != HPIC_ENV_FLAT && l.envelope != HPIC_ENV_GAUSS) ||
      (l.moore_cap != 0 && l.moore_cap != 1))
    return "unknown envelope or Moore flag";
  if (l.envelope == HPIC_ENV_GAUSS) {
    if (l.per_cell < 1 || !(l.r_fwhm_m > 0) || !(l.t_fwhm_s > 0) || !(l.f_min > 0 && l.f_min <= 1) ||
        !(l.g_min > 0 && l.g_min < 1))
      return "Gaussian envelope parameters out of range";
    return nullptr;  // only face cells inject: nothing has to fit
  }
  const double Ly = t.ny * t.dx_m, Lz = t.nz * t.dx_m;
  if (l.spot_y_m - l.spot_radius_m < 0 || l.spot_y_m + l.spot_radius_m > Ly ||
      l.spot_z_m - l.spot_radius_m < 0 || l.spot_z_m + l.spot_radius_m > Lz)
    return "injection disc does not fit on the x = 0 face";
  return nullptr;
}

namespace {

void fold_constants(hpic_ctx *c) {
  hpic::fold(c->tgt, c->run, c->have_laser ? &c->laser : nullptr, c->K);
}

double eta_host(const hpic_ctx *c, double T) { return hpic::eta_of(c->K, T); }

}  // namespace

double hpic::eta_of(const Consts &K, double T) {
  const double kT = KB * T;
  double tau = K.A_hot * kT * std::sqrt(kT);
  if (K.lambda1 > 0.0) {
    const double tc = K.B_cold / std::sqrt(kT);
    tau = tc > tau ? tc : tau;
  }
  const double e = K.eta_num / tau;
  return e < K.eta_max ? e : K.eta_max;
}

double hpic::fsigma_of(const Consts &K, double Ti) {
  return 1.0 + K.fs_q * (0.5 * std::log(Ti) + K.fs_c);
}

// App. B: the x = 0 face cells (k outer, j inner) whose centre has
// f(r) = exp(-4 ln2 r^2/r_fwhm^2) >= f_min, with sqrt(f)
std::vector<hpic::InjCell> hpic::injection_cells(const hpic_target_desc &t,
                                                 const hpic_laser_desc &l) {
  std::vector<InjCell> out;
  if (l.envelope != HPIC_ENV_GAUSS) return out;
  for (int k = 0; k < t.nz; ++k)
    for (int j = 0; j < t.ny; ++j) {
      const double y = (j + 0.5) * t.dx_m - l.spot_y_m, z = (k + 0.5) * t.dx_m - l.spot_z_m;
      const double f = std::exp(-4.0 * std::log(2.0) * (y * y + z * z) / (l.r_fwhm_m * l.r_fwhm_m));
      if (f >= l.f_min) out.push_back(InjCell{j, k, std::sqrt(f)});
    }
  return out;
}

namespace {

void destroy_all(hpic_ctx *c) {
  cudaFree(c->pbuf[0]);
  cudaFree(c->pbuf[1]);
  cudaFree(c->keys);
  cudaFree(c->counts);
  cudaFree(c->partials);
  cudaFree(c->fields);
  cudaFree(c->T);
  cudaFree(c->eta);
  cudaFree(c->eta_r);
  cudaFree(c->Ti);
  cudaFree(c->Fsig);
  cudaFree(c->inj_cells);
  cudaFree(c->H);
  cudaFree(c->tal);
  cudaFree(c->hist);
  cudaFree(c->history);
  cudaFree(c->scratch);
  cudaFree(c->t64);
  cudaFree(c->t32);
  cudaFree(c->cnt);
  cudaFree(c->xfer);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
}

double grid_scale(const hpic_ctx *c, int which) {
  const double dx = c->tgt.dx_m, dt = c->run.dt_s;
  switch (which) {
    case HPIC_GRID_EX: case HPIC_GRID_EY: case HPIC_GRID_EZ: return -ME * CL / (QE * dt);
    case HPIC_GRID_BX: case HPIC_GRID_BY: case HPIC_GRID_BZ: return -ME / (QE * dt);
    case HPIC_GRID_JX: case HPIC_GRID_JY: case HPIC_GRID_JZ: return -QE * CL / (dx * dx * dx);
    case HPIC_GRID_HEAT: return MC2;
    default: return 1.0;
  }
}

template <typename R>
int step_impl(hpic_ctx *ctx, long long nsteps) {
  auto P = [&](int b) { return pview<R>(ctx, b); };
  const hpic::GView<R> G = gview<R>(ctx);
  const hpic::TallyView tv = tview(ctx);
  const R *tab = ctx->fp32 ? reinterpret_cast<const R *>(ctx->t32)
                           : reinterpret_cast<const R *>(ctx->t64);
  const int gp = grid_blocks(ctx, ctx->cap);
  const int gg = field_blocks(ctx, ctx->K.nvec);
  const bool grid_on = !(ctx->K.physics & hpic::P_UNBOUNDED);
  for (long long s = 0; s < nsteps; ++s) {
    if (grid_on) {
      CK(cudaMemsetAsync(G.J[0], 0, 3 * ctx->vstride * ctx->rsz, ctx->stream));
      CK(cudaMemsetAsync(ctx->H, 0, ctx->K.ncell * sizeof(double), ctx->stream));
    }
    // every sort_interval steps the cell sort rides on the step: its keys
    // come from the start-of-step state one step further ahead, and the push
    // writes each electron to its sorted slot in the other buffer.  The keys,
    // ranks and counts are computed by the push of the step before when that
    // step injects nothing (the new electrons would need keys too), else by a
    // key pass at the start of the sorting step.
    const int si = ctx->run.sort_interval;
    const bool sort_now = si > 0 && (ctx->host_step + 1) % si == 0 && ctx->keys;
    const bool inject_now =
        ctx->have_laser && ctx->host_step < ctx->K.n_inj_steps && injection_total(ctx) > 0;
    const bool keys_now = si >= 2 && (ctx->host_step + 2) % si == 0 && ctx->keys && !inject_now;
    uint32_t *ranks = ctx->keys ? ctx->keys + ctx->cap : nullptr;
    hpic::SortOut<R> so{};
    hpic::KeyOut<R> ko{};
    if (sort_now) {
      if (ctx->keys_step == ctx->host_step) {
        ctx->launches += hpic::launch_scan(ctx->counts, ctx->K.nkeys + 1, ctx->partials, ctx->stream);
      } else {
        ctx->launches += hpic::launch_sort_keys<R>(ctx->K, P(ctx->cur), ctx->cnt, ctx->keys, ranks,
                                                   ctx->counts, ctx->partials, gp, ctx->stream,
                                                   hpic::sort_lead(si) + 1.0);
      }
      so.dst = P(ctx->cur ^ 1);
      so.keys = ctx->keys;
      so.ranks = ranks;
      so.offsets = ctx->counts;
    } else if (keys_now) {
      CK(cudaMemsetAsync(ctx->counts, 0, (ctx->K.nkeys + 1) * sizeof(uint32_t), ctx->stream));
      ko.keys = ctx->keys;
      ko.ranks = ranks;
      ko.counts = ctx->counts;
      ko.lead = R((hpic::sort_lead(si) + 1.0) * ctx->K.cdt_dx);
    }
    ctx->keys_step = keys_now ? ctx->host_step + 1 : -1;
    if (ctx->prof) {
      if (ctx->ev_used + 2 > ctx->ev.size()) {
        for (int q = 0; q < 64; ++q) {
          cudaEvent_t e;
          CK(cudaEventCreate(&e));
          ctx->ev.push_back(e);
        }
      }
      CK(cudaEventRecord(ctx->ev[ctx->ev_used], ctx->stream));
    }
    hpic::launch_push<R>(ctx->K, P(ctx->cur), G, tab, ctx->cnt, tv,
                         ctx->sm_count * hpic::push_blocks_per_sm<R>(), ctx->stream, so, ko);
    ctx->launches += 1;
    if (ctx->prof) {
      CK(cudaEventRecord(ctx->ev[ctx->ev_used + 1], ctx->stream));
      ctx->ev_used += 2;
      ctx->prof_launches += 1;
    }
    if (grid_on && (ctx->K.physics & hpic::P_FIELDS)) {
      hpic::launch_efield<R>(ctx->K, G, gg, ctx->stream);
      ctx->launches += 1;
    }
    if (grid_on) {
      hpic::launch_bheat<R>(ctx->K, G, tv, gg, ctx->stream);
      ctx->launches += 1;
    }
    if (sort_now) {  // the kept electrons now fill the front of the other buffer
      ctx->launches += hpic::launch_sort_finish(ctx->K, ctx->cnt, ctx->counts, ctx->stream);
      ctx->cur ^= 1;
    }
    if (inject_now) {
      const long long S = ctx->K.n_inj_steps, N = ctx->K.n_macro, st = ctx->host_step;
      const long long c = ctx->K.weighted ? ctx->K.per_cell * ctx->K.n_inj_cells
                                          : (N * (st + 1)) / S - (N * st) / S;
      hpic::launch_inject<R>(ctx->K, P(ctx->cur), ctx->cnt, ctx->cap, tv,
                             grid_blocks(ctx, c > 0 ? c : 1), ctx->stream);
      ctx->launches += 1;
    }
    hpic::launch_advance(ctx->cnt, ctx->cap, ctx->stream);
    ctx->launches += 1;
    ctx->host_step += 1;
    CK(cudaGetLastError());
  }
  return HPIC_OK;
}

template <typename R>
int sort_impl(hpic_ctx *ctx) {
  ctx->launches += hpic::launch_sort<R>(ctx->K, pview<R>(ctx, ctx->cur), pview<R>(ctx, ctx->cur ^ 1),
                                        ctx->cnt, ctx->keys, ctx->counts, ctx->partials,
                                        grid_blocks(ctx, ctx->cap), ctx->stream, 0.0);
  ctx->cur ^= 1;
  CK(cudaGetLastError());
  return HPIC_OK;
}

// device scratch of at least `bytes` for the host transfers
int xfer_reserve(hpic_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->xfer_bytes) return HPIC_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  cudaFree(ctx->xfer);
  ctx->xfer = nullptr;
  ctx->xfer_bytes = 0;
  const size_t want = (bytes + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
  if (cudaMalloc(&ctx->xfer, want) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, HPIC_ENOMEM, "transfer scratch allocation failed");
  }
  ctx->xfer_bytes = want;
  return HPIC_OK;
}

int xfer_grid(const hpic_ctx *ctx, long long n) {
  const long long want = (n + 255) / 256, cap = 8LL * ctx->sm_count;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

// The live electrons in storage order.  On the device: the live slots are
// counted per chunk and scanned, then each array is compacted and
// converted to double (positions back to metres) into the transfer scratch
// and copied to the caller's array; the ids likewise.
template <typename R>
int read_particles_impl(hpic_ctx *ctx, double *x, double *y, double *z, double *ux, double *uy,
                        double *uz, double *tau, uint32_t *id, int64_t cap, int64_t *n_out) {
  hpic::Counters h;
  int rc = read_counters(ctx, &h);
  if (rc) return rc;
  const long long n = h.n;
  const long long nb = hpic::xfer_chunks(n);
  const size_t cc_bytes = (size_t)(nb + 1) * sizeof(uint32_t);
  const size_t data_off = (cc_bytes + 255) & ~(size_t)255;
  rc = xfer_reserve(ctx, data_off + (size_t)(n > 0 ? n : 1) * sizeof(double));
  if (rc) return rc;
  uint32_t *cc = static_cast<uint32_t *>(ctx->xfer);
  void *data = static_cast<char *>(ctx->xfer) + data_off;
  const hpic::PView<R> P = pview<R>(ctx, ctx->cur);
  hpic::launch_live_scan(P.id, n, cc, ctx->stream);
  uint32_t live32 = 0;
  CK(cudaMemcpyAsync(&live32, cc + nb, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const long long live = live32;
  *n_out = live;
  if (live > cap) return fail(ctx, HPIC_EINVAL, "output capacity below the live particle count");
  const double dx = ctx->tgt.dx_m;
  const R *src[7] = {P.x, P.y, P.z, P.ux, P.uy, P.uz, P.tau};
  double *dst[7] = {x, y, z, ux, uy, uz, tau};
  for (int q = 0; q < 7; ++q) {
    if (!dst[q] || live == 0) continue;
    hpic::launch_compact<R, double>(src[q], P.id, n, cc, q < 3 ? dx : 1.0,
                                    static_cast<double *>(data), ctx->stream);
    CK(cudaMemcpyAsync(dst[q], data, live * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (id && live > 0) {
    hpic::launch_compact<uint32_t, uint32_t>(P.id, P.id, n, cc, 1.0,
                                             static_cast<uint32_t *>(data), ctx->stream);
    CK(cudaMemcpyAsync(id, data, live * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  CK(cudaGetLastError());
  return HPIC_OK;
}

// Replace the population with n host electrons.  Every array is copied to
// the transfer scratch as it is; a first pass checks the positions and ids
// on the device (nothing is written to the state unless all pass), a second
// converts each array into the particle storage.
template <typename R>
int load_particles_impl(hpic_ctx *ctx, int64_t n, const double *x, const double *y,
                        const double *z, const double *ux, const double *uy, const double *uz,
                        const double *tau, const uint32_t *id) {
  const double dx = ctx->tgt.dx_m;
  const int nn[3] = {ctx->tgt.nx, ctx->tgt.ny, ctx->tgt.nz};
  const int unbounded = (ctx->K.physics & hpic::P_UNBOUNDED) != 0;
  const size_t data_off = 256;  // the error count first
  int rc = xfer_reserve(ctx, data_off + (size_t)(n > 0 ? n : 1) * sizeof(double));
  if (rc) return rc;
  unsigned *bad = static_cast<unsigned *>(ctx->xfer);
  double *data = reinterpret_cast<double *>(static_cast<char *>(ctx->xfer) + data_off);
  const int grid = xfer_grid(ctx, n);
  CK(cudaMemsetAsync(bad, 0, sizeof(unsigned), ctx->stream));
  const double *src[7] = {x, y, z, ux, uy, uz, tau};
  if (n > 0) {
    for (int a = 0; a < 3; ++a) {
      CK(cudaMemcpyAsync(data, src[a], n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      hpic::launch_load_convert<R>(data, n, 1.0, static_cast<R *>(nullptr), 1, dx, (double)nn[a],
                                   unbounded, bad, grid, ctx->stream);
    }
    CK(cudaMemcpyAsync(data, id, n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
    hpic::launch_check_ids(reinterpret_cast<const uint32_t *>(data), n, bad, grid, ctx->stream);
  }
  unsigned nbad = 0;
  CK(cudaMemcpyAsync(&nbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  if (nbad) {
    // the host's own reading of the first offence, for the message
    for (int64_t i = 0; i < n; ++i) {
      if (id[i] == hpic::kDead) return fail(ctx, HPIC_EINVAL, "id 0xFFFFFFFF is reserved");
      for (int a = 0; a < 3; ++a) {
        const double X = src[a][i] / dx;
        if (unbounded ? !std::isfinite(X) : !(X >= 0.0 && X <= (double)nn[a]))
          return fail(ctx, HPIC_EINVAL, "particle position outside the target");
      }
    }
    return fail(ctx, HPIC_EINVAL, "particle position outside the target");
  }
  const long long extra = injection_total(ctx);
  rc = reserve(ctx, n + extra);
  if (rc) return rc;
  const hpic::PView<R> P = pview<R>(ctx, ctx->cur);
  R *dst[7] = {P.x, P.y, P.z, P.ux, P.uy, P.uz, P.tau};
  if (n > 0) {
    CK(cudaMemcpyAsync(P.id, id, n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
    for (int q = 0; q < 7; ++q) {
      CK(cudaMemcpyAsync(data, src[q], n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      hpic::launch_load_convert<R>(data, n, q < 3 ? 1.0 / dx : 1.0, dst[q], 0, dx, 0.0, unbounded,
                                   bad, grid, ctx->stream);
    }
    if (ctx->K.weighted)  // the envelope's weights come from hpic_load_weights
      hpic::launch_fill<R>(P.w, n, (R)ctx->K.w, grid, ctx->stream);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
  }
  hpic::Counters h;
  rc = read_counters(ctx, &h);
  if (rc) return rc;
  h.n = n;
  return write_counters(ctx, &h);
}

bool valid_grid(int which) { return which >= HPIC_GRID_T && which <= HPIC_GRID_TI; }

// cell-centred double arrays: T, eta, drag heat, T_i
double *cell_array(const hpic_ctx *ctx, int which) {
  switch (which) {
    case HPIC_GRID_T: return ctx->T;
    case HPIC_GRID_ETA: return ctx->eta;
    case HPIC_GRID_HEAT: return ctx->H;
    case HPIC_GRID_TI: return ctx->Ti;
    default: return nullptr;
  }
}

// device array of a vector-field component (HPIC_GRID_EX .. HPIC_GRID_JZ)
void *vector_array(const hpic_ctx *ctx, int which) {
  const int slot = which - HPIC_GRID_EX;  // 0..8: E, B, J
  char *base = static_cast<char *>(slot < 6 ? ctx->fields : ctx->jfield);
  return base + (slot % 6) * ctx->vstride * ctx->rsz;
}

// entry points that step or reshape a context are the batch's business
int refuse_batch_target(hpic_ctx *ctx) {
  return fail(ctx, HPIC_ESTATE, "this context is a target of a batch: use the hpic_batch_* calls");
}

}  // namespace

extern "C" {

int hpic_init_target(hpic_ctx **out, const hpic_target_desc *t, const hpic_run_params *r,
                     int device, void *cuda_stream) {
  if (!out) return fail(nullptr, HPIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!t || !r) return fail(nullptr, HPIC_EINVAL, "target or run params NULL");
  if (const char *why = hpic::check_target(*t, *r)) return fail(nullptr, HPIC_EINVAL, why);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(nullptr, HPIC_ECUDA, "no such CUDA device");
  }
  hpic_ctx *ctx = new hpic_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->tgt = *t;
  ctx->run = *r;
  ctx->fp32 = r->precision == HPIC_FP32_MIXED;
  ctx->rsz = ctx->fp32 ? 4 : 8;
  auto bail = [&](int code) {
    const std::string m = ctx->err;
    destroy_all(ctx);
    delete ctx;
    g_create_error = m;
    return code;
  };
  if (cudaSetDevice(device) != cudaSuccess) { cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice"); return bail(HPIC_ECUDA); }
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (const cudaError_t e = hpic::prepare_push(); e != cudaSuccess) {
    cuda_fail(ctx, e, "push kernel shared memory");
    return bail(HPIC_ECUDA);
  }
  fold_constants(ctx);
  const hpic::Consts &K = ctx->K;
  ctx->vstride = round_up(K.nvec + 4, 64);
  const long long m = K.nkeys + 1;
  bool ok = cudaMalloc(&ctx->fields, 9 * ctx->vstride * ctx->rsz) == cudaSuccess &&
            cudaMalloc(&ctx->T, K.ncell * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ctx->eta, K.ncell * sizeof(double)) == cudaSuccess &&
            (!ctx->fp32 || cudaMalloc(&ctx->eta_r, K.ncell * sizeof(float)) == cudaSuccess) &&
            cudaMalloc(&ctx->Ti, K.ncell * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ctx->Fsig, K.ncell * ctx->rsz) == cudaSuccess &&
            cudaMalloc(&ctx->H, K.ncell * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ctx->counts, m * sizeof(uint32_t)) == cudaSuccess &&
            cudaMalloc(&ctx->partials, hpic::scan_partials(m) * sizeof(uint32_t)) == cudaSuccess &&
            cudaMalloc(&ctx->tal, hpic::T_COUNT * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ctx->hist, 2 * hist_len(ctx) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ctx->history, (r->max_history > 0 ? r->max_history : 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ctx->scratch, 2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ctx->t64, (size_t)r->table_rows * r->table_cols * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&ctx->t32, (size_t)r->table_rows * r->table_cols * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&ctx->cnt, sizeof(hpic::Counters)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    fail(ctx, HPIC_ENOMEM, "device allocation failed");
    return bail(HPIC_ENOMEM);
  }
  ctx->jfield = static_cast<char *>(ctx->fields) + 6 * ctx->vstride * ctx->rsz;
  int rc = reserve(ctx, 1024);
  if (rc) return bail(rc);
  cudaStream_t st = ctx->stream;
  std::vector<double> T0(K.ncell, t->T0_K), E0(K.ncell, eta_host(ctx, t->T0_K));
  std::vector<float> E0f(ctx->fp32 ? K.ncell : 0, (float)E0[0]);
  const double F0 = hpic::fsigma_of(K, t->T0_K);
  std::vector<float> F0f(ctx->fp32 ? K.ncell : 0, (float)F0);
  std::vector<double> F0d(ctx->fp32 ? 0 : K.ncell, F0);
  if (cudaMemsetAsync(ctx->fields, 0, 9 * ctx->vstride * ctx->rsz, st) != cudaSuccess ||
      cudaMemsetAsync(ctx->H, 0, K.ncell * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(ctx->tal, 0, hpic::T_COUNT * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(ctx->hist, 0, 2 * hist_len(ctx) * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(ctx->history, 0, (r->max_history > 0 ? r->max_history : 1) * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(ctx->cnt, 0, sizeof(hpic::Counters), st) != cudaSuccess ||
      cudaMemcpyAsync(ctx->T, T0.data(), K.ncell * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(ctx->eta, E0.data(), K.ncell * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (ctx->fp32 && cudaMemcpyAsync(ctx->eta_r, E0f.data(), K.ncell * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      cudaMemcpyAsync(ctx->Ti, T0.data(), K.ncell * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(ctx->Fsig, ctx->fp32 ? (const void *)F0f.data() : (const void *)F0d.data(),
                      K.ncell * ctx->rsz, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cuda_fail(ctx, cudaGetLastError(), "initialisation");
    return bail(HPIC_ECUDA);
  }
  hpic::launch_table(K, r->k_min_J / MC2, r->table_Emax_J / MC2, ctx->t64, ctx->t32, st);
  ctx->launches += 1;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    cuda_fail(ctx, e, "table build");
    return bail(HPIC_ECUDA);
  }
  *out = ctx;
  return HPIC_OK;
}

int hpic_inject_electrons(hpic_ctx *ctx, const hpic_laser_desc *l) {
  if (!ctx || !l) return fail(ctx, HPIC_EINVAL, "NULL argument");
  if (ctx->owner) return refuse_batch_target(ctx);
  if (ctx->have_laser) return fail(ctx, HPIC_ESTATE, "a laser is already scheduled");
  ctx->keys_step = -1;
  if (const char *why = hpic::check_laser(*l, ctx->tgt)) return fail(ctx, HPIC_EINVAL, why);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  hpic::Counters h;
  int rc = read_counters(ctx, &h);
  if (rc) return rc;
  const hpic_laser_desc keep = ctx->laser;
  ctx->laser = *l;
  ctx->have_laser = true;
  fold_constants(ctx);
  const long long total = injection_total(ctx);
  std::vector<hpic::InjCell> cells = hpic::injection_cells(ctx->tgt, *l);
  auto undo = [&](int code, const char *msg) {
    ctx->laser = keep;
    ctx->have_laser = false;
    fold_constants(ctx);
    return fail(ctx, code, msg);
  };
  if (h.next_id + total >= 0xFFFFFFFFll) return undo(HPIC_EINVAL, "id space exhausted");
  rc = reserve(ctx, h.n + total);
  if (rc) return undo(rc, ctx->err.c_str());
  if (!cells.empty()) {
    if (cudaMalloc(&ctx->inj_cells, cells.size() * sizeof(hpic::InjCell)) != cudaSuccess) {
      cudaGetLastError();
      return undo(HPIC_ENOMEM, "injection cell list allocation failed");
    }
    CK(cudaMemcpyAsync(ctx->inj_cells, cells.data(), cells.size() * sizeof(hpic::InjCell),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->K.inj_cells = ctx->inj_cells;
  }
  return HPIC_OK;
}

int hpic_seed_electrons(hpic_ctx *ctx, int64_t n, double mean_energy_J) {
  if (!ctx) return HPIC_EINVAL;
  if (ctx->owner) return refuse_batch_target(ctx);
  ctx->keys_step = -1;
  if (n < 0 || !(mean_energy_J > 0)) return fail(ctx, HPIC_EINVAL, "bad seeding arguments");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  hpic::Counters h;
  int rc = read_counters(ctx, &h);
  if (rc) return rc;
  if (h.next_id + n >= 0xFFFFFFFFll) return fail(ctx, HPIC_EINVAL, "id space exhausted");
  rc = reserve(ctx, h.n + n + injection_total(ctx));
  if (rc) return rc;
  if (n == 0) return HPIC_OK;
  const int grid = grid_blocks(ctx, n);
  if (ctx->fp32)
    hpic::launch_seed<float>(ctx->K, pview<float>(ctx, ctx->cur), ctx->cnt, ctx->cap, n,
                             mean_energy_J / MC2, tview(ctx), grid, ctx->stream);
  else
    hpic::launch_seed<double>(ctx->K, pview<double>(ctx, ctx->cur), ctx->cnt, ctx->cap, n,
                              mean_energy_J / MC2, tview(ctx), grid, ctx->stream);
  ctx->launches += 2;
  CK(cudaGetLastError());
  return HPIC_OK;
}

int hpic_step(hpic_ctx *ctx, int64_t n) {
  if (!ctx) return HPIC_EINVAL;
  if (ctx->owner) return refuse_batch_target(ctx);
  if (n < 0) return fail(ctx, HPIC_EINVAL, "negative step count");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  return ctx->fp32 ? step_impl<float>(ctx, n) : step_impl<double>(ctx, n);
}

int hpic_sort(hpic_ctx *ctx) {
  if (!ctx) return HPIC_EINVAL;
  if (ctx->owner) return refuse_batch_target(ctx);
  ctx->keys_step = -1;  // the sort reuses the key buffers
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  return ctx->fp32 ? sort_impl<float>(ctx) : sort_impl<double>(ctx);
}

int hpic_read_tallies(hpic_ctx *ctx, hpic_tallies *out) {
  if (!ctx || !out) return fail(ctx, HPIC_EINVAL, "NULL argument");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  CK(cudaMemsetAsync(ctx->scratch, 0, 2 * sizeof(double), ctx->stream));
  const int gp = grid_blocks(ctx, ctx->cap), gg = grid_blocks(ctx, ctx->K.nvec);
  if (ctx->fp32) {
    hpic::launch_live_energy<float>(ctx->K, pview<float>(ctx, ctx->cur), ctx->cnt, ctx->scratch, gp, ctx->stream);
    hpic::launch_field_energy<float>(ctx->K, gview<float>(ctx), ctx->scratch + 1, gg, ctx->stream);
  } else {
    hpic::launch_live_energy<double>(ctx->K, pview<double>(ctx, ctx->cur), ctx->cnt, ctx->scratch, gp, ctx->stream);
    hpic::launch_field_energy<double>(ctx->K, gview<double>(ctx), ctx->scratch + 1, gg, ctx->stream);
  }
  ctx->launches += 2;
  CK(cudaGetLastError());
  double t[hpic::T_COUNT], sc[2];
  CK(cudaMemcpyAsync(t, ctx->tal, sizeof(t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(sc, ctx->scratch, sizeof(sc), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  out->E_injected = t[hpic::T_E_INJ] * MC2;
  out->N_injected = t[hpic::T_N_INJ];
  out->W_field = t[hpic::T_W_FIELD] * MC2;
  out->E_drag = t[hpic::T_E_DRAG] * MC2;
  out->E_xray = t[hpic::T_E_XRAY] * MC2;
  out->E_xray_above = t[hpic::T_E_XRAY_ABOVE] * MC2;
  out->E_escaped = t[hpic::T_E_ESC] * MC2;
  out->E_reflux = t[hpic::T_E_REFLUX] * MC2;
  out->E_ohmic_grid = t[hpic::T_E_OHMIC];
  out->n_injected = t[hpic::T_N_INJECTED];
  out->n_escaped = t[hpic::T_N_ESC];
  out->n_refluxed = t[hpic::T_N_REFLUX];
  out->n_reflux_absorbed = t[hpic::T_N_REFLUX_ABS];
  out->n_cut = t[hpic::T_N_CUT];
  out->n_emitted = t[hpic::T_N_EMIT];
  out->particle_steps = t[hpic::T_PSTEPS];
  out->n_nonfinite = t[hpic::T_N_NONFINITE];
  out->E_live = sc[0] * MC2;
  const double bs = ME / (QE * ctx->run.dt_s);
  out->E_B_field = sc[1] * bs * bs * ctx->K.dx3 / (2.0 * MU0);
  return t[hpic::T_N_NONFINITE] > 0 ? HPIC_ENONFINITE : HPIC_OK;
}

int hpic_reset_tallies(hpic_ctx *ctx) {
  if (!ctx) return HPIC_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  CK(cudaMemsetAsync(ctx->tal, 0, hpic::T_COUNT * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->hist, 0, 2 * hist_len(ctx) * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->history, 0, (ctx->run.max_history > 0 ? ctx->run.max_history : 1) * sizeof(double), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return HPIC_OK;
}

int hpic_read_hist(hpic_ctx *ctx, double *ew, double *nw) {
  if (!ctx) return HPIC_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  const long long L = hist_len(ctx);
  if (ew) CK(cudaMemcpyAsync(ew, ctx->hist, L * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (nw) CK(cudaMemcpyAsync(nw, ctx->hist + L, L * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ew) for (long long i = 0; i < L; ++i) ew[i] *= MC2;
  return HPIC_OK;
}

int hpic_read_history(hpic_ctx *ctx, double *out) {
  if (!ctx || !out) return fail(ctx, HPIC_EINVAL, "NULL argument");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  const int L = ctx->run.max_history;
  if (L > 0) {
    CK(cudaMemcpyAsync(out, ctx->history, L * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < L; ++i) out[i] *= MC2;
  }
  return HPIC_OK;
}

int hpic_grid_len(const hpic_ctx *ctx, int which, int64_t *len) {
  if (!ctx || !len || !valid_grid(which)) return HPIC_EINVAL;
  *len = cell_array(ctx, which) ? ctx->K.ncell : ctx->K.nvec;
  return HPIC_OK;
}

int hpic_read_grid(hpic_ctx *ctx, int which, double *out) {
  if (!ctx || !out || !valid_grid(which)) return fail(ctx, HPIC_EINVAL, "bad grid request");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  int64_t L;
  hpic_grid_len(ctx, which, &L);
  const double s = grid_scale(ctx, which);
  if (const double *src = cell_array(ctx, which)) {
    CK(cudaMemcpyAsync(out, src, L * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int64_t i = 0; i < L; ++i) out[i] *= s;
    return HPIC_OK;
  }
  const char *src = static_cast<const char *>(vector_array(ctx, which));
  if (ctx->fp32) {
    std::vector<float> b(L);
    CK(cudaMemcpyAsync(b.data(), src, L * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int64_t i = 0; i < L; ++i) out[i] = (double)b[i] * s;
  } else {
    CK(cudaMemcpyAsync(out, src, L * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int64_t i = 0; i < L; ++i) out[i] *= s;
  }
  return HPIC_OK;
}

int hpic_write_grid(hpic_ctx *ctx, int which, const double *in) {
  if (!ctx || !in || !valid_grid(which)) return fail(ctx, HPIC_EINVAL, "bad grid request");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  int64_t L;
  hpic_grid_len(ctx, which, &L);
  const double s = 1.0 / grid_scale(ctx, which);
  if (double *dst = cell_array(ctx, which)) {
    std::vector<double> b(in, in + L);
    for (auto &v : b) v *= s;
    CK(cudaMemcpyAsync(dst, b.data(), L * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (which == HPIC_GRID_ETA && ctx->fp32) {  // the field solve's FP32 copy
      std::vector<float> f(b.begin(), b.end());
      CK(cudaMemcpyAsync(ctx->eta_r, f.data(), L * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
    if (which == HPIC_GRID_TI) {  // F_sigma follows T_i
      std::vector<double> F(L);
      for (int64_t i = 0; i < L; ++i) F[i] = hpic::fsigma_of(ctx->K, b[i]);
      std::vector<float> Ff(ctx->fp32 ? L : 0);
      for (size_t i = 0; i < Ff.size(); ++i) Ff[i] = (float)F[i];
      CK(cudaMemcpyAsync(ctx->Fsig, ctx->fp32 ? (const void *)Ff.data() : (const void *)F.data(),
                         L * ctx->rsz, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return HPIC_OK;
  }
  char *dst = static_cast<char *>(vector_array(ctx, which));
  if (ctx->fp32) {
    std::vector<float> b(L);
    for (int64_t i = 0; i < L; ++i) b[i] = (float)(in[i] * s);
    CK(cudaMemcpyAsync(dst, b.data(), L * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    std::vector<double> b(in, in + L);
    for (auto &v : b) v *= s;
    CK(cudaMemcpyAsync(dst, b.data(), L * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return HPIC_OK;
}

int hpic_count_particles(hpic_ctx *ctx, int64_t *n) {
  if (!ctx || !n) return fail(ctx, HPIC_EINVAL, "NULL argument");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  hpic::Counters h;
  int rc = read_counters(ctx, &h);
  if (rc) return rc;
  // the live slots counted on the device (the chunk counts of the transfers)
  const long long nb = hpic::xfer_chunks(h.n);
  rc = xfer_reserve(ctx, (size_t)(nb + 1) * sizeof(uint32_t));
  if (rc) return rc;
  uint32_t *cc = static_cast<uint32_t *>(ctx->xfer);
  const uint32_t *src = ctx->fp32 ? pview<float>(ctx, ctx->cur).id : pview<double>(ctx, ctx->cur).id;
  hpic::launch_live_scan(src, h.n, cc, ctx->stream);
  uint32_t live = 0;
  CK(cudaMemcpyAsync(&live, cc + nb, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  *n = live;
  return HPIC_OK;
}

int hpic_read_particles(hpic_ctx *ctx, double *x, double *y, double *z, double *ux, double *uy,
                        double *uz, double *tau, uint32_t *id, int64_t cap, int64_t *n) {
  if (!ctx || !n) return fail(ctx, HPIC_EINVAL, "NULL argument");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  return ctx->fp32 ? read_particles_impl<float>(ctx, x, y, z, ux, uy, uz, tau, id, cap, n)
                   : read_particles_impl<double>(ctx, x, y, z, ux, uy, uz, tau, id, cap, n);
}

int hpic_read_weights(hpic_ctx *ctx, double *w, int64_t cap, int64_t *n_out) {
  if (!ctx || !n_out) return fail(ctx, HPIC_EINVAL, "NULL argument");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  hpic::Counters h;
  int rc = read_counters(ctx, &h);
  if (rc) return rc;
  const long long n = h.n;
  std::vector<uint32_t> ids(n);
  std::vector<char> wb(n * ctx->rsz);
  const uint32_t *id_src = ctx->fp32 ? pview<float>(ctx, ctx->cur).id : pview<double>(ctx, ctx->cur).id;
  const void *w_src = ctx->fp32 ? (const void *)pview<float>(ctx, ctx->cur).w
                                : (const void *)pview<double>(ctx, ctx->cur).w;
  if (n) {
    CK(cudaMemcpyAsync(ids.data(), id_src, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->K.weighted)
      CK(cudaMemcpyAsync(wb.data(), w_src, n * ctx->rsz, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  long long live = 0;
  for (long long i = 0; i < n; ++i) live += ids[i] != hpic::kDead;
  *n_out = live;
  if (live > cap) return fail(ctx, HPIC_EINVAL, "output capacity below the live particle count");
  long long m = 0;
  for (long long i = 0; i < n; ++i) {
    if (ids[i] == hpic::kDead) continue;
    double v = ctx->K.w;
    if (ctx->K.weighted)
      v = ctx->fp32 ? (double)reinterpret_cast<const float *>(wb.data())[i]
                    : reinterpret_cast<const double *>(wb.data())[i];
    if (w) w[m] = v;
    ++m;
  }
  return HPIC_OK;
}

int hpic_load_weights(hpic_ctx *ctx, int64_t n, const double *w) {
  if (!ctx || n < 0 || (n > 0 && !w)) return fail(ctx, HPIC_EINVAL, "bad weight arguments");
  ctx->keys_step = -1;
  if (!ctx->K.weighted) return fail(ctx, HPIC_ESTATE, "per-electron weights need the Gaussian envelope");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  hpic::Counters h;
  int rc = read_counters(ctx, &h);
  if (rc) return rc;
  if (n > h.n) return fail(ctx, HPIC_EINVAL, "more weights than loaded electrons");
  for (int64_t i = 0; i < n; ++i)
    if (!(w[i] > 0) || !std::isfinite(w[i])) return fail(ctx, HPIC_EINVAL, "weights must be positive");
  if (n == 0) return HPIC_OK;
  if (ctx->fp32) {
    std::vector<float> b(w, w + n);
    CK(cudaMemcpyAsync(pview<float>(ctx, ctx->cur).w, b.data(), n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    CK(cudaMemcpyAsync(pview<double>(ctx, ctx->cur).w, w, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return HPIC_OK;
}

int hpic_load_particles(hpic_ctx *ctx, int64_t n, const double *x, const double *y,
                        const double *z, const double *ux, const double *uy, const double *uz,
                        const double *tau, const uint32_t *id) {
  if (!ctx || n < 0 || (n > 0 && (!x || !y || !z || !ux || !uy || !uz || !tau || !id)))
    return fail(ctx, HPIC_EINVAL, "bad particle arguments");
  ctx->keys_step = -1;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  return ctx->fp32 ? load_particles_impl<float>(ctx, n, x, y, z, ux, uy, uz, tau, id)
                   : load_particles_impl<double>(ctx, n, x, y, z, ux, uy, uz, tau, id);
}

int hpic_get_clock(hpic_ctx *ctx, int64_t *step, int64_t *next_id) {
  if (!ctx) return HPIC_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  hpic::Counters h;
  int rc = read_counters(ctx, &h);
  if (rc) return rc;
  if (step) *step = h.step;
  if (next_id) *next_id = h.next_id;
  return HPIC_OK;
}

int hpic_set_clock(hpic_ctx *ctx, int64_t step, int64_t next_id) {
  if (!ctx || step < 0 || next_id < 0 || step >= 0xFFFFFFFFll || next_id >= 0xFFFFFFFFll)
    return fail(ctx, HPIC_EINVAL, "clock out of range");
  ctx->keys_step = -1;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  hpic::Counters h;
  int rc = read_counters(ctx, &h);
  if (rc) return rc;
  h.step = step;
  h.next_id = next_id;
  ctx->host_step = step;
  return write_counters(ctx, &h);
}

int hpic_profile(hpic_ctx *ctx, int enable) {
  if (!ctx) return HPIC_EINVAL;
  if (ctx->owner) return refuse_batch_target(ctx);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof = enable != 0;
  ctx->ev_used = 0;
  ctx->prof_launches = 0;
  double ps;
  CK(cudaMemcpy(&ps, ctx->tal + hpic::T_PSTEPS, sizeof(double), cudaMemcpyDeviceToHost));
  ctx->prof_ps0 = ps;
  return HPIC_OK;
}

int hpic_kernel_time(hpic_ctx *ctx, double *ms, int64_t *launches, double *psteps) {
  if (!ctx) return HPIC_EINVAL;
  if (ctx->owner) return refuse_batch_target(ctx);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  CK(cudaStreamSynchronize(ctx->stream));
  double total = 0.0;
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ctx->ev[i], ctx->ev[i + 1]));
    total += t;
  }
  double ps;
  CK(cudaMemcpy(&ps, ctx->tal + hpic::T_PSTEPS, sizeof(double), cudaMemcpyDeviceToHost));
  if (ms) *ms = total;
  if (launches) *launches = ctx->prof_launches;
  if (psteps) *psteps = ps - ctx->prof_ps0;
  ctx->ev_used = 0;
  ctx->prof_launches = 0;
  ctx->prof_ps0 = ps;
  return HPIC_OK;
}

int hpic_launch_count(const hpic_ctx *ctx, int64_t *launches) {
  if (!ctx || !launches) return HPIC_EINVAL;
  *launches = ctx->launches;
  return HPIC_OK;
}

}  // extern "C"

namespace {

constexpr char kCkptMagic[8] = {'H', 'P', 'I', 'C', 'C', 'K', 'P', '1'};

// a device array of `bytes` to the file (through host memory)
int save_dev(hpic_ctx *ctx, FILE *f, const void *dev, size_t bytes) {
  std::vector<char> b(bytes);
  if (bytes) {
    CK(cudaMemcpyAsync(b.data(), dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (bytes && fwrite(b.data(), 1, bytes, f) != bytes) return fail(ctx, HPIC_EINVAL, "checkpoint write failed");
  return HPIC_OK;
}

int load_dev(hpic_ctx *ctx, FILE *f, void *dev, size_t bytes) {
  std::vector<char> b(bytes);
  if (bytes && fread(b.data(), 1, bytes, f) != bytes) return fail(ctx, HPIC_EINVAL, "checkpoint truncated");
  if (bytes) {
    CK(cudaMemcpyAsync(dev, b.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return HPIC_OK;
}

// the state arrays of a context in file order: particle slots [0, n) of the
// current buffer (7 reals, weight, id), then the grids, tallies, histograms
// and history; `fn` is save_dev or load_dev
template <typename Fn>
int each_array(hpic_ctx *ctx, FILE *f, long long n, Fn fn) {
  char *b = static_cast<char *>(ctx->pbuf[ctx->cur]);
  const size_t rs = ctx->rsz, st = (size_t)ctx->stride * rs;
  int rc = HPIC_OK;
  for (int a = 0; a < 8 && !rc; ++a) rc = fn(ctx, f, b + a * st + ctx->poff * rs, n * rs);
  if (!rc) rc = fn(ctx, f, reinterpret_cast<uint32_t *>(b + 8 * st) + ctx->poff, n * sizeof(uint32_t));
  const size_t nv = ctx->vstride * rs, nc = ctx->K.ncell * sizeof(double);
  if (!rc) rc = fn(ctx, f, ctx->fields, 6 * nv);
  if (!rc) rc = fn(ctx, f, ctx->jfield, 3 * nv);
  if (!rc) rc = fn(ctx, f, ctx->T, nc);
  if (!rc) rc = fn(ctx, f, ctx->eta, nc);
  if (!rc) rc = fn(ctx, f, ctx->H, nc);
  if (!rc) rc = fn(ctx, f, ctx->Ti, nc);
  if (!rc) rc = fn(ctx, f, ctx->Fsig, ctx->K.ncell * rs);
  if (!rc && ctx->fp32) rc = fn(ctx, f, ctx->eta_r, ctx->K.ncell * sizeof(float));
  if (!rc) rc = fn(ctx, f, ctx->tal, hpic::T_COUNT * sizeof(double));
  if (!rc) rc = fn(ctx, f, ctx->hist, 2 * hist_len(ctx) * sizeof(double));
  if (!rc) rc = fn(ctx, f, ctx->history, (ctx->run.max_history > 0 ? ctx->run.max_history : 1) * sizeof(double));
  return rc;
}

struct CkptHeader {
  char magic[8];
  hpic_target_desc tgt;
  hpic_run_params run;
  hpic_laser_desc laser;
  int32_t have_laser, pad;
  long long host_step;
  hpic::Counters cnt;
};

}  // namespace

extern "C" {

int hpic_save(hpic_ctx *ctx, const char *path) {
  if (!ctx || !path) return fail(ctx, HPIC_EINVAL, "NULL argument");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, 8);
  h.tgt = ctx->tgt;
  h.run = ctx->run;
  h.laser = ctx->laser;
  h.have_laser = ctx->have_laser;
  h.host_step = ctx->host_step;
  int rc = read_counters(ctx, &h.cnt);
  if (rc) return rc;
  FILE *f = std::fopen(path, "wb");
  if (!f) return fail(ctx, HPIC_EINVAL, std::string("cannot write ") + path);
  rc = fwrite(&h, sizeof(h), 1, f) == 1 ? HPIC_OK : fail(ctx, HPIC_EINVAL, "checkpoint write failed");
  if (!rc) rc = each_array(ctx, f, h.cnt.n, save_dev);
  if (std::fclose(f) != 0 && !rc) rc = fail(ctx, HPIC_EINVAL, "checkpoint write failed");
  return rc;
}

int hpic_load(hpic_ctx **out, const char *path, int device, void *cuda_stream) {
  if (!out || !path) return fail(nullptr, HPIC_EINVAL, "NULL argument");
  *out = nullptr;
  FILE *f = std::fopen(path, "rb");
  if (!f) return fail(nullptr, HPIC_EINVAL, std::string("cannot read ") + path);
  CkptHeader h{};
  if (fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.cnt.n < 0) {
    std::fclose(f);
    return fail(nullptr, HPIC_EINVAL, "not a checkpoint of this library");
  }
  hpic_ctx *ctx = nullptr;
  int rc = hpic_init_target(&ctx, &h.tgt, &h.run, device, cuda_stream);
  if (!rc && h.have_laser) {
    rc = hpic_inject_electrons(ctx, &h.laser);
    if (rc) g_create_error = ctx->err;
  }
  if (!rc) {
    rc = reserve(ctx, h.cnt.n + injection_total(ctx));
    if (rc) g_create_error = ctx->err;
  }
  if (!rc) {
    rc = each_array(ctx, f, h.cnt.n, load_dev);
    if (!rc) rc = write_counters(ctx, &h.cnt);
    ctx->host_step = h.host_step;
    if (rc) g_create_error = ctx->err;
  }
  std::fclose(f);
  if (rc) {
    if (ctx) {
      cudaStreamSynchronize(ctx->stream);
      destroy_all(ctx);
      delete ctx;
    }
    return rc;
  }
  *out = ctx;
  return HPIC_OK;
}

int hpic_destroy(hpic_ctx *ctx) {
  if (!ctx) return HPIC_EINVAL;
  if (ctx->owner) return refuse_batch_target(ctx);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  destroy_all(ctx);
  delete ctx;
  return HPIC_OK;
}

const char *hpic_last_error(const hpic_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
