/*
 * Oracle, part 2: one time step of the fast-electron hybrid-PIC method,
 * serial, SI units, FP64.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * A step, in the order this reading of the paper fixes (the paper gives the
 * equations but no order):
 *   for every electron present at the start of the step
 *     gather E, B at x^n (trilinear on the Yee lattice)
 *     relativistic Boris push of the momentum             (Lorentz force)
 *     ionisation drag, explicit in energy                 Eq. (5)
 *     Davies angular scatter                              Eq. (B4)
 *     optical-depth bremsstrahlung emission               App. B
 *     position update x^{n+1} = x^n + v dt
 *     escape / reflux at each face crossed                Sec. II.A
 *     current deposit at x^{n+1}                          j_h of Eq. (A2)
 *   E = eta (curl B / mu0 - j_h) on edges                 Eq. (A2)
 *   B -= dt curl E on faces                               Eq. (A3)
 *   Ohmic + drag heating, T and eta update                Eqs. (A4)-(A8)
 *   e-i equilibration of T_e and T_i (optional)           App. A
 *   injection of this step's new electrons at x = 0+     Eq. (B1), Sec. II.B
 * Random numbers: Philox4x32-10 with counter (step, id, block, target) and
 * key (seed low, seed high); block 0 = scatter, 1 = emission, 2..4 = reflux
 * on the x, y, z faces, 8 and 9 = injection.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q_E 1.602176634e-19
#define M_E 9.1093837015e-31
#define C_L 299792458.0
#define EPS0 8.8541878128e-12
#define MU0 (1.0 / (EPS0 * C_L * C_L))
#define K_B 1.380649e-23
#define PI 3.14159265358979323846
#define MC2 (M_E * C_L * C_L)

struct orc_sim {
  orc_target t;
  orc_laser l;
  orc_run r;
  double a0, T_hot, w, eps_esc, du_reflux;
  int64_t n_inj_steps;
  int64_t n, cap;
  double *x, *y, *z, *ux, *uy, *uz, *tau, *wt;  /* wt: real electrons per macro */
  uint32_t *id;
  unsigned char *alive;
  int64_t nvec, ncell;
  double *g[13];
  int64_t step, next_id;
  orc_tallies tal;
  double *histE, *histN, *history;
  double *table;
  double *ohm;  /* Ohmic energy of each cell in the current step (heating) */
};

static double kinetic(const double u[3]) {
  double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return MC2 * u2 / (1.0 + sqrt(1.0 + u2));
}

static double u_of_eps(double eps) {
  double e = eps / MC2;
  return sqrt(e * (e + 2.0));
}

static void draw(const orc_sim *s, uint32_t id, uint32_t block, double u[4]) {
  uint32_t ctr[4] = {(uint32_t)s->step, id, block, s->r.target_index};
  uint32_t key[2] = {(uint32_t)s->r.seed, (uint32_t)(s->r.seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  for (int c = 0; c < 4; ++c) u[c] = orc_uniform(out[c]);
}

/* ---------------- grid helpers ---------------- */
static int64_t vidx(const orc_sim *s, int i, int j, int k) {
  return (int64_t)i + (int64_t)(s->t.nx + 1) * ((int64_t)j + (int64_t)(s->t.ny + 1) * k);
}
static int64_t cidx(const orc_sim *s, int i, int j, int k) {
  return (int64_t)i + (int64_t)s->t.nx * ((int64_t)j + (int64_t)s->t.ny * k);
}

/* staggering of each vector component (in half cells) along x, y, z */
static const int STAG[12][3] = {
    {0, 0, 0}, {0, 0, 0},                       /* T, eta (unused) */
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1},            /* Ex Ey Ez */
    {0, 1, 1}, {1, 0, 1}, {1, 1, 0},            /* Bx By Bz */
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1},            /* jx jy jz */
    {0, 0, 0}};

/* linear (cloud-in-cell) weights along one axis.  X is the position in
 * cells, n the cell count.  A component staggered by half a cell is held at
 * its outermost value within half a cell of a wall. */
static void cic_axis(double X, int n, int stag, int *i0, double *f) {
  double q = X;
  if (stag) {
    q = X - 0.5;
    if (q < 0.0) q = 0.0;
    if (q > (double)(n - 1)) q = (double)(n - 1);
  }
  int i = (int)floor(q);
  if (i > n - 1) i = n - 1;
  if (i < 0) i = 0;
  *i0 = i;
  *f = q - (double)i;
}

static double gather(const orc_sim *s, int which, const double X[3]) {
  int i0[3];
  double f[3];
  int n[3] = {s->t.nx, s->t.ny, s->t.nz};
  for (int a = 0; a < 3; ++a) cic_axis(X[a], n[a], STAG[which][a], &i0[a], &f[a]);
  const double *G = s->g[which];
  double v = 0.0;
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        double wgt = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1]) * (c ? f[2] : 1.0 - f[2]);
        v += wgt * G[vidx(s, i0[0] + a, i0[1] + b, i0[2] + c)];
      }
  return v;
}

static void deposit(orc_sim *s, int which, const double X[3], double val) {
  int i0[3];
  double f[3];
  int n[3] = {s->t.nx, s->t.ny, s->t.nz};
  for (int a = 0; a < 3; ++a) cic_axis(X[a], n[a], STAG[which][a], &i0[a], &f[a]);
  double *G = s->g[which];
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        double wgt = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1]) * (c ? f[2] : 1.0 - f[2]);
        G[vidx(s, i0[0] + a, i0[1] + b, i0[2] + c)] += wgt * val;
      }
}

/* bin of one photon in the energy x angle tallies (Sec. III.A spectra and
 * angular distributions): row 0 below tally_E_min, rows 1..n_E the log bins
 * of equal width in ln k, row n_E + 1 at or above tally_E_max; column the
 * polar angle theta in [0, pi] (measured by the caller from +x, the laser
 * axis) in n_theta equal bins, theta = pi in the last */
void orc_tally_bin(const orc_run *r, double k, double theta, int *row_out, int *col_out) {
  int nE = r->n_E, nth = r->n_theta;
  int row;
  if (k < r->tally_E_min) row = 0;
  else if (k >= r->tally_E_max) row = nE + 1;
  else {
    row = 1 + (int)floor((double)nE * log(k / r->tally_E_min) /
                         log(r->tally_E_max / r->tally_E_min));
    if (row < 1) row = 1;
    if (row > nE) row = nE;
  }
  int col = (int)floor(theta / PI * (double)nth);
  if (col < 0) col = 0;
  if (col > nth - 1) col = nth - 1;
  *row_out = row;
  *col_out = col;
}

/* photon tally: energy row (underflow, n_E log bins, overflow) x polar bin */
static void tally_photon(orc_sim *s, double k, double theta, double wph) {
  int nth = s->r.n_theta, row, col;
  orc_tally_bin(&s->r, k, theta, &row, &col);
  s->histE[row * nth + col] += wph * k;
  s->histN[row * nth + col] += wph;
  s->tal.E_xray += wph * k;
  if (k >= s->r.ce_threshold) {
    s->tal.E_xray_above += wph * k;
    if (s->step < s->r.max_history) s->history[s->step] += wph * k;
  }
}

/* ---------------- one electron, one step ---------------- */
static void kill_with_heat(orc_sim *s, int64_t ip, int64_t cell, double eps) {
  if (!(s->r.physics & ORC_UNBOUNDED)) s->g[ORC_HEAT][cell] += s->wt[ip] * eps;
  s->tal.E_drag += s->wt[ip] * eps;
  s->tal.n_cut += 1.0;
  s->alive[ip] = 0;
}

static void particle_update(orc_sim *s, int64_t ip) {
  const orc_target *t = &s->t;
  const orc_run *r = &s->r;
  const double dx = t->dx, dt = r->dt, w = s->wt[ip];
  double X[3] = {s->x[ip] / dx, s->y[ip] / dx, s->z[ip] / dx};
  double u[3] = {s->ux[ip], s->uy[ip], s->uz[ip]};
  double R0[4];
  draw(s, s->id[ip], 0, R0);
  s->tal.particle_steps += 1.0;

  /* field gather at x^n */
  const int unbounded = (r->physics & ORC_UNBOUNDED) != 0;
  double E[3] = {0.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 0.0};
  if (!unbounded)
    for (int c = 0; c < 3; ++c) {
      E[c] = gather(s, ORC_EX + c, X);
      B[c] = gather(s, ORC_BX + c, X);
    }
  int ci = (int)floor(X[0]), cj = (int)floor(X[1]), ck = (int)floor(X[2]);
  if (ci > t->nx - 1) ci = t->nx - 1;
  if (cj > t->ny - 1) cj = t->ny - 1;
  if (ck > t->nz - 1) ck = t->nz - 1;
  if (ci < 0) ci = 0;
  if (cj < 0) cj = 0;
  if (ck < 0) ck = 0;
  int64_t cell = cidx(s, ci, cj, ck);

  /* relativistic push; the energy change is the work of E */
  double eps_before = kinetic(u);
  orc_boris(u, E, B, dt);
  double eps = kinetic(u);
  s->tal.W_field += w * (eps_before - eps);

  /* tracking cut, then ionisation drag with beta at the start of the drag */
  if (eps < r->E_cut) { kill_with_heat(s, ip, cell, eps); return; }
  if (r->physics & ORC_DRAG) {
    double gam = 1.0 + eps / MC2;
    double beta = sqrt(1.0 - 1.0 / (gam * gam));
    double de = orc_stop_ion(t, eps) * beta * C_L * dt;
    double eps1 = eps - de;
    if (eps1 < r->E_cut) { kill_with_heat(s, ip, cell, eps); return; }
    double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double scale = u_of_eps(eps1) / un;
    for (int c = 0; c < 3; ++c) u[c] *= scale;
    if (!unbounded) s->g[ORC_HEAT][cell] += w * de;
    s->tal.E_drag += w * de;
    eps = eps1;
  }

  /* Davies scatter: polar deflection Gamma*sigma, azimuth uniform */
  if (r->physics & ORC_SCATTER) {
    double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double sig = orc_davies_sigma(t, un * M_E * C_L, dt);
    double gauss = sqrt(-2.0 * log(R0[0])) * cos(2.0 * PI * R0[1]);
    double d[3] = {u[0] / un, u[1] / un, u[2] / un}, dn[3];
    orc_rotate(d, gauss * sig, 2.0 * PI * R0[2], dn);
    for (int c = 0; c < 3; ++c) u[c] = un * dn[c];
  }

  /* bremsstrahlung by optical depth: tau_rem -= n_i B sigma v dt */
  if ((r->physics & ORC_BREM) && eps > r->k_min) {
    double gam = 1.0 + eps / MC2;
    double beta = sqrt(1.0 - 1.0 / (gam * gam));
    double rate = orc_brem_rate(t, r->k_min, eps);  /* sum n_i sigma (1/m) */
    if (r->physics & ORC_FSIGMA) rate *= orc_f_sigma(t, s->g[ORC_TI][cell]);
    s->tau[ip] -= r->brem_boost * rate * beta * C_L * dt;
    if (s->tau[ip] <= 0.0) {
      double R1[4];
      draw(s, s->id[ip], 1, R1);
      double k = orc_brem_sample(s->table, r->table_rows, r->table_cols, r->k_min,
                                 r->table_E_max, eps, R1[0]);
      double thg = orc_photon_theta(gam, R1[1]);
      double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      double d[3] = {u[0] / un, u[1] / un, u[2] / un}, dg[3];
      orc_rotate(d, thg, 2.0 * PI * R1[2], dg);
      double cx = dg[0];
      if (cx > 1.0) cx = 1.0;
      if (cx < -1.0) cx = -1.0;
      tally_photon(s, k, acos(cx), w / r->brem_boost);
      s->tal.n_emitted += 1.0;
      s->tau[ip] = -log(1.0 - R1[3]);
      eps -= k / r->brem_boost;
      if (eps < r->E_cut) { kill_with_heat(s, ip, cell, eps); return; }
      double scale = u_of_eps(eps) / un;
      for (int c = 0; c < 3; ++c) u[c] *= scale;
    }
  }

  /* position update with the final momentum */
  double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double pos[3] = {s->x[ip] + u[0] / gam * C_L * dt, s->y[ip] + u[1] / gam * C_L * dt,
                   s->z[ip] + u[2] / gam * C_L * dt};

  /* escape or reflux at each face crossed, x then y then z */
  int n[3] = {t->nx, t->ny, t->nz};
  for (int a = 0; a < 3 && !unbounded; ++a) {
    double L = (double)n[a] * dx;
    if (pos[a] >= 0.0 && pos[a] <= L) continue;
    double e_out = kinetic(u);
    if (e_out >= s->eps_esc) {
      s->tal.E_escaped += w * e_out;
      s->tal.n_escaped += 1.0;
      s->alive[ip] = 0;
      return;
    }
    int low = pos[a] < 0.0;
    pos[a] = low ? -pos[a] : 2.0 * L - pos[a];
    u[a] = -u[a];
    double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double un2 = un - s->du_reflux;
    if (un2 <= 0.0) {
      s->tal.E_reflux += w * e_out;
      s->tal.n_reflux_absorbed += 1.0;
      s->alive[ip] = 0;
      return;
    }
    double R2[4];
    draw(s, s->id[ip], 2 + a, R2);
    double xi = r->sigma_dtheta * (R2[0] - 0.5);
    double d[3] = {u[0] / un, u[1] / un, u[2] / un}, dn[3];
    orc_rotate(d, xi, 2.0 * PI * R2[1], dn);
    if (low && dn[a] < 0.0) dn[a] = -dn[a];
    if (!low && dn[a] > 0.0) dn[a] = -dn[a];
    for (int c = 0; c < 3; ++c) u[c] = un2 * dn[c];
    s->tal.E_reflux += w * (e_out - kinetic(u));
    s->tal.n_refluxed += 1.0;
  }

  s->x[ip] = pos[0];
  s->y[ip] = pos[1];
  s->z[ip] = pos[2];
  s->ux[ip] = u[0];
  s->uy[ip] = u[1];
  s->uz[ip] = u[2];

  /* hot-electron current j_h = q w v S(x) / V at x^{n+1}, q = -e */
  if (unbounded) return;
  gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double Xn[3] = {pos[0] / dx, pos[1] / dx, pos[2] / dx};
  double jfac = -Q_E * w / (dx * dx * dx) * C_L / gam;
  for (int c = 0; c < 3; ++c) deposit(s, ORC_JX + c, Xn, jfac * u[c]);
}

/* ---------------- fields: Eqs. (A2), (A3) ---------------- */
static double eta_avg4(const orc_sim *s, int i0, int i1, int j0, int j1, int k0, int k1) {
  const double *eta = s->g[ORC_ETA];
  double v = 0.0;
  for (int k = k0; k <= k1; ++k)
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i) v += eta[cidx(s, i, j, k)];
  return 0.25 * v;
}

static void field_update(orc_sim *s) {
  const int nx = s->t.nx, ny = s->t.ny, nz = s->t.nz;
  const double dx = s->t.dx, dt = s->r.dt;
  double *Ex = s->g[ORC_EX], *Ey = s->g[ORC_EY], *Ez = s->g[ORC_EZ];
  double *Bx = s->g[ORC_BX], *By = s->g[ORC_BY], *Bz = s->g[ORC_BZ];
  const double *jx = s->g[ORC_JX], *jy = s->g[ORC_JY], *jz = s->g[ORC_JZ];
  const double cb = s->r.curlB_term ? 1.0 / MU0 : 0.0;
  if (s->r.physics & ORC_FIELDS) {
    /* Ohm's law with the return current on interior edges; tangential E is
     * zero on the outer faces (conducting walls) */
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= nz; ++k)
      for (int j = 0; j <= ny; ++j)
        for (int i = 0; i <= nx; ++i) {
          int64_t q = vidx(s, i, j, k);
          Ex[q] = Ey[q] = Ez[q] = 0.0;
          if (i < nx && j >= 1 && j <= ny - 1 && k >= 1 && k <= nz - 1) {
            double curl = (Bz[q] - Bz[vidx(s, i, j - 1, k)]) / dx -
                          (By[q] - By[vidx(s, i, j, k - 1)]) / dx;
            Ex[q] = eta_avg4(s, i, i, j - 1, j, k - 1, k) * (cb * curl - jx[q]);
          }
          if (j < ny && i >= 1 && i <= nx - 1 && k >= 1 && k <= nz - 1) {
            double curl = (Bx[q] - Bx[vidx(s, i, j, k - 1)]) / dx -
                          (Bz[q] - Bz[vidx(s, i - 1, j, k)]) / dx;
            Ey[q] = eta_avg4(s, i - 1, i, j, j, k - 1, k) * (cb * curl - jy[q]);
          }
          if (k < nz && i >= 1 && i <= nx - 1 && j >= 1 && j <= ny - 1) {
            double curl = (By[q] - By[vidx(s, i - 1, j, k)]) / dx -
                          (Bx[q] - Bx[vidx(s, i, j - 1, k)]) / dx;
            Ez[q] = eta_avg4(s, i - 1, i, j - 1, j, k, k) * (cb * curl - jz[q]);
          }
        }
  }
  if (s->r.physics & ORC_FARADAY) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= nz; ++k)
      for (int j = 0; j <= ny; ++j)
        for (int i = 0; i <= nx; ++i) {
          int64_t q = vidx(s, i, j, k);
          if (j < ny && k < nz)
            Bx[q] -= dt * ((Ez[vidx(s, i, j + 1, k)] - Ez[q]) / dx -
                           (Ey[vidx(s, i, j, k + 1)] - Ey[q]) / dx);
          if (i < nx && k < nz)
            By[q] -= dt * ((Ex[vidx(s, i, j, k + 1)] - Ex[q]) / dx -
                           (Ez[vidx(s, i + 1, j, k)] - Ez[q]) / dx);
          if (i < nx && j < ny)
            Bz[q] -= dt * ((Ey[vidx(s, i + 1, j, k)] - Ey[q]) / dx -
                           (Ex[vidx(s, i, j + 1, k)] - Ex[q]) / dx);
        }
  }
}

/* ---------------- background heating: Eqs. (A4)-(A8) ---------------- */
static void heating(orc_sim *s) {
  const int nx = s->t.nx, ny = s->t.ny, nz = s->t.nz;
  const double V = s->t.dx * s->t.dx * s->t.dx, dt = s->r.dt;
  const double *jx = s->g[ORC_JX], *jy = s->g[ORC_JY], *jz = s->g[ORC_JZ];
  double *T = s->g[ORC_T], *eta = s->g[ORC_ETA], *Ti = s->g[ORC_TI];
  const double *heat = s->g[ORC_HEAT];
  const int fields = (s->r.physics & ORC_FIELDS) != 0;
  double *ohm = s->ohm;
  /* each cell on its own (in parallel in the OpenMP build); the cells'
   * Ohmic energies are summed into the tally afterwards in cell order */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t c = cidx(s, i, j, k);
        double rho = heat[c] / V;
        if (fields) {
          double jbx = 0.25 * (jx[vidx(s, i, j, k)] + jx[vidx(s, i, j + 1, k)] +
                               jx[vidx(s, i, j, k + 1)] + jx[vidx(s, i, j + 1, k + 1)]);
          double jby = 0.25 * (jy[vidx(s, i, j, k)] + jy[vidx(s, i + 1, j, k)] +
                               jy[vidx(s, i, j, k + 1)] + jy[vidx(s, i + 1, j, k + 1)]);
          double jbz = 0.25 * (jz[vidx(s, i, j, k)] + jz[vidx(s, i + 1, j, k)] +
                               jz[vidx(s, i, j + 1, k)] + jz[vidx(s, i + 1, j + 1, k)]);
          double rho_ohm = eta[c] * (jbx * jbx + jby * jby + jbz * jbz) * dt;
          ohm[c] = rho_ohm * V;
          rho += rho_ohm;
        }
        if (s->r.physics & ORC_HEATING) T[c] += orc_temperature_rise(&s->t, T[c], rho);
        /* e-i equilibration over the step, rates frozen at the temperatures
         * after the heating: d = T_e - T_i decays as exp(-(a + b) dt) and
         * b T_e + a T_i is kept (a = rate_e, b = rate_i) */
        if (s->r.physics & ORC_EI) {
          double a, b;
          orc_ei_rates(&s->t, T[c], Ti[c], &a, &b);
          if (!(a + b > 0.0)) a = b = 0.0;
          double d = T[c] - Ti[c];
          double f = a + b > 0.0 ? expm1(-(a + b) * dt) / (a + b) : 0.0;  /* (e^{-(a+b)dt} - 1)/(a+b) */
          T[c] += a * d * f;
          Ti[c] -= b * d * f;
        }
        if (s->r.physics & (ORC_HEATING | ORC_EI)) eta[c] = orc_resistivity(&s->t, T[c]);
      }
  if (fields)
    for (int64_t c = 0; c < s->ncell; ++c) s->tal.E_ohmic_grid += ohm[c];
}

/* ---------------- injection: Eq. (B1) ---------------- */
static void reserve(orc_sim *s, int64_t need) {
  if (need <= s->cap) return;
  int64_t cap = s->cap ? s->cap : 1024;
  while (cap < need) cap *= 2;
  s->x = realloc(s->x, cap * sizeof(double));
  s->y = realloc(s->y, cap * sizeof(double));
  s->z = realloc(s->z, cap * sizeof(double));
  s->ux = realloc(s->ux, cap * sizeof(double));
  s->uy = realloc(s->uy, cap * sizeof(double));
  s->uz = realloc(s->uz, cap * sizeof(double));
  s->tau = realloc(s->tau, cap * sizeof(double));
  s->wt = realloc(s->wt, cap * sizeof(double));
  s->id = realloc(s->id, cap * sizeof(uint32_t));
  s->alive = realloc(s->alive, cap);
  s->cap = cap;
}

/* the cone half-angle for an electron of kinetic energy eps: the laser's,
 * or with the Moore cap (Sec. II.B) the smaller of it and
 * atan(sqrt(2/(gamma - 1))); returned as 1 - cos(theta) */
static double cone_omc(const orc_sim *s, double eps) {
  double th = s->l.cone_half;
  if (s->l.moore_cap) {
    double moore = atan(sqrt(2.0 / (eps / MC2)));
    if (moore < th) th = moore;
  }
  return 1.0 - cos(th);
}

/* Gaussian envelopes of Sec. II.B and App. B: f(r) = exp(-4 ln2 r^2/r_fwhm^2)
 * at the centre of each face cell, g(t) = exp(-4 ln2 (t - t_pk)^2/t_fwhm^2)
 * at mid-step t = (s + 1/2) dt with t_pk chosen so that g(0) = g_min; cells
 * with f >= f_min inject per_cell macro-electrons while g >= g_min, each of
 * weight N_cell/per_cell, N_cell = I0 f g A dt eta_le / <eps>, with the local
 * mean energy <eps> = a0 sqrt(f g) m_e c^2 (Eq. (N_cell)) */
static double g_of(const orc_sim *s, int64_t st) {
  const orc_laser *l = &s->l;
  double t_pk = 0.5 * l->t_fwhm * sqrt(log(1.0 / l->g_min) / log(2.0));
  double t = ((double)st + 0.5) * s->r.dt;
  double u = (t - t_pk) / l->t_fwhm;
  return exp(-4.0 * log(2.0) * u * u);
}

static void inject_gauss(orc_sim *s) {
  const orc_laser *l = &s->l;
  const double g = g_of(s, s->step);
  if (!(g >= l->g_min) || l->per_cell <= 0 || !(s->a0 > 0.0)) return;
  const double dx = s->t.dx, A = dx * dx;
  int64_t c = 0;
  for (int k = 0; k < s->t.nz; ++k)
    for (int j = 0; j < s->t.ny; ++j) {
      double yc = (j + 0.5) * dx - l->spot_y, zc = (k + 0.5) * dx - l->spot_z;
      double f = exp(-4.0 * log(2.0) * (yc * yc + zc * zc) / (l->r_fwhm * l->r_fwhm));
      if (!(f >= l->f_min)) continue;
      double mean = s->a0 * sqrt(f * g) * MC2;
      double N_cell = l->I0 * f * g * A * s->r.dt * l->eta_l2e / mean;
      double w = N_cell / (double)l->per_cell;
      reserve(s, s->n + l->per_cell);
      for (int32_t i = 0; i < l->per_cell; ++i) {
        uint32_t id = (uint32_t)(s->next_id + c * l->per_cell + i);
        double R8[4], R9[4];
        draw(s, id, 8, R8);
        draw(s, id, 9, R9);
        double eps = -mean * log(1.0 - R8[2]);
        double omc = R8[3] * cone_omc(s, eps);
        double ct = 1.0 - omc, st_ = sqrt(omc * (2.0 - omc)), cph = 2.0 * PI * R9[0];
        double un = u_of_eps(eps);
        int64_t q = s->n;
        s->x[q] = 1e-6 * dx;
        s->y[q] = (j + R8[0]) * dx;
        s->z[q] = (k + R8[1]) * dx;
        s->ux[q] = un * ct;
        s->uy[q] = un * st_ * cos(cph);
        s->uz[q] = un * st_ * sin(cph);
        s->tau[q] = -log(1.0 - R9[1]);
        s->wt[q] = w;
        s->id[q] = id;
        s->alive[q] = 1;
        s->tal.E_injected += w * eps;
        s->tal.N_injected += w;
        s->tal.n_injected += 1.0;
        s->n += 1;
      }
      ++c;
    }
  s->next_id += c * l->per_cell;
}

static void inject(orc_sim *s) {
  if (s->l.envelope == ORC_ENV_GAUSS) {
    inject_gauss(s);
    return;
  }
  int64_t st = s->step;
  if (st >= s->n_inj_steps || s->l.n_macro <= 0) return;
  int64_t S = s->n_inj_steps, N = s->l.n_macro;
  int64_t cnt = N * (st + 1) / S - N * st / S;
  reserve(s, s->n + cnt);
  double cosc = cos(s->l.cone_half);
  for (int64_t i = 0; i < cnt; ++i) {
    uint32_t id = (uint32_t)(s->next_id + i);
    double R8[4], R9[4];
    draw(s, id, 8, R8);
    draw(s, id, 9, R9);
    double rr = s->l.spot_r * sqrt(R8[0]);
    double ph = 2.0 * PI * R8[1];
    double eps = -s->T_hot * log(1.0 - R8[2]);
    double omc = R8[3] * (s->l.moore_cap ? cone_omc(s, eps) : 1.0 - cosc);  /* uniform in solid angle */
    double ct = 1.0 - omc;
    double st_ = sqrt(omc * (2.0 - omc));
    double cph = 2.0 * PI * R9[0];
    double un = u_of_eps(eps);
    int64_t q = s->n + i;
    s->x[q] = 1e-6 * s->t.dx;
    s->y[q] = s->l.spot_y + rr * cos(ph);
    s->z[q] = s->l.spot_z + rr * sin(ph);
    s->ux[q] = un * ct;
    s->uy[q] = un * st_ * cos(cph);
    s->uz[q] = un * st_ * sin(cph);
    s->tau[q] = -log(1.0 - R9[1]);
    s->wt[q] = s->w;
    s->id[q] = id;
    s->alive[q] = 1;
    s->tal.E_injected += s->w * eps;
    s->tal.N_injected += s->w;
    s->tal.n_injected += 1.0;
  }
  s->n += cnt;
  s->next_id += cnt;
}

/* ---------------- bulk seeding ----------------
 * n electrons uniform in the box, directions uniform on the sphere
 * (cos theta = 2u - 1), kinetic energy exponential with mean mean_eps,
 * fresh optical depth; draws: block 10 = (eps, cos theta, phi, x),
 * block 11 = (y, z, tau, unused) at the current step. */
void orc_seed(orc_sim *s, int64_t n, double mean_eps) {
  reserve(s, s->n + n);
  const double Lx = s->t.nx * s->t.dx, Ly = s->t.ny * s->t.dx, Lz = s->t.nz * s->t.dx;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t id = (uint32_t)(s->next_id + i);
    double R10[4], R11[4];
    draw(s, id, 10, R10);
    draw(s, id, 11, R11);
    double eps = -mean_eps * log(1.0 - R10[0]);
    double ct = 2.0 * R10[1] - 1.0;
    double st = sqrt((1.0 - ct) * (1.0 + ct));
    double ph = 2.0 * PI * R10[2];
    double un = u_of_eps(eps);
    int64_t q = s->n + i;
    s->x[q] = Lx * R10[3];
    s->y[q] = Ly * R11[0];
    s->z[q] = Lz * R11[1];
    s->ux[q] = un * ct;
    s->uy[q] = un * st * cos(ph);
    s->uz[q] = un * st * sin(ph);
    s->tau[q] = -log(1.0 - R11[2]);
    s->wt[q] = s->w;
    s->id[q] = id;
    s->alive[q] = 1;
    s->tal.E_injected += s->w * eps;
    s->tal.N_injected += s->w;
    s->tal.n_injected += 1.0;
  }
  s->n += n;
  s->next_id += n;
}

/* ---------------- public ---------------- */
orc_sim *orc_create(const orc_target *t, const orc_laser *l, const orc_run *r) {
  if (t->nx < 2 || t->ny < 2 || t->nz < 2) return NULL;
  if (C_L * r->dt >= t->dx) return NULL;
  orc_sim *s = calloc(1, sizeof(orc_sim));
  s->t = *t;
  s->l = *l;
  s->r = *r;
  s->a0 = orc_a0(l->I0, l->lambda);
  s->T_hot = s->a0 * MC2;
  double N_real = (s->a0 > 0.0)
      ? l->eta_l2e * l->I0 * PI * l->spot_r * l->spot_r * l->t_inj / (s->a0 * MC2) : 0.0;
  s->w = l->n_macro > 0 ? N_real / (double)l->n_macro : 1.0;
  s->eps_esc = r->kappa_esc * s->a0 * MC2;
  s->du_reflux = r->kappa_tnsa * s->a0;
  s->n_inj_steps = (int64_t)llround(l->t_inj / r->dt);
  if (s->n_inj_steps < 1) s->n_inj_steps = 1;
  s->nvec = (int64_t)(t->nx + 1) * (t->ny + 1) * (t->nz + 1);
  s->ncell = (int64_t)t->nx * t->ny * t->nz;
  for (int w = 0; w < 13; ++w) s->g[w] = calloc(orc_grid_len(s, w), sizeof(double));
  s->ohm = calloc(s->ncell, sizeof(double));
  for (int64_t c = 0; c < s->ncell; ++c) {
    s->g[ORC_T][c] = t->T0;
    s->g[ORC_TI][c] = t->T0;
    s->g[ORC_ETA][c] = orc_resistivity(t, t->T0);
  }
  int rows = r->n_E + 2;
  s->histE = calloc((size_t)rows * r->n_theta, sizeof(double));
  s->histN = calloc((size_t)rows * r->n_theta, sizeof(double));
  s->history = calloc(r->max_history > 0 ? r->max_history : 1, sizeof(double));
  s->table = malloc((size_t)r->table_rows * r->table_cols * sizeof(double));
  orc_brem_table(t, r->k_min, r->table_E_max, r->table_rows, r->table_cols, s->table);
  return s;
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  free(s->x); free(s->y); free(s->z); free(s->ux); free(s->uy); free(s->uz);
  free(s->tau); free(s->wt); free(s->id); free(s->alive);
  for (int w = 0; w < 13; ++w) free(s->g[w]);
  free(s->histE); free(s->histN); free(s->history); free(s->table); free(s->ohm);
  free(s);
}

#ifdef _OPENMP
/* The electrons of a step on nt threads (the OpenMP build, used only to time
 * the oracle on all host cores): each thread adds into private copies of
 * what the step accumulates (tallies, photon histograms and history,
 * current, drag heat), which are then added to the context's in thread
 * order.  The electrons' own state is written in place (one thread each). */
static void electrons_threads(orc_sim *s, int nt) {
  const size_t hl = (size_t)(s->r.n_E + 2) * (size_t)s->r.n_theta;
  const size_t hy = s->r.max_history > 0 ? (size_t)s->r.max_history : 1;
  const int acc[4] = {ORC_JX, ORC_JY, ORC_JZ, ORC_HEAT};
  orc_sim *loc = malloc((size_t)nt * sizeof(orc_sim));
  for (int t = 0; t < nt; ++t) {
    loc[t] = *s;
    memset(&loc[t].tal, 0, sizeof(orc_tallies));
    loc[t].histE = calloc(hl, sizeof(double));
    loc[t].histN = calloc(hl, sizeof(double));
    loc[t].history = calloc(hy, sizeof(double));
    for (int a = 0; a < 4; ++a) loc[t].g[acc[a]] = calloc(orc_grid_len(s, acc[a]), sizeof(double));
  }
#pragma omp parallel num_threads(nt)
  {
    orc_sim *me = loc + omp_get_thread_num();
#pragma omp for schedule(static)
    for (int64_t ip = 0; ip < s->n; ++ip) particle_update(me, ip);
  }
  double *dst = (double *)&s->tal;
  for (int t = 0; t < nt; ++t) {
    const double *src = (const double *)&loc[t].tal;
    for (size_t k = 0; k < sizeof(orc_tallies) / sizeof(double); ++k) dst[k] += src[k];
  }
  for (int a = 0; a < 4; ++a) {
    double *g = s->g[acc[a]];
    const int64_t len = orc_grid_len(s, acc[a]);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < len; ++q)
      for (int t = 0; t < nt; ++t) g[q] += loc[t].g[acc[a]][q];
  }
  for (int t = 0; t < nt; ++t) {
    for (size_t q = 0; q < hl; ++q) {
      s->histE[q] += loc[t].histE[q];
      s->histN[q] += loc[t].histN[q];
    }
    for (size_t q = 0; q < hy; ++q) s->history[q] += loc[t].history[q];
    free(loc[t].histE); free(loc[t].histN); free(loc[t].history);
    for (int a = 0; a < 4; ++a) free(loc[t].g[acc[a]]);
  }
  free(loc);
}
#endif

int orc_step(orc_sim *s, int64_t nsteps) {
  for (int64_t it = 0; it < nsteps; ++it) {
    memset(s->g[ORC_JX], 0, s->nvec * sizeof(double));
    memset(s->g[ORC_JY], 0, s->nvec * sizeof(double));
    memset(s->g[ORC_JZ], 0, s->nvec * sizeof(double));
    memset(s->g[ORC_HEAT], 0, s->ncell * sizeof(double));
#ifdef _OPENMP
    if (omp_get_max_threads() > 1 && s->n > 0) electrons_threads(s, omp_get_max_threads());
    else
#endif
    for (int64_t ip = 0; ip < s->n; ++ip) particle_update(s, ip);
    int64_t m = 0;
    for (int64_t ip = 0; ip < s->n; ++ip) {
      if (!s->alive[ip]) continue;
      s->x[m] = s->x[ip]; s->y[m] = s->y[ip]; s->z[m] = s->z[ip];
      s->ux[m] = s->ux[ip]; s->uy[m] = s->uy[ip]; s->uz[m] = s->uz[ip];
      s->tau[m] = s->tau[ip]; s->wt[m] = s->wt[ip]; s->id[m] = s->id[ip]; s->alive[m] = 1;
      ++m;
    }
    s->n = m;
    field_update(s);
    heating(s);
    inject(s);
    s->step += 1;
  }
  return 0;
}

void orc_fields(orc_sim *s) {
  field_update(s);
  heating(s);
}

int64_t orc_n_particles(const orc_sim *s) { return s->n; }

void orc_get_particles(const orc_sim *s, double *x, double *y, double *z, double *ux,
                       double *uy, double *uz, double *tau, uint32_t *id) {
  size_t b = (size_t)s->n * sizeof(double);
  memcpy(x, s->x, b); memcpy(y, s->y, b); memcpy(z, s->z, b);
  memcpy(ux, s->ux, b); memcpy(uy, s->uy, b); memcpy(uz, s->uz, b);
  memcpy(tau, s->tau, b);
  memcpy(id, s->id, (size_t)s->n * sizeof(uint32_t));
}

void orc_set_particles(orc_sim *s, int64_t n, const double *x, const double *y,
                       const double *z, const double *ux, const double *uy,
                       const double *uz, const double *tau, const uint32_t *id) {
  reserve(s, n);
  size_t b = (size_t)n * sizeof(double);
  memcpy(s->x, x, b); memcpy(s->y, y, b); memcpy(s->z, z, b);
  memcpy(s->ux, ux, b); memcpy(s->uy, uy, b); memcpy(s->uz, uz, b);
  memcpy(s->tau, tau, b);
  memcpy(s->id, id, (size_t)n * sizeof(uint32_t));
  memset(s->alive, 1, (size_t)n);
  for (int64_t i = 0; i < n; ++i) s->wt[i] = s->w;
  s->n = n;
}

int64_t orc_grid_len(const orc_sim *s, int which) {
  return (which == ORC_T || which == ORC_ETA || which == ORC_HEAT || which == ORC_TI) ? s->ncell
                                                                                       : s->nvec;
}

void orc_get_grid(const orc_sim *s, int which, double *out) {
  memcpy(out, s->g[which], (size_t)orc_grid_len(s, which) * sizeof(double));
}

void orc_set_grid(orc_sim *s, int which, const double *in) {
  memcpy(s->g[which], in, (size_t)orc_grid_len(s, which) * sizeof(double));
}

void orc_get_tallies(const orc_sim *s, orc_tallies *out) { *out = s->tal; }

void orc_reset_tallies(orc_sim *s) {
  memset(&s->tal, 0, sizeof(s->tal));
  int rows = s->r.n_E + 2;
  memset(s->histE, 0, (size_t)rows * s->r.n_theta * sizeof(double));
  memset(s->histN, 0, (size_t)rows * s->r.n_theta * sizeof(double));
  memset(s->history, 0, (size_t)(s->r.max_history > 0 ? s->r.max_history : 1) * sizeof(double));
}

void orc_get_hist(const orc_sim *s, double *hE, double *hN) {
  size_t b = (size_t)(s->r.n_E + 2) * s->r.n_theta * sizeof(double);
  memcpy(hE, s->histE, b);
  memcpy(hN, s->histN, b);
}

void orc_get_history(const orc_sim *s, double *out) {
  memcpy(out, s->history, (size_t)(s->r.max_history > 0 ? s->r.max_history : 0) * sizeof(double));
}

void orc_get_clock(const orc_sim *s, int64_t *step, int64_t *nid) {
  *step = s->step;
  *nid = s->next_id;
}

void orc_set_clock(orc_sim *s, int64_t step, int64_t nid) {
  s->step = step;
  s->next_id = nid;
}

double orc_live_energy(const orc_sim *s) {
  double e = 0.0;
  for (int64_t ip = 0; ip < s->n; ++ip) {
    double u[3] = {s->ux[ip], s->uy[ip], s->uz[ip]};
    e += s->wt[ip] * kinetic(u);
  }
  return e;
}

double orc_field_energy(const orc_sim *s) {
  double e = 0.0;
  for (int c = ORC_BX; c <= ORC_BZ; ++c)
    for (int64_t q = 0; q < s->nvec; ++q) e += s->g[c][q] * s->g[c][q];
  return e / (2.0 * MU0) * s->t.dx * s->t.dx * s->t.dx;
}

double orc_weight(const orc_sim *s) { return s->w; }

void orc_get_weights(const orc_sim *s, double *w) { memcpy(w, s->wt, (size_t)s->n * sizeof(double)); }

void orc_set_weights(orc_sim *s, int64_t n, const double *w) {
  if (n > s->n) n = s->n;
  memcpy(s->wt, w, (size_t)n * sizeof(double));
}
double orc_a0_of(const orc_sim *s) { return s->a0; }
