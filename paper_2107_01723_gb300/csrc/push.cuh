// Per-electron device code of the fast-electron step (arXiv 2107.01723),
// shared by the single-target and the batched push kernels.  See
// particles.cu for the order of the step and the random-number layout.
#pragma once

#include "kernels.h"

namespace hpic {

// ---------------------------------------------------------------- geometry
template <typename R>
struct Axis {
  int iN, iS;  // base node of the node-centred / half-staggered lattice
  R fN, fS;    // fractional offsets
};

// linear weights along one axis; X in cells, n cells.  The half-staggered
// lattice is held at its outermost value within half a cell of a wall.
template <typename R>
__device__ __forceinline__ Axis<R> axis_weights(R X, int n) {
  Axis<R> a;
  int i = (int)m_floor(X);
  i = min(max(i, 0), n - 1);
  a.iN = i;
  a.fN = X - R(i);
  R q = X - R(0.5);
  q = q < R(0) ? R(0) : q;
  q = q > R(n - 1) ? R(n - 1) : q;
  int is = (int)m_floor(q);
  is = min(max(is, 0), n - 1);
  a.iS = is;
  a.fS = q - R(is);
  return a;
}

// the x-neighbour pair (G[q], G[q+1]) through the read-only path.  (Aligned
// 16-byte pair loads and v4 vector reductions were measured slower here:
// the per-lane alignment selects and the +0 lanes cost more than they save.)
template <typename R>
__device__ __forceinline__ void ld_pair(const R *G, int q, R &v0, R &v1) {
  v0 = __ldg(G + q);
  v1 = __ldg(G + q + 1);
}

// the grid as the push kernel sees it; node (i, j, k) lives at i + sy*j + sz*k
template <typename R>
struct Grid {
  const R *F[6];  // Ex Ey Ez Bx By Bz
  R *J[3];
  double *H;
  const R *Fsig;  // F_sigma per cell
  int sy, sz, nx, ny, nz;
  __device__ __forceinline__ int node(int i, int j, int k) const { return i + sy * j + sz * k; }
};

template <typename R>
__device__ __forceinline__ Grid<R> make_grid(const HotK<R> &K, const GView<R> &gv) {
  Grid<R> g;
  for (int c = 0; c < 3; ++c) {
    g.F[c] = gv.E[c];
    g.F[3 + c] = gv.B[c];
    g.J[c] = gv.J[c];
  }
  g.H = gv.H;
  g.Fsig = gv.Fsig;
  g.sy = K.nx + 1;
  g.sz = (K.nx + 1) * (K.ny + 1);
  g.nx = K.nx;
  g.ny = K.ny;
  g.nz = K.nz;
  return g;
}

template <typename R>
__device__ __forceinline__ R trilerp(const Grid<R> &g, int c, int b, R fx, R fy, R fz) {
  const R gx = R(1) - fx;
  R a0, a1, b0, b1, c0, c1, d0, d1;
  ld_pair(g.F[c], b, a0, a1);
  ld_pair(g.F[c], b + g.sy, b0, b1);
  ld_pair(g.F[c], b + g.sz, c0, c1);
  ld_pair(g.F[c], b + g.sz + g.sy, d0, d1);
  const R e00 = a0 * gx + a1 * fx;
  const R e10 = b0 * gx + b1 * fx;
  const R e01 = c0 * gx + c1 * fx;
  const R e11 = d0 * gx + d1 * fx;
  const R e0 = e00 * (R(1) - fy) + e10 * fy;
  const R e1 = e01 * (R(1) - fy) + e11 * fy;
  return e0 * (R(1) - fz) + e1 * fz;
}

// G(u0) = integral_{u0}^{1} s(u)/u du for s(u) = (4/3)(1-u) + u^2
template <typename R>
__device__ __forceinline__ R shape_G(R u0) {
  return R(4.0 / 3.0) * (-m_flog(u0) - (R(1) - u0)) + R(0.5) * (R(1) - u0 * u0);
}

// Photon energy from the inverse-CDF table (rows: ln eps, columns: the
// uniform deviate).  The table holds w = ln(eps/k) / ln(eps/k_min), and the
// sampler returns ln(eps/k) = w ln(eps/k_min) >= 0: the caller forms k =
// eps e^{-x} and the electron's remainder with expm1, so a photon that takes
// nearly all of eps leaves a remainder as accurate as eps itself (k_min
// e^{v ln(eps/k_min)} subtracted from eps loses the digits of k in FP32).
// The column and its fraction come from the deviate's 23 bits m in integers,
// (m + 1/2) 2^-23 (cols-1) = (2m+1)(cols-1) 2^-24, exact in either precision.
template <typename R>
__device__ __forceinline__ R sample_log_ratio(R k_min, R t_inv_dlog, int rows, int cols,
                                              const R *__restrict__ tab, R eps, uint32_t bits) {
  const R lr = m_log(eps / k_min);
  R L = lr * t_inv_dlog;
  int i = (int)m_floor(L);
  i = min(max(i, 0), rows - 2);
  R f = L - R(i);
  f = f < R(0) ? R(0) : (f > R(1) ? R(1) : f);
  const unsigned long long cpos =
      (unsigned long long)(2u * (bits >> 9) + 1u) * (unsigned long long)(cols - 1);
  const int j = (int)(cpos >> 24);  // <= cols - 2 since 2m+1 < 2^24
  const R g = R((uint32_t)(cpos & 0xFFFFFFull)) * R(1.0 / 16777216.0);
  const R *t0 = tab + i * cols + j;
  const R *t1 = t0 + cols;
  const R va = __ldg(t0) * (R(1) - g) + __ldg(t0 + 1) * g;
  const R vb = __ldg(t1) * (R(1) - g) + __ldg(t1 + 1) * g;
  return (va * (R(1) - f) + vb * f) * lr;
}

// photon polar angle: theta = t/gamma, t ~ t/(1+t^2)^2 truncated at theta = pi
template <typename R>
__device__ __forceinline__ R photon_theta(R gamma, R u) {
  const R a = R(3.14159265358979323846) * gamma;
  const R a2 = a * a;
  const R F = u * a2 / (R(1) + a2);
  const R omF = (R(1) - u) + u / (R(1) + a2);
  return m_sqrt(F / omF) / gamma;
}

// per-thread tally accumulators
constexpr int kAccN = 13;
__device__ constexpr int kAccSlot[kAccN] = {
    T_W_FIELD, T_E_DRAG, T_E_ESC, T_E_REFLUX, T_E_XRAY, T_E_XRAY_ABOVE, T_N_ESC,
    T_N_REFLUX, T_N_REFLUX_ABS, T_N_CUT, T_N_EMIT, T_PSTEPS, T_N_NONFINITE};

// the frequent sums stay in registers; the rare ones (escape, reflux,
// photons, non-finite electrons) go straight into a shared-memory array of
// kAccN doubles indexed like kAccSlot, so they hold no registers
enum AccIndex { A_W = 0, A_DRAG, A_ESC, A_REF, A_X, A_XA, A_N_ESC, A_N_REF, A_N_REFABS, A_N_CUT,
                A_N_EMIT, A_N_STEPS, A_N_NF };

template <typename R>
struct Acc {
  R W = 0, drag = 0;
  int n_cut = 0, n_steps = 0;
  // in the order of kAccSlot (the rare slots are zero here)
  __device__ __forceinline__ void values(double (&v)[kAccN]) const {
#pragma unroll
    for (int q = 0; q < kAccN; ++q) v[q] = 0.0;
    v[A_W] = (double)W; v[A_DRAG] = (double)drag; v[A_N_CUT] = n_cut; v[A_N_STEPS] = n_steps;
  }
};

// Escape or reflux at each face the move crossed, in the order x, y, z
// (Sec. II.A).  Rare, so kept out of line.
template <typename R>
struct Crossing {
  R pos[3], u[3];
  double esc, ref;
  int n_esc, n_ref, n_refabs;
  bool alive;
};

template <typename R>
__device__ __noinline__ Crossing<R> cross_faces(R eps_esc, R du_reflux, R sigma_dtheta,
                                                uint32_t step, uint32_t target, uint32_t key0,
                                                uint32_t key1, uint32_t id, R w, int nx, int ny,
                                                int nz, R p0, R p1, R p2, R u0, R u1, R u2) {
  Crossing<R> c;
  c.pos[0] = p0; c.pos[1] = p1; c.pos[2] = p2;
  c.u[0] = u0; c.u[1] = u1; c.u[2] = u2;
  c.esc = 0.0; c.ref = 0.0; c.n_esc = 0; c.n_ref = 0; c.n_refabs = 0; c.alive = true;
  R *pos = c.pos, *u = c.u;
  const int nn[3] = {nx, ny, nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R L = R(nn[a]);
    if (pos[a] >= R(0) && pos[a] <= L) continue;
    const R e_out = kinetic(u[0], u[1], u[2]);
    if (e_out >= eps_esc) {
      c.esc += (double)(w * e_out);
      ++c.n_esc;
      c.alive = false;
      return c;
    }
    const bool low = pos[a] < R(0);
    pos[a] = low ? -pos[a] : R(2) * L - pos[a];
    u[a] = -u[a];
    const R un = m_sqrt_rn(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const R un2 = un - du_reflux;
    if (un2 <= R(0)) {
      c.ref += (double)(w * e_out);
      ++c.n_refabs;
      c.alive = false;
      return c;
    }
    const U4 r2 = philox10(step, id, 2u + a, target, key0, key1);
    const R xi = sigma_dtheta * (unif<R>(r2.a) - R(0.5));
    R st, ct, sp, cp;
    m_sincos(xi, &st, &ct);
    m_sincos2pi(unif<R>(r2.b), &sp, &cp);
    const R inv = m_div_rn(R(1), un);
    R d[3] = {u[0] * inv, u[1] * inv, u[2] * inv};
    rotate(d[0], d[1], d[2], ct, st, cp, sp);
    if (low && d[a] < R(0)) d[a] = -d[a];
    if (!low && d[a] > R(0)) d[a] = -d[a];
    u[0] = un2 * d[0]; u[1] = un2 * d[1]; u[2] = un2 * d[2];
    c.ref += (double)(w * (e_out - kinetic(u[0], u[1], u[2])));
    ++c.n_ref;
  }
  return c;
}

struct StepCtx {
  uint32_t step, key0, key1, target;
  long long step_ll;
};

// What the emission of one photon needs besides the electron (App. B);
// filled only on that rare path.
template <typename R>
struct EmitIn {
  const R *tab;
  double *hist, *history;
  double w_shared, inv_boost_d, ce_thr;
  long long max_history;
  int t_rows, t_cols, n_E, n_th, weighted;
  R k_min, t_inv_dlog, tE_min, tE_max, inv_dlogE, th_scale, inv_boost, E_cut;
};

template <typename R>
struct EmitOut {
  R eps, ux, uy, uz, tau, heat;
  double x, xa;
  bool alive;
};

// One photon at zero optical depth: energy from the table, polar angle about
// the electron, energy x angle tallies, fresh optical depth, and the
// electron's remainder (cut below E_cut).  Rare, so kept out of line.
template <typename R>
__device__ __noinline__ EmitOut<R> emit_photon(const EmitIn<R> e, StepCtx sc, uint32_t id, R w,
                                               R eps, R ux, R uy, R uz) {
  EmitOut<R> o;
  o.x = 0.0;
  o.xa = 0.0;
  o.heat = R(0);
  o.alive = true;
  const U4 r1 = philox10(sc.step, id, 1u, sc.target, sc.key0, sc.key1);
  const R xk = sample_log_ratio(e.k_min, e.t_inv_dlog, e.t_rows, e.t_cols, e.tab, eps, r1.a);
  const R k = eps * m_exp(-xk);
  const R thg = photon_theta(R(1) + eps, unif<R>(r1.b));
  const R un = m_sqrt_rn(ux * ux + uy * uy + uz * uz);
  R dx = ux / un, dy = uy / un, dz = uz / un;
  R st, ct, sp, cp;
  m_sincos(thg, &st, &ct);
  m_sincos2pi(unif<R>(r1.c), &sp, &cp);
  rotate(dx, dy, dz, ct, st, cp, sp);
  const R th = m_atan2(m_sqrt(dy * dy + dz * dz), dx);  // polar angle from +x
  // photon tally: energy row (underflow, log bins, overflow) x polar bin
  int row;
  if (k < e.tE_min) row = 0;
  else if (k >= e.tE_max) row = e.n_E + 1;
  else row = min(max(1 + (int)m_floor(e.inv_dlogE * m_log(k / e.tE_min)), 1), e.n_E);
  const int col = min(max((int)m_floor(th * e.th_scale), 0), e.n_th - 1);
  // photon weight: the electron's own, or the shared FP64 weight exactly
  const double wph = (e.weighted ? (double)w : e.w_shared) * e.inv_boost_d;
  const double ek = wph * (double)k;
  const int hb = row * e.n_th + col;
  atomicAdd(e.hist + hb, ek);
  atomicAdd(e.hist + (e.n_E + 2) * e.n_th + hb, wph);
  o.x = ek;
  if ((double)k >= e.ce_thr) {
    o.xa = ek;
    if (sc.step_ll < e.max_history) atomicAdd(e.history + sc.step_ll, ek);
  }
  o.tau = -m_log(R(1) - unif<R>(r1.d));
  // eps - k/boost = eps ((1 - 1/boost) + (1 - e^{-x})/boost)
  eps *= (R(1) - e.inv_boost) - e.inv_boost * m_expm1(-xk);
  if (eps < e.E_cut) {
    o.heat = w * eps;
    o.alive = false;
  } else {
    const R s = m_div_rn(u_of_eps(eps), un);
    ux *= s; uy *= s; uz *= s;
  }
  o.eps = eps; o.ux = ux; o.uy = uy; o.uz = uz;
  return o;
}

// Advance one live electron through the step.  Returns false when the
// electron is absorbed or escapes (the caller marks its slot dead).  On
// true, the state holds x^{n+1}, u^{n+1} and tau, ig = 1/gamma of u^{n+1}
// (the deposit's velocity factor), and its current is deposited.  NS: 1 for
// a single-element solid (the element loops vanish), 4 for up to four
// elements counted at run time.
template <typename R, int NS>
__device__ __forceinline__ bool advance(const Consts &K, const HotK<R> &h, const Grid<R> &g,
                                        const R *__restrict__ tab, const TallyView &tv,
                                        const StepCtx &sc, uint32_t id, R w, R &X, R &Y, R &Zc,
                                        R &ux, R &uy, R &uz, R &tau, Acc<R> &acc, double *rare,
                                        R &heat_out, int &heat_cell, R &ig) {
  const int nx = h.nx, ny = h.ny, nz = h.nz;

  // ---- gather at x^n
  const bool unbounded = (K.physics & P_UNBOUNDED) != 0;
  const Axis<R> ax = axis_weights(X, nx), ay = axis_weights(Y, ny), az = axis_weights(Zc, nz);
  R Ex = R(0), Ey = R(0), Ez = R(0), Bx = R(0), By = R(0), Bz = R(0);
  if (!unbounded) {
    Ex = trilerp(g, 0, g.node(ax.iS, ay.iN, az.iN), ax.fS, ay.fN, az.fN);
    Ey = trilerp(g, 1, g.node(ax.iN, ay.iS, az.iN), ax.fN, ay.fS, az.fN);
    Ez = trilerp(g, 2, g.node(ax.iN, ay.iN, az.iS), ax.fN, ay.fN, az.fS);
    Bx = trilerp(g, 3, g.node(ax.iN, ay.iS, az.iS), ax.fN, ay.fS, az.fS);
    By = trilerp(g, 4, g.node(ax.iS, ay.iN, az.iS), ax.fS, ay.fN, az.fS);
    Bz = trilerp(g, 5, g.node(ax.iS, ay.iS, az.iN), ax.fS, ay.fS, az.fN);
  }

  // ---- Boris push: half kick, rotation, half kick
  const R eps0 = kinetic(ux, uy, uz);
  {
    const R mx = ux + R(0.5) * Ex, my = uy + R(0.5) * Ey, mz = uz + R(0.5) * Ez;
    const R gm = m_sqrt(R(1) + mx * mx + my * my + mz * mz);
    const R hh = R(0.5) / gm;
    const R tx = Bx * hh, ty = By * hh, tz = Bz * hh;
    const R s2 = R(2) / (R(1) + tx * tx + ty * ty + tz * tz);
    const R sx = tx * s2, sy_ = ty * s2, sz_ = tz * s2;
    const R qx = mx + (my * tz - mz * ty), qy = my + (mz * tx - mx * tz), qz = mz + (mx * ty - my * tx);
    ux = mx + (qy * sz_ - qz * sy_) + R(0.5) * Ex;
    uy = my + (qz * sx - qx * sz_) + R(0.5) * Ey;
    uz = mz + (qx * sy_ - qy * sx) + R(0.5) * Ez;
  }
  R eps = kinetic(ux, uy, uz);
  acc.W += w * (eps0 - eps);
  R heat = 0;
  bool alive = true;

  // ---- tracking cut and ionisation drag, Eq. (5)
  if (eps < h.E_cut) {
    heat += w * eps;
    alive = false;
  } else if (K.physics & P_DRAG) {
    const R gam = R(1) + eps;
    const R beta = u_of_eps(eps) / gam;
    const R ig = R(1) / gam;
    const R le = m_flog(eps), lh = R(0.5) * m_flog(gam + R(1));
    const R a2 = R(0.909) * ig * ig, a1 = R(0.818) * ig;
    R de = R(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {  // the elements' stopping powers add
      if (NS > 1 && s >= h.n_solids) break;  // constant indices: no local-memory copy
      R br = le + h.L_I[s] + lh + a2 - a1 - R(0.246);
      br = br < R(0) ? R(0) : br;
      de += h.K_ion[s] / beta * br;
    }
    const R eps1 = eps - de;
    if (eps1 < h.E_cut) {
      heat += w * eps;
      alive = false;
    } else {
      const R s = m_div_rn(u_of_eps(eps1), m_sqrt_rn(ux * ux + uy * uy + uz * uz));
      ux *= s; uy *= s; uz *= s;
      heat += w * de;
      eps = eps1;
    }
  }

  // ---- Davies scatter, Eq. (B4): polar Gamma*sigma, azimuth uniform
  if (alive && (K.physics & P_SCATTER)) {
    const U4 r0 = philox10(sc.step, id, 0u, sc.target, sc.key0, sc.key1);
    const R u2 = ux * ux + uy * uy + uz * uz;
    const R inv = m_rsqrt_rn(u2);
    const R un = u2 * inv;
    const R gam = m_sqrt(R(1) + u2);
    R var = R(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {  // the elements' variances add
      if (NS > 1 && s >= h.n_solids) break;
      R lg = m_flog(h.K_lg[s] * un);
      lg = lg < R(0) ? R(0) : lg;
      var += h.K_sc[s] * gam / (un * un * un) * lg;
    }
    const R sig = m_sqrt(var);
    R s2, c2, st, ct;
    // Box-Muller normal deviate (its cosine changes only the deflection)
    const R gauss = m_sqrt(R(-2) * m_log(unif<R>(r0.a))) * m_fcos2pi(unif<R>(r0.b));
    m_sincos(gauss * sig, &st, &ct);
    m_sincos2pi(unif<R>(r0.c), &s2, &c2);
    R dx = ux * inv, dy = uy * inv, dz = uz * inv;
    rotate(dx, dy, dz, ct, st, c2, s2);
    ux = un * dx; uy = un * dy; uz = un * dz;
  }

  // ---- bremsstrahlung by optical depth (App. B)
  if (alive && (K.physics & P_BREM) && eps > h.k_min) {
    R dtau = h.K_tau * u_of_eps(eps) / eps * shape_G(h.k_min / eps);
    if (K.physics & P_FSIGMA) dtau *= __ldg(g.Fsig + ax.iN + nx * (ay.iN + ny * az.iN));
    tau -= dtau;
    if (tau <= R(0)) {
      EmitIn<R> e;
      e.tab = tab; e.hist = tv.hist; e.history = tv.history;
      e.w_shared = h.w_d; e.inv_boost_d = K.inv_boost; e.ce_thr = K.ce_thr;
      e.max_history = K.max_history;
      e.t_rows = K.t_rows; e.t_cols = K.t_cols; e.n_E = K.n_E; e.n_th = K.n_th;
      e.weighted = K.weighted;
      e.k_min = h.k_min; e.t_inv_dlog = h.t_inv_dlog; e.tE_min = h.tE_min; e.tE_max = h.tE_max;
      e.inv_dlogE = h.inv_dlogE; e.th_scale = h.th_scale; e.inv_boost = h.inv_boost;
      e.E_cut = h.E_cut;
      const EmitOut<R> o = emit_photon<R>(e, sc, id, w, eps, ux, uy, uz);
      atomicAdd(rare + A_X, o.x);
      if (o.xa != 0.0) atomicAdd(rare + A_XA, o.xa);
      atomicAdd(rare + A_N_EMIT, 1.0);
      tau = o.tau;
      eps = o.eps;
      ux = o.ux; uy = o.uy; uz = o.uz;
      heat += o.heat;
      alive = o.alive;
    }
  }

  acc.drag += heat;
  heat_out = heat;  // deposited by the warp in the cell of x^n
  heat_cell = ax.iN + nx * (ay.iN + ny * az.iN);
  if (!alive) {
    ++acc.n_cut;
    return false;
  }

  // ---- move, then escape or reflux at each face crossed (out of line: rare)
  ig = R(1) / m_sqrt(R(1) + ux * ux + uy * uy + uz * uz);
  R pos[3] = {X + ux * ig * h.cdt, Y + uy * ig * h.cdt, Zc + uz * ig * h.cdt};
  if (!unbounded && !(pos[0] >= R(0) && pos[0] <= R(nx) && pos[1] >= R(0) && pos[1] <= R(ny) &&
                      pos[2] >= R(0) && pos[2] <= R(nz))) {
    const Crossing<R> c = cross_faces<R>(h.eps_esc, h.du_reflux, h.sigma_dtheta, sc.step,
                                         sc.target, sc.key0, sc.key1, id, w, nx, ny, nz,
                                         pos[0], pos[1], pos[2], ux, uy, uz);
    if (c.esc != 0.0) atomicAdd(rare + A_ESC, c.esc);
    if (c.ref != 0.0) atomicAdd(rare + A_REF, c.ref);
    if (c.n_esc) atomicAdd(rare + A_N_ESC, (double)c.n_esc);
    if (c.n_ref) atomicAdd(rare + A_N_REF, (double)c.n_ref);
    if (c.n_refabs) atomicAdd(rare + A_N_REFABS, (double)c.n_refabs);
    if (!c.alive) return false;
    pos[0] = c.pos[0]; pos[1] = c.pos[1]; pos[2] = c.pos[2];
    ux = c.u[0]; uy = c.u[1]; uz = c.u[2];
    ig = R(1) / m_sqrt(R(1) + ux * ux + uy * uy + uz * uz);
  }
  X = pos[0]; Y = pos[1]; Zc = pos[2];

  return true;  // the caller's warp deposits the current at x^{n+1}
}

// ---------------------------------------------------------------- warp deposits
// A warp adds its electrons' current and drag heat to the grid together.
//
// Current.  The warp groups its electrons by the cell of x^{n+1} (lanes with
// equal cells found by one match instruction); each electron takes the row
// of its place in that grouping, so a cell's electrons hold consecutive rows,
// and writes its 24 CIC values (per component c the 8 corners of its own
// lattice, times w v_c / c) as row `row` of a column-major stage.  Lane l
// then walks column l down the 32 rows keeping two running sums, one for the
// rows whose half-staggered base along c is the cell's own node (off = 1)
// and one for those whose base is the node below (off = 0): with keep = 0
// on the first row of a cell and 1 elsewhere, (s0, s1) = keep (s0, s1) +
// (x [off = 0], x [off = 1]), one packed two-wide FMA per row.  At the last
// row of a cell the pair is that cell's sum for the two nodes of the column:
// one reduction per node, the lanes of a reduction instruction on distinct
// addresses.  Cell ends are tested once per four rows.
//
// Drag heat goes to the cell of x^n: a segmented scan across the lanes, in
// row order, over runs of equal heat cell, and one FP64 reduction per run.
//
// Node of a corner: with nk the node index of the cell of x^{n+1}, corner
// (a, b, e) of component c of an electron whose axis-c staggered index is
// i_c - 1 + off is nk + a + sy b + sz e - (1 - off) stride_c.
constexpr int kDepCols = 24;               // 3 components x 8 corners
constexpr uint32_t kNoKey = 0xFFFFFFFFu;   // row with nothing to deposit
constexpr uint32_t kNoCell = (1u << 27) - 1u;  // cell key of such a row (cells < 2^27 - 1)
constexpr unsigned kFull = 0xffffffffu;

// Stage of one warp, in elements of R: 24 columns of 32 rows, each column
// padded by 16 bytes (a 16-byte read of the same rows by eight lanes falls
// in eight distinct bank groups), then the keep pairs of the 32 rows, then
// the 32 rows' cell node keys (uint32; first the electron of each row).
template <typename R>
__host__ __device__ constexpr int dep_stride() { return 32 + 16 / (int)sizeof(R); }
template <typename R>
__host__ __device__ constexpr int dep_keep0() { return kDepCols * dep_stride<R>(); }
template <typename R>
__host__ __device__ constexpr int dep_words() {
  return dep_keep0<R>() + 64 + 32 * 4 / (int)sizeof(R);
}

template <typename R>
struct Pair;  // the two running sums of a column, and the segmented-sum step
template <>
struct Pair<float> {
  float2 v;
  __device__ __forceinline__ static Pair make(float a, float b) { Pair q; q.v = make_float2(a, b); return q; }
  __device__ __forceinline__ void fma_keep(const Pair &keep, const Pair &x) { v = __ffma2_rn(v, keep.v, x.v); }
  __device__ __forceinline__ float a() const { return v.x; }
  __device__ __forceinline__ float b() const { return v.y; }
};
template <>
struct Pair<double> {
  double2 v;
  __device__ __forceinline__ static Pair make(double a, double b) { Pair q; q.v = make_double2(a, b); return q; }
  __device__ __forceinline__ void fma_keep(const Pair &keep, const Pair &x) {
    v.x = fma(v.x, keep.v.x, x.v.x);
    v.y = fma(v.y, keep.v.y, x.v.y);
  }
  __device__ __forceinline__ double a() const { return v.x; }
  __device__ __forceinline__ double b() const { return v.y; }
};

template <typename R>
struct Vec16;  // the rows one 16-byte shared load covers
template <>
struct Vec16<float> {
  static constexpr int n = 4;
  __device__ __forceinline__ static void load(const float *p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <>
struct Vec16<double> {
  static constexpr int n = 2;
  __device__ __forceinline__ static void load(const double *p, double (&v)[2]) {
    const double2 q = *reinterpret_cast<const double2 *>(p);
    v[0] = q.x; v[1] = q.y;
  }
};

// current J += w (u/gamma) S(x^{n+1}) of the lanes with dep set (ig =
// 1/gamma), and drag heat into the cell heat_cell of x^n (heat == 0:
// nothing); buf is this warp's stage.  Every lane of the warp must call it.
template <typename R>
__device__ __forceinline__ void warp_deposit(const Grid<R> &g, R *__restrict__ buf,
                                             bool dep, R w, R X, R Y, R Zc, R ux, R uy, R uz,
                                             R ig, R heat, int heat_cell) {
  constexpr int S = dep_stride<R>();
  const int lane = threadIdx.x & 31;

  // ---- this lane's electron, written as row `row` of the cell grouping
  if (!dep) { X = R(0); Y = R(0); Zc = R(0); }  // finite weights, zero values
  const Axis<R> ax = axis_weights(X, g.nx), ay = axis_weights(Y, g.ny), az = axis_weights(Zc, g.nz);
  R v[3] = {R(0), R(0), R(0)};
  uint32_t nk = kNoKey, ck = kNoCell;
  if (dep) {
    v[0] = w * ux * ig;
    v[1] = w * uy * ig;
    v[2] = w * uz * ig;
    nk = (uint32_t)g.node(ax.iN, ay.iN, az.iN);
    ck = (uint32_t)(ax.iN + g.nx * (ay.iN + g.ny * az.iN));
  }
  const int offs = (ax.iS - ax.iN + 1) | ((ay.iS - ay.iN + 1) << 1) | ((az.iS - az.iN + 1) << 2);
  const uint32_t hk = (heat != R(0) && heat_cell >= 0) ? (uint32_t)heat_cell : kNoKey;
  // the lanes sharing a cell take consecutive rows, the groups in the order
  // of their first lanes (offsets: a prefix sum of the group sizes over the
  // groups' first lanes); lane p then learns which electron holds row p (src)
  const unsigned same = __match_any_sync(kFull, ck);
  const int lead = __ffs((int)same) - 1;
  const int size_here = lane == lead ? __popc(same) : 0;
  int incl = size_here;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  const int row = __shfl_sync(kFull, incl - size_here, lead) + __popc(same & ((1u << lane) - 1u));
  uint32_t *rowkey = reinterpret_cast<uint32_t *>(buf + dep_keep0<R>() + 64);
  rowkey[row] = (uint32_t)lane;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R fx = c == 0 ? ax.fS : ax.fN, fy = c == 1 ? ay.fS : ay.fN, fz = c == 2 ? az.fS : az.fN;
    const R z0 = v[c] * (R(1) - fz), z1 = v[c] * fz;
    const R yz[4] = {z0 * (R(1) - fy), z0 * fy, z1 * (R(1) - fy), z1 * fy};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      buf[(8 * c + 2 * q) * S + row] = yz[q] * (R(1) - fx);
      buf[(8 * c + 2 * q + 1) * S + row] = yz[q] * fx;
    }
  }
  __syncwarp();
  const int src = (int)rowkey[lane];
  // from here on lane p speaks for row p
  const uint32_t pnk = __shfl_sync(kFull, nk, src), phk = __shfl_sync(kFull, hk, src);
  const int poffs = __shfl_sync(kFull, offs, src);
  R ph = __shfl_sync(kFull, heat, src);
  const uint32_t nk_up = __shfl_up_sync(kFull, pnk, 1), nk_dn = __shfl_down_sync(kFull, pnk, 1);
  const uint32_t hk_up = __shfl_up_sync(kFull, phk, 1), hk_dn = __shfl_down_sync(kFull, phk, 1);
  const bool head_c = lane == 0 || nk_up != pnk;
  const uint32_t endc = __ballot_sync(kFull, lane == 31 || nk_dn != pnk);
  const uint32_t offx = __ballot_sync(kFull, poffs & 1);
  const uint32_t offy = __ballot_sync(kFull, poffs & 2);
  const uint32_t offz = __ballot_sync(kFull, poffs & 4);
  __syncwarp();
  {
    const R k = head_c ? R(0) : R(1);
    *reinterpret_cast<Pair<R> *>(buf + dep_keep0<R>() + 2 * lane) = Pair<R>::make(k, k);
    rowkey[lane] = pnk;
  }
  __syncwarp();

  // ---- column `lane` (lanes 24-31 walk column 23 again and add nothing)
  const int col = lane < kDepCols ? lane : kDepCols - 1;
  const int c = col >> 3;
  const uint32_t offm = c == 0 ? offx : (c == 1 ? offy : offz);
  R *J = c == 0 ? g.J[0] : (c == 1 ? g.J[1] : g.J[2]);
  const int o1 = (col & 1) + g.sy * ((col >> 1) & 1) + g.sz * ((col >> 2) & 1);
  const int sc = c == 0 ? 1 : (c == 1 ? g.sy : g.sz);
  const bool adds = lane < kDepCols;
  const R *colp = buf + col * S;
  const R *keep = buf + dep_keep0<R>();
  const uint32_t *rk = rowkey;
  uint32_t om = offm, em = endc;  // shifted down by the rows walked
  Pair<R> s = Pair<R>::make(R(0), R(0));
  constexpr int V = Vec16<R>::n;
  // rolled over the rows (a copy of the reduction code per chunk of rows
  // would not fit the instruction cache), unrolled within a chunk
#pragma unroll 1
  for (int r0 = 0; r0 < 32; r0 += V) {
    R x[V];
    Vec16<R>::load(colp, x);
    R kv[2 * V];  // the keep pairs of these rows, 16 bytes at a time
#pragma unroll
    for (int q = 0; q < 2 * V; q += Vec16<R>::n) {
      R t[Vec16<R>::n];
      Vec16<R>::load(keep + q, t);
#pragma unroll
      for (int e = 0; e < Vec16<R>::n; ++e) kv[q + e] = t[e];
    }
    Pair<R> sr[V];
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const bool up = (om >> q) & 1u;
      s.fma_keep(Pair<R>::make(kv[2 * q], kv[2 * q + 1]),
                 Pair<R>::make(up ? R(0) : x[q], up ? x[q] : R(0)));
      sr[q] = s;
    }
    const uint32_t ends = em & ((1u << V) - 1u);
    if (ends) {  // warp-uniform: a cell ends in these rows
#pragma unroll
      for (int q = 0; q < V; ++q) {
        if ((ends >> q) & 1u) {
          const uint32_t kc = rk[q];
          if (adds && kc != kNoKey) {
            const long long q1 = (long long)kc + o1;
            if (sr[q].b() != R(0)) atomicAdd(J + q1, sr[q].b());
            if (sr[q].a() != R(0)) atomicAdd(J + (q1 - sc), sr[q].a());
          }
        }
      }
    }
    om >>= V;
    em >>= V;
    colp += V;
    keep += 2 * V;
    rk += V;
  }

  // ---- drag heat: segmented scan over runs of equal heat cell in row order
  bool head_h = lane == 0 || hk_up != phk;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const R hu = __shfl_up_sync(kFull, ph, o);
    const bool fu = __shfl_up_sync(kFull, head_h, o);
    if (lane >= o && !head_h) {
      ph += hu;
      head_h = fu;
    }
  }
  if ((lane == 31 || hk_dn != phk) && phk != kNoKey && ph != R(0))
    atomicAdd(g.H + phk, (double)ph);
  __syncwarp();  // the stage is rewritten by the warp's next electrons
}

// ---------------------------------------------------------------- one warp's step
// evict-first access to the streaming electron state
template <typename R>
__device__ __forceinline__ R ld_stream(const R *p) { return __ldcs(p); }
template <typename R>
__device__ __forceinline__ void st_stream(R *p, R v) { __stcs(p, v); }

// The 32 lanes of a warp advance the electrons in slots ip (one per lane;
// in_range false: nothing there) through the step, then deposit their
// current and drag heat together through the warp's shared-memory stage
// (dep_words<R>() elements, 16-byte aligned).  Every lane of the warp must
// call it.  MODE kPushSort: the step also sorts, and *so (with *shift: see
// SortOut; read only then, so it may stay in shared memory) says where the
// electrons go; kPushKeys: the step also keys the next sort (*ko); the
// pointers may be null otherwise.
template <typename R, int NS, int MODE>
__device__ __forceinline__ void push_warp(const Consts &K, const HotK<R> &h, const Grid<R> &g,
                                          const R *__restrict__ tab, const TallyView &tv,
                                          const StepCtx &sc, const PView<R> &p, long long ip,
                                          bool in_range, Acc<R> &acc, double *rare,
                                          R *__restrict__ stage, const SortOut<R> *so,
                                          const long long *shift, const KeyOut<R> *ko) {
  constexpr bool SORT = MODE == kPushSort;
  bool live = false, dep = false;
  uint32_t id = kDead;
  R X = 0, Y = 0, Zc = 0, ux = 0, uy = 0, uz = 0, tau = 0, heat = 0, w = h.w, ig = 0;
  int heat_cell = -1;
  if (in_range) {
    // the state is loaded together with the id, not after testing it, so
    // that a slot costs one memory round trip (a dead slot's values are
    // read and left unused)
    id = ld_stream(p.id + ip);
    X = ld_stream(p.x + ip); Y = ld_stream(p.y + ip); Zc = ld_stream(p.z + ip);
    ux = ld_stream(p.ux + ip); uy = ld_stream(p.uy + ip); uz = ld_stream(p.uz + ip);
    tau = ld_stream(p.tau + ip);
    if (K.weighted) w = ld_stream(p.w + ip);  // uniform over the launch
    if (id != kDead) {
      if (isfinite(X) && isfinite(Y) && isfinite(Zc) && isfinite(ux) && isfinite(uy) &&
          isfinite(uz) && isfinite(tau)) {
        live = true;
      } else {
        if constexpr (SORT)
          so->dst.id[(long long)so->offsets[so->keys[ip]] + so->ranks[ip] + *shift] = kDead;
        else
          p.id[ip] = kDead;
        atomicAdd(rare + A_N_NF, 1.0);
      }
    }
  }
  if (live) {
    ++acc.n_steps;
    dep = advance<R, NS>(K, h, g, tab, tv, sc, id, w, X, Y, Zc, ux, uy, uz, tau, acc, rare, heat,
                         heat_cell, ig);
    if constexpr (SORT) {  // loaded here so that no register holds them through the step
      const long long q =
          (long long)so->offsets[ld_stream(so->keys + ip)] + ld_stream(so->ranks + ip) + *shift;
      const PView<R> &o = so->dst;
      if (dep) {
        st_stream(o.x + q, X); st_stream(o.y + q, Y); st_stream(o.z + q, Zc);
        st_stream(o.ux + q, ux); st_stream(o.uy + q, uy); st_stream(o.uz + q, uz);
        st_stream(o.tau + q, tau);
        if (K.weighted) st_stream(o.w + q, w);
        o.id[q] = id;
      } else {
        o.id[q] = kDead;
      }
    } else if (dep) {
      st_stream(p.x + ip, X); st_stream(p.y + ip, Y); st_stream(p.z + ip, Zc);
      st_stream(p.ux + ip, ux); st_stream(p.uy + ip, uy); st_stream(p.uz + ip, uz);
      st_stream(p.tau + ip, tau);
      if constexpr (MODE == kPushKeys) {  // the next sort's key and rank
        const R a = ko->lead * ig;
        int i = (int)m_floor(X + a * ux), j = (int)m_floor(Y + a * uy),
            k = (int)m_floor(Zc + a * uz);
        i = min(max(i, 0), K.nx - 1);
        j = min(max(j, 0), K.ny - 1);
        k = min(max(k, 0), K.nz - 1);
        const uint32_t key = tile_key(i, j, k, K.nti, K.ntj);
        ko->keys[ip] = key;
        ko->ranks[ip] = agg_inc(ko->counts, key);
      }
    } else {
      p.id[ip] = kDead;
    }
  }
  if (!(K.physics & P_UNBOUNDED))  // uniform over the warp
    warp_deposit(g, stage, dep, w, X, Y, Zc, ux, uy, uz, ig, heat, heat_cell);
}

// ---------------------------------------------------------------- injection
// One new electron of Eq. (B1) in slot q: at x = 1e-6 cells on the laser
// disc, kinetic energy exponential with mean a0 m_e c^2 (App. B), direction
// uniform in solid angle inside the cone about +x, fresh optical depth.
// Returns its kinetic energy (m_e c^2).
// 1 - cos of the cone half-angle for an electron of kinetic energy eps
// (m_e c^2): the laser's, or with the Moore cap the smaller of it and
// atan(sqrt(2/(gamma - 1))), whose 1 - cos is written without cancellation
// as (2/(gamma + 1)) / (1 + sqrt((gamma - 1)/(gamma + 1)))
template <typename R>
__device__ __forceinline__ R cone_omc(const Consts &K, R eps) {
  R omc = R(K.omc_cone);
  if (K.moore) {
    const R gp = R(2) + eps;  // gamma + 1
    const R m = (R(2) / gp) / (R(1) + m_sqrt(eps / gp));
    omc = m < omc ? m : omc;
  }
  return omc;
}

template <typename R>
__device__ __forceinline__ R inject_one(const Consts &K, const PView<R> &p, long long q,
                                        uint32_t id, uint32_t step) {
  const U4 r8 = philox10(step, id, 8u, K.target_index, K.key0, K.key1);
  const U4 r9 = philox10(step, id, 9u, K.target_index, K.key0, K.key1);
  const R rr = R(K.spot_r) * m_sqrt(unif<R>(r8.a));
  R sp, cp;
  m_sincos2pi(unif<R>(r8.b), &sp, &cp);
  const R eps = -R(K.T_hot) * m_log(R(1) - unif<R>(r8.c));
  const R omc = unif<R>(r8.d) * cone_omc(K, eps);  // 1 - cos(theta)
  const R ct = R(1) - omc;
  const R stt = m_sqrt(omc * (R(2) - omc));
  R sc, cc;
  m_sincos2pi(unif<R>(r9.a), &sc, &cc);
  const R un = u_of_eps(eps);
  p.x[q] = R(1e-6);
  p.y[q] = R(K.spot_y) + rr * cp;
  p.z[q] = R(K.spot_z) + rr * sp;
  p.ux[q] = un * ct;
  p.uy[q] = un * stt * cc;
  p.uz[q] = un * stt * sc;
  p.tau[q] = -m_log(R(1) - unif<R>(r9.b));
  p.id[q] = id;
  return eps;
}

// One electron of the Gaussian envelope (App. B) in face cell (j, k): uniform
// over the cell's face at x = 1e-6 cells, kinetic energy exponential with the
// local mean `mean` (m_e c^2), direction uniform in the (capped) cone; the
// caller stores its weight.  Returns its kinetic energy.
template <typename R>
__device__ __forceinline__ R inject_cell_one(const Consts &K, const PView<R> &p, long long q,
                                             uint32_t id, uint32_t step, int j, int k, R mean) {
  const U4 r8 = philox10(step, id, 8u, K.target_index, K.key0, K.key1);
  const U4 r9 = philox10(step, id, 9u, K.target_index, K.key0, K.key1);
  const R eps = -mean * m_log(R(1) - unif<R>(r8.c));
  const R omc = unif<R>(r8.d) * cone_omc(K, eps);
  const R ct = R(1) - omc;
  const R stt = m_sqrt(omc * (R(2) - omc));
  R sc, cc;
  m_sincos2pi(unif<R>(r9.a), &sc, &cc);
  const R un = u_of_eps(eps);
  p.x[q] = R(1e-6);
  p.y[q] = R(j) + unif<R>(r8.a);
  p.z[q] = R(k) + unif<R>(r8.b);
  p.ux[q] = un * ct;
  p.uy[q] = un * stt * cc;
  p.uz[q] = un * stt * sc;
  p.tau[q] = -m_log(R(1) - unif<R>(r9.b));
  p.id[q] = id;
  return eps;
}

}  // namespace hpic
