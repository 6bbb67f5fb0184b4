// Fused per-electron step of the hybrid-PIC method (arXiv 2107.01723) and
// the injection of new hot electrons.
//
// One thread advances one electron through the whole step, so its state is
// read once and written once per step:
//   gather E, B at x^n (trilinear on the Yee lattice)
//   relativistic Boris push                          (Lorentz force)
//   ionisation drag, explicit in energy              Eq. (5)
//   Davies angular scatter                           Eq. (B4)
//   bremsstrahlung by optical depth + photon tally   App. B
//   x^{n+1} = x^n + v dt, then escape/reflux         Sec. II.A
//   current deposit at x^{n+1}                       j_h of Eq. (A2)
// Random numbers: Philox4x32-10, counter (step, id, block, target), key = seed;
// block 0 scatter, 1 emission, 2..4 reflux on x/y/z faces, 8-9 injection.
#include "kernels.h"

namespace hpic {

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

template <typename R>
__device__ __forceinline__ R trilerp(const R *__restrict__ G, long long b, int sy, long long sz,
                                     R fx, R fy, R fz) {
  const R gx = R(1) - fx;
  const R c00 = __ldg(G + b) * gx + __ldg(G + b + 1) * fx;
  const R c10 = __ldg(G + b + sy) * gx + __ldg(G + b + sy + 1) * fx;
  const R c01 = __ldg(G + b + sz) * gx + __ldg(G + b + sz + 1) * fx;
  const R c11 = __ldg(G + b + sz + sy) * gx + __ldg(G + b + sz + sy + 1) * fx;
  const R c0 = c00 * (R(1) - fy) + c10 * fy;
  const R c1 = c01 * (R(1) - fy) + c11 * fy;
  return c0 * (R(1) - fz) + c1 * fz;
}

template <typename R>
__device__ __forceinline__ void spread(R *G, long long b, int sy, long long sz, R fx, R fy, R fz,
                                       R v) {
  const R gx = R(1) - fx, gy = R(1) - fy, gz = R(1) - fz;
  const R v0 = v * gz, v1 = v * fz;
  atomicAdd(G + b, v0 * gy * gx);
  atomicAdd(G + b + 1, v0 * gy * fx);
  atomicAdd(G + b + sy, v0 * fy * gx);
  atomicAdd(G + b + sy + 1, v0 * fy * fx);
  atomicAdd(G + b + sz, v1 * gy * gx);
  atomicAdd(G + b + sz + 1, v1 * gy * fx);
  atomicAdd(G + b + sz + sy, v1 * fy * gx);
  atomicAdd(G + b + sz + sy + 1, v1 * fy * fx);
}

// G(u0) = integral_{u0}^{1} s(u)/u du for s(u) = (4/3)(1-u) + u^2
template <typename R>
__device__ __forceinline__ R shape_G(R u0) {
  return R(4.0 / 3.0) * (-m_log(u0) - (R(1) - u0)) + R(0.5) * (R(1) - u0 * u0);
}

// photon energy from the inverse-CDF table (rows: ln eps, columns: r)
template <typename R>
__device__ __forceinline__ R sample_k(const Consts &K, const R *__restrict__ tab, R eps, R r) {
  const R lr = m_log(eps / R(K.k_min));
  R L = lr * R(K.t_inv_dlog);
  int i = (int)m_floor(L);
  i = min(max(i, 0), K.t_rows - 2);
  R f = L - R(i);
  f = f < R(0) ? R(0) : (f > R(1) ? R(1) : f);
  const R cpos = r * R(K.t_cols - 1);
  int j = (int)m_floor(cpos);
  j = min(max(j, 0), K.t_cols - 2);
  const R g = cpos - R(j);
  const R *t0 = tab + (long long)i * K.t_cols + j;
  const R *t1 = t0 + K.t_cols;
  const R va = __ldg(t0) * (R(1) - g) + __ldg(t0 + 1) * g;
  const R vb = __ldg(t1) * (R(1) - g) + __ldg(t1 + 1) * g;
  const R v = va * (R(1) - f) + vb * f;
  return R(K.k_min) * m_exp(v * lr);
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

template <typename R>
__global__ void __launch_bounds__(256)
k_push(const Consts K, PView<R> p, GView<R> g, const R *__restrict__ tab, Counters *cnt,
       TallyView tv) {
  __shared__ double smem[13 * 32];
  const long long n = cnt->n;
  const long long step_ll = cnt->step;
  const uint32_t step = (uint32_t)step_ll;
  const int nx = K.nx, ny = K.ny, nz = K.nz;
  const int sy = nx + 1;
  const long long sz = (long long)(nx + 1) * (ny + 1);
  const R w = R(K.w);
  const R cdt = R(K.cdt_dx);
  const R Ecut = R(K.E_cut);

  R a_W = 0, a_drag = 0;
  double a_esc = 0, a_ref = 0, a_x = 0, a_xa = 0;
  int c_esc = 0, c_ref = 0, c_refabs = 0, c_cut = 0, c_emit = 0, c_steps = 0, c_nf = 0;

  for (long long ip = blockIdx.x * (long long)blockDim.x + threadIdx.x; ip < n;
       ip += (long long)gridDim.x * blockDim.x) {
    const uint32_t id = p.id[ip];
    if (id == kDead) continue;
    R X = p.x[ip], Y = p.y[ip], Zc = p.z[ip];
    R ux = p.ux[ip], uy = p.uy[ip], uz = p.uz[ip];
    R tau = p.tau[ip];
    if (!(isfinite(X) && isfinite(Y) && isfinite(Zc) && isfinite(ux) && isfinite(uy) &&
          isfinite(uz) && isfinite(tau))) {
      p.id[ip] = kDead;
      ++c_nf;
      continue;
    }
    ++c_steps;
    const U4 r0 = philox10(step, id, 0u, K.target_index, K.key0, K.key1);

    // ---- gather at x^n
    const Axis<R> ax = axis_weights(X, nx), ay = axis_weights(Y, ny), az = axis_weights(Zc, nz);
    const R Ex = trilerp(g.E[0], ax.iS + sy * (long long)ay.iN + sz * az.iN, sy, sz, ax.fS, ay.fN, az.fN);
    const R Ey = trilerp(g.E[1], ax.iN + sy * (long long)ay.iS + sz * az.iN, sy, sz, ax.fN, ay.fS, az.fN);
    const R Ez = trilerp(g.E[2], ax.iN + sy * (long long)ay.iN + sz * az.iS, sy, sz, ax.fN, ay.fN, az.fS);
    const R Bx = trilerp(g.B[0], ax.iN + sy * (long long)ay.iS + sz * az.iS, sy, sz, ax.fN, ay.fS, az.fS);
    const R By = trilerp(g.B[1], ax.iS + sy * (long long)ay.iN + sz * az.iS, sy, sz, ax.fS, ay.fN, az.fS);
    const R Bz = trilerp(g.B[2], ax.iS + sy * (long long)ay.iS + sz * az.iN, sy, sz, ax.fS, ay.fS, az.fN);
    const long long cell = ax.iN + (long long)nx * (ay.iN + (long long)ny * az.iN);

    // ---- Boris push: half kick, rotation, half kick
    const R eps0 = kinetic(ux, uy, uz);
    {
      const R mx = ux + R(0.5) * Ex, my = uy + R(0.5) * Ey, mz = uz + R(0.5) * Ez;
      const R gm = m_sqrt(R(1) + mx * mx + my * my + mz * mz);
      const R h = R(0.5) / gm;
      const R tx = Bx * h, ty = By * h, tz = Bz * h;
      const R s2 = R(2) / (R(1) + tx * tx + ty * ty + tz * tz);
      const R sx = tx * s2, sy_ = ty * s2, sz_ = tz * s2;
      const R qx = mx + (my * tz - mz * ty), qy = my + (mz * tx - mx * tz), qz = mz + (mx * ty - my * tx);
      ux = mx + (qy * sz_ - qz * sy_) + R(0.5) * Ex;
      uy = my + (qz * sx - qx * sz_) + R(0.5) * Ey;
      uz = mz + (qx * sy_ - qy * sx) + R(0.5) * Ez;
    }
    R eps = kinetic(ux, uy, uz);
    a_W += w * (eps0 - eps);
    R heat = 0;
    bool alive = true;

    // ---- tracking cut and ionisation drag, Eq. (5)
    if (eps < Ecut) {
      heat += w * eps;
      alive = false;
    } else if (K.physics & P_DRAG) {
      const R gam = R(1) + eps;
      const R un = u_of_eps(eps);
      const R beta = un / gam;
      const R ig = R(1) / gam;
      R br = m_log(eps) + R(K.L_I) + R(0.5) * m_log(gam + R(1)) + R(0.909) * ig * ig -
             R(0.818) * ig - R(0.246);
      br = br < R(0) ? R(0) : br;
      const R de = R(K.K_ion) / beta * br;
      const R eps1 = eps - de;
      if (eps1 < Ecut) {
        heat += w * eps;
        alive = false;
      } else {
        const R sc = u_of_eps(eps1) / m_sqrt(ux * ux + uy * uy + uz * uz);
        ux *= sc; uy *= sc; uz *= sc;
        heat += w * de;
        eps = eps1;
      }
    }

    // ---- Davies scatter, Eq. (B4): polar Gamma*sigma, azimuth uniform
    if (alive && (K.physics & P_SCATTER)) {
      const R un = m_sqrt(ux * ux + uy * uy + uz * uz);
      const R gam = m_sqrt(R(1) + un * un);
      R lg = m_log(R(K.K_lg) * un);
      lg = lg < R(0) ? R(0) : lg;
      const R sig = m_sqrt(R(K.K_sc) * gam / (un * un * un) * lg);
      R s1, c1, s2, c2, st, ct;
      m_sincos2pi(unif<R>(r0.b), &s1, &c1);
      const R gauss = m_sqrt(R(-2) * m_log(unif<R>(r0.a))) * c1;
      m_sincos(gauss * sig, &st, &ct);
      m_sincos2pi(unif<R>(r0.c), &s2, &c2);
      const R inv = R(1) / un;
      R dx = ux * inv, dy = uy * inv, dz = uz * inv;
      rotate(dx, dy, dz, ct, st, c2, s2);
      ux = un * dx; uy = un * dy; uz = un * dz;
    }

    // ---- bremsstrahlung by optical depth (App. B)
    if (alive && (K.physics & P_BREM) && eps > R(K.k_min)) {
      const R un_e = u_of_eps(eps);
      tau -= R(K.K_tau) * un_e / eps * shape_G(R(K.k_min) / eps);
      if (tau <= R(0)) {
        const U4 r1 = philox10(step, id, 1u, K.target_index, K.key0, K.key1);
        const R k = sample_k(K, tab, eps, unif<R>(r1.a));
        const R gam = R(1) + eps;
        const R thg = photon_theta(gam, unif<R>(r1.b));
        const R un = m_sqrt(ux * ux + uy * uy + uz * uz);
        R dx = ux / un, dy = uy / un, dz = uz / un;
        R st, ct, sp, cp;
        m_sincos(thg, &st, &ct);
        m_sincos2pi(unif<R>(r1.c), &sp, &cp);
        rotate(dx, dy, dz, ct, st, cp, sp);
        dx = dx > R(1) ? R(1) : (dx < R(-1) ? R(-1) : dx);
        const R th = m_acos(dx);
        // photon tally: energy row (underflow, log bins, overflow) x polar bin
        int row;
        if (k < R(K.tE_min)) row = 0;
        else if (k >= R(K.tE_max)) row = K.n_E + 1;
        else {
          row = 1 + (int)m_floor(R(K.inv_dlogE) * m_log(k / R(K.tE_min)));
          row = min(max(row, 1), K.n_E);
        }
        int col = (int)m_floor(th * R(K.n_th / 3.14159265358979323846));
        col = min(max(col, 0), K.n_th - 1);
        const double wph = K.w * K.inv_boost;
        const double ek = wph * (double)k;
        const long long hb = (long long)row * K.n_th + col;
        atomicAdd(tv.hist + hb, ek);
        atomicAdd(tv.hist + (long long)(K.n_E + 2) * K.n_th + hb, wph);
        a_x += ek;
        if ((double)k >= K.ce_thr) {
          a_xa += ek;
          if (step_ll < K.max_history) atomicAdd(tv.history + step_ll, ek);
        }
        ++c_emit;
        tau = -m_log(R(1) - unif<R>(r1.d));
        eps -= k * R(K.inv_boost);
        if (eps < Ecut) {
          heat += w * eps;
          alive = false;
        } else {
          const R sc = u_of_eps(eps) / un;
          ux *= sc; uy *= sc; uz *= sc;
        }
      }
    }

    if (!alive) {
      ++c_cut;
      p.id[ip] = kDead;
    } else {
      // ---- move, then escape or reflux at each face crossed (x, y, z)
      R ig = R(1) / m_sqrt(R(1) + ux * ux + uy * uy + uz * uz);
      R pos[3] = {X + ux * ig * cdt, Y + uy * ig * cdt, Zc + uz * ig * cdt};
      R u[3] = {ux, uy, uz};
      const int nn[3] = {nx, ny, nz};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R L = R(nn[a]);
        if (!alive || (pos[a] >= R(0) && pos[a] <= L)) continue;
        const R e_out = kinetic(u[0], u[1], u[2]);
        if (e_out >= R(K.eps_esc)) {
          a_esc += (double)(w * e_out);
          ++c_esc;
          alive = false;
          continue;
        }
        const bool low = pos[a] < R(0);
        pos[a] = low ? -pos[a] : R(2) * L - pos[a];
        u[a] = -u[a];
        const R un = m_sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const R un2 = un - R(K.du_reflux);
        if (un2 <= R(0)) {
          a_ref += (double)(w * e_out);
          ++c_refabs;
          alive = false;
          continue;
        }
        const U4 r2 = philox10(step, id, 2u + a, K.target_index, K.key0, K.key1);
        const R xi = R(K.sigma_dtheta) * (unif<R>(r2.a) - R(0.5));
        R st, ct, sp, cp;
        m_sincos(xi, &st, &ct);
        m_sincos2pi(unif<R>(r2.b), &sp, &cp);
        const R inv = R(1) / un;
        R d[3] = {u[0] * inv, u[1] * inv, u[2] * inv};
        rotate(d[0], d[1], d[2], ct, st, cp, sp);
        if (low && d[a] < R(0)) d[a] = -d[a];
        if (!low && d[a] > R(0)) d[a] = -d[a];
        u[0] = un2 * d[0]; u[1] = un2 * d[1]; u[2] = un2 * d[2];
        a_ref += (double)(w * (e_out - kinetic(u[0], u[1], u[2])));
        ++c_ref;
      }
      if (!alive) {
        p.id[ip] = kDead;
      } else {
        p.x[ip] = pos[0]; p.y[ip] = pos[1]; p.z[ip] = pos[2];
        p.ux[ip] = u[0]; p.uy[ip] = u[1]; p.uz[ip] = u[2];
        p.tau[ip] = tau;
        // ---- current deposit at x^{n+1}: J += w (u/gamma) S(x)
        ig = R(1) / m_sqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const Axis<R> bx = axis_weights(pos[0], nx), by = axis_weights(pos[1], ny),
                      bz = axis_weights(pos[2], nz);
        spread(g.J[0], bx.iS + sy * (long long)by.iN + sz * bz.iN, sy, sz, bx.fS, by.fN, bz.fN, w * u[0] * ig);
        spread(g.J[1], bx.iN + sy * (long long)by.iS + sz * bz.iN, sy, sz, bx.fN, by.fS, bz.fN, w * u[1] * ig);
        spread(g.J[2], bx.iN + sy * (long long)by.iN + sz * bz.iS, sy, sz, bx.fN, by.fN, bz.fS, w * u[2] * ig);
      }
    }
    a_drag += heat;
    if (heat != R(0)) atomicAdd(g.H + cell, (double)heat);
  }

  const double v[13] = {(double)a_W, (double)a_drag, a_esc, a_ref, a_x, a_xa, (double)c_esc,
                        (double)c_ref, (double)c_refabs, (double)c_cut, (double)c_emit,
                        (double)c_steps, (double)c_nf};
  const int slot[13] = {T_W_FIELD, T_E_DRAG, T_E_ESC, T_E_REFLUX, T_E_XRAY, T_E_XRAY_ABOVE,
                        T_N_ESC, T_N_REFLUX, T_N_REFLUX_ABS, T_N_CUT, T_N_EMIT, T_PSTEPS,
                        T_N_NONFINITE};
  block_flush<13>(v, slot, tv.tal, smem);
}

// ---------------------------------------------------------------- injection
// Eq. (B1) with flat-top envelopes: step s < S injects floor((s+1)N/S) -
// floor(sN/S) electrons at x = 1e-6 cells on a disc, energies exponential
// with mean a0 m_e c^2 (App. B), directions uniform in solid angle in a cone.
template <typename R>
__global__ void __launch_bounds__(256)
k_inject(const Consts K, PView<R> p, Counters *cnt, long long cap, TallyView tv) {
  __shared__ double smem[3 * 32];
  const long long st = cnt->step;
  if (st >= K.n_inj_steps) return;
  const long long S = K.n_inj_steps, N = K.n_macro;
  const long long c = (N * (st + 1)) / S - (N * st) / S;
  const long long n0 = cnt->n, id0 = cnt->next_id;
  const uint32_t step = (uint32_t)st;
  double e_inj = 0.0, n_inj = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < c;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = n0 + i;
    if (q >= cap) {
      atomicOr(&cnt->flags, 1u);
      continue;
    }
    const uint32_t id = (uint32_t)(id0 + i);
    const U4 r8 = philox10(step, id, 8u, K.target_index, K.key0, K.key1);
    const U4 r9 = philox10(step, id, 9u, K.target_index, K.key0, K.key1);
    const R rr = R(K.spot_r) * m_sqrt(unif<R>(r8.a));
    R sp, cp;
    m_sincos2pi(unif<R>(r8.b), &sp, &cp);
    const R eps = -R(K.T_hot) * m_log(R(1) - unif<R>(r8.c));
    const R ct = R(1) - unif<R>(r8.d) * (R(1) - R(K.cos_cone));
    const R stt = m_sqrt((R(1) - ct) * (R(1) + ct));
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
    e_inj += K.w * (double)eps;
    n_inj += 1.0;
  }
  const double v[3] = {e_inj, n_inj * K.w, n_inj};
  const int slot[3] = {T_E_INJ, T_N_INJ, T_N_INJECTED};
  block_flush<3>(v, slot, tv.tal, smem);
  if (blockIdx.x == 0 && threadIdx.x == 0) cnt->inj_cnt = c;
}

// closes a step: append the injected electrons, advance the clock
__global__ void k_advance(Counters *cnt, long long cap) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const long long c = cnt->inj_cnt;
    long long n = cnt->n + c;
    cnt->n = n < cap ? n : cap;
    cnt->next_id += c;
    cnt->step += 1;
    cnt->inj_cnt = 0;
  }
}

// ---------------------------------------------------------------- launchers
template <typename R>
void launch_push(const Consts &K, PView<R> p, GView<R> g, const R *table, Counters *cnt,
                 TallyView tv, int grid, cudaStream_t st) {
  k_push<R><<<grid, 256, 0, st>>>(K, p, g, table, cnt, tv);
}

template <typename R>
void launch_inject(const Consts &K, PView<R> p, Counters *cnt, long long cap, TallyView tv,
                   int grid, cudaStream_t st) {
  k_inject<R><<<grid, 256, 0, st>>>(K, p, cnt, cap, tv);
}

void launch_advance(Counters *cnt, long long cap, cudaStream_t st) {
  k_advance<<<1, 32, 0, st>>>(cnt, cap);
}

template void launch_push<float>(const Consts &, PView<float>, GView<float>, const float *,
                                 Counters *, TallyView, int, cudaStream_t);
template void launch_push<double>(const Consts &, PView<double>, GView<double>, const double *,
                                  Counters *, TallyView, int, cudaStream_t);
template void launch_inject<float>(const Consts &, PView<float>, Counters *, long long, TallyView,
                                   int, cudaStream_t);
template void launch_inject<double>(const Consts &, PView<double>, Counters *, long long,
                                    TallyView, int, cudaStream_t);

}  // namespace hpic
