// Device-side building blocks of the fast-electron step (arXiv 2107.01723).
//
// Units inside the kernels are normalised so that FP32 keeps its range:
//   length in cells (dx), time in steps (dt), momentum u = p/(m_e c),
//   energy in m_e c^2, electric field as the per-step momentum kick
//   E_n = -e E dt/(m_e c), magnetic field as the per-step rotation
//   parameter B_n = -e B dt/m_e, current as J = sum w (u/gamma) S(x)
//   (electrons x beta per cell).  Every SI coefficient of the paper is folded
//   into these units once, in double precision, on the host (see api.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hpic {

constexpr uint32_t kDead = 0xFFFFFFFFu;  // id of an absorbed/escaped slot

// tally slots (device array of doubles); energies in m_e c^2 x weight
enum Tally {
  T_E_INJ = 0, T_N_INJ, T_W_FIELD, T_E_DRAG, T_E_XRAY, T_E_XRAY_ABOVE,
  T_E_ESC, T_E_REFLUX, T_E_OHMIC, T_N_INJECTED, T_N_ESC, T_N_REFLUX,
  T_N_REFLUX_ABS, T_N_CUT, T_N_EMIT, T_PSTEPS, T_N_NONFINITE,
  T_E_LIVE, T_E_BFIELD, T_COUNT
};

// device-resident counters
struct Counters {
  long long n;        // particle slots in use (live + dead until the next sort)
  long long step;     // step counter (Philox counter word 0)
  long long next_id;  // id of the next injected electron
  long long inj_cnt;  // electrons injected by the current step's injection
  unsigned int flags; // bit 0: capacity exceeded during injection
};

// Constants of one target, folded on the host.  R is the particle/field
// precision; temperature, resistivity and tallies are always double.
struct Consts {
  int nx, ny, nz;
  long long nvec, ncell;
  int nti, ntj, ntk;       // 4x4x4 cell tiles per axis (sort order)
  long long nkeys;         // nti*ntj*ntk*64 sort keys (the dead bin is nkeys)
  double cdt_dx;           // c dt / dx: cells per step at v = c
  double w;                // macro-electron weight (real electrons)
  // per element of the solid (a compound has up to kMaxSolids):
  // drag, Eq. (5): d_eps = sum K_ion/beta * bracket, L_I = ln(m_e c^2 / I_ex);
  // scatter, Eq. (B4): sigma^2 = sum K_sc gamma/u^3 ln(K_lg u)
  int n_solids;
  double K_ion[4], L_I[4], K_sc[4], K_lg[4];
  // heating of a compound, Eq. (A7): 1/C averaged with the weights ne_frac
  // (n_e of each element over the total), T' = T Tp_fac_s
  double ne_frac[4], Tp_fac_s[4];
  // bremsstrahlung optical depth: d_tau = K_tau u/eps G(k_min/eps)
  double K_tau, k_min, boost, inv_boost;
  // cut and reflux (Sec. II.A)
  double E_cut, eps_esc, du_reflux, sigma_dtheta;
  // photon tally
  int n_E, n_th;
  double tE_min, tE_max, inv_dlogE;   // n_E / ln(tE_max/tE_min)
  double ce_thr;
  int max_history;
  // inverse-CDF table
  int t_rows, t_cols;
  double t_inv_dlog;                  // (rows-1)/ln(E_max/k_min)
  // fields, Eqs. (A2)-(A3)
  double F_curl, F_j;
  // heating, Eqs. (A4)-(A8), SI
  double F_ohm, F_H, dx3, heat_den, Tp_fac;
  double eta_num, A_hot, B_cold, eta_max, lambda1;
  double eta_hot_c, eta_cold_c;  // eta_num / A_hot, eta_num / B_cold (0 without lambda1)
  double eta_Tlo, eta_Thi;            // eta(T) is at its cap for eta_Tlo < T < eta_Thi (K)
  // F_sigma (App. B) = 1 + fs_q (ln T_i / 2 + fs_c), T_i in K
  double fs_q, fs_c;
  // e-i equilibration (App. A): rate_e = ei_a / (T_e m_i + T_i m_e)^(3/2)
  // (masses in u), rate_i = Z* rate_e
  double ei_a, ei_mi, ei_me, Zstar;
  // injection, Eq. (B1)
  double T_hot, spot_r, spot_y, spot_z, omc_cone;  // omc_cone = 1 - cos(cone)
  long long n_macro, n_inj_steps;
  // RNG
  uint32_t key0, key1, target_index;
  int physics;
  // Gaussian injection envelope (App. B): per_cell electrons in each of the
  // n_inj_cells cells of inj_cells while g = exp(-g_c (s + 1/2 - t_pk)^2) >=
  // g_min (s in steps); weight inj_unit sqrt(f g), mean energy T_hot sqrt(f g)
  int weighted;   // electrons carry their own weight
  int moore;      // Moore-scaling cap on the cone half-angle
  long long per_cell, n_inj_cells;
  double g_c, t_pk, g_min, inj_unit;
  const void *inj_cells;
};

// one injecting face cell: indices and sqrt(f(r)) at its centre
struct InjCell {
  int j, k;
  double sf;
};

enum {
  P_DRAG = 1, P_SCATTER = 2, P_BREM = 4, P_FIELDS = 8, P_FARADAY = 16, P_HEATING = 32,
  P_UNBOUNDED = 64, P_FSIGMA = 128, P_EI = 256
};

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds, each two
// 32x32 multiplies whose high halves are mixed with the other counter words
// and a Weyl-sequence key.
struct U4 { uint32_t a, b, c, d; };

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// open-interval uniform from the top 23 bits; exact in float and double
template <typename R>
__device__ __forceinline__ R unif(uint32_t x) {
  return (R(x >> 9) + R(0.5)) * R(1.0 / 8388608.0);
}

// ---------------------------------------------------------------- math wrappers
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
// hardware log (absolute error ~5e-7) for terms of order 1-10 whose error
// budget allows it; exact log in double precision
__device__ __forceinline__ float m_flog(float x) { return __logf(x); }
__device__ __forceinline__ double m_flog(double x) { return log(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ void m_sincos(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void m_sincos(double x, double *s, double *c) { sincos(x, s, c); }
// sin/cos of 2 pi u without rounding 2 pi u first
__device__ __forceinline__ void m_sincos2pi(float u, float *s, float *c) { sincospif(2.0f * u, s, c); }
__device__ __forceinline__ void m_sincos2pi(double u, double *s, double *c) { sincospi(2.0 * u, s, c); }
// Round-to-nearest square root and division.  The FP32 particle kernels are
// compiled with approximate division and square root; these wrappers keep
// IEEE rounding where the push converts between an electron's energy and
// its momentum (kinetic, u_of_eps, the rescale after drag or a photon) and
// where it builds the frame of a rotation, so that no systematic rounding
// bias enters an energy change that no tally records.
__device__ __forceinline__ float m_sqrt_rn(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ double m_sqrt_rn(double x) { return sqrt(x); }
__device__ __forceinline__ float m_div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double m_div_rn(double a, double b) { return a / b; }
__device__ __forceinline__ float m_rsqrt_rn(float x) { return __frsqrt_rn(x); }
__device__ __forceinline__ double m_rsqrt_rn(double x) { return 1.0 / sqrt(x); }
// cos(2 pi u) for u in (0, 1): in FP32 from the hardware unit on the angle
// 2 pi (u - 1) for u > 1/2 (exact shift, |angle| <= pi, absolute error
// about 5e-7); exact cospi in FP64
__device__ __forceinline__ float m_fcos2pi(float u) {
  return __cosf(6.28318530717958647692f * (u > 0.5f ? u - 1.0f : u));
}
__device__ __forceinline__ double m_fcos2pi(double u) { return cospi(2.0 * u); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }

// Sort key of cell (i, j, k): 4x4x4 tiles in x-fastest tile order, cells
// x-fastest inside a tile, so consecutive electrons share a compact box.
__host__ __device__ __forceinline__ uint32_t tile_key(int i, int j, int k, int nti, int ntj) {
  const uint32_t t = (uint32_t)(((k >> 2) * ntj + (j >> 2)) * nti + (i >> 2));
  return t * 64u + (uint32_t)(((k & 3) << 4) | ((j & 3) << 2) | (i & 3));
}

// kinetic energy (m_e c^2) of momentum u, without the gamma - 1 cancellation
template <typename R>
__device__ __forceinline__ R kinetic(R ux, R uy, R uz) {
  const R u2 = ux * ux + uy * uy + uz * uz;
  return m_div_rn(u2, R(1) + m_sqrt_rn(R(1) + u2));
}

// momentum |u| of kinetic energy e (m_e c^2)
template <typename R>
__device__ __forceinline__ R u_of_eps(R e) { return m_sqrt_rn(e * (e + R(2))); }

// Rotate unit d by polar angle (cos ct, sin st) at azimuth (cp, sp) in the
// orthonormal frame of Duff et al., "Building an orthonormal basis,
// revisited", JCGT 6(1), 2017.
template <typename R>
__device__ __forceinline__ void rotate(R &dx, R &dy, R &dz, R ct, R st, R cp, R sp) {
  const R sg = dz >= R(0) ? R(1) : R(-1);
  const R a = m_div_rn(R(-1), sg + dz);
  const R b = dx * dy * a;
  const R e1x = R(1) + sg * dx * dx * a, e1y = sg * b, e1z = -sg * dx;
  const R e2x = b, e2y = sg + dy * dy * a, e2z = -dy;
  const R px = e1x * cp + e2x * sp, py = e1y * cp + e2y * sp, pz = e1z * cp + e2z * sp;
  const R ox = dx * ct + px * st, oy = dy * ct + py * st, oz = dz * ct + pz * st;
  dx = ox; dy = oy; dz = oz;
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// warp-aggregated atomic increment: lanes with equal keys share one atomic
__device__ __forceinline__ uint32_t agg_inc(uint32_t *ctr, uint32_t key) {
  const unsigned mask = __activemask();
  const unsigned peers = __match_any_sync(mask, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(ctr + key, (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + rank;
}

// Sum `nq` per-thread values over the block and add them to dst[slot[q]].
// smem must hold nq * 32 doubles.  All threads of the block must call it.
template <int NQ>
__device__ __forceinline__ void block_flush(const double (&v)[NQ], const int (&slot)[NQ],
                                            double *dst, double *smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double s = warp_sum(v[q]);
    if (lane == 0) smem[q * 32 + warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
    for (int w = 0; w < nwarps; ++w) s += smem[threadIdx.x * 32 + w];
    if (s != 0.0) atomicAdd(dst + slot[threadIdx.x], s);
  }
  __syncthreads();
}

}  // namespace hpic
