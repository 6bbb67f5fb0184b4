// The paper's three-macro-electron estimate of the hot-electron loss
// channels (arXiv 2107.01723, Sec. III.B), one GPU thread per parameter set.
//
// Per set: the exponential injection spectrum is cut at the X-ray threshold
// and the escape energy into three macro-electrons (warm, emitting,
// escaping), each integrated by RK4 in its path length through the four
// continuous stopping powers of Eqs. (stop_brem), (stop_ion), (stop_tnsa)
// and (stop_field).  FP64 throughout: the sets are independent and few, so
// the work is ALU-bound on GB300's FP64 units, not memory-bound.
#include <cmath>
#include <string>

#include "hpic.h"
#include "kernels.h"

namespace hpic {
namespace {

// CODATA 2018 SI values
constexpr double kQE = 1.602176634e-19;
constexpr double kME = 9.1093837015e-31;
constexpr double kC = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;
constexpr double kHbar = 6.62607015e-34 / (2.0 * kPi);
constexpr double kMC2 = kME * kC * kC;

struct Stopping {
  double Kb;        // S_brem = Kb gamma
  double Ki;        // S_ion = Ki / beta^2 * bracket
  double St;        // S_tnsa
  double Fc, r, tc; // S_field = Fc / (x tc + r)^2
  double I_ex, th;
  int mech;
};

// brem, ion, tnsa, field and the above-threshold photon rate at (eps, x)
__device__ __forceinline__ void rates(const Stopping &s, double eps, double x, double k[5]) {
  const double gam = 1.0 + eps / kMC2;
  k[0] = (s.mech & HPIC_MODEL_BREM) ? s.Kb * gam : 0.0;
  k[1] = 0.0;
  if ((s.mech & HPIC_MODEL_ION) && eps > 0.0) {
    const double ig = 1.0 / gam;
    const double br = log(eps / s.I_ex) + 0.5 * log(gam + 1.0) + 0.909 * ig * ig - 0.818 * ig - 0.246;
    if (br > 0.0) k[1] = s.Ki / (1.0 - ig * ig) * br;
  }
  k[2] = (s.mech & HPIC_MODEL_TNSA) ? s.St : 0.0;
  if (s.mech & HPIC_MODEL_FIELD) {
    const double rr = x * s.tc + s.r;
    k[3] = s.Fc / (rr * rr);
  } else {
    k[3] = 0.0;
  }
  k[4] = ((s.mech & HPIC_MODEL_BREM) && eps > s.th) ? s.Kb * (1.0 + (eps - s.th) / kMC2) : 0.0;
}

// one macro-electron; per-electron losses into acc[0..3] (channels), acc[4]
// (photons above threshold), acc[5] (escaped); returns the path length
__device__ double run_macro(const Stopping &s, const hpic_model_in &m, double eps, bool escaping,
                            double acc[6], long long &steps) {
  double x = 0.0;
  const double x_field = s.r / s.tc;
  for (long long it = 0; it < 10000000ll; ++it) {  // bounded: sets are validated
    if (!escaping && eps <= m.E_stop_J) {
      acc[1] += eps;
      return x;
    }
    if (escaping && x >= m.Lx_m) {
      acc[5] += eps;
      return x;
    }
    if (eps <= 0.0) return x;
    double k1[5], k2[5], k3[5], k4[5];
    rates(s, eps, x, k1);
    const double t1 = k1[0] + k1[1] + k1[2] + k1[3];
    if (!(t1 > 0.0)) {  // nothing slows it down any more
      acc[escaping ? 5 : 1] += eps;
      return escaping ? m.Lx_m : x;
    }
    double h = m.rel_step * eps / t1;
    if (s.mech & HPIC_MODEL_FIELD) h = fmin(h, m.rel_step * (x + x_field));
    if (escaping && x + h > m.Lx_m) h = m.Lx_m - x;
    rates(s, eps - 0.5 * h * t1, x + 0.5 * h, k2);
    const double t2 = k2[0] + k2[1] + k2[2] + k2[3];
    rates(s, eps - 0.5 * h * t2, x + 0.5 * h, k3);
    const double t3 = k3[0] + k3[1] + k3[2] + k3[3];
    rates(s, eps - h * t3, x + h, k4);
    ++steps;
    double d[5], de = 0.0;
#pragma unroll
    for (int q = 0; q < 5; ++q) d[q] = h / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) de += d[q];
    if (de >= eps) {  // stops inside the step: share what is left
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += eps * d[q] / de;
      acc[4] += d[4] * eps / de;
      return x + h * eps / de;
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] += d[q];
    eps -= de;
    x += h;
  }
  return x;
}

__global__ void __launch_bounds__(128) k_model(long long n, const hpic_model_in *__restrict__ in,
                                               hpic_model_out *__restrict__ out) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const hpic_model_in m = in[p];
    hpic_model_out o;
    const double a0 = 8.5e-6 * sqrt(m.I0_Wm2 * m.lambda_m * m.lambda_m);  // Eq. (1)
    const double T = a0 * kMC2 * m.mean_sqrt_fg;
    Stopping s;
    const double Lrad = log(5.6 * kPi * kEps0 * kHbar * kC / (cbrt(m.Z) * kQE * kQE));
    const double e2 = kQE * kQE;
    s.Kb = e2 * e2 * e2 / (12.0 * kPi * kPi * kPi * kEps0 * kEps0 * kEps0 * kME * kC * kC * kC * kHbar) *
           m.n_i_m3 * m.Z * m.Z * Lrad;
    s.Ki = m.Z * m.n_i_m3 * e2 * e2 / (4.0 * kPi * kEps0 * kEps0 * kME * kC * kC);
    s.St = 3.0 * m.kappa_tnsa * a0 * kMC2 / (m.Lx_m + m.Ly_m + m.Lz_m);
    s.r = 0.5 * m.r_fwhm_m;
    s.tc = tan(m.theta_c_rad);
    s.Fc = e2 * m.eta_avg_ohm_m * m.I0_Wm2 * m.mean_fg * s.r * s.r * m.eta_l2e / T;
    s.I_ex = m.I_ex_J;
    s.th = m.eps_th_J;
    s.mech = m.mechanisms;
    o.N_e = m.I0_Wm2 * m.mean_fg * (kPi * m.r_fwhm_m * m.r_fwhm_m / 4.0) *
            (m.t_fwhm_s * sqrt(log(10.0) / log(2.0))) * m.eta_l2e / T;
    o.a0 = a0;
    for (int q = 0; q < 8; ++q) o.E[q] = 0.0;
    o.steps = 0;
    const double esc = m.kappa_esc * a0 * kMC2;
    const double lo[3] = {0.0, s.th, esc};
    const double hi[3] = {fmin(s.th, esc), esc, INFINITY};
    for (int b = 0; b < 3; ++b) {
      o.N_band[b] = o.eps_band[b] = o.x_end[b] = 0.0;
      if (!(hi[b] > lo[b])) continue;
      const bool open = isinf(hi[b]);
      const double ea = exp(-lo[b] / T), eb = open ? 0.0 : exp(-hi[b] / T);
      const double nb = o.N_e * (ea - eb);
      const double Eb = o.N_e * ((lo[b] + T) * ea - (open ? 0.0 : (hi[b] + T) * eb));
      if (!(nb > 0.0)) continue;
      double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      const double eps = Eb / nb;
      o.N_band[b] = nb;
      o.eps_band[b] = eps;
      long long steps = 0;
      o.x_end[b] = run_macro(s, m, eps, b == 2, acc, steps);
      o.steps += steps;
      o.E[HPIC_MODEL_E_INJ] += Eb;
      for (int q = 0; q < 6; ++q) o.E[1 + q] += nb * acc[q];
    }
    out[p] = o;
  }
}

}  // namespace
}  // namespace hpic

extern "C" {

int hpic_model_device(int64_t n, const hpic_model_in *in, hpic_model_out *out, int device,
                      void *cuda_stream) {
  if (n < 0 || (n > 0 && (!in || !out))) return HPIC_EINVAL;
  if (n == 0) return HPIC_OK;
  if (cudaSetDevice(device) != cudaSuccess) return HPIC_ECUDA;
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const long long want = (n + 127) / 128, cap = (long long)sms * 16;
  hpic::k_model<<<(int)(want < cap ? want : cap), 128, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      n, in, out);
  return cudaGetLastError() == cudaSuccess ? HPIC_OK : HPIC_ECUDA;
}

int hpic_model(int64_t n, const hpic_model_in *in, hpic_model_out *out, int device,
               void *cuda_stream) {
  if (n < 0 || (n > 0 && (!in || !out))) {
    hpic::set_global_error("hpic_model: bad arguments");
    return HPIC_EINVAL;
  }
  for (int64_t p = 0; p < n; ++p) {
    const hpic_model_in &m = in[p];
    if (!(m.rel_step >= 1e-6 && m.rel_step < 1) || !(m.Z > 0) || !(m.n_i_m3 > 0) || !(m.I_ex_J > 0) ||
        !(m.Lx_m > 0) || !(m.Ly_m > 0) || !(m.Lz_m > 0) || !(m.I0_Wm2 > 0) || !(m.lambda_m > 0) ||
        !(m.eta_l2e > 0) || !(m.r_fwhm_m > 0) || !(m.t_fwhm_s > 0) || !(m.mean_fg > 0) ||
        !(m.mean_sqrt_fg > 0) || !(m.kappa_esc >= 0) || !(m.kappa_tnsa >= 0) ||
        !(m.theta_c_rad > 0 && m.theta_c_rad < 1.5707963267948966) || !(m.eta_avg_ohm_m >= 0) ||
        !(m.eps_th_J > 0) || !(m.E_stop_J > 0) || (m.mechanisms & ~HPIC_MODEL_ALL) != 0 ||
        (m.mechanisms & (HPIC_MODEL_BREM | HPIC_MODEL_ION | HPIC_MODEL_TNSA)) == 0) {
      hpic::set_global_error(("hpic_model: parameter set " + std::to_string(p) + " out of range").c_str());
      return HPIC_EINVAL;
    }
  }
  if (n == 0) return HPIC_OK;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    hpic::set_global_error("hpic_model: no such CUDA device");
    return HPIC_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  hpic_model_in *din = nullptr;
  hpic_model_out *dout = nullptr;
  if (cudaMalloc(&din, n * sizeof(*din)) != cudaSuccess ||
      cudaMalloc(&dout, n * sizeof(*dout)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(din);
    hpic::set_global_error("hpic_model: device allocation failed");
    return HPIC_ENOMEM;
  }
  int rc = HPIC_OK;
  cudaError_t e = cudaMemcpyAsync(din, in, n * sizeof(*din), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) rc = hpic_model_device(n, din, dout, device, cuda_stream);
  if (e == cudaSuccess && rc == HPIC_OK)
    e = cudaMemcpyAsync(out, dout, n * sizeof(*dout), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(din);
  cudaFree(dout);
  if (e != cudaSuccess || rc != HPIC_OK) {
    hpic::set_global_error(("hpic_model: " + std::string(cudaGetErrorString(e))).c_str());
    return HPIC_ECUDA;
  }
  return HPIC_OK;
}

}  // extern "C"
