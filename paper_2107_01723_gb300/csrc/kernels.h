// Internal declarations shared by the kernel translation units and api.cu.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace hpic {

// particle storage: structure of arrays, positions in cells, momenta u = p/(m_e c)
template <typename R>
struct PView {
  R *x, *y, *z, *ux, *uy, *uz, *tau;
  uint32_t *id;
};

// grid storage: vector components as (nx+1)(ny+1)(nz+1) arrays (x fastest)
template <typename R>
struct GView {
  R *E[3], *B[3], *J[3];
  double *T, *eta, *H;  // cell-centred, double
};

struct TallyView {
  double *tal;      // T_COUNT scalars
  double *hist;     // 2 x (n_E+2) x n_th: energy-weighted, then number-weighted
  double *history;  // max_history
};

// the per-electron constants in the kernel's own precision (folded on the
// host so that no double->float conversion runs per electron)
template <typename R>
struct HotK {
  R w, cdt, E_cut, K_ion, L_I, K_sc, K_lg, K_tau, k_min, inv_boost;
  R eps_esc, du_reflux, sigma_dtheta, tE_min, tE_max, inv_dlogE, th_scale, t_inv_dlog;
};

// message returned by hpic_last_error(NULL) (entry points without a context)
void set_global_error(const char *msg);

template <typename R>
void launch_push(const Consts &K, PView<R> p, GView<R> g, const R *table, Counters *cnt,
                 TallyView tv, int grid, cudaStream_t st);
template <typename R>
void launch_inject(const Consts &K, PView<R> p, Counters *cnt, long long cap, TallyView tv,
                   int grid, cudaStream_t st);
void launch_advance(Counters *cnt, long long cap, cudaStream_t st);
// bulk seeding (two launches); mean kinetic energy in m_e c^2
template <typename R>
void launch_seed(const Consts &K, PView<R> p, Counters *cnt, long long cap, long long count,
                 double mean, TallyView tv, int grid, cudaStream_t st);

template <typename R>
void launch_efield(const Consts &K, GView<R> g, int grid, cudaStream_t st);
template <typename R>
void launch_bheat(const Consts &K, GView<R> g, TallyView tv, int grid, cudaStream_t st);

// counting sort by cell: keys/counts/offsets are scratch; returns launches made
template <typename R>
int launch_sort(const Consts &K, PView<R> src, PView<R> dst, Counters *cnt, uint32_t *keys,
                uint32_t *counts, uint32_t *partials, int grid, cudaStream_t st);

void launch_table(const Consts &K, double k_min, double E_max, double *t64, float *t32,
                  cudaStream_t st);

template <typename R>
void launch_live_energy(const Consts &K, PView<R> p, Counters *cnt, double *dst, int grid,
                        cudaStream_t st);
template <typename R>
void launch_field_energy(const Consts &K, GView<R> g, double *dst, int grid, cudaStream_t st);

}  // namespace hpic
