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
// On a step that also sorts (kPushSort) the new state goes to the electron's
// slot of the sorted order in the other buffer instead of its own slot; on
// the step before (kPushKeys) each surviving electron also gets its key and
// rank for that sort.
// Random numbers: Philox4x32-10, counter (step, id, block, target), key = seed;
// block 0 scatter, 1 emission, 2..4 reflux on x/y/z faces, 8-9 injection.
//
// Memory traffic: the electron state streams through once (evict-first
// loads and stores, so the grid stays resident in L2); the grid is read
// through the read-only path and the current is added by reductions in L2.
// Electrons are kept sorted by 4x4x4 cell tiles, so a warp's gathers and
// reductions fall on few L2 lines.
#include "push.cuh"

namespace hpic {

// MODE: a plain step, one that also keys the next sort (ko), or one that
// also sorts (so says where the electrons go); the other modes' code is
// compiled out.
template <typename R, int NS, int MODE>
// Launched as one persistent wave in the shape push_threads/push_blocks_per_sm
// give: the kernel is issue- and latency-bound and gains from the warps, up
// to the register count at which spills begin.
__global__ void __launch_bounds__(push_threads<R>(), push_blocks_per_sm<R>())
k_push(const Consts K, const HotK<R> h, PView<R> p, GView<R> gv, const R *__restrict__ tab,
       Counters *cnt, TallyView tv, const SortOut<R> so, const KeyOut<R> ko) {
  __shared__ double rare[kAccN];  // the rare tally sums of the block
  if (threadIdx.x < kAccN) rare[threadIdx.x] = 0.0;
  __syncthreads();
  extern __shared__ __align__(16) unsigned char dyn[];  // the warps' deposit stages
  R *stage = reinterpret_cast<R *>(dyn) + (threadIdx.x >> 5) * dep_words<R>();
  const long long n = cnt->n;
  StepCtx sc;
  sc.step_ll = cnt->step;
  sc.step = (uint32_t)sc.step_ll;
  sc.key0 = K.key0;
  sc.key1 = K.key1;
  sc.target = h.target_index;

  const Grid<R> g = make_grid(h, gv);
  Acc<R> acc;
  const long long no_shift = 0;  // one target: the sorted slot is offset + rank

  // warp-uniform loop: every lane reaches the warp-cooperative deposits
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x - lane); base < n;
       base += stride)
    push_warp<R, NS, MODE>(K, h, g, tab, tv, sc, p, base + lane, base + lane < n, acc, rare,
                           stage, MODE == kPushSort ? &so : nullptr,
                           MODE == kPushSort ? &no_shift : nullptr,
                           MODE == kPushKeys ? &ko : nullptr);

  double v[kAccN];
  acc.values(v);
  __syncthreads();  // every warp is past its deposits: the stages hold the block sums
  block_flush<kAccN>(v, kAccSlot, tv.tal, reinterpret_cast<double *>(dyn));  // synchronises
  if (threadIdx.x < kAccN && rare[threadIdx.x] != 0.0)
    atomicAdd(tv.tal + kAccSlot[threadIdx.x], rare[threadIdx.x]);
}

// ---------------------------------------------------------------- injection
// Eq. (B1) with flat-top envelopes: step s < S injects floor((s+1)N/S) -
// floor(sN/S) electrons (inject_one places each).
// Gaussian envelope (App. B): per_cell electrons in each injecting face cell
// while g(t) >= g_min, each of weight inj_unit sqrt(f g) and local mean
// energy a0 sqrt(f g) m_e c^2; ids run cell by cell in the cells' order.
template <typename R>
__device__ void inject_gauss(const Consts &K, PView<R> p, Counters *cnt, long long cap,
                             TallyView tv, double *smem) {
  const long long st = cnt->step;
  const double tm = (double)st + 0.5 - K.t_pk;
  const double g = exp(-K.g_c * tm * tm);
  const long long c = g >= K.g_min ? K.per_cell * K.n_inj_cells : 0;
  const long long n0 = cnt->n, id0 = cnt->next_id;
  const uint32_t step = (uint32_t)st;
  const double sg = sqrt(g);
  const InjCell *cells = static_cast<const InjCell *>(K.inj_cells);
  double e_inj = 0.0, w_inj = 0.0, n_inj = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < c;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = n0 + i;
    if (q >= cap) {
      atomicOr(&cnt->flags, 1u);
      continue;
    }
    const InjCell ic = cells[i / K.per_cell];
    const double sfg = ic.sf * sg;
    const R w = R(K.inj_unit * sfg);
    const R eps = inject_cell_one(K, p, q, (uint32_t)(id0 + i), step, ic.j, ic.k, R(K.T_hot * sfg));
    p.w[q] = w;
    e_inj += (double)w * (double)eps;
    w_inj += (double)w;
    n_inj += 1.0;
  }
  const double v[3] = {e_inj, w_inj, n_inj};
  const int slot[3] = {T_E_INJ, T_N_INJ, T_N_INJECTED};
  block_flush<3>(v, slot, tv.tal, smem);
  if (blockIdx.x == 0 && threadIdx.x == 0) cnt->inj_cnt = c;
}

template <typename R>
__global__ void __launch_bounds__(256)
k_inject(const Consts K, PView<R> p, Counters *cnt, long long cap, TallyView tv) {
  __shared__ double smem[3 * 32];
  if (K.weighted) {
    inject_gauss(K, p, cnt, cap, tv, smem);
    return;
  }
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
    const R eps = inject_one(K, p, q, (uint32_t)(id0 + i), step);
    e_inj += K.w * (double)eps;
    n_inj += 1.0;
  }
  const double v[3] = {e_inj, n_inj * K.w, n_inj};
  const int slot[3] = {T_E_INJ, T_N_INJ, T_N_INJECTED};
  block_flush<3>(v, slot, tv.tal, smem);
  if (blockIdx.x == 0 && threadIdx.x == 0) cnt->inj_cnt = c;
}

// Bulk seeding: n electrons uniform in the box, isotropic, kinetic energy
// exponential with mean `mean` (m_e c^2), fresh optical depth.  Draws: block
// 10 = (eps, cos theta, phi, x), block 11 = (y, z, tau, -) at the current step.
template <typename R>
__global__ void __launch_bounds__(256)
k_seed(const Consts K, PView<R> p, Counters *cnt, long long cap, long long count, double mean,
       TallyView tv) {
  __shared__ double smem[3 * 32];
  const long long n0 = cnt->n, id0 = cnt->next_id;
  const uint32_t step = (uint32_t)cnt->step;
  double e_inj = 0.0, n_inj = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = n0 + i;
    if (q >= cap) {
      atomicOr(&cnt->flags, 1u);
      continue;
    }
    const uint32_t id = (uint32_t)(id0 + i);
    const U4 a = philox10(step, id, 10u, K.target_index, K.key0, K.key1);
    const U4 b = philox10(step, id, 11u, K.target_index, K.key0, K.key1);
    const R eps = -R(mean) * m_log(R(1) - unif<R>(a.a));
    const R ct = R(2) * unif<R>(a.b) - R(1);
    const R st = m_sqrt((R(1) - ct) * (R(1) + ct));
    R sp, cp;
    m_sincos2pi(unif<R>(a.c), &sp, &cp);
    const R un = u_of_eps(eps);
    p.x[q] = R(K.nx) * unif<R>(a.d);
    p.y[q] = R(K.ny) * unif<R>(b.a);
    p.z[q] = R(K.nz) * unif<R>(b.b);
    p.ux[q] = un * ct;
    p.uy[q] = un * st * cp;
    p.uz[q] = un * st * sp;
    p.tau[q] = -m_log(R(1) - unif<R>(b.c));
    if (K.weighted) p.w[q] = R(K.w);
    p.id[q] = id;
    e_inj += K.w * (double)eps;
    n_inj += 1.0;
  }
  const double v[3] = {e_inj, n_inj * K.w, n_inj};
  const int slot[3] = {T_E_INJ, T_N_INJ, T_N_INJECTED};
  block_flush<3>(v, slot, tv.tal, smem);
}

__global__ void k_seed_done(Counters *cnt, long long count, long long cap) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const long long n = cnt->n + count;
    cnt->n = n < cap ? n : cap;
    cnt->next_id += count;
  }
}

template <typename R>
void launch_seed(const Consts &K, PView<R> p, Counters *cnt, long long cap, long long count,
                 double mean, TallyView tv, int grid, cudaStream_t st) {
  k_seed<R><<<grid, 256, 0, st>>>(K, p, cnt, cap, count, mean, tv);
  k_seed_done<<<1, 32, 0, st>>>(cnt, count, cap);
}
template void launch_seed<float>(const Consts &, PView<float>, Counters *, long long, long long,
                                 double, TallyView, int, cudaStream_t);
template void launch_seed<double>(const Consts &, PView<double>, Counters *, long long,
                                  long long, double, TallyView, int, cudaStream_t);

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
constexpr size_t push_stage_bytes() { return (push_threads<R>() / 32) * dep_words<R>() * sizeof(R); }

cudaError_t prepare_push() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *fn, size_t bytes) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  set((const void *)k_push<float, 1, kPushPlain>, push_stage_bytes<float>());
  set((const void *)k_push<float, 1, kPushKeys>, push_stage_bytes<float>());
  set((const void *)k_push<float, 1, kPushSort>, push_stage_bytes<float>());
  set((const void *)k_push<float, 4, kPushPlain>, push_stage_bytes<float>());
  set((const void *)k_push<float, 4, kPushKeys>, push_stage_bytes<float>());
  set((const void *)k_push<float, 4, kPushSort>, push_stage_bytes<float>());
  set((const void *)k_push<double, 1, kPushPlain>, push_stage_bytes<double>());
  set((const void *)k_push<double, 1, kPushKeys>, push_stage_bytes<double>());
  set((const void *)k_push<double, 1, kPushSort>, push_stage_bytes<double>());
  set((const void *)k_push<double, 4, kPushPlain>, push_stage_bytes<double>());
  set((const void *)k_push<double, 4, kPushKeys>, push_stage_bytes<double>());
  set((const void *)k_push<double, 4, kPushSort>, push_stage_bytes<double>());
  return e;
}

template <typename R, int NS>
void launch_push_ns(const Consts &K, const HotK<R> &h, PView<R> p, GView<R> g, const R *table,
                    Counters *cnt, TallyView tv, int grid, cudaStream_t st, const SortOut<R> &so,
                    const KeyOut<R> &ko) {
  const size_t sm = push_stage_bytes<R>();
  if (so.dst.x)
    k_push<R, NS, kPushSort><<<grid, push_threads<R>(), sm, st>>>(K, h, p, g, table, cnt, tv, so, ko);
  else if (ko.keys)
    k_push<R, NS, kPushKeys><<<grid, push_threads<R>(), sm, st>>>(K, h, p, g, table, cnt, tv, so, ko);
  else
    k_push<R, NS, kPushPlain><<<grid, push_threads<R>(), sm, st>>>(K, h, p, g, table, cnt, tv, so, ko);
}

template <typename R>
void launch_push(const Consts &K, PView<R> p, GView<R> g, const R *table, Counters *cnt,
                 TallyView tv, int grid, cudaStream_t st, const SortOut<R> &so,
                 const KeyOut<R> &ko) {
  const HotK<R> h = make_hot<R>(K);
  if (K.n_solids == 1)  // a single-element solid: the element loops vanish
    launch_push_ns<R, 1>(K, h, p, g, table, cnt, tv, grid, st, so, ko);
  else
    launch_push_ns<R, 4>(K, h, p, g, table, cnt, tv, grid, st, so, ko);
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
                                 Counters *, TallyView, int, cudaStream_t, const SortOut<float> &,
                                 const KeyOut<float> &);
template void launch_push<double>(const Consts &, PView<double>, GView<double>, const double *,
                                  Counters *, TallyView, int, cudaStream_t,
                                  const SortOut<double> &, const KeyOut<double> &);
template void launch_inject<float>(const Consts &, PView<float>, Counters *, long long, TallyView,
                                   int, cudaStream_t);
template void launch_inject<double>(const Consts &, PView<double>, Counters *, long long,
                                    TallyView, int, cudaStream_t);

}  // namespace hpic
