// Batched particle kernels: many independent targets advanced by one launch
// per kernel kind (the paper's parameter scans, Sec. III, as one job).
//
// Every target owns a fixed range of slots in one shared structure of
// arrays.  Per step a one-block plan turns the targets' live counts into a
// prefix of warp-sized tasks (32 consecutive slots of one target); the
// persistent push kernel's warps take tasks in a global sweep (task w,
// w + all warps, ...), so at any moment the whole GPU works on a narrow
// window of slots and each target's grid stays hot in L2 while it is swept.
// A warp meets each target once per sweep: it then copies the target's
// constants into shared memory and, when it moves on, adds its tally sums to
// a per-block shared array indexed by target, flushed to the targets'
// device tallies once at the end.  The per-electron physics is the same
// device code as the single-target kernel (push.cuh).
#include "push.cuh"

namespace hpic {

// Threads per block of the persistent push, by precision and blocks per SM
// (MINB): FP32 runs 512 at two blocks per SM (64 registers) and 384 at three
// (56 registers), 256 otherwise; FP64 runs 256.  A block's warps take
// consecutive tasks, so larger blocks share more of their gathers' L1 lines
// (the single-target kernel measured three blocks of 384 3.4 % faster than
// five of 256 at 48 registers).
// One definition serves the kernels' launch bounds, the launches and the
// dynamic shared memory sized for them (an FP32 request of one block per SM
// runs the two-block code, as launch_batch_push_ns does).
__host__ __device__ constexpr int batch_threads_for(bool fp32, int blocks_per_sm) {
  return !fp32 ? 256 : (blocks_per_sm <= 2 ? 512 : (blocks_per_sm == 3 ? 384 : 256));
}
template <typename R, int MINB>
__host__ __device__ constexpr int batch_threads() { return batch_threads_for(sizeof(R) == 4, MINB); }
constexpr int kBatchMaxWarps = 16;
static_assert(batch_threads_for(true, 2) / 32 <= kBatchMaxWarps &&
                  batch_threads_for(true, 3) / 32 <= kBatchMaxWarps &&
                  batch_threads_for(false, 2) / 32 <= kBatchMaxWarps,
              "the largest block's stages are what the shared-memory limit is set for");
static_assert(batch_threads_for(true, 1) == batch_threads_for(true, 2),
              "one block per SM in FP32 runs the two-block kernel");

// ---------------------------------------------------------------- plan
// wpref: warp tasks from the live slot counts; ipref: electrons injected in
// this step (Eq. (B1), flat-top: floor((s+1)N/S) - floor(sN/S) at step s < S)
template <typename R>
__global__ void __launch_bounds__(256) k_batch_plan(const BatchItem<R> *items, BatchDev d) {
  __shared__ long long wt[HPIC_BATCH_MAX_TARGETS], ct[HPIC_BATCH_MAX_TARGETS];
  for (int t = threadIdx.x; t < d.n; t += blockDim.x) {
    const BatchItem<R> &it = items[t];
    const long long n = it.cnt->n, st = it.cnt->step;
    wt[t] = (n + 31) / 32;
    const long long S = it.K.n_inj_steps, N = it.K.n_macro;
    ct[t] = (N > 0 && st < S) ? (N * (st + 1)) / S - (N * st) / S : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long a = 0, b = 0;
    for (int t = 0; t < d.n; ++t) {
      d.wpref[t] = a;
      d.ipref[t] = b;
      a += wt[t];
      b += ct[t];
    }
    d.wpref[d.n] = a;
    d.ipref[d.n] = b;
  }
}

// ---------------------------------------------------------------- push
template <typename R>
__device__ __forceinline__ void flush_acc(const Acc<R> &acc, double *dst) {
  double v[kAccN];
  acc.values(v);
#pragma unroll
  for (int q = 0; q < kAccN; ++q) {
    if (!__any_sync(0xffffffffu, v[q] != 0.0)) continue;  // rare events: mostly none
    const double s = warp_sum(v[q]);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(dst + q, s);
  }
}

// What a warp keeps of its current target: the per-target hot constants
// and the grid and tally views (the run-wide constants are the kernel's
// parameter Krun, read from the constant bank like the single-target
// kernel's).
template <typename R>
struct TargetHot {
  HotK<R> h;
  Grid<R> grid;  // read in place by the push (not held in registers)
  TallyView tv;
  long long off;  // first particle slot of the target
  long long step, n;  // the target's step and slot count
  long long sshift;   // a sorting step: the target's first slot minus its first sorted offset
};

// SORT: the step also sorts (so says where the electrons go; without it the
// sorting code is compiled out).  MINB = the blocks per SM the launch asks
// for, with batch_threads threads each: the register budget follows (FP32
// 5: 48 registers, 4: 64, 3: 56 at 384 threads, 2: 64 at 512; FP64 2: 128,
// 1: 255; the FP32 state spills a little below 64), and the autotuner picks
// among the variants by timing them
template <typename R, int MINB, int NS, bool SORT>
__global__ void __launch_bounds__(batch_threads<R, MINB>(), MINB)
k_batch_push(const Consts Krun, const BatchItem<R> *__restrict__ items, BatchDev d, PView<R> p,
             const R *__restrict__ tab, const SortOut<R> so) {
  constexpr int kBatchWarps = batch_threads<R, MINB>() / 32;
  __shared__ TargetHot<R> wc[kBatchWarps];  // each warp's current target
  // the warps' deposit stages, then n x kAccN tally sums, then the task prefix
  extern __shared__ __align__(16) double dyn[];
  R *stage = reinterpret_cast<R *>(dyn) + (threadIdx.x >> 5) * dep_words<R>();
  double *tal_s = dyn + kBatchWarps * dep_words<R>() * sizeof(R) / sizeof(double);
  long long *wpref_s = reinterpret_cast<long long *>(tal_s + d.n * kAccN);
  for (int i = threadIdx.x; i < d.n * kAccN; i += blockDim.x) tal_s[i] = 0.0;
  for (int t = threadIdx.x; t <= d.n; t += blockDim.x) wpref_s[t] = d.wpref[t];
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long ntask = wpref_s[d.n];
  const long long nwarps = (long long)gridDim.x * kBatchWarps;
  TargetHot<R> &it = wc[warp];
  int t = -1;
  Acc<R> acc;
  for (long long w = blockIdx.x * (long long)kBatchWarps + warp; w < ntask; w += nwarps) {
    int tn = t < 0 ? 0 : t;
    while (wpref_s[tn + 1] <= w) ++tn;
    if (tn != t) {  // warp-uniform: a new target
      if (t >= 0) {
        flush_acc(acc, tal_s + t * kAccN);
        acc = Acc<R>();
      }
      t = tn;
      __syncwarp();
      const BatchItem<R> *src = items + t;
      auto copy = [&](void *dst, const void *from, int bytes) {
        const uint32_t *a = static_cast<const uint32_t *>(from);
        uint32_t *b = static_cast<uint32_t *>(dst);
        for (int k = lane; k < bytes / 4; k += 32) b[k] = __ldg(a + k);
      };
      copy(&it.h, &src->h, (int)sizeof(HotK<R>));
      copy(&it.tv, &src->tv, (int)sizeof(TallyView));
      if (lane == 0) {
        it.grid = make_grid(src->h, src->g);
        it.off = src->off;
        if constexpr (SORT) it.sshift = src->off - d.sstart[t];
        it.step = src->cnt->step;
        it.n = src->cnt->n;
      }
      __syncwarp();
    }
    // rebuilt per task from shared memory rather than held in registers
    StepCtx sc;
    sc.step_ll = it.step;
    sc.step = (uint32_t)sc.step_ll;
    sc.key0 = Krun.key0;
    sc.key1 = Krun.key1;
    sc.target = it.h.target_index;
    const long long local = (w - wpref_s[t]) * 32 + lane;
    push_warp<R, NS, SORT ? kPushSort : kPushPlain>(
        Krun, it.h, it.grid, tab, it.tv, sc, p, it.off + local, local < it.n, acc,
        tal_s + t * kAccN, stage, SORT ? &so : nullptr, SORT ? &it.sshift : nullptr, nullptr);
  }
  if (t >= 0) flush_acc(acc, tal_s + t * kAccN);
  __syncthreads();
  for (int i = threadIdx.x; i < d.n * kAccN; i += blockDim.x)
    if (tal_s[i] != 0.0) atomicAdd(items[i / kAccN].tv.tal + kAccSlot[i % kAccN], tal_s[i]);
}

// ---------------------------------------------------------------- injection
__device__ __forceinline__ int forward_target(const long long *pref, int t, int n, long long q) {
  while (t + 1 < n && pref[t + 1] <= q) ++t;
  return t;
}

template <typename R>
__global__ void __launch_bounds__(256)
k_batch_inject(const BatchItem<R> *__restrict__ items, BatchDev d, PView<R> p) {
  extern __shared__ long long ipref_s[];  // n + 1 prefix, then 3 sums per target
  double *sum_s = reinterpret_cast<double *>(ipref_s + d.n + 1);
  for (int t = threadIdx.x; t <= d.n; t += blockDim.x) ipref_s[t] = d.ipref[t];
  for (int t = threadIdx.x; t < 3 * d.n; t += blockDim.x) sum_s[t] = 0.0;
  __syncthreads();
  const long long C = ipref_s[d.n];
  int t = 0;
  double e_inj = 0.0, n_inj = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < C;
       i += (long long)gridDim.x * blockDim.x) {
    const int tn = forward_target(ipref_s, t, d.n, i);
    if (tn != t) {
      if (n_inj > 0.0) {
        atomicAdd(sum_s + 3 * t, e_inj);
        atomicAdd(sum_s + 3 * t + 1, n_inj * items[t].K.w);
        atomicAdd(sum_s + 3 * t + 2, n_inj);
      }
      e_inj = n_inj = 0.0;
      t = tn;
    }
    const BatchItem<R> &it = items[t];
    const long long local = i - ipref_s[t];
    const long long q = it.cnt->n + local;
    if (q >= it.cap) {
      atomicOr(&it.cnt->flags, 1u);
      continue;
    }
    const uint32_t id = (uint32_t)(it.cnt->next_id + local);
    const R eps = inject_one(it.K, p, it.off + q, id, (uint32_t)it.cnt->step);
    e_inj += it.K.w * (double)eps;
    n_inj += 1.0;
  }
  if (n_inj > 0.0) {
    atomicAdd(sum_s + 3 * t, e_inj);
    atomicAdd(sum_s + 3 * t + 1, n_inj * items[t].K.w);
    atomicAdd(sum_s + 3 * t + 2, n_inj);
  }
  __syncthreads();
  const int slot[3] = {T_E_INJ, T_N_INJ, T_N_INJECTED};
  for (int u = threadIdx.x; u < 3 * d.n; u += blockDim.x)
    if (sum_s[u] != 0.0) atomicAdd(items[u / 3].tv.tal + slot[u % 3], sum_s[u]);
}

// closes a step of every target: append the injected electrons, advance the clock
template <typename R>
__global__ void k_batch_advance(const BatchItem<R> *items, BatchDev d) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d.n; t += gridDim.x * blockDim.x) {
    Counters *cnt = items[t].cnt;
    const long long c = d.ipref[t + 1] - d.ipref[t];
    const long long n = cnt->n + c, cap = items[t].cap;
    cnt->n = n < cap ? n : cap;
    cnt->next_id += c;
    cnt->step += 1;
    cnt->inj_cnt = 0;
  }
}

// ---------------------------------------------------------------- sort
// Counting sort of every target's slots by (target, 4x4x4 cell tile) over
// the concatenated key ranges (prefix d.kpref; the last key of each target's
// range is its dead bin).  Each target's electrons land in its own slots.
template <typename R>
__global__ void __launch_bounds__(256)
k_batch_sort_keys(const BatchItem<R> *__restrict__ items, BatchDev d, PView<R> p,
                  uint32_t *keys, uint32_t *ranks, uint32_t *counts, R lead) {
  const long long nslot = d.wpref[d.n] * 32;
  int t = 0;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nslot;
       s += (long long)gridDim.x * blockDim.x) {
    t = forward_target(d.wpref, t, d.n, s >> 5);  // uniform over the warp
    const BatchItem<R> &it = items[t];
    const long long local = s - d.wpref[t] * 32;
    if (local >= it.cnt->n) continue;
    const long long ip = it.off + local;
    uint32_t key = (uint32_t)(d.kpref[t] + it.K.nkeys);
    if (p.id[ip] != kDead) {
      R X = p.x[ip], Y = p.y[ip], Z = p.z[ip];
      if (lead != R(0)) {  // the cell reached `lead` steps ahead (cdt: cells per step at c)
        const R ux = p.ux[ip], uy = p.uy[ip], uz = p.uz[ip];
        const R a = lead * it.h.cdt / m_sqrt(R(1) + ux * ux + uy * uy + uz * uz);
        X += a * ux;
        Y += a * uy;
        Z += a * uz;
      }
      int i = (int)m_floor(X), j = (int)m_floor(Y), k = (int)m_floor(Z);
      i = min(max(i, 0), it.K.nx - 1);
      j = min(max(j, 0), it.K.ny - 1);
      k = min(max(k, 0), it.K.nz - 1);
      key = (uint32_t)d.kpref[t] + tile_key(i, j, k, it.K.nti, it.K.ntj);
    }
    keys[ip] = key;
    ranks[ip] = agg_inc(counts, key);
  }
}

// after the scan: each target's first offset and the slots it keeps (the
// exclusive offset of its dead bin minus its first offset)
template <typename R>
__global__ void k_batch_sort_starts(const BatchItem<R> *items, BatchDev d, const uint32_t *offs) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d.n; t += gridDim.x * blockDim.x) {
    const long long k0 = d.kpref[t];
    d.sstart[t] = offs[k0];
    d.snew[t] = (long long)offs[k0 + items[t].K.nkeys] - (long long)offs[k0];
  }
}

template <typename R>
__global__ void k_batch_sort_finish(const BatchItem<R> *items, BatchDev d) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d.n; t += gridDim.x * blockDim.x)
    items[t].cnt->n = d.snew[t];
}

// ---------------------------------------------------------------- launchers
template <typename R>
void launch_batch_plan(const BatchItem<R> *items, BatchDev d, cudaStream_t st) {
  k_batch_plan<R><<<1, 256, 0, st>>>(items, d);
}

template <typename R>
constexpr size_t batch_stage_bytes(int warps) { return (size_t)warps * dep_words<R>() * sizeof(R); }

// dynamic shared memory of the push for up to the maximum number of targets
// at the largest block
template <typename R>
constexpr size_t batch_push_smem_max() {
  return batch_stage_bytes<R>(kBatchMaxWarps) +
         (size_t)HPIC_BATCH_MAX_TARGETS * kAccN * sizeof(double) +
         (HPIC_BATCH_MAX_TARGETS + 1) * sizeof(long long);
}

cudaError_t prepare_batch_push() {
  const int f = (int)batch_push_smem_max<float>(), d = (int)batch_push_smem_max<double>();
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *fn, int bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, a, bytes);
  };
  set((const void *)k_batch_push<float, 2, 1, false>, f);
  set((const void *)k_batch_push<float, 2, 1, true>, f);
  set((const void *)k_batch_push<float, 3, 1, false>, f);
  set((const void *)k_batch_push<float, 3, 1, true>, f);
  set((const void *)k_batch_push<float, 4, 1, false>, f);
  set((const void *)k_batch_push<float, 4, 1, true>, f);
  set((const void *)k_batch_push<float, 5, 1, false>, f);
  set((const void *)k_batch_push<float, 5, 1, true>, f);
  set((const void *)k_batch_push<float, 2, 4, false>, f);
  set((const void *)k_batch_push<float, 2, 4, true>, f);
  set((const void *)k_batch_push<float, 3, 4, false>, f);
  set((const void *)k_batch_push<float, 3, 4, true>, f);
  set((const void *)k_batch_push<float, 4, 4, false>, f);
  set((const void *)k_batch_push<float, 4, 4, true>, f);
  set((const void *)k_batch_push<float, 5, 4, false>, f);
  set((const void *)k_batch_push<float, 5, 4, true>, f);
  set((const void *)k_batch_push<double, 1, 1, false>, d);
  set((const void *)k_batch_push<double, 1, 1, true>, d);
  set((const void *)k_batch_push<double, 2, 1, false>, d);
  set((const void *)k_batch_push<double, 2, 1, true>, d);
  set((const void *)k_batch_push<double, 1, 4, false>, d);
  set((const void *)k_batch_push<double, 1, 4, true>, d);
  set((const void *)k_batch_push<double, 2, 4, false>, d);
  set((const void *)k_batch_push<double, 2, 4, true>, d);
  return e;
}

template <typename R, int NS, bool SORT>
void launch_batch_push_ns(const Consts &Krun, const BatchItem<R> *items, BatchDev d, PView<R> p,
                          const R *table, int grid, int blocks_per_sm, size_t sm, cudaStream_t st,
                          const SortOut<R> &so) {
  if constexpr (sizeof(R) == 8) {  // FP64: one or two blocks per SM
    if (blocks_per_sm <= 1)
      k_batch_push<R, 1, NS, SORT><<<grid, batch_threads<R, 1>(), sm, st>>>(Krun, items, d, p,
                                                                            table, so);
    else
      k_batch_push<R, 2, NS, SORT><<<grid, batch_threads<R, 2>(), sm, st>>>(Krun, items, d, p,
                                                                            table, so);
  } else {  // FP32: two to five (one runs the two-block code)
    if (blocks_per_sm <= 2)
      k_batch_push<R, 2, NS, SORT><<<grid, batch_threads<R, 2>(), sm, st>>>(Krun, items, d, p,
                                                                            table, so);
    else if (blocks_per_sm == 3)
      k_batch_push<R, 3, NS, SORT><<<grid, batch_threads<R, 3>(), sm, st>>>(Krun, items, d, p,
                                                                            table, so);
    else if (blocks_per_sm == 4)
      k_batch_push<R, 4, NS, SORT><<<grid, batch_threads<R, 4>(), sm, st>>>(Krun, items, d, p,
                                                                            table, so);
    else
      k_batch_push<R, 5, NS, SORT><<<grid, batch_threads<R, 5>(), sm, st>>>(Krun, items, d, p,
                                                                            table, so);
  }
}

// single: every target is a single-element solid (the element loops vanish)
template <typename R>
void launch_batch_push(const Consts &Krun, const BatchItem<R> *items, BatchDev d, PView<R> p,
                       const R *table, int sm_count, int blocks_per_sm, bool single,
                       cudaStream_t st, const SortOut<R> &so) {
  const int warps = batch_threads_for(sizeof(R) == 4, blocks_per_sm) / 32;
  const size_t sm = batch_stage_bytes<R>(warps) + (size_t)d.n * kAccN * sizeof(double) +
                    (d.n + 1) * sizeof(long long);
  const int grid = sm_count * blocks_per_sm;
  const bool sort = so.dst.x != nullptr;
  if (single && sort)
    launch_batch_push_ns<R, 1, true>(Krun, items, d, p, table, grid, blocks_per_sm, sm, st, so);
  else if (single)
    launch_batch_push_ns<R, 1, false>(Krun, items, d, p, table, grid, blocks_per_sm, sm, st, so);
  else if (sort)
    launch_batch_push_ns<R, 4, true>(Krun, items, d, p, table, grid, blocks_per_sm, sm, st, so);
  else
    launch_batch_push_ns<R, 4, false>(Krun, items, d, p, table, grid, blocks_per_sm, sm, st, so);
}

template <typename R>
void launch_batch_inject(const BatchItem<R> *items, BatchDev d, PView<R> p, int grid,
                         cudaStream_t st) {
  const size_t sm = (d.n + 1) * sizeof(long long) + 3 * d.n * sizeof(double);
  k_batch_inject<R><<<grid, 256, sm, st>>>(items, d, p);
}

template <typename R>
void launch_batch_advance(const BatchItem<R> *items, BatchDev d, cudaStream_t st) {
  k_batch_advance<R><<<1, 256, 0, st>>>(items, d);
}

template <typename R>
int launch_batch_sort_keys(const BatchItem<R> *items, BatchDev d, PView<R> p, uint32_t *keys,
                           uint32_t *ranks, uint32_t *counts, uint32_t *partials,
                           long long nkeys_total, int grid, cudaStream_t st, double lead) {
  cudaMemsetAsync(counts, 0, nkeys_total * sizeof(uint32_t), st);
  k_batch_sort_keys<R><<<grid, 256, 0, st>>>(items, d, p, keys, ranks, counts, R(lead));
  const int launches = 1 + launch_scan(counts, nkeys_total, partials, st);
  k_batch_sort_starts<R><<<1, 256, 0, st>>>(items, d, counts);
  return launches + 1;
}

template <typename R>
int launch_batch_sort_finish(const BatchItem<R> *items, BatchDev d, cudaStream_t st) {
  k_batch_sort_finish<R><<<1, 256, 0, st>>>(items, d);
  return 1;
}

#define HPIC_INST(R)                                                                            \
  template void launch_batch_plan<R>(const BatchItem<R> *, BatchDev, cudaStream_t);             \
  template void launch_batch_push<R>(const Consts &, const BatchItem<R> *, BatchDev, PView<R>,  \
                                     const R *, int, int, bool, cudaStream_t,                   \
                                     const SortOut<R> &);                                       \
  template void launch_batch_inject<R>(const BatchItem<R> *, BatchDev, PView<R>, int,           \
                                       cudaStream_t);                                           \
  template void launch_batch_advance<R>(const BatchItem<R> *, BatchDev, cudaStream_t);          \
  template int launch_batch_sort_keys<R>(const BatchItem<R> *, BatchDev, PView<R>, uint32_t *, \
                                         uint32_t *, uint32_t *, uint32_t *, long long, int,    \
                                         cudaStream_t, double);                                 \
  template int launch_batch_sort_finish<R>(const BatchItem<R> *, BatchDev, cudaStream_t);
HPIC_INST(float)
HPIC_INST(double)
#undef HPIC_INST

}  // namespace hpic
