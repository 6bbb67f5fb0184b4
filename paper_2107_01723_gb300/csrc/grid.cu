// Grid-side kernels of the hybrid-PIC step (arXiv 2107.01723):
//   k_efield : E = eta (curl B / mu0 - j_h) on edges, Eq. (A2), tangential E
//              zero on the walls (conducting boundary)
//   k_bheat  : B -= dt curl E on faces, Eq. (A3), fused with the background
//              heating dT = rho/(Z n_i C k_B), Eqs. (A7)-(A8), rho = Ohmic
//              eta j_h.j_h dt + ionisation heat, and eta(T), Eqs. (A4)-(A6)
//   sort     : counting sort of electrons by cell (GPU data layout)
//   k_table  : inverse-CDF bremsstrahlung table from the closed-form CDF
#include "fields.cuh"

#include <type_traits>

namespace hpic {

template <typename R>
__global__ void __launch_bounds__(256, kFieldBlocksPerSm) k_efield(const Consts K, GView<R> g) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < K.nvec;
       q += (long long)gridDim.x * blockDim.x)
    efield_node(K, g, q);
}

template <typename R>
__global__ void __launch_bounds__(256, kFieldBlocksPerSm) k_bheat(const Consts K, GView<R> g, TallyView tv) {
  __shared__ double smem[32];
  double e_ohm = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < K.nvec;
       q += (long long)gridDim.x * blockDim.x)
    e_ohm += bheat_node(K, g, q);
  const double v[1] = {e_ohm};
  const int slot[1] = {T_E_OHMIC};
  block_flush<1>(v, slot, tv.tal, smem);
}

// ---------------------------------------------------------------- batched field kernels
// The targets' node ranges are concatenated (prefix d.npref); a thread walks
// its grid-stride nodes in increasing order, so its target index only moves
// forward.  Shared memory holds the prefix and the per-target Ohmic sums.
__device__ __forceinline__ int advance_target(const long long *pref, int t, int n, long long q) {
  while (t + 1 < n && pref[t + 1] <= q) ++t;
  return t;
}

template <typename R>
__global__ void __launch_bounds__(256, kBatchFieldBlocksPerSm)
k_batch_efield(const BatchItem<R> *items, BatchDev d) {
  extern __shared__ long long npref_s[];
  for (int t = threadIdx.x; t <= d.n; t += blockDim.x) npref_s[t] = d.npref[t];
  __syncthreads();
  const long long N = npref_s[d.n];
  int t = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
       q += (long long)gridDim.x * blockDim.x) {
    t = advance_target(npref_s, t, d.n, q);
    efield_node(items[t].K, items[t].g, q - npref_s[t]);
  }
}

template <typename R>
__global__ void __launch_bounds__(256, kBatchFieldBlocksPerSm)
k_batch_bheat(const BatchItem<R> *items, BatchDev d) {
  extern __shared__ long long npref_s[];
  double *ohm_s = reinterpret_cast<double *>(npref_s + d.n + 1);
  for (int t = threadIdx.x; t <= d.n; t += blockDim.x) npref_s[t] = d.npref[t];
  for (int t = threadIdx.x; t < d.n; t += blockDim.x) ohm_s[t] = 0.0;
  __syncthreads();
  const long long N = npref_s[d.n];
  int t = 0;
  double e_ohm = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
       q += (long long)gridDim.x * blockDim.x) {
    const int tn = advance_target(npref_s, t, d.n, q);
    if (tn != t) {
      if (e_ohm != 0.0) atomicAdd(ohm_s + t, e_ohm);
      e_ohm = 0.0;
      t = tn;
    }
    e_ohm += bheat_node(items[t].K, items[t].g, q - npref_s[t]);
  }
  if (e_ohm != 0.0) atomicAdd(ohm_s + t, e_ohm);
  __syncthreads();
  for (int u = threadIdx.x; u < d.n; u += blockDim.x)
    if (ohm_s[u] != 0.0) atomicAdd(items[u].tv.tal + T_E_OHMIC, ohm_s[u]);
}

// ---------------------------------------------------------------- counting sort
// Key of each slot: the tile key of the cell at x + lead (u/gamma), lead in
// cells per unit of u/gamma (0: the current cell), clamped to the grid.
template <typename R>
__global__ void __launch_bounds__(256)
k_sort_keys(const Consts K, PView<R> p, const Counters *cnt, uint32_t *keys, uint32_t *counts,
            R lead, uint32_t *ranks) {
  const long long n = cnt->n;
  for (long long ip = blockIdx.x * (long long)blockDim.x + threadIdx.x; ip < n;
       ip += (long long)gridDim.x * blockDim.x) {
    uint32_t key = (uint32_t)K.nkeys;
    if (p.id[ip] != kDead) {
      R X = p.x[ip], Y = p.y[ip], Z = p.z[ip];
      if (lead != R(0)) {  // uniform over the launch
        const R ux = p.ux[ip], uy = p.uy[ip], uz = p.uz[ip];
        const R a = lead / m_sqrt(R(1) + ux * ux + uy * uy + uz * uz);
        X += a * ux;
        Y += a * uy;
        Z += a * uz;
      }
      int i = (int)m_floor(X), j = (int)m_floor(Y), k = (int)m_floor(Z);
      i = min(max(i, 0), K.nx - 1);
      j = min(max(j, 0), K.ny - 1);
      k = min(max(k, 0), K.nz - 1);
      key = tile_key(i, j, k, K.nti, K.ntj);
    }
    keys[ip] = key;
    if (ranks)  // uniform over the launch
      ranks[ip] = agg_inc(counts, key);
    else
      agg_inc(counts, key);
  }
}


// per-tile sums of counts[0, m)
__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t *counts, long long m,
                                                     uint32_t *partials) {
  __shared__ uint32_t ws[32];
  const long long base = (long long)blockIdx.x * kScanTile;
  uint32_t s = 0;
  for (int t = threadIdx.x; t < kScanTile; t += blockDim.x) {
    const long long q = base + t;
    if (q < m) s += counts[q];
  }
  s = __reduce_add_sync(0xffffffffu, s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = ws[threadIdx.x];
    v = __reduce_add_sync(0xffffffffu, v);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
}

// exclusive scan of the tile sums in one block; total to partials[ntiles]
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *partials, int ntiles) {
  __shared__ uint32_t ws[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += blockDim.x) {
    const int t = base + threadIdx.x;
    const uint32_t v = t < ntiles ? partials[t] : 0u;
    // inclusive warp scan
    uint32_t x = v;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t z = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
      }
      ws[lane] = z;
    }
    __syncthreads();
    const uint32_t incl = x + (warp > 0 ? ws[warp - 1] : 0u) + carry;
    if (t < ntiles) partials[t] = incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[ntiles] = carry;
}

// exclusive scan within each tile plus its tile offset, in place
__global__ void __launch_bounds__(1024) k_scan_apply(uint32_t *counts, long long m,
                                                     const uint32_t *partials) {
  __shared__ uint32_t ws[32];
  __shared__ uint32_t carry;
  const long long base = (long long)blockIdx.x * kScanTile;
  if (threadIdx.x == 0) carry = partials[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 0; off < kScanTile; off += blockDim.x) {
    const long long q = base + off + threadIdx.x;
    const uint32_t v = q < m ? counts[q] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t z = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
      }
      ws[lane] = z;
    }
    __syncthreads();
    const uint32_t incl = x + (warp > 0 ? ws[warp - 1] : 0u) + carry;
    if (q < m) counts[q] = incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
}

template <typename R>
__global__ void __launch_bounds__(256)
k_sort_scatter(const Consts K, PView<R> src, PView<R> dst, const Counters *cnt,
               const uint32_t *keys, uint32_t *offsets) {
  const long long n = cnt->n;
  for (long long ip = blockIdx.x * (long long)blockDim.x + threadIdx.x; ip < n;
       ip += (long long)gridDim.x * blockDim.x) {
    const uint32_t key = keys[ip];
    if (key >= (uint32_t)K.nkeys) continue;
    const uint32_t q = agg_inc(offsets, key);
    dst.x[q] = src.x[ip];
    dst.y[q] = src.y[ip];
    dst.z[q] = src.z[ip];
    dst.ux[q] = src.ux[ip];
    dst.uy[q] = src.uy[ip];
    dst.uz[q] = src.uz[ip];
    dst.tau[q] = src.tau[ip];
    if (K.weighted) dst.w[q] = src.w[ip];
    dst.id[q] = src.id[ip];
  }
}

// live count = exclusive offset of the dead bin (the scatter never touches it)
__global__ void k_sort_finish(Counters *cnt, const uint32_t *offsets, long long ncell) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cnt->n = offsets[ncell];
}

// ---------------------------------------------------------------- photon table
// Row i: eps_i = k_min (E_max/k_min)^(i/(rows-1)); column j: the photon
// energy k with CDF(k/eps_i) = j/(cols-1), where CDF is the normalised
// integral of s(u)/u, s(u) = (4/3)(1-u) + u^2, from u0 = k_min/eps to u,
// stored as the log-ratio w = ln(eps_i/k) / ln(eps_i/k_min) (the sampler
// subtracts k from eps through it without cancellation).  Solved by
// Newton's method on y = ln u (dG/dy = s(e^y)) inside a bracket.
__global__ void k_table(int rows, int cols, double k_min, double E_max, double *t64, float *t32) {
  const long long nt = (long long)rows * cols;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nt;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q / cols), j = (int)(q - (long long)i * cols);
    const double r = (double)j / (double)(cols - 1);
    // w = ln(eps/k) / ln(eps/k_min): 1 at k = k_min, 0 at k = eps
    double w;
    if (i == 0 || j == 0 || j == cols - 1) {
      w = (i == 0) ? 1.0 - r : (j == 0 ? 1.0 : 0.0);
    } else {
      const double lu0 = ((double)i / (double)(rows - 1)) * -log(E_max / k_min);  // ln u0 < 0
      const double u0 = exp(lu0);
      // G(y) = (4/3)(y - lu0 - (e^y - u0)) + (e^{2y} - u0^2)/2, target r G(0)
      const double G1 = (4.0 / 3.0) * (-lu0 - (1.0 - u0)) + 0.5 * (1.0 - u0 * u0);
      const double target = r * G1;
      double lo = lu0, hi = 0.0, y = lu0 + r * (-lu0);
      for (int it = 0; it < 100; ++it) {
        const double e = exp(y);
        const double Gy = (4.0 / 3.0) * (y - lu0 - (e - u0)) + 0.5 * (e * e - u0 * u0) - target;
        if (Gy < 0.0) lo = y; else hi = y;
        const double dG = (4.0 / 3.0) * (1.0 - e) + e * e;
        double yn = y - Gy / dG;
        if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
        if (fabs(yn - y) < 1e-16 * fabs(lu0)) { y = yn; break; }
        y = yn;
      }
      w = y / lu0;  // y = ln(k/eps)
    }
    t64[q] = w;
    t32[q] = (float)w;
  }
}

// ---------------------------------------------------------------- read-time sums
template <typename R>
__global__ void __launch_bounds__(256)
k_live_energy(const Consts K, PView<R> p, const Counters *cnt, double *dst) {
  __shared__ double smem[32];
  const long long n = cnt->n;
  double e = 0.0;
  for (long long ip = blockIdx.x * (long long)blockDim.x + threadIdx.x; ip < n;
       ip += (long long)gridDim.x * blockDim.x) {
    if (p.id[ip] == kDead) continue;
    const double ux = p.ux[ip], uy = p.uy[ip], uz = p.uz[ip];
    const double u2 = ux * ux + uy * uy + uz * uz;
    e += (K.weighted ? (double)p.w[ip] : K.w) * u2 / (1.0 + sqrt(1.0 + u2));
  }
  const double v[1] = {e};
  const int slot[1] = {0};
  block_flush<1>(v, slot, dst, smem);
}

template <typename R>
__global__ void __launch_bounds__(256) k_field_energy(const Consts K, GView<R> g, double *dst) {
  __shared__ double smem[32];
  double e = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < K.nvec;
       q += (long long)gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const double b = g.B[c][q];
      e += b * b;
    }
  }
  const double v[1] = {e};
  const int slot[1] = {0};
  block_flush<1>(v, slot, dst, smem);
}

// ---------------------------------------------------------------- launchers
template <typename R>
void launch_efield(const Consts &K, GView<R> g, int grid, cudaStream_t st) {
  k_efield<R><<<grid, 256, 0, st>>>(K, g);
}

template <typename R>
void launch_bheat(const Consts &K, GView<R> g, TallyView tv, int grid, cudaStream_t st) {
  k_bheat<R><<<grid, 256, 0, st>>>(K, g, tv);
}

int launch_scan(uint32_t *counts, long long m, uint32_t *partials, cudaStream_t st) {
  const int ntiles = (int)((m + kScanTile - 1) / kScanTile);
  k_scan_tiles<<<ntiles, 1024, 0, st>>>(counts, m, partials);
  k_scan_top<<<1, 1024, 0, st>>>(partials, ntiles);
  k_scan_apply<<<ntiles, 1024, 0, st>>>(counts, m, partials);
  return 3;
}

template <typename R>
int launch_sort(const Consts &K, PView<R> src, PView<R> dst, Counters *cnt, uint32_t *keys,
                uint32_t *counts, uint32_t *partials, int grid, cudaStream_t st, double lead) {
  const long long m = K.nkeys + 1;
  cudaMemsetAsync(counts, 0, m * sizeof(uint32_t), st);
  k_sort_keys<R><<<grid, 256, 0, st>>>(K, src, cnt, keys, counts, R(lead * K.cdt_dx), nullptr);
  launch_scan(counts, m, partials, st);
  k_sort_scatter<R><<<grid, 256, 0, st>>>(K, src, dst, cnt, keys, counts);
  k_sort_finish<<<1, 32, 0, st>>>(cnt, counts, K.nkeys);
  return 6;
}

template <typename R>
int launch_sort_keys(const Consts &K, PView<R> p, Counters *cnt, uint32_t *keys, uint32_t *ranks,
                     uint32_t *counts, uint32_t *partials, int grid, cudaStream_t st, double lead) {
  const long long m = K.nkeys + 1;
  cudaMemsetAsync(counts, 0, m * sizeof(uint32_t), st);
  k_sort_keys<R><<<grid, 256, 0, st>>>(K, p, cnt, keys, counts, R(lead * K.cdt_dx), ranks);
  return 1 + launch_scan(counts, m, partials, st);
}

int launch_sort_finish(const Consts &K, Counters *cnt, const uint32_t *offsets, cudaStream_t st) {
  k_sort_finish<<<1, 32, 0, st>>>(cnt, offsets, K.nkeys);
  return 1;
}

void launch_table(const Consts &K, double k_min, double E_max, double *t64, float *t32,
                  cudaStream_t st) {
  const long long nt = (long long)K.t_rows * K.t_cols;
  const int grid = (int)((nt + 255) / 256);
  k_table<<<grid, 256, 0, st>>>(K.t_rows, K.t_cols, k_min, E_max, t64, t32);
}

template <typename R>
void launch_batch_efield(const BatchItem<R> *items, BatchDev d, int grid, cudaStream_t st) {
  k_batch_efield<R><<<grid, 256, (d.n + 1) * sizeof(long long), st>>>(items, d);
}

template <typename R>
void launch_batch_bheat(const BatchItem<R> *items, BatchDev d, int grid, cudaStream_t st) {
  const size_t sm = (d.n + 1) * sizeof(long long) + d.n * sizeof(double);
  k_batch_bheat<R><<<grid, 256, sm, st>>>(items, d);
}

template <typename R>
void launch_live_energy(const Consts &K, PView<R> p, Counters *cnt, double *dst, int grid,
                        cudaStream_t st) {
  k_live_energy<R><<<grid, 256, 0, st>>>(K, p, cnt, dst);
}

template <typename R>
void launch_field_energy(const Consts &K, GView<R> g, double *dst, int grid, cudaStream_t st) {
  k_field_energy<R><<<grid, 256, 0, st>>>(K, g, dst);
}

// ---------------------------------------------------------------- host transfers
// Reading the electrons out: the live slots in storage order, converted to
// double with a scale, compacted on the device so that one copy per array
// crosses to the host.  Slots go in chunks of kXferChunk (256 threads x 8
// consecutive slots): the live count of each chunk, an exclusive scan of the
// chunk counts, then each array written at the compacted positions.
constexpr int kXferChunk = 2048;

__global__ void __launch_bounds__(256) k_live_counts(const uint32_t *id, long long n,
                                                     uint32_t *cc) {
  __shared__ uint32_t ws[8];
  const long long base = (long long)blockIdx.x * kXferChunk + threadIdx.x * 8;
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) c += (base + k < n && id[base + k] != kDead) ? 1u : 0u;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    cc[blockIdx.x] = t;
  }
}

// exclusive scan of cc[0, nb) in one block; the total goes to cc[nb]
__global__ void __launch_bounds__(1024) k_scan_chunks(uint32_t *cc, long long nb) {
  __shared__ uint32_t part[1024];
  const long long per = (nb + 1023) / 1024;
  const long long b0 = threadIdx.x * per, b1 = b0 + per < nb ? b0 + per : nb;
  uint32_t s = 0;
  for (long long b = b0; b < b1; ++b) s += cc[b];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the slice sums
    const uint32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (long long b = b0; b < b1; ++b) {
    const uint32_t c = cc[b];
    cc[b] = run;
    run += c;
  }
  if (threadIdx.x == 1023) cc[nb] = part[1023];
}

// out[rank] = src[i] * scale (converted to O) for the live slots i of this
// block's chunk, rank = the slot's place among the live slots
template <typename T, typename O>
__global__ void __launch_bounds__(256) k_compact(const T *src, const uint32_t *id, long long n,
                                                 const uint32_t *cc, double scale, O *out) {
  __shared__ uint32_t ws[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long base = (long long)blockIdx.x * kXferChunk + threadIdx.x * 8;
  uint32_t live = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (base + k < n && id[base + k] != kDead) live |= 1u << k;
  const uint32_t c = __popc(live);
  uint32_t incl = c;  // inclusive scan over the warp, then over the warps
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += ws[w];
  long long pos = (long long)cc[blockIdx.x] + before + incl - c;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (live & (1u << k)) {
      if constexpr (std::is_floating_point<T>::value)
        out[pos++] = (O)((double)src[base + k] * scale);
      else
        out[pos++] = (O)src[base + k];
    }
}

// Loading electrons in: dst[i] = (R)(src[i] * scale); with check set, also
// count positions outside [0, hi] after division by dx (any non-finite
// value with unbounded), the test the host made before
template <typename R>
__global__ void __launch_bounds__(256) k_load_convert(const double *src, long long n,
                                                      double scale, R *dst, int check,
                                                      double dx, double hi, int unbounded,
                                                      unsigned *bad) {
  unsigned b = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = src[i];
    if (check) {
      const double X = v / dx;
      b += (unbounded ? !isfinite(X) : !(X >= 0.0 && X <= hi)) ? 1u : 0u;
    }
    if (dst) dst[i] = (R)(v * scale);
  }
  if (check && b) atomicAdd(bad, b);
}

__global__ void __launch_bounds__(256) k_check_ids(const uint32_t *id, long long n,
                                                   unsigned *bad) {
  unsigned b = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b += id[i] == kDead ? 1u : 0u;
  if (b) atomicAdd(bad, b);
}

template <typename R>
__global__ void __launch_bounds__(256) k_fill(R *dst, long long n, R v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = v;
}

long long xfer_chunks(long long n) { return (n + kXferChunk - 1) / kXferChunk; }

void launch_live_scan(const uint32_t *id, long long n, uint32_t *cc, cudaStream_t st) {
  const long long nb = xfer_chunks(n);
  if (nb > 0) k_live_counts<<<(unsigned)nb, 256, 0, st>>>(id, n, cc);
  k_scan_chunks<<<1, 1024, 0, st>>>(cc, nb);
}

template <typename T, typename O>
void launch_compact(const T *src, const uint32_t *id, long long n, const uint32_t *cc,
                    double scale, O *out, cudaStream_t st) {
  const long long nb = xfer_chunks(n);
  if (nb > 0) k_compact<T, O><<<(unsigned)nb, 256, 0, st>>>(src, id, n, cc, scale, out);
}

template <typename R>
void launch_load_convert(const double *src, long long n, double scale, R *dst, int check,
                         double dx, double hi, int unbounded, unsigned *bad, int grid,
                         cudaStream_t st) {
  k_load_convert<R><<<grid, 256, 0, st>>>(src, n, scale, dst, check, dx, hi, unbounded, bad);
}

void launch_check_ids(const uint32_t *id, long long n, unsigned *bad, int grid, cudaStream_t st) {
  k_check_ids<<<grid, 256, 0, st>>>(id, n, bad);
}

template <typename R>
void launch_fill(R *dst, long long n, R v, int grid, cudaStream_t st) {
  k_fill<R><<<grid, 256, 0, st>>>(dst, n, v);
}

template void launch_compact<uint32_t, uint32_t>(const uint32_t *, const uint32_t *, long long,
                                                 const uint32_t *, double, uint32_t *,
                                                 cudaStream_t);

#define HPIC_INST(R)                                                                          \
  template void launch_efield<R>(const Consts &, GView<R>, int, cudaStream_t);                \
  template void launch_bheat<R>(const Consts &, GView<R>, TallyView, int, cudaStream_t);      \
  template int launch_sort<R>(const Consts &, PView<R>, PView<R>, Counters *, uint32_t *,     \
                              uint32_t *, uint32_t *, int, cudaStream_t, double);             \
  template int launch_sort_keys<R>(const Consts &, PView<R>, Counters *, uint32_t *, uint32_t *, \
                                   uint32_t *, uint32_t *, int, cudaStream_t, double);        \
  template void launch_live_energy<R>(const Consts &, PView<R>, Counters *, double *, int,    \
                                      cudaStream_t);                                          \
  template void launch_field_energy<R>(const Consts &, GView<R>, double *, int, cudaStream_t); \
  template void launch_batch_efield<R>(const BatchItem<R> *, BatchDev, int, cudaStream_t);     \
  template void launch_batch_bheat<R>(const BatchItem<R> *, BatchDev, int, cudaStream_t);     \
  template void launch_compact<R, double>(const R *, const uint32_t *, long long,             \
                                          const uint32_t *, double, double *, cudaStream_t);  \
  template void launch_load_convert<R>(const double *, long long, double, R *, int, double,   \
                                       double, int, unsigned *, int, cudaStream_t);           \
  template void launch_fill<R>(R *, long long, R, int, cudaStream_t);
HPIC_INST(float)
HPIC_INST(double)
#undef HPIC_INST

}  // namespace hpic
