// Host side of the batch entry points in include/hpic.h: many independent
// targets (the paper's scans over thickness, material and intensity,
// Sec. III) advanced together, one launch per kernel kind per step, the step
// replayed from captured CUDA graphs, and an autotuner for the persistent
// particle kernel's blocks per SM and the sort interval.
//
// All state of all targets lives in one device allocation (the arena), so a
// snapshot for the autotuner is one device-to-device copy.  Each target is
// also exposed as an hpic_ctx whose pointers lie inside the arena, so the
// single-target read and write entry points serve batch targets unchanged.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

namespace {

thread_local std::string g_batch_error;

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }
size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

constexpr int kSortChoices[4] = {3, 5, 10, 20};
constexpr int kTrialPeriod = 40;  // every sort interval tried divides it

}  // namespace

struct hpic_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n = 0;
  bool fp32 = false;
  size_t rsz = 8;
  int sm_count = 1;
  hpic_run_params run{};
  std::vector<hpic_ctx *> tg;  // borrowed per-target contexts
  // state of every target: one allocation
  void *arena = nullptr;
  size_t arena_bytes = 0;
  void *pbuf[2] = {nullptr, nullptr};
  int cur = 0;
  long long slots = 0;  // elements per particle array (all targets)
  void *jall = nullptr;
  size_t jall_bytes = 0;
  double *hall = nullptr;
  long long cells = 0;
  // per-step scratch, constants and tables: a second allocation
  void *aux = nullptr;
  void *items = nullptr;  // BatchItem<R>[n]
  hpic::BatchDev d{};
  uint32_t *keys = nullptr, *counts = nullptr, *partials = nullptr;
  long long nkeys_total = 0, nodes_total = 0;
  double *t64 = nullptr;
  float *t32 = nullptr;
  bool any_inject = false;
  bool single = true;  // every target a single-element solid
  long long host_step = 0;
  hpic_batch_tuning tune{};
  cudaGraphExec_t gstep[2] = {nullptr, nullptr}, gsort[2] = {nullptr, nullptr};
  int kstep = 0, ksort = 0;  // kernels in each graph
  long long launches = 0;
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  long long prof_launches = 0;
  double prof_ps0 = 0.0;
  std::string err;
};

namespace {

int bfail(hpic_batch *b, int code, const std::string &msg) {
  if (b) b->err = msg; else g_batch_error = msg;
  return code;
}

int bcuda(hpic_batch *b, cudaError_t e, const char *where) {
  return bfail(b, HPIC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define BCK(call)                                                      \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call);                 \
  } while (0)

int grid_for(const hpic_batch *b, long long work) {
  const long long want = (work + 255) / 256, cap = (long long)b->sm_count * 8;
  const long long g = want < cap ? want : cap;
  return (int)(g < 1 ? 1 : g);
}

int max_blocks_per_sm(const hpic_batch *b) { return b->fp32 ? 5 : 2; }
int min_blocks_per_sm(const hpic_batch *b) { return b->fp32 ? 2 : 1; }

template <typename R>
hpic::PView<R> pview_all(const hpic_batch *b, int which) {
  char *base = static_cast<char *>(b->pbuf[which]);
  R *r = reinterpret_cast<R *>(base);
  hpic::PView<R> v;
  v.x = r;
  v.y = r + b->slots;
  v.z = r + 2 * b->slots;
  v.ux = r + 3 * b->slots;
  v.uy = r + 4 * b->slots;
  v.uz = r + 5 * b->slots;
  v.tau = r + 6 * b->slots;
  v.w = r + 7 * b->slots;
  v.id = reinterpret_cast<uint32_t *>(base + 8 * (size_t)b->slots * sizeof(R));
  return v;
}

void set_cur(hpic_batch *b, int cur) {
  b->cur = cur;
  for (hpic_ctx *c : b->tg) c->cur = cur;
}

void drop_graphs(hpic_batch *b) {
  for (int c = 0; c < 2; ++c) {
    if (b->gstep[c]) cudaGraphExecDestroy(b->gstep[c]);
    if (b->gsort[c]) cudaGraphExecDestroy(b->gsort[c]);
    b->gstep[c] = b->gsort[c] = nullptr;
  }
}

// one step of every target; returns the kernels launched, or < 0 on error
// One step of every target; with sort, the cell sort rides on it (keys from
// the start-of-step state one step further ahead, the push writing each
// electron to its sorted slot of the other buffer, injection into that one).
template <typename R>
int enqueue_step(hpic_batch *b, bool sort) {
  const auto *items = static_cast<const hpic::BatchItem<R> *>(b->items);
  const hpic::PView<R> P = pview_all<R>(b, b->cur);
  const hpic::PView<R> Pnext = sort ? pview_all<R>(b, b->cur ^ 1) : P;
  const R *tab = b->fp32 ? reinterpret_cast<const R *>(b->t32) : reinterpret_cast<const R *>(b->t64);
  const bool grid_on = !(b->run.physics & HPIC_UNBOUNDED);
  const int gg = (int)std::min<long long>((b->nodes_total + 255) / 256,
                                          (long long)b->sm_count * hpic::kBatchFieldBlocksPerSm);
  int k = 0;
  if (grid_on) {
    BCK(cudaMemsetAsync(b->jall, 0, b->jall_bytes, b->stream));
    BCK(cudaMemsetAsync(b->hall, 0, b->cells * sizeof(double), b->stream));
  }
  hpic::launch_batch_plan<R>(items, b->d, b->stream);
  ++k;
  hpic::SortOut<R> so{};
  if (sort) {
    uint32_t *ranks = b->keys + b->slots;
    k += hpic::launch_batch_sort_keys<R>(items, b->d, P, b->keys, ranks, b->counts, b->partials,
                                         b->nkeys_total, grid_for(b, b->slots), b->stream,
                                         hpic::sort_lead(b->tune.sort_interval) + 1.0);
    so.dst = Pnext;
    so.keys = b->keys;
    so.ranks = ranks;
    so.offsets = b->counts;
  }
  if (b->prof) {
    if (b->ev_used + 2 > b->ev.size()) {
      for (int q = 0; q < 64; ++q) {
        cudaEvent_t e;
        BCK(cudaEventCreate(&e));
        b->ev.push_back(e);
      }
    }
    BCK(cudaEventRecord(b->ev[b->ev_used], b->stream));
  }
  hpic::launch_batch_push<R>(b->tg[0]->K, items, b->d, P, tab, b->sm_count, b->tune.blocks_per_sm,
                             b->single, b->stream, so);
  ++k;
  if (b->prof) {
    BCK(cudaEventRecord(b->ev[b->ev_used + 1], b->stream));
    b->ev_used += 2;
    b->prof_launches += 1;
  }
  if (grid_on && (b->run.physics & HPIC_FIELDS)) {
    hpic::launch_batch_efield<R>(items, b->d, gg, b->stream);
    ++k;
  }
  if (grid_on) {
    hpic::launch_batch_bheat<R>(items, b->d, gg, b->stream);
    ++k;
  }
  if (sort) k += hpic::launch_batch_sort_finish<R>(items, b->d, b->stream);
  if (b->any_inject) {
    hpic::launch_batch_inject<R>(items, b->d, Pnext, b->sm_count * 2, b->stream);
    ++k;
  }
  hpic::launch_batch_advance<R>(items, b->d, b->stream);
  ++k;
  BCK(cudaGetLastError());
  return k;
}

int enqueue(hpic_batch *b, bool sort) {
  return b->fp32 ? enqueue_step<float>(b, sort) : enqueue_step<double>(b, sort);
}

// capture the plain step and the step that sorts, for both particle buffers
int capture_graphs(hpic_batch *b) {
  if (b->gstep[0]) return HPIC_OK;
  const int keep = b->cur;
  for (int c = 0; c < 2; ++c) {
    for (int sort = 0; sort < 2; ++sort) {
      b->cur = c;
      BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      const int k = enqueue(b, sort != 0);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      if (k < 0 || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        b->cur = keep;
        drop_graphs(b);
        return k < 0 ? k : bcuda(b, e, "cudaStreamEndCapture");
      }
      cudaGraphExec_t x = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        b->cur = keep;
        drop_graphs(b);
        return bcuda(b, ei, "cudaGraphInstantiate");
      }
      (sort ? b->gsort : b->gstep)[c] = x;
      (sort ? b->ksort : b->kstep) = k;
    }
  }
  b->cur = keep;
  for (int c = 0; c < 2; ++c) {
    BCK(cudaGraphUpload(b->gstep[c], b->stream));
    BCK(cudaGraphUpload(b->gsort[c], b->stream));
  }
  return HPIC_OK;
}

int run_steps(hpic_batch *b, long long nsteps) {
  const bool graphs = b->tune.use_graph && !b->prof;
  if (graphs) {
    const int rc = capture_graphs(b);
    if (rc) return rc;
  }
  for (long long s = 0; s < nsteps; ++s) {
    const int si = b->tune.sort_interval;
    const bool sort = si > 0 && (b->host_step + 1) % si == 0;
    if (graphs) {
      BCK(cudaGraphLaunch((sort ? b->gsort : b->gstep)[b->cur], b->stream));
      b->launches += sort ? b->ksort : b->kstep;
    } else {
      const int k = enqueue(b, sort);
      if (k < 0) return k;
      b->launches += k;
    }
    b->host_step += 1;
    for (hpic_ctx *c : b->tg) c->host_step = b->host_step;
    if (sort) set_cur(b, b->cur ^ 1);
  }
  return HPIC_OK;
}

double sum_psteps(hpic_batch *b, int *rc) {
  std::vector<double> t((size_t)b->n * hpic::T_COUNT);
  const double *tal = b->tg[0]->tal;  // the targets' tallies are consecutive
  cudaError_t e = cudaMemcpyAsync(t.data(), tal, t.size() * sizeof(double),
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    *rc = bcuda(b, e, "tally read");
    return 0.0;
  }
  double s = 0.0;
  for (int q = 0; q < b->n; ++q) s += t[(size_t)q * hpic::T_COUNT + hpic::T_PSTEPS];
  *rc = HPIC_OK;
  return s;
}

void destroy_batch(hpic_batch *b) {
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  cudaFree(b->arena);
  cudaFree(b->aux);
  for (hpic_ctx *c : b->tg) {
    cudaFree(c->xfer);
    delete c;
  }
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

template <typename R>
void fill_items(hpic_batch *b, std::vector<char> &out) {
  out.resize(sizeof(hpic::BatchItem<R>) * b->n);
  auto *it = reinterpret_cast<hpic::BatchItem<R> *>(out.data());
  for (int t = 0; t < b->n; ++t) {
    const hpic_ctx *c = b->tg[t];
    std::memset(&it[t], 0, sizeof(it[t]));
    it[t].K = c->K;
    it[t].h = hpic::make_hot<R>(c->K);
    it[t].g = gview<R>(c);
    it[t].tv = tview(c);
    it[t].cnt = c->cnt;
    it[t].off = c->poff;
    it[t].cap = c->cap;
  }
}

}  // namespace

extern "C" {

int hpic_batch_init(hpic_batch **out, int32_t n_targets, const hpic_target_desc *targets,
                    const hpic_laser_desc *lasers, const hpic_run_params *run,
                    const uint32_t *target_index, int64_t spare_slots, int device,
                    void *cuda_stream) {
  if (!out) return bfail(nullptr, HPIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!targets || !run) return bfail(nullptr, HPIC_EINVAL, "targets or run params NULL");
  if (n_targets < 1 || n_targets > HPIC_BATCH_MAX_TARGETS)
    return bfail(nullptr, HPIC_EINVAL, "n_targets must be 1.." + std::to_string(HPIC_BATCH_MAX_TARGETS));
  if (spare_slots < 0) return bfail(nullptr, HPIC_EINVAL, "negative spare_slots");
  for (int t = 0; t < n_targets; ++t) {
    if (const char *why = hpic::check_target(targets[t], *run))
      return bfail(nullptr, HPIC_EINVAL, "target " + std::to_string(t) + ": " + why);
    if (lasers) {
      if (const char *why = hpic::check_laser(lasers[t], targets[t]))
        return bfail(nullptr, HPIC_EINVAL, "laser " + std::to_string(t) + ": " + why);
      if (lasers[t].envelope != HPIC_ENV_FLAT)
        return bfail(nullptr, HPIC_EINVAL, "laser " + std::to_string(t) +
                                               ": batches inject with the flat-top envelope only");
      if (lasers[t].n_macro + spare_slots >= 0xFFFFFFFFll)
        return bfail(nullptr, HPIC_EINVAL, "id space exhausted");
    }
  }
  if (!target_index && (long long)run->target_index + n_targets > 0xFFFFFFFFll)
    return bfail(nullptr, HPIC_EINVAL, "target_index + n_targets exceeds 32 bits");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return bfail(nullptr, HPIC_ECUDA, "no such CUDA device");
  }
  if (cudaSetDevice(device) != cudaSuccess) return bcuda(nullptr, cudaGetLastError(), "cudaSetDevice");

  hpic_batch *b = new hpic_batch();
  b->device = device;
  b->n = n_targets;
  b->run = *run;
  b->fp32 = run->precision == HPIC_FP32_MIXED;
  b->rsz = b->fp32 ? 4 : 8;
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, device);
  auto bail = [&](int code) {
    const std::string m = b->err;
    destroy_batch(b);
    g_batch_error = m;
    return code;
  };
  if (const cudaError_t e = hpic::prepare_batch_push(); e != cudaSuccess) {
    bcuda(b, e, "batch push kernel shared memory");
    return bail(HPIC_ECUDA);
  }
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      bcuda(b, cudaGetLastError(), "cudaStreamCreate");
      return bail(HPIC_ECUDA);
    }
    b->own_stream = true;
  }

  // per-target contexts and the layout of the shared arrays
  std::vector<long long> npref(n_targets + 1, 0), kpref(n_targets + 1, 0);
  long long slots = 0, eb = 0, jv = 0, cells = 0;
  const long long hist_len = (long long)(run->n_Ebins + 2) * run->n_thbins;
  const long long hlen = run->max_history > 0 ? run->max_history : 1;
  for (int t = 0; t < n_targets; ++t) {
    hpic_ctx *c = new hpic_ctx();
    b->tg.push_back(c);
    c->owner = b;
    c->device = device;
    c->stream = b->stream;
    c->tgt = targets[t];
    c->run = *run;
    c->run.target_index = target_index ? target_index[t] : run->target_index + (uint32_t)t;
    c->have_laser = lasers != nullptr;
    if (lasers) c->laser = lasers[t];
    c->fp32 = b->fp32;
    c->rsz = b->rsz;
    c->sm_count = b->sm_count;
    hpic::fold(c->tgt, c->run, c->have_laser ? &c->laser : nullptr, c->K);
    if (c->have_laser && c->K.n_macro > 0) b->any_inject = true;
    if (c->K.n_solids != 1) b->single = false;
    const long long need = (c->have_laser ? c->K.n_macro : 0) + spare_slots;
    c->cap = round_up(need < 32 ? 32 : need, 32);
    c->poff = slots;
    slots += c->cap;
    c->vstride = round_up(c->K.nvec + 4, 64);
    eb += 6 * c->vstride;
    jv += 3 * c->vstride;
    cells += c->K.ncell;
    npref[t + 1] = npref[t] + c->K.nvec;
    kpref[t + 1] = kpref[t] + c->K.nkeys + 1;
  }
  slots = round_up(slots, 64);
  if (slots >= 0x7FFFFFFFll || kpref[n_targets] >= 0x7FFFFFFFll) {
    bfail(b, HPIC_EINVAL, "batch too large (particle slots and sort keys must stay below 2^31)");
    return bail(HPIC_EINVAL);
  }
  b->slots = slots;
  b->cells = cells;
  b->nodes_total = npref[n_targets];
  b->nkeys_total = kpref[n_targets];

  // arena: particles (x2), E and B, J, T, eta, heat, tallies, histograms,
  // histories, counters, read scratch
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t pb = (size_t)slots * (8 * b->rsz + sizeof(uint32_t));
  const size_t o_p0 = take(pb), o_p1 = take(pb);
  const size_t o_eb = take(eb * b->rsz), o_j = take(jv * b->rsz);
  const size_t o_T = take(cells * sizeof(double)), o_eta = take(cells * sizeof(double));
  const size_t o_H = take(cells * sizeof(double));
  const size_t o_er = take(b->fp32 ? cells * sizeof(float) : 0);
  const size_t o_Ti = take(cells * sizeof(double)), o_Fs = take(cells * b->rsz);
  const size_t o_tal = take((size_t)n_targets * hpic::T_COUNT * sizeof(double));
  const size_t o_hist = take((size_t)n_targets * 2 * hist_len * sizeof(double));
  const size_t o_hy = take((size_t)n_targets * hlen * sizeof(double));
  const size_t o_cnt = take((size_t)n_targets * sizeof(hpic::Counters));
  const size_t o_scr = take((size_t)n_targets * 2 * sizeof(double));
  b->arena_bytes = off;
  // aux: items, prefixes, sort scratch, tables
  const size_t isz = b->fp32 ? sizeof(hpic::BatchItem<float>) : sizeof(hpic::BatchItem<double>);
  const long long tab = (long long)run->table_rows * run->table_cols;
  off = 0;
  const size_t a_items = take(isz * n_targets);
  const size_t a_w = take((n_targets + 1) * sizeof(long long));
  const size_t a_i = take((n_targets + 1) * sizeof(long long));
  const size_t a_n = take((n_targets + 1) * sizeof(long long));
  const size_t a_k = take((n_targets + 1) * sizeof(long long));
  const size_t a_s0 = take(n_targets * sizeof(long long)), a_s1 = take(n_targets * sizeof(long long));
  const size_t a_keys = take(2 * slots * sizeof(uint32_t));  // sort keys, then ranks
  const size_t a_cnts = take(b->nkeys_total * sizeof(uint32_t));
  const size_t a_part = take(hpic::scan_partials(b->nkeys_total) * sizeof(uint32_t));
  const size_t a_t64 = take(tab * sizeof(double)), a_t32 = take(tab * sizeof(float));
  const size_t aux_bytes = off;
  if (cudaMalloc(&b->arena, b->arena_bytes) != cudaSuccess ||
      cudaMalloc(&b->aux, aux_bytes) != cudaSuccess) {
    cudaGetLastError();
    bfail(b, HPIC_ENOMEM, "device allocation failed (" + std::to_string(b->arena_bytes + aux_bytes) + " bytes)");
    return bail(HPIC_ENOMEM);
  }
  char *A = static_cast<char *>(b->arena), *X = static_cast<char *>(b->aux);
  b->pbuf[0] = A + o_p0;
  b->pbuf[1] = A + o_p1;
  b->jall = A + o_j;
  b->jall_bytes = jv * b->rsz;
  b->hall = reinterpret_cast<double *>(A + o_H);
  b->items = X + a_items;
  b->d.n = n_targets;
  b->d.wpref = reinterpret_cast<long long *>(X + a_w);
  b->d.ipref = reinterpret_cast<long long *>(X + a_i);
  b->d.npref = reinterpret_cast<long long *>(X + a_n);
  b->d.kpref = reinterpret_cast<long long *>(X + a_k);
  b->d.sstart = reinterpret_cast<long long *>(X + a_s0);
  b->d.snew = reinterpret_cast<long long *>(X + a_s1);
  b->keys = reinterpret_cast<uint32_t *>(X + a_keys);
  b->counts = reinterpret_cast<uint32_t *>(X + a_cnts);
  b->partials = reinterpret_cast<uint32_t *>(X + a_part);
  b->t64 = reinterpret_cast<double *>(X + a_t64);
  b->t32 = reinterpret_cast<float *>(X + a_t32);

  long long e_at = 0, j_at = 0, c_at = 0;
  for (int t = 0; t < n_targets; ++t) {
    hpic_ctx *c = b->tg[t];
    c->stride = slots;
    c->pbuf[0] = b->pbuf[0];
    c->pbuf[1] = b->pbuf[1];
    c->fields = A + o_eb + e_at * b->rsz;
    c->jfield = A + o_j + j_at * b->rsz;
    c->T = reinterpret_cast<double *>(A + o_T) + c_at;
    c->eta = reinterpret_cast<double *>(A + o_eta) + c_at;
    if (b->fp32) c->eta_r = reinterpret_cast<float *>(A + o_er) + c_at;
    c->Ti = reinterpret_cast<double *>(A + o_Ti) + c_at;
    c->Fsig = A + o_Fs + c_at * b->rsz;
    c->H = reinterpret_cast<double *>(A + o_H) + c_at;
    c->tal = reinterpret_cast<double *>(A + o_tal) + (size_t)t * hpic::T_COUNT;
    c->hist = reinterpret_cast<double *>(A + o_hist) + (size_t)t * 2 * hist_len;
    c->history = reinterpret_cast<double *>(A + o_hy) + (size_t)t * hlen;
    c->cnt = reinterpret_cast<hpic::Counters *>(A + o_cnt) + t;
    c->scratch = reinterpret_cast<double *>(A + o_scr) + 2 * t;
    c->t64 = b->t64;
    c->t32 = b->t32;
    e_at += 6 * c->vstride;
    j_at += 3 * c->vstride;
    c_at += c->K.ncell;
  }

  // initial state: zero everything, then T0 and eta(T0) per target
  cudaStream_t st = b->stream;
  std::vector<double> T0(cells), E0(cells), F0(cells);
  c_at = 0;
  for (int t = 0; t < n_targets; ++t) {
    const hpic_ctx *c = b->tg[t];
    const double e0 = hpic::eta_of(c->K, c->tgt.T0_K), f0 = hpic::fsigma_of(c->K, c->tgt.T0_K);
    std::fill(T0.begin() + c_at, T0.begin() + c_at + c->K.ncell, c->tgt.T0_K);
    std::fill(E0.begin() + c_at, E0.begin() + c_at + c->K.ncell, e0);
    std::fill(F0.begin() + c_at, F0.begin() + c_at + c->K.ncell, f0);
    c_at += c->K.ncell;
  }
  std::vector<float> F0f(b->fp32 ? cells : 0);
  for (size_t i = 0; i < F0f.size(); ++i) F0f[i] = (float)F0[i];
  std::vector<float> E0f(b->fp32 ? cells : 0);
  for (size_t i = 0; i < E0f.size(); ++i) E0f[i] = (float)E0[i];
  std::vector<char> items;
  if (b->fp32) fill_items<float>(b, items); else fill_items<double>(b, items);
  if (cudaMemsetAsync(b->arena, 0, b->arena_bytes, st) != cudaSuccess ||
      cudaMemcpyAsync(b->tg[0]->T, T0.data(), cells * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b->tg[0]->eta, E0.data(), cells * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (b->fp32 && cudaMemcpyAsync(b->tg[0]->eta_r, E0f.data(), cells * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      cudaMemcpyAsync(b->tg[0]->Ti, T0.data(), cells * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b->tg[0]->Fsig, b->fp32 ? (const void *)F0f.data() : (const void *)F0.data(),
                      cells * b->rsz, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b->items, items.data(), items.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(X + a_n, npref.data(), npref.size() * sizeof(long long), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(X + a_k, kpref.data(), kpref.size() * sizeof(long long), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    bcuda(b, cudaGetLastError(), "initialisation");
    return bail(HPIC_ECUDA);
  }
  const hpic::Consts &K0 = b->tg[0]->K;
  hpic::launch_table(K0, K0.k_min, K0.k_min * (run->table_Emax_J / run->k_min_J), b->t64, b->t32, st);
  b->launches += 1;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    bcuda(b, e, "batch initialisation");
    return bail(HPIC_ECUDA);
  }
  b->tune.blocks_per_sm = max_blocks_per_sm(b);
  b->tune.sort_interval = run->sort_interval;
  b->tune.use_graph = 1;
  *out = b;
  return HPIC_OK;
}

int hpic_batch_target(hpic_batch *b, int32_t t, hpic_ctx **out) {
  if (!b || !out) return bfail(b, HPIC_EINVAL, "NULL argument");
  if (t < 0 || t >= b->n) return bfail(b, HPIC_EINVAL, "no such target");
  *out = b->tg[t];
  return HPIC_OK;
}

int hpic_batch_step(hpic_batch *b, int64_t n) {
  if (!b) return HPIC_EINVAL;
  if (n < 0) return bfail(b, HPIC_EINVAL, "negative step count");
  BCK(cudaSetDevice(b->device));
  return run_steps(b, n);
}

int hpic_batch_get_tuning(const hpic_batch *b, hpic_batch_tuning *out) {
  if (!b || !out) return HPIC_EINVAL;
  *out = b->tune;
  return HPIC_OK;
}

int hpic_batch_set_tuning(hpic_batch *b, const hpic_batch_tuning *in) {
  if (!b || !in) return bfail(b, HPIC_EINVAL, "NULL argument");
  if (in->blocks_per_sm < 1 || in->blocks_per_sm > max_blocks_per_sm(b) || in->sort_interval < 0)
    return bfail(b, HPIC_EINVAL, "tuning out of range");
  BCK(cudaSetDevice(b->device));
  BCK(cudaStreamSynchronize(b->stream));
  drop_graphs(b);
  b->tune.blocks_per_sm = in->blocks_per_sm;
  b->tune.sort_interval = in->sort_interval;
  b->tune.use_graph = in->use_graph != 0;
  return HPIC_OK;
}

int hpic_batch_autotune(hpic_batch *b, int32_t trial_steps, hpic_batch_tuning *out) {
  if (!b) return HPIC_EINVAL;
  if (trial_steps < 1) return bfail(b, HPIC_EINVAL, "trial_steps must be >= 1");
  if (b->prof) return bfail(b, HPIC_ESTATE, "disable profiling before autotuning");
  BCK(cudaSetDevice(b->device));
  BCK(cudaStreamSynchronize(b->stream));
  const long long L = round_up(trial_steps, kTrialPeriod);
  void *snap = nullptr;
  if (cudaMalloc(&snap, b->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, HPIC_ENOMEM, "no device memory for the autotuner's snapshot");
  }
  const int cur0 = b->cur;
  const long long step0 = b->host_step;
  const long long launches0 = b->launches;  // the trials' launches are not the run's
  const hpic_batch_tuning keep = b->tune;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HPIC_OK;
  hpic_batch_tuning best = keep;
  best.ms_per_step = -1.0;
  auto restore = [&]() -> int {
    BCK(cudaMemcpyAsync(b->arena, snap, b->arena_bytes, cudaMemcpyDeviceToDevice, b->stream));
    set_cur(b, cur0);
    b->host_step = step0;
    for (hpic_ctx *c : b->tg) c->host_step = step0;
    b->launches = launches0;
    return HPIC_OK;
  };
  if (cudaMemcpyAsync(snap, b->arena, b->arena_bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = bcuda(b, cudaGetLastError(), "autotune setup");
  }
  for (int bps = min_blocks_per_sm(b); rc == HPIC_OK && bps <= max_blocks_per_sm(b); ++bps) {
    for (int s = 0; rc == HPIC_OK && s < 4; ++s) {
      rc = restore();
      if (rc) break;
      drop_graphs(b);
      b->tune.blocks_per_sm = bps;
      b->tune.sort_interval = kSortChoices[s];
      b->tune.use_graph = 1;
      rc = capture_graphs(b);
      if (rc) break;
      cudaError_t e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess) rc = run_steps(b, L);
      if (e == cudaSuccess && rc == HPIC_OK) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess && rc == HPIC_OK) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess && rc == HPIC_OK) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) rc = bcuda(b, e, "autotune trial");
      if (rc) break;
      if (best.ms_per_step < 0.0 || ms / L < best.ms_per_step) {
        best = b->tune;
        best.ms_per_step = ms / L;
      }
    }
  }
  const int rr = restore();
  if (rc == HPIC_OK) rc = rr;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess && rc == HPIC_OK) rc = bcuda(b, e, "autotune restore");
  cudaFree(snap);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  drop_graphs(b);
  b->tune = rc == HPIC_OK ? best : keep;
  if (rc == HPIC_OK && out) *out = best;
  return rc;
}

int hpic_batch_profile(hpic_batch *b, int enable) {
  if (!b) return HPIC_EINVAL;
  BCK(cudaSetDevice(b->device));
  BCK(cudaStreamSynchronize(b->stream));
  b->prof = enable != 0;
  b->ev_used = 0;
  b->prof_launches = 0;
  int rc;
  b->prof_ps0 = sum_psteps(b, &rc);
  return rc;
}

int hpic_batch_kernel_time(hpic_batch *b, double *ms, int64_t *launches, double *psteps) {
  if (!b) return HPIC_EINVAL;
  BCK(cudaSetDevice(b->device));
  BCK(cudaStreamSynchronize(b->stream));
  double total = 0.0;
  for (size_t i = 0; i + 1 < b->ev_used; i += 2) {
    float t = 0.f;
    BCK(cudaEventElapsedTime(&t, b->ev[i], b->ev[i + 1]));
    total += t;
  }
  int rc;
  const double ps = sum_psteps(b, &rc);
  if (rc) return rc;
  if (ms) *ms = total;
  if (launches) *launches = b->prof_launches;
  if (psteps) *psteps = ps - b->prof_ps0;
  b->ev_used = 0;
  b->prof_launches = 0;
  b->prof_ps0 = ps;
  return HPIC_OK;
}

int hpic_batch_launch_count(const hpic_batch *b, int64_t *launches) {
  if (!b || !launches) return HPIC_EINVAL;
  *launches = b->launches;
  return HPIC_OK;
}

int hpic_batch_destroy(hpic_batch *b) {
  if (!b) return HPIC_EINVAL;
  destroy_batch(b);
  return HPIC_OK;
}

const char *hpic_batch_last_error(const hpic_batch *b) {
  return b ? b->err.c_str() : g_batch_error.c_str();
}

}  // extern "C"
