// Internal declarations shared by the kernel translation units and api.cu.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "hpic.h"

namespace hpic {

// particle storage: structure of arrays, positions in cells, momenta u = p/(m_e c)
template <typename R>
struct PView {
  R *x, *y, *z, *ux, *uy, *uz, *tau;
  R *w;  // per-electron weight (read only when Consts::weighted)
  uint32_t *id;
};

// grid storage: vector components as (nx+1)(ny+1)(nz+1) arrays (x fastest)
template <typename R>
struct GView {
  R *E[3], *B[3], *J[3];
  double *T, *eta, *H;  // cell-centred, double
  R *eta_r;             // eta in the field precision (its own FP32 copy, or eta itself)
  double *Ti;           // ion temperature (K)
  R *Fsig;              // F_sigma of each cell, from T_i
};

struct TallyView {
  double *tal;      // T_COUNT scalars
  double *hist;     // 2 x (n_E+2) x n_th: energy-weighted, then number-weighted
  double *history;  // max_history
};

// the per-electron constants in the kernel's own precision (folded on the
// host so that no double->float conversion runs per electron)
//
// Everything the per-electron code needs that differs between the targets
// of a batch is here (with the grid and tally views); from Consts it reads
// only run-wide values, so the batched kernel can take Consts as a kernel
// parameter and keep just these per target.
template <typename R>
struct HotK {
  R w, cdt, E_cut, K_tau, k_min, inv_boost;
  R K_ion[4], L_I[4], K_sc[4], K_lg[4];  // per element (n_solids used)
  R eps_esc, du_reflux, sigma_dtheta, tE_min, tE_max, inv_dlogE, th_scale, t_inv_dlog;
  double w_d;                // the weight in FP64 (photon weights)
  int nx, ny, nz, n_solids;  // the target's cells and elements
  uint32_t target_index;     // fourth Philox counter word
};

// the hot constants in precision R
template <typename R>
inline HotK<R> make_hot(const Consts &K) {
  HotK<R> h;
  h.w = R(K.w);
  h.cdt = R(K.cdt_dx);
  h.E_cut = R(K.E_cut);
  for (int s = 0; s < 4; ++s) {
    h.K_ion[s] = R(K.K_ion[s]);
    h.L_I[s] = R(K.L_I[s]);
    h.K_sc[s] = R(K.K_sc[s]);
    h.K_lg[s] = R(K.K_lg[s]);
  }
  h.K_tau = R(K.K_tau);
  h.k_min = R(K.k_min);
  h.inv_boost = R(K.inv_boost);
  h.eps_esc = R(K.eps_esc);
  h.du_reflux = R(K.du_reflux);
  h.sigma_dtheta = R(K.sigma_dtheta);
  h.tE_min = R(K.tE_min);
  h.tE_max = R(K.tE_max);
  h.inv_dlogE = R(K.inv_dlogE);
  h.th_scale = R(K.n_th / 3.14159265358979323846);
  h.t_inv_dlog = R(K.t_inv_dlog);
  h.w_d = K.w;
  h.nx = K.nx;
  h.ny = K.ny;
  h.nz = K.nz;
  h.n_solids = K.n_solids;
  h.target_index = K.target_index;
  return h;
}

// message returned by hpic_last_error(NULL) (entry points without a context)
void set_global_error(const char *msg);

// fold one target's SI parameters into normalised kernel constants (laser may
// be NULL: a0 = 0, weight 1), and the resistivity eta(T) of Eqs. (A4)-(A6)
void fold(const hpic_target_desc &t, const hpic_run_params &r, const hpic_laser_desc *laser,
          Consts &K);
double eta_of(const Consts &K, double T);
// F_sigma of App. B at ion temperature Ti (K)
double fsigma_of(const Consts &K, double Ti);
// the injecting face cells of a Gaussian-envelope laser (empty otherwise)
std::vector<InjCell> injection_cells(const hpic_target_desc &t, const hpic_laser_desc &l);

// Launch shape of the single-target particle kernel: resident blocks per SM
// (it is launched as one persistent wave of sm_count times this many blocks)
// and threads per block (one deposit stage per warp).  FP32: three blocks of
// 384 threads, 36 warps at 56 registers with few spills; a block's twelve
// warps take consecutive slots, so their gathers share L1 lines.  (Against
// it: five blocks of 256 at 48 registers, 84 B of spills, 3.5 % slower; six
// of 192 at 56 registers 3.2 %; four of 288 1.2 %; two of 576 level.)  FP64:
// two blocks of 256.
template <typename R>
constexpr int push_blocks_per_sm() { return sizeof(R) == 4 ? 3 : 2; }
template <typename R>
constexpr int push_threads() { return sizeof(R) == 4 ? 384 : 256; }
// resident 256-thread blocks per SM of the field and heating kernels (their
// launch bounds); they are launched as one wave of sm_count times this many
// blocks (grid-stride over the nodes), so no partial second wave trails
constexpr int kFieldBlocksPerSm = 6;
constexpr int kBatchFieldBlocksPerSm = 5;

// host transfers of the electron state (the C-ABI's read and load calls):
// live-slot compaction in storage order and FP64 <-> R conversion on the device
long long xfer_chunks(long long n);  // chunk counts needed: xfer_chunks(n) + 1
void launch_live_scan(const uint32_t *id, long long n, uint32_t *cc, cudaStream_t st);
template <typename T, typename O>
void launch_compact(const T *src, const uint32_t *id, long long n, const uint32_t *cc,
                    double scale, O *out, cudaStream_t st);
template <typename R>
void launch_load_convert(const double *src, long long n, double scale, R *dst, int check,
                         double dx, double hi, int unbounded, unsigned *bad, int grid,
                         cudaStream_t st);
void launch_check_ids(const uint32_t *id, long long n, unsigned *bad, int grid, cudaStream_t st);
template <typename R>
void launch_fill(R *dst, long long n, R v, int grid, cudaStream_t st);

// allow the push kernels their shared-memory deposit stages (above the
// default 48 KB for FP64 and the batch); once per device, before any launch
cudaError_t prepare_push();
cudaError_t prepare_batch_push();
// Where a step that also sorts writes its electrons: an electron live at
// the start of the step goes to slot offsets[key] + rank (+ a shift: 0 for
// one target; a batch target's first slot minus its first offset) of dst,
// where the counting sort's key pass ran on that start-of-step state (key
// and rank of each slot) and its scan turned the counts into offsets; one
// that is absorbed or escapes leaves its slot there marked dead.
// dst.x == nullptr: the electrons stay in their slots.
template <typename R>
struct SortOut {
  PView<R> dst;
  const uint32_t *keys, *ranks, *offsets;
};

// The sort key pass folded into the step before a sort: each electron that
// survives the step gets, from its new state, the key of the cell it reaches
// `lead` cells per unit of u/gamma ahead (as the key pass computes it from
// the start of the sorting step) and its rank among its key's electrons
// (counts must be cleared before).  keys == nullptr: no keys.
template <typename R>
struct KeyOut {
  uint32_t *keys, *ranks, *counts;
  R lead;
};

// the push kernel's modes: a plain step, a step that also computes the next
// sort's keys (KeyOut), a step that also sorts (SortOut)
enum PushMode { kPushPlain = 0, kPushKeys = 1, kPushSort = 2 };

template <typename R>
void launch_push(const Consts &K, PView<R> p, GView<R> g, const R *table, Counters *cnt,
                 TallyView tv, int grid, cudaStream_t st, const SortOut<R> &so,
                 const KeyOut<R> &ko);
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

// counting sort by cell: keys/counts/offsets are scratch; electrons are keyed
// by the cell they reach `lead` steps ahead at their current velocity (0: the
// cell they are in); returns launches made
template <typename R>
int launch_sort(const Consts &K, PView<R> src, PView<R> dst, Counters *cnt, uint32_t *keys,
                uint32_t *counts, uint32_t *partials, int grid, cudaStream_t st, double lead);

// Lead (steps) of the sort that runs every `interval` steps: the cell each
// electron reaches halfway through the coming interval, so that the gathers
// at x^n and the deposits at x^{n+1} of the steps until the next sort find
// a warp's electrons in as few cells as the drift allows
inline double sort_lead(int interval) { return interval > 0 ? 0.5 * (interval + 1) : 0.0; }

// The counting sort folded into a step: keys, ranks (each slot's place among
// the slots of its key) and the scanned offsets of the electrons in p, keyed
// `lead` steps ahead; the step's push then writes each electron to its
// sorted slot (SortOut) and launch_sort_finish sets the slot count to the
// electrons kept.  Return launches made.
template <typename R>
int launch_sort_keys(const Consts &K, PView<R> p, Counters *cnt, uint32_t *keys, uint32_t *ranks,
                     uint32_t *counts, uint32_t *partials, int grid, cudaStream_t st, double lead);
int launch_sort_finish(const Consts &K, Counters *cnt, const uint32_t *offsets, cudaStream_t st);

void launch_table(const Consts &K, double k_min, double E_max, double *t64, float *t32,
                  cudaStream_t st);

template <typename R>
void launch_live_energy(const Consts &K, PView<R> p, Counters *cnt, double *dst, int grid,
                        cudaStream_t st);
template <typename R>
void launch_field_energy(const Consts &K, GView<R> g, double *dst, int grid, cudaStream_t st);

// ---------------------------------------------------------------- batches
// One target of a batch as the batched kernels see it (a device array of
// these, one per target).
template <typename R>
struct BatchItem {
  Consts K;
  HotK<R> h;
  GView<R> g;
  TallyView tv;
  Counters *cnt;
  long long off, cap;  // particle slots [off, off + cap) of the shared arrays
};

// device arrays shared by the batched kernels (n + 1 prefix sums over targets)
struct BatchDev {
  int n;                  // targets
  long long *wpref;       // warp-sized particle tasks, from the live counts
  long long *ipref;       // electrons injected in this step
  const long long *npref; // vector-grid nodes
  const long long *kpref; // sort keys (each target's tile keys, then its dead bin)
  long long *sstart;      // sort: first sorted offset of each target (n entries)
  long long *snew;        // sort: slots kept per target (n entries)
};

// counts per step and per target: warp tasks and injections (one block)
template <typename R>
void launch_batch_plan(const BatchItem<R> *items, BatchDev d, cudaStream_t st);
// persistent particle kernel, sm_count * blocks_per_sm blocks; Krun: the
// run-wide constants (any target's Consts: those fields are common);
// single: every target is a single-element solid
template <typename R>
void launch_batch_push(const Consts &Krun, const BatchItem<R> *items, BatchDev d, PView<R> p,
                       const R *table, int sm_count, int blocks_per_sm, bool single,
                       cudaStream_t st, const SortOut<R> &so);
template <typename R>
void launch_batch_inject(const BatchItem<R> *items, BatchDev d, PView<R> p, int grid,
                         cudaStream_t st);
template <typename R>
void launch_batch_advance(const BatchItem<R> *items, BatchDev d, cudaStream_t st);
template <typename R>
void launch_batch_efield(const BatchItem<R> *items, BatchDev d, int grid, cudaStream_t st);
template <typename R>
void launch_batch_bheat(const BatchItem<R> *items, BatchDev d, int grid, cudaStream_t st);
// the cell sort of every target inside its own slots, folded into a step as
// for one target: keys, ranks and scan over the targets' concatenated key
// ranges, each target's first offset and kept slots (the step's plan must
// have run), then the push writes each electron to its sorted slot and the
// finish sets each target's slot count; return launches made
template <typename R>
int launch_batch_sort_keys(const BatchItem<R> *items, BatchDev d, PView<R> p, uint32_t *keys,
                           uint32_t *ranks, uint32_t *counts, uint32_t *partials,
                           long long nkeys_total, int grid, cudaStream_t st, double lead);
template <typename R>
int launch_batch_sort_finish(const BatchItem<R> *items, BatchDev d, cudaStream_t st);
// counts summed per block of the scan; the partials scratch of a scan of m
// counts holds scan_partials(m) words
constexpr long long kScanTile = 4096;
constexpr long long scan_partials(long long m) { return (m + kScanTile - 1) / kScanTile + 1; }
// exclusive scan of counts[0, m) in place (partials: scratch of
// scan_partials(m) words); returns launches made
int launch_scan(uint32_t *counts, long long m, uint32_t *partials, cudaStream_t st);

}  // namespace hpic
