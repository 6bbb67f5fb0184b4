// Internal: the state behind an hpic_ctx handle, shared by the single-target
// entry points (api.cu) and the batch (batch.cu).
#pragma once

#include <string>
#include <vector>

#include "hpic.h"
#include "kernels.h"

namespace hpic {
// validation shared by the single and batch entry points: NULL when the
// parameters are usable, else the reason
const char *check_target(const hpic_target_desc &t, const hpic_run_params &r);
const char *check_laser(const hpic_laser_desc &l, const hpic_target_desc &t);
}  // namespace hpic

struct hpic_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  hpic_target_desc tgt{};
  hpic_run_params run{};
  hpic_laser_desc laser{};
  bool have_laser = false;
  bool fp32 = false;
  size_t rsz = 8;  // bytes per particle/field real
  hpic::Consts K{};
  int sm_count = 1;
  // particles: two SoA buffers (the sort ping-pongs between them); this
  // context's slots are [poff, poff + cap) of arrays `stride` elements long
  long long cap = 0;
  long long stride = 0;
  long long poff = 0;
  void *pbuf[2] = {nullptr, nullptr};
  int cur = 0;
  uint32_t *keys = nullptr;
  uint32_t *counts = nullptr;
  uint32_t *partials = nullptr;
  // device scratch of the host transfers (read/load of the electron state),
  // grown on demand; owned by this context (also a borrowed batch target)
  void *xfer = nullptr;
  size_t xfer_bytes = 0;
  // grid
  void *fields = nullptr;  // E[3], B[3] of R, each nvec long, vstride apart
  void *jfield = nullptr;  // J[3], vstride apart (just after B in a single context)
  long long vstride = 0;   // nvec + >= 4 padding, a multiple of 64 (aligned vector access)
  double *T = nullptr, *eta = nullptr, *H = nullptr;
  void *eta_r = nullptr;  // FP32 copy of eta read by the FP32 field solve (mixed precision)
  double *Ti = nullptr;   // ion temperature
  void *inj_cells = nullptr;  // InjCell list of the Gaussian envelope
  void *Fsig = nullptr;   // F_sigma per cell, in the particle precision
  // tallies and tables
  double *tal = nullptr, *hist = nullptr, *history = nullptr, *scratch = nullptr;
  double *t64 = nullptr;
  float *t32 = nullptr;
  hpic::Counters *cnt = nullptr;
  long long host_step = 0;
  // the host step whose start-of-step state the stored sort keys and ranks
  // (with their counts) describe, computed by the step before it; -1: none.
  // Every call that changes the electrons between steps clears it.
  long long keys_step = -1;
  long long launches = 0;
  // profiling of the particle kernel
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  long long prof_launches = 0;
  double prof_ps0 = 0.0;
  std::string err;
  // set for the per-target contexts of a batch: the batch owns every buffer
  // and steps the target; the read/write entry points work unchanged
  hpic_batch *owner = nullptr;
};


template <typename R>
inline hpic::PView<R> pview(const hpic_ctx *c, int which) {
  char *b = static_cast<char *>(c->pbuf[which]);
  const size_t s = (size_t)c->stride * sizeof(R);
  R *r = reinterpret_cast<R *>(b) + c->poff;
  hpic::PView<R> v;
  v.x = r;
  v.y = r + c->stride;
  v.z = r + 2 * c->stride;
  v.ux = r + 3 * c->stride;
  v.uy = r + 4 * c->stride;
  v.uz = r + 5 * c->stride;
  v.tau = r + 6 * c->stride;
  v.w = r + 7 * c->stride;
  v.id = reinterpret_cast<uint32_t *>(b + 8 * s) + c->poff;
  return v;
}

template <typename R>
inline hpic::GView<R> gview(const hpic_ctx *c) {
  hpic::GView<R> g;
  R *f = static_cast<R *>(c->fields);
  R *j = static_cast<R *>(c->jfield);
  const long long nv = c->vstride;
  for (int a = 0; a < 3; ++a) {
    g.E[a] = f + a * nv;
    g.B[a] = f + (3 + a) * nv;
    g.J[a] = j + a * nv;
  }
  g.T = c->T;
  g.eta = c->eta;
  g.eta_r = c->fp32 ? static_cast<R *>(c->eta_r) : reinterpret_cast<R *>(c->eta);
  g.Ti = c->Ti;
  g.Fsig = static_cast<R *>(c->Fsig);
  g.H = c->H;
  return g;
}

inline hpic::TallyView tview(const hpic_ctx *c) { return hpic::TallyView{c->tal, c->hist, c->history}; }

