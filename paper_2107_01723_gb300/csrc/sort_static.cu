// hpic_sort_cells_noalloc: the cell sort of the electron population for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs while a CUDA
// stream is being captured into a graph (allocation is not a capturable
// operation and breaks the capture), real-time or embedded hosts that fix
// their device-memory budget at start-up, and plug-ins whose host framework
// owns every device allocation through its own pool.  This entry point
// sorts caller-owned electron arrays into caller-owned output arrays and
// takes its scratch (sort keys, per-key counts and offsets, scan partials,
// the live count) from one fixed array in this file, so it allocates
// nothing, on the device or the host.
//
// The scratch array is a file-scope __device__ variable: every GPU that
// loads this library holds it (8 MiB + 64 KiB) until the process exits.
// Host code cannot pass the variable's name to a kernel (on the host it is
// only a stand-in symbol); its device address is looked up once per device
// with cudaGetSymbolAddress, with that device current, the first time the
// entry point runs on that device.  That first call should therefore come
// before any stream capture.  Every call reuses the same scratch, which
// keeps the previous call's contents: the per-key counts are cleared at the
// start of each call, and everything else is overwritten before it is read.
// Calls that overlap on the GPU (on different streams, or from several host
// threads) share the scratch and race; serialise them.  The looked-up
// address stays valid for the life of the device's primary context: after
// cudaDeviceReset (or any reset of that context) the module is loaded again
// and the array may move, so this entry point must not be called again in a
// process that has reset the device.  The output arrays must not overlap the
// input arrays (the scatter reads one while it writes the other); overlapping
// ranges are refused.
#include <mutex>

#include "hpic.h"
#include "kernels.h"

namespace {

constexpr long long kMaxElectrons = 1ll << 20;  // HPIC_NOALLOC_MAX_ELECTRONS
constexpr long long kMaxKeys = 1ll << 20;       // HPIC_NOALLOC_MAX_TILE_CELLS

// scratch layout (bytes): keys | counts | scan partials | counters, every
// region starting on a 256-byte boundary (the counters hold 64-bit fields)
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kKeysOff = 0;
constexpr size_t kCountsOff = align256(kKeysOff + sizeof(uint32_t) * kMaxElectrons);
constexpr size_t kPartialsOff = align256(kCountsOff + sizeof(uint32_t) * (kMaxKeys + 1));
// the scan runs over the nkeys + 1 counts (tile keys and the dead bin) with
// the scan tile of launch_scan
constexpr size_t kCountersOff =
    align256(kPartialsOff + sizeof(uint32_t) * hpic::scan_partials(kMaxKeys + 1));
constexpr size_t kScratchBytes = (8u << 20) + (64u << 10);
static_assert(kCountsOff % 256 == 0 && kPartialsOff % 256 == 0 && kCountersOff % 256 == 0,
              "scratch regions must be 256-byte aligned");
static_assert(kCountersOff + sizeof(hpic::Counters) <= kScratchBytes, "scratch layout");
static_assert(kPartialsOff + sizeof(uint32_t) * hpic::scan_partials(kMaxKeys + 1) <= kCountersOff,
              "the scan's partials must end before the counters");

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

__global__ void k_noalloc_begin(hpic::Counters *cnt, long long n) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cnt->n = n;
    cnt->step = 0;
    cnt->next_id = 0;
    cnt->inj_cnt = 0;
    cnt->flags = 0;
  }
}

__global__ void k_noalloc_end(const hpic::Counters *cnt, long long *n_live) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_live = cnt->n;
}

int noalloc_fail(int code, const char *msg) {
  hpic::set_global_error(msg);
  return code;
}

template <typename R>
hpic::PView<R> view_of(void *const a[8]) {
  hpic::PView<R> v;
  v.x = static_cast<R *>(a[0]);
  v.y = static_cast<R *>(a[1]);
  v.z = static_cast<R *>(a[2]);
  v.ux = static_cast<R *>(a[3]);
  v.uy = static_cast<R *>(a[4]);
  v.uz = static_cast<R *>(a[5]);
  v.tau = static_cast<R *>(a[6]);
  v.id = static_cast<uint32_t *>(a[7]);
  v.w = nullptr;  // weights are not part of this entry point
  return v;
}

}  // namespace

extern "C" int hpic_sort_cells_noalloc(int32_t nx, int32_t ny, int32_t nz, int32_t precision,
                                       int64_t n, const void *const in_soa[8],
                                       void *const out_soa[8], int64_t *n_live_dev, int device,
                                       void *cuda_stream) {
  if (nx < 2 || ny < 2 || nz < 2)
    return noalloc_fail(HPIC_EINVAL, "hpic_sort_cells_noalloc: each dimension must be >= 2");
  if (precision != HPIC_FP64 && precision != HPIC_FP32_MIXED)
    return noalloc_fail(HPIC_EINVAL, "hpic_sort_cells_noalloc: unknown precision");
  if (n < 0 || n > kMaxElectrons)
    return noalloc_fail(HPIC_EINVAL,
                        "hpic_sort_cells_noalloc: more than 1048576 electrons (the fixed scratch limit)");
  const long long nti = (nx + 3) / 4, ntj = (ny + 3) / 4, ntk = (nz + 3) / 4;
  const long long nkeys = nti * ntj * ntk * 64;
  if (nkeys > kMaxKeys)
    return noalloc_fail(HPIC_EINVAL,
                        "hpic_sort_cells_noalloc: more than 1048576 cells after rounding each "
                        "dimension up to a multiple of 4 (the fixed scratch limit)");
  if (!in_soa || !out_soa || !n_live_dev)
    return noalloc_fail(HPIC_EINVAL, "hpic_sort_cells_noalloc: NULL argument");
  for (int a = 0; a < 8; ++a)
    if (n > 0 && (!in_soa[a] || !out_soa[a]))
      return noalloc_fail(HPIC_EINVAL, "hpic_sort_cells_noalloc: NULL array");
  // the scatter reads in_soa while it writes out_soa: no output range may
  // overlap an input range
  if (n > 0) {
    const size_t rb = precision == HPIC_FP32_MIXED ? sizeof(float) : sizeof(double);
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b) {
        const uintptr_t i0 = reinterpret_cast<uintptr_t>(in_soa[a]);
        const uintptr_t o0 = reinterpret_cast<uintptr_t>(out_soa[b]);
        const uintptr_t i1 = i0 + (size_t)n * (a < 7 ? rb : sizeof(uint32_t));
        const uintptr_t o1 = o0 + (size_t)n * (b < 7 ? rb : sizeof(uint32_t));
        if (i0 < o1 && o0 < i1)
          return noalloc_fail(HPIC_EINVAL,
                              "hpic_sort_cells_noalloc: an output array overlaps an input array");
      }
  }
  if (device < 0 || device >= kMaxDevices)
    return noalloc_fail(HPIC_EINVAL, "hpic_sort_cells_noalloc: device index out of range");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return noalloc_fail(HPIC_ECUDA, cudaGetErrorString(e));

  unsigned char *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[device]) {
      // once per device, with that device current
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_sort_scratch);
      if (e != cudaSuccess) return noalloc_fail(HPIC_ECUDA, cudaGetErrorString(e));
      g_scratch_addr[device] = static_cast<unsigned char *>(p);
    }
    scratch = g_scratch_addr[device];
  }
  uint32_t *keys = reinterpret_cast<uint32_t *>(scratch + kKeysOff);
  uint32_t *counts = reinterpret_cast<uint32_t *>(scratch + kCountsOff);
  uint32_t *partials = reinterpret_cast<uint32_t *>(scratch + kPartialsOff);
  hpic::Counters *cnt = reinterpret_cast<hpic::Counters *>(scratch + kCountersOff);

  hpic::Consts K{};
  K.nx = nx;
  K.ny = ny;
  K.nz = nz;
  K.ncell = (long long)nx * ny * nz;
  K.nvec = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  K.nti = (int)nti;
  K.ntj = (int)ntj;
  K.ntk = (int)ntk;
  K.nkeys = nkeys;
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  long long want = (n + 255) / 256;
  const int grid = (int)(want < 1 ? 1 : (want < sms * 8ll ? want : sms * 8ll));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void *const *in = const_cast<void *const *>(in_soa);

  k_noalloc_begin<<<1, 32, 0, st>>>(cnt, n);
  if (precision == HPIC_FP32_MIXED)
    hpic::launch_sort<float>(K, view_of<float>(in), view_of<float>(out_soa), cnt, keys, counts,
                             partials, grid, st, 0.0);
  else
    hpic::launch_sort<double>(K, view_of<double>(in), view_of<double>(out_soa), cnt, keys,
                              counts, partials, grid, st, 0.0);
  k_noalloc_end<<<1, 32, 0, st>>>(cnt, reinterpret_cast<long long *>(n_live_dev));
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(HPIC_ECUDA, cudaGetErrorString(e));
  return HPIC_OK;
}
