// md_potential_noalloc: the potential energy of a state in caller-owned device
// memory, computed without allocating anything.
//
// Some callers cannot allocate device memory: a host framework whose caching
// allocator has reserved (almost) all of the GPU's memory, so that a fresh
// cudaMalloc fails or fragments its pool; or a latency-critical loop in which
// cudaMalloc / cudaFree, which can synchronise the device, are not acceptable.
// For them this entry point takes its scratch memory (per-tile partial sums,
// half-angle table, per-CTA partials, completion ticket) from one file-scope
// device array that every GPU loading the library holds until the process
// exits.  The kernels are those of md_energy, with the same summation order.
#include <mutex>

#include "md_internal.cuh"

namespace {

constexpr int64_t kMaxN = 65536;                     // largest N the scratch holds
constexpr int kTile = 256;                           // potential tile (particles per side)
constexpr int64_t kMaxTiles = kMaxN / kTile;         // 256
constexpr int kMaxCtas = 2048;                       // cap on reduction CTAs
constexpr size_t kUnitSums = kMaxTiles * kMaxTiles;  // doubles
constexpr size_t kHalfAngles = 2 * kMaxN;            // doubles (N double2)
constexpr size_t kPartials = 2 * kMaxCtas;           // doubles
constexpr size_t kSums = 8;                          // doubles
constexpr size_t kTicket = 8;                        // doubles' worth, holds an unsigned
constexpr size_t kScratchDoubles = kUnitSums + kHalfAngles + kPartials + kSums + kTicket;  // 1.6 MB

// The scratch.  Host code must not pass this name to a kernel: on the host it is
// a stand-in, not a device address; the address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};
int g_nsm[kMaxDevices] = {};
// Completion of the last call queued on each device: every call waits for it on its
// own stream before touching the scratch, so calls on different streams or from
// different threads run one after another on the GPU (an event holds no device memory).
cudaEvent_t g_done[kMaxDevices] = {};

// Once per device, with that device current: the scratch's device address and the
// ordering event.  The caller holds g_mu.
int setup(int dev, double **addr, int *nsm) {
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_err(nullptr, MD_ECUDA, "md_potential_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return MD_ECUDA;
    }
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      set_err(nullptr, MD_ECUDA, "md_potential_noalloc: device attribute: %s", cudaGetErrorString(e));
      return MD_ECUDA;
    }
    e = cudaEventCreateWithFlags(&g_done[dev], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      set_err(nullptr, MD_ECUDA, "md_potential_noalloc: event: %s", cudaGetErrorString(e));
      return MD_ECUDA;
    }
    g_addr[dev] = (double *)p;
    g_nsm[dev] = n;
  }
  *addr = g_addr[dev];
  *nsm = g_nsm[dev];
  return MD_OK;
}

}  // namespace

extern "C" int md_potential_noalloc(int model, int64_t N, double eps, const double *q, double *V, void *stream) {
  if (model != MD_HMF && model != MD_RING && model != MD_GRAV2D && model != MD_GRAV3D && model != MD_SHEET1D)
    return set_err(nullptr, MD_EINVAL, "md_potential_noalloc: unknown model %d", model);
  if (N < 1 || N > kMaxN)
    return set_err(nullptr, MD_EINVAL,
                   "md_potential_noalloc: N = %lld is outside [1, %lld], the size its static scratch holds",
                   (long long)N, (long long)kMaxN);
  if (!eps_valid(model, eps))
    return set_err(nullptr, MD_EINVAL, "md_potential_noalloc: bad eps %g (finite; 0 only for HMF and sheets, else >= %g)",
                   eps, kEpsMin);
  if (!q || !V) return set_err(nullptr, MD_EINVAL, "md_potential_noalloc: NULL pointer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_err(nullptr, MD_ECUDA, "md_potential_noalloc: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_err(nullptr, MD_EINVAL, "md_potential_noalloc: device %d", dev);
  // the scratch address and the ordering event belong to the current device, so the
  // stream must be one of its streams
  int sdev = dev;
  e = cudaStreamGetDevice((cudaStream_t)stream, &sdev);
  if (e != cudaSuccess) return set_err(nullptr, MD_ECUDA, "md_potential_noalloc: stream device: %s", cudaGetErrorString(e));
  if (sdev != dev)
    return set_err(nullptr, MD_EINVAL, "md_potential_noalloc: the stream belongs to device %d, the current device is %d",
                   sdev, dev);
  double *base = nullptr;
  int nsm = 0;
  std::lock_guard<std::mutex> lk(g_mu);  // one call enqueues at a time, in host order
  int rc = setup(dev, &base, &nsm);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // Under stream capture an event recorded outside it cannot be waited on: the
  // captured graph's own order is the caller's to keep.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return set_err(nullptr, MD_ECUDA, "md_potential_noalloc: %s", cudaGetErrorString(e));
  const bool ordered = cap == cudaStreamCaptureStatusNone;
  if (ordered && (e = cudaStreamWaitEvent(st, g_done[dev], 0)) != cudaSuccess)
    return set_err(nullptr, MD_ECUDA, "md_potential_noalloc: wait: %s", cudaGetErrorString(e));
  double *unit_sums = base;
  double2 *ag = (double2 *)(base + kUnitSums);
  double *partials = base + kUnitSums + kHalfAngles;
  double *sums = partials + kPartials;
  unsigned *ticket = (unsigned *)(sums + kSums);
  // the array keeps the previous call's contents: clear what must start at zero
  const int64_t ntiles = (N + kTile - 1) / kTile;
  e = cudaMemsetAsync(ticket, 0, sizeof(double) * kTicket, st);
  if (e == cudaSuccess && model != MD_HMF)
    e = cudaMemsetAsync(unit_sums, 0, sizeof(double) * (size_t)(ntiles * ntiles), st);
  if (e != cudaSuccess) return set_err(nullptr, MD_ECUDA, "md_potential_noalloc: memset: %s", cudaGetErrorString(e));
  rc = potential_with_scratch(st, nsm, kMaxCtas, model, N, eps, q, unit_sums, ag, partials, sums, ticket, V);
  if (rc) return set_err(nullptr, rc, "md_potential_noalloc: launch: %s", cudaGetErrorString(cudaGetLastError()));
  if (ordered && (e = cudaEventRecord(g_done[dev], st)) != cudaSuccess)
    return set_err(nullptr, MD_ECUDA, "md_potential_noalloc: record: %s", cudaGetErrorString(e));
  return MD_OK;
}
