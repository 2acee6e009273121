// nb_noalloc.cu -- nb_force_noalloc: a force evaluation that allocates nothing.
//
// The regular entry points work inside a device workspace that the caller
// allocates.  Some callers cannot allocate device memory at the point where
// they need forces -- for example code running inside a host callback or a
// library hook where another framework owns every device allocation, or
// embedded runtimes that forbid cudaMalloc after start-up.  For them this
// entry point takes plain device arrays (positions, velocities, masses,
// target indices, outputs) and keeps everything else it needs -- the packed
// source layout, the i-split partial sums and the plan words -- in one fixed
// device array compiled into the library.
//
// Properties a caller must know:
//   * the array is kNoAllocBytes (6,705,664) bytes, lives on every GPU that loads the
//     library, and is held until the process exits;
//   * at most NB_NOALLOC_MAX_SOURCES sources per call; larger calls are
//     rejected with NB_EINVAL before anything is launched;
//   * every call on a device uses the same array, and a call leaves its
//     contents behind; each call rewrites everything it reads before reading
//     it, but two calls whose kernels overlap on the GPU (different streams
//     without ordering, or different host threads) race on the array;
//   * the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress with that device current) and the SM count; that
//     first call should come before any stream capture on that device.
#include <cmath>
#include <mutex>

#include "../../include/nbody_gb300.h"
#include "nb_integrator.cuh"

namespace nb {
namespace {

constexpr int64_t kNoAllocMaxSources = NB_NOALLOC_MAX_SOURCES;
constexpr int64_t kNoAllocSlots = kNoAllocMaxSources + 4;
constexpr int64_t kNoAllocItems = 320;  // i-split work items with partial sums
constexpr size_t kAlignNA = 256;

constexpr size_t align_up(size_t x) { return (x + kAlignNA - 1) / kAlignNA * kAlignNA; }

// Sub-array offsets inside the fixed array.
constexpr size_t kOffSources = 0;  // mixed float4 groups or FP64 pos+vel (the larger)
constexpr size_t kSourceBytes = align_up(64 * kNoAllocSlots);
constexpr size_t kOffPartials = kOffSources + kSourceBytes;
constexpr size_t kPartialBytes = align_up((size_t)kNoAllocItems * kPartialComps * kMixNI * 8);
constexpr int64_t kNoAllocTiles = (kNoAllocSlots + kMixJT - 1) / kMixJT;
constexpr size_t kOffTiles = kOffPartials + kPartialBytes;
constexpr size_t kTileBytes = align_up(16 * kTileRecF4 * (size_t)kNoAllocTiles);
constexpr size_t kOffSmall = kOffTiles + kTileBytes;
constexpr size_t kSmallBytes = 4096;  // offsets, plan words, status, counters
constexpr size_t kNoAllocBytes = kOffSmall + kSmallBytes;  // 6,705,664 bytes
// the status word of the last call (read back by nb_noalloc_status)
constexpr size_t kOffStatus = kOffSmall + 256 + 12 * sizeof(int32_t);
static_assert(kNoAllocBytes == 6705664, "documented size of the fixed array");

static_assert(64 + wide_counter_entries(kNoAllocItems) <= (kSmallBytes - 256) / 4,
              "the reduction counters fit in the small area");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Per-device set-up results.
constexpr int kMaxDevices = 64;
struct DeviceSetup {
  bool ready = false;
  unsigned char* base = nullptr;
  int sms = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Single-cluster offsets, the identity source order, the zeroed status and
// the zeroed arrival counters of the wide-split reduction (a call whose
// reduction did not finish must not leave them behind for the next one).
__global__ void k_noalloc_setup(int64_t n, int64_t n_pad, int64_t m, int32_t n_tiles,
                                int64_t* off, int64_t* soff, int32_t* act_off, int32_t* toff,
                                uint32_t* status, int32_t* wide_cnt, int64_t n_wide) {
  for (int64_t i = threadIdx.x; i < n_wide; i += blockDim.x) wide_cnt[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    off[0] = 0;
    off[1] = n;
    soff[0] = 0;
    soff[1] = n_pad;
    act_off[0] = 0;
    act_off[1] = static_cast<int32_t>(m);
    toff[0] = 0;
    toff[1] = n_tiles;
    *status = 0u;
  }
}

// FP64 sources straight from the caller's arrays (pads: massless, far away).
__global__ void k_noalloc_pack64(const double* pos, const double* vel, const double* mass,
                                 int64_t n, int64_t n_pad, dbl4* src_pos, dbl4* src_vel) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad;
       s += (int64_t)gridDim.x * blockDim.x) {
    if (s < n) {
      src_pos[s] = dbl4{pos[3 * s], pos[3 * s + 1], pos[3 * s + 2], mass[s]};
      src_vel[s] = dbl4{vel[3 * s], vel[3 * s + 1], vel[3 * s + 2], 0.0};
    } else {
      src_pos[s] = dbl4{kDummyPos, kDummyPos, kDummyPos, 0.0};
      src_vel[s] = dbl4{0.0, 0.0, 0.0, 0.0};
    }
  }
}

// Mixed source tiles (one CTA of kMixJT threads per tile) from the caller's
// arrays, in particle order.
__global__ void __launch_bounds__(kMixJT) k_noalloc_pack_mix(const double* pos, const double* vel,
                                                             const double* mass, int64_t n,
                                                             int64_t n_pad, float4* src,
                                                             float4* tiles) {
  __shared__ float sh[kMixJT / 32];
  const int64_t s = (int64_t)blockIdx.x * kMixJT + threadIdx.x;
  const bool in = s < n_pad, valid = s < n;
  double3 x = make_double3(0.0, 0.0, 0.0), v = make_double3(0.0, 0.0, 0.0);
  double m = 0.0;
  if (valid) {
    x = make_double3(pos[3 * s], pos[3 * s + 1], pos[3 * s + 2]);
    v = make_double3(vel[3 * s], vel[3 * s + 1], vel[3 * s + 2]);
    m = mass[s];
  }
  build_mixed_tile(src, tiles, blockIdx.x, s, in, valid, x, m, v, sh);
}

int setup_device(DeviceSetup** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NB_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return NB_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* p = nullptr;
    // host code must not use g_noalloc_scratch directly: its name here is a
    // host-side shadow, not the device address
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return NB_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return NB_ECUDA;
    if (integrator_setup() != cudaSuccess) return NB_ECUDA;
    s.base = static_cast<unsigned char*>(p);
    s.sms = sms;
    s.ready = true;
  }
  *out = &s;
  return NB_OK;
}

}  // namespace
}  // namespace nb

using namespace nb;

extern "C" int nb_force_noalloc(const double* pos, const double* vel, const double* mass,
                                int64_t n, const int32_t* target_idx, int64_t m, double G,
                                double eps, int32_t precision, double* acc, double* jerk,
                                double* pot, void* stream) {
  if (n < 1 || n > kNoAllocMaxSources || m < 0 || m > n) return NB_EINVAL;
  if (precision != NB_MIXED && precision != NB_FP64) return NB_EINVAL;
  if (!(eps >= 0.0) || !std::isfinite(eps) || !std::isfinite(G)) return NB_EINVAL;
  if (!pos || !vel || !mass) return NB_EINVAL;
  if (m == 0) return NB_OK;
  if (!target_idx || !acc || !jerk) return NB_EINVAL;
  DeviceSetup* ds = nullptr;
  const int rc = setup_device(&ds);
  if (rc != NB_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool f64 = precision == NB_FP64;
  const int64_t n_pad = round_up64(n, 4);

  unsigned char* base = ds->base;
  int64_t* small64 = reinterpret_cast<int64_t*>(base + kOffSmall);
  int32_t* small32 = reinterpret_cast<int32_t*>(base + kOffSmall + 256);
  Dev d;
  d.N = n;
  d.S = n_pad;
  d.K = 1;
  d.off = small64;           // 2 entries
  d.soff = small64 + 2;      // 2 entries
  d.t_cur = small64 + 4;     // unused by a plan outside a block step
  d.t_min = small64 + 5;
  d.counters = reinterpret_cast<unsigned long long*>(small64 + 8);  // 4 entries
  d.act_off = small32;       // 2 entries
  d.item_off = small32 + 4;  // 2 entries
  d.bfac = small32 + 8;      // 1 entry
  d.status = reinterpret_cast<uint32_t*>(base + kOffStatus);  // small32 + 12
  d.src_mix = reinterpret_cast<float4*>(base + kOffSources);
  d.src64_pos = reinterpret_cast<dbl4*>(base + kOffSources);
  d.src64_vel = reinterpret_cast<dbl4*>(base + kOffSources + 32 * kNoAllocSlots);
  d.partials = reinterpret_cast<double*>(base + kOffPartials);
  d.part_items = kNoAllocItems;
  d.tiles = reinterpret_cast<float4*>(base + kOffTiles);
  d.toff = small32 + 16;     // 2 entries
  d.wt_off = small32 + 20;   // 2 entries
  d.work_ctr = small32 + 24; // the force kernel's dynamic item counter (zeroed by the plan)
  d.wide_cnt = small32 + 64; // wide_counter_entries(kNoAllocItems), zeroed by the set-up
  const int32_t n_tiles = static_cast<int32_t>((n_pad + kMixJT - 1) / kMixJT);

  k_noalloc_setup<<<1, 256, 0, st>>>(n, n_pad, m, n_tiles, d.off, d.soff, d.act_off, d.toff,
                                     d.status, d.wide_cnt, wide_counter_entries(kNoAllocItems));
  if (f64)
    k_noalloc_pack64<<<static_cast<int>((n_pad + 255) / 256), 256, 0, st>>>(
        pos, vel, mass, n, n_pad, d.src64_pos, d.src64_vel);
  else
    k_noalloc_pack_mix<<<n_tiles, kMixJT, 0, st>>>(pos, vel, mass, n, n_pad, d.src_mix,
                                                   d.tiles);
  if (cudaGetLastError() != cudaSuccess) return NB_ECUDA;

  const int grid = ds->sms * (f64 ? force_fp64_ctas_per_sm() : force_mixed_ctas_per_sm(kMixDefaultVariant));
  PlanArgs p{};
  p.NI = f64 ? kF64NI : force_mixed_ni(kMixDefaultVariant);
  p.JT = f64 ? kF64JT : kMixJT;
  p.grid = grid;
  p.forced_b = 0;
  p.part_items = kNoAllocItems;
  p.step_mode = 0;
  p.count = 0;
  if (launch_plan(d, p, st) != cudaSuccess) return NB_ECUDA;

  ForceArgs a{};
  a.off = d.off;
  a.soff = d.soff;
  a.active = target_idx;
  a.act_off = d.act_off;
  a.item_off = d.item_off;
  a.wt_off = d.wt_off;
  a.wide_cnt = d.wide_cnt;
  a.bfac = d.bfac;
  a.sinv = nullptr;  // sources in particle order
  a.tiles = d.tiles;
  a.toff = d.toff;
  a.rows = nullptr;
  a.tile_counts = nullptr;
  a.K = 1;
  a.src_a = f64 ? static_cast<const void*>(d.src64_pos) : static_cast<const void*>(d.src_mix);
  a.src_b = f64 ? d.src64_vel : nullptr;
  a.out_acc = acc;
  a.sa = 3;
  a.out_jerk = jerk;
  a.sj = 3;
  a.out_pot = pot;
  a.sp = 1;
  a.partials = d.partials;
  a.G = G;
  a.eps2 = eps * eps;
  a.status = d.status;
  a.work_ctr = d.work_ctr;
  cudaError_t e = f64 ? launch_force_fp64(a, grid, kF64Full, st)
                      : launch_force_mixed(a, grid, pot != nullptr, kMixDefaultVariant, st);
  if (e != cudaSuccess) return NB_ECUDA;
  if (launch_reduce(a, p.NI, true, m, ds->sms, st) != cudaSuccess) return NB_ECUDA;
  return NB_OK;
}

extern "C" int nb_noalloc_status(void* stream) {
  DeviceSetup* ds = nullptr;
  const int rc = setup_device(&ds);
  if (rc != NB_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t s = 0;
  const void* word = ds->base + kOffStatus;
  if (cudaMemcpyAsync(&s, word, sizeof s, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return NB_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return NB_ECUDA;
  if (s & kStatusTimeout) return NB_ETIMEOUT;
  if (s & kStatusNonFinite) return NB_ENONFINITE;
  if (s & kStatusInval) return NB_EINVAL;
  return NB_OK;
}
