// nb_integrator.cu -- block-time-step machinery around the force kernels.
//
// One block step (Sec. 2 items 1 and 2) is a fixed sequence of seven launches
// whose sizes all live on the device, so it can be captured in a CUDA graph:
//   k_tmin       t_next(k) = min_i (t_i + dt_i) per cluster        (O(N))
//   k_predict    Taylor predictor of EVERY particle to t_next, written
//                as the source arrays; counts due particles per tile (O(N))
//   k_scan_plan  exclusive scan of the per-tile counts, each cluster's
//                offset in the active list, and the plan: per-cluster
//                i-split factor B_k and work-item offsets (one CTA)
//   k_scatter    active list {i : t_i + dt_i = t_next}, ascending (O(N))
//   force        (nb_force_mixed.cu / nb_force_fp64.cu)          O(m N)
//   k_reduce     fixed-order sum of the B_k partials per target
//   k_correct    Hermite corrector, step criterion, power-of-two level (O(m))
// A force evaluation on a caller's list (nb_force) uses k_scan and k_plan
// on their own.
#include <cfloat>
#include <climits>

#include <math_constants.h>

#include "nb_integrator.cuh"

namespace nb {
namespace {

__device__ __forceinline__ int64_t step_ticks(int32_t level, int T) {
  return (int64_t)1 << (T - level);
}

// Taylor predictor of the Hermite scheme: x + v t + a t^2/2 + j t^3/6 and
// v + a t + j t^2/2 (Horner form).
__device__ __forceinline__ void predict1(const dbl4& p, const dbl4& v, const dbl4& a,
                                         const dbl4& j, double t, double3& xp, double3& vp) {
  const double h = 0.5 * t, s = t * (1.0 / 3.0);
  xp.x = p.x + t * (v.x + h * (a.x + s * j.x));
  xp.y = p.y + t * (v.y + h * (a.y + s * j.y));
  xp.z = p.z + t * (v.z + h * (a.z + s * j.z));
  vp.x = v.x + t * (a.x + h * j.x);
  vp.y = v.y + t * (a.y + h * j.y);
  vp.z = v.z + t * (a.z + h * j.z);
}

// Taylor predictor of the 6th-order scheme (Horner form): x + v t + a t^2/2
// + j t^3/6 + s t^4/24 + c t^5/120, its velocity and its acceleration
// a + j t + s t^2/2 + c t^3/6 (the sources' accelerations of the snap term).
__device__ __forceinline__ void predict6(const dbl4& p, const dbl4& v, const dbl4& a,
                                         const dbl4& j, const dbl4& sn, const dbl4& cr, double t,
                                         double3& xp, double3& vp, double3& ap) {
  const double h = 0.5 * t, t3 = t * (1.0 / 3.0), t4 = 0.25 * t, t5 = 0.2 * t;
  xp.x = p.x + t * (v.x + h * (a.x + t3 * (j.x + t4 * (sn.x + t5 * cr.x))));
  xp.y = p.y + t * (v.y + h * (a.y + t3 * (j.y + t4 * (sn.y + t5 * cr.y))));
  xp.z = p.z + t * (v.z + h * (a.z + t3 * (j.z + t4 * (sn.z + t5 * cr.z))));
  vp.x = v.x + t * (a.x + h * (j.x + t3 * (sn.x + t4 * cr.x)));
  vp.y = v.y + t * (a.y + h * (j.y + t3 * (sn.y + t4 * cr.y)));
  vp.z = v.z + t * (a.z + h * (j.z + t3 * (sn.z + t4 * cr.z)));
  ap.x = a.x + t * (j.x + h * (sn.x + t3 * cr.x));
  ap.y = a.y + t * (j.y + h * (sn.y + t3 * cr.y));
  ap.z = a.z + t * (j.z + h * (sn.z + t3 * cr.z));
}

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T* sh, T ident) {
  // blockDim.x a multiple of 32, <= 1024
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (wid == 0) {
    v = lane < nw ? sh[lane] : ident;
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) sh[0] = v;
  }
  __syncthreads();
  T r = sh[0];
  __syncthreads();
  return r;
}

// inclusive warp scan
__device__ __forceinline__ int32_t warp_incl_scan(int32_t v) {
  const int lane = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// exclusive block scan (blockDim.x <= 1024); returns the block total in *total
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* sh, int32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int32_t inc = warp_incl_scan(v);
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int32_t x = lane < nw ? sh[lane] : 0;
    x = warp_incl_scan(x);
    sh[lane] = x;  // inclusive warp totals
  }
  __syncthreads();
  const int32_t base = wid > 0 ? sh[wid - 1] : 0;
  *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + inc - v;
}

// ----------------------------------------------------------------- kernels

__global__ void k_fill_i64(int64_t* p, int64_t n, int64_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// Next block time of every cluster whose time is below the end time.
__global__ void k_tmin(Dev d, int T) {
  pdl_wait();  // the previous kernel of the chain has completed
  pdl_launch();
  __shared__ long long sh[32];
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x;
  const int64_t i = i0 + threadIdx.x;
  const int64_t t_end = *d.t_end;
  int64_t due = LLONG_MAX;
  int32_t c = -1;
  if (i < d.N) {
    c = d.cid[i];
    if (d.t_cur[c] < t_end) due = d.t[i] + step_ticks(d.level[i], T);
  }
  // whole block inside one cluster: block min + one atomic
  const int64_t ilast = min(i0 + (int64_t)blockDim.x, d.N) - 1;
  const int32_t c0 = d.cid[i0], c1 = d.cid[ilast];
  if (c0 == c1) {
    const long long mn = block_reduce<long long>(
        (long long)due, [](long long x, long long y) { return x < y ? x : y; }, sh, LLONG_MAX);
    if (threadIdx.x == 0 && mn != LLONG_MAX)
      atomicMin(reinterpret_cast<long long*>(d.t_min + c0), mn);
  } else if (due != LLONG_MAX) {
    atomicMin(reinterpret_cast<long long*>(d.t_min + c), (long long)due);
  }
}

// In-place exclusive scan of the n counts cnt[0 .. n) by one CTA of
// blockDim.x <= kScanThreads threads; returns the total (in every thread).
// Chunks of kScanPerThread counts per thread are staged in shared memory by
// coalesced loads; each thread sums its consecutive counts, one block scan
// gives its offset, and it writes its counts' prefixes back: one block scan
// per chunk of blockDim.x * kScanPerThread counts instead of one per
// blockDim.x.
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 8;
__device__ __forceinline__ int32_t scan_counts(int32_t* cnt, int32_t n, int32_t* sh,
                                               int32_t* chunk) {
  const int32_t per = blockDim.x * kScanPerThread;
  const int32_t b0 = threadIdx.x * kScanPerThread;
  int32_t carry = 0;
  for (int32_t c0 = 0; c0 < n; c0 += per) {
    const int32_t len = min(per, n - c0);
    for (int32_t q = threadIdx.x; q < len; q += blockDim.x) chunk[q] = cnt[c0 + q];
    __syncthreads();
    int32_t local = 0;
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) local += b0 + q < len ? chunk[b0 + q] : 0;
    int32_t tot;
    int32_t run = carry + block_excl_scan(local, sh, &tot);
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
      if (b0 + q < len) {
        const int32_t v = chunk[b0 + q];
        chunk[b0 + q] = run;
        run += v;
      }
    }
    __syncthreads();
    for (int32_t q = threadIdx.x; q < len; q += blockDim.x) cnt[c0 + q] = chunk[q];
    carry += tot;
    __syncthreads();  // the chunk buffer is refilled next
  }
  return carry;
}

// Exclusive scan of nblk block counts (one CTA of 1024 threads); the total
// goes to act_off[K].
__global__ void __launch_bounds__(kScanThreads) k_scan(Dev d, int32_t nblk) {
  __shared__ int32_t sh[32];
  __shared__ int32_t chunk[kScanThreads * kScanPerThread];
  const int32_t total = scan_counts(d.blk_count, nblk, sh, chunk);
  if (threadIdx.x == 0) d.act_off[d.K] = total;
}

// Predict the particles of one source tile (one CTA of kMixJT threads, one
// slot per thread) to the target time of their cluster (t_tgt[k], or t_fixed
// when t_tgt is null; a cluster whose target is LLONG_MAX is skipped) and
// write them in the force kernels' layouts: FP64 sources, and/or the mixed
// tile (centre, radius, double-single offsets).  With count_due, also count
// the tile's particles due at the target time.
__global__ void __launch_bounds__(kMixJT) k_predict_tiles(Dev d, const int64_t* t_tgt,
                                                          int64_t t_fixed, int T, int write_mix,
                                                          int write64, int count_due,
                                                          int zero_tau) {
  pdl_wait();  // the previous kernel of the chain has completed
  pdl_launch();
  __shared__ float shd[kMixJT / 32];
  __shared__ int32_t shi[32];
  const int32_t tile = blockIdx.x;
  const int32_t k = upper_bound_i32(d.toff, d.K + 1, tile) - 1;
  const int64_t s = d.soff[k] + (int64_t)(tile - d.toff[k]) * kMixJT + threadIdx.x;
  const bool in = s < d.soff[k + 1];
  const int32_t p = in ? d.sperm[s] : -1;
  const int64_t tn = t_tgt ? t_tgt[k] : t_fixed;
  if (tn == LLONG_MAX) {  // uniform over the CTA: the whole tile is one cluster
    if (count_due) {
      if (threadIdx.x == 0) d.blk_count[tile] = 0;
      if ((threadIdx.x & 31) == 0) d.due_mask[tile * (kMixJT / 32) + (threadIdx.x >> 5)] = 0u;
    }
    return;
  }
  int32_t due = 0;
  double3 xp = make_double3(0.0, 0.0, 0.0), vp = make_double3(0.0, 0.0, 0.0);
  double3 ap = make_double3(0.0, 0.0, 0.0);
  double m = 0.0;
  const bool o6 = d.order == 6;
  if (p >= 0) {
    const int64_t ti = d.t[p];
    due = (count_due && ti + step_ticks(d.level[p], T) == tn) ? 1 : 0;
    const double tau = zero_tau ? 0.0 : ldexp((double)(tn - ti), -T);
    const dbl4 P = d.pos[p], V = d.vel[p], A = d.acc[p], J = d.jerk[p];
    if (o6)
      predict6(P, V, A, J, d.snap[p], d.crackle[p], tau, xp, vp, ap);
    else
      predict1(P, V, A, J, tau, xp, vp);
    m = P.w;
  }
  if (count_due) {
    // the due slots as one bit per lane and warp, for k_scatter_tiles
    const uint32_t bal = __ballot_sync(0xffffffffu, due != 0);
    if ((threadIdx.x & 31) == 0) d.due_mask[tile * (kMixJT / 32) + (threadIdx.x >> 5)] = bal;
    const int32_t tot =
        block_reduce<int32_t>(due, [](int32_t x, int32_t y) { return x + y; }, shi, 0);
    if (threadIdx.x == 0) d.blk_count[tile] = tot;
  }
  if (write64 && in) {
    if (p >= 0) {
      d.src64_pos[s] = dbl4{xp.x, xp.y, xp.z, m};
      d.src64_vel[s] = dbl4{vp.x, vp.y, vp.z, 0.0};
    } else {
      d.src64_pos[s] = dbl4{kDummyPos, kDummyPos, kDummyPos, 0.0};
      d.src64_vel[s] = dbl4{0.0, 0.0, 0.0, 0.0};
    }
    if (o6) d.src64_acc[s] = dbl4{ap.x, ap.y, ap.z, 0.0};  // pads: zero
  }
  if (o6 && write_mix && in) {  // [ax][ay][az] float4 groups of 4 slots
    float* g = reinterpret_cast<float*>(d.src_acc_mix + (s >> 2) * 3) + (s & 3);
    g[0] = __double2float_rn(ap.x);
    g[4] = __double2float_rn(ap.y);
    g[8] = __double2float_rn(ap.z);
  }
  if (write_mix) build_mixed_tile(d.src_mix, d.tiles, tile, s, in, p >= 0, xp, m, vp, shd);
}

// Active list in source-slot order (spatially sorted targets), from the
// predictor's due bits and the scanned per-tile counts.
constexpr int kScatterThreads = 256;
__global__ void __launch_bounds__(kScatterThreads) k_scatter_tiles(Dev d, int T) {
  pdl_wait();  // the previous kernel of the chain has completed
  pdl_launch();
  (void)T;
  // one warp per word of the predictor's due bits (a tile has kMixJT / 32),
  // a grid of a few CTAs per SM striding over them (a CTA per tile spends
  // more on launching CTAs than on the work when few particles are due): a
  // slot's place in the active list is its tile's offset (the scan) plus the
  // due slots before it in the tile (population counts).  Words without due
  // slots cost one load; the particle map is read for due slots only.  (Each
  // cluster's offset in the list, act_off[k], was set by the scan.)
  constexpr int kWords = kMixJT / 32;
  const int lane = threadIdx.x & 31;
  const int64_t nw = d.n_tiles * kWords;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < nw;
       gw += stride) {
    const uint32_t mine = d.due_mask[gw];
    if (!((mine >> lane) & 1u)) continue;
    const int32_t tile = static_cast<int32_t>(gw / kWords);
    const int w = static_cast<int>(gw - (int64_t)tile * kWords);
    int32_t before = 0;
    for (int q = 0; q < w; ++q) before += __popc(d.due_mask[(int64_t)tile * kWords + q]);
    const int32_t ex = before + __popc(mine & ((1u << lane) - 1u));
    const int32_t k = upper_bound_i32(d.toff, d.K + 1, tile) - 1;
    const int64_t slot = d.soff[k] + (int64_t)(tile - d.toff[k]) * kMixJT + w * 32 + lane;
    d.active[d.blk_count[tile] + ex] = d.sperm[slot];
  }
}

// Work plan: per-cluster active count m_k, i-split factor B_k (Sec. 2 item 3)
// and work-item offsets.  One CTA (every thread calls it).  In step mode the
// cluster's new block time t_min[k] becomes t_cur[k]; t_min itself is reset
// here (reset_tmin) or, when the active list is still to be built from it,
// by the step's corrector.
__device__ __forceinline__ void plan_body(const Dev& d, const PlanArgs& p0, bool reset_tmin) {
  __shared__ unsigned long long shu[32];
  __shared__ int32_t shi[32];
  __shared__ int32_t bg_sh;
  __shared__ int32_t var_sh;
  const int32_t K = d.K;
  PlanArgs p = p0;
  if (p0.use_table) {
    // the shape and split of the autotune table for ceil(log2 m) of the
    // step's active count (the list is complete: act_off is final here)
    if (threadIdx.x == 0) {
      const int32_t m = d.act_off[K] - d.act_off[0];
      const int b = m <= 1 ? 0 : min(kTuneBuckets - 1, 32 - __clz(m - 1));
      const int v = d.tune[2 * b];
      var_sh = v;
      bg_sh = d.tune[2 * b + 1];
      d.sel[0] = v;
      d.sel[1] = p0.ni_v[v];
    }
    __syncthreads();
    p.NI = p0.ni_v[var_sh];
    p.grid = p0.grid_v[var_sh];
    p.forced_b = p0.forced_b > 0 ? p0.forced_b : bg_sh;  // a configured B wins
    __syncthreads();  // bg_sh is rewritten below
  }
  // the force kernel's dynamic item counter starts from zero every launch
  if (threadIdx.x == 0 && d.work_ctr) *d.work_ctr = 0;
  unsigned long long nit = 0, inter = 0;
  for (int32_t k = threadIdx.x; k < K; k += blockDim.x) {
    const int64_t mk = d.act_off[k + 1] - d.act_off[k];
    nit += (unsigned long long)ceil_div64(mk, p.NI);
    int64_t nk = d.off[k + 1] - d.off[k];
    if (p.parts > 1) {  // the real particles of the piece (pad slots at the end)
      int64_t pb, pe;
      src_piece(d.soff[k + 1] - d.soff[k], p.part, p.parts, &pb, &pe);
      nk = min(pe, nk) - min(pb, nk);
    }
    inter += (unsigned long long)mk * (unsigned long long)nk;
  }
  auto add = [](unsigned long long x, unsigned long long y) { return x + y; };
  nit = block_reduce<unsigned long long>(nit, add, shu, 0ull);
  inter = block_reduce<unsigned long long>(inter, add, shu, 0ull);
  if (threadIdx.x == 0) {
    int64_t bg = 1;
    if (nit > 0) {
      if (p.forced_b > 0) {
        bg = p.forced_b;
      } else {
        // fill the persistent grid, then pick the split whose last round of
        // work items is fullest: a few candidates above the fill point (the
        // per-cluster clamp below bounds B by the cluster's tile count), in
        // 32-bit integers and FP32, since one thread's FP64 division costs
        // microseconds on this part.  n b = (q g + r) b items take
        // q b + ceil(r b / g) rounds, and r b < 10 g fits 32 bits.
        const uint32_t g = static_cast<uint32_t>(p.grid);
        const uint32_t n = nit > (1ull << 30) ? (1u << 30) : static_cast<uint32_t>(nit);
        const uint32_t b0 = n >= g ? 1u : (g + n - 1) / n;
        const uint32_t q = n / g, r = n - q * g;
        float best = -1.f;
        for (uint32_t b = b0; b <= b0 + 8; ++b) {
          const uint32_t rounds = q * b + (r * b + g - 1) / g;
          const float e = __fdiv_rn((float)n * (float)b, (float)rounds * (float)g);
          if (e > best + 1e-3f) { best = e; bg = b; }
        }
        // at least kItemsPerCta items per CTA, so that the dynamic item order
        // can even out CTAs that run at different speeds
        const uint32_t bmin = (kItemsPerCta * g + n - 1) / n;
        if (bg < (int64_t)bmin) bg = bmin;
      }
      const int64_t cap = max((int64_t)1, p.part_items / (int64_t)nit);
      if (bg > cap) bg = cap;
    }
    bg_sh = static_cast<int32_t>(bg);
    if (p.count) {
      atomicAdd(d.counters + 0, inter);
      if (p.step_mode) atomicAdd(d.counters + 1, 1ull);
    }
  }
  __syncthreads();
  const int32_t bg = bg_sh;
  int32_t carry = 0, wcarry = 0;
  for (int32_t k0 = 0; k0 < K; k0 += blockDim.x) {
    const int32_t k = k0 + threadIdx.x;
    int32_t items = 0, wide = 0;
    if (k < K) {
      const int64_t mk = d.act_off[k + 1] - d.act_off[k];
      int64_t Sk = d.soff[k + 1] - d.soff[k];
      if (p.parts > 1) {  // B splits this process's piece of the sources
        int64_t pb, pe;
        src_piece(Sk, p.part, p.parts, &pb, &pe);
        Sk = pe - pb;
      }
      int64_t B = min((int64_t)bg, ceil_div64(Sk, p.JT));
      if (B < 1) B = 1;
      // every chunk non-empty (an empty piece: one empty chunk, zero sums)
      if (Sk > 0) B = ceil_div64(Sk, chunk_len(Sk, B, p.JT));
      d.bfac[k] = static_cast<int32_t>(B);
      items = static_cast<int32_t>(ceil_div64(mk, p.NI) * B);
      if (B > kReduceSerial)  // (i-tile, row segment) units of k_reduce
        wide = static_cast<int32_t>(ceil_div64(mk, p.NI) * ceil_div64(B, kWideRows));
      if (p.step_mode) {
        const int64_t tn = d.t_min[k];
        if (tn != LLONG_MAX) d.t_cur[k] = tn;
        if (reset_tmin) d.t_min[k] = LLONG_MAX;
      }
    }
    int32_t tot, wtot;
    const int32_t ex = block_excl_scan(items, shi, &tot);
    const int32_t wex = block_excl_scan(wide, shi, &wtot);
    if (k < K) {
      d.item_off[k] = carry + ex;
      d.wt_off[k] = wcarry + wex;
    }
    carry += tot;
    wcarry += wtot;
  }
  if (threadIdx.x == 0) {
    d.item_off[K] = carry;
    d.wt_off[K] = wcarry;
  }
}

__global__ void k_plan(Dev d, PlanArgs p) {
  pdl_wait();  // the previous kernel of the chain has completed
  pdl_launch();
  plan_body(d, p, true);
}

// Block step: the scan of the per-tile due counts (k_scan), each cluster's
// offset in the active list (the scanned count of its first tile) and the
// plan, in one CTA of 1024 threads.  t_min stays for k_scatter_tiles; the
// corrector resets it.
__global__ void __launch_bounds__(kScanThreads) k_scan_plan(Dev d, int32_t nblk, PlanArgs p) {
  pdl_wait();  // the previous kernel of the chain has completed
  pdl_launch();
  __shared__ int32_t sh[32];
  __shared__ int32_t chunk[kScanThreads * kScanPerThread];
  const int32_t total = scan_counts(d.blk_count, nblk, sh, chunk);
  if (threadIdx.x == 0) d.act_off[d.K] = total;
  __syncthreads();
  for (int32_t k = threadIdx.x; k < d.K; k += blockDim.x) d.act_off[k] = d.blk_count[d.toff[k]];
  __syncthreads();
  plan_body(d, p, false);
}

// Fixed-order sum of the B_k partials of every target whose cluster was
// split (Sec. 2 item 3); the order depends on B_k alone.
//   1 < B_k <= kReduceSerial: each lane owns one target and sums
//     b = 0 .. B_k - 1 in order (the lanes of a warp read consecutive targets
//     of one partial row).
//   B_k > kReduceSerial (few active targets split over many
//     source chunks): the partial rows of an i-tile are cut into segments of
//     kWideRows rows; one CTA of kWideRows warps takes one segment of one
//     block of 32 targets, warp r holding row r, and combines the rows in
//     pairs (r, r + o) for o = 16, 8, 4, 2, 1.  With one segment that is the
//     result; otherwise the CTA writes its segment sum over the segment's
//     first row, and the last CTA of the block (arrival counter) adds the
//     segment sums in segment order.  GB300 runs FP64 at ~2 lanes per SM per
//     clock, so the segments spread the additions over many SMs.
// C partial components per target: 7 (acceleration, jerk, potential) or 10
// (and snap, for the 6th-order force).
template <int C>
__device__ __forceinline__ void write_reduced(const ForceArgs& a, int32_t s, const double* v,
                                              int with_acc) {
  const int64_t row = a.rows ? (int64_t)a.rows[s] : (int64_t)s;
  if (with_acc) {
    if (a.out_acc) for (int c = 0; c < 3; ++c) a.out_acc[row * a.sa + c] = a.G * v[c];
    if (a.out_jerk) for (int c = 0; c < 3; ++c) a.out_jerk[row * a.sj + c] = a.G * v[3 + c];
    if (C > kPartialComps && a.out_snap)
      for (int c = 0; c < 3; ++c) a.out_snap[row * a.ss + c] = a.G * v[kPartialComps + c];
  }
  if (a.out_pot) a.out_pot[row * a.sp] = a.G * v[6];
}

constexpr size_t kWideSmem = sizeof(double) * kPartialCompsSnap * kWideRows * 32;

template <int C>
__global__ void __launch_bounds__(32 * kWideRows) k_reduce(ForceArgs a, int NI,
                                                           int with_acc) {
  pdl_wait();  // the previous kernel of the chain has completed
  pdl_launch();
  extern __shared__ double red[];  // [component][row r][lane]
  __shared__ int last_sh;
  const int32_t K = a.K;
  if (a.sel) NI = a.sel[1];  // the shape the plan chose (block steps with a table)
  // small splits: one lane per target
  const int32_t m = a.act_off[K];
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < m; s += gridDim.x * blockDim.x) {
    const int32_t k = upper_bound_i32(a.act_off, K + 1, s) - 1;
    const int32_t B = a.bfac[k];
    if (B <= 1 || B > kReduceSerial) continue;
    const int32_t local = s - a.act_off[k];
    const int32_t it = local / NI;
    const int32_t q = local - it * NI;
    const int32_t w0 = a.item_off[k] + it * B;
    double v[C];
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = 0.0;
    for (int32_t b = 0; b < B; ++b) {
      const double* P = a.partials + (size_t)(w0 + b) * C * NI + q;
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] += P[(size_t)c * NI];
    }
    write_reduced<C>(a, s, v, with_acc);
  }
  // large splits: (i-tile, row segment, block of 32 targets) units
  const int32_t cbs = NI / 32;
  const int32_t units = a.wt_off[K] * cbs;
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5;
  for (int32_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int32_t ws = u / cbs;             // (i-tile, segment) unit
    const int32_t cb = u - ws * cbs;        // block of 32 targets
    const int32_t k = upper_bound_i32(a.wt_off, K + 1, ws) - 1;
    const int32_t B = a.bfac[k];
    const int32_t nseg = (B + kWideRows - 1) / kWideRows;
    const int32_t lw = ws - a.wt_off[k];
    const int32_t it = lw / nseg;
    const int32_t g = lw - it * nseg;
    const int32_t m_k = a.act_off[k + 1] - a.act_off[k];
    const int32_t q = cb * 32 + lane;
    const int32_t local = it * NI + q;
    const bool valid = local < m_k;
    const int32_t w0 = a.item_off[k] + it * B;
    const int32_t b = g * kWideRows + r;
    double v[C];
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = 0.0;
    if (valid && b < B) {
      const double* P = a.partials + (size_t)(w0 + b) * C * NI + q;
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = P[(size_t)c * NI];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) red[(c * kWideRows + r) * 32 + lane] = v[c];
    __syncthreads();
    for (int o = kWideRows / 2; o > 0; o >>= 1) {
      if (r < o) {
#pragma unroll
        for (int c = 0; c < C; ++c)
          red[(c * kWideRows + r) * 32 + lane] += red[(c * kWideRows + r + o) * 32 + lane];
      }
      __syncthreads();
    }
    if (nseg == 1) {
      if (r == 0 && valid) {
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = red[(c * kWideRows) * 32 + lane];
        write_reduced<C>(a, a.act_off[k] + local, v, with_acc);
      }
    } else {
      // segment sum over the segment's first row (only this CTA reads or
      // writes those columns of that row until the block's last CTA)
      if (r == 0) {
        if (valid) {
          double* P0 = a.partials + (size_t)(w0 + g * kWideRows) * C * NI + q;
#pragma unroll
          for (int c = 0; c < C; ++c) P0[(size_t)c * NI] = red[(c * kWideRows) * 32 + lane];
        }
        __threadfence();
      }
      __syncthreads();
      int32_t* cnt = a.wide_cnt + (size_t)(a.wt_off[k] + it * nseg) * cbs + cb;
      if (threadIdx.x == 0) last_sh = atomicAdd(cnt, 1) == nseg - 1;
      __syncthreads();
      if (last_sh) {
        // warp r < C adds component r of the segment sums in
        // segment order, eight loads in flight at a time
        if (r < C) {
          __threadfence();
          double acc = 0.0;
          for (int32_t h0 = 0; h0 < nseg; h0 += 8) {
            double x[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const double* P0 =
                  a.partials + (size_t)(w0 + (h0 + j) * kWideRows) * C * NI + q;
              x[j] = (valid && h0 + j < nseg) ? __ldcg(P0 + (size_t)r * NI) : 0.0;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (h0 + j < nseg) acc += x[j];
          }
          red[r * 32 + lane] = acc;
        }
        __syncthreads();
        if (r == 0) {
          if (valid) {
#pragma unroll
            for (int c = 0; c < C; ++c) v[c] = red[c * 32 + lane];
            write_reduced<C>(a, a.act_off[k] + local, v, with_acc);
          }
          if (lane == 0) *cnt = 0;  // ready for the next launch
        }
      }
    }
    __syncthreads();  // red[] and last_sh are rewritten by the next unit
  }
}

__device__ __forceinline__ double norm3(double x, double y, double z) {
  return sqrt(x * x + y * y + z * z);
}

// Step criterion of Aarseth (the paper's reference for its block steps):
// dt = sqrt(eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2)); +inf when the
// denominator vanishes.
__device__ __forceinline__ double aarseth(double na, double nj, double n2, double n3, double eta) {
  const double den = nj * n3 + n2 * n2;
  if (!(den > 0.0)) return CUDART_INF;
  return sqrt(eta * (na * n2 + nj * nj) / den);
}

// Power-of-two level: the largest 2^-L not above dt (via frexp), clamped to
// [lmin, lmax]; growth by one level at most and only when the new time is a
// multiple of the doubled step; L_old < 0 means no previous level.
__device__ __forceinline__ int32_t new_level(double dt, int32_t L_old, int64_t t_new, int T,
                                             int lmin, int lmax) {
  int L;
  if (!(dt > 0.0)) {
    L = lmax;
  } else if (isinf(dt)) {
    L = lmin;
  } else {
    int e;
    (void)frexp(dt, &e);
    L = 1 - e;
  }
  L = min(max(L, lmin), lmax);
  if (L_old < 0 || L >= L_old) return L;
  const int Ld = L_old - 1;
  if (Ld < lmin) return L_old;
  return (t_new % ((int64_t)1 << (T - Ld)) == 0) ? Ld : L_old;
}

// Hermite corrector (Sec. 2 item 1) of the listed particles, new step level,
// and the state write-back.
// One active particle per group of 4 lanes: lane q < 3 takes component q of
// the predictor and corrector, and the four norms of the step criterion are
// summed across the group in the order (x^2 + y^2) + z^2; lane q then takes
// the square root of norm q.  The per-lane FP64 work is about a third of a
// particle's (GB300's FP64 pipe is the bound here).
__global__ void k_correct(Dev d, CorrectArgs c) {
  pdl_wait();  // the previous kernel of the chain has completed
  pdl_launch();
  const int64_t m = c.count_dev ? (int64_t)*c.count_dev : c.count_host;
  if (c.reset_tmin && blockIdx.x == 0)  // the block step's t_min is used up
    for (int32_t k = threadIdx.x; k < d.K; k += blockDim.x) d.t_min[k] = LLONG_MAX;
  const int q = threadIdx.x & 3;
  const unsigned gmask = 0xfu << (threadIdx.x & 28);
  const int64_t g0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 2;
  const int64_t gs = ((int64_t)gridDim.x * blockDim.x) >> 2;
  for (int64_t s = g0; s < m; s += gs) {
    const int32_t i = c.active[s];
    if (i < 0 || i >= d.N) {
      if (q == 0) atomicOr(d.status, kStatusInval);
      continue;
    }
    const int32_t cl = d.cid[i];
    const int64_t tn = c.t_tgt ? c.t_tgt[cl] : c.t_fixed;
    const int64_t ti = d.t[i];
    if (tn <= ti) {  // a step must move forward in time
      if (q == 0) atomicOr(d.status, kStatusInval);
      continue;
    }
    const double t = ldexp((double)(tn - ti), -c.T);
    // component q of the state (q == 3: the fourth word of each record)
    const double x0 = reinterpret_cast<const double*>(d.pos + i)[q];
    const double v0 = reinterpret_cast<const double*>(d.vel + i)[q];
    const double a0 = reinterpret_cast<const double*>(d.acc + i)[q];
    const double j0 = reinterpret_cast<const double*>(d.jerk + i)[q];
    const double a1 = q < 3 ? c.acc[s * c.sa + q] : 0.0;
    const double j1 = q < 3 ? c.jerk[s * c.sj + q] : 0.0;
    // Taylor predictor (Horner form), as predict1
    const double h = 0.5 * t, th = t * (1.0 / 3.0);
    const double xp = x0 + t * (v0 + h * (a0 + th * j0));
    const double vp = v0 + t * (a0 + h * j0);
    // the Hermite fit's divisions as multiplications by 1/t^2, 1/t^3 (exact
    // powers of two in a block step) and the Taylor coefficients
    const double t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t;
    int te;
    const bool pow2 = frexp(t, &te) == 0.5;
    const double it2 = pow2 ? ldexp(1.0, 2 - 2 * te) : 1.0 / t2;
    const double it3 = pow2 ? ldexp(1.0, 3 - 3 * te) : it2 / t;
    const double c24 = t4 * (1.0 / 24.0), c120 = t5 * (1.0 / 120.0), c6 = t3 * (1.0 / 6.0);
    const double da = a0 - a1;
    const double a2 = (-6.0 * da - t * (4.0 * j0 + 2.0 * j1)) * it2;
    const double a3 = (12.0 * da + 6.0 * t * (j0 + j1)) * it3;
    const double x1 = xp + a2 * c24 + a3 * c120;
    const double v1 = vp + a2 * c6 + a3 * c24;
    const double a2e = a2 + a3 * t;
    // squared norms over the group: lanes (0 + 1) then + 2 (lane 3 adds 0)
    double n[4];
    n[0] = q < 3 ? a1 * a1 : 0.0;
    n[1] = q < 3 ? j1 * j1 : 0.0;
    n[2] = q < 3 ? a2e * a2e : 0.0;
    n[3] = q < 3 ? a3 * a3 : 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      n[k] += __shfl_xor_sync(gmask, n[k], 1, 4);
      n[k] += __shfl_xor_sync(gmask, n[k], 2, 4);
    }
    // lane q takes sqrt of norm q; gather the four
    const double mine = sqrt(q == 0 ? n[0] : q == 1 ? n[1] : q == 2 ? n[2] : n[3]);
    const double na = __shfl_sync(gmask, mine, 0, 4), nj = __shfl_sync(gmask, mine, 1, 4);
    const double n2 = __shfl_sync(gmask, mine, 2, 4), n3 = __shfl_sync(gmask, mine, 3, 4);
    const double dt = aarseth(na, nj, n2, n3, c.eta);
    const int32_t L = new_level(dt, d.level[i], tn, c.T, c.lmin, c.lmax);
    const bool bad = q < 3 && !(isfinite(x1) && isfinite(v1));
    if (__any_sync(gmask, bad) && q == 0) atomicOr(d.status, kStatusNonFinite);
    double* P = reinterpret_cast<double*>(d.pos + i);
    double* V = reinterpret_cast<double*>(d.vel + i);
    double* A = reinterpret_cast<double*>(d.acc + i);
    double* J = reinterpret_cast<double*>(d.jerk + i);
    if (q < 3) {
      P[q] = x1;
      V[q] = v1;
      A[q] = a1;
      J[q] = j1;
    } else {  // the fourth words: mass kept, potential from this step when given
      V[3] = 0.0;
      if (c.pot) A[3] = c.pot[s * c.sp];
      J[3] = 0.0;
    }
    if (q == 0) {
      d.t[i] = tn;
      d.level[i] = L;
    }
  }
}

// 6th-order Hermite corrector (Sec. 2 item 1, the order of the paper's
// template code) of the listed particles, one thread per particle.  Over the
// step t from (x0, v0, a0, j0, s0) to the force (a1, j1, s1) at the predicted
// end, the quintic through (a0, j0, s0) and (a1, j1, s1) integrates to
//   v1 = v0 + t/2 (a0 + a1) - t^2/10 (j1 - j0) + t^3/120 (s0 + s1),
//   x1 = x0 + t/2 (v0 + v1) - t^2/10 (a1 - a0) + t^3/120 (j0 + j1),
// and its derivatives at the end (D = a1 - a0) are
//   crackle t^3 = 60 D - t (24 j0 + 36 j1) - t^2 (3 s0 - 9 s1),
//   pop t^4     = 360 D - t (168 j0 + 192 j1) - t^2 (24 s0 - 36 s1),
//   a5 t^5      = 720 D - 360 t (j0 + j1) - 60 t^2 (s0 - s1).
// The step criterion is the generalised Aarseth form of the p-th order
// Hermite schemes at p = 6, dt = eta (A1 / A4)^(1/3) with
// A_k = sqrt(|a^(k-1)| |a^(k+1)|) + |a^(k)| over a, j, s, crackle, pop, a5 at
// the end of the step; the power-of-two level follows the 4th-order rules.
// The crackle is kept for the next prediction.
__global__ void k_correct6(Dev d, CorrectArgs c) {
  pdl_wait();  // the previous kernel of the chain has completed
  pdl_launch();
  const int64_t m = c.count_dev ? (int64_t)*c.count_dev : c.count_host;
  if (c.reset_tmin && blockIdx.x == 0)  // the block step's t_min is used up
    for (int32_t k = threadIdx.x; k < d.K; k += blockDim.x) d.t_min[k] = LLONG_MAX;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < m;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = c.active[s];
    if (i < 0 || i >= d.N) {
      atomicOr(d.status, kStatusInval);
      continue;
    }
    const int32_t cl = d.cid[i];
    const int64_t tn = c.t_tgt ? c.t_tgt[cl] : c.t_fixed;
    const int64_t ti = d.t[i];
    if (tn <= ti) {  // a step must move forward in time
      atomicOr(d.status, kStatusInval);
      continue;
    }
    const double t = ldexp((double)(tn - ti), -c.T);
    int te;
    const bool pow2 = frexp(t, &te) == 0.5;
    const double it = pow2 ? ldexp(1.0, 1 - te) : 1.0 / t;  // exact for a block step
    const double t2 = t * t, t3 = t2 * t, it2 = it * it, it3 = it2 * it;
    const double h = 0.5 * t, c10 = t2 * 0.1, c120 = t3 * (1.0 / 120.0);
    const dbl4 X0 = d.pos[i], V0 = d.vel[i], A0 = d.acc[i], J0 = d.jerk[i], S0 = d.snap[i];
    const double x0[3] = {X0.x, X0.y, X0.z}, v0[3] = {V0.x, V0.y, V0.z};
    const double a0[3] = {A0.x, A0.y, A0.z}, j0[3] = {J0.x, J0.y, J0.z};
    const double s0[3] = {S0.x, S0.y, S0.z};
    double a1[3], j1[3], s1[3], x1[3], v1[3], cr[3], po[3], a5[3];
    bool finite = true;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      a1[q] = c.acc[s * c.sa + q];
      j1[q] = c.jerk[s * c.sj + q];
      s1[q] = c.snap[s * c.ss + q];
      v1[q] = v0[q] + h * (a0[q] + a1[q]) - c10 * (j1[q] - j0[q]) + c120 * (s0[q] + s1[q]);
      x1[q] = x0[q] + h * (v0[q] + v1[q]) - c10 * (a1[q] - a0[q]) + c120 * (j0[q] + j1[q]);
      const double D = a1[q] - a0[q];
      cr[q] = (60.0 * D - t * (24.0 * j0[q] + 36.0 * j1[q]) - t2 * (3.0 * s0[q] - 9.0 * s1[q])) *
              it3;
      po[q] = (360.0 * D - t * (168.0 * j0[q] + 192.0 * j1[q]) -
               t2 * (24.0 * s0[q] - 36.0 * s1[q])) * (it3 * it);
      a5[q] = (720.0 * D - 360.0 * t * (j0[q] + j1[q]) - 60.0 * t2 * (s0[q] - s1[q])) *
              (it3 * it2);
      finite = finite && isfinite(x1[q]) && isfinite(v1[q]);
    }
    const double na = norm3(a1[0], a1[1], a1[2]), nj = norm3(j1[0], j1[1], j1[2]);
    const double ns = norm3(s1[0], s1[1], s1[2]), nc = norm3(cr[0], cr[1], cr[2]);
    const double np = norm3(po[0], po[1], po[2]), nq = norm3(a5[0], a5[1], a5[2]);
    const double A1 = sqrt(na * ns) + nj, A4 = sqrt(nc * nq) + np;
    const double dt = A4 > 0.0 ? c.eta * cbrt(A1 / A4) : CUDART_INF;
    const int32_t L = new_level(dt, d.level[i], tn, c.T, c.lmin, c.lmax);
    if (!finite) atomicOr(d.status, kStatusNonFinite);
    d.pos[i] = dbl4{x1[0], x1[1], x1[2], X0.w};
    d.vel[i] = dbl4{v1[0], v1[1], v1[2], 0.0};
    d.acc[i] = dbl4{a1[0], a1[1], a1[2], c.pot ? c.pot[s * c.sp] : A0.w};
    d.jerk[i] = dbl4{j1[0], j1[1], j1[2], 0.0};
    d.snap[i] = dbl4{s1[0], s1[1], s1[2], 0.0};
    d.crackle[i] = dbl4{cr[0], cr[1], cr[2], 0.0};
    d.t[i] = tn;
    d.level[i] = L;
  }
}

// Initial state: a0, jerk0 from the t = 0 force (identity active list) and
// the first level from eta_start |a| / |jerk|.
__global__ void k_init_levels(Dev d, double eta_s, int T, int lmin, int lmax) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const dbl4 a = d.acc_new[i], j = d.jerk_new[i];
    d.acc[i] = a;
    d.jerk[i] = dbl4{j.x, j.y, j.z, 0.0};
    const double nj = norm3(j.x, j.y, j.z);
    const double dt = nj > 0.0 ? eta_s * norm3(a.x, a.y, a.z) / nj : CUDART_INF;
    d.level[i] = new_level(dt, -1, 0, T, lmin, lmax);
    d.t[i] = 0;
  }
}

// A caller's target list: mark[p] = its row k (list[k] = p), checking that
// every entry lies in [0, N) and appears once.  mark must hold -1 before.
__global__ void k_mark_list(Dev d, const int32_t* list, int64_t m) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = list[k];
    if (p < 0 || p >= d.N) {
      atomicOr(d.status, kStatusInval);
      continue;
    }
    if (atomicExch(d.mark + p, static_cast<int32_t>(k)) != -1) atomicOr(d.status, kStatusInval);
  }
}

// Marked particles per source tile (one CTA of kMixJT threads per tile).
__global__ void __launch_bounds__(kMixJT) k_count_marked(Dev d) {
  __shared__ int32_t sh[32];
  const int32_t tile = blockIdx.x;
  const int32_t k = upper_bound_i32(d.toff, d.K + 1, tile) - 1;
  const int64_t s = d.soff[k] + (int64_t)(tile - d.toff[k]) * kMixJT + threadIdx.x;
  const int32_t p = s < d.soff[k + 1] ? d.sperm[s] : -1;
  const int32_t f = (p >= 0 && d.mark[p] >= 0) ? 1 : 0;
  const int32_t tot =
      block_reduce<int32_t>(f, [](int32_t x, int32_t y) { return x + y; }, sh, 0);
  if (threadIdx.x == 0) d.blk_count[tile] = tot;
}

// The marked particles in source-slot order (spatially coherent targets),
// their caller rows, each cluster's offset in the list; clears the marks.
__global__ void __launch_bounds__(kMixJT) k_scatter_marked(Dev d) {
  __shared__ int32_t sh[32];
  const int32_t tile = blockIdx.x;
  const int32_t k = upper_bound_i32(d.toff, d.K + 1, tile) - 1;
  const int64_t s = d.soff[k] + (int64_t)(tile - d.toff[k]) * kMixJT + threadIdx.x;
  const int32_t p = s < d.soff[k + 1] ? d.sperm[s] : -1;
  const int32_t row = p >= 0 ? d.mark[p] : -1;
  const int32_t f = row >= 0 ? 1 : 0;
  int32_t tot;
  const int32_t ex = block_excl_scan(f, sh, &tot);
  const int32_t run = d.blk_count[tile];
  if (f) {
    d.active[run + ex] = p;
    d.rows[run + ex] = row;
    d.mark[p] = -1;
  }
  if (s == d.soff[k]) d.act_off[k] = run;
}

// Identity active list: every particle of every cluster is a target.
__global__ void k_actoff_identity(Dev d) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= d.K;
       k += (int64_t)gridDim.x * blockDim.x)
    d.act_off[k] = static_cast<int32_t>(d.off[k]);
}

// Energy: per-block partial sums (fixed ranges) of 1/2 m v^2 from the FP64
// predicted velocities and of 1/2 m pot; then one CTA sums the partials in
// block order (deterministic).
__global__ void k_energy_partial(Dev d, const double* pot, int sp, int64_t lo, int64_t hi,
                                 double* out) {
  __shared__ double sh[32];
  double ek = 0.0, ep = 0.0;
  for (int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hi;
       i += (int64_t)gridDim.x * blockDim.x) {
    const dbl4 v = d.src64_vel[d.sinv[i]];
    const double m = d.pos[i].w;
    ek += 0.5 * m * (v.x * v.x + v.y * v.y + v.z * v.z);
    ep += 0.5 * m * pot[i * sp];
  }
  auto add = [](double x, double y) { return x + y; };
  ek = block_reduce<double>(ek, add, sh, 0.0);
  ep = block_reduce<double>(ep, add, sh, 0.0);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = ek;
    out[2 * blockIdx.x + 1] = ep;
  }
}

__global__ void k_energy_final(double* part, int nblk, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double hk = 0.0, lk = 0.0, hp = 0.0, lp = 0.0;
    for (int b = 0; b < nblk; ++b) {
      two_sum_acc(hk, lk, part[2 * b]);
      two_sum_acc(hp, lp, part[2 * b + 1]);
    }
    out[0] = hk + lk;
    out[1] = hp + lp;
  }
}

// (n, 3) rows <-> double4 rows; keep_w keeps the destination's 4th lane
// (mass in pos, potential in acc), otherwise it is zeroed.
__global__ void k_pack3(const double* src3, dbl4* dst, int64_t n, int keep_w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double w = keep_w ? dst[i].w : 0.0;
    dst[i] = dbl4{src3[3 * i], src3[3 * i + 1], src3[3 * i + 2], w};
  }
}

__global__ void k_unpack3(const dbl4* src, double* dst3, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const dbl4 v = src[i];
    dst3[3 * i] = v.x;
    dst3[3 * i + 1] = v.y;
    dst3[3 * i + 2] = v.z;
  }
}

// Current block time of each cluster = the latest particle time in it.
// Kick-drift-kick leapfrog halves on every particle (nb_step_leapfrog).
// a_new == nullptr: kick with the stored acceleration and drift,
//   v <- v + h a, x <- x + dt v, t <- t + dt_ticks;
// otherwise: kick with the new acceleration (rows of 4 doubles) and store it,
//   v <- v + h a_new, a <- a_new (the potential word is kept).
__global__ void k_leapfrog(Dev d, const double* a_new, double h, double dt, int64_t dt_ticks) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    dbl4 v = d.vel[i];
    if (a_new == nullptr) {
      const dbl4 a = d.acc[i];
      v.x = v.x + h * a.x;
      v.y = v.y + h * a.y;
      v.z = v.z + h * a.z;
      dbl4 p = d.pos[i];
      p.x = p.x + dt * v.x;
      p.y = p.y + dt * v.y;
      p.z = p.z + dt * v.z;
      d.pos[i] = p;
      d.t[i] += dt_ticks;
    } else {
      const double ax = a_new[4 * i], ay = a_new[4 * i + 1], az = a_new[4 * i + 2];
      v.x = v.x + h * ax;
      v.y = v.y + h * ay;
      v.z = v.z + h * az;
      dbl4 a = d.acc[i];
      a.x = ax;
      a.y = ay;
      a.z = az;
      d.acc[i] = a;
    }
    d.vel[i] = v;
  }
}

// Every particle as a target list in source-slot order (the spatial order
// of the tiles, so the warps of the force kernel get compact target groups):
// active[off[k] + r] = sperm[soff[k] + r] for the N_k leading slots of each
// cluster (its pad slots come last).
__global__ void k_slot_list(Dev d) {
  const int64_t S = d.soff[d.K];
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = upper_bound_i64(d.soff, d.K + 1, s) - 1;
    const int64_t r = s - d.soff[k];
    if (r < d.off[k + 1] - d.off[k]) d.active[d.off[k] + r] = d.sperm[s];
  }
}

// Self-check of the bounded device waits: an mbarrier phase that nothing
// completes (one expected arrival, none made); the wait gives up after
// `budget` clock cycles and reports it in the sticky status, as the force
// kernels do when a bulk copy never lands.  Nothing is in flight on the
// barrier, so the CTA simply returns.
__global__ void k_wait_probe(uint32_t* status, long long budget) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0u, budget);
  if (!ok && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

__global__ void k_tcur_from_t(Dev d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.N;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicMax(reinterpret_cast<long long*>(d.t_cur + d.cid[i]), (long long)d.t[i]);
}

}  // namespace

// ----------------------------------------------------------- launchers
static inline int blocks_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t b = ceil_div64(n > 0 ? n : 1, threads);
  return static_cast<int>(b < cap ? b : cap);
}

cudaError_t launch_fill_i64(int64_t* p, int64_t n, int64_t v, cudaStream_t st) {
  k_fill_i64<<<blocks_for(n, 256), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}
cudaError_t launch_tmin(const Dev& d, int T, cudaStream_t st) {
  return launch_chain(k_tmin, dim3(static_cast<unsigned>(ceil_div64(d.N, 256))), dim3(256), 0,
                      st, d, T);
}
cudaError_t launch_predict(const Dev& d, const int64_t* t_tgt, int64_t t_fixed, int T,
                           bool mix, bool f64, bool count_due, cudaStream_t st, bool zero_tau) {
  return launch_chain(k_predict_tiles, dim3(static_cast<unsigned>(d.n_tiles)), dim3(kMixJT), 0,
                      st, d, t_tgt, t_fixed, T, mix ? 1 : 0, f64 ? 1 : 0, count_due ? 1 : 0,
                      zero_tau ? 1 : 0);
}
cudaError_t launch_wait_probe(uint32_t* status, long long budget, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(status, budget);
  return cudaGetLastError();
}
cudaError_t launch_slot_list(const Dev& d, cudaStream_t st) {
  k_slot_list<<<blocks_for(d.N + 4 * d.K, 256), 256, 0, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_leapfrog(const Dev& d, const double* a_new, double h, double dt,
                            int64_t dt_ticks, cudaStream_t st) {
  k_leapfrog<<<blocks_for(d.N, 256), 256, 0, st>>>(d, a_new, h, dt, dt_ticks);
  return cudaGetLastError();
}
cudaError_t launch_scan_plan_scatter(const Dev& d, const PlanArgs& p, int T, cudaStream_t st) {
  cudaError_t e = launch_chain(k_scan_plan, dim3(1), dim3(1024), 0, st, d,
                               static_cast<int32_t>(d.n_tiles), p);
  if (e != cudaSuccess) return e;
  return launch_chain(k_scatter_tiles,
                      dim3(blocks_for(d.n_tiles * kMixJT, kScatterThreads)),
                      dim3(kScatterThreads), 0, st, d, T);
}
cudaError_t launch_plan(const Dev& d, const PlanArgs& p, cudaStream_t st) {
  return launch_chain(k_plan, dim3(1), dim3(512), 0, st, d, p);
}
cudaError_t launch_reduce(const ForceArgs& a, int NI, bool with_acc, int64_t m_bound,
                          int grid, cudaStream_t st) {
  // one persistent CTA of 1024 threads per SM (its 82 KB of shared memory
  // serve the large splits); exits at once when the plan split nothing
  (void)m_bound;
  const int g = grid > 0 ? grid : 1;
  if (a.comps == kPartialCompsSnap)
    return launch_chain(k_reduce<kPartialCompsSnap>, dim3(g), dim3(32 * kWideRows), kWideSmem, st,
                        a, NI, with_acc ? 1 : 0);
  return launch_chain(k_reduce<kPartialComps>, dim3(g), dim3(32 * kWideRows), kWideSmem, st, a,
                      NI, with_acc ? 1 : 0);
}
cudaError_t integrator_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_reduce<kPartialComps>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kWideSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_reduce<kPartialCompsSnap>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kWideSmem));
}
cudaError_t launch_correct(const Dev& d, const CorrectArgs& c, int64_t m_bound, cudaStream_t st) {
  // 4 lanes per particle; the grid strides over the active list, whose
  // length is on the device in a block step (m_bound = N then): 128-thread
  // CTAs, at most 4 per SM, the same lanes as 32-thread CTAs at 16 per SM but
  // a quarter of the CTA launches when few particles are active
  return launch_chain(k_correct, dim3(blocks_for(4 * m_bound, 128, 152 * 4)), dim3(128), 0, st,
                      d, c);
}
cudaError_t launch_correct6(const Dev& d, const CorrectArgs& c, int64_t m_bound,
                            cudaStream_t st) {
  // one thread per particle, grid-stride, 128-thread CTAs (as k_correct)
  return launch_chain(k_correct6, dim3(blocks_for(m_bound, 128, 152 * 4)), dim3(128), 0, st, d,
                      c);
}
cudaError_t launch_init_levels(const Dev& d, double eta_s, int T, int lmin, int lmax,
                               cudaStream_t st) {
  k_init_levels<<<blocks_for(d.N, 256), 256, 0, st>>>(d, eta_s, T, lmin, lmax);
  return cudaGetLastError();
}
cudaError_t launch_list_to_slots(const Dev& d, const int32_t* list, int64_t m,
                                 cudaStream_t st) {
  k_mark_list<<<blocks_for(m, 256), 256, 0, st>>>(d, list, m);
  k_count_marked<<<static_cast<int>(d.n_tiles), kMixJT, 0, st>>>(d);
  k_scan<<<1, 1024, 0, st>>>(d, static_cast<int32_t>(d.n_tiles));
  k_scatter_marked<<<static_cast<int>(d.n_tiles), kMixJT, 0, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_actoff_identity(const Dev& d, cudaStream_t st) {
  k_actoff_identity<<<blocks_for(d.K + 1, 256), 256, 0, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_energy(const Dev& d, const double* pot, int sp, int64_t lo, int64_t hi,
                          double* part, int nblk, double* out, cudaStream_t st) {
  k_energy_partial<<<nblk, 256, 0, st>>>(d, pot, sp, lo, hi, part);
  k_energy_final<<<1, 32, 0, st>>>(part, nblk, out);
  return cudaGetLastError();
}

cudaError_t launch_pack3(const double* src3, dbl4* dst, int64_t n, bool keep_w, cudaStream_t st) {
  k_pack3<<<blocks_for(n, 256), 256, 0, st>>>(src3, dst, n, keep_w ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t launch_unpack3(const dbl4* src, double* dst3, int64_t n, cudaStream_t st) {
  k_unpack3<<<blocks_for(n, 256), 256, 0, st>>>(src, dst3, n);
  return cudaGetLastError();
}
cudaError_t launch_tcur_from_t(const Dev& d, cudaStream_t st) {
  k_tcur_from_t<<<blocks_for(d.N, 256), 256, 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace nb
