// nb_force_mixed.cu -- mixed-precision direct-summation force kernel (sm_103a).
//
// Computes, for each target i, Eq. 1 with the softening of Eq. 2 plus the
// jerk and potential:
//   a_i  =  sum_j m_j d / s^3,   jerk_i = sum_j m_j (w / s^3 - 3 (d.w) d / s^5),
//   pot_i = -sum_j m_j / s,       d = r_j - r_i, w = v_j - v_i, s^2 = d.d + eps^2
// (G applied on output).  Precision follows Sec. 2 item 4: the separation is
// formed from double-single positions, (xh_j - xh_i) + (xl_j - xl_i), so it
// keeps FP64-like resolution for close pairs; everything after that, square
// root included, is FP32 (hardware rsqrt); sums are accumulated per tile in
// FP32 and folded into a compensated (hi, lo) FP32 pair per tile (two-sum),
// then combined in FP64.
//
// GB300 mapping:
//   * persistent CTAs loop over work items (cluster, i-tile, j-chunk); the
//     j-chunk split is the i-splitting of Sec. 2 item 3 (Bfactor): B chunks
//     of the source range per i-tile, partial sums reduced afterwards in a
//     fixed order;
//   * source tiles are staged in shared memory (Sec. 2 item 5) by one bulk
//     copy (TMA engine, cp.async.bulk) per tile into a two-stage ring guarded
//     by mbarriers; waits are bounded and report NB_ETIMEOUT instead of
//     hanging;
//   * every pair operation is a packed f32x2 instruction over two sources, so
//     the FP32 pipe is fed at full width while the SFU (rsqrt), shared-memory
//     loads and loop overhead use the remaining issue slots; each thread owns
//     two targets so one shared-memory load serves two interactions per lane.
#include "nb_internal.cuh"

namespace nb {
namespace {

constexpr int NT = kMixNT, IPT = kMixIPT, NI = kMixNI, JT = kMixJT;
constexpr int kGroupF4 = 10;                      // float4 per group of 4 sources
constexpr int kTileF4 = JT / 4 * kGroupF4;        // float4 per tile
constexpr uint32_t kGroupBytes = kGroupF4 * 16;

struct Target {
  f2 nxh, nyh, nzh, nxl, nyl, nzl, nvx, nvy, nvz;   // -r_i, -v_i as broadcast pairs
  f2 ax, ay, az, j1x, j1y, j1z, j2x, j2y, j2z, pt;  // per-tile sums (2 lanes)
  float th[10], tl[10];                             // compensated totals
  int64_t slot;
};

__device__ __forceinline__ f2 bcast(float v) { return f2_pack(v, v); }

// Two interactions (sources js, js + 1) for one target.
template <bool POT, bool MASK>
__device__ __forceinline__ void pair_step(Target& s, f2 xh, f2 yh, f2 zh, f2 m, f2 xl, f2 yl,
                                          f2 zl, f2 vx, f2 vy, f2 vz, f2 eps2, int64_t js) {
  const f2 dx = f2_add(f2_add(xh, s.nxh), f2_add(xl, s.nxl));
  const f2 dy = f2_add(f2_add(yh, s.nyh), f2_add(yl, s.nyl));
  const f2 dz = f2_add(f2_add(zh, s.nzh), f2_add(zl, s.nzl));
  const f2 wx = f2_add(vx, s.nvx);
  const f2 wy = f2_add(vy, s.nvy);
  const f2 wz = f2_add(vz, s.nvz);
  f2 r2 = f2_fma(dx, dx, eps2);
  r2 = f2_fma(dy, dy, r2);
  r2 = f2_fma(dz, dz, r2);
  f2 rv = f2_mul(dx, wx);
  rv = f2_fma(dy, wy, rv);
  rv = f2_fma(dz, wz, rv);
  const float2 q = f2_unpack(r2);
  float ri0 = rsqrt_approx(q.x);
  float ri1 = rsqrt_approx(q.y);
  if (MASK) {  // j == i is excluded by index (Eq. 1)
    if (js == s.slot) ri0 = 0.f;
    if (js + 1 == s.slot) ri1 = 0.f;
  }
  const f2 rinv = f2_pack(ri0, ri1);
  const f2 r2inv = f2_mul(rinv, rinv);
  const f2 mri = f2_mul(m, rinv);
  const f2 mr3 = f2_mul(mri, r2inv);
  if (POT) s.pt = f2_add(s.pt, mri);
  const f2 u = f2_mul(rv, r2inv);
  const f2 bb = f2_mul(u, mr3);
  s.ax = f2_fma(mr3, dx, s.ax);
  s.ay = f2_fma(mr3, dy, s.ay);
  s.az = f2_fma(mr3, dz, s.az);
  s.j1x = f2_fma(mr3, wx, s.j1x);
  s.j1y = f2_fma(mr3, wy, s.j1y);
  s.j1z = f2_fma(mr3, wz, s.j1z);
  s.j2x = f2_fma(bb, dx, s.j2x);
  s.j2y = f2_fma(bb, dy, s.j2y);
  s.j2z = f2_fma(bb, dz, s.j2z);
}

template <bool POT, bool MASK>
__device__ __forceinline__ void tile_compute(const float4* __restrict__ tile, int ngroups,
                                             int64_t slot0, Target (&tg)[IPT], f2 eps2) {
#pragma unroll 2
  for (int g = 0; g < ngroups; ++g) {
    const ulonglong2* G = reinterpret_cast<const ulonglong2*>(tile + g * kGroupF4);
    const ulonglong2 xh = G[0], yh = G[1], zh = G[2], m = G[3], xl = G[4], yl = G[5],
                     zl = G[6], vx = G[7], vy = G[8], vz = G[9];
    const int64_t js = slot0 + 4 * g;
#pragma unroll
    for (int r = 0; r < IPT; ++r) {
      pair_step<POT, MASK>(tg[r], xh.x, yh.x, zh.x, m.x, xl.x, yl.x, zl.x, vx.x, vy.x, vz.x,
                           eps2, js);
      pair_step<POT, MASK>(tg[r], xh.y, yh.y, zh.y, m.y, xl.y, yl.y, zl.y, vx.y, vy.y, vz.y,
                           eps2, js + 2);
    }
  }
}

__device__ __forceinline__ float lanes_sum(f2& v) {
  const float2 p = f2_unpack(v);
  v = 0ull;
  return p.x + p.y;
}

// Fold the per-tile FP32 sums into the compensated totals.
__device__ __forceinline__ void flush(Target& s) {
  two_sum_acc(s.th[0], s.tl[0], lanes_sum(s.ax));
  two_sum_acc(s.th[1], s.tl[1], lanes_sum(s.ay));
  two_sum_acc(s.th[2], s.tl[2], lanes_sum(s.az));
  two_sum_acc(s.th[3], s.tl[3], lanes_sum(s.j1x));
  two_sum_acc(s.th[4], s.tl[4], lanes_sum(s.j1y));
  two_sum_acc(s.th[5], s.tl[5], lanes_sum(s.j1z));
  two_sum_acc(s.th[6], s.tl[6], lanes_sum(s.j2x));
  two_sum_acc(s.th[7], s.tl[7], lanes_sum(s.j2y));
  two_sum_acc(s.th[8], s.tl[8], lanes_sum(s.j2z));
  two_sum_acc(s.th[9], s.tl[9], lanes_sum(s.pt));
}

__device__ __forceinline__ void issue_tile(float4* stage, uint64_t* bar, const float4* src,
                                           int64_t t0, int64_t cnt) {
  const uint32_t bytes = static_cast<uint32_t>(cnt / 4) * kGroupBytes;
  mbar_arrive_expect(bar, bytes);
  bulk_g2s(stage, src + (t0 >> 2) * kGroupF4, bytes, bar);
}

template <bool POT>
__global__ void __launch_bounds__(NT, 2) k_force_mixed(const ForceArgs a) {
  __shared__ __align__(128) float4 stage[2][kTileF4];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    abort_flag = 0;
  }
  __syncthreads();
  uint32_t used[2] = {0u, 0u};  // completed phases per stage
  const float4* __restrict__ src = static_cast<const float4*>(a.src_a);
  const float e2 = static_cast<float>(a.eps2);
  const f2 eps2 = f2_pack(e2, e2);
  const int32_t n_items = a.item_off[a.K];
  bool pending[2] = {false, false};

  for (int32_t w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int32_t k = upper_bound_i32(a.item_off, a.K + 1, w) - 1;
    const int32_t B = a.bfac[k];
    const int32_t l = w - a.item_off[k];
    const int32_t it = l / B;
    const int32_t b = l - it * B;
    const int64_t sk0 = a.soff[k];
    const int64_t S_k = a.soff[k + 1] - sk0;
    const int64_t L = chunk_len(S_k, B, JT);
    const int64_t j0 = sk0 + b * L;
    const int64_t j1 = sk0 + min(S_k, (int64_t)(b + 1) * L);
    const int32_t a0 = a.act_off[k];
    const int32_t m_k = a.act_off[k + 1] - a0;
    const int64_t p0 = a.off[k], p1 = a.off[k + 1];

    Target tg[IPT];
    bool valid[IPT];
#pragma unroll
    for (int r = 0; r < IPT; ++r) {
      const int32_t q = it * NI + r * NT + tid;
      valid[r] = q < m_k;
      float xh = 0.f, yh = 0.f, zh = 0.f, xl = 0.f, yl = 0.f, zl = 0.f, vx = 0.f, vy = 0.f,
            vz = 0.f;
      tg[r].slot = -1;
      if (valid[r]) {
        const int32_t s = a0 + q;
        const int64_t p = a.active ? (int64_t)a.active[s] : (int64_t)s;
        if (p < p0 || p >= p1) {
          valid[r] = false;
          atomicOr(a.status, kStatusInval);
        } else {
          const int64_t slot = sk0 + (p - p0);
          const float* gp = reinterpret_cast<const float*>(src + (slot >> 2) * kGroupF4) + (slot & 3);
          xh = gp[0]; yh = gp[4]; zh = gp[8];
          xl = gp[16]; yl = gp[20]; zl = gp[24];
          vx = gp[28]; vy = gp[32]; vz = gp[36];
          tg[r].slot = slot;
        }
      }
      tg[r].nxh = bcast(-xh); tg[r].nyh = bcast(-yh); tg[r].nzh = bcast(-zh);
      tg[r].nxl = bcast(-xl); tg[r].nyl = bcast(-yl); tg[r].nzl = bcast(-zl);
      tg[r].nvx = bcast(-vx); tg[r].nvy = bcast(-vy); tg[r].nvz = bcast(-vz);
      tg[r].ax = tg[r].ay = tg[r].az = 0ull;
      tg[r].j1x = tg[r].j1y = tg[r].j1z = 0ull;
      tg[r].j2x = tg[r].j2y = tg[r].j2z = 0ull;
      tg[r].pt = 0ull;
#pragma unroll
      for (int c = 0; c < 10; ++c) { tg[r].th[c] = 0.f; tg[r].tl[c] = 0.f; }
    }

    const int64_t ntile = ceil_div64(j1 - j0, JT);
    if (tid == 0) {
      issue_tile(stage[0], &bar[0], src, j0, min((int64_t)JT, j1 - j0));
      pending[0] = true;
      if (ntile > 1) {
        issue_tile(stage[1], &bar[1], src, j0 + JT, min((int64_t)JT, j1 - j0 - JT));
        pending[1] = true;
      }
    }
    for (int64_t t = 0; t < ntile; ++t) {
      const int st = static_cast<int>(t & 1);
      const int64_t t0 = j0 + t * JT;
      const int64_t cnt = min((int64_t)JT, j1 - t0);
      const bool ok = mbar_wait(&bar[st], used[st] & 1u, kWaitBudget);
      used[st] += 1;
      if (tid == 0) pending[st] = false;
      if (!ok) {
        abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
      } else {
        bool self = false;
#pragma unroll
        for (int r = 0; r < IPT; ++r) self |= (tg[r].slot >= t0) && (tg[r].slot < t0 + cnt);
        const int ng = static_cast<int>(cnt >> 2);
        if (self)
          tile_compute<POT, true>(stage[st], ng, t0, tg, eps2);
        else
          tile_compute<POT, false>(stage[st], ng, t0, tg, eps2);
#pragma unroll
        for (int r = 0; r < IPT; ++r) flush(tg[r]);
      }
      __syncthreads();
      if (abort_flag) goto drain;
      if (tid == 0 && t + 2 < ntile) {
        issue_tile(stage[st], &bar[st], src, t0 + 2 * JT, min((int64_t)JT, j1 - t0 - 2 * JT));
        pending[st] = true;
      }
    }

#pragma unroll
    for (int r = 0; r < IPT; ++r) {
      if (!valid[r]) continue;
      const Target& s = tg[r];
      double v[kPartialComps];
      v[0] = (double)s.th[0] + (double)s.tl[0];
      v[1] = (double)s.th[1] + (double)s.tl[1];
      v[2] = (double)s.th[2] + (double)s.tl[2];
      v[3] = ((double)s.th[3] + (double)s.tl[3]) - 3.0 * ((double)s.th[6] + (double)s.tl[6]);
      v[4] = ((double)s.th[4] + (double)s.tl[4]) - 3.0 * ((double)s.th[7] + (double)s.tl[7]);
      v[5] = ((double)s.th[5] + (double)s.tl[5]) - 3.0 * ((double)s.th[8] + (double)s.tl[8]);
      v[6] = -((double)s.th[9] + (double)s.tl[9]);
      const int32_t ql = r * NT + tid;
      if (B == 1) {
        const int64_t srow = a0 + it * NI + ql;
        if (a.out_acc) for (int c = 0; c < 3; ++c) a.out_acc[srow * a.sa + c] = a.G * v[c];
        if (a.out_jerk) for (int c = 0; c < 3; ++c) a.out_jerk[srow * a.sj + c] = a.G * v[3 + c];
        if (POT && a.out_pot) a.out_pot[srow * a.sp] = a.G * v[6];
      } else {
        double* P = a.partials + (size_t)w * kPartialComps * NI + ql;
#pragma unroll
        for (int c = 0; c < kPartialComps; ++c) P[(size_t)c * NI] = v[c];
      }
    }
  }
  return;

drain:
  // A wait gave up: let any copy still in flight land (bounded) before the
  // CTA's shared memory is released.
  if (tid == 0) {
    for (int st = 0; st < 2; ++st)
      if (pending[st]) (void)mbar_wait(&bar[st], used[st] & 1u, kWaitBudget);
  }
}

}  // namespace

cudaError_t launch_force_mixed(const ForceArgs& a, int grid, bool with_pot, cudaStream_t st) {
  if (with_pot)
    k_force_mixed<true><<<grid, NT, 0, st>>>(a);
  else
    k_force_mixed<false><<<grid, NT, 0, st>>>(a);
  return cudaGetLastError();
}

int force_mixed_ctas_per_sm() {
  int n1 = 0, n2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_force_mixed<true>, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, k_force_mixed<false>, NT, 0);
  int n = n1 < n2 ? n1 : n2;
  return n > 0 ? n : 1;
}

size_t force_mixed_smem() { return sizeof(float4) * 2 * kTileF4; }

}  // namespace nb
