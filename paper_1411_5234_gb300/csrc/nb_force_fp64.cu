// nb_force_fp64.cu -- FP64 direct-summation force kernel (sm_103a).
//
// Same quantities as the mixed kernel (Eq. 1 with the softening of Eq. 2,
// the jerk and the potential), every operation in IEEE FP64; the reciprocal
// square root is CUDA's double-precision rsqrt().  Per-tile FP64 sums are
// folded into a two-sum (hi, lo) pair, so the summation error stays at the
// level of the individual terms' rounding.  A potential-only mode serves the
// FP64 energy, and a snap mode the 6th-order Hermite scheme (Sec. 2 item 1):
// with u = a_j - a_i (the predicted accelerations), alpha = d.w / s^2 and
// beta = (w.w + d.u) / s^2 + alpha^2, the pair term A = m d / s^3 has the
// time derivatives J = m (w - 3 alpha d) / s^3 and
// S = m (u - 6 alpha (w - 3 alpha d) - 3 beta d) / s^3.
//
// GB300 mapping: the FP64 pipe (about 1/64 of the FP32 rate on this part)
// bounds this kernel, so it keeps the simplest layout that feeds it -- one
// target per thread, double4 source tiles staged in shared memory by bulk
// copies (two-stage ring, bounded mbarrier waits), persistent CTAs over
// (cluster, i-tile, j-chunk) work items as in the mixed kernel.
#include "nb_internal.cuh"

namespace nb {
namespace {

constexpr int NT = kF64NT, NI = kF64NI, JT = kF64JT;

struct Target64 {
  double x, y, z, vx, vy, vz, ax, ay, az;
  double th[10], tl[10];
  int64_t slot;
};

template <int MODE, bool MASK>
__device__ __forceinline__ void tile_compute64(const dbl4* __restrict__ sp,
                                               const dbl4* __restrict__ sv, int cnt,
                                               int64_t slot0, Target64& s, double eps2) {
  double ax = 0, ay = 0, az = 0, j1x = 0, j1y = 0, j1z = 0, j2x = 0, j2y = 0, j2z = 0, pt = 0;
#pragma unroll 4
  for (int j = 0; j < cnt; ++j) {
    const dbl4 p = sp[j];
    const double dx = p.x - s.x, dy = p.y - s.y, dz = p.z - s.z;
    double r2 = fma(dx, dx, eps2);
    r2 = fma(dy, dy, r2);
    r2 = fma(dz, dz, r2);
    double rinv = rsqrt(r2);
    if (MASK && slot0 + j == s.slot) rinv = 0.0;  // j == i excluded (Eq. 1)
    const double mri = p.w * rinv;
    pt += mri;
    if (MODE == kF64Full) {
      const dbl4 v = sv[j];
      const double wx = v.x - s.vx, wy = v.y - s.vy, wz = v.z - s.vz;
      double rv = dx * wx;
      rv = fma(dy, wy, rv);
      rv = fma(dz, wz, rv);
      const double r2inv = rinv * rinv;
      const double mr3 = mri * r2inv;
      const double bb = rv * r2inv * mr3;
      ax = fma(mr3, dx, ax);
      ay = fma(mr3, dy, ay);
      az = fma(mr3, dz, az);
      j1x = fma(mr3, wx, j1x);
      j1y = fma(mr3, wy, j1y);
      j1z = fma(mr3, wz, j1z);
      j2x = fma(bb, dx, j2x);
      j2y = fma(bb, dy, j2y);
      j2z = fma(bb, dz, j2z);
    }
  }
  if (MODE == kF64Full) {
    two_sum_acc(s.th[0], s.tl[0], ax);
    two_sum_acc(s.th[1], s.tl[1], ay);
    two_sum_acc(s.th[2], s.tl[2], az);
    two_sum_acc(s.th[3], s.tl[3], j1x);
    two_sum_acc(s.th[4], s.tl[4], j1y);
    two_sum_acc(s.th[5], s.tl[5], j1z);
    two_sum_acc(s.th[6], s.tl[6], j2x);
    two_sum_acc(s.th[7], s.tl[7], j2y);
    two_sum_acc(s.th[8], s.tl[8], j2z);
  }
  two_sum_acc(s.th[9], s.tl[9], pt);
}

// Snap mode: acceleration, jerk, snap and potential of one target against a
// tile; sums per tile folded into the target's two-sum pairs
// th/tl[0..2] = A, [3..5] = J, [6..8] = S, [9] = potential.
template <bool MASK>
__device__ __forceinline__ void tile_compute64_snap(const dbl4* __restrict__ sp,
                                                    const dbl4* __restrict__ sv,
                                                    const dbl4* __restrict__ sa, int cnt,
                                                    int64_t slot0, Target64& s, double eps2) {
  double A[3] = {0, 0, 0}, J[3] = {0, 0, 0}, S[3] = {0, 0, 0}, pt = 0;
#pragma unroll 2
  for (int j = 0; j < cnt; ++j) {
    const dbl4 p = sp[j], v = sv[j], q = sa[j];
    const double d[3] = {p.x - s.x, p.y - s.y, p.z - s.z};
    const double w[3] = {v.x - s.vx, v.y - s.vy, v.z - s.vz};
    const double u[3] = {q.x - s.ax, q.y - s.ay, q.z - s.az};
    double r2 = fma(d[0], d[0], eps2);
    r2 = fma(d[1], d[1], r2);
    r2 = fma(d[2], d[2], r2);
    double rinv = rsqrt(r2);
    if (MASK && slot0 + j == s.slot) rinv = 0.0;  // j == i excluded (Eq. 1)
    const double mri = p.w * rinv;
    pt += mri;
    const double r2inv = rinv * rinv;
    const double mr3 = mri * r2inv;
    const double dw = fma(d[2], w[2], fma(d[1], w[1], d[0] * w[0]));
    const double wwdu = fma(d[2], u[2], fma(d[1], u[1], fma(d[0], u[0],
                        fma(w[2], w[2], fma(w[1], w[1], w[0] * w[0])))));
    const double alpha = dw * r2inv;
    const double beta = fma(wwdu, r2inv, alpha * alpha);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double jc = fma(-3.0 * alpha, d[c], w[c]);          // w - 3 alpha d
      const double sc = fma(-3.0 * beta, d[c], fma(-6.0 * alpha, jc, u[c]));
      A[c] = fma(mr3, d[c], A[c]);
      J[c] = fma(mr3, jc, J[c]);
      S[c] = fma(mr3, sc, S[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    two_sum_acc(s.th[c], s.tl[c], A[c]);
    two_sum_acc(s.th[3 + c], s.tl[3 + c], J[c]);
    two_sum_acc(s.th[6 + c], s.tl[6 + c], S[c]);
  }
  two_sum_acc(s.th[9], s.tl[9], pt);
}

template <int MODE>
__device__ __forceinline__ void issue64(dbl4* stp, dbl4* stv, dbl4* sta, uint64_t* bar,
                                        const dbl4* gp, const dbl4* gv, const dbl4* ga,
                                        int64_t t0, int64_t cnt) {
  const uint32_t bytes = static_cast<uint32_t>(cnt) * 32u;
  const uint32_t arrays = MODE == kF64Snap ? 3u : MODE == kF64Full ? 2u : 1u;
  mbar_arrive_expect(bar, arrays * bytes);
  bulk_g2s(stp, gp + t0, bytes, bar);
  if (MODE != kF64PotOnly) bulk_g2s(stv, gv + t0, bytes, bar);
  if (MODE == kF64Snap) bulk_g2s(sta, ga + t0, bytes, bar);
}

template <int MODE>
__global__ void __launch_bounds__(NT) k_force_fp64(const ForceArgs a) {
  pdl_wait();  // the previous kernel of the chain has completed
  pdl_launch();
  __shared__ __align__(128) dbl4 sp[2][JT];
  __shared__ __align__(128) dbl4 sv[2][JT];
  __shared__ __align__(128) dbl4 sa[2][MODE == kF64Snap ? JT : 1];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int abort_flag;
  __shared__ int32_t item_sh;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    abort_flag = 0;
  }
  __syncthreads();
  uint32_t used[2] = {0u, 0u};
  bool pending[2] = {false, false};
  const dbl4* __restrict__ gp = static_cast<const dbl4*>(a.src_a);
  const dbl4* __restrict__ gv = static_cast<const dbl4*>(a.src_b);
  const dbl4* __restrict__ ga = static_cast<const dbl4*>(a.src_c);
  constexpr int C = MODE == kF64Snap ? kPartialCompsSnap : kPartialComps;
  const int32_t n_items = a.item_off[a.K];

  // dynamic item order when the plan provided a counter (see k_force_mixed)
  const bool dyn = a.work_ctr != nullptr;
  for (int32_t w = dyn ? grab_item(a.work_ctr, &item_sh) : (int32_t)blockIdx.x; w < n_items;
       w = dyn ? grab_item(a.work_ctr, &item_sh) : w + (int32_t)gridDim.x) {
    const int32_t k = upper_bound_i32(a.item_off, a.K + 1, w) - 1;
    const int32_t B = a.bfac[k];
    const int32_t l = w - a.item_off[k];
    const int32_t it = l / B;
    const int32_t b = l - it * B;
    const int64_t sk0 = a.soff[k];
    const int64_t S_k = a.soff[k + 1] - sk0;
    // chunk b of B of the cluster's sources, or of this process's piece
    int64_t pb = 0, pe = S_k;
    if (a.parts > 1) src_piece(S_k, a.part, a.parts, &pb, &pe);
    const int64_t L = chunk_len(pe - pb, B, JT);
    const int64_t j0 = sk0 + pb + b * L;
    const int64_t j1 = sk0 + pb + min(pe - pb, (int64_t)(b + 1) * L);
    const int32_t a0 = a.act_off[k];
    const int32_t m_k = a.act_off[k + 1] - a0;
    const int64_t p0 = a.off[k], p1 = a.off[k + 1];

    Target64 s;
    const int32_t q = it * NI + tid;
    bool valid = q < m_k;
    s.x = s.y = s.z = s.vx = s.vy = s.vz = s.ax = s.ay = s.az = 0.0;
    s.slot = -1;
    if (valid) {
      const int64_t p = a.active ? (int64_t)a.active[a0 + q] : (int64_t)(a0 + q);
      if (p < p0 || p >= p1) {
        valid = false;
        atomicOr(a.status, kStatusInval);
      } else {
        s.slot = a.sinv ? (int64_t)a.sinv[p] : sk0 + (p - p0);
        const dbl4 ip = gp[s.slot];
        s.x = ip.x; s.y = ip.y; s.z = ip.z;
        if (MODE != kF64PotOnly) {
          const dbl4 iv = gv[s.slot];
          s.vx = iv.x; s.vy = iv.y; s.vz = iv.z;
        }
        if (MODE == kF64Snap) {
          const dbl4 ia = ga[s.slot];
          s.ax = ia.x; s.ay = ia.y; s.az = ia.z;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 10; ++c) { s.th[c] = 0.0; s.tl[c] = 0.0; }

    const int64_t ntile = ceil_div64(j1 - j0, JT);  // 0: an empty piece
    if (tid == 0 && ntile > 0) {
      issue64<MODE>(sp[0], sv[0], sa[0], &bar[0], gp, gv, ga, j0, min((int64_t)JT, j1 - j0));
      pending[0] = true;
      if (ntile > 1) {
        issue64<MODE>(sp[1], sv[1], sa[MODE == kF64Snap ? 1 : 0], &bar[1], gp, gv, ga, j0 + JT,
                      min((int64_t)JT, j1 - j0 - JT));
        pending[1] = true;
      }
    }
    for (int64_t t = 0; t < ntile; ++t) {
      const int st = static_cast<int>(t & 1);
      const int64_t t0 = j0 + t * JT;
      const int cnt = static_cast<int>(min((int64_t)JT, j1 - t0));
      const bool ok = mbar_wait(&bar[st], used[st] & 1u, kWaitBudget);
      used[st] += 1;
      if (tid == 0) pending[st] = false;
      if (!ok) {
        abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
      } else {
        const bool own = s.slot >= t0 && s.slot < t0 + cnt;
        if constexpr (MODE == kF64Snap) {
          if (own)
            tile_compute64_snap<true>(sp[st], sv[st], sa[st], cnt, t0, s, a.eps2);
          else
            tile_compute64_snap<false>(sp[st], sv[st], sa[st], cnt, t0, s, a.eps2);
        } else {
          if (own)
            tile_compute64<MODE, true>(sp[st], sv[st], cnt, t0, s, a.eps2);
          else
            tile_compute64<MODE, false>(sp[st], sv[st], cnt, t0, s, a.eps2);
        }
      }
      __syncthreads();
      if (abort_flag) goto drain;
      if (tid == 0 && t + 2 < ntile) {
        issue64<MODE>(sp[st], sv[st], sa[MODE == kF64Snap ? st : 0], &bar[st], gp, gv, ga,
                      t0 + 2 * JT, min((int64_t)JT, j1 - t0 - 2 * JT));
        pending[st] = true;
      }
    }

    if (valid) {
      double v[C];
      v[0] = s.th[0] + s.tl[0];
      v[1] = s.th[1] + s.tl[1];
      v[2] = s.th[2] + s.tl[2];
      if constexpr (MODE == kF64Snap) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          v[3 + c] = s.th[3 + c] + s.tl[3 + c];
          v[kPartialComps + c] = s.th[6 + c] + s.tl[6 + c];
        }
      } else {
        v[3] = (s.th[3] + s.tl[3]) - 3.0 * (s.th[6] + s.tl[6]);
        v[4] = (s.th[4] + s.tl[4]) - 3.0 * (s.th[7] + s.tl[7]);
        v[5] = (s.th[5] + s.tl[5]) - 3.0 * (s.th[8] + s.tl[8]);
      }
      v[6] = -(s.th[9] + s.tl[9]);
      if (B == 1) {
        int64_t srow = a0 + q;
        if (a.rows) srow = a.rows[srow];
        if (MODE != kF64PotOnly) {
          if (a.out_acc) for (int c = 0; c < 3; ++c) a.out_acc[srow * a.sa + c] = a.G * v[c];
          if (a.out_jerk) for (int c = 0; c < 3; ++c) a.out_jerk[srow * a.sj + c] = a.G * v[3 + c];
        }
        if (MODE == kF64Snap && a.out_snap)
          for (int c = 0; c < 3; ++c) a.out_snap[srow * a.ss + c] = a.G * v[kPartialComps + c];
        if (a.out_pot) a.out_pot[srow * a.sp] = a.G * v[6];
      } else {
        double* P = a.partials + (size_t)w * C * NI + tid;
#pragma unroll
        for (int c = 0; c < C; ++c) P[(size_t)c * NI] = v[c];
      }
    }
  }
  return;

drain:
  if (tid == 0) {
    for (int st = 0; st < 2; ++st)
      if (pending[st]) (void)mbar_wait(&bar[st], used[st] & 1u, kWaitBudget);
  }
}

}  // namespace

cudaError_t launch_force_fp64(const ForceArgs& a, int grid, int mode, cudaStream_t st) {
  if (mode == kF64PotOnly)
    return launch_chain(k_force_fp64<kF64PotOnly>, dim3(grid), dim3(NT), 0, st, a);
  if (mode == kF64Snap)
    return launch_chain(k_force_fp64<kF64Snap>, dim3(grid), dim3(NT), 0, st, a);
  return launch_chain(k_force_fp64<kF64Full>, dim3(grid), dim3(NT), 0, st, a);
}

int force_fp64_ctas_per_sm() {
  int n1 = 0, n2 = 0, n3 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_force_fp64<kF64Full>, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, k_force_fp64<kF64PotOnly>, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n3, k_force_fp64<kF64Snap>, NT, 0);
  int n = n1 < n2 ? n1 : n2;
  n = n < n3 ? n : n3;
  return n > 0 ? n : 1;
}

size_t force_fp64_smem() { return sizeof(dbl4) * 4 * JT; }

}  // namespace nb
