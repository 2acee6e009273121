// nb_force_mixed.cuh -- mixed-precision direct-summation force kernel (sm_103a),
// templated on its shape.
//
// Computes, for each target i, Eq. 1 with the softening of Eq. 2 plus the
// jerk and potential:
//   a_i  =  sum_j m_j d / s^3,   jerk_i = sum_j m_j (w - 3 (d.w / s^2) d) / s^3,
//   pot_i = -sum_j m_j / s,       d = r_j - r_i, w = v_j - v_i, s^2 = d.d + eps^2
// (G applied on output).
//
// Precision (Sec. 2 item 4: DP resolution for the separations and the sums,
// SP for the rest, square roots included).  Sources are stored relative to
// the centre c_J of their tile of kMixJT spatially sorted slots, as
// double-single offsets delta_j = dh_j + dl_j from the centre c of their cell
// (kMixJD consecutive slots, two cells per tile); a target's position
// relative to the centre, e = c - r_i, is formed per cell in double-single
// (eh + el).
//   * near cells (some target of the warp within 2 cell radii h of the
//     centre, the own cell included): d = (dh_j + eh) + (dl_j + el), FP64-like
//     resolution for close pairs;
//   * far cells (every target of the warp beyond 2 h): d = dh_j + eh.  The
//     three roundings (of dh_j, of eh, of the sum) are at most
//     2^-24 (|delta_j| + |e| + |d|), and |e| <= |d| + |delta_j|, so the error
//     stays within 4 units of 2^-24 |d| whenever |delta_j| <= |d|, which
//     |e| > 2 h guarantees for every source of the cell: the separation keeps
//     the relative accuracy of the FP32 arithmetic after it, without the
//     cancellation that absolute FP32 positions suffer.
// Everything after the separation is FP32 (hardware rsqrt and reciprocal);
// the jerk term is formed per pair as m (w + t d) / s^3 with t = -3 d.w / s^2
// (its rounding is relative to |w| + 3 |d.w| |d| / s^2, the magnitude of the
// two terms taken apart); sums are accumulated per pipeline stage in FP32
// and folded into a compensated (hi, lo) FP32 pair per stage (two-sum), then
// combined in FP64.
//
// GB300 mapping:
//   * persistent CTAs take work items (cluster, i-tile, j-chunk) from a
//     device counter that the plan zeroes before every launch; the j-chunk
//     split is the i-splitting of Sec. 2 item 3 (Bfactor): B chunks of the
//     source range per i-tile, partial sums reduced afterwards in a fixed
//     order.  Items are handed out dynamically because the warp scheduler
//     favours older warps: with a fixed share per CTA the younger CTAs of an
//     SM finish late and run alone on their sub-partition, where one warp
//     cannot keep the FMA pipe busy (measured: 1 ms spread of finish times in
//     a 2.4 ms launch of identical shares);
//   * source tiles and their cell records (centre, radius) are staged in
//     shared memory (Sec. 2 item 5) by bulk copies (TMA engine,
//     cp.async.bulk), ST tiles per stage, into a two-stage ring guarded by
//     mbarriers; waits are bounded and report NB_ETIMEOUT instead of hanging;
//   * every pair operation is a packed f32x2 instruction over two sources,
//     feeding the FP32 pipe at full width; IPT targets per thread share each
//     shared-memory load.
//
// Shape parameters (MixShape): NT threads per CTA, IPT targets per thread
// (NT * IPT <= kMixNI targets per work item), POT computes the potential, RCP takes 1/s^2 from the
// SFU reciprocal instead of an FP32 multiply, SMT keeps the compensated
// totals in shared memory instead of registers, UNR unrolls the source loop,
// MINB is the CTAs-per-SM hint of __launch_bounds__, JERK false computes the
// acceleration (and potential) alone: no velocities, 12 f32x2 instructions
// per two interactions instead of 26 (for acceleration-only integrators),
// SEP the separation mode, NU unrolls the near-cell loop (it runs one target
// at a time, so its groups are independent chains worth interleaving), ST
// tiles of kMixJT sources per pipeline stage: the per-tile FP32 sums are
// folded into the compensated totals once per stage, so ST = 2 halves the
// flushes, syncs and waits (FP32 runs of 128 terms per lane instead of 64).
#pragma once
#include <type_traits>

#include "nb_internal.cuh"

namespace nb {
namespace mixk {

constexpr int JT = kMixJT;
constexpr int kGroupF4 = 10;                      // float4 per group of 4 sources
constexpr int kTileF4 = JT / 4 * kGroupF4;        // float4 per tile
constexpr uint32_t kGroupBytes = kGroupF4 * 16;
constexpr int kCellGroups = kMixJD / 4;           // groups of 4 sources per cell
// far cell: |e| > 2 h, which gives |d| > h >= |delta_j| for every source of
// the cell, the condition of the error bound above
constexpr float kFarRatio2 = 4.0f;

// component order inside a group of 4 sources (float4 index)
enum { cDXH = 0, cDYH, cDZH, cM, cVX, cVY, cVZ, cDXL, cDYL, cDZL };

// separation modes: the far/near vote of the mixed path; double-single
// separations for every cell; plain FP32 separations (no low words) for every
// cell, the targets' own cell still through the masked single-target loop
enum { kSepMixed = 0, kSepDS = 1, kSepFP32 = 2 };

template <int NT_, int IPT_, bool POT_, bool RCP_, bool SMT_, int UNR_, int MINB_,
          bool JERK_ = true, int SEP_ = kSepMixed, int NU_ = 1, int ST_ = 1, bool SNAP_ = false>
struct MixShape {
  static constexpr int NT = NT_, IPT = IPT_, NI = NT_ * IPT_, UNR = UNR_, MINB = MINB_;
  static constexpr bool POT = POT_, RCP = RCP_, SMT = SMT_, JERK = JERK_, SNAP = SNAP_;
  static constexpr int SEP = SEP_, NU = NU_, ST = ST_;
  // compensated totals (and partial-sum components) per target
  static constexpr int TC = SNAP_ ? kPartialCompsSnap : kPartialComps;
  static_assert(NT_ * IPT_ <= kMixNI, "partial-sum rows hold at most kMixNI targets");
  static_assert(!SNAP_ || JERK_, "the snap needs the jerk terms");
};

// What the source loop needs of one target in registers; the target's
// absolute double-single position and its slot stay in shared memory.
struct Target {
  f2 nvx, nvy, nvz;              // -v_i as broadcast pairs
  f2 ex, ey, ez;                 // hi part of c_J - r_i (broadcast)
  f2 ax, ay, az, jx, jy, jz, pt; // per-stage sums (2 lanes)
};
// ... and of a snap shape (kept apart, so that the other shapes compile to
// the same code as without the snap)
struct TargetS : Target {
  f2 nax, nay, naz;              // -a_i (the predicted acceleration, broadcast)
  f2 sx, sy, sz;                 // per-stage snap sums
};
template <class Sh>
using TargetOf = typename std::conditional<Sh::SNAP, TargetS, Target>::type;

// compensated totals per target: a (3), jerk (3), potential, [snap (3)]
constexpr int kTotComps = kPartialCompsSnap;

// Per-thread shared-memory record of a target: r_i as double-single and its
// source slot (-1: no target); component-major so a warp's loads are
// conflict-free.
template <int IPT, int NT>
struct TargetPosSh {
  float c[IPT][6][NT];
  long long slot[IPT][NT];
};
struct TargetPos {
  float xh, yh, zh, xl, yl, zl;
  long long slot;
};
template <int IPT, int NT>
__device__ __forceinline__ TargetPos load_tpos(const TargetPosSh<IPT, NT>& t, int r, int tid) {
  return TargetPos{t.c[r][0][tid], t.c[r][1][tid], t.c[r][2][tid], t.c[r][3][tid],
                   t.c[r][4][tid], t.c[r][5][tid], t.slot[r][tid]};
}

__device__ __forceinline__ f2 bcast(float v) { return f2_pack(v, v); }

// (ah + al) - (bh + bl) in double-single, renormalised.
__device__ __forceinline__ void ds_sub(float ah, float al, float bh, float bl, float& rh,
                                       float& rl) {
  const float s = ah - bh;
  const float bb = s - ah;
  float err = (ah - (s - bb)) + (-bh - bb);
  err += al - bl;
  rh = s + err;
  rl = err - (rh - s);
}

// c - (bh + bl) in double-single for an FP32 value c (a cell centre, whose
// double-single low part is zero).
__device__ __forceinline__ void ds_sub0(float c, float bh, float bl, float& rh, float& rl) {
  const float s = c - bh;
  const float bb = s - c;
  float err = (c - (s - bb)) + (-bh - bb);
  err -= bl;
  rh = s + err;
  rl = err - (rh - s);
}

// One pair step, from the separation d and relative velocity w to the
// accumulators: pair_head forms 1/s, m/s^3, the potential and acceleration
// terms (shared by every shape); pair_tail adds the jerk term.
template <class Sh, bool MASK>
__device__ __forceinline__ void pair_head(Target& s, f2 dx, f2 dy, f2 dz, f2 m, f2 eps2,
                                          int64_t js, int64_t slot, f2& mr3, f2& r2inv) {
  f2 r2 = f2_fma(dx, dx, eps2);
  r2 = f2_fma(dy, dy, r2);
  r2 = f2_fma(dz, dz, r2);
  f2 rinv = f2_rsqrt(r2);
  f2 rr = Sh::RCP ? f2_rcp(r2) : 0ull;
  if (MASK) {  // j == i is excluded by index (Eq. 1)
    float2 a = f2_unpack(rinv), c = f2_unpack(rr);
    if (js == slot) a.x = c.x = 0.f;
    if (js + 1 == slot) a.y = c.y = 0.f;
    rinv = f2_pack(a.x, a.y);
    rr = f2_pack(c.x, c.y);
  }
  r2inv = Sh::RCP ? rr : f2_mul(rinv, rinv);
  const f2 mri = f2_mul(m, rinv);
  mr3 = f2_mul(mri, r2inv);
  if (Sh::POT) s.pt = f2_add(s.pt, mri);
  s.ax = f2_fma(mr3, dx, s.ax);
  s.ay = f2_fma(mr3, dy, s.ay);
  s.az = f2_fma(mr3, dz, s.az);
}

template <class Sh, bool MASK>
__device__ __forceinline__ void pair_tail(Target& s, f2 dx, f2 dy, f2 dz, f2 wx, f2 wy, f2 wz,
                                          f2 m, f2 eps2, int64_t js, int64_t slot) {
  f2 mr3, r2inv;
  pair_head<Sh, MASK>(s, dx, dy, dz, m, eps2, js, slot, mr3, r2inv);
  if constexpr (Sh::JERK) {
    f2 rv = f2_mul(dx, wx);
    rv = f2_fma(dy, wy, rv);
    rv = f2_fma(dz, wz, rv);
    const f2 t = f2_mul(f2_mul(rv, r2inv), f2_pack(-3.f, -3.f));  // -3 d.w / s^2
    s.jx = f2_fma(mr3, f2_fma(t, dx, wx), s.jx);
    s.jy = f2_fma(mr3, f2_fma(t, dy, wy), s.jy);
    s.jz = f2_fma(mr3, f2_fma(t, dz, wz), s.jz);
  } else {
    (void)wx; (void)wy; (void)wz;
  }
}

// The snap shapes' tail: also u = a_j - a_i, and the snap term
// m (u - 6 alpha (w - 3 alpha d) - 3 beta d) / s^3, alpha = d.w / s^2,
// beta = (w.w + d.u) / s^2 + alpha^2 (the second time derivative of the pair
// term of Eq. 2; 22 more FP32 lane-ops per interaction).
template <class Sh, bool MASK>
__device__ __forceinline__ void pair_tail_snap(TargetS& s, f2 dx, f2 dy, f2 dz, f2 wx, f2 wy,
                                               f2 wz, f2 ux, f2 uy, f2 uz, f2 m, f2 eps2,
                                               int64_t js, int64_t slot) {
  f2 mr3, r2inv;
  pair_head<Sh, MASK>(s, dx, dy, dz, m, eps2, js, slot, mr3, r2inv);
  f2 rv = f2_mul(dx, wx);
  rv = f2_fma(dy, wy, rv);
  rv = f2_fma(dz, wz, rv);
  f2 wdu = f2_mul(wx, wx);  // w.w + d.u
  wdu = f2_fma(wy, wy, wdu);
  wdu = f2_fma(wz, wz, wdu);
  wdu = f2_fma(dx, ux, wdu);
  wdu = f2_fma(dy, uy, wdu);
  wdu = f2_fma(dz, uz, wdu);
  const f2 r2m3 = f2_mul(r2inv, f2_pack(-3.f, -3.f));
  const f2 t = f2_mul(rv, r2m3);                 // -3 alpha
  const f2 alpha = f2_mul(rv, r2inv);
  const f2 c2 = f2_fma(alpha, t, f2_mul(wdu, r2m3));  // -3 beta
  const f2 c1 = f2_add(t, t);                    // -6 alpha
  const f2 jx = f2_fma(t, dx, wx), jy = f2_fma(t, dy, wy), jz = f2_fma(t, dz, wz);
  s.jx = f2_fma(mr3, jx, s.jx);
  s.jy = f2_fma(mr3, jy, s.jy);
  s.jz = f2_fma(mr3, jz, s.jz);
  s.sx = f2_fma(mr3, f2_fma(c2, dx, f2_fma(c1, jx, ux)), s.sx);
  s.sy = f2_fma(mr3, f2_fma(c2, dy, f2_fma(c1, jy, uy)), s.sy);
  s.sz = f2_fma(mr3, f2_fma(c2, dz, f2_fma(c1, jz, uz)), s.sz);
}

// Source accelerations of the snap shapes: 3 float4 per group of 4 slots
// ([ax][ay][az]), beside the group's 10 float4.
constexpr int kAccGroupF4 = 3;
constexpr int kAccTileF4 = JT / 4 * kAccGroupF4;

// Far cell: d = dh_j + eh.  NG > 0: a full cell with a compile-time trip
// count (no remainder code, better interleaving); NG == 0: ngroups groups.
template <class Sh, int NG = 0>
__device__ __forceinline__ void tile_far(const float4* __restrict__ tile,
                                         const float4* __restrict__ acc, int ngroups,
                                         TargetOf<Sh> (&tg)[Sh::IPT], f2 eps2, uint32_t live) {
  const int n = NG > 0 ? NG : ngroups;
#pragma unroll Sh::UNR
  for (int g = 0; g < n; ++g) {
    const ulonglong2* G = reinterpret_cast<const ulonglong2*>(tile + g * kGroupF4);
    const ulonglong2 dxh = G[cDXH], dyh = G[cDYH], dzh = G[cDZH], m = G[cM], vx = G[cVX],
                     vy = G[cVY], vz = G[cVZ];
    if constexpr (Sh::SNAP) {
      const ulonglong2* A = reinterpret_cast<const ulonglong2*>(acc + g * kAccGroupF4);
      const ulonglong2 ax = A[0], ay = A[1], az = A[2];
#pragma unroll
      for (int r = 0; r < Sh::IPT; ++r) {
        if constexpr (Sh::IPT <= 2) {
          if (!((live >> r) & 1u)) continue;  // no active target in this row of the warp
        }
        TargetS& s = tg[r];
        pair_tail_snap<Sh, false>(s, f2_add(dxh.x, s.ex), f2_add(dyh.x, s.ey),
                                  f2_add(dzh.x, s.ez), f2_add(vx.x, s.nvx), f2_add(vy.x, s.nvy),
                                  f2_add(vz.x, s.nvz), f2_add(ax.x, s.nax), f2_add(ay.x, s.nay),
                                  f2_add(az.x, s.naz), m.x, eps2, 0, -1);
        pair_tail_snap<Sh, false>(s, f2_add(dxh.y, s.ex), f2_add(dyh.y, s.ey),
                                  f2_add(dzh.y, s.ez), f2_add(vx.y, s.nvx), f2_add(vy.y, s.nvy),
                                  f2_add(vz.y, s.nvz), f2_add(ax.y, s.nax), f2_add(ay.y, s.nay),
                                  f2_add(az.y, s.naz), m.y, eps2, 0, -1);
      }
    } else {
      (void)acc;
#pragma unroll
      for (int r = 0; r < Sh::IPT; ++r) {
        if constexpr (Sh::IPT <= 2) {
          if (!((live >> r) & 1u)) continue;  // no active target in this row of the warp
        }
        Target& s = tg[r];
        pair_tail<Sh, false>(s, f2_add(dxh.x, s.ex), f2_add(dyh.x, s.ey), f2_add(dzh.x, s.ez),
                             f2_add(vx.x, s.nvx), f2_add(vy.x, s.nvy), f2_add(vz.x, s.nvz), m.x,
                             eps2, 0, -1);
        pair_tail<Sh, false>(s, f2_add(dxh.y, s.ex), f2_add(dyh.y, s.ey), f2_add(dzh.y, s.ez),
                             f2_add(vx.y, s.nvx), f2_add(vy.y, s.nvy), f2_add(vz.y, s.nvz), m.y,
                             eps2, 0, -1);
      }
    }
  }
}

// Near cell, one target: d = (dh_j + eh) + (dl_j + el).  Near cells are a
// small fraction, so each target takes its own pass over the cell and only
// one target's low parts are live at a time.  (Plain FP32 separation mode:
// d = dh_j + eh, the low words unused.)
template <class Sh, bool MASK>
__device__ __forceinline__ void tile_near_one(const float4* __restrict__ tile,
                                              const float4* __restrict__ acc, int ngroups,
                                              int64_t slot0, TargetOf<Sh>& s, f2 elx, f2 ely,
                                              f2 elz, int64_t slot, f2 eps2) {
#pragma unroll Sh::NU
  for (int g = 0; g < ngroups; ++g) {
    const ulonglong2* G = reinterpret_cast<const ulonglong2*>(tile + g * kGroupF4);
    const ulonglong2 dxh = G[cDXH], dyh = G[cDYH], dzh = G[cDZH], m = G[cM], vx = G[cVX],
                     vy = G[cVY], vz = G[cVZ], dxl = G[cDXL], dyl = G[cDYL], dzl = G[cDZL];
    const int64_t js = slot0 + 4 * g;
    f2 dx0, dy0, dz0, dx1, dy1, dz1;
    if constexpr (Sh::SEP == kSepFP32) {
      dx0 = f2_add(dxh.x, s.ex);
      dy0 = f2_add(dyh.x, s.ey);
      dz0 = f2_add(dzh.x, s.ez);
      dx1 = f2_add(dxh.y, s.ex);
      dy1 = f2_add(dyh.y, s.ey);
      dz1 = f2_add(dzh.y, s.ez);
      (void)dxl; (void)dyl; (void)dzl; (void)elx; (void)ely; (void)elz;
    } else {
      dx0 = f2_add(f2_add(dxh.x, s.ex), f2_add(dxl.x, elx));
      dy0 = f2_add(f2_add(dyh.x, s.ey), f2_add(dyl.x, ely));
      dz0 = f2_add(f2_add(dzh.x, s.ez), f2_add(dzl.x, elz));
      dx1 = f2_add(f2_add(dxh.y, s.ex), f2_add(dxl.y, elx));
      dy1 = f2_add(f2_add(dyh.y, s.ey), f2_add(dyl.y, ely));
      dz1 = f2_add(f2_add(dzh.y, s.ez), f2_add(dzl.y, elz));
    }
    if constexpr (Sh::SNAP) {
      const ulonglong2* A = reinterpret_cast<const ulonglong2*>(acc + g * kAccGroupF4);
      const ulonglong2 ax = A[0], ay = A[1], az = A[2];
      pair_tail_snap<Sh, MASK>(s, dx0, dy0, dz0, f2_add(vx.x, s.nvx), f2_add(vy.x, s.nvy),
                               f2_add(vz.x, s.nvz), f2_add(ax.x, s.nax), f2_add(ay.x, s.nay),
                               f2_add(az.x, s.naz), m.x, eps2, js, slot);
      pair_tail_snap<Sh, MASK>(s, dx1, dy1, dz1, f2_add(vx.y, s.nvx), f2_add(vy.y, s.nvy),
                               f2_add(vz.y, s.nvz), f2_add(ax.y, s.nax), f2_add(ay.y, s.nay),
                               f2_add(az.y, s.naz), m.y, eps2, js + 2, slot);
    } else {
      (void)acc;
      pair_tail<Sh, MASK>(s, dx0, dy0, dz0, f2_add(vx.x, s.nvx), f2_add(vy.x, s.nvy),
                          f2_add(vz.x, s.nvz), m.x, eps2, js, slot);
      pair_tail<Sh, MASK>(s, dx1, dy1, dz1, f2_add(vx.y, s.nvx), f2_add(vy.y, s.nvy),
                          f2_add(vz.y, s.nvz), m.y, eps2, js + 2, slot);
    }
  }
}

__device__ __forceinline__ float lanes_sum(f2& v) {
  const float2 p = f2_unpack(v);
  v = 0ull;
  return p.x + p.y;
}

// Compensated totals of one target: TC (hi, lo) pairs, in registers or in
// shared memory (one column per thread).
template <bool SMT, int NT, int TC>
struct Totals {
  float h[TC], l[TC];
  __device__ __forceinline__ void zero(float*) {
#pragma unroll
    for (int c = 0; c < TC; ++c) h[c] = l[c] = 0.f;
  }
  __device__ __forceinline__ void add(float*, int c, float x) { two_sum_acc(h[c], l[c], x); }
  __device__ __forceinline__ double get(float*, int c) const { return (double)h[c] + (double)l[c]; }
};
template <int NT, int TC>
struct Totals<true, NT, TC> {
  // column of this thread: col[(2 c) NT] = hi, col[(2 c + 1) NT] = lo
  __device__ __forceinline__ void zero(float* col) {
#pragma unroll
    for (int c = 0; c < 2 * TC; ++c) col[c * NT] = 0.f;
  }
  // components c, c + 1 at once: packed two-sum of x = (x_c, x_c+1)
  __device__ __forceinline__ void add2(float* col, int c, f2 x) {
    const f2 h = f2_pack(col[(2 * c) * NT], col[(2 * c + 2) * NT]);
    f2 l = f2_pack(col[(2 * c + 1) * NT], col[(2 * c + 3) * NT]);
    const f2 sm = f2_add(h, x);
    const f2 bp = f2_sub(sm, h);
    l = f2_add(l, f2_add(f2_sub(h, f2_sub(sm, bp)), f2_sub(x, bp)));
    const float2 hh = f2_unpack(sm), ll = f2_unpack(l);
    col[(2 * c) * NT] = hh.x;
    col[(2 * c + 2) * NT] = hh.y;
    col[(2 * c + 1) * NT] = ll.x;
    col[(2 * c + 3) * NT] = ll.y;
  }
  __device__ __forceinline__ void add(float* col, int c, float x) {
    float hi = col[(2 * c) * NT], lo = col[(2 * c + 1) * NT];
    two_sum_acc(hi, lo, x);
    col[(2 * c) * NT] = hi;
    col[(2 * c + 1) * NT] = lo;
  }
  __device__ __forceinline__ double get(float* col, int c) const {
    return (double)col[(2 * c) * NT] + (double)col[(2 * c + 1) * NT];
  }
};

// (a.x + a.y, b.x + b.y), clearing a and b
__device__ __forceinline__ f2 lanes_sum2(f2& a, f2& b) {
  const float2 pa = f2_unpack(a), pb = f2_unpack(b);
  a = 0ull;
  b = 0ull;
  return f2_add(f2_pack(pa.x, pb.x), f2_pack(pa.y, pb.y));
}

template <class Sh>
__device__ __forceinline__ void flush(TargetOf<Sh>& s, Totals<Sh::SMT, Sh::NT, Sh::TC>& T,
                                      float* col) {
  if constexpr (!Sh::JERK) {  // acceleration (and potential) only
    if constexpr (Sh::SMT) {
      T.add2(col, 0, lanes_sum2(s.ax, s.ay));
    } else {
      T.add(col, 0, lanes_sum(s.ax));
      T.add(col, 1, lanes_sum(s.ay));
    }
    T.add(col, 2, lanes_sum(s.az));
  } else if constexpr (Sh::SMT) {  // packed two-sums, two components at a time
    T.add2(col, 0, lanes_sum2(s.ax, s.ay));
    T.add2(col, 2, lanes_sum2(s.az, s.jx));
    T.add2(col, 4, lanes_sum2(s.jy, s.jz));
  } else {
    T.add(col, 0, lanes_sum(s.ax));
    T.add(col, 1, lanes_sum(s.ay));
    T.add(col, 2, lanes_sum(s.az));
    T.add(col, 3, lanes_sum(s.jx));
    T.add(col, 4, lanes_sum(s.jy));
    T.add(col, 5, lanes_sum(s.jz));
  }
  if constexpr (Sh::SNAP) {
    if constexpr (Sh::SMT) {
      T.add2(col, 7, lanes_sum2(s.sx, s.sy));
    } else {
      T.add(col, 7, lanes_sum(s.sx));
      T.add(col, 8, lanes_sum(s.sy));
    }
    T.add(col, 9, lanes_sum(s.sz));
  }
  if (Sh::POT) T.add(col, 6, lanes_sum(s.pt));
}

// Slots t0 .. t0 + cnt (cnt a multiple of 4, at most a stage) plus the cell
// records (centre, radius) of the tiles they span; t0 starts a tile.
// Snap shapes (acc != nullptr) also copy the slots' accelerations.
__device__ __forceinline__ void issue_tile(float4* stage, float4* rec, float4* stage_acc,
                                           uint64_t* bar, const float4* src, const float4* tiles,
                                           const float4* acc, int64_t t0, int64_t cnt,
                                           int64_t tile_idx) {
  const uint32_t bytes = static_cast<uint32_t>(cnt / 4) * kGroupBytes;
  const uint32_t rec_bytes = 16u * kTileRecF4 * static_cast<uint32_t>(ceil_div64(cnt, JT));
  const uint32_t acc_bytes = acc ? static_cast<uint32_t>(cnt / 4) * 16u * kAccGroupF4 : 0u;
  mbar_arrive_expect(bar, bytes + rec_bytes + acc_bytes);
  bulk_g2s(stage, src + (t0 >> 2) * kGroupF4, bytes, bar);
  bulk_g2s(rec, tiles + kTileRecF4 * tile_idx, rec_bytes, bar);
  if (acc) bulk_g2s(stage_acc, acc + (t0 >> 2) * kAccGroupF4, acc_bytes, bar);
}

template <class Sh>
__global__ void __launch_bounds__(Sh::NT, Sh::MINB) k_force_mixed(const ForceArgs a) {
  pdl_wait();  // the previous kernel of the chain has completed
  pdl_launch();
  constexpr int NT = Sh::NT, IPT = Sh::IPT, NI = Sh::NI;
  constexpr int SJ = Sh::ST * JT;  // sources per pipeline stage
  // a block step launches every shape of its autotune table; only the one
  // the plan chose for this step's active count works
  if (a.sel && a.sel[0] != a.my_variant) return;
  __shared__ __align__(128) float4 stage[2][Sh::ST * kTileF4];
  __shared__ __align__(16) float4 rec[2][Sh::ST * kTileRecF4];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int abort_flag;
  __shared__ int32_t item_sh;
  constexpr int TC = Sh::TC;
  __shared__ __align__(16) float4 stage_acc[Sh::SNAP ? 2 : 1][Sh::SNAP ? Sh::ST * kAccTileF4 : 1];
  __shared__ float tot_sh[Sh::SMT ? IPT * 2 * TC * NT : 1];
  __shared__ TargetPosSh<IPT, NT> tpos;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    abort_flag = 0;
  }
  __syncthreads();
  uint32_t used[2] = {0u, 0u};  // completed phases per stage
  bool pending[2] = {false, false};
  const float4* __restrict__ src = static_cast<const float4*>(a.src_a);
  const float4* __restrict__ tiles = a.tiles;
  // snap shapes: the sources' predicted accelerations (3 float4 per group)
  const float4* __restrict__ gacc = Sh::SNAP ? static_cast<const float4*>(a.src_c) : nullptr;
  const float e2 = static_cast<float>(a.eps2);
  const f2 eps2 = f2_pack(e2, e2);
  const int32_t n_items = a.item_off[a.K];

  // dynamic item order when the plan provided a counter, else a fixed share
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
    // the item's j-chunk: chunk b of B of the cluster's sources, or of this
    // process's piece of them in a j-partition
    int64_t pb = 0, pe = S_k;
    if (a.parts > 1) src_piece(S_k, a.part, a.parts, &pb, &pe);
    const int64_t L = chunk_len(pe - pb, B, JT);
    const int64_t j0 = sk0 + pb + b * L;
    const int64_t j1 = sk0 + pb + min(pe - pb, (int64_t)(b + 1) * L);
    const int64_t tk0 = a.toff[k];
    const int32_t a0 = a.act_off[k];
    const int32_t m_k = a.act_off[k + 1] - a0;
    const int64_t p0 = a.off[k], p1 = a.off[k + 1];

    TargetOf<Sh> tg[IPT];
    Totals<Sh::SMT, NT, TC> tot[IPT];
    bool valid[IPT];
    // warp wp owns the 32 * IPT consecutive targets [wp * 32 * IPT, ...):
    // target r of lane ln is wp * 32 * IPT + r * 32 + ln (spatially compact
    // warps, coalesced rows per r)
    const int wp = tid >> 5, ln = tid & 31;
#pragma unroll
    for (int r = 0; r < IPT; ++r) {
      const int32_t q = it * NI + wp * 32 * IPT + r * 32 + ln;
      valid[r] = q < m_k;
      float xh = 0.f, yh = 0.f, zh = 0.f, xl = 0.f, yl = 0.f, zl = 0.f, vx = 0.f, vy = 0.f,
            vz = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
      long long slot_r = -1;
      if (valid[r]) {
        const int32_t s = a0 + q;
        const int64_t p = a.active ? (int64_t)a.active[s] : (int64_t)s;
        if (p < p0 || p >= p1) {
          valid[r] = false;
          atomicOr(a.status, kStatusInval);
        } else {
          const int64_t slot = a.sinv ? (int64_t)a.sinv[p] : sk0 + (p - p0);
          const float* gp =
              reinterpret_cast<const float*>(src + (slot >> 2) * kGroupF4) + (slot & 3);
          // absolute position = own cell centre + offset, in double-single
          const float4* tr = tiles + kTileRecF4 * (tk0 + (slot - sk0) / JT) +
                             2 * (((slot - sk0) % JT) / kMixJD);
          const float4 ch = tr[0], cl = tr[1];
          ds_sub(ch.x, cl.x, -gp[4 * cDXH], -gp[4 * cDXL], xh, xl);
          ds_sub(ch.y, cl.y, -gp[4 * cDYH], -gp[4 * cDYL], yh, yl);
          ds_sub(ch.z, cl.z, -gp[4 * cDZH], -gp[4 * cDZL], zh, zl);
          vx = gp[4 * cVX];
          vy = gp[4 * cVY];
          vz = gp[4 * cVZ];
          if constexpr (Sh::SNAP) {
            const float* ga =
                reinterpret_cast<const float*>(gacc + (slot >> 2) * kAccGroupF4) + (slot & 3);
            ax = ga[0];
            ay = ga[4];
            az = ga[8];
          }
          slot_r = slot;
        }
      }
      tpos.c[r][0][tid] = xh;
      tpos.c[r][1][tid] = yh;
      tpos.c[r][2][tid] = zh;
      tpos.c[r][3][tid] = xl;
      tpos.c[r][4][tid] = yl;
      tpos.c[r][5][tid] = zl;
      tpos.slot[r][tid] = slot_r;
      tg[r].nvx = bcast(-vx); tg[r].nvy = bcast(-vy); tg[r].nvz = bcast(-vz);
      tg[r].ax = tg[r].ay = tg[r].az = 0ull;
      tg[r].jx = tg[r].jy = tg[r].jz = 0ull;
      tg[r].pt = 0ull;
      if constexpr (Sh::SNAP) {
        tg[r].nax = bcast(-ax); tg[r].nay = bcast(-ay); tg[r].naz = bcast(-az);
        tg[r].sx = tg[r].sy = tg[r].sz = 0ull;
      } else {
        (void)ax; (void)ay; (void)az;
      }
      tot[r].zero(tot_sh + r * 2 * TC * NT + tid);
    }
    // the rows of this warp's targets that hold an active target: the
    // 2-target shapes, which serve small active sets, skip the others (with
    // m below an item's width whole rows are empty); bit r for row r
    uint32_t live = (1u << IPT) - 1u;
    if constexpr (IPT <= 2) {
      live = 0u;
#pragma unroll
      for (int r = 0; r < IPT; ++r)
        if (__any_sync(0xffffffffu, valid[r])) live |= 1u << r;
    }

    // pipeline stages of SJ slots (the chunk starts on a tile boundary)
    const int64_t ntile = ceil_div64(j1 - j0, SJ);  // 0: an empty piece
    uint32_t n_near = 0;  // cells this warp took on the near path
    if (tid == 0 && ntile > 0) {
      issue_tile(stage[0], rec[0], stage_acc[0], &bar[0], src, tiles, gacc, j0,
                 min((int64_t)SJ, j1 - j0), tk0 + (j0 - sk0) / JT);
      pending[0] = true;
      if (ntile > 1) {
        issue_tile(stage[1], rec[1], stage_acc[Sh::SNAP ? 1 : 0], &bar[1], src, tiles, gacc,
                   j0 + SJ, min((int64_t)SJ, j1 - j0 - SJ), tk0 + (j0 - sk0) / JT + Sh::ST);
        pending[1] = true;
      }
    }
    for (int64_t t = 0; t < ntile; ++t) {
      const int st = static_cast<int>(t & 1);
      const int64_t t0 = j0 + t * SJ;
      const int64_t cnt = min((int64_t)SJ, j1 - t0);
      const bool ok_me = mbar_wait(&bar[st], used[st] & 1u, kWaitBudget);
      used[st] += 1;
      if (tid == 0) pending[st] = false;
      if (!ok_me) {
        abort_flag = 1;
        atomicOr(a.status, kStatusTimeout);
      }
      // one decision for the whole CTA, so every thread takes the same path
      // through the warp votes below
      const bool ok = __syncthreads_and(ok_me) != 0;
      const int ng = ok ? static_cast<int>(cnt >> 2) : 0;
#pragma unroll 1
      for (int q = 0; q < Sh::ST * kMixCells; ++q) {
        const int g0 = q * kCellGroups;
        const int ngq = min(ng - g0, kCellGroups);
        if (ngq <= 0) break;  // uniform: ng is the same in every thread
        // the centre is an FP32 point (its double-single low part is zero)
        const float4 ch = rec[st][2 * q];
        const float far_lim = kFarRatio2 * ch.w * ch.w;
        bool far = true;
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
          const TargetPos tp = load_tpos(tpos, r, tid);
          float exh, exl, eyh, eyl, ezh, ezl;
          ds_sub0(ch.x, tp.xh, tp.xl, exh, exl);
          ds_sub0(ch.y, tp.yh, tp.yl, eyh, eyl);
          ds_sub0(ch.z, tp.zh, tp.zl, ezh, ezl);
          tg[r].ex = bcast(exh);
          tg[r].ey = bcast(eyh);
          tg[r].ez = bcast(ezh);
          const float d2 = exh * exh + eyh * eyh + ezh * ezh;
          far = far && (!valid[r] || d2 > far_lim);
        }
        const float4* cell = stage[st] + g0 * kGroupF4;
        const float4* cacc = Sh::SNAP ? stage_acc[st] + g0 * kAccGroupF4 : nullptr;
        const int64_t c0 = t0 + 4 * g0;
        bool take_far;
        if constexpr (Sh::SEP == kSepMixed) {
          take_far = __all_sync(0xffffffffu, far);
        } else if constexpr (Sh::SEP == kSepDS) {
          take_far = false;
        } else {  // FP32: far arithmetic unless the cell holds a target of the warp
          bool own = false;
#pragma unroll
          for (int r = 0; r < IPT; ++r) {
            const long long sl = tpos.slot[r][tid];
            own = own || (sl >= c0 && sl < c0 + 4 * ngq);
          }
          take_far = !__any_sync(0xffffffffu, own);
        }
        if (take_far) {
          if (ngq == kCellGroups)
            tile_far<Sh, kCellGroups>(cell, cacc, ngq, tg, eps2, live);
          else
            tile_far<Sh>(cell, cacc, ngq, tg, eps2, live);
        } else {
          ++n_near;
#pragma unroll
          for (int r = 0; r < IPT; ++r) {
            if constexpr (IPT <= 2) {
              if (!((live >> r) & 1u)) continue;
            }
            const TargetPos tp = load_tpos(tpos, r, tid);
            float h, lx, ly, lz;
            ds_sub0(ch.x, tp.xh, tp.xl, h, lx);
            ds_sub0(ch.y, tp.yh, tp.yl, h, ly);
            ds_sub0(ch.z, tp.zh, tp.zl, h, lz);
            // the slot test excludes j == i where the target's own cell is near
            tile_near_one<Sh, true>(cell, cacc, ngq, c0, tg[r], bcast(lx), bcast(ly),
                                    bcast(lz), tp.slot, eps2);
          }
        }
      }
      if (ok) {
#pragma unroll
        for (int r = 0; r < IPT; ++r) flush<Sh>(tg[r], tot[r], tot_sh + r * 2 * TC * NT + tid);
      }
      __syncthreads();
      if (abort_flag) goto drain;
      if (tid == 0 && t + 2 < ntile) {
        issue_tile(stage[st], rec[st], stage_acc[Sh::SNAP ? st : 0], &bar[st], src, tiles, gacc,
                   t0 + 2 * SJ, min((int64_t)SJ, j1 - t0 - 2 * SJ),
                   tk0 + (t0 - sk0) / JT + 2 * Sh::ST);
        pending[st] = true;
      }
    }

    if (ln == 0 && a.tile_counts) {
      atomicAdd(a.tile_counts, (unsigned long long)ceil_div64(j1 - j0, kMixJD));
      atomicAdd(a.tile_counts + 1, (unsigned long long)n_near);
    }
#pragma unroll
    for (int r = 0; r < IPT; ++r) {
      if (!valid[r]) continue;
      float* col = tot_sh + r * 2 * TC * NT + tid;
      double v[TC];
      v[0] = tot[r].get(col, 0);
      v[1] = tot[r].get(col, 1);
      v[2] = tot[r].get(col, 2);
      v[3] = Sh::JERK ? tot[r].get(col, 3) : 0.0;
      v[4] = Sh::JERK ? tot[r].get(col, 4) : 0.0;
      v[5] = Sh::JERK ? tot[r].get(col, 5) : 0.0;
      v[6] = Sh::POT ? -tot[r].get(col, 6) : 0.0;
      if constexpr (Sh::SNAP) {
        v[7] = tot[r].get(col, 7);
        v[8] = tot[r].get(col, 8);
        v[9] = tot[r].get(col, 9);
      }
      const int32_t ql = wp * 32 * IPT + r * 32 + ln;
      if (B == 1) {
        int64_t srow = a0 + it * NI + ql;
        if (a.rows) srow = a.rows[srow];
        if (a.out_acc) for (int c = 0; c < 3; ++c) a.out_acc[srow * a.sa + c] = a.G * v[c];
        if (Sh::JERK && a.out_jerk)
          for (int c = 0; c < 3; ++c) a.out_jerk[srow * a.sj + c] = a.G * v[3 + c];
        if (Sh::POT && a.out_pot) a.out_pot[srow * a.sp] = a.G * v[6];
        if constexpr (Sh::SNAP) {
          if (a.out_snap)
            for (int c = 0; c < 3; ++c) a.out_snap[srow * a.ss + c] = a.G * v[kPartialComps + c];
        }
      } else {
        double* P = a.partials + (size_t)w * TC * NI + ql;
#pragma unroll
        for (int c = 0; c < TC; ++c) P[(size_t)c * NI] = v[c];
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

}  // namespace mixk
}  // namespace nb
