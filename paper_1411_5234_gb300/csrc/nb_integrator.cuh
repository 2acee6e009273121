// nb_integrator.cuh -- launch interface of the block-step kernels.
#pragma once
#include <math_constants.h>

#include "nb_internal.cuh"

namespace nb {

// Min or max of v over the threads of one cell (kMixJD = 64 threads, two
// warps) of a CTA of kMixJT threads; every thread gets its cell's result.
// `sh` holds >= kMixJT / 32 doubles.
__device__ __forceinline__ double nb_half_reduce_d(double v, bool is_max, double* sh) {
  static_assert(kMixJD == 64 && kMixJT % kMixJD == 0, "two warps per cell");
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmax(v, u) : fmin(v, u);
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[wid] = v;
  __syncthreads();
  const double a = sh[wid & ~1], b = sh[wid | 1];
  __syncthreads();
  return is_max ? fmax(a, b) : fmin(a, b);
}

// Write one mixed source tile (one CTA of kMixJT threads, one slot each).
// The tile holds kMixCells cells of kMixJD slots; for each cell: centre c = the
// midpoint of its valid particles' bounding box, rounded to a double-single
// pair (ch, cl), radius h = max |r_j - c| (rounded up).  Each valid slot
// stores its double-single offset r_j - c from its cell's centre, its mass
// and FP32 velocity; pad slots (in == true, valid == false) hold massless
// dummies far away.  Record of tile t: float4 [kTileRecF4 t + 2q] = (ch, h)
// and [kTileRecF4 t + 2q + 1] = (cl, 0) for cell q.  Every thread must call
// this.
__device__ __forceinline__ void build_mixed_tile(float4* src, float4* tiles, int64_t tile,
                                                 int64_t s, bool in, bool valid, double3 x,
                                                 double m, double3 v, double* sh) {
  const double inf = CUDART_INF;
  const double lx = nb_half_reduce_d(valid ? x.x : inf, false, sh);
  const double ly = nb_half_reduce_d(valid ? x.y : inf, false, sh);
  const double lz = nb_half_reduce_d(valid ? x.z : inf, false, sh);
  const double hx = nb_half_reduce_d(valid ? x.x : -inf, true, sh);
  const double hy = nb_half_reduce_d(valid ? x.y : -inf, true, sh);
  const double hz = nb_half_reduce_d(valid ? x.z : -inf, true, sh);
  const bool any = lx <= hx;
  const double cx = any ? 0.5 * (lx + hx) : 0.0, cy = any ? 0.5 * (ly + hy) : 0.0,
               cz = any ? 0.5 * (lz + hz) : 0.0;
  const float chx = __double2float_rn(cx), chy = __double2float_rn(cy), chz = __double2float_rn(cz);
  const float clx = __double2float_rn(cx - (double)chx), cly = __double2float_rn(cy - (double)chy),
              clz = __double2float_rn(cz - (double)chz);
  const double ux = (double)chx + (double)clx, uy = (double)chy + (double)cly,
               uz = (double)chz + (double)clz;  // the centre as represented
  const double dx = x.x - ux, dy = x.y - uy, dz = x.z - uz;
  const double r = valid ? sqrt(dx * dx + dy * dy + dz * dz) : 0.0;
  const double h = nb_half_reduce_d(r, true, sh);
  if (in) {
    float* g = reinterpret_cast<float*>(src + (s >> 2) * 10) + (s & 3);
    if (valid) {
      const float dxh = __double2float_rn(dx), dyh = __double2float_rn(dy),
                  dzh = __double2float_rn(dz);
      g[0] = dxh;
      g[4] = dyh;
      g[8] = dzh;
      g[12] = __double2float_rn(m);
      g[16] = __double2float_rn(v.x);
      g[20] = __double2float_rn(v.y);
      g[24] = __double2float_rn(v.z);
      g[28] = __double2float_rn(dx - (double)dxh);
      g[32] = __double2float_rn(dy - (double)dyh);
      g[36] = __double2float_rn(dz - (double)dzh);
    } else {
      g[0] = g[4] = g[8] = static_cast<float>(kDummyPos);
      g[12] = 0.f;
      g[16] = g[20] = g[24] = 0.f;
      g[28] = g[32] = g[36] = 0.f;
    }
  }
  if ((threadIdx.x & (kMixJD - 1)) == 0) {
    const int q = threadIdx.x / kMixJD;
    tiles[kTileRecF4 * tile + 2 * q] = make_float4(chx, chy, chz, __double2float_ru(h));
    tiles[kTileRecF4 * tile + 2 * q + 1] = make_float4(clx, cly, clz, 0.f);
  }
}

struct PlanArgs {
  int NI;               // targets per work item of the force kernel
  int JT;               // sources per tile of the force kernel
  int grid;             // persistent CTAs of the force kernel
  int forced_b;         // fixed i-split factor (0: chosen here)
  int64_t part_items;   // capacity of the partial-sum buffer in work items
  int step_mode;        // block step: adopt t_min as t_cur, reset t_min
  int count;            // add the interactions (and the step) to the counters
};

struct CorrectArgs {
  const int32_t* active;
  const int32_t* count_dev;  // device count (act_off[K]) or nullptr
  int64_t count_host;
  const double* acc; int sa;
  const double* jerk; int sj;
  const double* pot; int sp;  // nullptr: keep the stored potential
  const int64_t* t_tgt;       // per-cluster target time or nullptr
  int64_t t_fixed;
  double eta;
  int T, lmin, lmax;
};

cudaError_t launch_fill_i64(int64_t* p, int64_t n, int64_t v, cudaStream_t st);
cudaError_t launch_tmin(const Dev& d, int T, cudaStream_t st);
cudaError_t launch_predict(const Dev& d, const int64_t* t_tgt, int64_t t_fixed, int T, bool mix,
                           bool f64, bool count_due, cudaStream_t st);
cudaError_t launch_compact(const Dev& d, int T, cudaStream_t st);
cudaError_t launch_plan(const Dev& d, const PlanArgs& p, cudaStream_t st);
cudaError_t launch_reduce(const ForceArgs& a, int NI, bool with_acc, int64_t m_bound,
                          cudaStream_t st);
cudaError_t launch_correct(const Dev& d, const CorrectArgs& c, int64_t m_bound, cudaStream_t st);
cudaError_t launch_init_levels(const Dev& d, double eta_s, int T, int lmin, int lmax,
                               cudaStream_t st);
// caller list -> d.active (slot order), d.rows (caller rows), act_off
cudaError_t launch_list_to_slots(const Dev& d, const int32_t* list, int64_t m, cudaStream_t st);
cudaError_t launch_actoff_identity(const Dev& d, cudaStream_t st);
cudaError_t launch_energy(const Dev& d, const double* pot, int sp, int64_t lo, int64_t hi,
                          double* part, int nblk, double* out, cudaStream_t st);

cudaError_t launch_pack3(const double* src3, dbl4* dst, int64_t n, bool keep_w, cudaStream_t st);
cudaError_t launch_unpack3(const dbl4* src, double* dst3, int64_t n, cudaStream_t st);
cudaError_t launch_tcur_from_t(const Dev& d, cudaStream_t st);

}  // namespace nb
