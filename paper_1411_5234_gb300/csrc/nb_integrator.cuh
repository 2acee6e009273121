// nb_integrator.cuh -- launch interface of the block-step kernels.
#pragma once
#include <math_constants.h>

#include "nb_internal.cuh"

namespace nb {

// i-split factors up to kReduceSerial are reduced by one lane per target
// (k_reduce); larger ones, in the same kernel, in segments of kWideRows partial
// rows (one per warp of its CTA).
constexpr int kReduceSerial = 16;
// The plan splits the sources so that a force launch has at least this many
// work items per persistent CTA (taken in dynamic order).
constexpr uint32_t kItemsPerCta = 4;
constexpr int kWideRows = 32;

// Entries of k_reduce's arrival counters (large splits) for a partial-sum buffer of
// part_items work items.  The plan keeps sum_k T_k B_k <= part_items (T_k
// i-tiles of cluster k), so the units (i-tile, row segment) of clusters with
// B_k > kReduceSerial, sum_k T_k ceil(B_k / kWideRows), stay below
// part_items / kWideRows + part_items / (kReduceSerial + 1); one counter per
// unit and block of 32 targets (at most kMixNI / 32 blocks).
constexpr int64_t wide_counter_entries(int64_t part_items) {
  return (part_items / kWideRows + part_items / (kReduceSerial + 1) + 2) * (kMixNI / 32);
}

// Min or max of v over the threads of one cell (kMixJD = 64 threads, two
// warps) of a CTA of kMixJT threads; every thread gets its cell's result.
// `sh` holds >= kMixJT / 32 floats.
__device__ __forceinline__ float nb_half_reduce_f(float v, bool is_max, float* sh) {
  static_assert(kMixJD == 64 && kMixJT % kMixJD == 0, "two warps per cell");
  for (int o = 16; o > 0; o >>= 1) {
    const float u = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmaxf(v, u) : fminf(v, u);
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[wid] = v;
  __syncthreads();
  const float a = sh[wid & ~1], b = sh[wid | 1];
  __syncthreads();
  return is_max ? fmaxf(a, b) : fminf(a, b);
}

// Write one mixed source tile (one CTA of kMixJT threads, one slot each).
// The tile holds kMixCells cells of kMixJD slots; for each cell: centre c = the
// midpoint of its valid particles' bounding box, taken in FP32 (c is only a
// reference point, exactly representable as a float), radius h >= max |r_j - c|.
// Each valid slot stores its double-single offset r_j - c (formed in FP64) from
// its cell's centre, its mass and FP32 velocity; pad slots (in == true,
// valid == false) hold massless dummies far away.  Record of tile t: float4
// [kTileRecF4 t + 2q] = (c, h) and [kTileRecF4 t + 2q + 1] = (0, 0, 0, 0)
// (the low part of a double-single centre) for cell q.  The FP64 work per slot
// is the offset and its split; the box and the radius use the FP32 pipe.
// Every thread must call this.
__device__ __forceinline__ void build_mixed_tile(float4* src, float4* tiles, int64_t tile,
                                                 int64_t s, bool in, bool valid, double3 x,
                                                 double m, double3 v, float* sh) {
  const float inf = CUDART_INF_F;
  const float fx = __double2float_rn(x.x), fy = __double2float_rn(x.y),
              fz = __double2float_rn(x.z);
  const float lx = nb_half_reduce_f(valid ? fx : inf, false, sh);
  const float ly = nb_half_reduce_f(valid ? fy : inf, false, sh);
  const float lz = nb_half_reduce_f(valid ? fz : inf, false, sh);
  const float hx = nb_half_reduce_f(valid ? fx : -inf, true, sh);
  const float hy = nb_half_reduce_f(valid ? fy : -inf, true, sh);
  const float hz = nb_half_reduce_f(valid ? fz : -inf, true, sh);
  const bool any = lx <= hx;
  // lx + hx cannot overflow for positions far below FLT_MAX
  const float chx = any ? 0.5f * (lx + hx) : 0.f, chy = any ? 0.5f * (ly + hy) : 0.f,
              chz = any ? 0.5f * (lz + hz) : 0.f;
  const double dx = x.x - (double)chx, dy = x.y - (double)chy, dz = x.z - (double)chz;
  const float dxh = __double2float_rn(dx), dyh = __double2float_rn(dy),
              dzh = __double2float_rn(dz);
  // |r_j - c| from the rounded offsets, then rounded up by 2^-18 relative: a
  // bound on the true distance (the FP32 rounding of the offsets and of the
  // sum and square root stays below 2^-21 relative)
  const float r = valid ? __fmul_ru(sqrtf(dxh * dxh + dyh * dyh + dzh * dzh), 1.0f + 0x1p-18f)
                        : 0.f;
  const float h = nb_half_reduce_f(r, true, sh);
  if (in) {
    float* g = reinterpret_cast<float*>(src + (s >> 2) * 10) + (s & 3);
    if (valid) {
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
    tiles[kTileRecF4 * tile + 2 * q] = make_float4(chx, chy, chz, h);
    tiles[kTileRecF4 * tile + 2 * q + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

struct PlanArgs {
  int NI;               // targets per work item of the force kernel
  int JT;               // sources per tile of the force kernel
  int grid;             // persistent CTAs of the force kernel
  int forced_b;         // fixed i-split factor (0: chosen here)
  int64_t part_items;   // capacity of the partial-sum buffer in work items
  // j-partition: the force runs over piece `part` of `parts` of each
  // cluster's sources (parts <= 1: all of them); B splits the piece
  int part, parts;
  // autotune table (block steps of the mixed path; 0: not used): the plan
  // takes (variant, B) from d.tune for ceil(log2 m) of the step's active
  // count, the variant's NI and grid from these arrays, and records the
  // choice in d.sel
  int use_table;
  int ni_v[kMixVariants], grid_v[kMixVariants];
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
  const double* snap; int ss; // 6th order: the new snap (m rows)
  const int64_t* t_tgt;       // per-cluster target time or nullptr
  int64_t t_fixed;
  double eta;
  int T, lmin, lmax;
  int reset_tmin;             // block step: reset the clusters' t_min (used up)
};

cudaError_t launch_fill_i64(int64_t* p, int64_t n, int64_t v, cudaStream_t st);
cudaError_t launch_tmin(const Dev& d, int T, cudaStream_t st);
// zero_tau: sources at the stored positions (no Taylor step)
cudaError_t launch_predict(const Dev& d, const int64_t* t_tgt, int64_t t_fixed, int T, bool mix,
                           bool f64, bool count_due, cudaStream_t st, bool zero_tau = false);
// a bounded wait that nothing completes: sets the timeout bit after `budget`
// clock cycles (the self-check behind nb_check_wait_timeout)
cudaError_t launch_wait_probe(uint32_t* status, long long budget, cudaStream_t st);
// every particle in source-slot order into d.active (use it as the rows too)
cudaError_t launch_slot_list(const Dev& d, cudaStream_t st);
// leapfrog halves (a_new == nullptr: kick + drift + time; else kick + store)
cudaError_t launch_leapfrog(const Dev& d, const double* a_new, double h, double dt,
                            int64_t dt_ticks, cudaStream_t st);
// block step: scan + plan (one CTA), then the active list
cudaError_t launch_scan_plan_scatter(const Dev& d, const PlanArgs& p, int T, cudaStream_t st);
cudaError_t launch_plan(const Dev& d, const PlanArgs& p, cudaStream_t st);
// grid: persistent CTAs of the reduction (one per SM)
cudaError_t launch_reduce(const ForceArgs& a, int NI, bool with_acc, int64_t m_bound,
                          int grid, cudaStream_t st);
// one-time kernel attributes (the reduction's dynamic shared memory)
cudaError_t integrator_setup();
cudaError_t launch_correct(const Dev& d, const CorrectArgs& c, int64_t m_bound, cudaStream_t st);
// 6th-order Hermite corrector, step criterion and level of the listed particles
cudaError_t launch_correct6(const Dev& d, const CorrectArgs& c, int64_t m_bound, cudaStream_t st);
cudaError_t launch_init_levels(const Dev& d, double eta_s, int T, int lmin, int lmax,
                               cudaStream_t st);
// caller list -> d.active (slot order), d.rows (caller rows), act_off
cudaError_t launch_list_to_slots(const Dev& d, const int32_t* list, int64_t m, cudaStream_t st);
cudaError_t launch_actoff_identity(const Dev& d, cudaStream_t st);
cudaError_t launch_energy(const Dev& d, const double* pot, int sp, int64_t lo, int64_t hi,
                          double* part, int nblk, double* out, cudaStream_t st);

// arithmetic-rate probe (nb_probe.cu): mode 0 f32x2 FMA, 1 FP32 FMA, 2 FP64 FMA;
// scratch holds probe_scratch_bytes(ctas); records (smid, start, end clock)
// per CTA follow ctas * 256 floats
size_t probe_scratch_bytes(int ctas);
cudaError_t launch_rate_probe(int mode, int ctas, int iters, void* scratch, cudaStream_t st);
double probe_lanes_per_launch(int mode, int ctas, int iters);

cudaError_t launch_pack3(const double* src3, dbl4* dst, int64_t n, bool keep_w, cudaStream_t st);
cudaError_t launch_unpack3(const dbl4* src, double* dst3, int64_t n, cudaStream_t st);
cudaError_t launch_tcur_from_t(const Dev& d, cudaStream_t st);

}  // namespace nb
