// nb_integrator.cuh -- launch interface of the block-step kernels.
#pragma once
#include "nb_internal.cuh"

namespace nb {

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
cudaError_t launch_init_pads(const Dev& d, cudaStream_t st);
cudaError_t launch_tmin(const Dev& d, int T, cudaStream_t st);
int scan_blocks(int64_t N);
cudaError_t launch_predict(const Dev& d, const int64_t* t_tgt, int64_t t_fixed, int T, bool mix,
                           bool f64, bool count_due, cudaStream_t st);
cudaError_t launch_compact(const Dev& d, int T, cudaStream_t st);
cudaError_t launch_plan(const Dev& d, const PlanArgs& p, cudaStream_t st);
cudaError_t launch_reduce(const ForceArgs& a, int NI, bool with_acc, int64_t m_bound,
                          cudaStream_t st);
cudaError_t launch_correct(const Dev& d, const CorrectArgs& c, int64_t m_bound, cudaStream_t st);
cudaError_t launch_init_levels(const Dev& d, double eta_s, int T, int lmin, int lmax,
                               cudaStream_t st);
cudaError_t launch_actoff_list(const Dev& d, const int32_t* list, int64_t m, cudaStream_t st);
cudaError_t launch_actoff_identity(const Dev& d, cudaStream_t st);
cudaError_t launch_energy(const Dev& d, const double* pot, int sp, int64_t lo, int64_t hi,
                          double* part, int nblk, double* out, cudaStream_t st);

cudaError_t launch_pack3(const double* src3, dbl4* dst, int64_t n, bool keep_w, cudaStream_t st);
cudaError_t launch_unpack3(const dbl4* src, double* dst3, int64_t n, cudaStream_t st);
cudaError_t launch_tcur_from_t(const Dev& d, cudaStream_t st);

}  // namespace nb
