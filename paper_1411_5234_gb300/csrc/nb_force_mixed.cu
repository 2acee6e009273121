// nb_force_mixed.cu -- instantiation and launch of the mixed-precision force
// kernel (the kernel itself is in nb_force_mixed.cuh).
//
// Shapes compiled in (selected per context by nb_config.variant; each
// handles NT x IPT targets per work item; all take work items in dynamic
// order):
//   0:  64 threads x 4 targets, shared-memory totals, two tiles per stage,
//       near loop unrolled x4 (the default: 60.9 % of the FP32 peak at
//       N = m = 2^20 on GB300, against 59.5-60.7 % for the next shapes)
//   1:  as 0 with the near loop unrolled x8
//   2:  64 x 4, one tile per stage, near loop unrolled x2
//   3:  32 x 4 (one warp per CTA, 8 CTAs per SM), one tile per stage
//   4:  64 x 3, two tiles per stage (10 warps per SM)
//   5: 128 x 2, totals in registers, source loop unrolled x2, two tiles per stage
//   6:  64 x 2 (8 CTAs per SM), one tile per stage: 128 targets per work item
//   7:  32 x 2 (16 CTAs per SM), one tile per stage: 64 targets per work item
// (6 and 7 serve small active sets: fewer targets per item means more
// i-tiles and fewer source chunks for the same grid)
// and, for nb_force calls that want no jerk, one acceleration-only shape.
#include "../../include/nbody_gb300.h"
#include "nb_force_mixed.cuh"

namespace nb {
namespace {
template <bool POT> using S0 = mixk::MixShape<64, 4, POT, false, true, 1, 4, true, mixk::kSepMixed, 4, 2>;
template <bool POT> using S1 = mixk::MixShape<64, 4, POT, false, true, 1, 4, true, mixk::kSepMixed, 8, 2>;
template <bool POT> using S2 = mixk::MixShape<64, 4, POT, false, true, 1, 4, true, mixk::kSepMixed, 2, 1>;
template <bool POT> using S3 = mixk::MixShape<32, 4, POT, false, true, 1, 8, true, mixk::kSepMixed, 4, 1>;
template <bool POT> using S4 = mixk::MixShape<64, 3, POT, false, true, 1, 5, true, mixk::kSepMixed, 4, 2>;
template <bool POT> using S5 = mixk::MixShape<128, 2, POT, false, false, 2, 2, true, mixk::kSepMixed, 4, 2>;
template <bool POT> using S6 = mixk::MixShape<64, 2, POT, false, true, 1, 8, true, mixk::kSepMixed, 4, 1>;
template <bool POT> using S7 = mixk::MixShape<32, 2, POT, false, true, 1, 16, true, mixk::kSepMixed, 4, 1>;
// acceleration (and potential) only: 64 x 4 at 6 CTAs per SM was the fastest
// of the 64x4 (5 or 6 CTAs/SM, unrolled or not), 128x2 and 256x1 shapes at
// N = m = 2^20 (measured on GB300)
template <bool POT> using SA = mixk::MixShape<64, 4, POT, false, true, 1, 6, false, mixk::kSepMixed, 4, 2>;
// acceleration, jerk and snap (the 6th-order Hermite force): 64 x 2
template <bool POT> using SS = mixk::MixShape<64, 2, POT, false, true, 1, 5, true, mixk::kSepMixed, 4, 1, true>;
// the default shape with double-single separations everywhere, and with plain
// FP32 separations (NB_DS, NB_FP32: accuracy and speed bounds of the mixed path)
template <bool POT> using SD = mixk::MixShape<64, 4, POT, false, true, 1, 4, true, mixk::kSepDS, 4, 2>;
template <bool POT> using SF = mixk::MixShape<64, 4, POT, false, true, 1, 4, true, mixk::kSepFP32, 4, 2>;

template <class Sh>
cudaError_t launch_shape(const ForceArgs& a, int grid, cudaStream_t st) {
  return launch_chain(mixk::k_force_mixed<Sh>, dim3(grid), dim3(Sh::NT), 0, st, a);
}

template <class Sh>
int occupancy() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mixk::k_force_mixed<Sh>, Sh::NT, 0);
  return n;
}

template <template <bool> class S>
int occupancy_both() {
  const int a = occupancy<S<true>>(), b = occupancy<S<false>>();
  const int n = a < b ? a : b;
  return n > 0 ? n : 1;
}
}  // namespace

static_assert(kMixVariants == NB_MIXED_VARIANTS, "the shapes the ABI announces");
static_assert(kTuneBuckets == NB_TUNE_BUCKETS, "the autotune table the ABI announces");

int force_mixed_variants() { return NB_MIXED_VARIANTS; }

int force_mixed_ni(int variant) {
  switch (variant) {
    case 1: return S1<false>::NI;
    case 2: return S2<false>::NI;
    case 3: return S3<false>::NI;
    case 4: return S4<false>::NI;
    case 5: return S5<false>::NI;
    case 6: return S6<false>::NI;
    case 7: return S7<false>::NI;
    default: return S0<false>::NI;
  }
}

cudaError_t launch_force_mixed(const ForceArgs& a, int grid, bool with_pot, int variant,
                               cudaStream_t st) {
  switch (variant) {
    case 1: return with_pot ? launch_shape<S1<true>>(a, grid, st) : launch_shape<S1<false>>(a, grid, st);
    case 2: return with_pot ? launch_shape<S2<true>>(a, grid, st) : launch_shape<S2<false>>(a, grid, st);
    case 3: return with_pot ? launch_shape<S3<true>>(a, grid, st) : launch_shape<S3<false>>(a, grid, st);
    case 4: return with_pot ? launch_shape<S4<true>>(a, grid, st) : launch_shape<S4<false>>(a, grid, st);
    case 5: return with_pot ? launch_shape<S5<true>>(a, grid, st) : launch_shape<S5<false>>(a, grid, st);
    case 6: return with_pot ? launch_shape<S6<true>>(a, grid, st) : launch_shape<S6<false>>(a, grid, st);
    case 7: return with_pot ? launch_shape<S7<true>>(a, grid, st) : launch_shape<S7<false>>(a, grid, st);
    default: return with_pot ? launch_shape<S0<true>>(a, grid, st) : launch_shape<S0<false>>(a, grid, st);
  }
}

int force_mixed_ctas_per_sm(int variant) {
  switch (variant) {
    case 1: return occupancy_both<S1>();
    case 2: return occupancy_both<S2>();
    case 3: return occupancy_both<S3>();
    case 4: return occupancy_both<S4>();
    case 5: return occupancy_both<S5>();
    case 6: return occupancy_both<S6>();
    case 7: return occupancy_both<S7>();
    default: return occupancy_both<S0>();
  }
}

int force_mixed_acc_ni() { return SA<false>::NI; }
int force_mixed_sep_ctas_per_sm(int sep) {
  return sep == mixk::kSepDS ? occupancy_both<SD>() : occupancy_both<SF>();
}
cudaError_t launch_force_mixed_sep(const ForceArgs& a, int grid, bool with_pot, int sep,
                                   cudaStream_t st) {
  if (sep == mixk::kSepDS)
    return with_pot ? launch_shape<SD<true>>(a, grid, st) : launch_shape<SD<false>>(a, grid, st);
  return with_pot ? launch_shape<SF<true>>(a, grid, st) : launch_shape<SF<false>>(a, grid, st);
}
int force_mixed_acc_ctas_per_sm() { return occupancy_both<SA>(); }
cudaError_t launch_force_mixed_acc(const ForceArgs& a, int grid, bool with_pot, cudaStream_t st) {
  return with_pot ? launch_shape<SA<true>>(a, grid, st) : launch_shape<SA<false>>(a, grid, st);
}

int force_mixed_snap_ni() { return SS<false>::NI; }
int force_mixed_snap_ctas_per_sm() { return occupancy_both<SS>(); }
cudaError_t launch_force_mixed_snap(const ForceArgs& a, int grid, bool with_pot, cudaStream_t st) {
  if (with_pot) return launch_shape<SS<true>>(a, grid, st);
  return launch_shape<SS<false>>(a, grid, st);
}

size_t force_mixed_smem() { return sizeof(float4) * 2 * mixk::kTileF4; }

}  // namespace nb
