// nb_internal.cuh -- internal types and device helpers of libnbody_gb300.
//
// Data layout in HBM (one caller-owned workspace, carved by nb_layout()):
//   per particle i (N):   pos dbl4 (x, y, z, m)      vel dbl4 (vx, vy, vz, 0)
//                         acc dbl4 (ax, ay, az, pot) jerk dbl4 (jx, jy, jz, 0)
//                         t int64 ticks, level int32, cluster id int32,
//                         active list int32, new acc/jerk dbl4 per active slot
//   per source slot (S = sum over clusters of N_k rounded up to 4; pad slots
//   hold massless dummies far away):
//     mixed sources: groups of 4 slots, 10 float4 per group, component-major
//       [xh][yh][zh][m][xl][yl][zl][vx][vy][vz], x = xh + xl (double-single),
//       so one 16-byte shared-memory load yields a component of 4 sources and
//       two f32x2 operand pairs;
//     FP64 sources: dbl4 (x, y, z, m) and dbl4 (vx, vy, vz, 0).
//   per cluster k (K):    particle / slot offsets, current block time,
//                         running min for the next block time, active-list
//                         offsets, i-split factor B_k, work-item offsets.
//   i-split partial sums: [item][7][NI] doubles (acc xyz, jerk xyz, pot).
#pragma once
#include <cstddef>
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

// 32-byte aligned double vector (CUDA 13 names the alignment explicitly).
typedef double4_32a dbl4;

namespace nb {

constexpr int kMaxTickExp = 60;
constexpr int kPartialComps = 7;     // ax ay az jx jy jz pot
constexpr int kPartialCompsSnap = 10; // ... and sx sy sz (the 6th-order force)
constexpr double kDummyPos = 1.0e18; // where massless pad sources sit

// Mixed-precision force kernel shape.
constexpr int kMixNT = 128;          // threads per CTA
constexpr int kMixIPT = 2;           // targets (i) per thread
constexpr int kMixNI = kMixNT * kMixIPT;
constexpr int kMixJT = 128;          // sources per shared-memory tile (multiple of 4)
constexpr int kMixJD = 64;           // sources per cell (one centre/radius record)
constexpr int kMixCells = kMixJT / kMixJD;  // cells per tile
constexpr int kMixDefaultVariant = 0;       // mixed kernel shape of nb_default_config
constexpr int kMixVariants = 8;             // compiled mixed kernel shapes
constexpr int kTuneBuckets = 32;            // autotune table: one entry per ceil(log2 m)
constexpr int kTileRecF4 = 2 * kMixCells;   // float4 of cell records per tile
// FP64 force kernel shape.
constexpr int kF64NT = 128;
constexpr int kF64NI = kF64NT;
constexpr int kF64JT = 64;

// Device status bits (sticky; the host maps the lowest set code).
constexpr uint32_t kStatusInval = 1u << 0;
constexpr uint32_t kStatusTimeout = 1u << 1;
constexpr uint32_t kStatusNonFinite = 1u << 2;

struct Dev {
  int64_t N = 0, S = 0;
  int32_t K = 0;
  dbl4 *pos = nullptr, *vel = nullptr, *acc = nullptr, *jerk = nullptr;
  int64_t* t = nullptr;
  int32_t* level = nullptr;
  int32_t* cid = nullptr;
  int32_t* active = nullptr;
  dbl4 *acc_new = nullptr, *jerk_new = nullptr;
  float4* src_mix = nullptr;     // (S / 4) * 10 float4
  float4* tiles = nullptr;       // kTileRecF4 float4 per mixed source tile: per cell (c, h), (c_lo = 0, 0)
  int32_t* toff = nullptr;       // K + 1: first tile of each cluster
  int64_t n_tiles = 0;
  int32_t* sperm = nullptr;      // S: particle of each source slot (-1: pad)
  int32_t* sinv = nullptr;       // N: source slot of each particle
  int32_t* mark = nullptr;       // N: caller row of each listed particle (-1: none)
  int32_t* rows = nullptr;       // N: caller row of each target in slot order
  dbl4* src64_pos = nullptr;  // S
  dbl4* src64_vel = nullptr;  // S
  double* partials = nullptr;    // part_items * 7 * NI_max
  int64_t part_items = 0;
  int32_t* blk_count = nullptr;  // n_tiles + 1 (due particles per source tile)
  uint32_t* due_mask = nullptr;  // kMixJT / 32 words per source tile: the slots due in the
                                 // block step (bit = lane of the slot's warp), by the predictor
  int64_t *off = nullptr, *soff = nullptr;   // K + 1
  int64_t *t_cur = nullptr, *t_min = nullptr; // K
  int32_t *act_off = nullptr, *item_off = nullptr; // K + 1
  int32_t* wt_off = nullptr;     // K + 1: (i-tile, row segment) units of k_reduce's large splits
  int32_t* wide_cnt = nullptr;   // their arrival counters (zero between launches)
  int32_t* bfac = nullptr;       // K
  double* esum = nullptr;        // energy partial sums
  uint32_t* status = nullptr;
  unsigned long long* counters = nullptr;  // [0] interactions [1] block steps
                                           // [2] warp-tiles [3] near warp-tiles
  int64_t* t_end = nullptr;      // 1
  int32_t* work_ctr = nullptr;   // next work item of the force kernels (zeroed by the plan)
  int32_t* tune = nullptr;       // autotune table: (variant, B) per ceil(log2 m), kTuneBuckets
  int32_t* sel = nullptr;        // the plan's choice from it: variant, targets per work item
  // 6th-order Hermite (order == 6; null otherwise): snap and crackle per
  // particle (dbl4, w unused), the new snap per active slot, and the
  // predicted accelerations of the sources (mixed: groups of 4 slots, 3 float4
  // per group [ax][ay][az]; FP64: dbl4 per slot)
  int32_t order = 4;
  dbl4 *snap = nullptr, *crackle = nullptr, *snap_new = nullptr;
  float4* src_acc_mix = nullptr;
  dbl4* src64_acc = nullptr;
};

// Targets, sources and outputs of one force launch.
struct ForceArgs {
  const int64_t* off;       // particle offsets of the clusters (K + 1)
  const int64_t* soff;      // source-slot offsets (K + 1)
  const int32_t* active;    // target particle indices (nullptr: identity)
  const int32_t* act_off;   // target offsets per cluster (K + 1)
  const int32_t* item_off;  // work-item offsets per cluster (K + 1)
  const int32_t* wt_off;    // offsets of the wide-split reduction units per cluster (K + 1)
  int32_t* wide_cnt;        // arrival counters of the wide-split reduction
  const int32_t* bfac;      // i-split factor per cluster (K)
  const int32_t* sinv;      // source slot of each particle (nullptr: slot order = particle order)
  const float4* tiles;      // mixed source tile records
  const int32_t* toff;      // first tile of each cluster (K + 1)
  const int32_t* rows;      // output row of each target (nullptr: its position in the list)
  unsigned long long* tile_counts;  // [0] warp-tiles, [1] of them near (nullptr: not counted)
  int32_t K;
  const void* src_a;        // mixed: float4 groups; FP64: positions
  const void* src_b;        // FP64: velocities
  double* out_acc; int sa;  // row stride in doubles (nullptr: not written)
  double* out_jerk; int sj;
  double* out_pot; int sp;
  double* partials;         // [item][7][NI]
  double G;
  double eps2;
  uint32_t* status;
  int32_t* work_ctr;        // next work item (zeroed by the plan; nullptr: a fixed share per CTA)
  // force with snap (the 6th-order scheme): the sources' predicted
  // accelerations (mixed: float4 groups [ax][ay][az] of 4 slots; FP64: dbl4
  // per slot), the snap output (nullptr: no snap) and its row stride
  const void* src_c;
  double* out_snap; int ss;
  int comps;                // partial-sum components per target: 7, or 10 with snap
  // j-partition: the sum runs over piece `part` of `parts` of every
  // cluster's sources (src_piece); parts <= 1: all sources
  int32_t part, parts;
  // block steps with an autotune table: the plan writes the shape it chose
  // for the step's active count (sel[0]: variant, sel[1]: its targets per
  // work item); a force kernel launched as variant my_variant exits at once
  // when it is not the chosen one, and the reduction takes sel[1] as NI
  const int32_t* sel;       // nullptr: no selection (the launch is the chosen shape)
  int32_t my_variant;
};

// ---------------------------------------------------------------- helpers

// Programmatic dependent launch.  The kernels of a block step (t_next,
// predictor, scan and plan, scatter, force, reduction, corrector) run one
// after the other, and with few active particles each takes a few
// microseconds, about as long as a launch.  Launched with launch_chain, the
// next kernel of the chain is put on the GPU while the current one runs:
// every chain kernel first waits until the kernel before it has completed
// and its writes are visible (pdl_wait, which is why each of them, even one
// that exits at once, waits before anything else: the wait is what carries
// the ordering down the chain), then allows the kernel after it to launch
// (pdl_launch).  Outside a programmatic launch both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_chain(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                         cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One-dimensional bulk copy global -> shared (TMA engine); completion is
// signalled on `bar` as transaction bytes.  dst, src and bytes must be
// multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Spin on an mbarrier phase with a clock budget; false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > budget) return false;
  }
}

constexpr long long kWaitBudget = 4000000000LL;  // ~2 s of SM clock

// Packed FP32 pairs (f32x2): one instruction does the same operation on two
// independent lanes held in a 64-bit register pair.
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(f2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// Hardware approximate reciprocal square root / reciprocal (SFU, FP32).
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// SFU on both lanes of a pair, results written straight into the pair's
// halves (one asm block, so no register moves are needed to repack them).
__device__ __forceinline__ f2 f2_rsqrt(f2 x) {
  f2 y;
  asm("{\n\t.reg .f32 a, b;\n\t"
      "mov.b64 {a, b}, %1;\n\t"
      "rsqrt.approx.ftz.f32 a, a;\n\t"
      "rsqrt.approx.ftz.f32 b, b;\n\t"
      "mov.b64 %0, {a, b};\n\t}"
      : "=l"(y)
      : "l"(x));
  return y;
}
__device__ __forceinline__ f2 f2_rcp(f2 x) {
  f2 y;
  asm("{\n\t.reg .f32 a, b;\n\t"
      "mov.b64 {a, b}, %1;\n\t"
      "rcp.approx.ftz.f32 a, a;\n\t"
      "rcp.approx.ftz.f32 b, b;\n\t"
      "mov.b64 %0, {a, b};\n\t}"
      : "=l"(y)
      : "l"(x));
  return y;
}

// Knuth's error-free two-sum: hi + lo accumulates x exactly up to the final
// rounding of lo.
template <typename T>
__device__ __forceinline__ void two_sum_acc(T& hi, T& lo, T x) {
  T s = hi + x;
  T bp = s - hi;
  T err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

// Next work item of a persistent force kernel from the device counter
// (every thread of the CTA calls it; one atomic per item, broadcast through
// shared memory).
__device__ __forceinline__ int32_t grab_item(int32_t* ctr, int32_t* sh) {
  __syncthreads();  // every thread has read the previous value
  if (threadIdx.x == 0) *sh = atomicAdd(ctr, 1);
  __syncthreads();
  return *sh;
}

__device__ __forceinline__ int32_t upper_bound_i32(const int32_t* a, int32_t n, int32_t v) {
  // first index k in [0, n) with a[k] > v (a ascending)
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) > v) hi = mid; else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ int32_t upper_bound_i64(const int64_t* a, int32_t n, int64_t v) {
  // first index k in [0, n) with a[k] > v (a ascending)
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) > v) hi = mid; else lo = mid + 1;
  }
  return lo;
}

__host__ __device__ __forceinline__ int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t round_up64(int64_t a, int64_t b) { return ceil_div64(a, b) * b; }

// Chunk length (in source slots) of the j-range split of a cluster with S_k
// slots into B chunks; a multiple of the tile length JT.  The plan shrinks B
// so that every one of the B chunks is non-empty.
__host__ __device__ __forceinline__ int64_t chunk_len(int64_t S_k, int64_t B, int64_t JT) {
  return round_up64(ceil_div64(S_k, B), JT);
}

// Piece `part` of `parts` of a cluster's S_k source slots, [*b, *e) relative
// to the cluster's first slot: contiguous pieces of ceil(S_k / parts) slots
// rounded up to a whole tile of both force kernels, so that every piece
// starts on a tile; the last pieces may be empty.  The pieces of a
// j-partition of the force sum (one per process).
constexpr int kSrcPieceAlign = kMixJT;
static_assert(kMixJT % kF64JT == 0, "a piece starts on a tile of both force kernels");
__host__ __device__ __forceinline__ void src_piece(int64_t S_k, int32_t part, int32_t parts,
                                                   int64_t* b, int64_t* e) {
  const int64_t per = round_up64(ceil_div64(S_k, parts), kSrcPieceAlign);
  const int64_t lo = (int64_t)part * per;
  *b = lo < S_k ? lo : S_k;
  *e = lo + per < S_k ? lo + per : S_k;
}

// ------------------------------------------------------- launch wrappers
// (defined in the .cu files; all enqueue on `st` and return the launch error)
cudaError_t launch_force_mixed(const ForceArgs& a, int grid, bool with_pot, int variant,
                               cudaStream_t st);
cudaError_t launch_force_fp64(const ForceArgs& a, int grid, int mode, cudaStream_t st);
int force_mixed_variants();
int force_mixed_ni(int variant);  // targets per work item of a mixed shape
int force_mixed_ctas_per_sm(int variant);
// the acceleration-only mixed kernel (no velocities, no jerk)
cudaError_t launch_force_mixed_acc(const ForceArgs& a, int grid, bool with_pot, cudaStream_t st);
int force_mixed_acc_ni();
int force_mixed_acc_ctas_per_sm();
// acceleration, jerk and snap (the 6th-order force): one mixed shape
cudaError_t launch_force_mixed_snap(const ForceArgs& a, int grid, bool with_pot, cudaStream_t st);
int force_mixed_snap_ni();
int force_mixed_snap_ctas_per_sm();
// the 64 x 4 shape (force_mixed_ni(2) targets per item) with another
// separation mode: 1 double-single everywhere, 2 plain FP32
cudaError_t launch_force_mixed_sep(const ForceArgs& a, int grid, bool with_pot, int sep,
                                   cudaStream_t st);
int force_mixed_sep_ctas_per_sm(int sep);
int force_fp64_ctas_per_sm();
size_t force_mixed_smem();
size_t force_fp64_smem();

enum { kF64Full = 0, kF64PotOnly = 1, kF64Snap = 2 };

}  // namespace nb
