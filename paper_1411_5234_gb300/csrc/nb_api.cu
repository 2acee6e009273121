// nb_api.cu -- the C ABI of libnbody_gb300 (declared in include/nbody_gb300.h).
//
// Host side only: argument checks, workspace layout, and the enqueue order of
// the kernels in nb_force_*.cu and nb_integrator.cu.  No device memory is
// allocated here; the caller's workspace is carved into the arrays below.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/nbody_gb300.h"
#include "nb_integrator.cuh"

using namespace nb;

namespace {

// Host-side NVTX range around an ABI call (the span in which it enqueues its
// work, or waits for it when the call synchronises); a no-op unless a
// profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr size_t kAlign = 256;
constexpr int kEnergyBlocks = 304;
// kinds of timed launches (nb_profile_kernels, in this order)
enum { kProfTnext = 0, kProfPredict, kProfPlan, kProfForce, kProfReduce, kProfCorrect };
static_assert(kProfCorrect + 1 == NB_PROFILE_KINDS, "the kinds the ABI announces");

struct Layout {
  size_t snap, crackle, snap_new, src_acc_mix, src64_acc;  // 6th order only (else empty)
  size_t pos, vel, acc, jerk, acc_new, jerk_new, t, level, cid, active, src_mix, src64_pos,
      src64_vel, partials, blk_count, off, soff, t_cur, t_min, act_off, item_off, wt_off, wide_cnt, bfac, esum,
      status, counters, t_end, work, tune, sel, due_mask, tiles, toff, sperm, sinv, mark, rows,
      total;
  int64_t S, part_items, n_tiles;
};

size_t take(size_t& cur, size_t bytes) {
  const size_t o = cur;
  cur += (bytes + kAlign - 1) / kAlign * kAlign;
  return o;
}

Layout make_layout(int64_t N, int32_t K, int64_t S, int64_t n_tiles, int order) {
  Layout L{};
  const bool o6 = order == 6;
  const int comps = o6 ? kPartialCompsSnap : kPartialComps;
  L.S = S;
  L.n_tiles = n_tiles;
  const int64_t nitile = ceil_div64(N, 128) + K;  // smallest targets-per-item of any shape
  L.part_items = 2 * nitile > 2048 ? 2 * nitile : 2048;
  const size_t ni_max = kMixNI > kF64NI ? kMixNI : kF64NI;
  size_t c = 0;
  L.pos = take(c, 32 * N);
  L.vel = take(c, 32 * N);
  L.acc = take(c, 32 * N);
  L.jerk = take(c, 32 * N);
  L.acc_new = take(c, 32 * N);
  L.jerk_new = take(c, 32 * N);
  L.t = take(c, 8 * N);
  L.level = take(c, 4 * N);
  L.cid = take(c, 4 * N);
  L.active = take(c, 4 * N);
  L.src_mix = take(c, 40 * S);
  L.src64_pos = take(c, 32 * S);
  L.src64_vel = take(c, 32 * S);
  L.partials = take(c, (size_t)L.part_items * comps * ni_max * 8);
  L.blk_count = take(c, 4 * ((size_t)n_tiles + 1));
  L.off = take(c, 8 * ((size_t)K + 1));
  L.soff = take(c, 8 * ((size_t)K + 1));
  L.t_cur = take(c, 8 * (size_t)K);
  L.t_min = take(c, 8 * (size_t)K);
  L.act_off = take(c, 4 * ((size_t)K + 1));
  L.item_off = take(c, 4 * ((size_t)K + 1));
  L.wt_off = take(c, 4 * ((size_t)K + 1));
  L.wide_cnt = take(c, 4 * (size_t)wide_counter_entries(L.part_items));
  L.bfac = take(c, 4 * (size_t)K);
  L.esum = take(c, 8 * (2 * (size_t)kEnergyBlocks + 2));
  L.status = take(c, 4);
  L.counters = take(c, 8 * 4);
  L.t_end = take(c, 8);
  L.work = take(c, 4);
  L.tune = take(c, 8 * (size_t)kTuneBuckets);
  L.sel = take(c, 8);
  L.due_mask = take(c, 4 * (kMixJT / 32) * (size_t)n_tiles);
  L.tiles = take(c, 16 * kTileRecF4 * (size_t)n_tiles);
  L.toff = take(c, 4 * ((size_t)K + 1));
  L.sperm = take(c, 4 * (size_t)S);
  L.sinv = take(c, 4 * (size_t)N);
  L.mark = take(c, 4 * (size_t)N);
  L.rows = take(c, 4 * (size_t)N);
  L.snap = take(c, o6 ? 32 * (size_t)N : 0);
  L.crackle = take(c, o6 ? 32 * (size_t)N : 0);
  L.snap_new = take(c, o6 ? 32 * (size_t)N : 0);
  L.src_acc_mix = take(c, o6 ? 12 * (size_t)S : 0);
  L.src64_acc = take(c, o6 ? 32 * (size_t)S : 0);
  L.total = c;
  return L;
}

bool config_ok(const nb_config* c) {
  if (!c) return false;
  if (!std::isfinite(c->G) || !std::isfinite(c->eps) || c->eps < 0.0) return false;
  if (!(c->eta > 0.0) || !std::isfinite(c->eta)) return false;
  if (!(c->eta_start > 0.0) || !std::isfinite(c->eta_start)) return false;
  if (c->tick_exp < 1 || c->tick_exp > kMaxTickExp) return false;
  if (c->level_min < 0 || c->level_min > c->level_max || c->level_max > c->tick_exp) return false;
  if (c->precision < NB_FP64 || c->precision > NB_FP32) return false;
  if (c->bfactor < 0 || c->graph_steps < 0) return false;
  if (c->sort_sources != 0 && c->sort_sources != 1) return false;
  if (c->variant < 0 || c->variant >= force_mixed_variants()) return false;
  if (c->order != 4 && c->order != 6) return false;
  return true;
}

int64_t slots_of(const int64_t* off, int32_t K) {
  int64_t S = 0;
  for (int32_t k = 0; k < K; ++k) S += round_up64(off[k + 1] - off[k], 4);
  return S;
}

int64_t tiles_of(const int64_t* off, int32_t K) {
  int64_t n = 0;
  for (int32_t k = 0; k < K; ++k) n += ceil_div64(round_up64(off[k + 1] - off[k], 4), kMixJT);
  return n;
}

// 3-D Hilbert-curve key of a point quantised to `bits` bits per axis (Skilling,
// "Programming the Hilbert curve", AIP Conf. Proc. 707, 381, 2004): the axes
// are transformed in place into the transposed Hilbert index, whose bits are
// then interleaved most significant first.  Consecutive keys are neighbouring
// cells (no jumps), so fixed-size runs of sorted particles are compact.
uint64_t hilbert_key(uint32_t x, uint32_t y, uint32_t z, int bits) {
  uint32_t X[3] = {x, y, z};
  const uint32_t M = 1u << (bits - 1);
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    const uint32_t P = Q - 1;
    for (int i = 0; i < 3; ++i) {
      if (X[i] & Q) {
        X[0] ^= P;
      } else {
        const uint32_t t = (X[0] ^ X[i]) & P;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  X[1] ^= X[0];
  X[2] ^= X[1];
  uint32_t t = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1)
    if (X[2] & Q) t ^= Q - 1;
  for (int i = 0; i < 3; ++i) X[i] ^= t;
  uint64_t key = 0;
  for (int b = bits - 1; b >= 0; --b)
    for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
  return key;
}

// Source slots of every cluster: particles in Hilbert-curve order of their
// positions (pos: n x 3 host), or in particle order when `sorted` is false.  Pad slots
// get -1.  sperm: S entries, sinv: N entries.
void source_order(const double* pos, const int64_t* off, int32_t K, const int64_t* soff,
                  bool sorted, std::vector<int32_t>& sperm, std::vector<int32_t>& sinv) {
  for (int32_t k = 0; k < K; ++k) {
    const int64_t n0 = off[k], nk = off[k + 1] - off[k];
    std::vector<std::pair<uint64_t, int64_t>> key(nk);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nk; ++i)
      for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(lo[c], pos[3 * (n0 + i) + c]);
        hi[c] = std::max(hi[c], pos[3 * (n0 + i) + c]);
      }
    double span = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
    for (int64_t i = 0; i < nk; ++i) {
      uint64_t code = 0;
      if (sorted) {
        uint32_t u[3];
        for (int c = 0; c < 3; ++c) {
          const double q = (pos[3 * (n0 + i) + c] - lo[c]) / span * 2097151.0;
          u[c] = (uint32_t)std::min(std::max(q, 0.0), 2097151.0);
        }
        code = hilbert_key(u[0], u[1], u[2], 21);
      }
      key[i] = {code, i};
    }
    if (sorted) std::sort(key.begin(), key.end());
    for (int64_t r = 0; r < round_up64(nk, 4); ++r) {
      if (r < nk) {
        sperm[soff[k] + r] = static_cast<int32_t>(n0 + key[r].second);
        sinv[n0 + key[r].second] = static_cast<int32_t>(soff[k] + r);
      } else {
        sperm[soff[k] + r] = -1;
      }
    }
  }
}

}  // namespace

struct nb_ctx {
  nb_config cfg{};
  Dev d;
  Layout L{};
  cudaStream_t st = nullptr;
  int grid_mix = 0, grid_f64 = 0, grid_acc = 0, grid_snap = 0, sms = 0;
  int grid_v[kMixVariants] = {};  // persistent CTAs of each mixed shape
  // autotune table, host copy: (variant, B) per ceil(log2 m); `tabled` once
  // nb_autotune filled it (nb_force and block steps then follow it)
  std::vector<int32_t> tune_host;
  bool tabled = false;
  std::vector<int64_t> off_host;
  std::vector<double> mass_host;
  std::vector<int32_t> sperm_host;  // source slot order (for the autotuner's target lists)
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
  bool graph_broken = false;
  // kernel timing (nb_profile_enable): event pairs around the launches of
  // each kind (kProf*), summed per kind; the force kind also feeds
  // nb_profile_read's own total
  bool prof = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
  std::vector<int> ev_kind;
  double prof_ms = 0.0;
  int64_t prof_launches = 0;
  double kind_ms[NB_PROFILE_KINDS] = {};
  int64_t kind_n[NB_PROFILE_KINDS] = {};
  // j-partition: the piece of every cluster's sources the force launches of
  // the current call sum over (parts <= 1: all sources; set by PieceScope)
  int32_t part = 0, parts = 1;
  // a block step split by nb_block_force, waiting for nb_block_correct
  bool block_open = false;
};

namespace {

#define NB_TRY(x)                              \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return NB_ECUDA;    \
  } while (0)

static_assert(kSrcPieceAlign == NB_PIECE_ALIGN, "piece alignment of the ABI");

// every mode but FP64 uses the mixed source layout and kernel family
bool is_mixed(const nb_ctx* c) { return c->cfg.precision != NB_FP64; }
// separation mode of the mixed kernel (0: mixed vote, 1: DS, 2: plain FP32)
int sep_mode(const nb_ctx* c) {
  return c->cfg.precision == NB_DS ? 1 : c->cfg.precision == NB_FP32 ? 2 : 0;
}

ForceArgs force_args(nb_ctx* c, const int32_t* active, const int32_t* rows, double* acc, int sa,
                     double* jerk, int sj, double* pot, int sp, bool f64_sources) {
  ForceArgs a{};
  a.off = c->d.off;
  a.soff = c->d.soff;
  a.active = active;
  a.act_off = c->d.act_off;
  a.item_off = c->d.item_off;
  a.wt_off = c->d.wt_off;
  a.wide_cnt = c->d.wide_cnt;
  a.bfac = c->d.bfac;
  a.sinv = c->d.sinv;
  a.tiles = c->d.tiles;
  a.toff = c->d.toff;
  a.rows = rows;
  a.tile_counts = c->d.counters + 2;
  a.K = c->d.K;
  if (f64_sources) {
    a.src_a = c->d.src64_pos;
    a.src_b = c->d.src64_vel;
  } else {
    a.src_a = c->d.src_mix;
    a.src_b = nullptr;
  }
  a.out_acc = acc;
  a.sa = sa;
  a.out_jerk = jerk;
  a.sj = sj;
  a.out_pot = pot;
  a.sp = sp;
  a.partials = c->d.partials;
  a.G = c->cfg.G;
  a.eps2 = c->cfg.eps * c->cfg.eps;
  a.status = c->d.status;
  a.work_ctr = c->d.work_ctr;
  a.src_c = nullptr;
  a.out_snap = nullptr;
  a.ss = 0;
  a.comps = kPartialComps;
  a.sel = nullptr;
  a.my_variant = c->cfg.variant;
  a.part = c->part;
  a.parts = c->parts;
  return a;
}

// The force launches enqueued while a PieceScope lives sum over piece `part`
// of `parts` of each cluster's sources.
struct PieceScope {
  nb_ctx* c;
  PieceScope(nb_ctx* c_, int32_t part, int32_t parts) : c(c_) {
    c->part = part;
    c->parts = parts;
  }
  ~PieceScope() {
    c->part = 0;
    c->parts = 1;
  }
};

// The autotune table's bucket of an active count: ceil(log2 m).
int tune_bucket(int64_t m) {
  int b = 0;
  while (b < kTuneBuckets - 1 && ((int64_t)1 << b) < m) ++b;
  return b;
}

// Whether a force evaluation of this context takes its mixed shape from the
// autotune table (the plain mixed path with jerk, once nb_autotune ran).
bool uses_table(const nb_ctx* c, bool f64, bool acc_only, bool snap) {
  return c->tabled && !f64 && !acc_only && !snap && sep_mode(c) == 0;
}

// variant, forced_b: the mixed shape and i-split to plan for (-1: the
// context's); device_select: the plan takes both from the table instead.
PlanArgs plan_args(nb_ctx* c, bool f64, int step_mode, int count, bool acc_only = false,
                   bool snap = false, int variant = -1, int forced_b = -1,
                   bool device_select = false) {
  if (variant < 0) variant = c->cfg.variant;
  if (forced_b < 0) forced_b = c->cfg.bfactor;
  PlanArgs p{};
  p.NI = f64 ? kF64NI
             : snap ? force_mixed_snap_ni()
                    : acc_only ? force_mixed_acc_ni() : force_mixed_ni(variant);
  p.JT = f64 ? kF64JT : kMixJT;
  p.grid = f64        ? c->grid_f64
           : snap     ? c->grid_snap
           : acc_only ? c->grid_acc
           : sep_mode(c) ? c->grid_mix
                         : c->grid_v[variant];
  p.forced_b = forced_b;
  p.use_table = device_select ? 1 : 0;
  for (int v = 0; v < kMixVariants; ++v) {
    p.ni_v[v] = force_mixed_ni(v);
    p.grid_v[v] = c->grid_v[v];
  }
  p.part_items = c->L.part_items;
  p.step_mode = step_mode;
  p.count = count;
  p.part = c->part;
  p.parts = c->parts;
  return p;
}

// Fold finished event pairs into the running total (blocking when `all`).
cudaError_t prof_collect(nb_ctx* c, bool all) {
  size_t k = 0;
  for (; k < c->ev_pending.size(); ++k) {
    auto& p = c->ev_pending[k];
    if (all) {
      cudaError_t e = cudaEventSynchronize(p.second);
      if (e != cudaSuccess) return e;
    } else if (cudaEventQuery(p.second) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, p.first, p.second);
    if (e != cudaSuccess) return e;
    const int kind = c->ev_kind[k];
    c->kind_ms[kind] += ms;
    c->kind_n[kind] += 1;
    if (kind == kProfForce) {
      c->prof_ms += ms;
      c->prof_launches += 1;
    }
    c->ev_free.push_back(p.first);
    c->ev_free.push_back(p.second);
  }
  c->ev_pending.erase(c->ev_pending.begin(), c->ev_pending.begin() + k);
  c->ev_kind.erase(c->ev_kind.begin(), c->ev_kind.begin() + k);
  return cudaSuccess;
}

cudaError_t prof_events(nb_ctx* c, std::pair<cudaEvent_t, cudaEvent_t>* ev) {
  if (c->ev_pending.size() >= 512) {
    cudaError_t e = prof_collect(c, true);
    if (e != cudaSuccess) return e;
  }
  cudaEvent_t x[2];
  for (int q = 0; q < 2; ++q) {
    if (!c->ev_free.empty()) {
      x[q] = c->ev_free.back();
      c->ev_free.pop_back();
    } else {
      cudaError_t e = cudaEventCreate(&x[q]);
      if (e != cudaSuccess) return e;
    }
  }
  *ev = {x[0], x[1]};
  return cudaSuccess;
}

// Profiling only (c->prof): an event before and after the launches of one
// kind; nothing otherwise.
cudaError_t prof_begin(nb_ctx* c, std::pair<cudaEvent_t, cudaEvent_t>* ev) {
  if (!c->prof) return cudaSuccess;
  cudaError_t e = prof_events(c, ev);
  if (e != cudaSuccess) return e;
  return cudaEventRecord(ev->first, c->st);
}
cudaError_t prof_end(nb_ctx* c, const std::pair<cudaEvent_t, cudaEvent_t>& ev, int kind) {
  if (!c->prof) return cudaSuccess;
  cudaError_t e = cudaEventRecord(ev.second, c->st);
  if (e != cudaSuccess) return e;
  c->ev_pending.push_back(ev);
  c->ev_kind.push_back(kind);
  return cudaSuccess;
}

// plan + force + partial reduce on the active list already described by
// act_off (and `active`, or the identity when null).  m_host: the active
// count when the host knows it (nb_force: the table entry is applied here);
// -1 for a block step, whose plan (`planned`) picks the entry on the device.
cudaError_t enqueue_force(nb_ctx* c, const int32_t* active, const int32_t* rows, double* acc,
                          int sa, double* jerk, int sj, double* pot, int sp, bool f64,
                          int step_mode, int count, bool pot_only, int64_t m_bound,
                          bool planned = false, int64_t m_host = -1) {
  cudaError_t e = cudaSuccess;
  // no jerk wanted (and not the FP64 energy pass): the mixed path runs the
  // acceleration-only kernel
  const bool acc_only = !f64 && jerk == nullptr;
  const bool tabled = uses_table(c, f64, acc_only, false);
  int variant = c->cfg.variant, forced_b = c->cfg.bfactor;
  if (tabled && m_host >= 0) {
    const int b = tune_bucket(m_host);
    variant = c->tune_host[2 * b];
    if (forced_b == 0) forced_b = c->tune_host[2 * b + 1];
  }
  const bool device_select = tabled && m_host < 0;
  if (!planned) {
    std::pair<cudaEvent_t, cudaEvent_t> pev{nullptr, nullptr};
    e = prof_begin(c, &pev);
    if (e == cudaSuccess)
      e = launch_plan(c->d,
                      plan_args(c, f64, step_mode, count, acc_only, false, variant, forced_b,
                                device_select),
                      c->st);
    if (e == cudaSuccess) e = prof_end(c, pev, kProfPlan);
    if (e != cudaSuccess) return e;
  }
  ForceArgs fa = force_args(c, active, rows, acc, sa, jerk, sj, pot, sp, f64);
  fa.my_variant = variant;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (c->prof) {
    e = prof_events(c, &ev);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev.first, c->st);
    if (e != cudaSuccess) return e;
  }
  if (f64)
    e = launch_force_fp64(fa, c->grid_f64, pot_only ? kF64PotOnly : kF64Full, c->st);
  else if (acc_only)
    e = launch_force_mixed_acc(fa, c->grid_acc, pot != nullptr, c->st);
  else if (sep_mode(c))
    e = launch_force_mixed_sep(fa, c->grid_mix, pot != nullptr, sep_mode(c), c->st);
  else if (device_select) {
    // every distinct shape of the table; each exits at once unless the plan
    // chose it for this step's active count
    fa.sel = c->d.sel;
    bool launched[kMixVariants] = {};
    for (int b = 0; b < kTuneBuckets && e == cudaSuccess; ++b) {
      const int v = c->tune_host[2 * b];
      if (launched[v]) continue;
      launched[v] = true;
      fa.my_variant = v;
      e = launch_force_mixed(fa, c->grid_v[v], pot != nullptr, v, c->st);
    }
  } else {
    e = launch_force_mixed(fa, c->grid_v[variant], pot != nullptr, variant, c->st);
  }
  if (e != cudaSuccess) return e;
  if (c->prof) {
    e = cudaEventRecord(ev.second, c->st);
    if (e != cudaSuccess) return e;
    c->ev_pending.push_back(ev);
    c->ev_kind.push_back(kProfForce);
  }
  const int ni = f64 ? kF64NI : acc_only ? force_mixed_acc_ni() : force_mixed_ni(variant);
  std::pair<cudaEvent_t, cudaEvent_t> rev{nullptr, nullptr};
  e = prof_begin(c, &rev);
  if (e == cudaSuccess) e = launch_reduce(fa, ni, !pot_only, m_bound, c->sms, c->st);
  return e != cudaSuccess ? e : prof_end(c, rev, kProfReduce);
}

// plan + force with snap + partial reduce (the 6th-order scheme's force; the
// sources' predicted accelerations must be in place: an order-6 context's
// predictor writes them).  snap, ss: the snap rows and their stride.
cudaError_t enqueue_force_snap(nb_ctx* c, const int32_t* active, const int32_t* rows,
                               double* acc, int sa, double* jerk, int sj, double* snap, int ss,
                               double* pot, int sp, int step_mode, int count, int64_t m_bound,
                               bool planned = false) {
  const bool f64 = !is_mixed(c);
  cudaError_t e = cudaSuccess;
  if (!planned) {
    e = launch_plan(c->d, plan_args(c, f64, step_mode, count, false, true), c->st);
    if (e != cudaSuccess) return e;
  }
  ForceArgs fa = force_args(c, active, rows, acc, sa, jerk, sj, pot, sp, f64);
  fa.src_c = f64 ? static_cast<const void*>(c->d.src64_acc)
                 : static_cast<const void*>(c->d.src_acc_mix);
  fa.out_snap = snap;
  fa.ss = ss;
  fa.comps = kPartialCompsSnap;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (c->prof) {
    e = prof_events(c, &ev);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev.first, c->st);
    if (e != cudaSuccess) return e;
  }
  if (f64)
    e = launch_force_fp64(fa, c->grid_f64, kF64Snap, c->st);
  else
    e = launch_force_mixed_snap(fa, c->grid_snap, pot != nullptr, c->st);
  if (e != cudaSuccess) return e;
  if (c->prof) {
    e = cudaEventRecord(ev.second, c->st);
    if (e != cudaSuccess) return e;
    c->ev_pending.push_back(ev);
    c->ev_kind.push_back(kProfForce);
  }
  const int ni = f64 ? kF64NI : force_mixed_snap_ni();
  std::pair<cudaEvent_t, cudaEvent_t> rev{nullptr, nullptr};
  e = prof_begin(c, &rev);
  if (e == cudaSuccess) e = launch_reduce(fa, ni, true, m_bound, c->sms, c->st);
  return e != cudaSuccess ? e : prof_end(c, rev, kProfReduce);
}

// First half of a block step: the next block time, the prediction, the
// active list and its force (rows of 4 doubles in acc_new, jerk_new and, in
// the 6th-order scheme, snap_new, in active-list order).
cudaError_t enqueue_block_force(nb_ctx* c) {
  const int T = c->cfg.tick_exp;
  const bool f64 = !is_mixed(c);
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  cudaError_t e = prof_begin(c, &ev);
  if (e == cudaSuccess) e = launch_tmin(c->d, T, c->st);
  if (e == cudaSuccess) e = prof_end(c, ev, kProfTnext);
  if (e == cudaSuccess) e = prof_begin(c, &ev);
  if (e == cudaSuccess) e = launch_predict(c->d, c->d.t_min, 0, T, !f64, f64, true, c->st);
  if (e == cudaSuccess) e = prof_end(c, ev, kProfPredict);
  if (e != cudaSuccess) return e;
  const bool o6 = c->cfg.order == 6;
  e = prof_begin(c, &ev);
  if (e == cudaSuccess)
    e = launch_scan_plan_scatter(
        c->d, plan_args(c, f64, 1, 1, false, o6, -1, -1, uses_table(c, f64, false, o6)), T,
        c->st);
  if (e == cudaSuccess) e = prof_end(c, ev, kProfPlan);
  if (e != cudaSuccess) return e;
  double* an = reinterpret_cast<double*>(c->d.acc_new);
  double* jn = reinterpret_cast<double*>(c->d.jerk_new);
  if (o6) {
    double* sn = reinterpret_cast<double*>(c->d.snap_new);
    return enqueue_force_snap(c, c->d.active, nullptr, an, 4, jn, 4, sn, 4, nullptr, 0, 1, 1,
                              c->d.N, true);
  }
  // the integrator needs no potential: the force kernel skips it here
  return enqueue_force(c, c->d.active, nullptr, an, 4, jn, 4, nullptr, 0, f64, 1, 1, false,
                       c->d.N, true);
}

// Second half: the corrector of the step's active list from those rows.
cudaError_t enqueue_block_correct(nb_ctx* c) {
  CorrectArgs ca{};
  ca.active = c->d.active;
  ca.count_dev = c->d.act_off + c->d.K;
  ca.acc = reinterpret_cast<double*>(c->d.acc_new);
  ca.sa = 4;
  ca.jerk = reinterpret_cast<double*>(c->d.jerk_new);
  ca.sj = 4;
  ca.pot = nullptr;
  ca.sp = 0;
  ca.t_tgt = c->d.t_cur;
  ca.eta = c->cfg.eta;
  ca.T = c->cfg.tick_exp;
  ca.lmin = c->cfg.level_min;
  ca.lmax = c->cfg.level_max;
  ca.reset_tmin = 1;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  cudaError_t e = prof_begin(c, &ev);
  if (e != cudaSuccess) return e;
  if (c->cfg.order == 6) {
    ca.snap = reinterpret_cast<double*>(c->d.snap_new);
    ca.ss = 4;
    e = launch_correct6(c->d, ca, c->d.N, c->st);
  } else {
    e = launch_correct(c->d, ca, c->d.N, c->st);
  }
  return e != cudaSuccess ? e : prof_end(c, ev, kProfCorrect);
}

cudaError_t enqueue_block_step(nb_ctx* c) {
  const cudaError_t e = enqueue_block_force(c);
  return e != cudaSuccess ? e : enqueue_block_correct(c);
}

int sync_status(nb_ctx* c) {
  uint32_t s = 0;
  if (cudaMemcpyAsync(&s, c->d.status, sizeof s, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
    return NB_ECUDA;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return NB_ECUDA;
  if (s & kStatusTimeout) return NB_ETIMEOUT;
  if (s & kStatusNonFinite) return NB_ENONFINITE;
  if (s & kStatusInval) return NB_EINVAL;
  return NB_OK;
}

bool finite_all(const double* x, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}


// ---- autotune table: cache key, cache file, application

// The problem class a table belongs to: the GPU (name, SMs), the precision
// and Hermite order, ceil(log2 N) and the number of clusters.
std::string tune_key(const nb_ctx* c) {
  int dev = 0;
  cudaDeviceProp prop{};
  std::string name = "unknown";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
    name = prop.name;
  for (char& ch : name)
    if (ch == ' ' || ch == '=' || ch == ';') ch = '_';
  char buf[512];
  std::snprintf(buf, sizeof buf, "nbody-tune-1 gpu=%s sms=%d prec=%d order=%d logN=%d K=%d",
                name.c_str(), c->sms, c->cfg.precision, c->cfg.order, tune_bucket(c->d.N),
                c->d.K);
  return buf;
}

// The last line of `path` with this key: "<key> table=v,b;v,b;..." with
// kTuneBuckets valid entries.
bool tune_load(const char* path, const std::string& key, std::vector<int32_t>& tab) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  bool found = false;
  std::vector<char> line(1 << 16);
  while (std::fgets(line.data(), static_cast<int>(line.size()), f)) {
    std::string s(line.data());
    while (!s.empty() && (s.back() == '\n' || s.back() == '\r')) s.pop_back();
    const size_t pos = s.find(" table=");
    if (pos == std::string::npos || s.compare(0, pos, key) != 0 || pos != key.size()) continue;
    std::vector<int32_t> t;
    const char* p = s.c_str() + pos + 7;
    bool ok = true;
    for (int b = 0; b < kTuneBuckets && ok; ++b) {
      int v = -1, bf = -1, n = 0;
      ok = std::sscanf(p, "%d,%d%n", &v, &bf, &n) == 2 && v >= 0 && v < kMixVariants &&
           bf >= 0 && bf <= (1 << 20);
      if (!ok) break;
      t.push_back(v);
      t.push_back(bf);
      p += n;
      if (b + 1 < kTuneBuckets) ok = *p++ == ';';
    }
    if (ok) {
      tab = t;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

bool tune_save(const char* path, const std::string& key, const std::vector<int32_t>& tab) {
  FILE* f = std::fopen(path, "a");
  if (!f) return false;
  std::fprintf(f, "%s table=", key.c_str());
  for (int b = 0; b < kTuneBuckets; ++b)
    std::fprintf(f, "%d,%d%s", tab[2 * b], tab[2 * b + 1], b + 1 < kTuneBuckets ? ";" : "\n");
  return std::fclose(f) == 0;
}

// Make c->tune_host the context's table: on the device for the block steps'
// plan, the shape of the largest bucket as the context's own, and graphs
// captured with the old shapes dropped.
cudaError_t tune_apply(nb_ctx* c) {
  cudaError_t e = cudaMemcpyAsync(c->d.tune, c->tune_host.data(), 8 * (size_t)kTuneBuckets,
                                  cudaMemcpyHostToDevice, c->st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(c->st);  // the host copy may change after this
  if (e != cudaSuccess) return e;
  c->tabled = true;
  c->cfg.variant = c->tune_host[2 * tune_bucket(c->d.N)];
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

void nb_default_config(nb_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->G = 1.0;
  cfg->eps = 1e-4;
  cfg->eta = 0.01;
  cfg->eta_start = 0.01;
  cfg->level_min = 0;
  cfg->level_max = 30;
  cfg->tick_exp = 40;
  cfg->precision = NB_MIXED;
  cfg->bfactor = 0;
  cfg->graph_steps = 16;
  cfg->sort_sources = 1;
  cfg->variant = kMixDefaultVariant;
  cfg->order = 4;
}

int nb_workspace_size(int64_t n_total, int32_t n_clusters, const nb_config* cfg, size_t* bytes) {
  if (!bytes || !config_ok(cfg) || n_clusters < 1 || n_total < n_clusters ||
      n_total > (int64_t)INT32_MAX - 1024)
    return NB_EINVAL;
  // worst case of the slot padding (3 pad slots per cluster) and of the
  // tile count (one partial tile per cluster)
  const int64_t S = n_total + 3 * (int64_t)n_clusters;
  *bytes = make_layout(n_total, n_clusters, S, S / kMixJT + n_clusters, cfg->order).total;
  return NB_OK;
}

int nb_init(nb_ctx** out, const nb_config* cfg, int32_t n_clusters, const int64_t* offsets,
            const double* mass, const double* pos, const double* vel, void* workspace,
            size_t workspace_bytes, void* stream) {
  NvtxRange nvtx_range("nb_init");
  if (!out || !config_ok(cfg) || n_clusters < 1 || !offsets || !mass || !pos || !vel ||
      !workspace)
    return NB_EINVAL;
  *out = nullptr;
  if (offsets[0] != 0) return NB_EINVAL;
  for (int32_t k = 0; k < n_clusters; ++k)
    if (offsets[k + 1] <= offsets[k]) return NB_EINVAL;
  const int64_t N = offsets[n_clusters];
  if (N > (int64_t)INT32_MAX - 1024) return NB_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return NB_EINVAL;
  if (!finite_all(mass, N) || !finite_all(pos, 3 * N) || !finite_all(vel, 3 * N)) return NB_EINVAL;
  for (int64_t i = 0; i < N; ++i)
    if (mass[i] < 0.0) return NB_EINVAL;
  size_t need = 0;
  if (nb_workspace_size(N, n_clusters, cfg, &need) != NB_OK) return NB_EINVAL;
  if (workspace_bytes < need) return NB_ENOMEM;

  nb_ctx* c = new nb_ctx();
  c->cfg = *cfg;
  if (c->cfg.precision == NB_DS || c->cfg.precision == NB_FP32) c->cfg.variant = kMixDefaultVariant;
  c->st = static_cast<cudaStream_t>(stream);
  c->off_host.assign(offsets, offsets + n_clusters + 1);
  c->mass_host.assign(mass, mass + N);
  const int64_t S = slots_of(offsets, n_clusters);
  const int64_t n_tiles = tiles_of(offsets, n_clusters);
  c->L = make_layout(N, n_clusters, S, n_tiles, cfg->order);
  char* w = static_cast<char*>(workspace);
  Dev& d = c->d;
  d.N = N;
  d.S = S;
  d.K = n_clusters;
  d.pos = reinterpret_cast<dbl4*>(w + c->L.pos);
  d.vel = reinterpret_cast<dbl4*>(w + c->L.vel);
  d.acc = reinterpret_cast<dbl4*>(w + c->L.acc);
  d.jerk = reinterpret_cast<dbl4*>(w + c->L.jerk);
  d.acc_new = reinterpret_cast<dbl4*>(w + c->L.acc_new);
  d.jerk_new = reinterpret_cast<dbl4*>(w + c->L.jerk_new);
  d.t = reinterpret_cast<int64_t*>(w + c->L.t);
  d.level = reinterpret_cast<int32_t*>(w + c->L.level);
  d.cid = reinterpret_cast<int32_t*>(w + c->L.cid);
  d.active = reinterpret_cast<int32_t*>(w + c->L.active);
  d.src_mix = reinterpret_cast<float4*>(w + c->L.src_mix);
  d.src64_pos = reinterpret_cast<dbl4*>(w + c->L.src64_pos);
  d.src64_vel = reinterpret_cast<dbl4*>(w + c->L.src64_vel);
  d.partials = reinterpret_cast<double*>(w + c->L.partials);
  d.part_items = c->L.part_items;
  d.blk_count = reinterpret_cast<int32_t*>(w + c->L.blk_count);
  d.off = reinterpret_cast<int64_t*>(w + c->L.off);
  d.soff = reinterpret_cast<int64_t*>(w + c->L.soff);
  d.t_cur = reinterpret_cast<int64_t*>(w + c->L.t_cur);
  d.t_min = reinterpret_cast<int64_t*>(w + c->L.t_min);
  d.act_off = reinterpret_cast<int32_t*>(w + c->L.act_off);
  d.item_off = reinterpret_cast<int32_t*>(w + c->L.item_off);
  d.wt_off = reinterpret_cast<int32_t*>(w + c->L.wt_off);
  d.wide_cnt = reinterpret_cast<int32_t*>(w + c->L.wide_cnt);
  d.bfac = reinterpret_cast<int32_t*>(w + c->L.bfac);
  d.esum = reinterpret_cast<double*>(w + c->L.esum);
  d.status = reinterpret_cast<uint32_t*>(w + c->L.status);
  d.counters = reinterpret_cast<unsigned long long*>(w + c->L.counters);
  d.t_end = reinterpret_cast<int64_t*>(w + c->L.t_end);
  d.work_ctr = reinterpret_cast<int32_t*>(w + c->L.work);
  d.tune = reinterpret_cast<int32_t*>(w + c->L.tune);
  d.sel = reinterpret_cast<int32_t*>(w + c->L.sel);
  d.due_mask = reinterpret_cast<uint32_t*>(w + c->L.due_mask);
  d.order = cfg->order;
  if (cfg->order == 6) {
    d.snap = reinterpret_cast<dbl4*>(w + c->L.snap);
    d.crackle = reinterpret_cast<dbl4*>(w + c->L.crackle);
    d.snap_new = reinterpret_cast<dbl4*>(w + c->L.snap_new);
    d.src_acc_mix = reinterpret_cast<float4*>(w + c->L.src_acc_mix);
    d.src64_acc = reinterpret_cast<dbl4*>(w + c->L.src64_acc);
  }
  d.tiles = reinterpret_cast<float4*>(w + c->L.tiles);
  d.toff = reinterpret_cast<int32_t*>(w + c->L.toff);
  d.n_tiles = n_tiles;
  d.sperm = reinterpret_cast<int32_t*>(w + c->L.sperm);
  d.sinv = reinterpret_cast<int32_t*>(w + c->L.sinv);
  d.mark = reinterpret_cast<int32_t*>(w + c->L.mark);
  d.rows = reinterpret_cast<int32_t*>(w + c->L.rows);

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete c;
    return NB_ECUDA;
  }
  c->grid_mix = sep_mode(c) ? sms * force_mixed_sep_ctas_per_sm(sep_mode(c))
                            : sms * force_mixed_ctas_per_sm(c->cfg.variant);
  for (int v = 0; v < kMixVariants; ++v) c->grid_v[v] = sms * force_mixed_ctas_per_sm(v);
  c->tune_host.assign(2 * kTuneBuckets, 0);
  for (int b = 0; b < kTuneBuckets; ++b) {
    c->tune_host[2 * b] = c->cfg.variant;
    c->tune_host[2 * b + 1] = c->cfg.bfactor;
  }
  c->grid_f64 = sms * force_fp64_ctas_per_sm();
  c->grid_acc = sms * force_mixed_acc_ctas_per_sm();
  c->grid_snap = sms * force_mixed_snap_ctas_per_sm();
  c->sms = sms;
  if (integrator_setup() != cudaSuccess) {
    delete c;
    return NB_ECUDA;
  }

  // host staging of the initial state
  std::vector<double> p4(4 * N), v4(4 * N, 0.0);
  std::vector<int32_t> cid(N);
  std::vector<int64_t> soff(n_clusters + 1, 0);
  std::vector<int32_t> toff(n_clusters + 1, 0);
  for (int32_t k = 0; k < n_clusters; ++k) {
    soff[k + 1] = soff[k] + round_up64(offsets[k + 1] - offsets[k], 4);
    toff[k + 1] = toff[k] + static_cast<int32_t>(ceil_div64(soff[k + 1] - soff[k], kMixJT));
    for (int64_t i = offsets[k]; i < offsets[k + 1]; ++i) cid[i] = k;
  }
  std::vector<int32_t> sperm(S), sinv(N);
  source_order(pos, offsets, n_clusters, soff.data(), cfg->sort_sources != 0, sperm, sinv);
  c->sperm_host = sperm;
  for (int64_t i = 0; i < N; ++i) {
    p4[4 * i] = pos[3 * i];
    p4[4 * i + 1] = pos[3 * i + 1];
    p4[4 * i + 2] = pos[3 * i + 2];
    p4[4 * i + 3] = mass[i];
    v4[4 * i] = vel[3 * i];
    v4[4 * i + 1] = vel[3 * i + 1];
    v4[4 * i + 2] = vel[3 * i + 2];
  }
  const int64_t big = LLONG_MAX;
  int rc = NB_OK;
  cudaStream_t st = c->st;
  do {
    if (cudaMemcpyAsync(d.pos, p4.data(), 32 * N, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(d.vel, v4.data(), 32 * N, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(d.cid, cid.data(), 4 * N, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(d.off, offsets, 8 * (n_clusters + 1), cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(d.soff, soff.data(), 8 * (n_clusters + 1), cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(d.toff, toff.data(), 4 * (n_clusters + 1), cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(d.sperm, sperm.data(), 4 * S, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(d.sinv, sinv.data(), 4 * N, cudaMemcpyHostToDevice, st) ||
        cudaMemsetAsync(d.acc, 0, 32 * N, st) || cudaMemsetAsync(d.jerk, 0, 32 * N, st) ||
        cudaMemsetAsync(d.t, 0, 8 * N, st) || cudaMemsetAsync(d.level, 0, 4 * N, st) ||
        cudaMemsetAsync(d.t_cur, 0, 8 * n_clusters, st) ||
        cudaMemsetAsync(d.status, 0, 4, st) || cudaMemsetAsync(d.counters, 0, 32, st) ||
        cudaMemsetAsync(d.wide_cnt, 0, 4 * (size_t)wide_counter_entries(c->L.part_items), st) ||
        cudaMemsetAsync(d.mark, 0xff, 4 * N, st) ||
        cudaMemcpyAsync(d.tune, c->tune_host.data(), 8 * (size_t)kTuneBuckets,
                        cudaMemcpyHostToDevice, st) ||
        (cfg->order == 6 && (cudaMemsetAsync(d.snap, 0, 32 * N, st) ||
                             cudaMemsetAsync(d.crackle, 0, 32 * N, st)))) {
      rc = NB_ECUDA;
      break;
    }
    if (launch_fill_i64(d.t_min, n_clusters, big, st) || launch_fill_i64(d.t_end, 1, big, st)) {
      rc = NB_ECUDA;
      break;
    }
    const bool f64 = !is_mixed(c);
    double* an = reinterpret_cast<double*>(d.acc_new);
    double* jn = reinterpret_cast<double*>(d.jerk_new);
    // every particle, targets in slot order, results to their particle rows
    if (launch_predict(d, nullptr, 0, cfg->tick_exp, !f64, f64, false, st) ||
        launch_slot_list(d, st) || launch_actoff_identity(d, st) ||
        enqueue_force(c, d.active, d.active, an, 4, jn, 4, an + 3, 4, f64, 0, 0, false, N) ||
        launch_init_levels(d, cfg->eta_start, cfg->tick_exp, cfg->level_min, cfg->level_max, st)) {
      rc = NB_ECUDA;
      break;
    }
    if (cfg->order == 6) {
      // snap at t = 0 from the sources' accelerations a0 (the predictor at
      // tau = 0 writes them; snap and crackle were zeroed above, and the
      // crackle stays zero): the start of the 6th-order scheme
      if (launch_predict(d, nullptr, 0, cfg->tick_exp, !f64, f64, false, st, true) ||
          launch_slot_list(d, st) || launch_actoff_identity(d, st) ||
          enqueue_force_snap(c, d.active, d.active, an, 4, jn, 4,
                             reinterpret_cast<double*>(d.snap), 4, nullptr, 0, 0, 0, N)) {
        rc = NB_ECUDA;
        break;
      }
    }
    rc = sync_status(c);
  } while (false);
  if (rc != NB_OK) {
    cudaStreamSynchronize(st);
    delete c;
    return rc;
  }
  *out = c;
  return NB_OK;
}

void nb_free(nb_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (auto& p : c->ev_pending) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  for (auto e : c->ev_free) cudaEventDestroy(e);
  delete c;
}

int nb_predict(nb_ctx* c, int64_t t_ticks) {
  NvtxRange nvtx_range("nb_predict");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || t_ticks < 0) return NB_EINVAL;
  const bool f64 = !is_mixed(c);
  NB_TRY(launch_predict(c->d, nullptr, t_ticks, c->cfg.tick_exp, !f64, f64, false, c->st));
  return NB_OK;
}

int nb_force(nb_ctx* c, const int32_t* active_idx, int64_t m, double* acc, double* jerk,
             double* pot) {
  NvtxRange nvtx_range("nb_force");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || m < 0 || m > c->d.N) return NB_EINVAL;
  if (m == 0) return NB_OK;
  if (!active_idx || !acc) return NB_EINVAL;
  const bool f64 = !is_mixed(c);
  // targets in source-slot order (spatially coherent warps), rows mapped back
  NB_TRY(launch_list_to_slots(c->d, active_idx, m, c->st));
  NB_TRY(enqueue_force(c, c->d.active, c->d.rows, acc, 3, jerk, 3, pot, 1, f64, 0, 1, false, m,
                       false, m));
  return NB_OK;
}

int nb_force_snap(nb_ctx* c, const int32_t* active_idx, int64_t m, double* acc, double* jerk,
                  double* snap, double* pot) {
  NvtxRange nvtx_range("nb_force_snap");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || m < 0 || m > c->d.N) return NB_EINVAL;
  if (c->cfg.order != 6) return NB_ESTATE;
  if (m == 0) return NB_OK;
  if (!active_idx || !acc || !jerk || !snap) return NB_EINVAL;
  NB_TRY(launch_list_to_slots(c->d, active_idx, m, c->st));
  NB_TRY(enqueue_force_snap(c, c->d.active, c->d.rows, acc, 3, jerk, 3, snap, 3, pot, 1, 0, 1,
                            m));
  return NB_OK;
}

int nb_source_piece(int64_t n_slots, int32_t part, int32_t n_parts, int64_t* slot_begin,
                    int64_t* slot_end) {
  if (n_slots < 0 || n_parts < 1 || part < 0 || part >= n_parts || !slot_begin || !slot_end)
    return NB_EINVAL;
  src_piece(n_slots, part, n_parts, slot_begin, slot_end);
  return NB_OK;
}

int nb_source_order(nb_ctx* c, int64_t* n_slots, int32_t* particle_of_slot,
                    int64_t* slot_offsets) {
  if (!c || !n_slots) return NB_EINVAL;
  *n_slots = c->d.S;
  if (particle_of_slot)
    std::copy(c->sperm_host.begin(), c->sperm_host.end(), particle_of_slot);
  if (slot_offsets) {
    slot_offsets[0] = 0;
    for (int32_t k = 0; k < c->d.K; ++k)
      slot_offsets[k + 1] =
          slot_offsets[k] + round_up64(c->off_host[k + 1] - c->off_host[k], 4);
  }
  return NB_OK;
}

int nb_force_range(nb_ctx* c, const int32_t* active_idx, int64_t m, int32_t part,
                   int32_t n_parts, double* acc, double* jerk, double* pot) {
  NvtxRange nvtx_range("nb_force_range");
  if (!c || n_parts < 1 || part < 0 || part >= n_parts) return NB_EINVAL;
  PieceScope piece(c, part, n_parts);
  return nb_force(c, active_idx, m, acc, jerk, pot);
}

int nb_block_force(nb_ctx* c, int32_t part, int32_t n_parts, int64_t* m_out, double** acc_rows,
                   double** jerk_rows, double** snap_rows) {
  NvtxRange nvtx_range("nb_block_force");
  if (!c || !m_out || n_parts < 1 || part < 0 || part >= n_parts) return NB_EINVAL;
  if (c->block_open) return NB_ESTATE;
  {
    PieceScope piece(c, part, n_parts);
    NB_TRY(enqueue_block_force(c));
  }
  int32_t m = 0;
  NB_TRY(cudaMemcpyAsync(&m, c->d.act_off + c->d.K, sizeof m, cudaMemcpyDeviceToHost, c->st));
  const int rc = sync_status(c);
  if (rc != NB_OK) return rc;
  c->block_open = true;
  *m_out = m;
  if (acc_rows) *acc_rows = reinterpret_cast<double*>(c->d.acc_new);
  if (jerk_rows) *jerk_rows = reinterpret_cast<double*>(c->d.jerk_new);
  if (snap_rows) *snap_rows = reinterpret_cast<double*>(c->d.snap_new);
  return NB_OK;
}

int nb_block_correct(nb_ctx* c) {
  NvtxRange nvtx_range("nb_block_correct");
  if (!c) return NB_EINVAL;
  if (!c->block_open) return NB_ESTATE;
  c->block_open = false;
  NB_TRY(enqueue_block_correct(c));
  return NB_OK;
}

int nb_resort_sources(nb_ctx* c) {
  NvtxRange nvtx_range("nb_resort_sources");
  if (!c) return NB_EINVAL;
  if (c->block_open) return NB_ESTATE;
  Dev& d = c->d;
  const int64_t N = d.N;
  const int32_t K = d.K;
  std::vector<double> p4(4 * N), p3(3 * N);
  NB_TRY(cudaMemcpyAsync(p4.data(), d.pos, 32 * N, cudaMemcpyDeviceToHost, c->st));
  int rc = sync_status(c);
  if (rc != NB_OK) return rc;
  for (int64_t i = 0; i < N; ++i)
    for (int q = 0; q < 3; ++q) p3[3 * i + q] = p4[4 * i + q];
  std::vector<int64_t> soff(K + 1, 0);
  for (int32_t k = 0; k < K; ++k)
    soff[k + 1] = soff[k] + round_up64(c->off_host[k + 1] - c->off_host[k], 4);
  std::vector<int32_t> sperm(d.S), sinv(N);
  source_order(p3.data(), c->off_host.data(), K, soff.data(), c->cfg.sort_sources != 0, sperm,
               sinv);
  NB_TRY(cudaMemcpyAsync(d.sperm, sperm.data(), 4 * d.S, cudaMemcpyHostToDevice, c->st));
  NB_TRY(cudaMemcpyAsync(d.sinv, sinv.data(), 4 * N, cudaMemcpyHostToDevice, c->st));
  // the sources in the new order, predicted to each cluster's block time
  const bool f64 = !is_mixed(c);
  NB_TRY(launch_predict(d, d.t_cur, 0, c->cfg.tick_exp, !f64, f64, false, c->st));
  rc = sync_status(c);  // the host vectors are released after this
  if (rc != NB_OK) return rc;
  c->sperm_host = sperm;
  return NB_OK;
}

int nb_correct_snap(nb_ctx* c, int64_t t_ticks, const int32_t* active_idx, int64_t m,
                    const double* acc, const double* jerk, const double* snap) {
  NvtxRange nvtx_range("nb_correct_snap");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || m < 0 || m > c->d.N || t_ticks < 0) return NB_EINVAL;
  if (c->cfg.order != 6) return NB_ESTATE;
  if (m == 0) return NB_OK;
  if (!active_idx || !acc || !jerk || !snap) return NB_EINVAL;
  CorrectArgs ca{};
  ca.active = active_idx;
  ca.count_dev = nullptr;
  ca.count_host = m;
  ca.acc = acc;
  ca.sa = 3;
  ca.jerk = jerk;
  ca.sj = 3;
  ca.snap = snap;
  ca.ss = 3;
  ca.pot = nullptr;
  ca.t_tgt = nullptr;
  ca.t_fixed = t_ticks;
  ca.eta = c->cfg.eta;
  ca.T = c->cfg.tick_exp;
  ca.lmin = c->cfg.level_min;
  ca.lmax = c->cfg.level_max;
  NB_TRY(launch_correct6(c->d, ca, m, c->st));
  return NB_OK;
}

int nb_get_derivs(nb_ctx* c, double* snap, double* crackle) {
  NvtxRange nvtx_range("nb_get_derivs");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c) return NB_EINVAL;
  if (c->cfg.order != 6) return NB_ESTATE;
  const int64_t N = c->d.N;
  const dbl4* srcs[2] = {c->d.snap, c->d.crackle};
  double* dsts[2] = {snap, crackle};
  double* stage[2] = {reinterpret_cast<double*>(c->d.acc_new),
                      reinterpret_cast<double*>(c->d.jerk_new)};
  for (int q = 0; q < 2; ++q) {
    if (!dsts[q]) continue;
    NB_TRY(launch_unpack3(srcs[q], stage[q], N, c->st));
    NB_TRY(cudaMemcpyAsync(dsts[q], stage[q], 24 * N, cudaMemcpyDeviceToHost, c->st));
  }
  NB_TRY(cudaStreamSynchronize(c->st));
  return NB_OK;
}

int nb_set_derivs(nb_ctx* c, const double* snap, const double* crackle) {
  NvtxRange nvtx_range("nb_set_derivs");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || !snap || !crackle) return NB_EINVAL;
  if (c->cfg.order != 6) return NB_ESTATE;
  const int64_t N = c->d.N;
  if (!finite_all(snap, 3 * N) || !finite_all(crackle, 3 * N)) return NB_EINVAL;
  double* sa = reinterpret_cast<double*>(c->d.acc_new);
  double* sb = reinterpret_cast<double*>(c->d.jerk_new);
  NB_TRY(cudaMemcpyAsync(sa, snap, 24 * N, cudaMemcpyHostToDevice, c->st));
  NB_TRY(cudaMemcpyAsync(sb, crackle, 24 * N, cudaMemcpyHostToDevice, c->st));
  NB_TRY(launch_pack3(sa, c->d.snap, N, false, c->st));
  NB_TRY(launch_pack3(sb, c->d.crackle, N, false, c->st));
  NB_TRY(cudaStreamSynchronize(c->st));
  return NB_OK;
}

int nb_correct(nb_ctx* c, int64_t t_ticks, const int32_t* active_idx, int64_t m,
               const double* acc, const double* jerk) {
  NvtxRange nvtx_range("nb_correct");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || m < 0 || m > c->d.N || t_ticks < 0) return NB_EINVAL;
  if (c->cfg.order == 6) return NB_ESTATE;
  if (m == 0) return NB_OK;
  if (!active_idx || !acc || !jerk) return NB_EINVAL;
  CorrectArgs ca{};
  ca.active = active_idx;
  ca.count_dev = nullptr;
  ca.count_host = m;
  ca.acc = acc;
  ca.sa = 3;
  ca.jerk = jerk;
  ca.sj = 3;
  ca.pot = nullptr;
  ca.t_tgt = nullptr;
  ca.t_fixed = t_ticks;
  ca.eta = c->cfg.eta;
  ca.T = c->cfg.tick_exp;
  ca.lmin = c->cfg.level_min;
  ca.lmax = c->cfg.level_max;
  NB_TRY(launch_correct(c->d, ca, m, c->st));
  return NB_OK;
}

int nb_step_leapfrog(nb_ctx* c, int64_t n_steps, int64_t dt_ticks) {
  NvtxRange nvtx_range("nb_step_leapfrog");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || n_steps < 0 || dt_ticks <= 0 || dt_ticks > ((int64_t)1 << 52)) return NB_EINVAL;
  if (n_steps == 0) return NB_OK;
  const bool f64 = !is_mixed(c);
  const int T = c->cfg.tick_exp;
  const double dt = std::ldexp(static_cast<double>(dt_ticks), -T);
  double* an = reinterpret_cast<double*>(c->d.acc_new);
  for (int64_t s = 0; s < n_steps; ++s) {
    NB_TRY(launch_leapfrog(c->d, nullptr, 0.5 * dt, dt, dt_ticks, c->st));  // kick, drift
    NB_TRY(launch_predict(c->d, nullptr, 0, T, !f64, f64, false, c->st, true));
    NB_TRY(launch_slot_list(c->d, c->st));
    NB_TRY(launch_actoff_identity(c->d, c->st));
    // acceleration at the new positions: no jerk (the acceleration-only
    // kernel), targets in slot order, results to their particle rows
    NB_TRY(enqueue_force(c, c->d.active, c->d.active, an, 4, nullptr, 0, nullptr, 0, f64, 0, 1,
                         false, c->d.N));
    NB_TRY(launch_leapfrog(c->d, an, 0.5 * dt, dt, 0, c->st));  // kick
  }
  NB_TRY(launch_tcur_from_t(c->d, c->st));
  return NB_OK;
}

int nb_step_block(nb_ctx* c, int64_t n_steps, int64_t* t_ticks_out, int64_t* m_last_out) {
  NvtxRange nvtx_range("nb_step_block");
  if (!c || n_steps < 0) return NB_EINVAL;
  if (c->block_open) return NB_ESTATE;
  if (n_steps == 0 && m_last_out) {
    // nothing corrected: clear the count the report below reads
    NB_TRY(cudaMemsetAsync(c->d.act_off + c->d.K, 0, sizeof(int32_t), c->st));
  }
  const int G = c->cfg.graph_steps;
  const bool graphs = G > 0 && c->st != nullptr && !c->graph_broken && !c->prof;
  if (graphs && c->graph == nullptr && n_steps >= G) {
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      for (int s = 0; s < G && ok; ++s) ok = enqueue_block_step(c) == cudaSuccess;
      const bool ended = cudaStreamEndCapture(c->st, &g) == cudaSuccess;
      ok = ok && ended && cudaGraphInstantiate(&c->graph, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
    }
    if (!ok) {
      c->graph = nullptr;
      c->graph_broken = true;  // fall back to direct launches of the same kernels
      cudaGetLastError();
    } else {
      c->graph_len = G;
    }
  }
  int64_t left = n_steps;
  if (c->graph && !c->prof) {
    while (left >= c->graph_len) {
      NB_TRY(cudaGraphLaunch(c->graph, c->st));
      left -= c->graph_len;
    }
  }
  for (; left > 0; --left) NB_TRY(enqueue_block_step(c));
  if (!t_ticks_out && !m_last_out) return NB_OK;
  // report: the last step's active count (act_off[K], which its plan wrote)
  // and the clusters' block times
  int32_t m_last = 0;
  std::vector<int64_t> tc(c->d.K);
  NB_TRY(cudaMemcpyAsync(&m_last, c->d.act_off + c->d.K, sizeof m_last, cudaMemcpyDeviceToHost,
                         c->st));
  NB_TRY(cudaMemcpyAsync(tc.data(), c->d.t_cur, 8 * (size_t)c->d.K, cudaMemcpyDeviceToHost,
                         c->st));
  const int rc = sync_status(c);
  if (rc != NB_OK) return rc;
  if (t_ticks_out) *t_ticks_out = *std::min_element(tc.begin(), tc.end());
  if (m_last_out) *m_last_out = m_last;
  return NB_OK;
}

int nb_set_end_time(nb_ctx* c, int64_t t_end_ticks) {
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || t_end_ticks < 0) return NB_EINVAL;
  NB_TRY(launch_fill_i64(c->d.t_end, 1, t_end_ticks, c->st));
  return NB_OK;
}

int nb_energy(nb_ctx* c, int32_t cluster, double* ekin, double* epot) {
  NvtxRange nvtx_range("nb_energy");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || !ekin || !epot || cluster < -1 || cluster >= c->d.K) return NB_EINVAL;
  Dev& d = c->d;
  double* an = reinterpret_cast<double*>(d.acc_new);
  NB_TRY(launch_predict(d, d.t_cur, 0, c->cfg.tick_exp, false, true, false, c->st));
  NB_TRY(launch_actoff_identity(d, c->st));
  NB_TRY(enqueue_force(c, nullptr, nullptr, nullptr, 0, nullptr, 0, an + 3, 4, true, 0, 0, true,
                       d.N));
  const int64_t lo = cluster < 0 ? 0 : c->off_host[cluster];
  const int64_t hi = cluster < 0 ? d.N : c->off_host[cluster + 1];
  double* out = d.esum + 2 * kEnergyBlocks;
  NB_TRY(launch_energy(d, an + 3, 4, lo, hi, d.esum, kEnergyBlocks, out, c->st));
  double h[2];
  NB_TRY(cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, c->st));
  const int rc = sync_status(c);
  if (rc != NB_OK) return rc;
  *ekin = h[0];
  *epot = h[1];
  return NB_OK;
}

int nb_energies(nb_ctx* c, double* ekin, double* epot) {
  NvtxRange nvtx_range("nb_energies");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || !ekin || !epot) return NB_EINVAL;
  Dev& d = c->d;
  double* an = reinterpret_cast<double*>(d.acc_new);
  NB_TRY(launch_predict(d, d.t_cur, 0, c->cfg.tick_exp, false, true, false, c->st));
  NB_TRY(launch_actoff_identity(d, c->st));
  NB_TRY(enqueue_force(c, nullptr, nullptr, nullptr, 0, nullptr, 0, an + 3, 4, true, 0, 0, true,
                       d.N));
  std::vector<double> h(2 * (size_t)d.K);
  double* out = d.esum + 2 * kEnergyBlocks;
  for (int32_t k = 0; k < d.K; ++k) {
    NB_TRY(launch_energy(d, an + 3, 4, c->off_host[k], c->off_host[k + 1], d.esum, kEnergyBlocks,
                         out, c->st));
    NB_TRY(cudaMemcpyAsync(h.data() + 2 * k, out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                           c->st));
  }
  const int rc = sync_status(c);
  if (rc != NB_OK) return rc;
  for (int32_t k = 0; k < d.K; ++k) {
    ekin[k] = h[2 * k];
    epot[k] = h[2 * k + 1];
  }
  return NB_OK;
}

int nb_get_state(nb_ctx* c, double* pos, double* vel, double* acc, double* jerk, int64_t* t,
                 int32_t* level) {
  NvtxRange nvtx_range("nb_get_state");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c) return NB_EINVAL;
  const int64_t N = c->d.N;
  // pack (n, 3) rows into the step scratch (acc_new / jerk_new), then copy
  // straight into the caller's arrays
  double* sa = reinterpret_cast<double*>(c->d.acc_new);
  double* sb = reinterpret_cast<double*>(c->d.jerk_new);
  const dbl4* srcs[4] = {c->d.pos, c->d.vel, c->d.acc, c->d.jerk};
  double* dsts[4] = {pos, vel, acc, jerk};
  for (int q = 0; q < 4; q += 2) {
    for (int r = 0; r < 2; ++r) {
      if (!dsts[q + r]) continue;
      double* stage = r == 0 ? sa : sb;
      NB_TRY(launch_unpack3(srcs[q + r], stage, N, c->st));
      NB_TRY(cudaMemcpyAsync(dsts[q + r], stage, 24 * N, cudaMemcpyDeviceToHost, c->st));
    }
    NB_TRY(cudaStreamSynchronize(c->st));  // stage reuse by the next pair
  }
  if (t) NB_TRY(cudaMemcpyAsync(t, c->d.t, 8 * N, cudaMemcpyDeviceToHost, c->st));
  if (level) NB_TRY(cudaMemcpyAsync(level, c->d.level, 4 * N, cudaMemcpyDeviceToHost, c->st));
  NB_TRY(cudaStreamSynchronize(c->st));
  return NB_OK;
}

int nb_set_state(nb_ctx* c, const double* pos, const double* vel, const double* acc,
                 const double* jerk, const int64_t* t, const int32_t* level) {
  NvtxRange nvtx_range("nb_set_state");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || !pos || !vel || !acc || !jerk || !t || !level) return NB_EINVAL;
  const int64_t N = c->d.N;
  const int T = c->cfg.tick_exp;
  for (int64_t i = 0; i < N; ++i) {
    if (level[i] < c->cfg.level_min || level[i] > c->cfg.level_max || t[i] < 0) return NB_EINVAL;
    if (t[i] & (((int64_t)1 << (T - level[i])) - 1)) return NB_EINVAL;
  }
  if (!finite_all(pos, 3 * N) || !finite_all(vel, 3 * N) || !finite_all(acc, 3 * N) ||
      !finite_all(jerk, 3 * N))
    return NB_EINVAL;
  double* sa = reinterpret_cast<double*>(c->d.acc_new);
  double* sb = reinterpret_cast<double*>(c->d.jerk_new);
  NB_TRY(cudaMemcpyAsync(sa, pos, 24 * N, cudaMemcpyHostToDevice, c->st));
  NB_TRY(cudaMemcpyAsync(sb, vel, 24 * N, cudaMemcpyHostToDevice, c->st));
  NB_TRY(launch_pack3(sa, c->d.pos, N, true, c->st));    // keeps the masses
  NB_TRY(launch_pack3(sb, c->d.vel, N, false, c->st));
  NB_TRY(cudaStreamSynchronize(c->st));  // host arrays may be pageable: stage reuse
  NB_TRY(cudaMemcpyAsync(sa, acc, 24 * N, cudaMemcpyHostToDevice, c->st));
  NB_TRY(cudaMemcpyAsync(sb, jerk, 24 * N, cudaMemcpyHostToDevice, c->st));
  NB_TRY(launch_pack3(sa, c->d.acc, N, true, c->st));    // keeps the potentials
  NB_TRY(launch_pack3(sb, c->d.jerk, N, false, c->st));
  NB_TRY(cudaMemcpyAsync(c->d.t, t, 8 * N, cudaMemcpyHostToDevice, c->st));
  NB_TRY(cudaMemcpyAsync(c->d.level, level, 4 * N, cudaMemcpyHostToDevice, c->st));
  NB_TRY(cudaMemsetAsync(c->d.t_cur, 0, 8 * (size_t)c->d.K, c->st));
  NB_TRY(launch_tcur_from_t(c->d, c->st));
  NB_TRY(cudaStreamSynchronize(c->st));
  return NB_OK;
}

int nb_stats(nb_ctx* c, int64_t* block_steps, int64_t* interactions, int64_t* t_min,
             int64_t* t_max) {
  if (!c) return NB_EINVAL;
  unsigned long long ctr[4];
  std::vector<int64_t> tc(c->d.K);
  NB_TRY(cudaMemcpyAsync(ctr, c->d.counters, sizeof ctr, cudaMemcpyDeviceToHost, c->st));
  NB_TRY(cudaMemcpyAsync(tc.data(), c->d.t_cur, 8 * c->d.K, cudaMemcpyDeviceToHost, c->st));
  NB_TRY(cudaStreamSynchronize(c->st));
  if (block_steps) *block_steps = (int64_t)ctr[1];
  if (interactions) *interactions = (int64_t)ctr[0];
  int64_t lo = LLONG_MAX, hi = LLONG_MIN;
  for (int64_t v : tc) {
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
  if (t_min) *t_min = lo;
  if (t_max) *t_max = hi;
  return NB_OK;
}

int nb_profile_enable(nb_ctx* c, int enable) {
  if (!c) return NB_EINVAL;
  c->prof = enable != 0;
  return NB_OK;
}

int nb_profile_read(nb_ctx* c, double* force_ms, int64_t* launches) {
  if (!c) return NB_EINVAL;
  NB_TRY(prof_collect(c, true));
  if (force_ms) *force_ms = c->prof_ms;
  if (launches) *launches = c->prof_launches;
  c->prof_ms = 0.0;
  c->prof_launches = 0;
  return NB_OK;
}

int nb_profile_kernels(nb_ctx* c, double* ms_by_kind, int64_t* launches_by_kind) {
  if (!c) return NB_EINVAL;
  NB_TRY(prof_collect(c, true));
  for (int k = 0; k < NB_PROFILE_KINDS; ++k) {
    if (ms_by_kind) ms_by_kind[k] = c->kind_ms[k];
    if (launches_by_kind) launches_by_kind[k] = c->kind_n[k];
    c->kind_ms[k] = 0.0;
    c->kind_n[k] = 0;
  }
  return NB_OK;
}

int nb_tile_stats(nb_ctx* c, int64_t* warp_tiles, int64_t* near_warp_tiles) {
  if (!c) return NB_EINVAL;
  unsigned long long ctr[2];
  NB_TRY(cudaMemcpyAsync(ctr, c->d.counters + 2, sizeof ctr, cudaMemcpyDeviceToHost, c->st));
  NB_TRY(cudaStreamSynchronize(c->st));
  if (warp_tiles) *warp_tiles = (int64_t)ctr[0];
  if (near_warp_tiles) *near_warp_tiles = (int64_t)ctr[1];
  return NB_OK;
}

int nb_autotune(nb_ctx* c, const char* cache_path, int32_t* variant_out, double* ms_out) {
  NvtxRange nvtx_range("nb_autotune");
  if (!c) return NB_EINVAL;
  if (c->block_open) return NB_ESTATE;
  if (ms_out)
    for (int q = 0; q < NB_TUNE_POINTS * kMixVariants; ++q) ms_out[q] = 0.0;
  if (c->cfg.precision != NB_MIXED) {  // FP64, DS, FP32: one shape each, nothing to choose
    if (variant_out) *variant_out = c->cfg.variant;
    return NB_OK;
  }
  const std::string key = tune_key(c);
  std::vector<int32_t> tab;
  if (cache_path && tune_load(cache_path, key, tab)) {
    c->tune_host = tab;
    NB_TRY(tune_apply(c));
    if (variant_out) *variant_out = c->cfg.variant;
    return sync_status(c);
  }
  Dev& d = c->d;
  const int saved_b = c->cfg.bfactor;
  c->tabled = false;  // every timed launch below runs the shape and B it is given
  cudaEvent_t e0, e1;
  NB_TRY(cudaEventCreate(&e0));
  NB_TRY(cudaEventCreate(&e1));
  double* an = reinterpret_cast<double*>(d.acc_new);
  double* jn = reinterpret_cast<double*>(d.jerk_new);
  std::vector<int64_t> soff(d.K + 1, 0);
  for (int32_t k = 0; k < d.K; ++k)
    soff[k + 1] = soff[k] + round_up64(c->off_host[k + 1] - c->off_host[k], 4);
  int rc = NB_OK;
  // one launch of shape v with split B on the current list: its time (ms);
  // launches under 5 ms are repeated and the best of five is kept
  auto time_one = [&](int v, int B, double* out) -> bool {
    c->cfg.variant = v;
    c->cfg.bfactor = B;
    double best = 1e30;
    for (int r = 0; r < 5; ++r) {
      if (cudaEventRecord(e0, c->st) ||
          enqueue_force(c, d.active, nullptr, an, 4, jn, 4, nullptr, 0, false, 0, 0, false,
                        d.N) ||
          cudaEventRecord(e1, c->st) || cudaEventSynchronize(e1))
        return false;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      best = std::min(best, (double)t);
      if (best >= 5.0) break;
    }
    *out = best;
    return true;
  };
  struct Point { int64_t m; int v, B; };
  std::vector<Point> pts;
  for (int k = 0; k < NB_TUNE_POINTS && rc == NB_OK; ++k) {
    // every 4^k-th source slot of each cluster, in slot order
    const int64_t stride = (int64_t)1 << (2 * k);
    std::vector<int32_t> list;
    std::vector<int32_t> aoff(d.K + 1, 0);
    int64_t nit_max = 0;
    for (int32_t q = 0; q < d.K; ++q) {
      aoff[q] = static_cast<int32_t>(list.size());
      for (int64_t sl = soff[q]; sl < soff[q + 1]; sl += stride)
        if (c->sperm_host[sl] >= 0) list.push_back(c->sperm_host[sl]);
    }
    aoff[d.K] = static_cast<int32_t>(list.size());
    const int64_t m = static_cast<int64_t>(list.size());
    if (m == 0 || (k > 0 && m < 64)) break;
    if (cudaMemcpyAsync(d.active, list.data(), 4 * list.size(), cudaMemcpyHostToDevice, c->st) ||
        cudaMemcpyAsync(d.act_off, aoff.data(), 4 * aoff.size(), cudaMemcpyHostToDevice, c->st) ||
        cudaStreamSynchronize(c->st)) {
      rc = NB_ECUDA;
      break;
    }
    double warm = 0.0;
    if (!time_one(kMixDefaultVariant, 0, &warm)) { rc = NB_ECUDA; break; }
    // every shape with the plan's B
    int vbest = 0;
    double tbest = 1e30;
    for (int v = 0; v < kMixVariants; ++v) {
      double t = 0.0;
      if (!time_one(v, 0, &t)) { rc = NB_ECUDA; break; }
      if (ms_out) ms_out[k * kMixVariants + v] = t;
      if (t < tbest) { tbest = t; vbest = v; }
    }
    if (rc != NB_OK) break;
    const double ms_best_plan = tbest;
    // the fastest shape with B = 1, 2, 4, ... up to the partial-sum buffer's
    // capacity (the plan's own cap) and the clusters' tile counts
    const int ni = force_mixed_ni(vbest);
    for (int32_t q = 0; q < d.K; ++q) nit_max += ceil_div64(aoff[q + 1] - aoff[q], ni);
    const int64_t bcap = std::min<int64_t>(
        {c->L.part_items / std::max<int64_t>(nit_max, 1), ceil_div64(d.N, kMixJT), 4096});
    // the smallest B within 0.3 % of the fastest (timing noise): fewer
    // partial sums written and reduced for the same speed; the plan's own
    // choice (B = 0) last
    std::vector<std::pair<int, double>> cand;
    for (int64_t B = 1; B <= bcap && rc == NB_OK; B *= 2) {
      double t = 0.0;
      if (!time_one(vbest, static_cast<int>(B), &t)) { rc = NB_ECUDA; break; }
      cand.push_back({static_cast<int>(B), t});
      tbest = std::min(tbest, t);
    }
    if (rc != NB_OK) break;
    cand.push_back({0, ms_best_plan});
    int bbest = 0;
    for (const auto& cb : cand)
      if (cb.second <= tbest * 1.003) {
        bbest = cb.first;
        break;
      }
    pts.push_back({m, vbest, bbest});
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->cfg.bfactor = saved_b;
  if (rc != NB_OK || pts.empty()) {
    c->tabled = false;
    c->cfg.variant = c->tune_host.empty() ? kMixDefaultVariant : c->tune_host[2 * tune_bucket(d.N)];
    return rc != NB_OK ? rc : sync_status(c);
  }
  // every bucket from the measured point nearest in log2 m (ties: the larger
  // m); B scaled by the ratio of the active counts, the same fill of the grid
  tab.assign(2 * kTuneBuckets, 0);
  for (int b = 0; b < kTuneBuckets; ++b) {
    size_t best = 0;
    double dist = 1e30;
    for (size_t q = 0; q < pts.size(); ++q) {
      const double dq = std::fabs(std::log2((double)pts[q].m) - b);
      if (dq < dist - 1e-9) { dist = dq; best = q; }
    }
    const Point& p = pts[best];
    int B = p.B;
    if (B > 0) {
      const double scaled = p.B * (double)p.m / std::ldexp(1.0, b);
      B = static_cast<int>(std::min(4096.0, std::max(1.0, std::floor(scaled + 0.5))));
    }
    tab[2 * b] = p.v;
    tab[2 * b + 1] = B;
  }
  c->tune_host = tab;
  NB_TRY(tune_apply(c));
  if (variant_out) *variant_out = c->cfg.variant;
  if (cache_path && !tune_save(cache_path, key, tab)) return NB_EINVAL;
  return sync_status(c);
}

int nb_tune_table(nb_ctx* c, int32_t* variant_by_bucket, int32_t* bfactor_by_bucket) {
  if (!c) return NB_EINVAL;
  for (int b = 0; b < kTuneBuckets; ++b) {
    if (variant_by_bucket) variant_by_bucket[b] = c->tune_host[2 * b];
    if (bfactor_by_bucket) bfactor_by_bucket[b] = c->tune_host[2 * b + 1];
  }
  return NB_OK;
}

int nb_status(nb_ctx* c) {
  if (!c) return NB_EINVAL;
  return sync_status(c);
}

int nb_measure_rate(nb_ctx* c, int32_t kind, double* lanes_per_sm_clock) {
  NvtxRange nvtx_range("nb_measure_rate");
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || kind < 0 || kind > 2 || !lanes_per_sm_clock) return NB_EINVAL;
  const int per_sm = 4;
  const int ctas = c->sms * per_sm;
  const int iters = kind == 2 ? 2000 : 100000;
  // the partial-sum buffer is scratch between force evaluations
  const size_t need = probe_scratch_bytes(ctas);
  if (need > c->L.part_items * kPartialComps * (size_t)kMixNI * sizeof(double)) return NB_ENOMEM;
  void* scratch = c->d.partials;
  for (int rep = 0; rep < 2; ++rep) NB_TRY(launch_rate_probe(kind, ctas, iters, scratch, c->st));
  std::vector<long long> rec(3 * (size_t)ctas);
  const char* recp = static_cast<const char*>(scratch) + need - rec.size() * sizeof(long long);
  NB_TRY(cudaMemcpyAsync(rec.data(), recp, rec.size() * sizeof(long long), cudaMemcpyDeviceToHost,
                         c->st));
  NB_TRY(cudaStreamSynchronize(c->st));
  // per SM: its CTAs' operations over the span from first start to last end
  const double lanes_per_cta = probe_lanes_per_launch(kind, ctas, iters) / ctas;
  std::vector<long long> lo, hi;
  std::vector<int> n;
  std::vector<long long> ids;
  for (int b = 0; b < ctas; ++b) {
    const long long sm = rec[3 * b], t0 = rec[3 * b + 1], t1 = rec[3 * b + 2];
    size_t k = 0;
    while (k < ids.size() && ids[k] != sm) ++k;
    if (k == ids.size()) {
      ids.push_back(sm);
      lo.push_back(t0);
      hi.push_back(t1);
      n.push_back(0);
    }
    lo[k] = std::min(lo[k], t0);
    hi[k] = std::max(hi[k], t1);
    n[k] += 1;
  }
  std::vector<double> rate;
  for (size_t k = 0; k < ids.size(); ++k)
    if (hi[k] > lo[k]) rate.push_back(n[k] * lanes_per_cta / (double)(hi[k] - lo[k]));
  if (rate.empty()) return NB_ECUDA;
  std::sort(rate.begin(), rate.end());
  *lanes_per_sm_clock = rate[rate.size() / 2];
  return NB_OK;
}

int nb_check_wait_timeout(nb_ctx* c, double seconds) {
  if (c && c->block_open) return NB_ESTATE;  // a split block step is open
  if (!c || !(seconds > 0.0) || seconds > 10.0) return NB_EINVAL;
  int dev = 0, khz = 0;
  NB_TRY(cudaGetDevice(&dev));
  NB_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  const long long budget = static_cast<long long>(seconds * 1e3 * (khz > 0 ? khz : 2000000));
  NB_TRY(launch_wait_probe(c->d.status, budget, c->st));
  return NB_OK;
}

int nb_clear_status(nb_ctx* c) {
  if (!c) return NB_EINVAL;
  NB_TRY(cudaMemsetAsync(c->d.status, 0, 4, c->st));
  NB_TRY(cudaStreamSynchronize(c->st));
  return NB_OK;
}

const char* nb_strerror(int code) {
  switch (code) {
    case NB_OK: return "ok";
    case NB_EINVAL: return "invalid argument";
    case NB_ENOMEM: return "workspace too small";
    case NB_ECUDA: return "CUDA runtime error";
    case NB_ETIMEOUT: return "device wait timed out";
    case NB_ENONFINITE: return "non-finite value produced";
    case NB_ESTATE: return "invalid context state";
    default: return "unknown status";
  }
}

}  // extern "C"
