/*
 * nbody_gb300.h -- C ABI of libnbody_gb300.so: direct-summation N-body forces
 * with a 4th- or 6th-order Hermite block-time-step integrator on one NVIDIA
 * GB300 (sm_103a).
 *
 * The library computes, for a set of "active" particles, the softened
 * Newtonian acceleration, its time derivative (jerk) and the potential due to
 * all N sources of the same cluster (Eq. 1 with the softening of Eq. 2), and
 * drives it with the Hermite predictor-corrector (Sec. 2 item 1) on
 * power-of-two block time steps (Sec. 2 item 2).  Several independent
 * clusters may share one context (a batch); forces never cross clusters.
 * The i-split of Sec. 2 item 3 and the kernel shape follow a table per
 * ceil(log2 m) that nb_autotune measures; the force sum can be split over
 * processes (one GPU each) by pieces of the source order (nb_force_range,
 * nb_block_force / nb_block_correct), as the paper's multi-GPU runs split it
 * (Sec. 2.1).
 *
 * Conventions
 *   - Units: G is a parameter (default 1).  Softening eps >= 0; with eps == 0
 *     two distinct particles at the same position give non-finite values.
 *   - Particle i's acceleration sums j != i of its own cluster:
 *       a_i    =  G sum m_j d / s^3,           d = r_j - r_i, s^2 = |d|^2 + eps^2
 *       jerk_i =  G sum m_j (w / s^3 - 3 (d.w) d / s^5),    w = v_j - v_i
 *       pot_i  = -G sum m_j / s
 *   - Time is an integer number of ticks of 2^-tick_exp time units; a
 *     particle on level L has the step dt = 2^-L time units.
 *   - Host vectors are row-major (n, 3) doubles; device result vectors are
 *     row-major (m, 3) doubles.
 *
 * Precision (nb_config.precision)
 *   NB_FP64  : every operation in IEEE FP64.
 *   NB_MIXED : the pair arithmetic in FP32 with double-single (hi + lo FP32)
 *              positions so that the separation keeps FP64-like resolution
 *              (Sec. 2 item 4: DP for distances and accumulation, the rest,
 *              square roots included, in SP); sums over sources accumulated
 *              with a compensated FP32 pair per tile and combined in FP64;
 *              predictor, corrector, time, state and energy stay FP64.
 *   NB_DS    : as NB_MIXED with double-single separations for every source
 *              (no far-cell shortcut): the accuracy bound of the mixed path,
 *              at a lower speed.
 *   NB_FP32  : as NB_MIXED with plain FP32 separations for every source
 *              (the offsets' low words unused): the speed bound, whose
 *              separation error is relative to the cell size rather than to
 *              the separation, so close pairs lose accuracy.
 *   NB_DS and NB_FP32 use the default kernel shape (variant 0); nb_force
 *   without jerk uses the mixed separations in every non-FP64 mode.
 *
 * Memory ownership
 *   All device memory is the caller's: nb_workspace_size() gives the bytes of
 *   ONE device buffer that the caller allocates (e.g. a torch uint8 tensor)
 *   and passes to nb_init(); it must stay allocated until nb_free().  The
 *   library keeps a small host struct (nb_ctx), never allocates device memory
 *   itself, and keeps no host pointer after a call returns.
 *
 * Streams and synchronisation
 *   Every call runs on the stream given to nb_init() (NULL = legacy default
 *   stream).  nb_predict, nb_force, nb_correct and nb_step_block only enqueue
 *   work and return; nb_init, nb_energy, nb_get_state, nb_set_state,
 *   nb_stats and nb_status synchronise that stream.
 *
 * Errors
 *   Every int-returning call returns NB_OK or a positive NB_E* code and never
 *   aborts, exits or traps.  Argument errors are reported immediately.
 *   Errors found on the device (bad active list, non-finite results, a device
 *   wait that gave up) set a sticky status word in the workspace; the
 *   synchronising calls return it, and nb_status() reads it.
 *
 * Thread safety: a context is used by one host thread at a time.
 */
#ifndef NBODY_GB300_H
#define NBODY_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define NB_OK          0
#define NB_EINVAL      1   /* bad argument (NULL, size, range, order)        */
#define NB_ENOMEM      2   /* workspace smaller than nb_workspace_size()     */
#define NB_ECUDA       3   /* a CUDA runtime call failed                     */
#define NB_ETIMEOUT    4   /* a device-side wait gave up (bounded spin)      */
#define NB_ENONFINITE  5   /* NaN/Inf produced by the corrector              */
#define NB_ESTATE      6   /* call not valid in the context's current state  */

typedef struct nb_ctx nb_ctx;

typedef enum { NB_FP64 = 0, NB_MIXED = 1, NB_DS = 2, NB_FP32 = 3 } nb_precision;

typedef struct {
    double  G;          /* gravitational constant (Eq. 1)                      */
    double  eps;        /* softening length (Eq. 2), >= 0                      */
    double  eta;        /* accuracy parameter of the step criterion            */
    double  eta_start;  /* accuracy parameter of the initial step              */
    int32_t level_min;  /* largest step  = 2^-level_min, 0 <= level_min        */
    int32_t level_max;  /* smallest step = 2^-level_max, level_min <= level_max */
    int32_t tick_exp;   /* one tick = 2^-tick_exp time units, level_max <= tick_exp <= 60 */
    int32_t precision;  /* nb_precision                                        */
    int32_t bfactor;    /* i-split factor B: 0 = chosen per step by the plan   */
    int32_t graph_steps;/* block steps captured per CUDA graph (0 = no graph)  */
    int32_t sort_sources;/* 1: force sources kept in spatial (Hilbert) order of
                            the initial positions, 0: in particle order.  Only
                            speed depends on it, never the results' accuracy. */
    int32_t variant;    /* shape of the mixed force kernel, 0 .. NB_MIXED_VARIANTS-1
                           (see nb_autotune); all give results of the same
                           accuracy */
    int32_t order;      /* order of the Hermite scheme: 4 (default) or 6 (the
                           order of the paper's template code, Sec. 2 item 1):
                           the force then also yields the snap, the state also
                           holds snap and crackle, and nb_step_block predicts,
                           corrects and picks steps with the 6th-order rules */
} nb_config;

/* Defaults: G = 1, eps = 1e-4, eta = 0.01, eta_start = 0.01, level_min = 0,
 * level_max = 30, tick_exp = 40, NB_MIXED, bfactor = 0, graph_steps = 16,
 * sort_sources = 1, variant = 0, order = 4. */
void nb_default_config(nb_config *cfg);

/* Bytes of the device workspace for n_total particles in n_clusters clusters
 * (n_clusters >= 1; every cluster holds >= 1 particle).  NB_EINVAL on bad
 * sizes or config. */
int nb_workspace_size(int64_t n_total, int32_t n_clusters, const nb_config *cfg,
                      size_t *bytes);

/* Create a context.  offsets (host, n_clusters + 1, offsets[0] = 0, strictly
 * increasing, offsets[n_clusters] = n_total) delimit the clusters; mass (n),
 * pos and vel (n x 3) are host arrays copied during the call.  workspace is a
 * device pointer (256-byte aligned) of at least nb_workspace_size() bytes.
 * stream is a cudaStream_t (or NULL).  Computes the acceleration and jerk of
 * every particle at t = 0 (one force evaluation), sets every time to 0 and
 * assigns the first levels from eta_start |a| / |jerk| (clamped to
 * [level_min, level_max]).  Synchronises the stream. */
int nb_init(nb_ctx **out, const nb_config *cfg, int32_t n_clusters,
            const int64_t *offsets, const double *mass, const double *pos,
            const double *vel, void *workspace, size_t workspace_bytes,
            void *stream);

/* Release the host context (the workspace stays the caller's). */
void nb_free(nb_ctx *ctx);

/* Predict EVERY particle to time t_ticks with the Taylor predictor of the
 * Hermite scheme (Sec. 2 items 1 and 2) and store the result as the source
 * set used by nb_force.  Asynchronous. */
int nb_predict(nb_ctx *ctx, int64_t t_ticks);

/* Acceleration, jerk and potential (Eq. 1, Eq. 2) of the m particles listed in
 * active_idx (device int32, m entries, global particle indices in any order,
 * no repeats) from the predicted sources of their own cluster (the last
 * nb_predict).  acc: device (m x 3) doubles; jerk: device (m x 3) doubles or
 * NULL; pot: device m doubles or NULL.  With jerk == NULL only the
 * acceleration (and the potential) is wanted: a mixed-precision context
 * then runs a kernel without the velocity terms (about half the arithmetic
 * per interaction, for acceleration-only integrators such as leapfrog); an
 * FP64 context computes the jerk and drops it.  Row k of the outputs belongs
 * to active_idx[k].  The targets are evaluated in the library's spatial
 * source order and written back to their rows.  m == 0 is a no-op.
 * Asynchronous; an out-of-range or repeated entry sets the sticky status to
 * NB_EINVAL and the rows of the offending entries are left unwritten. */
int nb_force(nb_ctx *ctx, const int32_t *active_idx, int64_t m, double *acc,
             double *jerk, double *pot);

/* Acceleration, jerk, snap and potential for the 6th-order Hermite scheme
 * (the order of the paper's template code, Sec. 2 item 1): as nb_force, plus
 * the snap, the second time derivative of the softened pair term of Eq. 2,
 *   snap_i = G sum_j m_j (u - 6 alpha (w - 3 alpha d) - 3 beta d) / s^3,
 *   u = a_j - a_i, alpha = d.w / s^2, beta = (w.w + d.u) / s^2 + alpha^2,
 * with the predicted accelerations a of the last nb_predict.  snap: device
 * (m x 3) doubles; jerk required; pot may be NULL.  Order-6 contexts only
 * (NB_ESTATE otherwise).  Asynchronous. */
int nb_force_snap(nb_ctx *ctx, const int32_t *active_idx, int64_t m, double *acc,
                  double *jerk, double *snap, double *pot);

/* ---- j-partition of the force sum (Sec. 2.1: the template code spreads
 * its force work over many GPUs, MPI between the processes).  The force on a
 * target is a sum over sources (Eq. 1), so P processes that each hold the
 * whole particle set can each sum over one piece of the sources and add the
 * partial results (an all-reduce); each then corrects the same particles
 * from the same sums, and the replicated states stay identical. */

/* Slot range [*slot_begin, *slot_end) of piece `part` (0 <= part < n_parts)
 * of a cluster with n_slots source slots: contiguous pieces of
 * ceil(n_slots / n_parts) slots rounded up to NB_PIECE_ALIGN, so every piece
 * starts on a tile of the force kernels; together they cover [0, n_slots)
 * once, and the last ones may be empty.  Host arithmetic only (no context,
 * no device).  NB_EINVAL for a bad argument. */
int nb_source_piece(int64_t n_slots, int32_t part, int32_t n_parts, int64_t *slot_begin,
                    int64_t *slot_end);
#define NB_PIECE_ALIGN 128

/* The context's source order: *n_slots, the number of source slots (each
 * cluster's particles padded to a multiple of 4 slots, in the spatial order
 * nb_init or nb_resort_sources chose); particle_of_slot (host, n_slots
 * entries, or NULL): the particle held by each slot, -1 for a padding slot;
 * slot_offsets (host, n_clusters + 1 entries, or NULL): each cluster's first
 * slot.  A piece of cluster k (nb_source_piece over its slot count) covers
 * the slots slot_offsets[k] + [begin, end).  Host data only; does not
 * synchronise. */
int nb_source_order(nb_ctx *ctx, int64_t *n_slots, int32_t *particle_of_slot,
                    int64_t *slot_offsets);

/* nb_force restricted to the sources in piece `part` of `n_parts` of every
 * cluster's source order (nb_source_piece): the partial acceleration, jerk
 * and potential, whose sum over part = 0 .. n_parts-1 is nb_force's result
 * up to rounding.  n_parts == 1 is nb_force itself.  The targets, outputs,
 * asynchrony and errors are nb_force's; NB_EINVAL for a bad part. */
int nb_force_range(nb_ctx *ctx, const int32_t *active_idx, int64_t m, int32_t part,
                   int32_t n_parts, double *acc, double *jerk, double *pot);

/* One block step (nb_step_block, Sec. 2 item 2) split around the sum of its
 * force over processes.  nb_block_force takes the next block time, predicts,
 * lists the active set and evaluates its force from piece `part` of
 * `n_parts` of the sources, then waits and reports *m_out, the number of
 * active particles, and the device addresses of the step's force rows:
 * *acc_rows, *jerk_rows and, in an order-6 context, *snap_rows (NULL in
 * order 4), each m rows of 4 doubles (x, y, z, and one unused double), row k
 * for the k-th particle of the step's active list.  These rows belong to the
 * context's workspace; the caller may add the other processes' partial rows
 * into them in place (an all-reduce over the first 4 m doubles of each), on
 * the context's stream or after it.  nb_block_correct then applies the
 * corrector of Sec. 2 item 1 (nb_correct, or nb_correct_snap in order 6) to
 * those rows and closes the step.  While a step is open, every call that
 * does device work other than nb_block_correct (nb_predict, nb_force and its
 * variants, nb_correct, the step calls, energies, state and derivative
 * copies, nb_autotune, nb_resort_sources, the probes) returns NB_ESTATE:
 * the open step's active list and force rows must stay as they are.
 * nb_block_correct with no step open is NB_ESTATE as well.  Output pointers
 * other than m_out may be NULL. */
int nb_block_force(nb_ctx *ctx, int32_t part, int32_t n_parts, int64_t *m_out,
                   double **acc_rows, double **jerk_rows, double **snap_rows);
int nb_block_correct(nb_ctx *ctx);

/* Re-sort every cluster's source slots along the Hilbert curve of the
 * particles' current positions.  nb_init orders the slots by the initial
 * positions; as the particles move, the cells of consecutive slots spread
 * out and more (target warp, cell) pairs take the mixed kernel's near path
 * (the double-single separations of Sec. 2 item 4), which is slower.  The
 * sources are then predicted to each cluster's current block time (call
 * nb_predict again before nb_force at another time).  Later force results
 * change by rounding only (the summation follows the slot order).
 * Synchronises; NB_ESTATE while a split block step is open. */
int nb_resort_sources(nb_ctx *ctx);

/* Hermite correction (Sec. 2 item 1) of the m particles in active_idx
 * (device, as for nb_force) from their own times to t_ticks, given their new
 * acceleration and jerk evaluated at the predicted state (device m x 3, as
 * written by nb_force).  Sets each particle's time to t_ticks and a new level
 * from the step criterion.  Asynchronous. */
int nb_correct(nb_ctx *ctx, int64_t t_ticks, const int32_t *active_idx,
               int64_t m, const double *acc, const double *jerk);

/* 6th-order Hermite correction of the m particles in active_idx from their
 * own times to t_ticks, given the force with snap at the predicted state
 * (device m x 3 each, as written by nb_force_snap): over the step t,
 *   v1 = v0 + t/2 (a0 + a1) - t^2/10 (j1 - j0) + t^3/120 (s0 + s1),
 *   x1 = x0 + t/2 (v0 + v1) - t^2/10 (a1 - a0) + t^3/120 (j0 + j1)
 * (the quintic through both ends' a, j, s); keeps the quintic's crackle for
 * the next prediction and sets a new level from dt = eta (A1 / A4)^(1/3),
 * A_k = sqrt(|a^(k-1)| |a^(k+1)|) + |a^(k)| over a, j, s, crackle, pop,
 * a^(5) at the end of the step.  Order-6 contexts only (nb_correct serves
 * order 4 and returns NB_ESTATE here).  Asynchronous. */
int nb_correct_snap(nb_ctx *ctx, int64_t t_ticks, const int32_t *active_idx,
                    int64_t m, const double *acc, const double *jerk,
                    const double *snap);

/* Run n_steps block steps (Sec. 2 item 2).  In one block step EVERY cluster
 * whose time is below the end time (nb_set_end_time) independently takes its
 * next block time t_next = min_i (t_i + dt_i), predicts all its particles to
 * t_next, evaluates the force on its active set {i : t_i + dt_i = t_next}
 * and corrects that set.  All sizes live on the device, so the sequence is
 * launched without host synchronisation (CUDA graphs of graph_steps steps).
 * Asynchronous when both outputs are NULL.  Otherwise the call waits for the
 * steps and reports (host outputs): t_ticks_out, the smallest cluster block
 * time after the last step (the common time of a single cluster);
 * m_last_out, the number of particles corrected in the last step, summed over
 * the clusters that stepped (0 when n_steps == 0 or every cluster had
 * reached its end time). */
int nb_step_block(nb_ctx *ctx, int64_t n_steps, int64_t *t_ticks_out,
                  int64_t *m_last_out);

/* Clusters stop stepping once their time reaches t_end_ticks (a multiple of
 * 2^-level_min time units keeps every particle synchronised there).
 * Default: no end time. */
int nb_set_end_time(nb_ctx *ctx, int64_t t_end_ticks);

/* Kick-drift-kick leapfrog with one shared step of dt_ticks ticks (> 0,
 * at most 2^52), n_steps times, on every particle: v += a dt/2; x += v dt;
 * a = the acceleration at the new positions (Eq. 1, Eq. 2; in a mixed
 * context the acceleration-only kernel of nb_force without jerk); v += a dt/2;
 * each particle's time advances by dt.  The acceleration-only workload of
 * the same force sum, next to the Hermite block steps.  It starts from the
 * stored acceleration, takes the sources at their stored positions (so every
 * particle of a cluster should share one time, as after nb_init or an
 * nb_set_state with equal times), leaves the stored jerk and potential as
 * they were, and is not meant to be interleaved with nb_step_block.
 * Asynchronous. */
int nb_step_leapfrog(nb_ctx *ctx, int64_t n_steps, int64_t dt_ticks);

/* FP64 kinetic and softened potential energy of cluster `cluster` (-1: all
 * clusters summed), with every particle predicted to its cluster's current
 * block time: E_kin = 1/2 sum_i m_i |v_i|^2 and E_pot = 1/2 sum_i m_i pot_i,
 * pot_i = -G sum_{j != i} m_j / (|r_ij|^2 + eps^2)^(1/2), the potential whose
 * gradient is the softened force of Eq. 2 (Sec. 1: the softening enters the
 * gravitational potential).  Host outputs; synchronises. */
int nb_energy(nb_ctx *ctx, int32_t cluster, double *ekin, double *epot);

/* The same energies (as nb_energy, the softened potential of Eq. 2) for
 * every cluster from ONE potential evaluation of the whole context: ekin[k],
 * epot[k] for k < n_clusters (host arrays).  Synchronises. */
int nb_energies(nb_ctx *ctx, double *ekin, double *epot);

/* Copy the state to host arrays (any pointer may be NULL): pos, vel, acc,
 * jerk (n x 3), t (n ticks), level (n) -- the particle state of Eq. 1
 * (positions, velocities, masses) plus the Hermite scheme's derivatives and
 * the block-step bookkeeping of Sec. 2 items 1 and 2.  The vectors are packed
 * on the device and copied straight into the caller's arrays (pinned arrays
 * copy at full host-link bandwidth).  Synchronises. */
int nb_get_state(nb_ctx *ctx, double *pos, double *vel, double *acc,
                 double *jerk, int64_t *t, int32_t *level);

/* Overwrite the state (as nb_get_state describes it, Eq. 1 and Sec. 2
 * items 1 and 2) from host arrays (all six required; masses keep their
 * nb_init values).  Levels must lie in [level_min, level_max] and each time
 * must be a multiple of its step (Sec. 2 item 2: power-of-two steps).
 * Synchronises. */
int nb_set_state(nb_ctx *ctx, const double *pos, const double *vel,
                 const double *acc, const double *jerk, const int64_t *t,
                 const int32_t *level);

/* The 6th-order scheme's extra state (order-6 contexts; NB_ESTATE
 * otherwise): snap and crackle (n x 3 host arrays; get: either may be NULL,
 * set: both required and finite).  nb_init starts from the snap of the t = 0
 * force and a zero crackle.  Synchronise. */
int nb_get_derivs(nb_ctx *ctx, double *snap, double *crackle);
int nb_set_derivs(nb_ctx *ctx, const double *snap, const double *crackle);

/* Counters since nb_init (host outputs, any may be NULL): block steps taken,
 * pair interactions evaluated (sum over force evaluations of m x N_cluster),
 * smallest and largest cluster time in ticks.  Synchronises. */
int nb_stats(nb_ctx *ctx, int64_t *block_steps, int64_t *interactions,
             int64_t *t_min, int64_t *t_max);

/* Force-kernel timing.  While enabled, CUDA events bracket every launch of
 * the force kernel on the context's stream (block steps are then launched
 * directly instead of through CUDA graphs).  nb_profile_read synchronises and
 * returns the summed device milliseconds of those launches and their count
 * since the previous read (either pointer may be NULL). */
int nb_profile_enable(nb_ctx *ctx, int enable);
int nb_profile_read(nb_ctx *ctx, double *force_ms, int64_t *launches);

/* The same timing for every kind of launch of a block step (and of
 * nb_force): host arrays of NB_PROFILE_KINDS entries (either may be NULL),
 * in this order: next block time, predictor, active list and plan (scan,
 * plan and scatter, or the plan alone), force kernel, i-split reduction,
 * corrector.  Summed device milliseconds and launch counts since the
 * previous nb_profile_kernels (a count apart from nb_profile_read's).  The
 * sum over kinds leaves out the gaps between launches.  Synchronises. */
#define NB_PROFILE_KINDS 6
int nb_profile_kernels(nb_ctx *ctx, double *ms_by_kind, int64_t *launches_by_kind);

/* Mixed force kernel diagnostics since nb_init (host outputs, either may be
 * NULL): source cells (64 slots each) processed by a warp, and how many of
 * those took the near (full double-single) path because some target of the
 * warp lay within 2 cell radii of the cell centre.  The near share measures
 * how well the spatial source order fits the targets; it affects speed only.
 * The counts accumulate over every mixed launch of the context (nb_init's
 * own force evaluation included); take differences to cover a span.
 * Synchronises. */
int nb_tile_stats(nb_ctx *ctx, int64_t *warp_tiles, int64_t *near_warp_tiles);

/* Autotuner: the shape of the mixed force kernel (nb_config.variant) and the
 * i-split factor B (Sec. 2 item 3: the best Bfactor depends on the number of
 * active particles and has to be chosen step by step), per ceil(log2 m) of
 * the active count m -- a table of NB_TUNE_BUCKETS (variant, B) entries, B 0
 * for the plan's own choice.  Measured on this context's own sources at
 * m = every 4^k-th source slot (k = 0 .. NB_TUNE_POINTS-1, while m >= 64):
 * every shape with the plan's B, then the fastest shape with B = 1, 2, 4, ...
 * (the smallest B within 0.3 % of the fastest time is kept: fewer partial
 * sums to write and reduce for the same speed).
 * Buckets between two measured points take the nearer point's shape, and its
 * B scaled by the ratio of the active counts (the same fill of the grid).
 * nb_force then takes the entry of its m, and the plan of every block step
 * the entry of the step's active count (on the device: a block step launches
 * every shape the table holds, and each one exits at once unless the plan
 * chose it).  cache_path (may be NULL): a text file of tables, one line per
 * problem class (GPU name, SM count, precision, Hermite order, ceil(log2 N),
 * cluster count); a table found there is applied without measuring, and a
 * measured one is appended.  variant_out (host, may be NULL): the shape of
 * the largest bucket (also the context's nb_config.variant from now on);
 * ms_out (host, may be NULL): NB_TUNE_POINTS x NB_MIXED_VARIANTS doubles,
 * the time of each shape at each point with the plan's B (0: not measured).
 * Uses the workspace's active-list buffers (call it between steps).  Mixed
 * precision only (other precisions have one shape and return it).
 * Synchronises; NB_EINVAL when a measured table cannot be appended to
 * cache_path (the table is applied all the same). */
#define NB_TUNE_POINTS 8
#define NB_TUNE_BUCKETS 32
#define NB_MIXED_VARIANTS 8
int nb_autotune(nb_ctx *ctx, const char *cache_path, int32_t *variant_out, double *ms_out);

/* The context's autotune table (host arrays of NB_TUNE_BUCKETS entries,
 * either may be NULL): the shape and B (0: the plan's choice) used for
 * active counts m with ceil(log2 m) = bucket.  Before nb_autotune every
 * entry is (nb_config.variant, nb_config.bfactor). */
int nb_tune_table(nb_ctx *ctx, int32_t *variant_by_bucket, int32_t *bfactor_by_bucket);

/* Arithmetic-rate probe for the roofline of the force kernels (the paper has
 * no counterpart): runs independent FMA chains in 4 CTAs of 256 threads per
 * SM and returns the FMA lanes per SM per SM-clock cycle (lanes_per_sm_clock,
 * host; the median over SMs, counted with the SM cycle counter, so it does
 * not depend on the clock the GPU ran at).  kind 0: packed f32x2 FMA (two
 * lanes per instruction, the mixed kernel's arithmetic), 1: FP32 FMA, 2: FP64
 * FMA.  Nominal: 128 FP32 lanes per SM per clock.  Uses the workspace's
 * partial-sum buffer as scratch (call it between force evaluations).
 * Synchronises. */
int nb_measure_rate(nb_ctx *ctx, int32_t kind, double *lanes_per_sm_clock);

/* Sticky device status (NB_OK or an NB_E* code); synchronises. */
int nb_status(nb_ctx *ctx);

/* Clear the sticky device status. */
int nb_clear_status(nb_ctx *ctx);

/* Self-check of the failure detection: launch one kernel whose device wait
 * (an mbarrier phase that nothing completes) runs out after `seconds`
 * (0 < seconds <= 10) of SM clock, exactly as a force kernel's wait for a
 * source tile would; the sticky status becomes NB_ETIMEOUT (nb_status reads
 * it, nb_clear_status clears it) and the context stays usable.  Nothing
 * faults, traps or hangs.  Asynchronous. */
int nb_check_wait_timeout(nb_ctx *ctx, double seconds);

/* Text for a status code (static storage). */
const char *nb_strerror(int code);

/* ---- Forces without a workspace ------------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory where they need forces (code running in a
 * host callback or library hook while another framework owns all device
 * allocations, or runtimes that forbid cudaMalloc after start-up) and so
 * cannot provide the workspace nb_init() needs.  It computes the same
 * quantities as nb_force() for one cluster, directly from device arrays:
 * pos, vel (n x 3), mass (n), target_idx (m int32 in [0, n), any order),
 * outputs acc, jerk (m x 3) and pot (m, or NULL), on `stream`.
 * precision is NB_MIXED or NB_FP64.  Asynchronous; a target index outside
 * [0, n) leaves its row unspecified and sets the status that
 * nb_noalloc_status() reports, as does a device wait that gave up (its rows
 * are then unspecified too).
 *
 * It allocates nothing: the packed sources, the i-split partial sums and the
 * plan words live in one fixed device array of 6,705,664 bytes compiled into
 * the library, present on every GPU that loads the library until the process
 * exits.  Limits: 1 <= n <= NB_NOALLOC_MAX_SOURCES (larger n returns
 * NB_EINVAL without launching anything), 0 <= m <= n.  All calls on a device
 * share that array and each call leaves its contents behind; a call rewrites
 * everything it reads first, but calls whose work overlaps on the GPU (other
 * streams without ordering, other host threads) race on it.  The first call
 * on each device looks up the array's device address with that device
 * current; make that first call before any stream capture on the device. */
#define NB_NOALLOC_MAX_SOURCES 32768
int nb_force_noalloc(const double *pos, const double *vel, const double *mass,
                     int64_t n, const int32_t *target_idx, int64_t m, double G,
                     double eps, int32_t precision, double *acc, double *jerk,
                     double *pot, void *stream);

/* Device status of the last nb_force_noalloc call enqueued on `stream` on the
 * current device: NB_OK, NB_EINVAL (a target index outside [0, n)),
 * NB_ETIMEOUT (a device wait gave up) or NB_ECUDA.  Every call starts from a
 * cleared status, so the answer covers that one call, provided no call on
 * another stream of the device ran in between (calls share the fixed array).
 * Copies one word from the fixed array and synchronises `stream`; allocates
 * nothing. */
int nb_noalloc_status(void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NBODY_GB300_H */
