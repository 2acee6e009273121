/*
 * nbody_oracle.c -- plain, slow, FP64 CPU oracle for the direct-summation
 * N-body method (softened Newtonian forces + 4th-order Hermite integrator
 * with power-of-two block time steps).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * GPU library is checked against.  Only the test suite, the package's smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, constant or helper with the GPU library, and the GPU library
 * never calls it.
 *
 * Every function restates the paper's definition in the most direct form:
 *   - Eq. 1: the Newtonian equations of motion, the sum running over j != i,
 *     with r_ij the separation of i and j;
 *   - Eq. 2: the softened pair force, -G m_i m_j r_ij / (r_ij^2 + eps^2)^(3/2);
 *     acceleration drops m_i and sums the pair terms over j != i;
 *   - Sec. 2, item 1: Hermite integrator -- Taylor predictor of position and
 *     velocity, ONE force (acceleration + jerk) evaluation per step,
 *     corrector from the Hermite interpolation of the acceleration;
 *   - Sec. 2, item 2: block time steps -- each particle has its own step,
 *     forced to a power of two; only the m <= N particles due at the next
 *     block time are corrected, all others are only predicted (Taylor).
 * The paper gives no formula for the jerk, the potential, the corrector, the
 * time-step criterion or the level rules; the readings used are stated at
 * each function (they follow the standard Hermite literature the paper cites
 * for its integrator, Aarseth 2003).
 *
 * Precision: IEEE FP64 throughout, round-to-nearest; sums over sources use
 * Neumaier's compensated summation so the oracle's own summation error is
 * far below the 1e-12 parity bar.  Build WITHOUT -ffast-math and WITH
 * -ffp-contract=off so the results do not depend on FMA contraction (the
 * oracle is built on x86-64 and on aarch64 hosts).
 *
 * Threads: OpenMP over target particles; each target's sum runs over j in
 * ascending order, so the result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Neumaier compensated summation (improved Kahan).                     */
/* ------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_get(const nsum *a) { return a->s + a->c; }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* Force: Eq. 1 with the softening of Eq. 2.                            */
/*                                                                      */
/* For each requested target i (index idx[k]) and every source j != i:  */
/*   d  = r_j - r_i            (so -r_ij, r_ij = r_i - r_j of Eq. 1)    */
/*   w  = v_j - v_i                                                     */
/*   s  = sqrt(|d|^2 + eps^2)                                           */
/*   acc_i  += G m_j d / s^3                        (Eq. 1, Eq. 2)      */
/*   jerk_i += G m_j ( w / s^3 - 3 (d.w) d / s^5 )  (time derivative    */
/*                    of the softened acceleration; Sec. 2 item 1 needs */
/*                    it, the paper does not print it)                  */
/*   pot_i  -= G m_j / s        (softened potential whose gradient      */
/*                               gives Eq. 2)                           */
/* The excluded term is j == i by index (Eq. 1's j != i).               */
/* pos, vel: n x 3 row-major; mass: n; idx: m target indices in [0,n);  */
/* acc, jerk: m x 3; pot: m (any of the three may be NULL).             */
/* Returns 0, or -1 on a bad index.                                     */
/* ------------------------------------------------------------------ */
int oracle_force(int64_t n, const double *pos, const double *vel,
                 const double *mass, double G, double eps, int64_t m,
                 const int64_t *idx, double *acc, double *jerk, double *pot)
{
    for (int64_t k = 0; k < m; k++)
        if (idx[k] < 0 || idx[k] >= n) return -1;
    const double eps2 = eps * eps;
    int64_t k;
#pragma omp parallel for schedule(dynamic, 16)
    for (k = 0; k < m; k++) {
        const int64_t i = idx[k];
        nsum a[3], jk[3], p;
        memset(a, 0, sizeof a);
        memset(jk, 0, sizeof jk);
        memset(&p, 0, sizeof p);
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3], w[3];
            for (int c = 0; c < 3; c++) {
                d[c] = pos[3 * j + c] - pos[3 * i + c];
                w[c] = vel[3 * j + c] - vel[3 * i + c];
            }
            double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
            double s = sqrt(s2);
            double s3 = s2 * s;
            double s5 = s3 * s2;
            double dw = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
            double gm = G * mass[j];
            for (int c = 0; c < 3; c++) {
                nsum_add(&a[c], gm * d[c] / s3);
                nsum_add(&jk[c], gm * (w[c] / s3 - 3.0 * dw * d[c] / s5));
            }
            nsum_add(&p, -gm / s);
        }
        for (int c = 0; c < 3; c++) {
            if (acc) acc[3 * k + c] = nsum_get(&a[c]);
            if (jerk) jerk[3 * k + c] = nsum_get(&jk[c]);
        }
        if (pot) pot[k] = nsum_get(&p);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Energy: kinetic 1/2 sum m v^2 and softened potential energy          */
/* -G sum_{i<j} m_i m_j / sqrt(r_ij^2 + eps^2) (the pair energy whose   */
/* gradient is Eq. 2).  Both Neumaier-summed; per-i partial sums are    */
/* combined in ascending i, so the result is thread-count independent.  */
/* ------------------------------------------------------------------ */
void oracle_energy(int64_t n, const double *pos, const double *vel,
                   const double *mass, double G, double eps,
                   double *ekin, double *epot)
{
    const double eps2 = eps * eps;
    double *row = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < n; i++) {
        nsum p;
        memset(&p, 0, sizeof p);
        for (int64_t j = i + 1; j < n; j++) {
            double dx = pos[3 * j] - pos[3 * i];
            double dy = pos[3 * j + 1] - pos[3 * i + 1];
            double dz = pos[3 * j + 2] - pos[3 * i + 2];
            double s = sqrt(dx * dx + dy * dy + dz * dz + eps2);
            nsum_add(&p, -G * mass[i] * mass[j] / s);
        }
        row[i] = nsum_get(&p);
    }
    nsum k, p;
    memset(&k, 0, sizeof k);
    memset(&p, 0, sizeof p);
    for (i = 0; i < n; i++) {
        double v2 = vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] +
                    vel[3 * i + 2] * vel[3 * i + 2];
        nsum_add(&k, 0.5 * mass[i] * v2);
        nsum_add(&p, row[i]);
    }
    free(row);
    *ekin = nsum_get(&k);
    *epot = nsum_get(&p);
}

/* Total angular momentum L = sum m r x v and linear momentum P = sum m v. */
void oracle_momenta(int64_t n, const double *pos, const double *vel,
                    const double *mass, double *L, double *P)
{
    nsum l[3], p[3];
    memset(l, 0, sizeof l);
    memset(p, 0, sizeof p);
    for (int64_t i = 0; i < n; i++) {
        const double *r = pos + 3 * i, *v = vel + 3 * i;
        nsum_add(&l[0], mass[i] * (r[1] * v[2] - r[2] * v[1]));
        nsum_add(&l[1], mass[i] * (r[2] * v[0] - r[0] * v[2]));
        nsum_add(&l[2], mass[i] * (r[0] * v[1] - r[1] * v[0]));
        for (int c = 0; c < 3; c++) nsum_add(&p[c], mass[i] * v[c]);
    }
    for (int c = 0; c < 3; c++) {
        L[c] = nsum_get(&l[c]);
        P[c] = nsum_get(&p[c]);
    }
}

/* ------------------------------------------------------------------ */
/* Hermite predictor (Sec. 2 item 1: Taylor series of position and      */
/* velocity, truncated after the jerk term):                            */
/*   x_p = x + v tau + a tau^2/2 + j tau^3/6                            */
/*   v_p = v + a tau + j tau^2/2                                        */
/* tau[i] is the time from particle i's own time to the target time.    */
/* ------------------------------------------------------------------ */
void oracle_predict(int64_t n, const double *pos, const double *vel,
                    const double *acc, const double *jerk, const double *tau,
                    double *xp, double *vp)
{
    for (int64_t i = 0; i < n; i++) {
        double t = tau[i];
        for (int c = 0; c < 3; c++) {
            int64_t q = 3 * i + c;
            xp[q] = pos[q] + vel[q] * t + acc[q] * t * t / 2.0 +
                    jerk[q] * t * t * t / 6.0;
            vp[q] = vel[q] + acc[q] * t + jerk[q] * t * t / 2.0;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Hermite corrector (Sec. 2 item 1).  Given a0, j0 at the start of the */
/* step and a1, j1 evaluated once at the predicted state, the cubic     */
/* a(t) = a0 + j0 t + a2 t^2/2 + a3 t^3/6 that matches a and its time   */
/* derivative at both ends has                                          */
/*   a2 tau^2 = -6 (a0 - a1) - tau (4 j0 + 2 j1)                        */
/*   a3 tau^3 = 12 (a0 - a1) + 6 tau (j0 + j1)                          */
/* and the corrected state adds the next two Taylor terms:              */
/*   x1 = x_p + a2 tau^4/24 + a3 tau^5/120                              */
/*   v1 = v_p + a2 tau^3/6  + a3 tau^4/24                               */
/* Also returns the second and third derivatives of a at the END of the */
/* step (a2 + a3 tau and a3) for the time-step criterion.               */
/* All arrays are m x 3 for the m corrected particles.                  */
/* ------------------------------------------------------------------ */
void oracle_correct(int64_t m, const double *tau, const double *xp,
                    const double *vp, const double *a0, const double *j0,
                    const double *a1, const double *j1, double *x1, double *v1,
                    double *a2_end, double *a3_end)
{
    for (int64_t k = 0; k < m; k++) {
        double t = tau[k];
        double t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t;
        for (int c = 0; c < 3; c++) {
            int64_t q = 3 * k + c;
            double da = a0[q] - a1[q];
            double a2 = (-6.0 * da - t * (4.0 * j0[q] + 2.0 * j1[q])) / t2;
            double a3 = (12.0 * da + 6.0 * t * (j0[q] + j1[q])) / t3;
            x1[q] = xp[q] + a2 * t4 / 24.0 + a3 * t5 / 120.0;
            v1[q] = vp[q] + a2 * t3 / 6.0 + a3 * t4 / 24.0;
            if (a2_end) a2_end[q] = a2 + a3 * t;
            if (a3_end) a3_end[q] = a3;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Time-step criterion.  The paper gives each particle its own step as  */
/* a function of its kinematic state and refers to Aarseth 2003 for the */
/* rule (Sec. 2 item 2).  Reading: Aarseth's standard criterion         */
/*   dt = sqrt( eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2) )            */
/* with a, j the new acceleration and jerk and a2, a3 their second and  */
/* third derivatives at the end of the step.  A zero denominator gives  */
/* +inf (the level clamp then takes the largest allowed step).          */
/* ------------------------------------------------------------------ */
static double norm3(const double *x)
{
    return sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
}

double oracle_aarseth_dt(const double *a, const double *j, const double *a2,
                         const double *a3, double eta)
{
    double na = norm3(a), nj = norm3(j), n2 = norm3(a2), n3 = norm3(a3);
    double num = na * n2 + nj * nj;
    double den = nj * n3 + n2 * n2;
    if (!(den > 0.0)) return INFINITY;
    return sqrt(eta * num / den);
}

/* Initial step (reading; the paper is silent): dt = eta_s |a| / |j|.   */
double oracle_initial_dt(const double *a, const double *j, double eta_s)
{
    double na = norm3(a), nj = norm3(j);
    if (!(nj > 0.0)) return INFINITY;
    return eta_s * na / nj;
}

/* ------------------------------------------------------------------ */
/* Power-of-two level (Sec. 2 item 2: "the time step is forced to be a  */
/* power of two").  A level L means dt = 2^-L.  Reading of the rules:   */
/*   L_want = smallest L with 2^-L <= dt_crit  (largest power of two    */
/*            not above dt_crit; exact via frexp), clamped to           */
/*            [lmin, lmax] (lmin = largest step, lmax = smallest);      */
/*   shrinking (L_want > L_old) is always allowed;                      */
/*   growing is limited to one doubling (L_old - 1) and allowed only if */
/*   the particle's new time is a multiple of the doubled step, so the  */
/*   block hierarchy stays synchronised; otherwise L_old is kept.       */
/* L_old < 0 marks the initial assignment (no growth limit).            */
/* Times are integer ticks of 2^-tick_exp.                              */
/* ------------------------------------------------------------------ */
int oracle_level(double dt_crit, int L_old, int64_t t_new_ticks, int tick_exp,
                 int lmin, int lmax)
{
    int L;
    if (!(dt_crit > 0.0)) {
        L = lmax;                   /* zero or NaN: smallest step */
    } else if (isinf(dt_crit)) {
        L = lmin;
    } else {
        int e;
        (void)frexp(dt_crit, &e);   /* dt_crit = f 2^e, f in [0.5,1) */
        L = 1 - e;                  /* 2^(e-1) <= dt_crit < 2^e      */
    }
    if (L < lmin) L = lmin;
    if (L > lmax) L = lmax;
    if (L_old < 0) return L;
    if (L >= L_old) return L;
    /* wants a larger step: at most one doubling, and only when the new */
    /* time is commensurate with the doubled step                        */
    int Ld = L_old - 1;
    if (Ld < lmin) return L_old;
    int64_t step2 = (int64_t)1 << (tick_exp - Ld);
    if (t_new_ticks % step2 == 0) return Ld;
    return L_old;
}

/* ------------------------------------------------------------------ */
/* One block time step (Sec. 2 items 1 and 2), all state in FP64:       */
/*  1. t_next = min_i (t_i + dt_i)                                      */
/*  2. active set = { i : t_i + dt_i == t_next }, ascending index       */
/*  3. predict EVERY particle to t_next (Taylor; Sec. 2 item 2 says the */
/*     non-updated particles are only estimated by Taylor expansion)    */
/*  4. one force evaluation for the active particles from the predicted */
/*     positions and velocities of all N sources (Eq. 1, Eq. 2)         */
/*  5. Hermite correction of the active particles                       */
/*  6. new power-of-two step from the criterion, new t_i = t_next       */
/* State (updated in place): pos, vel, acc, jerk (n x 3), t (ticks),    */
/* level.  Optional outputs: active index list (n), the m value, the    */
/* raw criterion dt_crit per active particle (n).                       */
/* Returns 0, or -1 on an invalid level.                                */
/* ------------------------------------------------------------------ */
int oracle_block_step(int64_t n, double *pos, double *vel, double *acc,
                      double *jerk, const double *mass, int64_t *t,
                      int32_t *level, double G, double eps, double eta,
                      int tick_exp, int lmin, int lmax, int64_t *t_next_out,
                      int64_t *m_out, int64_t *active_out, double *dtcrit_out)
{
    if (n <= 0) return -1;
    int64_t t_next = INT64_MAX;
    for (int64_t i = 0; i < n; i++) {
        if (level[i] < 0 || level[i] > tick_exp) return -1;
        int64_t due = t[i] + ((int64_t)1 << (tick_exp - level[i]));
        if (due < t_next) t_next = due;
    }
    int64_t *act = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (t[i] + ((int64_t)1 << (tick_exp - level[i])) == t_next)
            act[m++] = i;

    double *tau = (double *)malloc((size_t)n * sizeof(double));
    double *xp = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *vp = (double *)malloc((size_t)n * 3 * sizeof(double));
    for (int64_t i = 0; i < n; i++)
        tau[i] = ldexp((double)(t_next - t[i]), -tick_exp);
    oracle_predict(n, pos, vel, acc, jerk, tau, xp, vp);

    double *a1 = (double *)malloc((size_t)m * 3 * sizeof(double));
    double *j1 = (double *)malloc((size_t)m * 3 * sizeof(double));
    oracle_force(n, xp, vp, mass, G, eps, m, act, a1, j1, NULL);

    double *tk = (double *)malloc((size_t)m * sizeof(double));
    double *xa = (double *)malloc((size_t)m * 3 * sizeof(double));
    double *va = (double *)malloc((size_t)m * 3 * sizeof(double));
    double *a0 = (double *)malloc((size_t)m * 3 * sizeof(double));
    double *j0 = (double *)malloc((size_t)m * 3 * sizeof(double));
    double *x1 = (double *)malloc((size_t)m * 3 * sizeof(double));
    double *v1 = (double *)malloc((size_t)m * 3 * sizeof(double));
    double *a2 = (double *)malloc((size_t)m * 3 * sizeof(double));
    double *a3 = (double *)malloc((size_t)m * 3 * sizeof(double));
    for (int64_t k = 0; k < m; k++) {
        int64_t i = act[k];
        tk[k] = tau[i];
        for (int c = 0; c < 3; c++) {
            xa[3 * k + c] = xp[3 * i + c];
            va[3 * k + c] = vp[3 * i + c];
            a0[3 * k + c] = acc[3 * i + c];
            j0[3 * k + c] = jerk[3 * i + c];
        }
    }
    oracle_correct(m, tk, xa, va, a0, j0, a1, j1, x1, v1, a2, a3);
    for (int64_t k = 0; k < m; k++) {
        int64_t i = act[k];
        double dtc = oracle_aarseth_dt(a1 + 3 * k, j1 + 3 * k, a2 + 3 * k,
                                       a3 + 3 * k, eta);
        if (dtcrit_out) dtcrit_out[k] = dtc;
        for (int c = 0; c < 3; c++) {
            pos[3 * i + c] = x1[3 * k + c];
            vel[3 * i + c] = v1[3 * k + c];
            acc[3 * i + c] = a1[3 * k + c];
            jerk[3 * i + c] = j1[3 * k + c];
        }
        t[i] = t_next;
        level[i] = oracle_level(dtc, level[i], t_next, tick_exp, lmin, lmax);
    }
    if (t_next_out) *t_next_out = t_next;
    if (m_out) *m_out = m;
    if (active_out)
        for (int64_t k = 0; k < m; k++) active_out[k] = act[k];
    free(act); free(tau); free(xp); free(vp); free(a1); free(j1); free(tk);
    free(xa); free(va); free(a0); free(j0); free(x1); free(v1); free(a2);
    free(a3);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Start of an integration: acceleration and jerk of every particle at  */
/* t = 0 (one full force evaluation), all t_i = 0, and the first level  */
/* from the initial-step rule (reading; see oracle_initial_dt).         */
/* ------------------------------------------------------------------ */
int oracle_init(int64_t n, const double *pos, const double *vel,
                const double *mass, double *acc, double *jerk, int64_t *t,
                int32_t *level, double G, double eps, double eta_s,
                int tick_exp, int lmin, int lmax)
{
    int64_t *all = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!all) return -1;
    for (int64_t i = 0; i < n; i++) all[i] = i;
    int rc = oracle_force(n, pos, vel, mass, G, eps, n, all, acc, jerk, NULL);
    free(all);
    if (rc) return rc;
    for (int64_t i = 0; i < n; i++) {
        t[i] = 0;
        double dt0 = oracle_initial_dt(acc + 3 * i, jerk + 3 * i, eta_s);
        level[i] = oracle_level(dt0, -1, 0, tick_exp, lmin, lmax);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Kick-drift-kick leapfrog with one shared step: the acceleration-only */
/* workload the same force sum (Eq. 1, Eq. 2) drives.  The paper's      */
/* method needs the jerk for its Hermite scheme; this second-order,     */
/* time-symmetric integrator needs the acceleration alone.  Per step:   */
/*   kick  v <- v + a dt/2,  drift  x <- x + v dt,  a <- a(x),          */
/*   kick  v <- v + a dt/2.                                             */
/* oracle_kick and oracle_drift are the two halves on n x 3 arrays;     */
/* oracle_leapfrog takes n_steps steps, acc holding a(x) at the start   */
/* on entry and at the end on return.  Returns 0, or -1 when memory     */
/* runs out.                                                            */
/* ------------------------------------------------------------------ */
void oracle_kick(int64_t n, double *vel, const double *acc, double h)
{
    for (int64_t i = 0; i < 3 * n; i++) vel[i] = vel[i] + h * acc[i];
}

void oracle_drift(int64_t n, double *pos, const double *vel, double dt)
{
    for (int64_t i = 0; i < 3 * n; i++) pos[i] = pos[i] + dt * vel[i];
}

int oracle_leapfrog(int64_t n, double *pos, double *vel, double *acc,
                    const double *mass, double G, double eps, double dt,
                    int64_t n_steps)
{
    int64_t *idx = malloc(sizeof *idx * (size_t)(n > 0 ? n : 1));
    if (!idx) return -1;
    for (int64_t i = 0; i < n; i++) idx[i] = i;
    const double h = 0.5 * dt;
    for (int64_t s = 0; s < n_steps; s++) {
        oracle_kick(n, vel, acc, h);
        oracle_drift(n, pos, vel, dt);
        oracle_force(n, pos, vel, mass, G, eps, n, idx, acc, NULL, NULL);
        oracle_kick(n, vel, acc, h);
    }
    free(idx);
    return 0;
}

/* ------------------------------------------------------------------ */
/* 6th-order Hermite scheme (the order of the paper's template code,    */
/* Sec. 2 item 1; the paper prints no formula for it).                  */
/*                                                                      */
/* Force with snap.  With d = r_j - r_i, w = v_j - v_i, u = a_j - a_i   */
/* (the sources' and the target's accelerations at the same time),     */
/* s^2 = d.d + eps^2, alpha = (d.w)/s^2 and                             */
/* beta = (w.w + d.u)/s^2 + alpha^2, the pair term of Eq. 2 and its     */
/* first two time derivatives are                                       */
/*   A = G m_j d / s^3,                                                 */
/*   J = G m_j w / s^3 - 3 alpha A,                                     */
/*   S = G m_j u / s^3 - 6 alpha J - 3 beta A                           */
/* (differentiate A in time twice; d(alpha)/dt = beta - 3 alpha^2).     */
/* acc_src: n x 3 accelerations of all particles (the sources' and the  */
/* targets' own); out: acc, jerk, snap (m x 3), Neumaier-summed.        */
/* Returns 0, or -1 on a bad index.                                     */
/* ------------------------------------------------------------------ */
int oracle_force_snap(int64_t n, const double *pos, const double *vel,
                      const double *acc_src, const double *mass, double G,
                      double eps, int64_t m, const int64_t *idx, double *acc,
                      double *jerk, double *snap)
{
    for (int64_t k = 0; k < m; k++)
        if (idx[k] < 0 || idx[k] >= n) return -1;
    const double eps2 = eps * eps;
    int64_t k;
#pragma omp parallel for schedule(dynamic, 16)
    for (k = 0; k < m; k++) {
        const int64_t i = idx[k];
        nsum sa[3], sj[3], ss[3];
        memset(sa, 0, sizeof sa);
        memset(sj, 0, sizeof sj);
        memset(ss, 0, sizeof ss);
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3], w[3], u[3];
            for (int c = 0; c < 3; c++) {
                d[c] = pos[3 * j + c] - pos[3 * i + c];
                w[c] = vel[3 * j + c] - vel[3 * i + c];
                u[c] = acc_src[3 * j + c] - acc_src[3 * i + c];
            }
            double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
            double s3 = s2 * sqrt(s2);
            double dw = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
            double ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
            double du = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
            double alpha = dw / s2;
            double beta = (ww + du) / s2 + alpha * alpha;
            double gm = G * mass[j];
            for (int c = 0; c < 3; c++) {
                double A = gm * d[c] / s3;
                double J = gm * w[c] / s3 - 3.0 * alpha * A;
                double S = gm * u[c] / s3 - 6.0 * alpha * J - 3.0 * beta * A;
                nsum_add(&sa[c], A);
                nsum_add(&sj[c], J);
                nsum_add(&ss[c], S);
            }
        }
        for (int c = 0; c < 3; c++) {
            if (acc) acc[3 * k + c] = nsum_get(&sa[c]);
            if (jerk) jerk[3 * k + c] = nsum_get(&sj[c]);
            if (snap) snap[3 * k + c] = nsum_get(&ss[c]);
        }
    }
    return 0;
}

/* 6th-order Hermite corrector over a step h, from (x0, v0, a0, j0, s0) */
/* at the start and the force (a1, j1, s1) at the predicted end: the    */
/* quintic through (a0, j0, s0) and (a1, j1, s1) integrates exactly to   */
/*   v1 = v0 + h/2 (a0 + a1) - h^2/10 (j1 - j0) + h^3/120 (s0 + s1),     */
/* and the same rule on v (derivatives a, j) gives                      */
/*   x1 = x0 + h/2 (v0 + v1) - h^2/10 (a1 - a0) + h^3/120 (j0 + j1).     */
/* The quintic's derivatives at the end, for the next prediction and    */
/* the step criterion (Delta = a1 - a0):                                */
/*   crackle h^3 = 60 Delta - h (24 j0 + 36 j1) - h^2 (3 s0 - 9 s1),     */
/*   pop h^4     = 360 Delta - h (168 j0 + 192 j1) - h^2 (24 s0 - 36 s1),*/
/*   a5 h^5      = 720 Delta - 360 h (j0 + j1) - 60 h^2 (s0 - s1).       */
/* m particles, all arrays m x 3; h per particle.                       */
/* ------------------------------------------------------------------ */
void oracle_hermite6_correct(int64_t m, const double *h, const double *x0,
                             const double *v0, const double *a0,
                             const double *j0, const double *s0,
                             const double *a1, const double *j1,
                             const double *s1, double *x1, double *v1,
                             double *crackle, double *pop, double *a5)
{
    for (int64_t k = 0; k < m; k++) {
        const double t = h[k], t2 = t * t, t3 = t2 * t;
        for (int q = 0; q < 3; q++) {
            const int64_t i = 3 * k + q;
            /* every input is read before any output is written: the
               outputs may alias the inputs (x1 = x0, v1 = v0) */
            const double xo = x0[i], vo = v0[i];
            const double vv = vo + t / 2.0 * (a0[i] + a1[i])
                              - t2 / 10.0 * (j1[i] - j0[i])
                              + t3 / 120.0 * (s0[i] + s1[i]);
            const double xx = xo + t / 2.0 * (vo + vv)
                              - t2 / 10.0 * (a1[i] - a0[i])
                              + t3 / 120.0 * (j0[i] + j1[i]);
            v1[i] = vv;
            x1[i] = xx;
            const double D = a1[i] - a0[i];
            if (crackle)
                crackle[i] = (60.0 * D - t * (24.0 * j0[i] + 36.0 * j1[i])
                              - t2 * (3.0 * s0[i] - 9.0 * s1[i])) / t3;
            if (pop)
                pop[i] = (360.0 * D - t * (168.0 * j0[i] + 192.0 * j1[i])
                          - t2 * (24.0 * s0[i] - 36.0 * s1[i])) / (t3 * t);
            if (a5)
                a5[i] = (720.0 * D - 360.0 * t * (j0[i] + j1[i])
                         - 60.0 * t2 * (s0[i] - s1[i])) / (t3 * t2);
        }
    }
}

/* Step criterion of the 6th-order scheme: the generalised Aarseth      */
/* form of the p-th order Hermite schemes at p = 6,                     */
/*   dt = eta ( A1 / A4 )^(1/3),  A_k = sqrt(|a^(k-1)| |a^(k+1)|) + |a^(k)|, */
/* with a^(0..5) = a, jerk, snap, crackle, pop, a5; zero denominator    */
/* gives +inf.                                                          */
/* ------------------------------------------------------------------ */
double oracle_hermite6_dt(const double *a, const double *j, const double *s,
                          const double *c, const double *p, const double *q,
                          double eta)
{
    const double na = norm3(a), nj = norm3(j), ns = norm3(s);
    const double nc = norm3(c), np_ = norm3(p), nq = norm3(q);
    const double A1 = sqrt(na * ns) + nj;
    const double A4 = sqrt(nc * nq) + np_;
    if (!(A4 > 0.0)) return INFINITY;
    return eta * cbrt(A1 / A4);
}

/* Taylor predictor of the 6th-order scheme over t (per particle):       */
/*   x_p = x + v t + a t^2/2 + j t^3/6 + s t^4/24 + c t^5/120,          */
/*   v_p = v + a t + j t^2/2 + s t^3/6 + c t^4/24,                      */
/*   a_p = a + j t + s t^2/2 + c t^3/6                                  */
/* (s snap, c crackle).  m particles, arrays m x 3; t per particle.     */
/* ------------------------------------------------------------------ */
void oracle_hermite6_predict(int64_t m, const double *t, const double *x,
                             const double *v, const double *a, const double *j,
                             const double *s, const double *c, double *xp,
                             double *vp, double *ap)
{
    for (int64_t k = 0; k < m; k++) {
        const double h = t[k], h2 = h * h, h3 = h2 * h, h4 = h3 * h, h5 = h4 * h;
        for (int q = 0; q < 3; q++) {
            const int64_t i = 3 * k + q;
            xp[i] = x[i] + v[i] * h + a[i] * h2 / 2.0 + j[i] * h3 / 6.0
                    + s[i] * h4 / 24.0 + c[i] * h5 / 120.0;
            vp[i] = v[i] + a[i] * h + j[i] * h2 / 2.0 + s[i] * h3 / 6.0
                    + c[i] * h4 / 24.0;
            ap[i] = a[i] + j[i] * h + s[i] * h2 / 2.0 + c[i] * h3 / 6.0;
        }
    }
}

/* Shared-step 6th-order Hermite integration of every particle: n_steps */
/* steps of h.  Start: acc and jerk from oracle_force, snap from        */
/* oracle_force_snap with those accelerations, crackle zero (the first  */
/* prediction lacks its c tau^5/120 term; one step's error, so the      */
/* scheme stays 6th order).  Per step: predict every particle with      */
/*   x_p = x + v t + a t^2/2 + j t^3/6 + s t^4/24 + c t^5/120,          */
/*   v_p = v + a t + j t^2/2 + s t^3/6 + c t^4/24,                      */
/*   a_p = a + j t + s t^2/2 + c t^3/6,                                 */
/* take the force with snap at (x_p, v_p, a_p) and correct.             */
/* Returns 0, or -1 when memory runs out.                               */
/* ------------------------------------------------------------------ */
int oracle_hermite6_run(int64_t n, double *pos, double *vel,
                        const double *mass, double G, double eps, double h,
                        int64_t n_steps)
{
    const size_t b = sizeof(double) * 3 * (size_t)(n > 0 ? n : 1);
    double *a = malloc(b), *j = malloc(b), *s = malloc(b), *c = malloc(b);
    double *xp = malloc(b), *vp = malloc(b), *ap = malloc(b);
    double *a1 = malloc(b), *j1 = malloc(b), *s1 = malloc(b);
    double *hh = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t *idx = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int rc = 0;
    if (!a || !j || !s || !c || !xp || !vp || !ap || !a1 || !j1 || !s1 || !hh || !idx) {
        rc = -1;
        goto done;
    }
    for (int64_t i = 0; i < n; i++) {
        idx[i] = i;
        hh[i] = h;
    }
    oracle_force(n, pos, vel, mass, G, eps, n, idx, a, j, NULL);
    oracle_force_snap(n, pos, vel, a, mass, G, eps, n, idx, NULL, NULL, s);
    memset(c, 0, b);
    for (int64_t st = 0; st < n_steps; st++) {
        oracle_hermite6_predict(n, hh, pos, vel, a, j, s, c, xp, vp, ap);
        oracle_force_snap(n, xp, vp, ap, mass, G, eps, n, idx, a1, j1, s1);
        oracle_hermite6_correct(n, hh, pos, vel, a, j, s, a1, j1, s1, pos, vel,
                                c, NULL, NULL);
        memcpy(a, a1, b);
        memcpy(j, j1, b);
        memcpy(s, s1, b);
    }
done:
    free(a); free(j); free(s); free(c); free(xp); free(vp); free(ap);
    free(a1); free(j1); free(s1); free(hh); free(idx);
    return rc;
}
