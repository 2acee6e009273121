"""Pins of the FP64 CPU oracle against facts fixed by physics and mathematics.

None of these re-types the oracle's formulas: each compares it with a closed
form, a symmetry, a conservation law, a finite-difference derivative or an
extended-precision brute force, chosen so that a dropped term, a wrong sign or
exponent, or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1411_5234_gb300 import inputs


# ---------------------------------------------------------------- force ---

def test_two_body_exact_values():
    # d = 3, eps = 4: (d^2 + eps^2)^(1/2) = 5 exactly, so |a| = G m d / 125 and
    # phi = -G m / 5 exactly (Eq. 2 and the potential it derives from).
    pos = np.array([[0.0, 0, 0], [3.0, 0, 0]])
    vel = np.zeros((2, 3))
    mass = np.array([2.0, 5.0])
    acc, jerk, pot = oracle.force(pos, vel, mass, eps=4.0, G=1.0)
    assert acc[0] == pytest.approx([5.0 * 3 / 125, 0, 0], abs=1e-16)
    assert acc[1] == pytest.approx([-2.0 * 3 / 125, 0, 0], abs=1e-16)
    assert pot == pytest.approx([-5.0 / 5, -2.0 / 5], rel=1e-15)
    assert np.all(jerk == 0.0)
    # unsoftened unit case: attraction toward the other body, |a| = 1
    acc, _, pot = oracle.force(np.array([[0, 0, 0], [0, 0, 1.0]]), vel,
                               np.array([1.0, 1.0]), eps=0.0)
    assert acc[0].tolist() == [0.0, 0.0, 1.0]
    assert acc[1].tolist() == [0.0, 0.0, -1.0]
    assert pot.tolist() == [-1.0, -1.0]


def test_G_scales_linearly():
    cl = inputs.plummer(64, seed=3)
    a1, j1, p1 = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2, G=1.0)
    a2, j2, p2 = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2, G=2.5)
    # compensated sums: equal up to a few ulps of each vector's norm
    for x2, x1 in ((a2, a1), (j2, j1)):
        nrm = np.linalg.norm(x1, axis=1, keepdims=True)
        assert np.all(np.abs(x2 - 2.5 * x1) <= 4e-16 * 2.5 * nrm)
    np.testing.assert_allclose(p2, 2.5 * p1, rtol=1e-15)


def test_lagrange_equilateral_triangle():
    # Three equal masses on an equilateral triangle of side L: each is pulled
    # toward the centroid with |a| = sqrt(3) G m / L^2 (vector geometry).
    L, m = 0.7, 1.3
    pos = np.array([[0, 0, 0], [L, 0, 0], [L / 2, L * math.sqrt(3) / 2, 0]])
    acc, _, _ = oracle.force(pos, np.zeros((3, 3)), np.full(3, m), eps=0.0)
    c = pos.mean(0)
    for i in range(3):
        u = (c - pos[i]) / np.linalg.norm(c - pos[i])
        np.testing.assert_allclose(acc[i], math.sqrt(3) * m / L ** 2 * u,
                                   rtol=1e-14, atol=1e-15)


def _icosahedron(radius):
    p = (1 + math.sqrt(5)) / 2
    v = []
    for a in (-1, 1):
        for b in (-p, p):
            v += [(0, a, b), (a, b, 0), (b, 0, a)]
    v = np.array(v, dtype=np.float64)
    return radius * v / np.linalg.norm(v, axis=1, keepdims=True)


def test_shell_theorem_icosahedron():
    # The 12 vertices of an icosahedron form a spherical 5-design: the shell's
    # exterior field equals that of a point mass up to degree-6 multipoles,
    # so at distance R = 20 r it matches G M / R^2 to ~ (r/R)^6 ~ 1e-8, and the
    # potential matches -G M / R.  At the centre the pull cancels exactly by
    # symmetry.
    r, R = 0.05, 1.0
    shell = _icosahedron(r)
    mshell = np.full(12, 1.0 / 12)
    probe = np.array([[0.3 * R, -0.4 * R, math.sqrt(0.75) * R]])
    pos = np.vstack([shell, probe, [[0.0, 0.0, 0.0]]])
    mass = np.concatenate([mshell, [0.0, 0.0]])
    vel = np.zeros((14, 3))
    acc, _, pot = oracle.force(pos, vel, mass, eps=0.0, idx=[12, 13])
    np.testing.assert_allclose(acc[0], -probe[0] / R ** 3, rtol=1e-7)
    assert pot[0] == pytest.approx(-1.0 / R, rel=1e-7)
    np.testing.assert_allclose(acc[1], 0.0, atol=1e-13)
    assert pot[1] == pytest.approx(-1.0 / r, rel=1e-14)


def test_newton_third_law():
    cl = inputs.plummer(300, seed=7, imf="kroupa")
    acc, jerk, _ = oracle.force(cl.pos, cl.vel, cl.mass, eps=1e-3)
    m = cl.mass[:, None]
    scale_a = np.abs(m * acc).sum()
    scale_j = np.abs(m * jerk).sum()
    assert np.abs((m * acc).sum(0)).max() < 1e-14 * scale_a
    assert np.abs((m * jerk).sum(0)).max() < 1e-14 * scale_j


def test_acceleration_is_minus_gradient_of_potential():
    # a_i = -grad_i phi_i, checked by a 4th-order central difference of the
    # oracle's own potential (pins acc against pot: a wrong exponent or sign
    # in either one fails).
    cl = inputs.plummer(40, seed=11)
    eps = 0.05
    idx = [0, 5, 17, 39]
    acc, _, _ = oracle.force(cl.pos, cl.vel, cl.mass, eps, idx=idx)
    h = 1e-3
    for k, i in enumerate(idx):
        g = np.zeros(3)
        for c in range(3):
            vals = []
            for s in (-2, -1, 1, 2):
                p = cl.pos.copy()
                p[i, c] += s * h
                vals.append(oracle.force(p, cl.vel, cl.mass, eps, idx=[i])[2][0])
            g[c] = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
        np.testing.assert_allclose(acc[k], -g, rtol=1e-8, atol=1e-9 * np.abs(acc[k]).max())


def test_jerk_is_time_derivative_of_acceleration():
    # Along straight-line motion x_j(t) = x_j + v_j t the exact d/dt of the
    # softened acceleration at t = 0 is the jerk (it depends on x and v only).
    cl = inputs.plummer(40, seed=12)
    eps = 0.05
    idx = [1, 9, 33]
    _, jerk, _ = oracle.force(cl.pos, cl.vel, cl.mass, eps, idx=idx)
    h = 1e-3
    vals = [oracle.force(cl.pos + s * h * cl.vel, cl.vel, cl.mass, eps, idx=idx)[0]
            for s in (-2, -1, 1, 2)]
    fd = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
    np.testing.assert_allclose(jerk, fd, rtol=1e-7, atol=1e-8 * np.abs(jerk).max())


def test_circular_orbit_jerk_closed_form():
    # Two-body circular orbit: each body moves uniformly on a circle about the
    # centre of mass, so a = -w^2 x and da/dt = -w^2 v, w^2 = G M / r^3.
    m1, m2, r = 0.7, 0.3, 1.7
    M = m1 + m2
    w = math.sqrt(M / r ** 3)
    pos = np.array([[-m2 / M * r, 0, 0], [m1 / M * r, 0, 0]])
    vel = np.array([[0, -m2 / M * r * w, 0], [0, m1 / M * r * w, 0]])
    acc, jerk, _ = oracle.force(pos, vel, np.array([m1, m2]), eps=0.0)
    np.testing.assert_allclose(acc, -w * w * pos, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(jerk, -w * w * vel, rtol=1e-14, atol=1e-16)


def test_brute_force_extended_precision():
    # 50-digit brute force on a tiny system bounds the oracle's own FP64
    # rounding (it runs the definition in mpmath, not the oracle's code path).
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    cl = inputs.plummer(16, seed=5, imf="kroupa")
    eps = 1e-3
    acc, jerk, pot = oracle.force(cl.pos, cl.vel, cl.mass, eps)
    P = [[mp.mpf(float(x)) for x in row] for row in cl.pos]
    V = [[mp.mpf(float(x)) for x in row] for row in cl.vel]
    Mm = [mp.mpf(float(x)) for x in cl.mass]
    e2 = mp.mpf(eps) ** 2
    for i in range(16):
        a = [mp.mpf(0)] * 3
        jk = [mp.mpf(0)] * 3
        ph = mp.mpf(0)
        ca = cj = mp.mpf(0)            # sums of |terms| (the conditioning)
        for j in range(16):
            if j == i:
                continue
            d = [P[j][c] - P[i][c] for c in range(3)]
            w = [V[j][c] - V[i][c] for c in range(3)]
            s = mp.sqrt(sum(x * x for x in d) + e2)
            dw = sum(d[c] * w[c] for c in range(3))
            for c in range(3):
                ta = Mm[j] * d[c] / s ** 3
                tj = Mm[j] * (w[c] / s ** 3 - 3 * dw * d[c] / s ** 5)
                a[c] += ta
                jk[c] += tj
                ca += abs(ta)
                cj += abs(tj)
            ph -= Mm[j] / s
        ref_a = np.array([float(x) for x in a])
        ref_j = np.array([float(x) for x in jk])
        # each FP64 term carries a few ulps; compensated summation adds ~1 ulp
        assert np.abs(acc[i] - ref_a).max() <= 1e-15 * float(ca)
        assert np.abs(jerk[i] - ref_j).max() <= 1e-15 * float(cj)
        assert abs(pot[i] - float(ph)) <= 4e-16 * abs(float(ph))


def test_force_subset_equals_full():
    cl = inputs.plummer(100, seed=2)
    a, j, p = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2)
    idx = np.array([99, 3, 50])
    a2, j2, p2 = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2, idx=idx)
    assert np.array_equal(a2, a[idx]) and np.array_equal(j2, j[idx])
    assert np.array_equal(p2, p[idx])
    with pytest.raises(ValueError):
        oracle.force(cl.pos, cl.vel, cl.mass, 1e-2, idx=[100])


# --------------------------------------------------------------- energy ---

def test_energy_closed_forms():
    # softened pair energy at d = 3, eps = 4: -G m1 m2 / 5 exactly
    ek, ep = oracle.energy(np.array([[0, 0, 0], [0, 3.0, 0]]),
                           np.array([[1.0, 0, 0], [0, 0, 2.0]]),
                           np.array([2.0, 5.0]), eps=4.0)
    assert ep == pytest.approx(-2.0, rel=1e-15)
    assert ek == pytest.approx(0.5 * 2 * 1 + 0.5 * 5 * 4, rel=1e-15)
    # circular orbit: virial 2K = -W and E = -G m1 m2 / (2 r)
    m1, m2, r = 0.7, 0.3, 1.7
    M = m1 + m2
    w = math.sqrt(M / r ** 3)
    pos = np.array([[-m2 / M * r, 0, 0], [m1 / M * r, 0, 0]])
    vel = np.array([[0, -m2 / M * r * w, 0], [0, m1 / M * r * w, 0]])
    ek, ep = oracle.energy(pos, vel, np.array([m1, m2]), eps=0.0)
    assert 2 * ek == pytest.approx(-ep, rel=1e-14)
    assert ek + ep == pytest.approx(-m1 * m2 / (2 * r), rel=1e-14)
    L, P = oracle.momenta(pos, vel, np.array([m1, m2]))
    mu = m1 * m2 / M
    assert L[2] == pytest.approx(mu * r * r * w, rel=1e-14)
    np.testing.assert_allclose(P, 0.0, atol=1e-16)


def test_potential_energy_is_half_sum_m_phi():
    cl = inputs.plummer(200, seed=4, imf="kroupa")
    _, _, pot = oracle.force(cl.pos, cl.vel, cl.mass, 1e-3)
    _, ep = oracle.energy(cl.pos, cl.vel, cl.mass, 1e-3)
    assert ep == pytest.approx(0.5 * np.dot(cl.mass, pot), rel=1e-13)


# ------------------------------------------------------------ integrator ---

def test_predictor_exact_for_constant_jerk_motion():
    rng = np.random.default_rng(0)
    x, v, a, j = (rng.normal(size=(5, 3)) for _ in range(4))
    tau = np.array([0.0, 0.1, -0.2, 1.5, 0.03125])
    xp, vp = oracle.predict(x, v, a, j, tau)
    t = tau[:, None]
    np.testing.assert_allclose(xp, x + v * t + a * t ** 2 / 2 + j * t ** 3 / 6, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(vp, v + a * t + j * t ** 2 / 2, rtol=1e-14, atol=1e-14)


def test_corrector_recovers_quintic_trajectory():
    # If a(t) is exactly a cubic, a = a0 + j0 t + s t^2/2 + c t^3/6, the
    # two-point Hermite fit recovers s and c, and the corrected state is the
    # exact x(tau), v(tau) of that motion.
    rng = np.random.default_rng(1)
    m = 4
    x0, v0, a0, j0, s, c = (rng.normal(size=(m, 3)) for _ in range(6))
    tau = np.array([0.5, 0.125, 1.0, 0.015625])
    t = tau[:, None]
    a1 = a0 + j0 * t + s * t ** 2 / 2 + c * t ** 3 / 6
    j1 = j0 + s * t + c * t ** 2 / 2
    xp, vp = oracle.predict(x0, v0, a0, j0, tau)
    x1, v1, a2e, a3e = oracle.correct(tau, xp, vp, a0, j0, a1, j1)
    x_ex = x0 + v0 * t + a0 * t ** 2 / 2 + j0 * t ** 3 / 6 + s * t ** 4 / 24 + c * t ** 5 / 120
    v_ex = v0 + a0 * t + j0 * t ** 2 / 2 + s * t ** 3 / 6 + c * t ** 4 / 24
    np.testing.assert_allclose(x1, x_ex, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(v1, v_ex, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(a3e, c, rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(a2e, s + c * t, rtol=1e-9, atol=1e-9)


def test_aarseth_dt_circular_orbit():
    # uniform circular motion: |a| = w^2 r, |j| = w^3 r, |a2| = w^4 r,
    # |a3| = w^5 r, so the criterion gives dt = sqrt(eta) / w.
    w, r, eta = 3.0, 0.4, 0.01
    ang = 0.3
    u = np.array([math.cos(ang), math.sin(ang), 0.0])
    p = np.array([-math.sin(ang), math.cos(ang), 0.0])
    dt = oracle.aarseth_dt(-w ** 2 * r * u, -w ** 3 * r * p, w ** 4 * r * u, w ** 5 * r * p, eta)
    assert dt == pytest.approx(math.sqrt(eta) / w, rel=1e-14)
    assert oracle.aarseth_dt(u, np.zeros(3), np.zeros(3), np.zeros(3), eta) == math.inf
    assert oracle.initial_dt(2 * u, 8 * p, 0.01) == pytest.approx(0.0025, rel=1e-15)


def test_level_rules():
    T = 40
    # largest power of two not above dt_crit
    assert oracle.level(0.3, -1, 0, T, 0, 30) == 2
    assert oracle.level(0.25, -1, 0, T, 0, 30) == 2
    assert oracle.level(0.2499999, -1, 0, T, 0, 30) == 3
    assert oracle.level(2.0 ** -20 * 1.5, -1, 0, T, 0, 30) == 20
    # clamps
    assert oracle.level(1e-30, -1, 0, T, 3, 20) == 20
    assert oracle.level(100.0, -1, 0, T, 3, 20) == 3
    assert oracle.level(math.inf, -1, 0, T, 3, 20) == 3
    assert oracle.level(0.0, -1, 0, T, 3, 20) == 20
    # shrinking is always allowed, to any depth
    assert oracle.level(2.0 ** -9, 5, 3 << (T - 5), T, 0, 30) == 9
    # growing: one doubling at most, and only on a commensurate time
    t_ok = 4 << (T - 5)        # multiple of 2^-4
    t_bad = 3 << (T - 5)       # odd multiple of 2^-5
    assert oracle.level(0.9, 5, t_ok, T, 0, 30) == 4
    assert oracle.level(0.9, 5, t_bad, T, 0, 30) == 5
    assert oracle.level(5.0, 0, 0, T, 0, 30) == 0     # already the largest step
    assert oracle.level(0.9, 0, 0, T, 0, 30) == 1     # 0.5 <= 0.9 < 1: shrink


def _kepler_state(a, e, M_tot, t, phase0=0.0):
    """Relative position/velocity of a Kepler orbit at time t (periapsis at 0)."""
    n = math.sqrt(M_tot / a ** 3)
    Mn = n * t + phase0
    E = Mn
    for _ in range(100):
        E = E - (E - e * math.sin(E) - Mn) / (1 - e * math.cos(E))
    r = a * (1 - e * math.cos(E))
    x = np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])
    v = np.array([-a * a * n * math.sin(E) / r, a * a * n * math.sqrt(1 - e * e) * math.cos(E) / r, 0.0])
    return x, v


def _kepler_run(level, e=0.5, t_end=1.0):
    # period 1 time unit: a = 1, G M = 4 pi^2
    M = 4 * math.pi ** 2
    m1, m2 = 0.6 * M, 0.4 * M
    x, v = _kepler_state(1.0, e, M, 0.0)
    pos = np.array([-m2 / M * x, m1 / M * x])
    vel = np.array([-m2 / M * v, m1 / M * v])
    st = oracle.State(pos, vel, np.array([m1, m2]), eps=0.0, tick_exp=40,
                      lmin=level, lmax=level)
    nsteps = int(round(t_end * 2 ** level))
    for _ in range(nsteps):
        st.block_step()
    xr, vr = _kepler_state(1.0, e, M, t_end)
    rel = st.pos[1] - st.pos[0]
    return np.linalg.norm(rel - xr), st


def test_hermite4_kepler_fourth_order():
    # Closed-form Kepler orbit (e = 0.5, one period): the Hermite scheme is
    # 4th order (Sec. 2 item 1), so halving dt cuts the error by ~2^4.
    errs = [_kepler_run(L)[0] for L in (8, 9, 10)]
    assert errs[0] < 1e-4
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0, errs


def test_hermite4_kepler_mid_orbit_and_conservation():
    err, st = _kepler_run(10, e=0.3, t_end=0.375)
    assert err < 1e-8
    ek, ep = oracle.energy(st.pos, st.vel, st.mass, 0.0)
    # Kepler energy -G m1 m2 / (2a), a = 1; 4th-order truncation error only
    assert ek + ep == pytest.approx(-st.mass[0] * st.mass[1] / 2.0, rel=1e-8)
    assert st.time() == 0.375


def test_block_step_equals_shared_step_composition():
    # With every particle on one level the block step is one shared Hermite
    # step; compose it from the primitive predictor / force / corrector.
    cl = inputs.plummer(24, seed=9)
    eps, L = 1e-2, 7
    st = oracle.State(cl.pos, cl.vel, cl.mass, eps=eps, lmin=L, lmax=L)
    x, v, a, j = st.pos.copy(), st.vel.copy(), st.acc.copy(), st.jerk.copy()
    for _ in range(3):
        tau = np.full(24, 2.0 ** -L)
        xp, vp = oracle.predict(x, v, a, j, tau)
        a1, j1, _ = oracle.force(xp, vp, cl.mass, eps)
        x, v, _, _ = oracle.correct(tau, xp, vp, a, j, a1, j1)
        a, j = a1, j1
        t_next, act, _ = st.block_step()
        assert len(act) == 24
    assert np.array_equal(st.pos, x) and np.array_equal(st.vel, v)
    assert np.array_equal(st.acc, a) and np.array_equal(st.jerk, j)
    assert t_next == 3 << (40 - L)


def test_block_step_invariants_and_conservation():
    cl = inputs.plummer(64, seed=1)
    eps = 1e-2
    st = oracle.State(cl.pos, cl.vel, cl.mass, eps=eps, eta=0.02, lmin=3, lmax=16)
    e0 = sum(oracle.energy(st.pos, st.vel, st.mass, eps))
    L0, P0 = oracle.momenta(st.pos, st.vel, st.mass)
    T = st.tick_exp
    t_prev = 0
    levels_seen = set()
    while True:
        due = st.t + (np.int64(1) << (T - st.level.astype(np.int64)))
        t_next, act, _ = st.block_step()
        assert t_next == due.min() and t_next > t_prev
        assert np.array_equal(act, np.flatnonzero(due == t_next))
        assert np.all(st.t[act] == t_next)
        dt = np.int64(1) << (T - st.level.astype(np.int64))
        assert np.all(st.t % dt == 0)               # commensurate times
        assert st.level.min() >= 3 and st.level.max() <= 16
        levels_seen.update(st.level.tolist())
        t_prev = t_next
        if t_next == 1 << (T - 3):                  # everybody synchronised
            assert np.all(st.t == t_next)
            break
    assert len(levels_seen) > 1                     # really a block hierarchy
    e1 = sum(oracle.energy(st.pos, st.vel, st.mass, eps))
    L1, P1 = oracle.momenta(st.pos, st.vel, st.mass)
    assert abs((e1 - e0) / e0) < 1e-6
    # with individual steps the pair forces act at different times, so L and
    # P are conserved only to truncation level (scale: sum m |v| ~ 0.7)
    np.testing.assert_allclose(L1, L0, atol=1e-7)
    np.testing.assert_allclose(P1, P0, atol=1e-7)


# ------------------------------------------------- leapfrog (KDK) ----

def test_leapfrog_free_motion():
    # G = 0: no force, so velocities stay exactly and positions move by
    # n dt v (dt a power of two: every product exact, one rounding per add)
    rng = np.random.default_rng(5)
    pos, vel = rng.normal(size=(16, 3)), rng.normal(size=(16, 3))
    x, v, a = oracle.leapfrog(pos, vel, np.zeros((16, 3)), np.ones(16), 0.1, 2.0 ** -6, 64, G=0.0)
    assert np.array_equal(v, vel) and np.array_equal(a, np.zeros((16, 3)))
    assert np.allclose(x, pos + 64 * 2.0 ** -6 * vel, rtol=0, atol=1e-13)


def test_leapfrog_time_reversible():
    # kick-drift-kick is time-symmetric: n steps, reversed velocities, n
    # steps, reversed again returns the start to round-off
    cl = inputs.plummer(32, seed=4)
    a0 = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2)[0]
    x, v, a = oracle.leapfrog(cl.pos, cl.vel, a0, cl.mass, 1e-2, 2.0 ** -8, 64)
    x2, v2, _ = oracle.leapfrog(x, -v, a, cl.mass, 1e-2, 2.0 ** -8, 64)
    assert np.abs(x2 - cl.pos).max() < 1e-11
    assert np.abs(-v2 - cl.vel).max() < 1e-11
    assert np.abs(x - cl.pos).max() > 1e-3      # it did move


def test_leapfrog_second_order_kepler():
    # closed-form Kepler orbit (e = 0.5, one period): the scheme is second
    # order, so halving dt cuts the error by ~2^2
    M = 4 * math.pi ** 2
    m1, m2 = 0.6 * M, 0.4 * M
    xk, vk = _kepler_state(1.0, 0.5, M, 0.0)
    pos = np.array([-m2 / M * xk, m1 / M * xk])
    vel = np.array([-m2 / M * vk, m1 / M * vk])
    mass = np.array([m1, m2])
    a0 = oracle.force(pos, vel, mass, 0.0)[0]
    xr, _ = _kepler_state(1.0, 0.5, M, 1.0)
    errs = []
    for L in (10, 11, 12):
        x, v, _ = oracle.leapfrog(pos, vel, a0, mass, 0.0, 2.0 ** -L, 2 ** L)
        errs.append(np.linalg.norm((x[1] - x[0]) - xr))
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.5 < e1 / e2 < 4.5, errs


def test_leapfrog_conserves_momentum():
    cl = inputs.plummer(64, seed=6)
    a0 = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2)[0]
    p0 = (cl.mass[:, None] * cl.vel).sum(0)
    _, v, _ = oracle.leapfrog(cl.pos, cl.vel, a0, cl.mass, 1e-2, 2.0 ** -8, 32)
    assert np.abs((cl.mass[:, None] * v).sum(0) - p0).max() < 1e-13


def test_oracle_reproduces_stored_values():
    # tests/golden/plummer64_seed0_eps1e-2.txt, written by
    # tests/golden/make_golden.py from the oracle: the same numbers on every
    # host the oracle is built on (compensated sums, no FMA contraction)
    path = os.path.join(os.path.dirname(__file__), "golden", "plummer64_seed0_eps1e-2.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    ek_ref, ep_ref = (float(t) for t in rows[0][1:])
    force = np.array([[float(t) for t in r[1:]] for r in rows if r[0] == "force"])
    lf = np.array([[float(t) for t in r[1:]] for r in rows if r[0] == "leapfrog8"])
    cl = inputs.plummer(64, seed=0)
    acc, jerk, pot = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2)
    ek, ep = oracle.energy(cl.pos, cl.vel, cl.mass, 1e-2)
    x, v, _ = oracle.leapfrog(cl.pos, cl.vel, acc, cl.mass, 1e-2, 2.0 ** -6, 8)
    got = np.hstack([acc, jerk, pot[:, None]])
    assert np.allclose(got, force, rtol=1e-14, atol=1e-14)
    assert ek == pytest.approx(ek_ref, rel=1e-14) and ep == pytest.approx(ep_ref, rel=1e-14)
    assert np.allclose(np.hstack([x, v]), lf, rtol=1e-13, atol=1e-13)


# ------------------------------------------- 6th-order Hermite scheme ----

def test_snap_is_time_derivative_of_jerk():
    # every particle moves with its own constant acceleration u_i:
    # x(t) = x0 + v0 t + u t^2/2, v(t) = v0 + u t; the snap at t = 0 (with
    # the accelerations u) is d/dt of the jerk along that motion
    rng = np.random.default_rng(3)
    n = 12
    x0, v0, u = rng.normal(size=(n, 3)), rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    mass = rng.uniform(0.5, 1.5, n)
    eps = 0.1
    h = 1e-3
    jt = lambda t: oracle.force(x0 + v0 * t + u * t * t / 2, v0 + u * t, mass, eps)[1]
    fd = (8 * (jt(h) - jt(-h)) - (jt(2 * h) - jt(-2 * h))) / (12 * h)
    _, _, snap = oracle.force_snap(x0, v0, u, mass, eps)
    assert np.allclose(snap, fd, rtol=1e-7, atol=1e-7 * np.abs(snap).max())


def test_snap_circular_orbit_closed_form():
    # two bodies on a circular orbit about their centre of mass: every
    # derivative rotates with the orbit, a = -w^2 r, jerk = -w^2 v,
    # snap = w^4 r (r, v each body's from the centre of mass)
    m1, m2, R = 0.7, 0.3, 1.3
    w = math.sqrt((m1 + m2) / R ** 3)
    r1, r2 = np.array([-m2 / (m1 + m2) * R, 0, 0]), np.array([m1 / (m1 + m2) * R, 0, 0])
    v1, v2 = np.array([0, w * r1[0], 0]), np.array([0, w * r2[0], 0])   # w z x r
    pos, vel, mass = np.array([r1, r2]), np.array([v1, v2]), np.array([m1, m2])
    a = -w * w * pos
    acc, jerk, snap = oracle.force_snap(pos, vel, a, mass, 0.0)
    assert np.allclose(acc, a, rtol=1e-13, atol=1e-15)
    assert np.allclose(jerk, -w * w * vel, rtol=1e-13, atol=1e-15)
    assert np.allclose(snap, w ** 4 * pos, rtol=1e-12, atol=1e-15)


def test_snap_third_law():
    cl = inputs.plummer(80, seed=9, imf="kroupa")
    a = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2)[0]
    _, _, snap = oracle.force_snap(cl.pos, cl.vel, a, cl.mass, 1e-2)
    scale = (cl.mass[:, None] * np.abs(snap)).sum(0).max()
    assert np.abs((cl.mass[:, None] * snap).sum(0)).max() < 1e-13 * scale


def test_hermite6_corrector_exact_for_polynomials():
    # a degree-6 trajectory has a degree-4 acceleration, which the quintic
    # through (a, jerk, snap) at both ends reproduces: positions, velocities
    # and the end derivatives come out exactly (to rounding)
    rng = np.random.default_rng(8)
    P = rng.normal(size=(7, 3))                  # x(t) = sum_k P_k t^k
    def deriv(t, d):
        out = np.zeros(3)
        for k in range(d, 7):
            out += P[k] * math.factorial(k) / math.factorial(k - d) * t ** (k - d)
        return out
    h = 0.37
    x1, v1, c1, p1, q1 = oracle.hermite6_correct(
        h, deriv(0, 0), deriv(0, 1), deriv(0, 2), deriv(0, 3), deriv(0, 4),
        deriv(h, 2), deriv(h, 3), deriv(h, 4))
    assert np.allclose(x1[0], deriv(h, 0), rtol=1e-13, atol=1e-13)
    assert np.allclose(v1[0], deriv(h, 1), rtol=1e-13, atol=1e-13)
    assert np.allclose(c1[0], deriv(h, 5), rtol=1e-10, atol=1e-10)
    assert np.allclose(p1[0], deriv(h, 6), rtol=1e-9, atol=1e-9)
    assert np.allclose(q1[0], 0.0, atol=1e-8)    # the 7th derivative of x is zero


def test_hermite6_predictor_exact_for_quintic_motion():
    # x(t) = sum_{k<=5} P_k t^k: the 6th-order predictor's Taylor series in
    # (x, v, a, jerk, snap, crackle) is exact for it, and so are its velocity
    # and acceleration (to rounding)
    rng = np.random.default_rng(12)
    P = rng.normal(size=(6, 3))
    def deriv(t, d):
        out = np.zeros(3)
        for k in range(d, 6):
            out += P[k] * math.factorial(k) / math.factorial(k - d) * t ** (k - d)
        return out
    h = 0.43
    xp, vp, ap = oracle.hermite6_predict(h, *[deriv(0, d) for d in range(6)])
    assert np.allclose(xp[0], deriv(h, 0), rtol=1e-14, atol=1e-14)
    assert np.allclose(vp[0], deriv(h, 1), rtol=1e-14, atol=1e-14)
    assert np.allclose(ap[0], deriv(h, 2), rtol=1e-14, atol=1e-14)
    # several particles with their own steps
    hs = np.array([0.1, 0.25, 0.5])
    xs, vs, as_ = oracle.hermite6_predict(hs, *[np.array([deriv(0, d)] * 3) for d in range(6)])
    for k, hk in enumerate(hs):
        assert np.allclose(xs[k], deriv(hk, 0), rtol=1e-14, atol=1e-14)
        assert np.allclose(as_[k], deriv(hk, 2), rtol=1e-14, atol=1e-14)


def test_hermite6_sixth_order_kepler():
    # closed-form Kepler orbit (e = 0.5, one period), shared steps: halving
    # dt cuts the error by ~2^6
    M = 4 * math.pi ** 2
    m1, m2 = 0.6 * M, 0.4 * M
    xk, vk = _kepler_state(1.0, 0.5, M, 0.0)
    pos = np.array([-m2 / M * xk, m1 / M * xk])
    vel = np.array([-m2 / M * vk, m1 / M * vk])
    xr, _ = _kepler_state(1.0, 0.5, M, 1.0)
    errs = []
    for L in (7, 8, 9):
        x, _ = oracle.hermite6_run(pos, vel, np.array([m1, m2]), 0.0, 2.0 ** -L, 2 ** L)
        errs.append(np.linalg.norm((x[1] - x[0]) - xr))
    assert errs[0] < 1e-4
    for e1, e2 in zip(errs, errs[1:]):
        assert 48.0 < e1 / e2 < 80.0, errs


def test_hermite6_dt_circular_orbit():
    # on a circular orbit |a^(k)| = w^k |a|, so A1 = 2 w |a| ... the
    # generalised criterion gives eta / w exactly
    w, r = 2.5, 0.8
    vecs = [np.array([math.cos(0.3 + k * math.pi / 2), math.sin(0.3 + k * math.pi / 2), 0.0])
            * r * w ** (k + 2) for k in range(6)]
    assert oracle.hermite6_dt(*vecs, 0.2) == pytest.approx(0.2 / w, rel=1e-14)


# --------------------------------------------------------- symmetries ----

def _rotation(seed):
    q = np.random.default_rng(seed).normal(size=4)
    a, b, c, d = q / np.linalg.norm(q)
    return np.array([[a*a + b*b - c*c - d*d, 2*(b*c - a*d), 2*(b*d + a*c)],
                     [2*(b*c + a*d), a*a - b*b + c*c - d*d, 2*(c*d - a*b)],
                     [2*(b*d - a*c), 2*(c*d + a*b), a*a - b*b - c*c + d*d]])


def test_force_translation_and_rotation_covariance():
    cl = inputs.plummer(50, seed=21, imf="kroupa")
    a, j, p = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2)
    sa, sj = np.abs(a).max(), np.abs(j).max()
    a2, j2, p2 = oracle.force(cl.pos + np.array([3.0, -7.0, 11.0]), cl.vel, cl.mass, 1e-2)
    assert np.allclose(a2, a, rtol=0, atol=1e-12 * sa) and np.allclose(j2, j, rtol=0, atol=1e-12 * sj)
    assert np.allclose(p2, p, rtol=1e-12)
    R = _rotation(4)
    a3, j3, p3 = oracle.force(cl.pos @ R.T, cl.vel @ R.T, cl.mass, 1e-2)
    assert np.allclose(a3, a @ R.T, rtol=0, atol=1e-13 * sa)
    assert np.allclose(j3, j @ R.T, rtol=0, atol=1e-13 * sj)
    assert np.allclose(p3, p, rtol=1e-13)


def test_force_galilean_reversal_and_mass_scaling():
    cl = inputs.plummer(50, seed=22, imf="kroupa")
    a, j, p = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2)
    sj = np.abs(j).max()
    # a common velocity changes no relative velocity: acc and jerk stay
    a2, j2, _ = oracle.force(cl.pos, cl.vel + np.array([5.0, -2.0, 1.0]), cl.mass, 1e-2)
    assert np.array_equal(a2, a) and np.allclose(j2, j, rtol=0, atol=1e-12 * sj)
    # reversed velocities: acc stays, the jerk flips
    a3, j3, _ = oracle.force(cl.pos, -cl.vel, cl.mass, 1e-2)
    assert np.array_equal(a3, a) and np.allclose(j3, -j, rtol=0, atol=1e-14 * sj)
    # twice the masses: twice every sum
    a4, j4, p4 = oracle.force(cl.pos, cl.vel, 2.0 * cl.mass, 1e-2)
    assert np.allclose(a4, 2 * a, rtol=1e-14) and np.allclose(p4, 2 * p, rtol=1e-14)


def test_snap_invariant_under_a_common_acceleration():
    cl = inputs.plummer(40, seed=23)
    acc = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2)[0]
    _, _, s1 = oracle.force_snap(cl.pos, cl.vel, acc, cl.mass, 1e-2)
    _, _, s2 = oracle.force_snap(cl.pos, cl.vel, acc + np.array([0.3, 0.1, -0.2]), cl.mass, 1e-2)
    assert np.allclose(s2, s1, rtol=0, atol=1e-12 * np.abs(s1).max())
