"""GPU parity of the 6th-order Hermite path (the order of the paper's template
code, Sec. 2 item 1) against the FP64 CPU oracle.

* Force with snap (nb_force_snap) from an identical state: positions,
  velocities and accelerations set through nb_set_state, so the sources'
  accelerations in the snap term are the oracle's own inputs.  FP64 path:
  per-particle relative error <= 1e-12 for acceleration and jerk, and for
  the snap, whose three kinds of terms (u, alpha w, beta d) partly cancel,
  <= 1e-11.  Mixed path: condition-scaled errors ||d x_i|| / sum_j |x_ij|
  <= 1e-6 (acceleration), 3e-6 (jerk) and 2e-5 (snap: 48 FP32 operations
  per pair, the accelerations u = a_j - a_i rounded to FP32).
* Shared steps against oracle_hermite6_run (same start: a, jerk from the
  force, snap from the force with those accelerations, crackle zero).
* One block step of individual levels against the oracle's 6th-order
  predictor, force with snap, corrector and step criterion, per sampled
  particle; particles that are not due stay untouched.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1411_5234_gb300 import inputs

from test_gpu_parity import rel_err

pytestmark = pytest.mark.gpu


def snap_term_sums(pos, vel, acc, mass, eps, idx):
    """sum_j |a_ij|, |jerk_ij|, |snap_ij| per target (the FP64 pair terms of
    the oracle's formula, magnitudes summed)."""
    idx = np.asarray(idx)
    out = np.empty((len(idx), 3))
    for c0 in range(0, len(idx), 128):
        ii = idx[c0:c0 + 128]
        d = pos[None] - pos[ii, None]
        w = vel[None] - vel[ii, None]
        u = acc[None] - acc[ii, None]
        s2 = (d * d).sum(2) + eps * eps
        s2[np.arange(len(ii)), ii] = np.inf
        inv3 = s2 ** -1.5
        alpha = (d * w).sum(2) / s2
        beta = ((w * w).sum(2) + (d * u).sum(2)) / s2 + alpha ** 2
        m = mass[None, :, None]
        A = m * d * inv3[..., None]
        J = m * w * inv3[..., None] - 3 * alpha[..., None] * A
        S = m * u * inv3[..., None] - 6 * alpha[..., None] * J - 3 * beta[..., None] * A
        out[c0:c0 + 128, 0] = np.linalg.norm(A, axis=2).sum(1)
        out[c0:c0 + 128, 1] = np.linalg.norm(J, axis=2).sum(1)
        out[c0:c0 + 128, 2] = np.linalg.norm(S, axis=2).sum(1)
    return out


def synthetic_state(cl, eps, seed):
    """Oracle accelerations and jerks of the initial state, plus seeded
    snap and crackle of the size a Plummer sphere has."""
    a, j, _ = oracle.force(cl.pos, cl.vel, cl.mass, eps)
    s = inputs.random_vectors(cl.n, 50.0, seed=seed)
    c = inputs.random_vectors(cl.n, 300.0, seed=seed + 1)
    return a, j, s, c


@pytest.mark.parametrize("n,m", [(1024, 1024), (4099, 517)])
def test_force_snap_fp64_matches_oracle(nb, n, m):
    cl = inputs.plummer(n, seed=3, imf="kroupa")
    eps = 1e-4
    a0, j0, _, _ = synthetic_state(cl, eps, 5)
    idx = inputs.random_active(n, m, seed=2)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=eps, precision=nb.NB_FP64, order=6,
                 level_min=10, level_max=10)
    sim.set_state(cl.pos, cl.vel, a0, j0, np.zeros(n, dtype=np.int64),
                  np.full(n, 10, dtype=np.int32))
    sim.predict(0)
    a, j, s, p = (x.cpu().numpy() for x in sim.force_snap(torch.as_tensor(idx, device="cuda")))
    assert sim.status() == nb.NB_OK
    sim.close()
    ra, rj, rs = oracle.force_snap(cl.pos, cl.vel, a0, cl.mass, eps, idx=idx.astype(np.int64))
    _, _, rp = oracle.force(cl.pos, cl.vel, cl.mass, eps, idx=idx.astype(np.int64))
    assert rel_err(a, ra).max() <= 1e-12
    assert rel_err(j, rj).max() <= 1e-12
    assert rel_err(s, rs).max() <= 1e-11, rel_err(s, rs).max()
    assert np.abs(p / rp - 1).max() <= 1e-12


@pytest.mark.parametrize("n,m", [(4099, 4099), (8192, 333)])
def test_force_snap_mixed_matches_oracle(nb, n, m):
    cl = inputs.plummer(n, seed=4, imf="kroupa")
    eps = 1e-4
    a0, j0, _, _ = synthetic_state(cl, eps, 7)
    idx = inputs.random_active(n, m, seed=3)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=eps, precision=nb.NB_MIXED, order=6,
                 level_min=10, level_max=10)
    sim.set_state(cl.pos, cl.vel, a0, j0, np.zeros(n, dtype=np.int64),
                  np.full(n, 10, dtype=np.int32))
    sim.predict(0)
    a, j, s, _ = (x.cpu().numpy() for x in sim.force_snap(torch.as_tensor(idx, device="cuda")))
    assert sim.status() == nb.NB_OK
    sim.close()
    ii = idx.astype(np.int64)
    ra, rj, rs = oracle.force_snap(cl.pos, cl.vel, a0, cl.mass, eps, idx=ii)
    S = snap_term_sums(cl.pos, cl.vel, a0, cl.mass, eps, ii)
    ca = np.linalg.norm(a - ra, axis=1) / S[:, 0]
    cj = np.linalg.norm(j - rj, axis=1) / S[:, 1]
    cs = np.linalg.norm(s - rs, axis=1) / S[:, 2]
    assert ca.max() <= 1e-6, ca.max()
    assert cj.max() <= 3e-6, cj.max()
    assert cs.max() <= 2e-5, cs.max()
    assert np.median(rel_err(a, ra)) <= 1e-7
    assert np.median(rel_err(s, rs)) <= 1e-5, np.median(rel_err(s, rs))


def test_force_snap_needs_an_order6_context(nb):
    cl = inputs.plummer(64, seed=1)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-2)
    sim.predict(0)
    with pytest.raises(nb.NBError) as e:
        sim.force_snap(torch.arange(4, dtype=torch.int32, device="cuda"))
    assert e.value.code == nb.NB_ESTATE
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hermite6_shared_steps_match_oracle(nb, prec):
    """10 shared steps of 2^-10 (every particle on one level: a block step
    is a shared step) against oracle_hermite6_run from the same start."""
    cl = inputs.plummer(1024, seed=0)
    eps, L, steps = 1e-4, 10, 10
    p = nb.NB_FP64 if prec == "fp64" else nb.NB_MIXED
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=eps, precision=p, order=6, level_min=L,
                 level_max=L)
    t, m = sim.step(steps, report=True)
    s = sim.get_state()
    assert sim.status() == nb.NB_OK and m == 1024 and t == steps * sim.ticks(2.0 ** -L)
    sim.close()
    x, v = oracle.hermite6_run(cl.pos, cl.vel, cl.mass, eps, 2.0 ** -L, steps)
    tol = 1e-12 if prec == "fp64" else 1e-7
    ex = np.linalg.norm(s["pos"] - x, axis=1) / np.linalg.norm(x, axis=1)
    ev = np.linalg.norm(s["vel"] - v, axis=1) / np.linalg.norm(v, axis=1)
    assert ex.max() <= tol, ex.max()
    assert ev.max() <= 100 * tol, ev.max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hermite6_block_step_from_identical_state(nb, prec):
    """One block step from a set state with individual levels: the due
    particles (the finest level) against the oracle's 6th-order predictor,
    force with snap, corrector and criterion; the others untouched."""
    # eps = 1e-2 and steps no finer than 2^-12 keep the quintic's end
    # derivatives (crackle ~ differences of accelerations over t^3) well
    # above the FP64 rounding of their numerators, so that the criterion
    # and its level are reproducible
    cl = inputs.plummer(2048, seed=6, imf="kroupa")
    n, eps, T, lmin, lmax, eta = cl.n, 1e-2, 40, 3, 12, 0.01
    a0, j0, s0, c0 = synthetic_state(cl, eps, 9)
    lev0 = np.array([oracle.level(oracle.initial_dt(a0[i], j0[i], 0.01), -1, 0, T, lmin, lmax)
                     for i in range(n)], dtype=np.int32)
    p = nb.NB_FP64 if prec == "fp64" else nb.NB_MIXED
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=eps, precision=p, order=6, level_min=lmin,
                 level_max=lmax, graph_steps=0)
    sim.set_state(cl.pos, cl.vel, a0, j0, np.zeros(n, dtype=np.int64), lev0)
    sim.set_derivs(s0, c0)
    t_next, m = sim.step(1, report=True)
    st = sim.get_state()
    s1_gpu, c1_gpu = sim.get_derivs()
    assert sim.status() == nb.NB_OK
    sim.close()

    Lf = lev0.max()
    assert t_next == 1 << (T - Lf)
    due = lev0 == Lf
    assert m == int(due.sum())
    idle = np.flatnonzero(~due)
    for key, ref in (("pos", cl.pos), ("vel", cl.vel), ("acc", a0), ("jerk", j0)):
        assert np.array_equal(st[key][idle], ref[idle]), key
    assert np.array_equal(s1_gpu[idle], s0[idle]) and np.array_equal(c1_gpu[idle], c0[idle])

    tau = 2.0 ** -Lf
    xp, vp, ap = oracle.hermite6_predict(tau, cl.pos, cl.vel, a0, j0, s0, c0)
    sample = np.flatnonzero(due)[:256]
    ra, rj, rs = oracle.force_snap(xp, vp, ap, cl.mass, eps, idx=sample.astype(np.int64))
    ga, gj, gs = st["acc"][sample], st["jerk"][sample], s1_gpu[sample]
    if prec == "fp64":
        assert rel_err(ga, ra).max() <= 1e-12
        assert rel_err(gj, rj).max() <= 1e-12
        assert rel_err(gs, rs).max() <= 1e-11
    else:
        S = snap_term_sums(xp, vp, ap, cl.mass, eps, sample)
        assert (np.linalg.norm(ga - ra, axis=1) / S[:, 0]).max() <= 1e-6
        assert (np.linalg.norm(gj - rj, axis=1) / S[:, 1]).max() <= 3e-6
        assert (np.linalg.norm(gs - rs, axis=1) / S[:, 2]).max() <= 2e-5
    # the corrector and criterion on the GPU's own force: both sides then
    # apply the same formulas to the same inputs, up to FP64 rounding
    x1, v1, cr, po, a5 = oracle.hermite6_correct(tau, cl.pos[sample], cl.vel[sample],
                                                 a0[sample], j0[sample], s0[sample],
                                                 ga, gj, gs)
    nrm = lambda v: np.linalg.norm(v, axis=1)
    tolx = 1e-14 * (nrm(cl.pos[sample]) + tau * nrm(cl.vel[sample]) + tau ** 2 * nrm(a0[sample]))
    tolv = 1e-14 * (nrm(cl.vel[sample]) + tau * (nrm(a0[sample]) + nrm(ga)))
    assert np.all(nrm(st["pos"][sample] - x1) <= tolx + 1e-15)
    assert np.all(nrm(st["vel"][sample] - v1) <= tolv + 1e-15)
    # crackle = (60 D - t (24 j0 + 36 j1) - t^2 (3 s0 - 9 s1)) / t^3: its
    # rounding is relative to the magnitudes of the numerator's terms
    mag = (60 * (nrm(ga) + nrm(a0[sample])) + tau * (24 * nrm(j0[sample]) + 36 * nrm(gj))
           + tau ** 2 * (3 * nrm(s0[sample]) + 9 * nrm(gs))) / tau ** 3
    assert np.all(nrm(c1_gpu[sample] - cr) <= 64 * 2.0 ** -52 * mag)
    assert np.all(st["t"][sample] == t_next)
    dtc = np.array([oracle.hermite6_dt(ga[r], gj[r], gs[r], cr[r], po[r], a5[r], eta)
                    for r in range(len(sample))])
    lev_ref = np.array([oracle.level(dtc[r], int(lev0[i]), int(t_next), T, lmin, lmax)
                        for r, i in enumerate(sample)])
    e = np.log2(dtc)
    near_edge = np.abs(e - np.round(e)) < 1e-3
    got = st["level"][sample]
    assert np.array_equal(got[~near_edge], lev_ref[~near_edge])
    assert np.all(np.abs(got[near_edge] - lev_ref[near_edge]) <= 1)
