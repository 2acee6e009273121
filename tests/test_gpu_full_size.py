"""GPU parity at the benchmark's full size: Plummer N = 2^20 with Kroupa
masses, eps = 1e-4, in the launch configuration bench.py times (mixed
precision, autotuned kernel shape, every particle on the shared level 10,
direct launches), checked against the FP64 CPU oracle on sampled outputs that
the oracle computes one by one.

The step starts from seeded synthetic accelerations and jerks set through
nb_set_state, so the oracle's inputs never come from the GPU: both sides
predict all N particles from the same state, evaluate the force at the
predicted positions and correct.  Per sampled particle:
  * acceleration and jerk after the step (the force at the predicted
    positions) against the oracle's force, with the mixed-precision gates of
    test_gpu_parity;
  * position and velocity after the corrector within the error that the
    force error itself explains.  The 4th-order Hermite corrector is linear in
    (a1, j1), with dx1/da1 = 0.15 tau^2, dx1/dj1 = -tau^3 / 30,
    dv1/da1 = tau / 2, dv1/dj1 = -tau^2 / 12 (from the cubic Hermite fit of
    Sec. 2 item 1), plus FP64 rounding of the Taylor terms;
  * time and level exactly.
The FP64 path is checked at the same size on 1024 random targets of nb_force
with the 1e-12 per-particle gate.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1411_5234_gb300 import inputs

from test_gpu_parity import check_mixed, rel_err

pytestmark = pytest.mark.gpu

N = 1 << 20
EPS = 1e-4
LEVEL = 10


@pytest.fixture(scope="module")
def cluster():
    return inputs.plummer(N, seed=0, imf="kroupa")


def term_sums_big(pos, vel, mass, eps, idx, chunk=8):
    """sum_j |a_ij| and sum_j |jerk_ij| per target, in chunks small enough
    for N = 2^20 sources."""
    Sa = np.empty(len(idx))
    Sj = np.empty(len(idx))
    for c0 in range(0, len(idx), chunk):
        ii = np.asarray(idx[c0:c0 + chunk])
        d = pos[None, :, :] - pos[ii, None, :]
        w = vel[None, :, :] - vel[ii, None, :]
        r = np.sqrt((d * d).sum(2))
        s2 = r * r + eps * eps
        s2[np.arange(len(ii)), ii] = np.inf
        inv3 = s2 ** -1.5
        Sa[c0:c0 + chunk] = (mass[None, :] * r * inv3).sum(1)
        dw = np.abs((d * w).sum(2))
        Sj[c0:c0 + chunk] = (mass[None, :] * (np.sqrt((w * w).sum(2)) * inv3
                                             + 3 * dw * r * inv3 / s2)).sum(1)
    return Sa, Sj


def test_full_size_block_step_sampled(nb, cluster):
    cl = cluster
    a0 = inputs.random_vectors(N, 2.0, seed=11)
    j0 = inputs.random_vectors(N, 20.0, seed=12)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=EPS, precision=nb.NB_MIXED,
                 level_min=LEVEL, level_max=LEVEL, graph_steps=0)
    try:
        sim.autotune()
        sim.set_state(cl.pos, cl.vel, a0, j0, np.zeros(N, dtype=np.int64),
                      np.full(N, LEVEL, dtype=np.int32))
        sim.step(1)
        s = sim.get_state()
        pos1, vel1, acc1, jerk1, t1, lev1 = (s[k] for k in ("pos", "vel", "acc", "jerk", "t",
                                                            "level"))
        assert sim.status() == nb.NB_OK
        variant = sim.cfg.variant
    finally:
        sim.close()

    tau = 2.0 ** -LEVEL
    assert np.all(t1 == sim.ticks(tau)), "every particle advances by one step"
    assert np.all(lev1 == LEVEL)

    sample = inputs.random_active(N, 128, seed=7).astype(np.int64)
    xp, vp = oracle.predict(cl.pos, cl.vel, a0, j0, tau)
    ra, rj, _ = oracle.force(xp, vp, cl.mass, EPS, idx=sample)
    Sa, Sj = term_sums_big(xp, vp, cl.mass, EPS, sample)
    check_mixed(acc1[sample], jerk1[sample], ra, rj, Sa, Sj)

    x1, v1, _, _ = oracle.correct(tau, xp[sample], vp[sample], a0[sample], j0[sample], ra, rj)
    da = np.linalg.norm(acc1[sample] - ra, axis=1)
    dj = np.linalg.norm(jerk1[sample] - rj, axis=1)
    nrm = lambda v: np.linalg.norm(v, axis=1)
    amag = nrm(a0[sample]) + nrm(ra)
    jmag = nrm(j0[sample]) + nrm(rj)
    taylor_x = nrm(cl.pos[sample]) + nrm(cl.vel[sample]) * tau + amag * tau ** 2 + jmag * tau ** 3
    taylor_v = nrm(cl.vel[sample]) + amag * tau + jmag * tau ** 2
    tol_x = 1.01 * (0.15 * tau ** 2 * da + tau ** 3 / 30 * dj) + 8e-16 * taylor_x
    tol_v = 1.01 * (0.5 * tau * da + tau ** 2 / 12 * dj) + 8e-16 * taylor_v
    ex = np.linalg.norm(pos1[sample] - x1, axis=1)
    ev = np.linalg.norm(vel1[sample] - v1, axis=1)
    assert np.all(ex <= tol_x), (variant, float((ex / tol_x).max()))
    assert np.all(ev <= tol_v), (variant, float((ev / tol_v).max()))


def test_full_size_fp64_force_sampled(nb, cluster):
    cl = cluster
    idx = inputs.random_active(N, 1024, seed=5)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=EPS, precision=nb.NB_FP64)
    try:
        sim.predict(0)
        acc, jerk, pot = sim.force(torch.as_tensor(idx, device="cuda"))
        torch.cuda.synchronize()
        assert sim.status() == nb.NB_OK
        acc, jerk, pot = acc.cpu().numpy(), jerk.cpu().numpy(), pot.cpu().numpy()
    finally:
        sim.close()
    ra, rj, rp = oracle.force(cl.pos, cl.vel, cl.mass, EPS, idx=idx.astype(np.int64))
    assert rel_err(acc, ra).max() <= 1e-12
    assert rel_err(jerk, rj).max() <= 1e-12
    assert np.abs(pot / rp - 1).max() <= 1e-12
