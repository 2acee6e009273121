"""Degenerate inputs of the method, GPU (through the C ABI) against the FP64
CPU oracle, in FP64 and in mixed precision:

  * coincident particles (distinct indices, one position, eps > 0): Eq. 1
    excludes only j == i, so the partner adds nothing to the acceleration
    (d = 0), -m/eps to the potential and m w / eps^3 to the jerk;
  * a lone particle: no force; a block step moves it in a straight line;
  * massless test particles: they feel the cluster and exert nothing;
  * a cluster far from the origin (|x| ~ 2e3, internal scale ~ 1): the
    double-single offsets keep the separations' resolution, which plain FP32
    positions would lose (~1e-4 relative).  Velocities stay in the centre-
    of-mass frame: the mixed path stores them as FP32 values, so a large
    bulk velocity would limit the jerk's accuracy instead.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1411_5234_gb300 import inputs

from test_gpu_parity import check_mixed, gpu_force, rel_err, term_sums

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]


def _prec(nb, name):
    return nb.NB_FP64 if name == "fp64" else nb.NB_MIXED


def _compare(nb, cl, eps, idx, prec):
    a, j, p = gpu_force(nb, cl, eps, idx, _prec(nb, prec))
    ra, rj, rp = oracle.force(cl.pos, cl.vel, cl.mass, eps, idx=np.asarray(idx, dtype=np.int64))
    if prec == "fp64":
        assert rel_err(a, ra).max() <= 1e-12
        assert rel_err(j, rj).max() <= 1e-12
        assert np.abs(p / rp - 1).max() <= 1e-12
    else:
        check_mixed(a, j, ra, rj, *term_sums(cl, eps, idx))
        assert np.abs(p / rp - 1).max() <= 1e-6


@pytest.mark.parametrize("prec", PRECS)
def test_coincident_particles(nb, prec):
    """FP64: the oracle's values.  Mixed: every other particle meets the
    mixed gates; the coincident pair's separation is zero only to the
    double-single resolution, ~2^-47 of the offsets from the cell centre
    (below the cluster's extent R), which the softened pair force turns into
    at most G m 2^-46 R / eps^3 of spurious acceleration."""
    eps = 1e-4
    cl = inputs.plummer(256, seed=11)
    pos, vel = cl.pos.copy(), cl.vel.copy()
    pos[1] = pos[0]
    vel[1] = vel[0] + np.array([0.3, -0.2, 0.1])
    c2 = inputs.Cluster(pos, vel, cl.mass, cl.offsets)
    idx = np.arange(256)
    if prec == "fp64":
        _compare(nb, c2, eps, idx, prec)
        return
    a, j, p = gpu_force(nb, c2, eps, idx, nb.NB_MIXED)
    ra, rj, rp = oracle.force(pos, vel, cl.mass, eps, idx=idx)
    Sa, Sj = term_sums(c2, eps, idx)
    rest = idx[2:]
    check_mixed(a[rest], j[rest], ra[rest], rj[rest], Sa[rest], Sj[rest])
    pair = idx[:2]
    R = np.linalg.norm(pos - pos.mean(0), axis=1).max()
    bound = 1e-6 * Sa[pair] + cl.mass[1 - pair] * 2.0 ** -46 * R / eps ** 3
    assert np.all(np.linalg.norm(a[pair] - ra[pair], axis=1) <= bound)
    assert np.all(np.linalg.norm(j[pair] - rj[pair], axis=1) / Sj[pair] <= 3e-6)
    assert np.abs(p / rp - 1).max() <= 1e-6


@pytest.mark.parametrize("prec", PRECS)
def test_lone_particle(nb, prec):
    pos = np.array([[0.3, -0.2, 0.1]])
    vel = np.array([[0.5, 0.25, -0.125]])
    mass = np.array([1.0])
    sim = nb.Sim(pos, vel, mass, eps=1e-4, precision=_prec(nb, prec), level_min=4, level_max=20)
    try:
        sim.predict(0)
        a, j, p = sim.force(torch.zeros(1, dtype=torch.int32, device="cuda"))
        torch.cuda.synchronize()
        assert not a.any() and not j.any() and not p.any()
        sim.step(1)
        s = sim.get_state()
        assert sim.status() == nb.NB_OK
    finally:
        sim.close()
    st = oracle.State(pos, vel, mass, eps=1e-4, lmin=4, lmax=20)
    st.block_step()
    assert np.array_equal(s["t"], st.t) and np.array_equal(s["level"], st.level)
    assert np.allclose(s["pos"], st.pos, rtol=0, atol=1e-15)
    assert np.array_equal(s["vel"], vel)


@pytest.mark.parametrize("prec", PRECS)
def test_massless_test_particles(nb, prec):
    cl = inputs.plummer(1024, seed=12)
    mass = cl.mass.copy()
    mass[::16] = 0.0
    c2 = inputs.Cluster(cl.pos, cl.vel, mass, cl.offsets)
    _compare(nb, c2, 1e-4, np.arange(1024), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_cluster_far_from_origin(nb, prec):
    cl = inputs.plummer(2048, seed=13)
    pos = cl.pos + np.array([1.0e3, -2.0e3, 5.0e2])
    c2 = inputs.Cluster(pos, cl.vel, cl.mass, cl.offsets)
    _compare(nb, c2, 1e-4, np.arange(2048), prec)
