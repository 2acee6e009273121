"""The seeded synthetic inputs follow their stated recipes (CPU only).

Plummer spheres in Henon units (centre-of-mass frame, E = -1/4 and virial
ratio 1/2 up to sampling noise, half-mass radius 0.769), Kroupa masses
(the share of bodies below the 0.5 break), primordial binaries (the pair
count, log-uniform semi-major axes in [1e-4, 1e-2], thermal eccentricities
with mean 2/3) and the batch of log-uniform cluster sizes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1411_5234_gb300 import inputs


def test_plummer_henon_units_and_frame():
    cl = inputs.plummer(4096, seed=0)
    assert cl.mass.sum() == pytest.approx(1.0, rel=1e-14)
    assert np.abs((cl.mass[:, None] * cl.pos).sum(0)).max() < 1e-14
    assert np.abs((cl.mass[:, None] * cl.vel).sum(0)).max() < 1e-14
    ek, ep = oracle.energy(cl.pos, cl.vel, cl.mass, 0.0)
    assert ek + ep == pytest.approx(-0.25, rel=0.05)
    assert ek / abs(ep) == pytest.approx(0.5, abs=0.03)


def test_plummer_half_mass_radius():
    # Henon units put the Plummer scale at 3 pi / 16; the half-mass radius of
    # the model (mass fraction cut at 0.999) is then 0.768
    cl = inputs.plummer(16384, seed=1)
    r = np.sort(np.linalg.norm(cl.pos, axis=1))
    a = 3 * math.pi / 16
    x = 0.5 * 0.999
    r_h = a / math.sqrt(x ** (-2.0 / 3.0) - 1.0)
    assert r[len(r) // 2] == pytest.approx(r_h, rel=0.03)


def test_kroupa_share_below_the_break():
    # dN/dm ~ m^-1.3 on [0.1, 0.5), m^-2.3 on [0.5, 100], continuous at 0.5
    low = (0.1 ** -0.3 - 0.5 ** -0.3) / 0.3
    high = 0.5 * (0.5 ** -1.3 - 100.0 ** -1.3) / 1.3
    share = low / (low + high)
    cl = inputs.plummer(16384, seed=2, imf="kroupa")
    m = cl.mass / cl.mass.min() * 0.1            # back to solar masses (min ~ 0.1)
    assert cl.mass.sum() == pytest.approx(1.0, rel=1e-14)
    assert np.mean(m < 0.5) == pytest.approx(share, abs=0.02)
    assert m.max() <= 100.0 * 1.02


def test_binaries_recipe():
    n = 20000
    cl = inputs.plummer_binaries(n, seed=0)
    nb = n // 20                                  # 10 % of the bodies in pairs
    ns = n - 2 * nb
    assert cl.n == n and np.allclose(cl.mass, 1.0 / n)
    r = cl.pos[ns + 1::2] - cl.pos[ns::2]
    w = cl.vel[ns + 1::2] - cl.vel[ns::2]
    mb = 2.0 / n
    E = 0.5 * (w * w).sum(1) - mb / np.linalg.norm(r, axis=1)
    a = -mb / (2 * E)
    h2 = (np.cross(r, w) ** 2).sum(1)
    e = np.sqrt(np.maximum(0.0, 1 + 2 * E * h2 / mb ** 2))
    assert len(a) == nb
    assert a.min() >= 1e-4 * (1 - 1e-9) and a.max() <= 1e-2 * (1 + 1e-9)
    assert np.mean(np.log10(a)) == pytest.approx(-3.0, abs=0.1)   # log-uniform
    assert np.mean(e) == pytest.approx(2.0 / 3.0, abs=0.03)       # f(e) = 2e
    # the pairs' centres of mass form the Plummer body set with the singles
    com = 0.5 * (cl.pos[ns::2] + cl.pos[ns + 1::2])
    allpos = np.vstack([cl.pos[:ns], com])
    m_sys = np.concatenate([np.full(ns, 1.0 / n), np.full(nb, 2.0 / n)])
    assert np.abs((m_sys[:, None] * allpos).sum(0)).max() < 1e-12


def test_batch_sizes_log_uniform():
    sizes = inputs.batch_sizes(512, 256, 16384, seed0=0)
    assert sizes.min() >= 256 and sizes.max() <= 16384
    assert int(sizes.sum()) == 2007990
    assert float((sizes.astype(float) ** 2).sum()) == pytest.approx(1.7e10, rel=0.05)
    assert np.mean(np.log(sizes)) == pytest.approx(0.5 * (math.log(256) + math.log(16384)),
                                                   abs=0.2)
    cl = inputs.plummer_batch(8, 256, 1024, seed0=3)
    assert np.array_equal(np.diff(cl.offsets), inputs.batch_sizes(8, 256, 1024, seed0=3))


def test_random_active_is_a_sorted_subset():
    idx = inputs.random_active(1000, 137, seed=5)
    assert len(idx) == 137 and np.all(np.diff(idx) > 0)
    assert idx.min() >= 0 and idx.max() < 1000 and idx.dtype == np.int32
    assert np.array_equal(inputs.random_active(50, 50), np.arange(50))
