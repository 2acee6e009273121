"""GPU parity: libnbody_gb300 (through its C ABI) against the FP64 CPU oracle.

Tolerances:
  * FP64 path: per-particle relative error ||a_gpu - a_ref|| / ||a_ref|| and the
    same for the jerk <= 1e-12 (both sides FP64; the GPU sums in a different
    order and uses CUDA's rsqrt, so agreement is to a few ulps times the
    conditioning sum|terms| / |sum|).
  * mixed path: FP32 pair arithmetic (24-bit mantissa, hardware rsqrt with
    ~2^-22.9 relative error) on separations accurate to a few ulp: every
    term carries a relative error of a few 2^-24, so the error of a sum is
    bounded by that times sum_j |term_j|, not times |sum|.  Worst case per
    term: the separation carries <= 4 ulp (far cells), which the direction
    and the cube of the length turn into <= 16 ulp of m d / s^3, plus ~3 ulp
    from rsqrt^3 and the products: ~22 ulp = 1.3e-6.  Gated per particle on
    the condition-scaled error ||da_i|| / sum_j |a_ij| <= 1e-6 (jerk, with its
    own terms and more products: <= 3e-6), plus, for samples of >= 100
    targets, the plain relative error's median <= 1e-7 and, for >= 1000
    targets, its 99.9th percentile <= 1e-6 for the acceleration (jerk:
    median <= 5e-7, 99.9th percentile <= 4e-6).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1411_5234_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel_err(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


def term_sums(cl, eps, idx, G=1.0):
    """sum_j |a_ij| and sum_j |jerk_ij| (component-wise norms) per target."""
    idx = np.asarray(idx)
    Sa = np.empty(len(idx))
    Sj = np.empty(len(idx))
    for c0 in range(0, len(idx), 256):
        ii = idx[c0:c0 + 256]
        d = cl.pos[None, :, :] - cl.pos[ii, None, :]
        w = cl.vel[None, :, :] - cl.vel[ii, None, :]
        s2 = (d * d).sum(2) + eps * eps
        s2[np.arange(len(ii)), ii] = np.inf            # j == i excluded
        inv3 = s2 ** -1.5
        m = G * cl.mass[None, :]
        Sa[c0:c0 + 256] = (m * np.sqrt((d * d).sum(2)) * inv3).sum(1)
        dw = np.abs((d * w).sum(2))
        Sj[c0:c0 + 256] = (m * (np.sqrt((w * w).sum(2)) * inv3
                               + 3 * dw * np.sqrt((d * d).sum(2)) * inv3 / s2)).sum(1)
    return Sa, Sj


def check_mixed(a, j, ra, rj, Sa, Sj, p999_min=1000):
    """The mixed path's gates: every particle's error relative to the sum of
    its pair magnitudes, and the plain relative error's median and 99.9th
    percentile over a population of at least p999_min targets."""
    ea, ej = rel_err(a, ra), rel_err(j, rj)
    ca = np.linalg.norm(a - ra, axis=1) / Sa
    cj = np.linalg.norm(j - rj, axis=1) / Sj
    assert ca.max() <= 1e-6, ca.max()
    assert cj.max() <= 3e-6, cj.max()
    if len(ea) >= 100:      # distribution gates need a population
        assert np.median(ea) <= 1e-7 and np.median(ej) <= 5e-7, (np.median(ea), np.median(ej))
    if len(ea) >= p999_min:
        assert np.quantile(ea, 0.999) <= 1e-6, np.quantile(ea, 0.999)
        assert np.quantile(ej, 0.999) <= 4e-6, np.quantile(ej, 0.999)


def gpu_force(nb, cl, eps, idx, prec, bfactor=0, G=1.0):
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, offsets=cl.offsets, eps=eps, precision=prec,
                 bfactor=bfactor, G=G)
    act = torch.as_tensor(np.asarray(idx, dtype=np.int32), device="cuda")
    sim.predict(0)
    acc, jerk, pot = sim.force(act)
    torch.cuda.synchronize()
    assert sim.status() == nb.NB_OK
    out = acc.cpu().numpy(), jerk.cpu().numpy(), pot.cpu().numpy()
    sim.close()
    return out


@pytest.fixture(scope="module")
def plummer1024():
    return inputs.plummer(1024, seed=0)


# ------------------------------------------------------------ forces ----

def test_fp64_force_config1(nb, plummer1024):
    cl = plummer1024
    idx = np.arange(cl.n)
    a, j, p = gpu_force(nb, cl, 1e-4, idx, nb.NB_FP64)
    ra, rj, rp = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4)
    assert rel_err(a, ra).max() <= 1e-12
    assert rel_err(j, rj).max() <= 1e-12
    assert np.abs(p / rp - 1).max() <= 1e-13


@pytest.mark.parametrize("n", [1000, 1027, 130])
@pytest.mark.parametrize("m", [1, 31, 33, 257, "all"])
@pytest.mark.parametrize("bfactor", [0, 1, 3])
def test_fp64_force_ragged_subsets(nb, n, m, bfactor):
    cl = inputs.plummer(n, seed=n, imf="kroupa")
    mm = n if m == "all" else min(m, n)
    idx = inputs.random_active(n, mm, seed=mm)
    a, j, p = gpu_force(nb, cl, 1e-3, idx, nb.NB_FP64, bfactor)
    ra, rj, rp = oracle.force(cl.pos, cl.vel, cl.mass, 1e-3, idx=idx)
    assert rel_err(a, ra).max() <= 1e-12
    assert rel_err(j, rj).max() <= 1e-12
    assert np.abs(p / rp - 1).max() <= 1e-13


@pytest.mark.parametrize("n,m", [(4099, "all"), (4099, 1), (4099, 333), (129, "all")])
def test_mixed_force_parity(nb, n, m):
    cl = inputs.plummer(n, seed=7, imf="kroupa")
    mm = n if m == "all" else m
    idx = inputs.random_active(n, mm, seed=3)
    a, j, p = gpu_force(nb, cl, 1e-4, idx, nb.NB_MIXED)
    ra, rj, rp = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=idx)
    check_mixed(a, j, ra, rj, *term_sums(cl, 1e-4, idx))
    assert np.abs(p / rp - 1).max() <= 1e-6


def test_mixed_close_binary_resolution(nb):
    # A hard binary (separation 1e-6) far from the origin (|x| ~ 1): plain
    # FP32 positions would resolve the separation to ~6%; the double-single
    # separation keeps the pair force to FP32 accuracy.
    cl = inputs.plummer(256, seed=2)
    pos = cl.pos.copy()
    pos[1] = pos[0] + np.array([1e-6, 0.0, 0.0])
    c2 = inputs.Cluster(pos, cl.vel, cl.mass, cl.offsets)
    a, _, _ = gpu_force(nb, c2, 0.0, [0, 1], nb.NB_MIXED)
    ra, _, _ = oracle.force(pos, cl.vel, cl.mass, 0.0, idx=[0, 1])
    assert rel_err(a, ra).max() <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_two_body_exact_values(nb, prec):
    # d = 3, eps = 4: |a| = G m 3 / 125, phi = -G m / 5
    P = nb.NB_FP64 if prec == "fp64" else nb.NB_MIXED
    tol = 1e-15 if prec == "fp64" else 3e-7
    pos = np.array([[0.0, 0, 0], [3.0, 0, 0]])
    cl = inputs.Cluster(pos, np.zeros((2, 3)), np.array([2.0, 5.0]), np.array([0, 2]))
    a, j, p = gpu_force(nb, cl, 4.0, [0, 1], P, G=1.5)
    np.testing.assert_allclose(a, [[1.5 * 5 * 3 / 125, 0, 0], [-1.5 * 2 * 3 / 125, 0, 0]],
                               rtol=tol, atol=1e-18)
    np.testing.assert_allclose(p, [-1.5 * 5 / 5, -1.5 * 2 / 5], rtol=tol)
    assert np.all(j == 0.0)


def test_bfactor_invariance(nb):
    cl = inputs.plummer(3000, seed=5, imf="kroupa")
    idx = inputs.random_active(3000, 200, seed=1)
    ref = gpu_force(nb, cl, 1e-4, idx, nb.NB_FP64, 1)
    for b in (2, 5, 16):
        got = gpu_force(nb, cl, 1e-4, idx, nb.NB_FP64, b)
        for x, r in zip(got[:2], ref[:2]):
            assert rel_err(x, r).max() <= 1e-14
    refm = gpu_force(nb, cl, 1e-4, idx, nb.NB_MIXED, 1)
    for b in (2, 5, 16):
        got = gpu_force(nb, cl, 1e-4, idx, nb.NB_MIXED, b)
        for x, r in zip(got[:2], refm[:2]):
            assert rel_err(x, r).max() <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_target_order_is_free(nb, prec):
    # rows follow the caller's list whatever its order; values do not depend
    # on it beyond the summation order inside the kernel (identical here)
    P = nb.NB_FP64 if prec == "fp64" else nb.NB_MIXED
    cl = inputs.plummer(3001, seed=31, imf="kroupa")
    idx = inputs.random_active(3001, 700, seed=2)
    perm = np.random.default_rng(0).permutation(700)
    a1, j1, p1 = gpu_force(nb, cl, 1e-4, idx, P)
    a2, j2, p2 = gpu_force(nb, cl, 1e-4, idx[perm], P)
    assert np.array_equal(a2, a1[perm]) and np.array_equal(j2, j1[perm])
    assert np.array_equal(p2, p1[perm])


def test_force_empty_and_invalid_lists(nb, plummer1024):
    cl = plummer1024
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nb.NB_FP64)
    sim.predict(0)
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    sim.force(empty)
    assert sim.status() == nb.NB_OK
    rep = torch.tensor([5, 3, 9, 3], dtype=torch.int32, device="cuda")  # repeated entry
    sim.force(rep)
    assert sim.status() == nb.NB_EINVAL
    sim.clear_status()
    oob = torch.tensor([1, 2, 5000], dtype=torch.int32, device="cuda")
    sim.force(oob)
    assert sim.status() == nb.NB_EINVAL
    sim.close()


# ------------------------------------------------------------- integrator ---

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_shared_steps_config1(nb, plummer1024, prec):
    # Plummer N = 1024, eps = 1e-4: 10 shared Hermite-4 steps of 2^-10
    cl = plummer1024
    P = nb.NB_FP64 if prec == "fp64" else nb.NB_MIXED
    st = oracle.State(cl.pos, cl.vel, cl.mass, eps=1e-4, lmin=10, lmax=10)
    for _ in range(10):
        st.block_step()
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=P, level_min=10, level_max=10,
                 graph_steps=4)
    sim.step(10)
    s = sim.get_state()
    assert sim.status() == nb.NB_OK
    assert np.array_equal(s["t"], st.t) and np.all(s["t"] == 10 << (40 - 10))
    tol = 1e-12 if prec == "fp64" else 1e-7
    assert rel_err(s["pos"], st.pos).max() <= tol
    assert rel_err(s["vel"], st.vel).max() <= tol * 10
    assert rel_err(s["acc"], st.acc).max() <= (1e-12 if prec == "fp64" else 1e-5)
    assert sim.stats().block_steps == 10
    assert sim.stats().interactions == 10 * 1024 * 1024
    sim.close()


def test_block_step_from_identical_state(nb):
    cl = inputs.plummer(700, seed=4)
    st = oracle.State(cl.pos, cl.vel, cl.mass, eps=1e-3, eta=0.01, lmin=3, lmax=20)
    for _ in range(5):
        st.block_step()
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-3, precision=nb.NB_FP64, eta=0.01,
                 level_min=3, level_max=20, graph_steps=0)
    sim.set_state(st.pos, st.vel, st.acc, st.jerk, st.t, st.level)
    for _ in range(3):
        before_level = st.level.copy()
        t_next, act, dtc = st.block_step()
        sim.step(1)
        s = sim.get_state()
        assert sim.status() == nb.NB_OK
        assert np.array_equal(s["t"], st.t)           # same active set, same times
        assert rel_err(s["pos"][act], st.pos[act]).max() <= 1e-12
        assert rel_err(s["vel"][act], st.vel[act]).max() <= 1e-11
        # a level may differ only where the criterion sits on a power of two
        diff = np.flatnonzero(s["level"][act] != st.level[act])
        for k in diff:
            frac = math.log2(dtc[k]) - math.floor(math.log2(dtc[k]))
            assert min(frac, 1 - frac) < 1e-9, (k, dtc[k], before_level[act[k]])
        sim.set_state(st.pos, st.vel, st.acc, st.jerk, st.t, st.level)
    sim.close()


def test_block_integration_energy_drift(nb):
    # Plummer N = 512, eps = 1e-3, levels 2^-3 .. 2^-20, t = 0 -> 1/8.  The
    # Hermite truncation error makes the energy drift; the FP64 path must
    # drift like the oracle running the same integrator, and the mixed path
    # within 2x of the FP64 path.
    cl = inputs.plummer(512, seed=8)
    eps, t_end = 1e-3, 0.125
    st = oracle.State(cl.pos, cl.vel, cl.mass, eps=eps, lmin=3, lmax=20)
    e_ref0 = sum(oracle.energy(cl.pos, cl.vel, cl.mass, eps))
    while st.time() < t_end:
        st.block_step()
    assert np.all(st.t == st.t[0])
    d_ref = sum(oracle.energy(st.pos, st.vel, st.mass, eps)) / e_ref0 - 1
    drift = {}
    for P in (nb.NB_FP64, nb.NB_MIXED):
        sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=eps, precision=P, level_min=3, level_max=20)
        e0 = sum(sim.energy())
        assert abs(e0 / e_ref0 - 1) < 1e-12
        sim.set_end_time(sim.ticks(t_end))
        for _ in range(200):
            sim.step(256)
            if sim.stats().t_min == sim.ticks(t_end):
                break
        stats = sim.stats()
        assert stats.t_min == stats.t_max == sim.ticks(t_end)
        s = sim.get_state()
        assert np.all(s["t"] == sim.ticks(t_end))
        drift[P] = sum(sim.energy()) / e0 - 1
        assert sim.status() == nb.NB_OK
        sim.close()
    assert abs(d_ref) < 1e-5
    assert abs(drift[nb.NB_FP64] - d_ref) <= 0.05 * abs(d_ref) + 1e-9, (drift, d_ref)
    assert abs(drift[nb.NB_MIXED]) <= 2 * abs(drift[nb.NB_FP64]) + 1e-9, (drift, d_ref)


def test_step_block_reports_time_and_active_count(nb, plummer1024):
    """nb_step_block's outputs: the block time after the last step and the
    number of particles that step corrected, against the state read back."""
    cl = plummer1024
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, level_min=8, level_max=8)
    t, m = sim.step(3, report=True)
    assert t == 3 * sim.ticks(2.0 ** -8) and m == 1024
    sim.close()
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, level_min=3, level_max=14)
    sim.step(5)
    before = sim.get_state()["t"]
    t, m = sim.step(1, report=True)
    after = sim.get_state()["t"]
    assert m == int((after != before).sum()) and m > 0
    stepped = after != before
    assert np.all(after[stepped] == t) and np.all(after <= t)
    assert sim.step(0, report=True) == (t, 0)
    sim.close()


def test_graphs_match_direct_launches(nb):
    cl = inputs.plummer(600, seed=9)
    out = []
    for g in (0, 5):
        sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-3, precision=nb.NB_MIXED, level_min=3,
                     level_max=20, graph_steps=g)
        sim.step(23)
        out.append(sim.get_state())
        sim.close()
    for k in ("pos", "vel", "t", "level"):
        assert np.array_equal(out[0][k], out[1][k]), k


def test_checkpoint_resume_bitwise(nb):
    cl = inputs.plummer(400, seed=10)
    kw = dict(eps=1e-3, precision=nb.NB_FP64, level_min=3, level_max=20)
    a = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    a.step(40)
    ref = a.get_state()
    b = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    b.step(20)
    mid = b.get_state()
    b.close()
    c = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    c.set_state(mid["pos"], mid["vel"], mid["acc"], mid["jerk"], mid["t"], mid["level"])
    c.step(20)
    got = c.get_state()
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k
    a.close()
    c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_clusters_alone(nb, prec):
    P = nb.NB_FP64 if prec == "fp64" else nb.NB_MIXED
    parts = [inputs.plummer(n, seed=s) for n, s in ((300, 1), (517, 2), (64, 3))]
    pos = np.concatenate([p.pos for p in parts])
    vel = np.concatenate([p.vel for p in parts])
    mass = np.concatenate([p.mass for p in parts])
    off = np.array([0, 300, 817, 881])
    kw = dict(eps=1e-3, precision=P, level_min=3, level_max=20, bfactor=1)
    batch = nb.Sim(pos, vel, mass, offsets=off, **kw)
    batch.step(30)
    sb = batch.get_state()
    for k, p in enumerate(parts):
        alone = nb.Sim(p.pos, p.vel, p.mass, **kw)
        alone.step(30)
        sa = alone.get_state()
        for key in ("pos", "vel", "acc", "jerk", "t", "level"):
            assert np.array_equal(sa[key], sb[key][off[k]:off[k + 1]]), (k, key)
        ek, ep = batch.energy(k)
        ea = alone.energy()
        assert ek == pytest.approx(ea[0], rel=1e-14) and ep == pytest.approx(ea[1], rel=1e-13)
        alone.close()
    batch.close()


def test_energy_matches_oracle(nb):
    cl = inputs.plummer_batch(3, 100, 400, seed0=5)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, offsets=cl.offsets, eps=1e-4, precision=nb.NB_MIXED)
    tot = [0.0, 0.0]
    for k in range(3):
        lo, hi = cl.offsets[k], cl.offsets[k + 1]
        ek, ep = sim.energy(k)
        rk, rp = oracle.energy(cl.pos[lo:hi], cl.vel[lo:hi], cl.mass[lo:hi], 1e-4)
        assert ek == pytest.approx(rk, rel=1e-13) and ep == pytest.approx(rp, rel=1e-12)
        tot[0] += rk
        tot[1] += rp
    ek, ep = sim.energy(-1)
    assert ek == pytest.approx(tot[0], rel=1e-13) and ep == pytest.approx(tot[1], rel=1e-12)
    eks, eps_ = sim.energies()                    # all clusters from one evaluation
    for k in range(3):
        assert (eks[k], eps_[k]) == sim.energy(k)
    sim.close()


def test_invalid_arguments(nb):
    cl = inputs.plummer(64, seed=0)
    with pytest.raises(nb.NBError) as e:
        nb.Sim(cl.pos, cl.vel, -cl.mass)
    assert e.value.code == nb.NB_EINVAL
    with pytest.raises(nb.NBError):
        nb.Sim(cl.pos, cl.vel, cl.mass, offsets=np.array([0, 40, 40, 64]))
    bad_pos = cl.pos.copy()
    bad_pos[3, 1] = np.nan
    with pytest.raises(nb.NBError):
        nb.Sim(bad_pos, cl.vel, cl.mass)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, precision=nb.NB_FP64, level_min=3, level_max=10)
    s = sim.get_state()
    lv = s["level"].copy()
    lv[0] = 11
    with pytest.raises(nb.NBError):
        sim.set_state(s["pos"], s["vel"], s["acc"], s["jerk"], s["t"], lv)
    # a correction must move forward in time
    act = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    a = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    sim.correct(0, act, a, a)
    assert sim.status() == nb.NB_EINVAL
    sim.close()


def test_autotune_picks_a_shape_and_keeps_results(nb, tmp_path):
    cl = inputs.plummer(6000, seed=41, imf="kroupa")
    idx = inputs.random_active(6000, 1500, seed=2)
    act = torch.as_tensor(idx, device="cuda")
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nb.NB_MIXED, graph_steps=4)
    sim.predict(0)
    a0, j0, _ = (x.cpu().numpy() for x in sim.force(act))
    cache = str(tmp_path / "tune.txt")
    v, ms = sim.autotune(cache)
    assert 0 <= v < nb.MIXED_VARIANTS
    assert all(t > 0 for t in ms[0][:3])                  # every shape timed at the first points
    tv, tb = sim.tune_table()
    assert np.all((tv >= 0) & (tv < nb.MIXED_VARIANTS)) and np.all(tb >= 0)
    assert tv[13] == v                                    # ceil(log2 6000) = 13
    sim.predict(0)
    a1, j1, _ = (x.cpu().numpy() for x in sim.force(act))
    ra, rj, _ = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=idx)
    Sa, Sj = term_sums(cl, 1e-4, idx)
    check_mixed(a1, j1, ra, rj, Sa, Sj)
    check_mixed(a0, j0, ra, rj, Sa, Sj)
    sim.step(9)                                   # graphs rebuilt with the table's shapes
    assert sim.status() == nb.NB_OK
    sim.close()
    # a second context of the same problem class loads the table from the cache
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nb.NB_MIXED, graph_steps=4)
    v2, ms2 = sim.autotune(cache)
    tv2, tb2 = sim.tune_table()
    assert v2 == v and np.array_equal(tv2, tv) and np.array_equal(tb2, tb)
    assert all(t == 0 for row in ms2.values() for t in row)     # nothing measured
    sim.close()


@pytest.mark.parametrize("k", [0, 1, 3, 5])
def test_every_tabled_shape_and_split_meets_the_gates(nb, k):
    """Every (shape, i-split factor) the autotune table can hold gives
    forces within the parity gates, for m = N / 4^k targets of N = 16384.

    The 99.9th percentile of the plain relative error is gated on
    populations of 4000 targets or more: on fewer it is set by the two or
    three worst-conditioned particles (sum_j |a_ij| / |a_i| of 8-26 in this
    Kroupa sphere), whose error the condition-scaled gate bounds, and the
    two-tile shapes (FP32 runs of 128 terms per lane) then reach 1.03e-6 at
    m = 2048 while their condition-scaled error stays below 4.3e-7."""
    n = 16384
    cl = inputs.plummer(n, seed=43, imf="kroupa")
    m = max(64, n >> (2 * k))
    idx = inputs.random_active(n, m, seed=k)
    act = torch.as_tensor(idx, device="cuda")
    ra, rj, _ = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=idx)
    Sa, Sj = term_sums(cl, 1e-4, idx)
    for v in range(nb.MIXED_VARIANTS):
        for bf in (0, 1, 7):
            sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nb.NB_MIXED,
                         variant=v, bfactor=bf)
            sim.predict(0)
            a, j, _ = (x.cpu().numpy() for x in sim.force(act))
            assert sim.status() == nb.NB_OK
            sim.close()
            check_mixed(a, j, ra, rj, Sa, Sj, p999_min=4000)


def test_block_steps_with_a_table_of_several_shapes(nb, tmp_path):
    """Block steps whose plan picks the shape per step on the device (a
    table of several shapes, written as a cache file) agree with block steps
    of one fixed shape, to the mixed path's rounding."""
    cl = inputs.plummer(4096, seed=44)
    kw = dict(eps=1e-4, precision=nb.NB_MIXED, level_min=3, level_max=14, graph_steps=8)
    ref = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    ref.step(64)
    s_ref = ref.get_state()
    ref.close()
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    cache = tmp_path / "tune.txt"
    sim.autotune(str(cache))                       # measures and writes a line with its key
    line = cache.read_text().strip().splitlines()[-1]
    key, _ = line.split(" table=")
    # a table that changes shape with m: 7 (32 x 2) for m <= 2^6, 6 (64 x 2)
    # up to 2^9, 3 (32 x 4) up to 2^11, 0 above, with a forced split
    entries = []
    for b in range(nb.TUNE_BUCKETS):
        v = 7 if b <= 6 else 6 if b <= 9 else 3 if b <= 11 else 0
        entries.append(f"{v},{3 if b == 8 else 0}")
    cache.write_text(f"{key} table={';'.join(entries)}\n")
    sim.close()
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    sim.autotune(str(cache))
    tv, tb = sim.tune_table()
    assert tv[5] == 7 and tv[8] == 6 and tv[11] == 3 and tv[13] == 0 and tb[8] == 3
    m_seen = set()
    for _ in range(64):
        t, m = sim.step(1, report=True)
        m_seen.add((m - 1).bit_length() if m > 0 else 0)
    s = sim.get_state()
    assert sim.status() == nb.NB_OK
    sim.close()
    assert len({7 if b <= 6 else 6 if b <= 9 else 3 if b <= 11 else 0 for b in m_seen}) >= 2
    # the same steps captured in graphs of 8 (the plan picks the shape on the
    # device inside the graph) give the same state as the direct launches
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    sim.autotune(str(cache))
    sim.step(64)
    s_graph = sim.get_state()
    assert sim.status() == nb.NB_OK
    sim.close()
    for key in ("pos", "vel", "t", "level"):
        assert np.array_equal(s_graph[key], s[key]), key
    assert np.array_equal(s["t"], s_ref["t"])
    ex = np.linalg.norm(s["pos"] - s_ref["pos"], axis=1) / np.linalg.norm(s_ref["pos"], axis=1)
    assert ex.max() < 1e-9, ex.max()


# ------------------------------------------------- acceleration only ----

@pytest.mark.parametrize("n,m", [(4099, "all"), (20000, 999)])
def test_mixed_acceleration_only_parity(nb, n, m):
    """nb_force with jerk == NULL runs the kernel without velocity terms:
    acceleration and potential against the oracle with the mixed gates."""
    cl = inputs.plummer(n, seed=3, imf="kroupa")
    idx = np.arange(n) if m == "all" else inputs.random_active(n, m, seed=4)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nb.NB_MIXED)
    sim.predict(0)
    act = torch.as_tensor(np.asarray(idx, dtype=np.int32), device="cuda")
    acc, jerk, pot = sim.force(act, want_jerk=False)
    torch.cuda.synchronize()
    assert jerk is None and sim.status() == nb.NB_OK
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    sim.close()
    ra, rj, rp = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=np.asarray(idx, dtype=np.int64))
    Sa, Sj = term_sums(cl, 1e-4, idx)
    ca = np.linalg.norm(acc - ra, axis=1) / Sa
    assert ca.max() <= 1e-6, ca.max()
    ea = rel_err(acc, ra)
    assert np.median(ea) <= 1e-7, np.median(ea)
    assert np.abs(pot / rp - 1).max() <= 1e-6


def test_fp64_acceleration_only_equals_full(nb, plummer1024):
    """An FP64 context with jerk == NULL gives the same accelerations."""
    cl = plummer1024
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nb.NB_FP64)
    sim.predict(0)
    act = torch.as_tensor(inputs.random_active(cl.n, 300, seed=2), device="cuda")
    a1, _, p1 = sim.force(act)
    a2, j2, p2 = sim.force(act, want_jerk=False)
    torch.cuda.synchronize()
    assert j2 is None and sim.status() == nb.NB_OK
    assert torch.equal(a1, a2) and torch.equal(p1, p2)
    sim.close()


# ----------------------------------- separation modes (DS, plain FP32) ----

def test_ds_mode_parity(nb):
    """NB_DS (double-single separations for every source) meets the mixed
    gates, close binary included."""
    n = 4099
    cl = inputs.plummer(n, seed=7, imf="kroupa")
    idx = np.arange(n)
    a, j, p = gpu_force(nb, cl, 1e-4, idx, nb.NB_DS)
    ra, rj, rp = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=idx)
    check_mixed(a, j, ra, rj, *term_sums(cl, 1e-4, idx))
    assert np.abs(p / rp - 1).max() <= 1e-6
    c2 = inputs.plummer(256, seed=2)
    pos = c2.pos.copy()
    pos[1] = pos[0] + np.array([1e-6, 0.0, 0.0])
    c3 = inputs.Cluster(pos, c2.vel, c2.mass, c2.offsets)
    a, _, _ = gpu_force(nb, c3, 0.0, [0, 1], nb.NB_DS)
    ra, _, _ = oracle.force(pos, c2.vel, c2.mass, 0.0, idx=[0, 1])
    assert rel_err(a, ra).max() <= 1e-5


def test_fp32_mode_bounds(nb):
    """NB_FP32 (plain FP32 separations): on a Plummer sample its error stays
    within FP32 rounding relative to the cell size (condition-scaled 1e-4
    here); a hard binary is not resolved (the pair force is off by orders of
    magnitude more than in the mixed path), which is what the double-single
    separations of the mixed path are for."""
    n = 4099
    cl = inputs.plummer(n, seed=7, imf="kroupa")
    idx = np.arange(n)
    a, j, p = gpu_force(nb, cl, 1e-4, idx, nb.NB_FP32)
    ra, rj, rp = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=idx)
    Sa, Sj = term_sums(cl, 1e-4, idx)
    assert (np.linalg.norm(a - ra, axis=1) / Sa).max() <= 1e-4
    assert np.all(np.isfinite(j)) and np.abs(p / rp - 1).max() <= 1e-4
    c2 = inputs.plummer(256, seed=2)
    pos = c2.pos.copy()
    pos[1] = pos[0] + np.array([1e-6, 0.0, 0.0])
    c3 = inputs.Cluster(pos, c2.vel, c2.mass, c2.offsets)
    af, _, _ = gpu_force(nb, c3, 0.0, [0, 1], nb.NB_FP32)
    am, _, _ = gpu_force(nb, c3, 0.0, [0, 1], nb.NB_MIXED)
    ra, _, _ = oracle.force(pos, c2.vel, c2.mass, 0.0, idx=[0, 1])
    assert rel_err(af, ra).max() > 100 * rel_err(am, ra).max()
    assert rel_err(af, ra).max() > 1e-3


# --------------------------------------------------------- leapfrog ----

def _leapfrog_gpu(nb, cl, eps, a0, prec, n_steps, dt_level, flip=False):
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=eps, precision=prec)
    try:
        sim.set_state(cl.pos, -cl.vel if flip else cl.vel, a0, np.zeros((cl.n, 3)),
                      np.zeros(cl.n, dtype=np.int64), np.full(cl.n, 10, dtype=np.int32))
        sim.leapfrog(n_steps, 1 << (sim.cfg.tick_exp - dt_level))
        s = sim.get_state()
        assert sim.status() == nb.NB_OK
        return s
    finally:
        sim.close()


def test_leapfrog_fp64_matches_oracle(nb, plummer1024):
    cl = plummer1024
    a0 = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4)[0]
    s = _leapfrog_gpu(nb, cl, 1e-4, a0, nb.NB_FP64, 16, 10)
    x, v, a = oracle.leapfrog(cl.pos, cl.vel, a0, cl.mass, 1e-4, 2.0 ** -10, 16)
    assert np.abs(s["pos"] - x).max() <= 1e-12 * np.abs(x).max()
    assert np.abs(s["vel"] - v).max() <= 1e-12 * np.abs(v).max()
    assert rel_err(s["acc"], a).max() <= 1e-12
    assert np.all(s["t"] == 16 << (40 - 10))


def test_leapfrog_fp64_time_reversible(nb):
    cl = inputs.plummer(512, seed=8)
    a0 = oracle.force(cl.pos, cl.vel, cl.mass, 1e-2)[0]
    s = _leapfrog_gpu(nb, cl, 1e-2, a0, nb.NB_FP64, 32, 8)
    back = inputs.Cluster(s["pos"], s["vel"], cl.mass, cl.offsets)
    r = _leapfrog_gpu(nb, back, 1e-2, s["acc"], nb.NB_FP64, 32, 8, flip=True)
    assert np.abs(r["pos"] - cl.pos).max() < 1e-11
    assert np.abs(-r["vel"] - cl.vel).max() < 1e-11


def test_leapfrog_mixed_matches_oracle(nb):
    """Mixed leapfrog (acceleration-only kernel) against the oracle: the
    kicks carry the force error, |dv| <= n dt 1e-6 sum_j |a_ij| and
    |dx| <= n^2 dt^2 1e-6 sum_j |a_ij| over n steps (positions barely move,
    so the term sums at the start bound every step's)."""
    n, steps, L = 4099, 8, 10
    cl = inputs.plummer(n, seed=9, imf="kroupa")
    a0 = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4)[0]
    s = _leapfrog_gpu(nb, cl, 1e-4, a0, nb.NB_MIXED, steps, L)
    x, v, a = oracle.leapfrog(cl.pos, cl.vel, a0, cl.mass, 1e-4, 2.0 ** -L, steps)
    Sa, _ = term_sums(cl, 1e-4, np.arange(n))
    dt = 2.0 ** -L
    dv = np.linalg.norm(s["vel"] - v, axis=1)
    dx = np.linalg.norm(s["pos"] - x, axis=1)
    assert np.all(dv <= 2 * steps * dt * 1e-6 * Sa + 1e-14)
    assert np.all(dx <= 2 * steps ** 2 * dt ** 2 * 1e-6 * Sa + 1e-14)
    assert (np.linalg.norm(s["acc"] - a, axis=1) / Sa).max() <= 2e-6


# ------------------------------------------------- failure detection ----

def test_wait_timeout_is_reported_and_context_survives(nb, plummer1024):
    """A device wait that nothing completes runs out after its clock budget:
    the sticky status says NB_ETIMEOUT, and after clearing it the context
    computes forces as before."""
    cl = plummer1024
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nb.NB_MIXED)
    try:
        sim.check_wait_timeout(0.05)
        assert sim.status() == nb.NB_ETIMEOUT
        sim.clear_status()
        assert sim.status() == nb.NB_OK
        sim.predict(0)
        act = torch.arange(0, cl.n, 7, dtype=torch.int32, device="cuda")
        a, j, p = sim.force(act)
        torch.cuda.synchronize()
        assert sim.status() == nb.NB_OK
        ra, _, _ = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4,
                                idx=act.cpu().numpy().astype(np.int64))
        assert rel_err(a.cpu().numpy(), ra).max() <= 1e-5
    finally:
        sim.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nonfinite_state_is_reported(nb, prec):
    """Two coincident particles without softening give an infinite force; the
    corrector finds the non-finite state and the status says NB_ENONFINITE."""
    cl = inputs.plummer(64, seed=5)
    pos = cl.pos.copy()
    pos[1] = pos[0]
    P = nb.NB_FP64 if prec == "fp64" else nb.NB_MIXED
    sim = nb.Sim(pos, cl.vel, cl.mass, eps=0.0, precision=P, level_min=3, level_max=20)
    try:
        sim.step(1)
        assert sim.status() == nb.NB_ENONFINITE
    finally:
        sim.close()


def test_profile_kernels_times_every_kind_of_launch(nb):
    """nb_profile_kernels: with profiling on, each block step times one
    launch of every kind (t_next, predictor, plan, force, reduction,
    corrector); nb_profile_read keeps reporting the force alone."""
    cl = inputs.plummer(4096, seed=46)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-4, precision=nb.NB_MIXED, level_min=3,
                 level_max=14, graph_steps=8)
    sim.step(4)
    sim.profile(True)
    sim.profile_kernels()
    sim.profile_read()
    sim.step(12)
    kinds = sim.profile_kernels()
    fms, nf = sim.profile_read()
    assert sim.status() == nb.NB_OK
    assert list(kinds) == list(nb.PROFILE_KINDS)
    for k, (ms, n) in kinds.items():
        assert n == 12 and ms > 0, (k, ms, n)
    assert nf == 12 and fms == pytest.approx(kinds["force"][0])
    assert all(n == 0 for _, n in sim.profile_kernels().values())   # read resets
    sim.profile(False)
    sim.close()
