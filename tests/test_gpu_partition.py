"""The j-partition of the force sum and the source re-sort on the GPU (one
GPU; the processes of a partition are emulated by contexts of the same
particles, or run as a one-rank NCCL group).

Each piece of the source order gives the force of Eq. 1 summed over that
piece: against the oracle on the masses of the piece alone, and, summed over
the pieces, against the unpartitioned force.  A block step split around the
sum (nb_block_force / nb_block_correct) keeps the contexts of a partition in
lockstep and integrates like nb_step_block.
"""
import os
import socket

import numpy as np
import pytest
import torch

import oracle
from paper_1411_5234_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


def piece_masses(nb, sim, cl, part, n_parts):
    """The masses with every source outside piece `part` set to zero."""
    perm, soff = sim.source_order()
    mass = np.zeros(cl.n)
    for k in range(cl.n_clusters):
        b, e = nb.source_piece(int(soff[k + 1] - soff[k]), part, n_parts)
        p = perm[soff[k] + b:soff[k] + e]
        p = p[p >= 0]
        mass[p] = cl.mass[p]
    return mass


def pair_sum(cl, mass, eps, idx):
    """sum_j m_j |d_ij| / s_ij^3 over each target's own cluster (j != i)."""
    out = np.zeros(len(idx))
    for k in range(cl.n_clusters):
        o0, o1 = int(cl.offsets[k]), int(cl.offsets[k + 1])
        sel = np.nonzero((idx >= o0) & (idx < o1))[0]
        for c0 in range(0, len(sel), 512):
            ii = idx[sel[c0:c0 + 512]]
            d = cl.pos[None, o0:o1, :] - cl.pos[ii, None, :]
            r2 = (d * d).sum(2)
            s2 = r2 + eps * eps
            s2[np.arange(len(ii)), ii - o0] = np.inf
            out[sel[c0:c0 + 512]] = (mass[None, o0:o1] * np.sqrt(r2) * s2 ** -1.5).sum(1)
    return out


def oracle_force(cl, mass, eps, idx):
    """Oracle force on the global targets idx, each from its own cluster."""
    acc = np.zeros((len(idx), 3))
    jerk = np.zeros((len(idx), 3))
    pot = np.zeros(len(idx))
    for k in range(cl.n_clusters):
        o0, o1 = int(cl.offsets[k]), int(cl.offsets[k + 1])
        sel = np.nonzero((idx >= o0) & (idx < o1))[0]
        if len(sel) == 0:
            continue
        a, j, p = oracle.force(cl.pos[o0:o1], cl.vel[o0:o1], mass[o0:o1], eps, idx=idx[sel] - o0)
        acc[sel], jerk[sel], pot[sel] = a, j, p
    return acc, jerk, pot


@pytest.mark.parametrize("prec_name", ["NB_FP64", "NB_MIXED"])
@pytest.mark.parametrize("n_parts", [2, 3, 5])
def test_force_pieces_sum_to_the_whole(nb, prec_name, n_parts):
    prec = getattr(nb, prec_name)
    cl = inputs.plummer_batch(3, n_min=300, n_max=3000, seed0=61, imf="kroupa")
    eps = 1e-4
    idx = inputs.random_active(cl.n, cl.n // 2, seed=3)
    act = torch.as_tensor(idx, device="cuda")
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, offsets=cl.offsets, eps=eps, precision=prec)
    sim.predict(0)
    full = [x.cpu().numpy() for x in sim.force(act)]
    one = [x.cpu().numpy() for x in sim.force_range(act, 0, 1)]
    for x, y in zip(one, full):                      # one part is nb_force itself
        assert np.array_equal(x, y)
    pieces = [[x.cpu().numpy() for x in sim.force_range(act, r, n_parts)]
              for r in range(n_parts)]
    assert sim.status() == nb.NB_OK
    tot = [sum(p[c] for p in pieces) for c in range(3)]
    ra, rj, rp = oracle_force(cl, cl.mass, eps, idx)
    if prec == nb.NB_FP64:
        assert rel(tot[0], full[0]).max() <= 1e-12
        assert rel(tot[1], full[1]).max() <= 1e-12
        assert (np.abs(tot[2] - full[2]) / np.abs(full[2])).max() <= 1e-12
        assert rel(tot[0], ra).max() <= 1e-12
    else:
        assert np.median(rel(tot[0], ra)) <= 1e-7
        assert np.quantile(rel(tot[0], ra), 0.999) <= 1e-6
        assert np.median(rel(tot[1], rj)) <= 5e-7
    # every piece against the oracle on that piece's masses alone, relative
    # to the piece's own pair magnitudes (a partial sum may cancel); an empty
    # piece gives exact zeros
    for r, p in enumerate(pieces):
        mass = piece_masses(nb, sim, cl, r, n_parts)
        if not mass.any():
            assert all(not x.any() for x in p)
            continue
        pa, _, _ = oracle_force(cl, mass, eps, idx)
        S = pair_sum(cl, mass, eps, idx)
        err = np.linalg.norm(p[0] - pa, axis=1)
        has = S > 0
        assert not p[0][~has].any()
        gate = 1e-13 if prec == nb.NB_FP64 else 1e-6
        assert (err[has] / S[has]).max() <= gate, (err[has] / S[has]).max()
    sim.close()


def test_empty_pieces_and_bad_parts(nb):
    cl = inputs.plummer(300, seed=62)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=1e-3, precision=nb.NB_MIXED)
    n_slots = int(sim.source_order()[1][1])
    assert n_slots == 300
    pieces = [nb.source_piece(n_slots, r, 5) for r in range(5)]
    assert pieces[3] == (300, 300) and pieces[4] == (300, 300)   # 3 tiles over 5 parts
    act = torch.arange(300, dtype=torch.int32, device="cuda")
    sim.predict(0)
    for r in (3, 4):
        for x in sim.force_range(act, r, 5):
            assert not x.any()
    for bad in [(5, 5), (-1, 2), (0, 0)]:
        with pytest.raises(nb.NBError):
            sim.force_range(act, *bad)
    with pytest.raises(nb.NBError):
        sim.block_correct()                                   # no step open
    sim.block_force(0, 1)
    # while a split step is open, nothing may touch its active list or rows
    for call in (lambda: sim.step(1), lambda: sim.block_force(0, 1), lambda: sim.predict(0),
                 lambda: sim.force(act), lambda: sim.get_state(), lambda: sim.energy(),
                 lambda: sim.resort_sources()):
        with pytest.raises(nb.NBError) as err:
            call()
        assert err.value.code == nb.NB_ESTATE
    sim.block_correct()
    sim.step(1)
    assert sim.status() == nb.NB_OK
    sim.close()


@pytest.mark.parametrize("prec_name,order", [("NB_FP64", 4), ("NB_FP64", 6), ("NB_MIXED", 4),
                                             ("NB_MIXED", 6)])
def test_partitioned_block_steps_stay_in_lockstep(nb, prec_name, order):
    """Two contexts of the same particles as the two processes of a
    partition: each evaluates its piece, the test adds the rows (the
    all-reduce), each corrects.  Their states stay bitwise equal, and they
    integrate like one context's nb_step_block."""
    prec = getattr(nb, prec_name)
    cl = inputs.plummer(3000, seed=63, imf="kroupa")
    kw = dict(eps=1e-3, precision=prec, level_min=3, level_max=14, order=order, graph_steps=0)
    ref = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    ranks = [nb.Sim(cl.pos, cl.vel, cl.mass, **kw) for _ in range(2)]
    n_steps = 48
    ms = []
    for _ in range(n_steps):
        got = [s.block_force(r, 2) for r, s in enumerate(ranks)]
        assert got[0][0] == got[1][0]
        assert len(got[0][1]) == (3 if order == 6 else 2)
        ms.append(got[0][0])
        torch.cuda.synchronize()
        for q in range(len(got[0][1])):
            tot = got[0][1][q] + got[1][1][q]
            got[0][1][q].copy_(tot)
            got[1][1][q].copy_(tot)
        torch.cuda.synchronize()
        for s in ranks:
            s.block_correct()
    ref.step(n_steps)
    st = [s.get_state() for s in ranks]
    s_ref = ref.get_state()
    for s in ranks + [ref]:
        assert s.status() == nb.NB_OK
    for key in ("pos", "vel", "acc", "jerk", "t", "level"):
        assert np.array_equal(st[0][key], st[1][key]), key
    assert min(ms) < cl.n                        # block steps with a proper subset
    e_part = sum(ranks[0].energy())
    e_ref = sum(ref.energy())
    if prec == nb.NB_FP64:
        assert np.array_equal(st[0]["t"], s_ref["t"])
        assert rel(st[0]["pos"], s_ref["pos"]).max() <= 1e-10
        assert abs(e_part - e_ref) <= 1e-12 * abs(e_ref)
    else:   # the partial sums round apart: the runs agree to the mixed path's accuracy
        assert abs(e_part - e_ref) <= 1e-7 * abs(e_ref)
    for s in ranks + [ref]:
        s.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("prec_name", ["NB_FP64", "NB_MIXED"])
def test_partition_driver_on_one_nccl_rank_equals_block_steps(nb, prec_name):
    """The partition module's block step (nb_block_force, an NCCL all-reduce
    of the rows in place on the context's stream, nb_block_correct) over a
    one-rank group reproduces nb_step_block bit for bit."""
    import torch.distributed as dist
    from paper_1411_5234_gb300 import partition
    if not dist.is_nccl_available():
        pytest.skip("torch without NCCL")
    prec = getattr(nb, prec_name)
    cl = inputs.plummer(4096, seed=64)
    kw = dict(eps=1e-4, precision=prec, level_min=3, level_max=14, graph_steps=0)
    ref = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    ref.step(40)
    s_ref = ref.get_state()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        sim = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
        part = partition.Partition(sim)
        part.step(40)
        s = sim.get_state()
        assert sim.status() == nb.NB_OK
        for key in ("pos", "vel", "acc", "jerk", "t", "level"):
            assert np.array_equal(s[key], s_ref[key]), key
        # the full force through the partition: one rank, nb_force's bits
        act = torch.as_tensor(inputs.random_active(cl.n, 700, seed=9), device="cuda")
        sim.predict(0)
        a1, j1, p1 = (x.cpu().numpy() for x in part.force(act))
        a0, j0, p0 = (x.cpu().numpy() for x in sim.force(act))
        assert np.array_equal(a1, a0) and np.array_equal(j1, j0) and np.array_equal(p1, p0)
        sim.close()
    finally:
        dist.destroy_process_group()
    ref.close()


@pytest.mark.parametrize("prec_name", ["NB_FP64", "NB_MIXED"])
def test_resort_sources_keeps_forces_and_integration(nb, prec_name):
    """Re-sorting the source slots by the current positions changes the
    summation order only: the same forces (FP64 to rounding, mixed to its
    gates), and an integration that re-sorts midway follows one that does
    not."""
    prec = getattr(nb, prec_name)
    cl = inputs.plummer(4096, seed=65, imf="kroupa")
    kw = dict(eps=1e-4, precision=prec, level_min=3, level_max=14, graph_steps=8)
    ref = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, **kw)
    ref.step(64)
    sim.step(64)
    perm0, _ = sim.source_order()
    act = torch.as_tensor(inputs.random_active(cl.n, 1500, seed=4), device="cuda")
    t = sim.stats().t_min
    sim.predict(t)
    f0 = [x.cpu().numpy() for x in sim.force(act)]
    sim.resort_sources()
    perm1, soff = sim.source_order()
    assert not np.array_equal(perm0, perm1)                  # the particles moved
    assert np.array_equal(np.sort(perm1[perm1 >= 0]), np.arange(cl.n))
    assert (perm1[cl.n:] == -1).all() and soff[-1] == len(perm1)
    sim.predict(t)
    f1 = [x.cpu().numpy() for x in sim.force(act)]
    if prec == nb.NB_FP64:
        assert rel(f1[0], f0[0]).max() <= 1e-13 and rel(f1[1], f0[1]).max() <= 1e-12
    else:
        assert np.median(rel(f1[0], f0[0])) <= 1e-7
        assert np.quantile(rel(f1[0], f0[0]), 0.999) <= 2e-6
    ref.step(64)
    sim.step(64)
    s, s_ref = sim.get_state(), ref.get_state()
    assert sim.status() == nb.NB_OK and ref.status() == nb.NB_OK
    if prec == nb.NB_FP64:
        assert np.array_equal(s["t"], s_ref["t"])
        assert rel(s["pos"], s_ref["pos"]).max() <= 1e-10
    else:
        e, e_ref = sum(sim.energy()), sum(ref.energy())
        assert abs(e - e_ref) <= 1e-7 * abs(e_ref)
    sim.close()
    ref.close()
