"""nb_force_noalloc: the entry point for callers that cannot allocate.

Such callers (code in a host callback or library hook while another framework
owns every device allocation, or runtimes that forbid cudaMalloc after
start-up) cannot hand the library a workspace, so this entry point keeps its
scratch in a fixed device array inside the library.  It must give the same
forces as the regular nb_force on the same inputs, call after call, even
though each call finds the previous call's data in that array.

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1411_5234_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel_err(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


def regular_force(nb, cl, eps, idx, prec):
    sim = nb.Sim(cl.pos, cl.vel, cl.mass, eps=eps, precision=prec)
    sim.predict(0)
    act = torch.as_tensor(np.asarray(idx, dtype=np.int32), device="cuda")
    a, j, p = sim.force(act)
    torch.cuda.synchronize()
    assert sim.status() == nb.NB_OK
    out = a.cpu().numpy(), j.cpu().numpy(), p.cpu().numpy()
    sim.close()
    return out


def noalloc_force(nb, cl, eps, idx, prec, outs):
    dev = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt,
                                                      device="cuda")
    acc, jerk, pot = outs
    nb.force_noalloc(dev(cl.pos), dev(cl.vel), dev(cl.mass), dev(idx, torch.int32), eps=eps,
                     precision=prec, acc=acc, jerk=jerk, pot=pot)
    torch.cuda.synchronize()
    return acc.cpu().numpy(), jerk.cpu().numpy(), pot.cpu().numpy()


# the gates of the parity tests: FP64 per-particle relative error 1e-12;
# mixed: the condition-scaled error (difference over the sum of the terms'
# magnitudes) for every particle, twice the parity gate since both sides
# carry rounding, and the plain relative error's median.  The two entry
# points may sum the sources in different orders and group them differently
# (the workspace path keeps them spatially sorted), so the mixed results
# differ by FP32 rounding, not bit for bit.
def check(got, ref, prec, nb, cl, eps, idx, sample=None):
    """`sample`: rows whose condition-scaled error is checked (default: all)."""
    from test_gpu_parity import term_sums
    ea, ej = rel_err(got[0], ref[0]), rel_err(got[1], ref[1])
    ep = np.abs(got[2] / ref[2] - 1)
    if prec == nb.NB_FP64:
        assert ea.max() <= 1e-12 and ej.max() <= 1e-12 and ep.max() <= 1e-12
    else:
        rows = np.arange(len(idx)) if sample is None else np.asarray(sample)
        Sa, Sj = term_sums(cl, eps, np.asarray(idx)[rows])
        ca = np.linalg.norm(got[0][rows] - ref[0][rows], axis=1) / Sa
        cj = np.linalg.norm(got[1][rows] - ref[1][rows], axis=1) / Sj
        assert ca.max() <= 2e-6 and cj.max() <= 6e-6, (ca.max(), cj.max())
        assert np.median(ea) <= 1e-7 and np.median(ej) <= 5e-7
        assert ep.max() <= 1e-6


def new_outputs(m):
    """Outputs the no-allocation caller would already own (NaN-filled, so
    that a row left unwritten shows)."""
    return (torch.full((m, 3), np.nan, dtype=torch.float64, device="cuda"),
            torch.full((m, 3), np.nan, dtype=torch.float64, device="cuda"),
            torch.full((m,), np.nan, dtype=torch.float64, device="cuda"))


def test_noalloc_matches_nb_force_twice_in_a_row(nb):
    cases = [
        (inputs.plummer(5000, seed=21, imf="kroupa"), 1e-4,
         inputs.random_active(5000, 777, seed=5), nb.NB_MIXED),
        (inputs.plummer(20003, seed=22), 1e-3,
         inputs.random_active(20003, 20003, seed=6), nb.NB_FP64),
        (inputs.plummer(5000, seed=21, imf="kroupa"), 1e-4,
         inputs.random_active(5000, 3001, seed=7), nb.NB_MIXED),
    ]
    for cl, eps, idx, prec in cases:
        m = len(idx)
        # outputs the no-allocation caller would already own
        outs = (torch.full((m, 3), np.nan, dtype=torch.float64, device="cuda"),
                torch.full((m, 3), np.nan, dtype=torch.float64, device="cuda"),
                torch.full((m,), np.nan, dtype=torch.float64, device="cuda"))
        got = noalloc_force(nb, cl, eps, idx, prec, outs)
        ref = regular_force(nb, cl, eps, idx, prec)
        check(got, ref, prec, nb, cl, eps, idx)


def test_noalloc_rejects_sizes_beyond_its_array(nb):
    n = nb.NOALLOC_MAX_SOURCES + 1
    z = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    mass = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    idx = torch.arange(4, dtype=torch.int32, device="cuda")
    with pytest.raises(nb.NBError) as e:
        nb.force_noalloc(z, z, mass, idx)
    assert e.value.code == nb.NB_EINVAL


def test_noalloc_at_its_maximum_size_between_smaller_calls(nb):
    """n = NB_NOALLOC_MAX_SOURCES fills the fixed array's layout to its
    limit.  Each precision runs the maximum size with every particle a target
    and with a few targets (the wide i-split reduction), right after a call of
    the other size, so stale pad slots, tiles or counters of the previous call
    would show.  Every call matches nb_force, and a sample of its targets the
    FP64 CPU oracle, with the parity gates."""
    from test_gpu_parity import check_mixed, term_sums
    nmax = nb.NOALLOC_MAX_SOURCES
    big = inputs.plummer(nmax, seed=23, imf="kroupa")
    small = inputs.plummer(1001, seed=24)
    eps = 1e-4
    sample_rows = np.arange(0, 300, 7)
    for prec in (nb.NB_MIXED, nb.NB_FP64):
        seq = [(big, inputs.random_active(nmax, nmax, seed=8)),
               (small, inputs.random_active(1001, 500, seed=9)),
               (big, inputs.random_active(nmax, 300, seed=10)),
               (small, inputs.random_active(1001, 17, seed=11)),
               (big, inputs.random_active(nmax, nmax, seed=12))]
        for cl, idx in seq:
            m = len(idx)
            got = noalloc_force(nb, cl, eps, idx, prec, new_outputs(m))
            assert nb.noalloc_status() == nb.NB_OK
            ref = regular_force(nb, cl, eps, idx, prec)
            rows = sample_rows[sample_rows < m]
            check(got, ref, prec, nb, cl, eps, idx, sample=rows)
            ra, rj, rp = oracle.force(cl.pos, cl.vel, cl.mass, eps,
                                      idx=np.asarray(idx)[rows].astype(np.int64))
            if prec == nb.NB_FP64:
                assert rel_err(got[0][rows], ra).max() <= 1e-12
                assert rel_err(got[1][rows], rj).max() <= 1e-12
                assert np.abs(got[2][rows] / rp - 1).max() <= 1e-12
            else:
                Sa, Sj = term_sums(cl, eps, np.asarray(idx)[rows])
                check_mixed(got[0][rows], got[1][rows], ra, rj, Sa, Sj)


def test_noalloc_status_reports_a_bad_target_and_clears(nb):
    """A target index outside [0, n) is reported by nb_noalloc_status as
    NB_EINVAL (the kernels check every index before using it, so nothing is
    read out of bounds); the next good call starts from a cleared status."""
    cl = inputs.plummer(2000, seed=25)
    dev = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt,
                                                      device="cuda")
    for prec in (nb.NB_MIXED, nb.NB_FP64):
        idx = np.array([3, 2000, 7], dtype=np.int32)  # 2000 is out of range
        nb.force_noalloc(dev(cl.pos), dev(cl.vel), dev(cl.mass), dev(idx, torch.int32),
                         precision=prec)
        assert nb.noalloc_status() == nb.NB_EINVAL
        good = np.array([3, 1999, 7], dtype=np.int32)
        a, _, _ = nb.force_noalloc(dev(cl.pos), dev(cl.vel), dev(cl.mass),
                                   dev(good, torch.int32), precision=prec)
        assert nb.noalloc_status() == nb.NB_OK
        ra, _, _ = oracle.force(cl.pos, cl.vel, cl.mass, 1e-4, idx=good.astype(np.int64))
        tol = 1e-12 if prec == nb.NB_FP64 else 1e-5
        assert rel_err(a.cpu().numpy(), ra).max() <= tol
