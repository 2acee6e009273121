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
def check(got, ref, prec, nb, cl, eps, idx):
    from test_gpu_parity import term_sums
    ea, ej = rel_err(got[0], ref[0]), rel_err(got[1], ref[1])
    ep = np.abs(got[2] / ref[2] - 1)
    if prec == nb.NB_FP64:
        assert ea.max() <= 1e-12 and ej.max() <= 1e-12 and ep.max() <= 1e-12
    else:
        Sa, Sj = term_sums(cl, eps, idx)
        ca = np.linalg.norm(got[0] - ref[0], axis=1) / Sa
        cj = np.linalg.norm(got[1] - ref[1], axis=1) / Sj
        assert ca.max() <= 2e-6 and cj.max() <= 6e-6, (ca.max(), cj.max())
        assert np.median(ea) <= 1e-7 and np.median(ej) <= 5e-7
        assert ep.max() <= 1e-6


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
