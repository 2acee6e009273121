"""The j-partition of the force sum on CPU: the library's piece rule and two
gloo ranks, no GPU.

Each rank evaluates Eq. 1 over its piece of the source order -- here with
the oracle, on the masses of the other pieces set to zero, which adds exact
zeros to its compensated sums -- and the partition module's all-reduce
gives both ranks the full force.  The sum must equal the unpartitioned
force within the FP64 gate, and both ranks must hold the same bits (the
replicated states of a partitioned integration stay in lockstep only then).
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_built():
    from paper_1411_5234_gb300 import build
    return build.build()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_slots", [4, 128, 1000, 1024, 65536 + 4, 1 << 20])
@pytest.mark.parametrize("n_parts", [1, 2, 3, 7, 8])
def test_source_pieces_tile_the_slots(lib_built, n_slots, n_parts):
    from paper_1411_5234_gb300 import partition
    pieces = [partition.source_piece(n_slots, r, n_parts) for r in range(n_parts)]
    assert pieces[0][0] == 0 and pieces[-1][1] == n_slots
    for (b0, e0), (b1, e1) in zip(pieces, pieces[1:]):
        assert e0 == b1                                    # contiguous, no overlap
    per = -(-(-(-n_slots // n_parts)) // 128) * 128       # ceil(n / P) up to a tile
    for b, e in pieces:
        assert 0 <= b <= e <= n_slots
        assert b % 128 == 0 or b == n_slots                # tile-aligned starts
        assert e - b <= per                                # balanced to one tile
    if n_parts == 1:
        assert pieces == [(0, n_slots)]


def test_source_piece_rejects_bad_arguments(lib_built):
    from paper_1411_5234_gb300 import nbody
    for args in [(100, 2, 2), (100, -1, 2), (100, 0, 0), (-4, 0, 1)]:
        with pytest.raises(nbody.NBError):
            nbody.source_piece(*args)


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1411_5234_gb300 import inputs, partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cl = inputs.plummer(1000, seed=51, imf="kroupa")
    n = cl.n
    n_slots = -(-n // 4) * 4
    # a source order: any permutation of the particles, padded to a multiple
    # of 4 slots (the sum over sources does not depend on the order)
    slots = np.full(n_slots, -1, dtype=np.int64)
    slots[:n] = np.random.default_rng(5).permutation(n)
    b, e = partition.source_piece(n_slots, rank, world)
    mine = slots[b:e]
    mine = mine[mine >= 0]
    mass = np.zeros(n)
    mass[mine] = cl.mass[mine]
    idx = np.arange(0, n, 3)                         # the targets of the step
    acc, jerk, pot = oracle.force(cl.pos, cl.vel, mass, 1e-3, idx=idx)
    rows = [torch.from_numpy(np.ascontiguousarray(x)) for x in (acc, jerk, pot)]
    partition.allreduce_rows(rows, None)
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), acc=rows[0].numpy(), jerk=rows[1].numpy(),
             pot=rows[2].numpy(), n_mine=len(mine))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_force_sum_equals_the_whole(lib_built, world):
    pytest.importorskip("torch")
    import tempfile
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1411_5234_gb300 import inputs
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        r = [dict(np.load(os.path.join(d, f"r{k}.npz"))) for k in range(world)]
    cl = inputs.plummer(1000, seed=51, imf="kroupa")
    assert sum(int(x["n_mine"]) for x in r) == cl.n         # every source in one piece
    assert all(int(x["n_mine"]) > 0 for x in r)
    for x in r[1:]:                                          # the same bits on every rank
        for k in ("acc", "jerk", "pot"):
            assert np.array_equal(x[k], r[0][k])
    idx = np.arange(0, cl.n, 3)
    ra, rj, rp = oracle.force(cl.pos, cl.vel, cl.mass, 1e-3, idx=idx)
    # the FP64 gate: per particle, relative to the sum of the pair magnitudes
    d = cl.pos[None, :, :] - cl.pos[idx, None, :]
    s2 = (d * d).sum(2) + 1e-6
    s2[np.arange(len(idx)), idx] = np.inf
    Sa = (cl.mass[None, :] * np.sqrt((d * d).sum(2)) * s2 ** -1.5).sum(1)
    Sp = (cl.mass[None, :] * s2 ** -0.5).sum(1)
    ea = np.linalg.norm(r[0]["acc"] - ra, axis=1)
    assert (ea / Sa).max() <= 1e-14, (ea / Sa).max()
    assert (ea / np.linalg.norm(ra, axis=1)).max() <= 1e-12
    assert (np.abs(r[0]["pot"] - rp) / Sp).max() <= 1e-14
    ej = np.linalg.norm(r[0]["jerk"] - rj, axis=1) / np.linalg.norm(rj, axis=1)
    assert ej.max() <= 1e-12, ej.max()


class _FakeSim:
    """Stands in for a context on the host: block_force hands out this
    rank's partial rows (rank + 1 everywhere), block_correct records what
    the rows hold when the corrector would read them."""

    def __init__(self, rank, m):
        import torch
        self.stream = None
        self.rank, self.m = rank, m
        self.rows = [torch.full((m, 4), float(rank + 1), dtype=torch.float64) for _ in range(2)]
        self.seen = []

    def block_force(self, part, n_parts):
        assert part == self.rank
        for r in self.rows:
            r.fill_(float(part + 1))
        return self.m, self.rows

    def block_correct(self):
        self.seen.append([float(r.sum()) for r in self.rows])


def _driver_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1411_5234_gb300 import partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sim = _FakeSim(rank, m=5)
    p = partition.Partition(sim, check_every=2)
    m = p.step(4)
    np.save(os.path.join(out_dir, f"d{rank}.npy"), np.array(sim.seen + [[m, m]]))
    # a rank whose active count differs is caught by the lockstep check,
    # before any rows are summed
    sim.m = 5 + rank
    err = ""
    try:
        p.step(2)
    except RuntimeError as e:
        err = str(e)
    with open(os.path.join(out_dir, f"e{rank}.txt"), "w") as f:
        f.write(err)
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_step_sums_before_every_correction():
    pytest.importorskip("torch")
    import tempfile
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_driver_main, args=(2, _free_port(), d), nprocs=2, join=True,
                           start_method="spawn")
        s0, s1 = (np.load(os.path.join(d, f"d{k}.npy")) for k in (0, 1))
        e0, e1 = (open(os.path.join(d, f"e{k}.txt")).read() for k in (0, 1))
    # 4 corrections, each seeing the rows summed over ranks: (1 + 2) * 5 * 4
    assert np.array_equal(s0, s1)
    assert np.all(s0[:4] == 3.0 * 5 * 4) and s0[4, 0] == 5
    assert "out of lockstep" in e0 and "out of lockstep" in e1


class _FakeForceSim:
    """A context stand-in for Partition.force: this rank's partial rows are
    rank + 1 everywhere (the potential only when asked for)."""

    def __init__(self, rank):
        self.rank, self.stream = rank, None

    def force_range(self, active, part, n_parts, want_pot=True):
        import torch
        assert part == self.rank and n_parts == 2
        m = len(active)
        acc = torch.full((m, 3), float(part + 1), dtype=torch.float64)
        jerk = torch.full((m, 3), 10.0 * (part + 1), dtype=torch.float64)
        pot = torch.full((m,), -float(part + 1), dtype=torch.float64) if want_pot else None
        return acc, jerk, pot


def _force_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1411_5234_gb300 import partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = partition.Partition(_FakeForceSim(rank))
    acc, jerk, pot = p.force(list(range(7)))
    acc2, jerk2, pot2 = p.force(list(range(3)), want_pot=False)
    np.savez(os.path.join(out_dir, f"f{rank}.npz"), acc=acc.numpy(), jerk=jerk.numpy(),
             pot=pot.numpy(), acc2=acc2.numpy(), none=pot2 is None)
    dist.barrier()
    dist.destroy_process_group()


def test_partition_force_sums_every_row_array():
    pytest.importorskip("torch")
    import tempfile
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_force_main, args=(2, _free_port(), d), nprocs=2, join=True,
                           start_method="spawn")
        r = [dict(np.load(os.path.join(d, f"f{k}.npz"))) for k in (0, 1)]
    for x in r:
        assert np.all(x["acc"] == 3.0) and np.all(x["jerk"] == 30.0) and np.all(x["pot"] == -3.0)
        assert x["acc"].shape == (7, 3) and np.all(x["acc2"] == 3.0) and bool(x["none"])
