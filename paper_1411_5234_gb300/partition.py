"""j-partition of the force sum across processes, one GPU per process.

The paper's template code runs on clusters of GPUs, with MPI between the
processes, and its scaling result splits the force work among the GPUs
(Sec. 2.1, Fig. 2 left).  The force on a target is a sum over sources
(Eq. 1), so it splits exactly:

* every rank holds the whole particle set in its own context (the state is
  replicated: a few hundred bytes per particle, so the whole set fits one
  GPU's memory long before the O(N^2) work does);
* rank r evaluates the sum over piece r of each cluster's source order
  (``Sim.force_range`` / ``Sim.block_force`` with part = r, n_parts = world
  size; the library cuts each cluster's slots into contiguous, tile-aligned
  pieces);
* one all-reduce (sum) of the partial rows -- acceleration and jerk, plus
  the snap in the 6th-order scheme and the potential when asked for -- gives
  every rank the full force of the step's active particles;
* every rank then applies the same corrector to the same sums, so the
  replicated states, and with them the next block time and active set, stay
  identical on every rank without any exchange of particles.

The last point needs every rank to receive the same bits from the
all-reduce.  The reduction algorithms of NCCL and gloo reduce each element
once and then distribute the result, which gives that; ``Partition.step``
also compares the active counts of the ranks every ``check_every`` steps,
before their rows are summed, and raises if the ranks have drifted apart.

The all-reduce runs through torch.distributed (NCCL between GPUs, gloo on
the host) on the library's own step buffers, viewed in place and ordered on
the context's stream.  No kernel reads a peer's memory.
"""
from __future__ import annotations

import contextlib

import torch
import torch.distributed as dist


def source_piece(n_slots: int, part: int, n_parts: int) -> tuple[int, int]:
    """Slot range [begin, end) of piece ``part`` of ``n_parts`` of a cluster
    with ``n_slots`` source slots (the library's rule, nb_source_piece)."""
    from . import nbody
    return nbody.source_piece(n_slots, part, n_parts)


def allreduce_rows(tensors, group=None, stream: torch.cuda.Stream | None = None):
    """Sum every tensor over the ranks of ``group`` in place, one all-reduce
    per tensor in list order.  With ``stream`` the collectives are ordered
    on that stream (the context's), so that the library's next launch there
    sees the sums."""
    ctx = torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext()
    with ctx:
        for t in tensors:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


class Partition:
    """A context of the whole particle set whose force sums this rank
    shares with the other ranks of ``group`` (see the module docstring).

    ``sim`` is the rank's ``nbody.Sim`` (every rank builds it from the same
    particles and configuration, so that the source orders agree)."""

    def __init__(self, sim, group=None, check_every: int = 1):
        self.sim = sim
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.check_every = max(1, int(check_every))
        self._steps = 0

    def _stream(self):
        return self.sim.stream if torch.cuda.is_available() else None

    def force(self, active: torch.Tensor, want_pot: bool = True):
        """The full acceleration, jerk (and potential) of ``active`` from the
        last prediction: this rank's piece, summed over the ranks."""
        acc, jerk, pot = self.sim.force_range(active, self.rank, self.world, want_pot=want_pot)
        allreduce_rows([t for t in (acc, jerk, pot) if t is not None], self.group)
        return acc, jerk, pot

    def step(self, n_steps: int = 1) -> int:
        """``n_steps`` block steps of the partitioned integration; returns the
        active count of the last one."""
        m = 0
        for _ in range(int(n_steps)):
            m, rows = self.sim.block_force(self.rank, self.world)
            # before the sums: ranks whose row counts differ must not enter
            # the all-reduce (the step stays open after the error)
            if self._steps % self.check_every == 0:
                self._check_lockstep(m)
            if m > 0:
                allreduce_rows(rows, self.group, stream=self._stream())
            self.sim.block_correct()
            self._steps += 1
        return m

    def _check_lockstep(self, m: int):
        # the ranks' active counts must agree: (m, -m) reduced with MAX
        # gives (max m, -min m)
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        x = torch.tensor([m, -m], dtype=torch.int64, device=dev)
        dist.all_reduce(x, op=dist.ReduceOp.MAX, group=self.group)
        if int(x[0]) != -int(x[1]):
            raise RuntimeError(f"ranks out of lockstep: active counts {-int(x[1])}..{int(x[0])}")
