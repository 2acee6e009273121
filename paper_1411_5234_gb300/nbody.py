"""ctypes binding of libnbody_gb300.so (the C ABI in include/nbody_gb300.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  PyTorch supplies the device workspace (one uint8 tensor) and the
stream.  Importing this module loads the library; a missing library raises
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

NB_OK, NB_EINVAL, NB_ENOMEM, NB_ECUDA, NB_ETIMEOUT, NB_ENONFINITE, NB_ESTATE = range(7)
NB_FP64, NB_MIXED, NB_DS, NB_FP32 = 0, 1, 2, 3
MIXED_VARIANTS = 8    # NB_MIXED_VARIANTS: shapes of the mixed force kernel
TUNE_BUCKETS = 32     # NB_TUNE_BUCKETS: autotune table entries (ceil(log2 m))
TUNE_POINTS = 8       # NB_TUNE_POINTS: active counts the autotuner measures
DEFAULT_VARIANT = 0   # the shape nb_default_config selects

FUNCTIONS = [
    "nb_default_config", "nb_workspace_size", "nb_init", "nb_free", "nb_predict", "nb_force",
    "nb_correct", "nb_step_block", "nb_set_end_time", "nb_energy", "nb_get_state",
    "nb_set_state", "nb_stats", "nb_status", "nb_clear_status", "nb_strerror",
    "nb_profile_enable", "nb_profile_read", "nb_force_noalloc", "nb_tile_stats",
    "nb_energies", "nb_autotune", "nb_step_leapfrog", "nb_check_wait_timeout",
    "nb_noalloc_status", "nb_measure_rate", "nb_force_snap", "nb_correct_snap",
    "nb_get_derivs", "nb_set_derivs", "nb_source_piece", "nb_source_order", "nb_force_range",
    "nb_block_force", "nb_block_correct", "nb_resort_sources", "nb_tune_table", "nb_profile_kernels",
]
PROFILE_KINDS = ("t_next", "predictor", "active_list_and_plan", "force", "reduction",
                 "corrector")   # NB_PROFILE_KINDS, in the ABI's order
PIECE_ALIGN = 128     # NB_PIECE_ALIGN: slots per tile of a source piece


class NbConfig(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("eps", ctypes.c_double), ("eta", ctypes.c_double),
                ("eta_start", ctypes.c_double), ("level_min", ctypes.c_int32),
                ("level_max", ctypes.c_int32), ("tick_exp", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("bfactor", ctypes.c_int32),
                ("graph_steps", ctypes.c_int32), ("sort_sources", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("order", ctypes.c_int32)]


class NBError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


def library_path() -> str:
    return os.environ.get("NBODY_GB300_LIB", _build.LIB)


def _load() -> ctypes.CDLL:
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libnbody_gb300.so not found at {path}; build it with "
                           "`python -m paper_1411_5234_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    sig = {
        "nb_default_config": (None, [P]),
        "nb_workspace_size": (ctypes.c_int, [i64, i32, P, P]),
        "nb_init": (ctypes.c_int, [P, P, i32, P, P, P, P, P, ctypes.c_size_t, P]),
        "nb_free": (None, [P]),
        "nb_predict": (ctypes.c_int, [P, i64]),
        "nb_force": (ctypes.c_int, [P, P, i64, P, P, P]),
        "nb_correct": (ctypes.c_int, [P, i64, P, i64, P, P]),
        "nb_step_block": (ctypes.c_int, [P, i64, P, P]),
        "nb_step_leapfrog": (ctypes.c_int, [P, i64, i64]),
        "nb_check_wait_timeout": (ctypes.c_int, [P, ctypes.c_double]),
        "nb_set_end_time": (ctypes.c_int, [P, i64]),
        "nb_energy": (ctypes.c_int, [P, i32, P, P]),
        "nb_get_state": (ctypes.c_int, [P, P, P, P, P, P, P]),
        "nb_set_state": (ctypes.c_int, [P, P, P, P, P, P, P]),
        "nb_stats": (ctypes.c_int, [P, P, P, P, P]),
        "nb_status": (ctypes.c_int, [P]),
        "nb_clear_status": (ctypes.c_int, [P]),
        "nb_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "nb_profile_enable": (ctypes.c_int, [P, ctypes.c_int]),
        "nb_profile_read": (ctypes.c_int, [P, P, P]),
        "nb_tile_stats": (ctypes.c_int, [P, P, P]),
        "nb_energies": (ctypes.c_int, [P, P, P]),
        "nb_autotune": (ctypes.c_int, [P, ctypes.c_char_p, P, P]),
        "nb_tune_table": (ctypes.c_int, [P, P, P]),
        "nb_profile_kernels": (ctypes.c_int, [P, P, P]),
        "nb_force_noalloc": (ctypes.c_int, [P, P, P, i64, P, i64, ctypes.c_double,
                                            ctypes.c_double, i32, P, P, P, P]),
        "nb_noalloc_status": (ctypes.c_int, [P]),
        "nb_measure_rate": (ctypes.c_int, [P, i32, P]),
        "nb_force_snap": (ctypes.c_int, [P, P, i64, P, P, P, P]),
        "nb_correct_snap": (ctypes.c_int, [P, i64, P, i64, P, P, P]),
        "nb_get_derivs": (ctypes.c_int, [P, P, P]),
        "nb_set_derivs": (ctypes.c_int, [P, P, P]),
        "nb_source_piece": (ctypes.c_int, [i64, i32, i32, P, P]),
        "nb_source_order": (ctypes.c_int, [P, P, P, P]),
        "nb_force_range": (ctypes.c_int, [P, P, i64, i32, i32, P, P, P]),
        "nb_block_force": (ctypes.c_int, [P, i32, i32, P, P, P, P]),
        "nb_block_correct": (ctypes.c_int, [P]),
        "nb_resort_sources": (ctypes.c_int, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def strerror(code: int) -> str:
    return lib.nb_strerror(int(code)).decode()


def _check(rc, where):
    if rc != NB_OK:
        raise NBError(rc, where)


def default_config(**kw) -> NbConfig:
    cfg = NbConfig()
    lib.nb_default_config(ctypes.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise AttributeError(f"nb_config has no field {k!r}")
        setattr(cfg, k, v)
    return cfg


def source_piece(n_slots: int, part: int, n_parts: int) -> tuple[int, int]:
    """Slot range [begin, end) of piece ``part`` of ``n_parts`` of a cluster
    with ``n_slots`` source slots (nb_source_piece; host arithmetic)."""
    b, e = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.nb_source_piece(int(n_slots), int(part), int(n_parts), ctypes.byref(b),
                               ctypes.byref(e)), "nb_source_piece")
    return b.value, e.value


def workspace_size(n_total: int, n_clusters: int, cfg: NbConfig) -> int:
    out = ctypes.c_size_t()
    _check(lib.nb_workspace_size(int(n_total), int(n_clusters), ctypes.byref(cfg),
                                 ctypes.byref(out)), "nb_workspace_size")
    return int(out.value)


def _hptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@dataclass
class Stats:
    block_steps: int
    interactions: int
    t_min: int
    t_max: int


class Sim:
    """A library context over caller-owned device memory.

    ``offsets`` (n_clusters + 1) delimit independent clusters; ``mass`` (n),
    ``pos``/``vel`` (n, 3) are host arrays in any float type.  The workspace
    is one torch uint8 tensor on the current CUDA device; work runs on
    ``stream`` (a dedicated torch stream by default, so that block-step
    sequences can be captured in CUDA graphs).
    """

    def __init__(self, pos, vel, mass, offsets=None, cfg: NbConfig | None = None,
                 stream: torch.cuda.Stream | None = None, **cfg_kw):
        self.cfg = cfg if cfg is not None else default_config()
        for k, v in cfg_kw.items():
            setattr(self.cfg, k, v)
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        n = pos.shape[0]
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(n, 3)
        mass = np.ascontiguousarray(mass, dtype=np.float64).reshape(n)
        if offsets is None:
            offsets = np.array([0, n], dtype=np.int64)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.n = n
        self.n_clusters = int(offsets.shape[0] - 1)
        self.offsets = offsets.copy()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.ws_bytes = workspace_size(n, self.n_clusters, self.cfg)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        self._ctx = ctypes.c_void_p()
        torch.cuda.current_stream().synchronize()
        rc = lib.nb_init(ctypes.byref(self._ctx), ctypes.byref(self.cfg), self.n_clusters,
                         _hptr(offsets), _hptr(mass), _hptr(pos), _hptr(vel),
                         ctypes.c_void_p(self.workspace.data_ptr()), self.ws_bytes,
                         ctypes.c_void_p(self.stream.cuda_stream))
        _check(rc, "nb_init")

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib.nb_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- time ------------------------------------------------------------
    def ticks(self, t: float) -> int:
        return int(round(t * 2.0 ** self.cfg.tick_exp))

    def time(self, ticks: int) -> float:
        return float(np.ldexp(float(ticks), -self.cfg.tick_exp))

    # -- hot path --------------------------------------------------------
    def predict(self, t_ticks: int):
        _check(lib.nb_predict(self._ctx, int(t_ticks)), "nb_predict")

    def force(self, active: torch.Tensor, acc: torch.Tensor | None = None,
              jerk: torch.Tensor | None = None, pot: torch.Tensor | None = None,
              want_pot: bool = True, want_jerk: bool = True):
        """Forces on ``active`` (int32 CUDA tensor) from the last prediction.
        ``want_jerk=False`` asks for the acceleration (and potential) only
        (nb_force with jerk == NULL); the returned jerk is then None."""
        if active.dtype != torch.int32 or not active.is_cuda or not active.is_contiguous():
            raise ValueError("active must be a contiguous int32 CUDA tensor")
        m = active.numel()
        if acc is None:
            acc = torch.empty((m, 3), dtype=torch.float64, device="cuda")
        if jerk is None and want_jerk:
            jerk = torch.empty((m, 3), dtype=torch.float64, device="cuda")
        if pot is None and want_pot:
            pot = torch.empty(m, dtype=torch.float64, device="cuda")
        self._order_inputs(active, acc, jerk, pot)
        _check(lib.nb_force(self._ctx, _dptr(active), m, _dptr(acc), _dptr(jerk), _dptr(pot)),
               "nb_force")
        self._order_outputs(acc, jerk, pot)
        return acc, jerk, pot

    def force_range(self, active: torch.Tensor, part: int, n_parts: int,
                    want_pot: bool = True, want_jerk: bool = True):
        """Forces on ``active`` from piece ``part`` of ``n_parts`` of every
        cluster's sources (nb_force_range): one process's share of a
        j-partition; the sum over the parts is ``force``'s result."""
        if active.dtype != torch.int32 or not active.is_cuda or not active.is_contiguous():
            raise ValueError("active must be a contiguous int32 CUDA tensor")
        m = active.numel()
        acc = torch.empty((m, 3), dtype=torch.float64, device="cuda")
        jerk = torch.empty((m, 3), dtype=torch.float64, device="cuda") if want_jerk else None
        pot = torch.empty(m, dtype=torch.float64, device="cuda") if want_pot else None
        self._order_inputs(active, acc, jerk, pot)
        _check(lib.nb_force_range(self._ctx, _dptr(active), m, int(part), int(n_parts),
                                  _dptr(acc), _dptr(jerk), _dptr(pot)), "nb_force_range")
        self._order_outputs(acc, jerk, pot)
        return acc, jerk, pot

    def source_order(self):
        """(particle of each source slot, -1 for padding; each cluster's
        first slot), both host arrays (nb_source_order)."""
        n = ctypes.c_int64()
        _check(lib.nb_source_order(self._ctx, ctypes.byref(n), None, None), "nb_source_order")
        perm = np.empty(n.value, dtype=np.int32)
        soff = np.empty(self.n_clusters + 1, dtype=np.int64)
        _check(lib.nb_source_order(self._ctx, ctypes.byref(n), _hptr(perm), _hptr(soff)),
               "nb_source_order")
        return perm, soff

    def _rows(self, addr: int, m: int) -> torch.Tensor:
        # (m, 4) float64 view of workspace rows at device address addr
        off = addr - self.workspace.data_ptr()
        if off < 0 or off % 8 or off + 32 * m > self.ws_bytes:
            raise RuntimeError("step rows outside the workspace")
        return self.workspace[off:off + 32 * m].view(torch.float64).view(m, 4)

    def block_force(self, part: int = 0, n_parts: int = 1):
        """First half of a block step (nb_block_force): returns the active
        count m and the step's force rows -- [acc, jerk] or, in the 6th-order
        scheme, [acc, jerk, snap] -- as (m, 4) float64 views of the
        workspace (column 3 unused), to be summed over the processes of a
        j-partition in place before ``block_correct``."""
        m = ctypes.c_int64()
        ptr = [ctypes.c_void_p() for _ in range(3)]
        _check(lib.nb_block_force(self._ctx, int(part), int(n_parts), ctypes.byref(m),
                                  *(ctypes.byref(p) for p in ptr)), "nb_block_force")
        rows = [self._rows(p.value, m.value) for p in ptr if p.value]
        return m.value, rows

    def block_correct(self):
        """Second half of a block step (nb_block_correct)."""
        _check(lib.nb_block_correct(self._ctx), "nb_block_correct")

    def resort_sources(self):
        """Re-sort the source slots by the current positions (nb_resort_sources)."""
        _check(lib.nb_resort_sources(self._ctx), "nb_resort_sources")

    def force_snap(self, active: torch.Tensor, want_pot: bool = True):
        """Acceleration, jerk, snap (and potential) of ``active`` from the last
        prediction (order-6 contexts: nb_force_snap)."""
        if active.dtype != torch.int32 or not active.is_cuda or not active.is_contiguous():
            raise ValueError("active must be a contiguous int32 CUDA tensor")
        m = active.numel()
        acc, jerk, snap = (torch.empty((m, 3), dtype=torch.float64, device="cuda")
                           for _ in range(3))
        pot = torch.empty(m, dtype=torch.float64, device="cuda") if want_pot else None
        self._order_inputs(active, acc, jerk, snap, pot)
        _check(lib.nb_force_snap(self._ctx, _dptr(active), m, _dptr(acc), _dptr(jerk),
                                 _dptr(snap), _dptr(pot)), "nb_force_snap")
        self._order_outputs(acc, jerk, snap, pot)
        return acc, jerk, snap, pot

    def correct_snap(self, t_ticks: int, active: torch.Tensor, acc, jerk, snap):
        self._order_inputs(active, acc, jerk, snap)
        _check(lib.nb_correct_snap(self._ctx, int(t_ticks), _dptr(active), active.numel(),
                                   _dptr(acc), _dptr(jerk), _dptr(snap)), "nb_correct_snap")

    def get_derivs(self):
        """(snap, crackle) of an order-6 context, each (n, 3)."""
        snap, crackle = np.empty((self.n, 3)), np.empty((self.n, 3))
        _check(lib.nb_get_derivs(self._ctx, _hptr(snap), _hptr(crackle)), "nb_get_derivs")
        return snap, crackle

    def set_derivs(self, snap, crackle):
        snap = np.ascontiguousarray(snap, dtype=np.float64).reshape(self.n, 3)
        crackle = np.ascontiguousarray(crackle, dtype=np.float64).reshape(self.n, 3)
        _check(lib.nb_set_derivs(self._ctx, _hptr(snap), _hptr(crackle)), "nb_set_derivs")

    def correct(self, t_ticks: int, active: torch.Tensor, acc: torch.Tensor, jerk: torch.Tensor):
        self._order_inputs(active, acc, jerk)
        _check(lib.nb_correct(self._ctx, int(t_ticks), _dptr(active), active.numel(),
                              _dptr(acc), _dptr(jerk)), "nb_correct")

    def step(self, n_steps: int = 1, report: bool = False):
        """n_steps block steps (asynchronous).  With ``report`` the call waits
        and returns (smallest cluster time in ticks, particles corrected in
        the last step)."""
        if not report:
            _check(lib.nb_step_block(self._ctx, int(n_steps), None, None), "nb_step_block")
            return None
        t, m = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.nb_step_block(self._ctx, int(n_steps), ctypes.byref(t), ctypes.byref(m)),
               "nb_step_block")
        return t.value, m.value

    def leapfrog(self, n_steps: int, dt_ticks: int):
        """Kick-drift-kick leapfrog, shared step of ``dt_ticks`` ticks."""
        _check(lib.nb_step_leapfrog(self._ctx, int(n_steps), int(dt_ticks)), "nb_step_leapfrog")

    def set_end_time(self, t_end_ticks: int):
        _check(lib.nb_set_end_time(self._ctx, int(t_end_ticks)), "nb_set_end_time")

    # -- host-synchronising calls -----------------------------------------
    def energy(self, cluster: int = -1):
        ek, ep = ctypes.c_double(), ctypes.c_double()
        _check(lib.nb_energy(self._ctx, int(cluster), ctypes.byref(ek), ctypes.byref(ep)),
               "nb_energy")
        return ek.value, ep.value

    def energies(self):
        """(ekin[K], epot[K]) of every cluster from one potential evaluation."""
        ek = np.empty(self.n_clusters)
        ep = np.empty(self.n_clusters)
        _check(lib.nb_energies(self._ctx, _hptr(ek), _hptr(ep)), "nb_energies")
        return ek, ep

    def autotune(self, cache_path: str | None = None):
        """The autotune table of (shape, i-split) per ceil(log2 m), measured
        on this context or loaded from ``cache_path`` (nb_autotune); returns
        (shape of the largest bucket, {variant: [ms at m = every 4^k-th
        slot, k = 0 ..]}, all zero when the table came from the cache)."""
        v = ctypes.c_int32()
        ms = np.zeros(TUNE_POINTS * MIXED_VARIANTS)
        path = None if cache_path is None else os.fsencode(cache_path)
        _check(lib.nb_autotune(self._ctx, path, ctypes.byref(v), _hptr(ms)), "nb_autotune")
        self.cfg.variant = v.value
        ms = ms.reshape(TUNE_POINTS, MIXED_VARIANTS)
        return v.value, {k: ms[:, k].tolist() for k in range(MIXED_VARIANTS)}

    def profile_kernels(self):
        """{kind: (device ms, launches)} of every kind of launch since the
        previous call, while profiling is on (nb_profile_kernels)."""
        ms = np.zeros(len(PROFILE_KINDS))
        n = np.zeros(len(PROFILE_KINDS), dtype=np.int64)
        _check(lib.nb_profile_kernels(self._ctx, _hptr(ms), _hptr(n)), "nb_profile_kernels")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(PROFILE_KINDS)}

    def tune_table(self):
        """(shape, B) per ceil(log2 m) bucket: two int32 arrays (nb_tune_table)."""
        v = np.empty(TUNE_BUCKETS, dtype=np.int32)
        b = np.empty(TUNE_BUCKETS, dtype=np.int32)
        _check(lib.nb_tune_table(self._ctx, _hptr(v), _hptr(b)), "nb_tune_table")
        return v, b

    def get_state(self):
        n = self.n
        pos, vel, acc, jerk = (np.empty((n, 3)) for _ in range(4))
        t = np.empty(n, dtype=np.int64)
        level = np.empty(n, dtype=np.int32)
        _check(lib.nb_get_state(self._ctx, _hptr(pos), _hptr(vel), _hptr(acc), _hptr(jerk),
                                _hptr(t), _hptr(level)), "nb_get_state")
        return dict(pos=pos, vel=vel, acc=acc, jerk=jerk, t=t, level=level)

    def set_state(self, pos, vel, acc, jerk, t, level):
        n = self.n
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(n, 3) for a in (pos, vel, acc, jerk)]
        t = np.ascontiguousarray(t, dtype=np.int64).reshape(n)
        level = np.ascontiguousarray(level, dtype=np.int32).reshape(n)
        _check(lib.nb_set_state(self._ctx, *[_hptr(a) for a in arrs], _hptr(t), _hptr(level)),
               "nb_set_state")

    def stats(self) -> Stats:
        v = [ctypes.c_int64() for _ in range(4)]
        _check(lib.nb_stats(self._ctx, *[ctypes.byref(x) for x in v]), "nb_stats")
        return Stats(*[x.value for x in v])

    def profile(self, enable: bool = True):
        """Bracket every force-kernel launch with CUDA events (no graphs meanwhile)."""
        _check(lib.nb_profile_enable(self._ctx, int(bool(enable))), "nb_profile_enable")

    def profile_read(self):
        """(force-kernel milliseconds, launches) since the previous read."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib.nb_profile_read(self._ctx, ctypes.byref(ms), ctypes.byref(n)),
               "nb_profile_read")
        return ms.value, n.value

    def get_state_into(self, pos, vel, acc, jerk, t, level):
        """nb_get_state into caller-provided (e.g. pinned) numpy arrays."""
        _check(lib.nb_get_state(self._ctx, *[None if a is None else _hptr(a)
                                             for a in (pos, vel, acc, jerk, t, level)]),
               "nb_get_state")

    def tile_stats(self):
        """(warp-tiles, of which near) of the mixed force kernel since nb_init."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.nb_tile_stats(self._ctx, ctypes.byref(a), ctypes.byref(b)), "nb_tile_stats")
        return a.value, b.value

    def measure_rate(self, kind: int = 0) -> float:
        """nb_measure_rate: FMA lanes per SM per clock of this GPU (kind 0:
        f32x2, 1: FP32, 2: FP64)."""
        v = ctypes.c_double()
        _check(lib.nb_measure_rate(self._ctx, int(kind), ctypes.byref(v)), "nb_measure_rate")
        return v.value

    def status(self) -> int:
        return int(lib.nb_status(self._ctx))

    def check_wait_timeout(self, seconds: float = 0.05):
        """nb_check_wait_timeout: a device wait that runs out on purpose."""
        _check(lib.nb_check_wait_timeout(self._ctx, float(seconds)), "nb_check_wait_timeout")

    def clear_status(self):
        _check(lib.nb_clear_status(self._ctx), "nb_clear_status")

    def synchronize(self):
        self.stream.synchronize()

    # -- stream ordering between torch's current stream and the library's --
    def _order_inputs(self, *tensors):
        cur = torch.cuda.current_stream()
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)
        for t in tensors:
            if t is not None:
                t.record_stream(self.stream)

    def _order_outputs(self, *tensors):
        cur = torch.cuda.current_stream()
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)


NOALLOC_MAX_SOURCES = 32768


def force_noalloc(pos, vel, mass, targets, G=1.0, eps=1e-4, precision=NB_MIXED,
                  acc=None, jerk=None, pot=None, want_pot=True, stream=None):
    """nb_force_noalloc: forces from plain CUDA tensors, with no workspace.

    For callers that cannot allocate device memory at the call site: the
    library keeps its scratch in a fixed device array.  ``pos``/``vel``
    (n, 3) and ``mass`` (n,) float64 CUDA tensors, ``targets`` int32 CUDA
    tensor; outputs may be passed in (as the no-allocation caller would) or
    are created here for convenience.
    """
    n = mass.numel()
    m = targets.numel()
    for t, dt in ((pos, torch.float64), (vel, torch.float64), (mass, torch.float64),
                  (targets, torch.int32)):
        if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            raise ValueError("inputs must be contiguous CUDA tensors (float64 / int32)")
    if acc is None:
        acc = torch.empty((m, 3), dtype=torch.float64, device=pos.device)
    if jerk is None:
        jerk = torch.empty((m, 3), dtype=torch.float64, device=pos.device)
    if pot is None and want_pot:
        pot = torch.empty(m, dtype=torch.float64, device=pos.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib.nb_force_noalloc(_dptr(pos), _dptr(vel), _dptr(mass), n, _dptr(targets), m,
                                float(G), float(eps), int(precision), _dptr(acc), _dptr(jerk),
                                _dptr(pot), ctypes.c_void_p(st.cuda_stream)),
           "nb_force_noalloc")
    return acc, jerk, pot


def noalloc_status(stream=None) -> int:
    """nb_noalloc_status: the device status (NB_OK or an NB_E* code) of the
    last force_noalloc call on ``stream`` (synchronises it)."""
    st = stream if stream is not None else torch.cuda.current_stream()
    return int(lib.nb_noalloc_status(ctypes.c_void_p(st.cuda_stream)))
