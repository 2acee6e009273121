"""FP64 CPU oracle for the direct N-body method -- TEST INFRASTRUCTURE ONLY.

The oracle is a plain C restatement of the paper's definitions (Eq. 1, Eq. 2,
the Hermite integrator of Sec. 2 item 1 and the power-of-two block time steps
of Sec. 2 item 2), compiled with gcc (no -ffast-math, no FMA contraction) and
called through ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the GPU library (``paper_1411_5234_gb300``) and neither imports the other.

Arrays are numpy, float64 ``(n, 3)`` for vectors, int64 ticks for times
(a tick is ``2**-tick_exp`` time units) and int32 levels (``dt = 2**-level``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_nbody.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C source into a shared library (idempotent)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # NBODY_ORACLE_LIB points the wrapper at another build of the same C
        # source (the mutation tests use it to load deliberately broken copies)
        path = os.environ.get("NBODY_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.oracle_force.argtypes = [i64, P, P, P, f64, f64, i64, P, P, P, P]
        lib.oracle_force.restype = i32
        lib.oracle_energy.argtypes = [i64, P, P, P, f64, f64, P, P]
        lib.oracle_energy.restype = None
        lib.oracle_momenta.argtypes = [i64, P, P, P, P, P]
        lib.oracle_momenta.restype = None
        lib.oracle_predict.argtypes = [i64, P, P, P, P, P, P, P]
        lib.oracle_predict.restype = None
        lib.oracle_correct.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_correct.restype = None
        lib.oracle_aarseth_dt.argtypes = [P, P, P, P, f64]
        lib.oracle_aarseth_dt.restype = f64
        lib.oracle_initial_dt.argtypes = [P, P, f64]
        lib.oracle_initial_dt.restype = f64
        lib.oracle_level.argtypes = [f64, i32, i64, i32, i32, i32]
        lib.oracle_level.restype = i32
        lib.oracle_block_step.argtypes = [i64, P, P, P, P, P, P, P, f64, f64,
                                          f64, i32, i32, i32, P, P, P, P]
        lib.oracle_block_step.restype = i32
        lib.oracle_init.argtypes = [i64, P, P, P, P, P, P, P, f64, f64, f64,
                                    i32, i32, i32]
        lib.oracle_init.restype = i32
        lib.oracle_kick.argtypes = [i64, P, P, f64]
        lib.oracle_kick.restype = None
        lib.oracle_drift.argtypes = [i64, P, P, f64]
        lib.oracle_drift.restype = None
        lib.oracle_leapfrog.argtypes = [i64, P, P, P, P, f64, f64, f64, i64]
        lib.oracle_leapfrog.restype = i32
        lib.oracle_force_snap.argtypes = [i64, P, P, P, P, f64, f64, i64, P, P, P, P]
        lib.oracle_force_snap.restype = i32
        lib.oracle_hermite6_correct.argtypes = [i64] + [P] * 14
        lib.oracle_hermite6_correct.restype = None
        lib.oracle_hermite6_dt.argtypes = [P, P, P, P, P, P, f64]
        lib.oracle_hermite6_dt.restype = f64
        lib.oracle_hermite6_predict.argtypes = [i64] + [P] * 10
        lib.oracle_hermite6_predict.restype = None
        lib.oracle_hermite6_run.argtypes = [i64, P, P, P, f64, f64, f64, i64]
        lib.oracle_hermite6_run.restype = i32
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = i32
        lib.oracle_set_threads.argtypes = [i32]
        lib.oracle_set_threads.restype = None
        _lib = lib
        return lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def force(pos, vel, mass, eps, idx=None, G=1.0):
    """Acceleration, jerk and potential of targets ``idx`` from all sources.

    Eq. 1 with the softening of Eq. 2; the j == i term is excluded by index.
    Returns ``(acc (m,3), jerk (m,3), pot (m,))``.
    """
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    vel = _f64(vel, (n, 3))
    mass = _f64(mass, (n,))
    if idx is None:
        idx = np.arange(n, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m = idx.shape[0]
    acc = np.empty((m, 3))
    jerk = np.empty((m, 3))
    pot = np.empty(m)
    rc = _load().oracle_force(n, _ptr(pos), _ptr(vel), _ptr(mass), float(G),
                              float(eps), m, _ptr(idx), _ptr(acc), _ptr(jerk),
                              _ptr(pot))
    if rc != 0:
        raise ValueError("oracle_force: target index out of range")
    return acc, jerk, pot


def energy(pos, vel, mass, eps, G=1.0):
    """(kinetic, softened potential) energy of the whole system."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    vel = _f64(vel, (n, 3))
    mass = _f64(mass, (n,))
    ek = ctypes.c_double()
    ep = ctypes.c_double()
    _load().oracle_energy(n, _ptr(pos), _ptr(vel), _ptr(mass), float(G),
                          float(eps), ctypes.byref(ek), ctypes.byref(ep))
    return ek.value, ep.value


def momenta(pos, vel, mass):
    """(angular momentum L (3,), linear momentum P (3,))."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    vel = _f64(vel, (n, 3))
    mass = _f64(mass, (n,))
    L = np.empty(3)
    P = np.empty(3)
    _load().oracle_momenta(n, _ptr(pos), _ptr(vel), _ptr(mass), _ptr(L),
                           _ptr(P))
    return L, P


def predict(pos, vel, acc, jerk, tau):
    """Hermite (Taylor) predictor to per-particle offsets ``tau``."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    args = [_f64(a, (n, 3)) for a in (vel, acc, jerk)]
    tau = _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (n,)))
    xp = np.empty((n, 3))
    vp = np.empty((n, 3))
    _load().oracle_predict(n, _ptr(pos), _ptr(args[0]), _ptr(args[1]),
                           _ptr(args[2]), _ptr(tau), _ptr(xp), _ptr(vp))
    return xp, vp


def correct(tau, xp, vp, a0, j0, a1, j1):
    """Hermite corrector.  Returns ``(x1, v1, a2_end, a3_end)``."""
    xp = _f64(xp).reshape(-1, 3)
    m = xp.shape[0]
    vp, a0, j0, a1, j1 = (_f64(a, (m, 3)) for a in (vp, a0, j0, a1, j1))
    tau = _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (m,)))
    out = [np.empty((m, 3)) for _ in range(4)]
    _load().oracle_correct(m, _ptr(tau), _ptr(xp), _ptr(vp), _ptr(a0),
                           _ptr(j0), _ptr(a1), _ptr(j1), *[_ptr(o) for o in out])
    return tuple(out)


def aarseth_dt(a, j, a2, a3, eta):
    a, j, a2, a3 = (_f64(x, (3,)) for x in (a, j, a2, a3))
    return float(_load().oracle_aarseth_dt(_ptr(a), _ptr(j), _ptr(a2),
                                           _ptr(a3), float(eta)))


def initial_dt(a, j, eta_s):
    a, j = (_f64(x, (3,)) for x in (a, j))
    return float(_load().oracle_initial_dt(_ptr(a), _ptr(j), float(eta_s)))


def level(dt_crit, level_old, t_new_ticks, tick_exp, lmin, lmax):
    return int(_load().oracle_level(float(dt_crit), int(level_old),
                                    int(t_new_ticks), int(tick_exp), int(lmin),
                                    int(lmax)))


def kick(vel, acc, h):
    """Leapfrog half kick: returns ``vel + h * acc`` (copies)."""
    vel = _f64(vel).reshape(-1, 3).copy()
    n = vel.shape[0]
    acc = _f64(acc, (n, 3))
    _load().oracle_kick(n, _ptr(vel), _ptr(acc), float(h))
    return vel


def drift(pos, vel, dt):
    """Leapfrog drift: returns ``pos + dt * vel`` (copies)."""
    pos = _f64(pos).reshape(-1, 3).copy()
    n = pos.shape[0]
    vel = _f64(vel, (n, 3))
    _load().oracle_drift(n, _ptr(pos), _ptr(vel), float(dt))
    return pos


def leapfrog(pos, vel, acc, mass, eps, dt, n_steps, G=1.0):
    """Kick-drift-kick leapfrog with a shared step ``dt`` for ``n_steps``
    steps, from positions, velocities and the acceleration at the start.
    Returns ``(pos, vel, acc)`` at the end (copies)."""
    pos = _f64(pos).reshape(-1, 3).copy()
    n = pos.shape[0]
    vel = _f64(vel, (n, 3)).copy()
    acc = _f64(acc, (n, 3)).copy()
    mass = _f64(mass, (n,))
    rc = _load().oracle_leapfrog(n, _ptr(pos), _ptr(vel), _ptr(acc), _ptr(mass),
                                 float(G), float(eps), float(dt), int(n_steps))
    if rc != 0:
        raise MemoryError("oracle_leapfrog")
    return pos, vel, acc


def force_snap(pos, vel, acc, mass, eps, idx=None, G=1.0):
    """Acceleration, jerk and snap of targets ``idx`` (the 6th-order scheme's
    force), from positions, velocities and accelerations of all particles.
    Returns ``(acc, jerk, snap)``, each (m, 3)."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    vel, acc = _f64(vel, (n, 3)), _f64(acc, (n, 3))
    mass = _f64(mass, (n,))
    idx = np.arange(n, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, np.int64)
    m = idx.shape[0]
    out = [np.empty((m, 3)) for _ in range(3)]
    rc = _load().oracle_force_snap(n, _ptr(pos), _ptr(vel), _ptr(acc), _ptr(mass), float(G),
                                   float(eps), m, _ptr(idx), *[_ptr(o) for o in out])
    if rc != 0:
        raise ValueError("oracle_force_snap: target index out of range")
    return tuple(out)


def hermite6_correct(h, x0, v0, a0, j0, s0, a1, j1, s1):
    """6th-order Hermite corrector.  Returns ``(x1, v1, crackle, pop, a5)``
    (the last three: the interpolant's derivatives at the end)."""
    x0 = _f64(x0).reshape(-1, 3)
    m = x0.shape[0]
    args = [_f64(a, (m, 3)) for a in (v0, a0, j0, s0, a1, j1, s1)]
    h = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (m,)))
    out = [np.empty((m, 3)) for _ in range(5)]
    _load().oracle_hermite6_correct(m, _ptr(h), _ptr(x0), *[_ptr(a) for a in args],
                                    *[_ptr(o) for o in out])
    return tuple(out)


def hermite6_predict(t, x, v, a, j, s, c):
    """Taylor predictor of the 6th-order scheme over t (scalar or per
    particle).  Returns ``(x_p, v_p, a_p)``, each (m, 3)."""
    x = _f64(x).reshape(-1, 3)
    m = x.shape[0]
    args = [_f64(y, (m, 3)) for y in (v, a, j, s, c)]
    t = _f64(np.broadcast_to(np.asarray(t, dtype=np.float64), (m,)))
    out = [np.empty((m, 3)) for _ in range(3)]
    _load().oracle_hermite6_predict(m, _ptr(t), _ptr(x), *[_ptr(y) for y in args],
                                    *[_ptr(o) for o in out])
    return tuple(out)


def hermite6_dt(a, j, s, c, p, q, eta):
    """Step criterion of the 6th-order scheme (generalised Aarseth, p = 6)."""
    vs = [_f64(x, (3,)) for x in (a, j, s, c, p, q)]
    return float(_load().oracle_hermite6_dt(*[_ptr(x) for x in vs], float(eta)))


def hermite6_run(pos, vel, mass, eps, h, n_steps, G=1.0):
    """Shared-step 6th-order Hermite integration; returns ``(pos, vel)``."""
    pos = _f64(pos).reshape(-1, 3).copy()
    n = pos.shape[0]
    vel = _f64(vel, (n, 3)).copy()
    mass = _f64(mass, (n,))
    rc = _load().oracle_hermite6_run(n, _ptr(pos), _ptr(vel), _ptr(mass), float(G),
                                     float(eps), float(h), int(n_steps))
    if rc != 0:
        raise MemoryError("oracle_hermite6_run")
    return pos, vel


class State:
    """FP64 particle state driven by the oracle's block-step integrator."""

    def __init__(self, pos, vel, mass, *, eps, eta=0.01, eta_s=0.01, G=1.0,
                 tick_exp=40, lmin=0, lmax=30):
        self.pos = _f64(pos).reshape(-1, 3).copy()
        self.n = self.pos.shape[0]
        self.vel = _f64(vel, (self.n, 3)).copy()
        self.mass = _f64(mass, (self.n,)).copy()
        self.eps, self.eta, self.eta_s, self.G = eps, eta, eta_s, G
        self.tick_exp, self.lmin, self.lmax = tick_exp, lmin, lmax
        self.acc = np.empty((self.n, 3))
        self.jerk = np.empty((self.n, 3))
        self.t = np.zeros(self.n, dtype=np.int64)
        self.level = np.zeros(self.n, dtype=np.int32)
        rc = _load().oracle_init(self.n, _ptr(self.pos), _ptr(self.vel),
                                 _ptr(self.mass), _ptr(self.acc),
                                 _ptr(self.jerk), _ptr(self.t),
                                 _ptr(self.level), float(G), float(eps),
                                 float(eta_s), tick_exp, lmin, lmax)
        if rc != 0:
            raise RuntimeError("oracle_init failed")

    def copy(self):
        c = object.__new__(State)
        c.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                           for k, v in self.__dict__.items()})
        return c

    def block_step(self):
        """One block step.  Returns ``(t_next_ticks, active_idx, dt_crit)``."""
        t_next = ctypes.c_int64()
        m = ctypes.c_int64()
        act = np.empty(self.n, dtype=np.int64)
        dtc = np.empty(self.n)
        rc = _load().oracle_block_step(
            self.n, _ptr(self.pos), _ptr(self.vel), _ptr(self.acc),
            _ptr(self.jerk), _ptr(self.mass), _ptr(self.t), _ptr(self.level),
            float(self.G), float(self.eps), float(self.eta), self.tick_exp,
            self.lmin, self.lmax, ctypes.byref(t_next), ctypes.byref(m),
            _ptr(act), _ptr(dtc))
        if rc != 0:
            raise RuntimeError("oracle_block_step failed")
        k = m.value
        return t_next.value, act[:k].copy(), dtc[:k].copy()

    def time(self) -> float:
        """Largest particle time (the current block time) in time units."""
        return float(np.ldexp(float(self.t.max()), -self.tick_exp))

    def energy_at_sync(self):
        """(ekin, epot) -- valid when every particle sits at the same time."""
        return energy(self.pos, self.vel, self.mass, self.eps, self.G)
