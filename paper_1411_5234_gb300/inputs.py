"""Seeded synthetic inputs: star-cluster initial conditions and active sets.

This module holds only input generation -- no force, integrator or energy
arithmetic -- and is the one module that both the GPU library's callers and
the CPU oracle's callers share.  It uses its own counter-based generator
(SplitMix64, Steele, Lea & Flood 2014) so that the same seed gives the same
particles on every machine and numpy version.

Workloads (the paper integrates star clusters of 3.2e4..8e6 bodies and shows
a N ~ 260,000 cluster in Fig. 1; it names no dataset):
  * Plummer sphere (Aarseth, Henon & Wielen 1974 sampling), Henon units
    G = M = 1 via the analytic scaling (length x 3 pi / 16), centre-of-mass
    frame; equal masses or Kroupa (2001) broken power-law masses in
    [0.1, 100] renormalised to M = 1;
  * primordial binaries: a fraction of the bodies paired in Kepler orbits
    with log-uniform semi-major axis and thermal eccentricity f(e) = 2e;
  * batches of independent clusters with log-uniform sizes;
  * uniform random active subsets (sorted indices).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (finaliser) on a uint64 array."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


class Stream:
    """Counter-based uniform stream: u_k = mix64(key + (k + 1) * gamma)."""

    def __init__(self, seed: int, stream: int = 0):
        key = _mix64(np.array([(seed * 0x100000001B3 + stream) & 0xFFFFFFFFFFFFFFFF],
                              dtype=np.uint64))[0]
        self.key = np.uint64(key)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix64(self.key + k * _GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform_open(self, n: int) -> np.ndarray:
        """Doubles in (0, 1)."""
        return ((self.u64(n) >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


@dataclass
class Cluster:
    """Host-side initial conditions of one or more independent clusters."""
    pos: np.ndarray      # (n, 3) float64
    vel: np.ndarray      # (n, 3) float64
    mass: np.ndarray     # (n,) float64
    offsets: np.ndarray  # (n_clusters + 1,) int64; cluster k = [off[k], off[k+1])

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])

    @property
    def n_clusters(self) -> int:
        return int(self.offsets.shape[0] - 1)


def _isotropic(st: Stream, n: int) -> np.ndarray:
    cth = 2.0 * st.uniform(n) - 1.0
    phi = 2.0 * math.pi * st.uniform(n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def kroupa_masses(n: int, st: Stream, mlo=0.1, mbreak=0.5, mhi=100.0) -> np.ndarray:
    """Kroupa (2001) IMF: dN/dm ~ m^-1.3 on [mlo, mbreak), m^-2.3 on [mbreak, mhi].

    Inverse-CDF sampling of each power-law segment; the segments join
    continuously at ``mbreak``.  Returns raw masses (not normalised).
    """
    a1, a2 = 1.3, 2.3
    k1 = 1.0
    k2 = k1 * mbreak ** (a2 - a1)          # continuity at the break
    w1 = k1 * (mlo ** (1 - a1) - mbreak ** (1 - a1)) / (a1 - 1)
    w2 = k2 * (mbreak ** (1 - a2) - mhi ** (1 - a2)) / (a2 - 1)
    pick = st.uniform(n)
    u = st.uniform(n)
    first = pick < w1 / (w1 + w2)
    out = np.empty(n)

    def seg(lo, hi, alpha, uu):
        p = 1.0 - alpha
        return (lo ** p + uu * (hi ** p - lo ** p)) ** (1.0 / p)

    out[first] = seg(mlo, mbreak, a1, u[first])
    out[~first] = seg(mbreak, mhi, a2, u[~first])
    return out


def _plummer_raw(n: int, st: Stream):
    """Plummer sphere with scale length 1 and G = M = 1 (AHW 1974)."""
    # radius from the cumulative mass fraction X = r^3 / (1 + r^2)^(3/2);
    # X is cut at 0.999 to drop the far tail.
    X = 0.999 * st.uniform_open(n)
    r = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    pos = r[:, None] * _isotropic(st, n)
    # speed: q = v / v_esc from g(q) = q^2 (1 - q^2)^(7/2) by rejection
    # (the maximum of g is below 0.1), v_esc = sqrt(2) (1 + r^2)^(-1/4)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x = st.uniform(todo.size)
        y = 0.1 * st.uniform(todo.size)
        ok = y < x * x * (1.0 - x * x) ** 3.5
        q[todo[ok]] = x[ok]
        todo = todo[~ok]
    speed = q * math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    vel = speed[:, None] * _isotropic(st, n)
    return pos, vel


def _to_henon_cm(pos, vel, mass):
    """Henon units (E = -1/4 for the continuous Plummer model) + CM frame."""
    s = 3.0 * math.pi / 16.0
    pos = pos * s
    vel = vel / math.sqrt(s)
    mt = mass.sum()
    pos = pos - (mass[:, None] * pos).sum(0) / mt
    vel = vel - (mass[:, None] * vel).sum(0) / mt
    return pos, vel


def plummer(n: int, seed: int = 0, imf: str = "equal") -> Cluster:
    """One Plummer cluster of ``n`` bodies, total mass 1, Henon units."""
    if n < 1:
        raise ValueError("n must be >= 1")
    st = Stream(seed, 1)
    pos, vel = _plummer_raw(n, st)
    if imf == "equal":
        mass = np.full(n, 1.0 / n)
    elif imf == "kroupa":
        mass = kroupa_masses(n, Stream(seed, 2))
        mass = mass / mass.sum()
    else:
        raise ValueError(f"unknown imf {imf!r}")
    pos, vel = _to_henon_cm(pos, vel, mass)
    return Cluster(pos, vel, mass, np.array([0, n], dtype=np.int64))


def _solve_kepler(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Eccentric anomaly E from M = E - e sin E (Newton, fixed 50 iterations)."""
    E = np.where(e < 0.8, M, math.pi)
    for _ in range(50):
        E = E - (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
    return E


def _random_rotation(st: Stream, n: int) -> np.ndarray:
    """Uniform random rotation matrices (via uniform unit quaternions, Shoemake)."""
    u1, u2, u3 = st.uniform(n), st.uniform(n), st.uniform(n)
    a = np.sqrt(1 - u1) * np.sin(2 * math.pi * u2)
    b = np.sqrt(1 - u1) * np.cos(2 * math.pi * u2)
    c = np.sqrt(u1) * np.sin(2 * math.pi * u3)
    d = np.sqrt(u1) * np.cos(2 * math.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (c * c + d * d)
    R[:, 0, 1] = 2 * (b * c - a * d)
    R[:, 0, 2] = 2 * (b * d + a * c)
    R[:, 1, 0] = 2 * (b * c + a * d)
    R[:, 1, 1] = 1 - 2 * (b * b + d * d)
    R[:, 1, 2] = 2 * (c * d - a * b)
    R[:, 2, 0] = 2 * (b * d - a * c)
    R[:, 2, 1] = 2 * (c * d + a * b)
    R[:, 2, 2] = 1 - 2 * (b * b + c * c)
    return R


def plummer_binaries(n: int, seed: int = 0, binary_fraction: float = 0.1,
                     a_min: float = 1e-4, a_max: float = 1e-2) -> Cluster:
    """Plummer cluster where ``binary_fraction`` of the bodies are in binaries.

    floor(binary_fraction * n / 2) pairs of equal-mass members (1/n each);
    the pair's centre of mass is a Plummer body of mass 2/n.  Semi-major axis
    log-uniform in [a_min, a_max], eccentricity e = sqrt(U) (f(e) = 2e),
    uniform mean anomaly, isotropic orientation.  Binary members are stored
    next to each other after the single stars.
    """
    nb = int(math.floor(binary_fraction * n / 2))
    ns = n - 2 * nb
    nsys = ns + nb
    st = Stream(seed, 3)
    pos, vel = _plummer_raw(nsys, st)
    msys = np.full(nsys, 1.0 / n)
    msys[ns:] = 2.0 / n
    pos, vel = _to_henon_cm(pos, vel, msys)
    sb = Stream(seed, 4)
    a = np.exp(math.log(a_min) + sb.uniform(nb) * (math.log(a_max) - math.log(a_min)))
    e = np.sqrt(sb.uniform(nb))
    M = 2 * math.pi * sb.uniform(nb)
    E = _solve_kepler(M, e)
    mb = msys[ns:]  # total mass of each pair (G = 1)
    # relative orbit in the orbital plane
    x = a * (np.cos(E) - e)
    y = a * np.sqrt(1 - e * e) * np.sin(E)
    rr = a * (1 - e * np.cos(E))
    n_mean = np.sqrt(mb / a ** 3)
    vx = -a * n_mean * np.sin(E) * a / rr
    vy = a * n_mean * np.sqrt(1 - e * e) * np.cos(E) * a / rr
    rel = np.stack([x, y, np.zeros(nb)], 1)
    vrel = np.stack([vx, vy, np.zeros(nb)], 1)
    R = _random_rotation(sb, nb)
    rel = np.einsum("kij,kj->ki", R, rel)
    vrel = np.einsum("kij,kj->ki", R, vrel)
    out_p = np.empty((n, 3))
    out_v = np.empty((n, 3))
    out_p[:ns] = pos[:ns]
    out_v[:ns] = vel[:ns]
    # equal members: each sits at -/+ rel/2 from the pair's centre of mass
    out_p[ns::2] = pos[ns:] - 0.5 * rel
    out_p[ns + 1::2] = pos[ns:] + 0.5 * rel
    out_v[ns::2] = vel[ns:] - 0.5 * vrel
    out_v[ns + 1::2] = vel[ns:] + 0.5 * vrel
    mass = np.full(n, 1.0 / n)
    return Cluster(out_p, out_v, mass, np.array([0, n], dtype=np.int64))


def batch_sizes(n_clusters: int, n_min: int = 256, n_max: int = 16384,
                seed0: int = 0) -> np.ndarray:
    """Cluster sizes log-uniform in [n_min, n_max]; cluster k uses seed seed0 + k."""
    sizes = np.empty(n_clusters, dtype=np.int64)
    for k in range(n_clusters):
        u = Stream(seed0 + k, 5).uniform(1)[0]
        sizes[k] = int(round(math.exp(math.log(n_min) + u * (math.log(n_max) - math.log(n_min)))))
    return sizes


def plummer_batch(n_clusters: int, n_min: int = 256, n_max: int = 16384,
                  seed0: int = 0, imf: str = "equal") -> Cluster:
    """Independent Plummer clusters concatenated; cluster k from seed seed0 + k."""
    sizes = batch_sizes(n_clusters, n_min, n_max, seed0)
    parts = [plummer(int(s), seed0 + k, imf) for k, s in enumerate(sizes)]
    offsets = np.zeros(n_clusters + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return Cluster(np.concatenate([p.pos for p in parts]),
                   np.concatenate([p.vel for p in parts]),
                   np.concatenate([p.mass for p in parts]), offsets)


def random_active(n: int, m: int, seed: int = 0) -> np.ndarray:
    """Uniform random subset of m indices out of n, sorted ascending (int32)."""
    if not 0 <= m <= n:
        raise ValueError("need 0 <= m <= n")
    if m == n:
        return np.arange(n, dtype=np.int32)
    keys = Stream(seed, 6).u64(n)
    pick = np.argsort(keys, kind="stable")[:m]
    return np.sort(pick).astype(np.int32)


def random_vectors(n: int, scale: float, seed: int = 0, lo: float = 0.0) -> np.ndarray:
    """n isotropic vectors with lengths uniform in [lo, scale) (n x 3 float64):
    synthetic stand-ins for state a test sets directly (e.g. the acceleration
    and jerk at the start of a step)."""
    st = Stream(seed, 7)
    return _isotropic(st, n) * (lo + (scale - lo) * st.uniform(n))[:, None]


def morton_order(pos: np.ndarray, bits: int = 21) -> np.ndarray:
    """Permutation that sorts points along a 3-D Morton (Z-order) curve."""
    lo = pos.min(0)
    span = float(max((pos.max(0) - lo).max(), 1e-300))
    q = np.floor((pos - lo) / span * ((1 << bits) - 1)).astype(np.uint64)
    code = np.zeros(pos.shape[0], dtype=np.uint64)
    for b in range(bits):
        for c in range(3):
            code |= ((q[:, c] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + c)
    return np.argsort(code, kind="stable")


def reorder(cl: Cluster, perm: np.ndarray) -> Cluster:
    """Apply a permutation inside each cluster (perm indexes the whole set)."""
    return Cluster(cl.pos[perm], cl.vel[perm], cl.mass[perm], cl.offsets.copy())
