"""Seeded synthetic initial conditions (inputs only; no force or integrator math).

Both the CUDA path and the oracle are fed from this module, so it holds none
of the method's arithmetic: it draws random numbers, samples the Plummer
model and the Salpeter mass function, and scales to standard N-body units.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), used as a
counter-based generator: draw ``c`` of stream ``seed`` is the SplitMix64
output for state ``mix64(seed) + (c + 1) * GAMMA``.  Everything is
vectorised numpy uint64 arithmetic and gives the same bits on every machine.

Workloads follow Sec. 4 and Sec. 5 of the paper: Plummer models in standard
N-body units (G = M = r_v = 1, i.e. E = -1/4 for the virialised model), the
softening eps = 4/N unless a configuration states another value.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_DRAWS_PER_PARTICLE = 1 << 16  # counter stride between particles


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (published finaliser)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def u64(seed: int, counter) -> np.ndarray:
    """Raw 64-bit draw number ``counter`` of stream ``seed``."""
    key = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = key + (c + np.uint64(1)) * GAMMA
    return _mix64(state)


def uniform(seed: int, counter) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1): (k + 0.5) * 2^-53."""
    k = (u64(seed, counter) >> np.uint64(11)).astype(np.float64)
    return (k + 0.5) * (2.0 ** -53)


class _Streams:
    """Per-particle draw counters so rejection loops stay reproducible."""

    def __init__(self, seed: int, n: int):
        self.seed = seed
        self.base = np.arange(n, dtype=np.uint64) * np.uint64(_DRAWS_PER_PARTICLE)
        self.next = np.zeros(n, dtype=np.uint64)

    def draw(self, sel: np.ndarray) -> np.ndarray:
        c = self.base[sel] + self.next[sel]
        if np.any(self.next[sel] >= np.uint64(_DRAWS_PER_PARTICLE)):
            raise RuntimeError("random stream exhausted")
        self.next[sel] += np.uint64(1)
        return uniform(self.seed, c)


def _isotropic(st: _Streams, sel: np.ndarray, radius: np.ndarray) -> np.ndarray:
    x2 = st.draw(sel)
    x3 = st.draw(sel)
    z = (1.0 - 2.0 * x2) * radius
    rho = np.sqrt(np.maximum(radius * radius - z * z, 0.0))
    phi = 2.0 * math.pi * x3
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def plummer(n: int, seed: int, r_max: float = 10.0, masses=None):
    """Plummer sphere, Aarseth, Henon & Wielen (1974) sampling.

    In model units (scale radius 1, M = G = 1): the radius follows from the
    cumulative mass fraction X, r = (X^(-2/3) - 1)^(-1/2), rejected beyond
    ``r_max``; the speed is q times the local escape speed
    sqrt(2) (1 + r^2)^(-1/4), with q drawn by von Neumann rejection against
    g(q) = q^2 (1 - q^2)^(7/2) (bound 0.1); directions are isotropic.  The
    model is shifted to its centre of mass and scaled to standard N-body
    units (length x 3 pi/16, velocity x sqrt(16 / (3 pi))), so that the total
    energy is -1/4 up to sampling noise.

    Returns (m, r, v): m (n,), r and v (n, 3), float64.
    """
    if n <= 0:
        return np.zeros(0), np.zeros((0, 3)), np.zeros((0, 3))
    st = _Streams(seed, n)
    radius = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x1 = st.draw(todo)
        rr = 1.0 / np.sqrt(x1 ** (-2.0 / 3.0) - 1.0)
        ok = rr <= r_max
        radius[todo[ok]] = rr[ok]
        todo = todo[~ok]
    pos = _isotropic(st, np.arange(n), radius)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x4 = st.draw(todo)
        x5 = st.draw(todo)
        ok = 0.1 * x5 < x4 * x4 * (1.0 - x4 * x4) ** 3.5
        q[todo[ok]] = x4[ok]
        todo = todo[~ok]
    speed = q * math.sqrt(2.0) * (1.0 + radius * radius) ** (-0.25)
    vel = _isotropic(st, np.arange(n), speed)
    if masses is None:
        m = np.full(n, 1.0 / n)
    else:
        m = np.ascontiguousarray(masses, dtype=np.float64)
    mt = m.sum()
    pos -= (m[:, None] * pos).sum(axis=0) / mt
    vel -= (m[:, None] * vel).sum(axis=0) / mt
    lscale = 3.0 * math.pi / 16.0
    pos *= lscale
    vel *= 1.0 / math.sqrt(lscale)
    return m, np.ascontiguousarray(pos), np.ascontiguousarray(vel)


def salpeter_masses(n: int, seed: int, slope: float = 2.35, m_lo: float = 0.1,
                    m_hi: float = 10.0) -> np.ndarray:
    """dN/dm ~ m^-slope on [m_lo, m_hi] by inverse-CDF sampling, sum = 1."""
    u = uniform(seed, np.arange(n, dtype=np.uint64) + np.uint64(1 << 40))
    p = 1.0 - slope
    lo, hi = m_lo ** p, m_hi ** p
    m = (lo + u * (hi - lo)) ** (1.0 / p)
    return m / m.sum()


def permutation(n: int, seed: int) -> np.ndarray:
    """Seeded random permutation of range(n) (argsort of 64-bit draws)."""
    keys = u64(seed, np.arange(n, dtype=np.uint64) + np.uint64(1 << 41))
    return np.argsort(keys, kind="stable").astype(np.int64)


def ensemble_sizes(k: int, seed: int, n_lo: int = 256, n_hi: int = 8192):
    """Cluster sizes log-uniform in [n_lo, n_hi]."""
    u = uniform(seed, np.arange(k, dtype=np.uint64) + np.uint64(1 << 42))
    return np.rint(np.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))
                   ).astype(np.int64)


@dataclass(frozen=True)
class Workload:
    """One of the five benchmark workloads (Plummer, standard N-body units)."""
    name: str
    n: int
    seed: int
    eps: float
    eta: float = 0.02
    eta_start: float = 0.01
    dt_max: float = 1.0 / 16
    t_end: float = 1.0
    precision: str = "mixed"
    salpeter: bool = False

    def particles(self):
        masses = salpeter_masses(self.n, self.seed) if self.salpeter else None
        return plummer(self.n, self.seed, masses=masses)


# The five workloads the library is measured on.
FP64_N1K = Workload("plummer_n1024_fp64_t0.5", 1024, 1, 1.0 / 64, t_end=0.5,
                    precision="fp64")
FORCE_SWEEP_N16K = Workload("plummer_n16384_force_sweep", 16384, 2, 1.0 / 256,
                            t_end=0.0)
FORCE_SWEEP_NACT = (32, 256, 2048, 16384)
MIXED_N64K = Workload("plummer_n65536_mixed_t1", 65536, 3, 4.0 / 65536)
ENSEMBLE_K256 = dict(name="ensemble_256_plummer_n256_8192", k=256, size_seed=4,
                     member_seed0=1000, eta=0.02, eta_start=0.01,
                     dt_max=1.0 / 16, t_end=1.0)
SALPETER_N256K = Workload("plummer_salpeter_n262144_mixed_t0.25", 262144, 5,
                          1e-4, t_end=0.25, salpeter=True)


def ensemble(k: int = 256, size_seed: int = 4, member_seed0: int = 1000,
             n_lo: int = 256, n_hi: int = 8192):
    """Independent Plummer clusters: sizes, offsets, m, r, v, eps_k = 4 / N_k."""
    sizes = ensemble_sizes(k, size_seed, n_lo, n_hi)
    offsets = np.zeros(k + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    ms, rs, vs = [], [], []
    for c in range(k):
        m, r, v = plummer(int(sizes[c]), member_seed0 + c)
        ms.append(m)
        rs.append(r)
        vs.append(v)
    eps = 4.0 / sizes.astype(np.float64)
    return (sizes, offsets, np.concatenate(ms), np.concatenate(rs),
            np.concatenate(vs), eps)


def gate_sample(r: np.ndarray, seed: int, n_random: int = 256, n_central: int = 64) -> np.ndarray:
    """Particles an accuracy check samples at sizes where every particle would
    be too slow for the oracle: `n_random` drawn by a seeded permutation and
    the `n_central` closest to the origin (the densest region, where near
    neighbours cancel most), ascending, without repeats."""
    n = len(r)
    central = np.argsort(np.einsum("ij,ij->i", r, r), kind="stable")[:n_central]
    pick = np.concatenate([permutation(n, seed)[:n_random], central])
    return np.unique(pick).astype(np.int32)


def ensemble_subset(count: int = 16, n_max: int = 2048, **kw):
    """`count` members of the ensemble workload, drawn by a seeded permutation
    from those with N <= n_max: (member numbers, offsets, m, r, v, eps) of
    the sub-ensemble, members in ascending order."""
    sizes, off, ms, rs, vs, eps = ensemble(**kw)
    small = [q for q in range(len(sizes)) if sizes[q] <= n_max]
    pick = sorted(small[i] for i in permutation(len(small), 16)[:count])
    sub_off = np.zeros(count + 1, dtype=np.int64)
    sub_off[1:] = np.cumsum([sizes[q] for q in pick])

    def cat(a):
        return np.concatenate([a[off[q]:off[q + 1]] for q in pick])

    return pick, sub_off, cat(ms), cat(rs), cat(vs), np.array([eps[q] for q in pick])
