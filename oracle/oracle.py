"""ctypes wrapper of the plain FP64 CPU oracle (``hermite_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously correct
definition of the fourth-order Hermite block-timestep scheme (Sec. 2 of
arXiv:1104.2700) that the CUDA path is checked against.  Only the test
suite, the smoke check and the benchmark's CPU-baseline leg may import this
module.  It shares no code with the CUDA path and never imports it.

Arrays are numpy float64, C-contiguous; positions, velocities,
accelerations and jerks are (n, 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hermite_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libhermite_oracle.so")
_lock = threading.Lock()
_lib = None

# status codes of the C oracle
OK = 0
ENONFINITE = 4
EDTMIN = 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain FP64: no contraction, no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
           "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        P = ctypes.c_void_p
        lib.orc_force.argtypes = [i64, P, P, P, d, d, i64, P, P, P, P, i32]
        lib.orc_force.restype = None
        lib.orc_predict.argtypes = [i64, P, P, P, P, P, d, P, P]
        lib.orc_predict.restype = None
        lib.orc_hermite_correct.argtypes = [P, P, P, P, P, P, d, P, P, P, P]
        lib.orc_hermite_correct.restype = None
        lib.orc_aarseth_dt.argtypes = [d, P, P, P, P]
        lib.orc_aarseth_dt.restype = d
        lib.orc_pow2_floor.argtypes = [d]
        lib.orc_pow2_floor.restype = d
        lib.orc_quantize_dt.argtypes = [d, d, d, d, d, P]
        lib.orc_quantize_dt.restype = i32
        lib.orc_initial_dt.argtypes = [d, P, P, d, d, P]
        lib.orc_initial_dt.restype = i32
        lib.orc_select.argtypes = [i64, P, P, P, P]
        lib.orc_select.restype = i64
        lib.orc_energy.argtypes = [i64, P, P, P, d, d, P, P, i32]
        lib.orc_energy.restype = None
        lib.orc_init.argtypes = [i64, P, P, P, P, P, P, P, d, d, d, d, d, d, i32]
        lib.orc_init.restype = i32
        lib.orc_run.argtypes = [i64, P, P, P, P, P, P, P, d, d, d, d, d, d, i32,
                                i64, P, P]
        lib.orc_run.restype = i32
        lib.orc_has_openmp.argtypes = []
        lib.orc_has_openmp.restype = i32
        lib.orc_force_snap.argtypes = [i64, P, P, P, P, d, d, i64, P, P, P, P, P, i32]
        lib.orc_force_snap.restype = None
        lib.orc_predict6.argtypes = [i64, P, P, P, P, P, P, P, d, P, P, P]
        lib.orc_predict6.restype = None
        lib.orc_hermite6_correct.argtypes = [P, P, P, P, P, P, P, P, d, P, P, P, P, P]
        lib.orc_hermite6_correct.restype = None
        lib.orc_aarseth6_dt.argtypes = [d, P, P, P, P, P, P]
        lib.orc_aarseth6_dt.restype = d
        lib.orc_init6.argtypes = [i64, P, P, P, P, P, P, P, P, P, d, d, d, d, d, d, i32]
        lib.orc_init6.restype = i32
        lib.orc_run6.argtypes = [i64, P, P, P, P, P, P, P, P, P, d, d, d, d, d, d, i32,
                                 i64, P, P]
        lib.orc_run6.restype = i32
        _lib = lib
        return lib


def _f64(x, shape=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def has_openmp() -> bool:
    return bool(_load().orc_has_openmp())


def force(m, r, v, eps, G=1.0, idx=None, nthreads=1):
    """Eqs. acc, jrk, pot on the particles ``idx`` (default: all)."""
    lib = _load()
    m = _f64(m)
    n = m.shape[0]
    r = _f64(r, (n, 3))
    v = _f64(v, (n, 3))
    if idx is None:
        idx = np.arange(n, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    k = idx.shape[0]
    acc = np.empty((k, 3))
    jerk = np.empty((k, 3))
    pot = np.empty(k)
    lib.orc_force(n, _ptr(m), _ptr(r), _ptr(v), float(eps), float(G), k,
                  _ptr(idx), _ptr(acc), _ptr(jerk), _ptr(pot), int(nthreads))
    return acc, jerk, pot


def predict(r0, v0, a0, j0, t0, t):
    """Eqs. xpred, vpred for every particle to time ``t``."""
    lib = _load()
    t0 = _f64(t0)
    n = t0.shape[0]
    r0, v0, a0, j0 = (_f64(x, (n, 3)) for x in (r0, v0, a0, j0))
    rp = np.empty((n, 3))
    vp = np.empty((n, 3))
    lib.orc_predict(n, _ptr(r0), _ptr(v0), _ptr(a0), _ptr(j0), _ptr(t0),
                    float(t), _ptr(rp), _ptr(vp))
    return rp, vp


def hermite_correct(rp, vp, a0, j0, a1, j1, dt):
    """Sec. 2 snap, crackle and corrector for one particle (3-vectors)."""
    lib = _load()
    args = [_f64(x, (3,)) for x in (rp, vp, a0, j0, a1, j1)]
    r1, v1, s0, c0 = (np.empty(3) for _ in range(4))
    lib.orc_hermite_correct(*[_ptr(a) for a in args], float(dt), _ptr(r1),
                            _ptr(v1), _ptr(s0), _ptr(c0))
    return r1, v1, s0, c0


def aarseth_dt(eta, a, j, s, c):
    """Eq. timestep."""
    lib = _load()
    a, j, s, c = (_f64(x, (3,)) for x in (a, j, s, c))
    return lib.orc_aarseth_dt(float(eta), _ptr(a), _ptr(j), _ptr(s), _ptr(c))


def pow2_floor(x):
    return _load().orc_pow2_floor(float(x))


def quantize_dt(dt_old, dt_cand, t_next, dt_max, dt_min=2.0 ** -40):
    """Power-of-two timestep update; returns (status, dt_new)."""
    out = np.zeros(1)
    st = _load().orc_quantize_dt(float(dt_old), float(dt_cand), float(t_next),
                                 float(dt_max), float(dt_min), _ptr(out))
    return st, float(out[0])


def initial_dt(eta_start, a, j, dt_max, dt_min=2.0 ** -40):
    a, j = _f64(a, (3,)), _f64(j, (3,))
    out = np.zeros(1)
    st = _load().orc_initial_dt(float(eta_start), _ptr(a), _ptr(j),
                                float(dt_max), float(dt_min), _ptr(out))
    return st, float(out[0])


def select(t, dt):
    """Step 1: (t_next, active indices ascending)."""
    t, dt = _f64(t), _f64(dt)
    n = t.shape[0]
    idx = np.empty(max(n, 1), dtype=np.int64)
    tn = np.zeros(1)
    k = _load().orc_select(n, _ptr(t), _ptr(dt), _ptr(tn), _ptr(idx))
    return float(tn[0]), idx[:k].copy()


def energy(m, r, v, eps, G=1.0, nthreads=1):
    """(kinetic, potential) with the potential 1/2 sum m_i phi_i (Eq. pot)."""
    m = _f64(m)
    n = m.shape[0]
    r, v = _f64(r, (n, 3)), _f64(v, (n, 3))
    K, W = np.zeros(1), np.zeros(1)
    _load().orc_energy(n, _ptr(m), _ptr(r), _ptr(v), float(eps), float(G),
                       _ptr(K), _ptr(W), int(nthreads))
    return float(K[0]), float(W[0])


def force_snap(m, r, v, a, eps, G=1.0, idx=None, nthreads=1):
    """Acceleration, jerk, snap and potential on ``idx`` (default: all), the
    snap from the particles' predicted accelerations ``a`` (sixth-order
    variant)."""
    lib = _load()
    m = _f64(m)
    n = m.shape[0]
    r, v, a = _f64(r, (n, 3)), _f64(v, (n, 3)), _f64(a, (n, 3))
    if idx is None:
        idx = np.arange(n, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    k = idx.shape[0]
    acc, jerk, snap, pot = np.empty((k, 3)), np.empty((k, 3)), np.empty((k, 3)), np.empty(k)
    lib.orc_force_snap(n, _ptr(m), _ptr(r), _ptr(v), _ptr(a), float(eps), float(G), k,
                       _ptr(idx), _ptr(acc), _ptr(jerk), _ptr(snap), _ptr(pot), int(nthreads))
    return acc, jerk, snap, pot


def predict6(r0, v0, a0, j0, s0, c0, t0, t):
    """Sixth-order predictor of r, v, a to time ``t``."""
    lib = _load()
    t0 = _f64(t0)
    n = t0.shape[0]
    r0, v0, a0, j0, s0, c0 = (_f64(x, (n, 3)) for x in (r0, v0, a0, j0, s0, c0))
    rp, vp, ap = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
    lib.orc_predict6(n, _ptr(r0), _ptr(v0), _ptr(a0), _ptr(j0), _ptr(s0), _ptr(c0),
                     _ptr(t0), float(t), _ptr(rp), _ptr(vp), _ptr(ap))
    return rp, vp, ap


def hermite6_correct(r0, v0, a0, j0, s0, a1, j1, s1, h):
    """Sixth-order corrector for one particle: (r1, v1, crackle, pop, fifth
    derivative) at the end of a step ``h``."""
    lib = _load()
    args = [_f64(x, (3,)) for x in (r0, v0, a0, j0, s0, a1, j1, s1)]
    out = [np.empty(3) for _ in range(5)]
    lib.orc_hermite6_correct(*[_ptr(x) for x in args], float(h), *[_ptr(x) for x in out])
    return tuple(out)


def aarseth6_dt(eta, a, j, s, c, d, x):
    """The sixth-order timestep criterion (reading H2)."""
    vs = [_f64(q, (3,)) for q in (a, j, s, c, d, x)]
    return _load().orc_aarseth6_dt(float(eta), *[_ptr(q) for q in vs])


class State6:
    """Full state of one system under the sixth-order scheme (the oracle's copy)."""

    def __init__(self, m, r, v, eps, eta, G=1.0, eta_start=0.01, dt_max=1.0 / 16,
                 dt_min=2.0 ** -40, nthreads=1):
        self.m = _f64(m).copy()
        n = self.n = self.m.shape[0]
        self.r, self.v = _f64(r, (n, 3)).copy(), _f64(v, (n, 3)).copy()
        self.a, self.j, self.s, self.c = (np.empty((n, 3)) for _ in range(4))
        self.t, self.dt = np.empty(n), np.empty(n)
        self.eps, self.eta, self.G = float(eps), float(eta), float(G)
        self.dt_max, self.dt_min, self.nthreads = float(dt_max), float(dt_min), int(nthreads)
        self.n_steps, self.n_inter = 0, 0.0
        st = _load().orc_init6(n, _ptr(self.m), _ptr(self.r), _ptr(self.v), _ptr(self.a),
                               _ptr(self.j), _ptr(self.s), _ptr(self.c), _ptr(self.t),
                               _ptr(self.dt), 0.0, self.eps, self.G, float(eta_start),
                               self.dt_max, self.dt_min, self.nthreads)
        if st != OK:
            raise RuntimeError(f"oracle init failed with status {st}")

    def run(self, t_end, max_steps=0):
        steps, inter = np.zeros(1, dtype=np.int64), np.zeros(1)
        st = _load().orc_run6(self.n, _ptr(self.m), _ptr(self.r), _ptr(self.v), _ptr(self.a),
                              _ptr(self.j), _ptr(self.s), _ptr(self.c), _ptr(self.t),
                              _ptr(self.dt), float(t_end), self.eps, self.G, self.eta,
                              self.dt_max, self.dt_min, self.nthreads, int(max_steps),
                              _ptr(steps), _ptr(inter))
        self.n_steps += int(steps[0])
        self.n_inter += float(inter[0])
        return st

    def energy(self):
        K, W = energy(self.m, self.r, self.v, self.eps, self.G, self.nthreads)
        return K + W


class State:
    """Full Hermite state of one system (the oracle's own copy)."""

    def __init__(self, m, r, v, eps, eta, G=1.0, eta_start=0.01,
                 dt_max=1.0 / 16, dt_min=2.0 ** -40, t0=0.0, nthreads=1,
                 a=None, j=None, t=None, dt=None):
        self.m = _f64(m).copy()
        n = self.m.shape[0]
        self.n = n
        self.r = _f64(r, (n, 3)).copy()
        self.v = _f64(v, (n, 3)).copy()
        self.eps, self.eta, self.G = float(eps), float(eta), float(G)
        self.eta_start = float(eta_start)
        self.dt_max, self.dt_min = float(dt_max), float(dt_min)
        self.nthreads = int(nthreads)
        self.n_steps = 0
        self.n_inter = 0.0
        if a is None:
            self.a = np.empty((n, 3))
            self.j = np.empty((n, 3))
            self.t = np.empty(n)
            self.dt = np.empty(n)
            st = _load().orc_init(n, _ptr(self.m), _ptr(self.r), _ptr(self.v),
                                  _ptr(self.a), _ptr(self.j), _ptr(self.t),
                                  _ptr(self.dt), float(t0), self.eps, self.G,
                                  self.eta_start, self.dt_max, self.dt_min,
                                  self.nthreads)
            if st != OK:
                raise RuntimeError(f"oracle init failed with status {st}")
        else:
            self.a = _f64(a, (n, 3)).copy()
            self.j = _f64(j, (n, 3)).copy()
            self.t = _f64(t).copy()
            self.dt = _f64(dt).copy()

    def run(self, t_end, max_steps=0):
        """Steps 1-9 of Sec. 2 until the next block time would pass t_end."""
        steps = np.zeros(1, dtype=np.int64)
        inter = np.zeros(1)
        st = _load().orc_run(self.n, _ptr(self.m), _ptr(self.r), _ptr(self.v),
                             _ptr(self.a), _ptr(self.j), _ptr(self.t),
                             _ptr(self.dt), float(t_end), self.eps, self.G,
                             self.eta, self.dt_max, self.dt_min, self.nthreads,
                             int(max_steps), _ptr(steps), _ptr(inter))
        self.n_steps += int(steps[0])
        self.n_inter += float(inter[0])
        return st

    def energy(self):
        K, W = energy(self.m, self.r, self.v, self.eps, self.G, self.nthreads)
        return K + W
