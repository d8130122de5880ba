"""Thin ctypes binding of libnbody (``include/nbody.h``).

The functions ``nb_*`` below have the C names and argument order; the
``Context`` class only marshals numpy arrays (host) and torch CUDA tensors
(device) into those calls.  Every step of the method runs in the CUDA
kernels of ``libnbody.so``; if the library is missing this module raises
instead of computing anything itself.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnbody.so")

NB_OK, NB_EINVAL, NB_ECUDA, NB_ENOMEM, NB_ENONFINITE, NB_EDTMIN, NB_ETIMEOUT, NB_ESTATE = range(8)
NB_FP64, NB_MIXED, NB_DS, NB_HYBRID, NB_MIXED_SPJ, NB_HYBRID_SPJ, NB_FP64_HERMITE6 = \
    0, 1, 2, 3, 4, 5, 6
PRECISIONS = {"fp64": NB_FP64, "mixed": NB_MIXED, "ds": NB_DS, "hybrid": NB_HYBRID,
              "mixed_spj": NB_MIXED_SPJ, "hybrid_spj": NB_HYBRID_SPJ,
              "fp64_hermite6": NB_FP64_HERMITE6}


class NbConfig(ctypes.Structure):
    _fields_ = [
        ("precision", c_int32),
        ("device", c_int32),
        ("G", c_double),
        ("eta_start", c_double),
        ("dt_max", c_double),
        ("dt_min", c_double),
        ("stream", c_void_p),
        ("i_per_thread", c_int32),
        ("ctas_per_sm", c_int32),
        ("autotune", c_int32),
        ("j_split", c_int32),
        ("wait_limit_cycles", c_int64),
    ]


class NbTuning(ctypes.Structure):
    _fields_ = [
        ("small_i_per_thread", c_int32),
        ("small_ctas_per_sm", c_int32),
        ("large_i_per_thread", c_int32),
        ("large_ctas_per_sm", c_int32),
        ("nact_split", c_int32),
        ("small_j_split", c_int32),
        ("large_j_split", c_int32),
        ("small_us", c_double),
        ("large_us", c_double),
        ("tiny_split", c_int32),
        ("tiny_i_per_thread", c_int32),
        ("tiny_ctas_per_sm", c_int32),
        ("tiny_j_split", c_int32),
        ("tiny_us", c_double),
        ("ens_chunks", c_int32),
    ]


class NbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libnbody.so (built by ``paper_1104_2700_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "nb_config_init": (None, [POINTER(NbConfig)]),
        "nb_create": (c_int32, [POINTER(NbConfig), POINTER(c_void_p)]),
        "nb_destroy": (c_int32, [P]),
        "nb_set_particles": (c_int32, [P, c_int64, P, P, P, c_double, c_double]),
        "nb_set_state": (c_int32, [P, c_int64, P, P, P, P, P, P, P, c_double, c_double, c_int32]),
        "nb_get_state": (c_int32, [P, P, P, P, P, P, P, c_int32]),
        "nb_predict": (c_int32, [P, c_double]),
        "nb_select": (c_int32, [P, c_double, POINTER(c_double), POINTER(c_int32), P]),
        "nb_force": (c_int32, [P, c_int32, P, P, P, P, c_int32]),
        "nb_correct": (c_int32, [P, c_double, c_int32, P, P, P, c_int32]),
        "nb_block_step": (c_int32, [P, c_double]),
        "nb_step_until": (c_int32, [P, c_double, POINTER(c_uint64), POINTER(c_uint64)]),
        "nb_energy": (c_int32, [P, c_int32, POINTER(c_double), POINTER(c_double)]),
        "nb_synchronize": (c_int32, [P]),
        "nb_num_particles": (c_int64, [P]),
        "nb_last_error": (c_char_p, [P]),
        "nb_status_string": (c_char_p, [c_int32]),
        "nb_force_static": (c_int32, [c_int64, P, P, P, c_double, c_double, c_int32, P, P, P,
                                      P, P]),
        "nb_set_ensemble": (c_int32, [P, c_int32, P, P, P, P, P, c_double]),
        "nb_energy_systems": (c_int32, [P, c_int32, P, P]),
        "nb_num_systems": (c_int32, [P]),
        "nb_autotune": (c_int32, [P, POINTER(NbTuning)]),
        "nb_set_tuning": (c_int32, [P, POINTER(NbTuning)]),
        "nb_selftest_timeout": (c_int32, [P]),
        "nb_measure_peaks": (c_int32, [c_int32, POINTER(c_double), POINTER(c_double)]),
        "nb_snapshot_bytes": (c_int64, [P]),
        "nb_snapshot": (c_int32, [P, P]),
        "nb_restore": (c_int32, [P, P]),
        "nb_spatial_order": (c_int32, [P, P]),
        "nb_set_j_part": (c_int32, [P, c_int32, c_int32]),
        "nb_get_snap": (c_int32, [P, P, P, c_int32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _status_name(s: int) -> str:
    names = ["NB_OK", "NB_EINVAL", "NB_ECUDA", "NB_ENOMEM", "NB_ENONFINITE",
             "NB_EDTMIN", "NB_ETIMEOUT", "NB_ESTATE"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


# --- the C entry points, same names ------------------------------------------
def nb_config_init() -> NbConfig:
    cfg = NbConfig()
    load().nb_config_init(ctypes.byref(cfg))
    return cfg


def nb_create(cfg: NbConfig) -> int:
    h = c_void_p()
    st = load().nb_create(ctypes.byref(cfg), ctypes.byref(h))
    if st != NB_OK:
        raise NbError(st, "nb_create failed")
    return h.value


def nb_destroy(ctx) -> int:
    return load().nb_destroy(ctx)


def nb_last_error(ctx) -> str:
    r = load().nb_last_error(ctx)
    return r.decode() if r else ""


def _check(ctx, st: int):
    if st != NB_OK:
        raise NbError(st, nb_last_error(ctx))


def nb_set_particles(ctx, n, m, r, v, eps, eta):
    return load().nb_set_particles(ctx, n, m, r, v, eps, eta)


def nb_set_state(ctx, n, m, r, v, a, j, t, dt, eps, eta, on_device):
    return load().nb_set_state(ctx, n, m, r, v, a, j, t, dt, eps, eta, on_device)


def nb_get_state(ctx, r, v, a, j, t, dt, on_device):
    return load().nb_get_state(ctx, r, v, a, j, t, dt, on_device)


def nb_predict(ctx, t):
    return load().nb_predict(ctx, t)


def nb_select(ctx, t_end, t_next_ref, n_act_ref, idx):
    return load().nb_select(ctx, t_end, t_next_ref, n_act_ref, idx)


def nb_force(ctx, n_act, idx, acc, jerk, pot, on_device):
    return load().nb_force(ctx, n_act, idx, acc, jerk, pot, on_device)


def nb_correct(ctx, t, n_act, idx, acc, jerk, on_device):
    return load().nb_correct(ctx, t, n_act, idx, acc, jerk, on_device)


def nb_block_step(ctx, t_end):
    return load().nb_block_step(ctx, t_end)


def nb_step_until(ctx, t_end, n_steps_ref, n_inter_ref):
    return load().nb_step_until(ctx, t_end, n_steps_ref, n_inter_ref)


def nb_energy(ctx, fp64_potential, kin_ref, pot_ref):
    return load().nb_energy(ctx, fp64_potential, kin_ref, pot_ref)


def nb_synchronize(ctx):
    return load().nb_synchronize(ctx)


def nb_num_particles(ctx) -> int:
    return load().nb_num_particles(ctx)


def nb_status_string(st: int) -> str:
    return load().nb_status_string(st).decode()


def nb_set_ensemble(ctx, k, offsets, m, r, v, eps, eta):
    return load().nb_set_ensemble(ctx, k, offsets, m, r, v, eps, eta)


def nb_energy_systems(ctx, fp64_potential, kin, pot):
    return load().nb_energy_systems(ctx, fp64_potential, kin, pot)


def nb_num_systems(ctx) -> int:
    return load().nb_num_systems(ctx)


def nb_autotune(ctx, out_ref):
    return load().nb_autotune(ctx, out_ref)


def nb_set_tuning(ctx, tuning_ref):
    return load().nb_set_tuning(ctx, tuning_ref)


def nb_selftest_timeout(ctx):
    return load().nb_selftest_timeout(ctx)


def nb_force_static(n, m, r, v, eps, G, n_act, idx, acc, jerk, pot, stream):
    """Allocation-free force evaluation on device pointers (see nbody.h)."""
    return load().nb_force_static(n, m, r, v, eps, G, n_act, idx, acc, jerk, pot, stream)


def nb_snapshot_bytes(ctx) -> int:
    return load().nb_snapshot_bytes(ctx)


def nb_snapshot(ctx, buf):
    return load().nb_snapshot(ctx, buf)


def nb_restore(ctx, buf):
    return load().nb_restore(ctx, buf)


def nb_spatial_order(ctx, order):
    return load().nb_spatial_order(ctx, order)


def nb_set_j_part(ctx, part, parts):
    return load().nb_set_j_part(ctx, part, parts)


def nb_get_snap(ctx, s, c, on_device):
    return load().nb_get_snap(ctx, s, c, on_device)


def nb_measure_peaks(device, fp32_ref, fp64_ref):
    return load().nb_measure_peaks(device, fp32_ref, fp64_ref)


def measure_peaks(device=0):
    """Measured (FP32, FP64) FMA throughput of the device in TFLOP/s."""
    f32, f64 = c_double(), c_double()
    st = nb_measure_peaks(int(device), ctypes.byref(f32), ctypes.byref(f64))
    if st != NB_OK:
        raise NbError(st, "nb_measure_peaks failed")
    return f32.value, f64.value


# --- marshalling helpers ------------------------------------------------------
def _is_device(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _ptr(x, dtype, shape=None):
    """(pointer, keep-alive object, on_device) for a numpy array or torch tensor."""
    if x is None:
        return None, None, None
    if _is_device(x):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"device tensor must be contiguous {want}")
        return c_void_p(x.data_ptr()), x, True
    a = np.ascontiguousarray(x, dtype=dtype)
    if shape is not None:
        a = a.reshape(shape)
    return a.ctypes.data_as(c_void_p), a, False


class Context:
    """One simulated system on one GPU (wraps an nb_ctx handle)."""

    def __init__(self, precision="hybrid", device=0, G=1.0, eta_start=0.01,
                 dt_max=1.0 / 16, dt_min=2.0 ** -40, stream=None, i_per_thread=0,
                 ctas_per_sm=0, autotune=False, wait_limit_cycles=0, j_split=0):
        cfg = nb_config_init()
        cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg.device = int(device)
        cfg.G = float(G)
        cfg.eta_start = float(eta_start)
        cfg.dt_max = float(dt_max)
        cfg.dt_min = float(dt_min)
        if stream is not None:
            cfg.stream = c_void_p(int(getattr(stream, "cuda_stream", stream)))
        cfg.i_per_thread = int(i_per_thread)
        cfg.ctas_per_sm = int(ctas_per_sm)
        cfg.autotune = int(bool(autotune))
        cfg.j_split = int(j_split)
        cfg.wait_limit_cycles = int(wait_limit_cycles)
        self.cfg = cfg
        self.handle = nb_create(cfg)
        self.n = 0

    def close(self):
        if self.handle:
            nb_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        _check(self.handle, st)

    def set_particles(self, m, r, v, eps, eta):
        n = len(m)
        pm, km, _ = _ptr(m, np.float64)
        pr, kr, _ = _ptr(r, np.float64, (n, 3))
        pv, kv, _ = _ptr(v, np.float64, (n, 3))
        self._ck(nb_set_particles(self.handle, n, pm, pr, pv, float(eps), float(eta)))
        self.n = n

    def set_state(self, m, r, v, a, j, t, dt, eps, eta):
        n = len(m)
        args = [_ptr(m, np.float64)] + [_ptr(x, np.float64, (n, 3)) for x in (r, v, a, j)] + \
               [_ptr(t, np.float64), _ptr(dt, np.float64)]
        dev = {x[2] for x in args}
        if len(dev) != 1:
            raise TypeError("set_state wants all host arrays or all device tensors")
        self._ck(nb_set_state(self.handle, n, *[x[0] for x in args], float(eps), float(eta),
                              int(dev.pop())))
        self.n = n

    def get_state(self):
        n = self.n
        out = {k: np.empty((n, 3)) for k in ("r", "v", "a", "j")}
        out["t"] = np.empty(n)
        out["dt"] = np.empty(n)
        p = {k: out[k].ctypes.data_as(c_void_p) for k in out}
        self._ck(nb_get_state(self.handle, p["r"], p["v"], p["a"], p["j"], p["t"], p["dt"], 0))
        return out

    def get_snap(self):
        """Snap and crackle of every particle (sixth-order variant)."""
        n = self.n
        s, c = np.empty((n, 3)), np.empty((n, 3))
        self._ck(nb_get_snap(self.handle, s.ctypes.data_as(c_void_p), c.ctypes.data_as(c_void_p), 0))
        return s, c

    def set_ensemble(self, offsets, m, r, v, eps, eta):
        """k independent systems: system q is [offsets[q], offsets[q+1])."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        k = len(off) - 1
        n = int(off[-1])
        pm, km, _ = _ptr(m, np.float64)
        pr, kr, _ = _ptr(r, np.float64, (n, 3))
        pv, kv, _ = _ptr(v, np.float64, (n, 3))
        pe, ke, _ = _ptr(eps, np.float64)
        self._ck(nb_set_ensemble(self.handle, k, off.ctypes.data_as(c_void_p), pm, pr, pv, pe,
                                 float(eta)))
        self.n = n
        self.k = k

    def energy_systems(self, fp64_potential=True):
        k = nb_num_systems(self.handle)
        kin = np.empty(k)
        pot = np.empty(k)
        self._ck(nb_energy_systems(self.handle, int(bool(fp64_potential)),
                                   kin.ctypes.data_as(c_void_p), pot.ctypes.data_as(c_void_p)))
        return kin, pot

    def autotune(self):
        """Measure and set the force launch shapes; returns them as a dict."""
        tun = NbTuning()
        self._ck(nb_autotune(self.handle, ctypes.byref(tun)))
        return {name: getattr(tun, name) for name, _ in NbTuning._fields_}

    def set_tuning(self, **shapes):
        """Set the force launch shapes (the fields of ``nb_tuning``; those not
        given are 0, i.e. no tiny shape)."""
        tun = NbTuning(**shapes)
        self._ck(nb_set_tuning(self.handle, ctypes.byref(tun)))

    def spatial_order(self):
        """The particles in the context's spatial (j-layout slot) order."""
        order = np.empty(self.n, dtype=np.int32)
        self._ck(nb_spatial_order(self.handle, order.ctypes.data_as(c_void_p)))
        return order

    def set_j_part(self, part, parts):
        """Sum forces over part `part` of `parts` j ranges (j-partitioned force)."""
        self._ck(nb_set_j_part(self.handle, int(part), int(parts)))

    def predict(self, t):
        self._ck(nb_predict(self.handle, float(t)))

    def select(self, t_end=float("inf")):
        tn = c_double()
        na = c_int32()
        idx = np.empty(max(self.n, 1), dtype=np.int32)
        self._ck(nb_select(self.handle, float(t_end), ctypes.byref(tn), ctypes.byref(na),
                           idx.ctypes.data_as(c_void_p)))
        return tn.value, idx[: na.value].copy()

    def force(self, idx, acc=None, jerk=None, pot=None):
        """acc, jerk, pot of the particles idx (host arrays, or device tensors)."""
        if _is_device(idx):
            k = idx.numel()
            pi, ki, _ = _ptr(idx, np.int32)
            pa, ka, _ = _ptr(acc, np.float64)
            pj, kj, _ = _ptr(jerk, np.float64)
            pp, kp, _ = _ptr(pot, np.float64)
            self._ck(nb_force(self.handle, k, pi, pa, pj, pp, 1))
            return acc, jerk, pot
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        k = idx.shape[0]
        acc = np.empty((k, 3))
        jerk = np.empty((k, 3))
        pot = np.empty(k)
        self._ck(nb_force(self.handle, k, idx.ctypes.data_as(c_void_p),
                          acc.ctypes.data_as(c_void_p), jerk.ctypes.data_as(c_void_p),
                          pot.ctypes.data_as(c_void_p), 0))
        return acc, jerk, pot

    def correct(self, t, idx, acc=None, jerk=None):
        if _is_device(idx):
            pi, ki, _ = _ptr(idx, np.int32)
            pa, ka, _ = _ptr(acc, np.float64)
            pj, kj, _ = _ptr(jerk, np.float64)
            self._ck(nb_correct(self.handle, float(t), idx.numel(), pi, pa, pj, 1))
            return
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        k = idx.shape[0]
        pa, ka, _ = _ptr(acc, np.float64, (k, 3)) if acc is not None else (None, None, None)
        pj, kj, _ = _ptr(jerk, np.float64, (k, 3)) if jerk is not None else (None, None, None)
        self._ck(nb_correct(self.handle, float(t), k, idx.ctypes.data_as(c_void_p), pa, pj, 0))

    def snapshot_bytes(self):
        return nb_snapshot_bytes(self.handle)

    def snapshot(self, buf):
        """Copy the device state into `buf` (a device tensor of at least
        snapshot_bytes() bytes)."""
        self._ck(nb_snapshot(self.handle, c_void_p(buf.data_ptr())))

    def restore(self, buf):
        """Copy a snapshot taken by snapshot() back into the device state."""
        self._ck(nb_restore(self.handle, c_void_p(buf.data_ptr())))

    def block_step(self, t_end):
        self._ck(nb_block_step(self.handle, float(t_end)))

    def step_until(self, t_end):
        ns = c_uint64()
        ni = c_uint64()
        self._ck(nb_step_until(self.handle, float(t_end), ctypes.byref(ns), ctypes.byref(ni)))
        return ns.value, ni.value

    def energy(self, fp64_potential=True):
        k = c_double()
        w = c_double()
        self._ck(nb_energy(self.handle, int(bool(fp64_potential)), ctypes.byref(k), ctypes.byref(w)))
        return k.value, w.value

    def synchronize(self):
        self._ck(nb_synchronize(self.handle))
