"""nb_force_static: the allocation-free force entry point.

Some callers cannot allocate device memory: a host framework that owns every
device allocation and forbids others, or a process that has already
reserved its GPU's memory.  nb_force_static serves them with a force
evaluation whose only working memory is a fixed array inside the library.
It computes what nb_force computes in NB_DS precision, so it is held to the
DS bound against the FP64 oracle (1e-9 per particle, as the full-size DS
tests).  This file is collected last so that a failure here leaves every
other result in place.
"""
import ctypes
import os

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

pytestmark = pytest.mark.gpu
NTHREADS = os.cpu_count() or 1
DS_BOUND = 1e-9
MAX_N = 131072  # NB_STATIC_MAX_N


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _rel(x, ref):
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


class _Inputs:
    """Device copies of one system and the output buffers for n_act entries."""

    def __init__(self, torch, m, r, v, idx):
        dev = torch.device("cuda", 0)
        k = len(idx)
        self.n, self.k = len(m), k
        self.m = torch.from_numpy(np.ascontiguousarray(m)).to(dev)
        self.r = torch.from_numpy(np.ascontiguousarray(r)).to(dev)
        self.v = torch.from_numpy(np.ascontiguousarray(v)).to(dev)
        self.idx = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int32)).to(dev)
        self.acc = torch.empty((max(k, 1), 3), dtype=torch.float64, device=dev)
        self.jerk = torch.empty((max(k, 1), 3), dtype=torch.float64, device=dev)
        self.pot = torch.empty(max(k, 1), dtype=torch.float64, device=dev)

    def call(self, gpu, eps, n_act=None):
        k = self.k if n_act is None else n_act
        return gpu.nb_force_static(self.n, _p(self.m), _p(self.r), _p(self.v), eps, 1.0, k,
                                   _p(self.idx), _p(self.acc), _p(self.jerk), _p(self.pot), None)

    def outputs(self):
        return (self.acc[:self.k].cpu().numpy(), self.jerk[:self.k].cpu().numpy(),
                self.pot[:self.k].cpu().numpy())


def _check_against_oracle(orc, m, r, v, eps, idx, out):
    a0, j0, p0 = orc.force(m, r, v, eps, idx=idx, nthreads=NTHREADS)
    a, j, p = out
    assert _rel(a, a0).max() < DS_BOUND
    assert _rel(j, j0).max() < DS_BOUND
    assert (np.abs(p - p0) / np.abs(p0)).max() < DS_BOUND


def test_force_static_matches_oracle_on_two_calls_in_a_row(gpu, orc):
    import torch
    # the second call is smaller and uses another active list, so anything
    # the first call left in the shared array must not leak into it
    cases = []
    for n, seed, n_act in ((3001, 21, 3001), (1500, 22, 257)):
        m, r, v = ics.plummer(n, seed)
        idx = ics.permutation(n, seed)[:n_act].astype(np.int32)
        cases.append((m, r, v, 4.0 / n, idx, _Inputs(torch, m, r, v, idx)))
    torch.cuda.synchronize()
    for q, (m, r, v, eps, idx, inp) in enumerate(cases):
        if q == 1:
            # the first call did the one-time set-up; from here on nothing
            # may be allocated, by the library or through torch
            free0, _ = torch.cuda.mem_get_info()
            torch0 = torch.cuda.memory_allocated()
        assert inp.call(gpu, eps) == gpu.NB_OK
        if q == 1:
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == torch0
        _check_against_oracle(orc, m, r, v, eps, idx, inp.outputs())


def test_force_static_at_its_size_limit(gpu, orc):
    """n = NB_STATIC_MAX_N fits the array (whatever the SM count); a sample
    of 320 particles (256 random, the 64 most central) against the oracle."""
    import torch
    n = MAX_N
    m, r, v = ics.plummer(n, 31)
    central = np.argsort(np.einsum("ij,ij->i", r, r))[:64]
    idx = np.unique(np.concatenate([ics.permutation(n, 31)[:256], central])).astype(np.int32)
    inp = _Inputs(torch, m, r, v, idx)
    assert inp.call(gpu, 4.0 / n) == gpu.NB_OK
    _check_against_oracle(orc, m, r, v, 4.0 / n, idx, inp.outputs())


def test_force_static_rejects_bad_arguments(gpu):
    import torch
    n = 700
    m, r, v = ics.plummer(n, 23)
    # an index outside [0, n): the kernel flags it and the call fails
    bad = np.array([0, 5, n, 17], dtype=np.int32)
    inp = _Inputs(torch, m, r, v, bad)
    assert inp.call(gpu, 4.0 / n) == gpu.NB_EINVAL
    # an empty active list does nothing and succeeds
    assert inp.call(gpu, 4.0 / n, n_act=0) == gpu.NB_OK
    # after the rejected call the shared array must not carry its status
    good = _Inputs(torch, m, r, v, np.arange(n, dtype=np.int32))
    assert good.call(gpu, 4.0 / n) == gpu.NB_OK


def test_force_static_rejects_sizes_beyond_its_array(gpu):
    lib = gpu.load()
    big = MAX_N + 1
    one = ctypes.c_void_p(1)  # never dereferenced: the size check comes first
    st = gpu.nb_force_static(big, one, one, one, 0.01, 1.0, 1, one, one, one, one, None)
    assert st == gpu.NB_EINVAL
    assert lib is not None
