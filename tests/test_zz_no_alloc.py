"""nb_force_static: the allocation-free force entry point.

Callers that cannot allocate device memory (a host framework that owns all
device allocations, a process whose GPU memory is fully reserved) get a
force evaluation whose only working memory is a fixed array inside the
library.  It must give what nb_force gives in NB_DS precision.  This file is
collected last so that a failure here leaves every other result in place.
"""
import ctypes

import numpy as np
import pytest

from paper_1104_2700_gb300 import ics

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _reference(gpu, m, r, v, eps, idx):
    n = len(m)
    z = np.zeros((n, 3))
    with gpu.Context("ds") as ctx:
        ctx.set_state(m, r, v, z, z, np.zeros(n), np.full(n, 1.0 / 16), eps=eps, eta=0.02)
        ctx.predict(0.0)
        return ctx.force(idx)


def test_force_static_matches_nb_force_on_two_calls_in_a_row(gpu):
    import torch
    dev = torch.device("cuda", 0)
    # the second call is smaller and uses another active list, so anything
    # the first call left in the shared array must not leak into it
    for n, seed, n_act in ((3001, 21, 3001), (1500, 22, 257)):
        m, r, v = ics.plummer(n, seed)
        eps = 4.0 / n
        idx = ics.permutation(n, seed)[:n_act].astype(np.int32)
        a0, j0, p0 = _reference(gpu, m, r, v, eps, idx)
        md = torch.from_numpy(m).to(dev)
        rd = torch.from_numpy(np.ascontiguousarray(r)).to(dev)
        vd = torch.from_numpy(np.ascontiguousarray(v)).to(dev)
        idd = torch.from_numpy(idx).to(dev)
        acc = torch.empty((n_act, 3), dtype=torch.float64, device=dev)
        jerk = torch.empty((n_act, 3), dtype=torch.float64, device=dev)
        pot = torch.empty(n_act, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        st = gpu.nb_force_static(n, _p(md), _p(rd), _p(vd), eps, 1.0, n_act, _p(idd), _p(acc),
                                 _p(jerk), _p(pot), None)
        assert st == gpu.NB_OK
        a, j, p = acc.cpu().numpy(), jerk.cpu().numpy(), pot.cpu().numpy()
        # same double-single arithmetic; only the split of each j sum over
        # warps may differ, so the DS tolerance of the parity tests applies
        assert np.max(np.linalg.norm(a - a0, axis=1) / np.linalg.norm(a0, axis=1)) < 1e-10
        assert np.max(np.linalg.norm(j - j0, axis=1) / np.linalg.norm(j0, axis=1)) < 1e-10
        assert np.max(np.abs(p - p0) / np.abs(p0)) < 1e-10


def test_force_static_rejects_sizes_beyond_its_array(gpu):
    lib = gpu.load()
    big = 131072 + 1  # NB_STATIC_MAX_N + 1
    one = ctypes.c_void_p(1)  # never dereferenced: the size check comes first
    st = gpu.nb_force_static(big, one, one, one, 0.01, 1.0, 1, one, one, one, one, None)
    assert st == gpu.NB_EINVAL
    assert lib is not None
