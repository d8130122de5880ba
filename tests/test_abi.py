"""The C ABI library builds, loads and exports what include/nbody.h declares.

No compute call is made here: these run on a machine without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "nbody.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("nb_create", "nb_set_particles", "nb_predict", "nb_force", "nb_correct",
                 "nb_step_until", "nb_destroy", "nb_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(nbody_lib):
    lib = ctypes.CDLL(nbody_lib.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_config_defaults(nbody_lib):
    cfg = nbody_lib.nb_config_init()
    assert cfg.precision == nbody_lib.NB_HYBRID
    assert cfg.G == 1.0 and cfg.eta_start == 0.01
    assert cfg.dt_max == 1.0 / 16 and cfg.dt_min == 2.0 ** -40
    assert cfg.autotune == 0
    assert cfg.wait_limit_cycles == 0
    assert ctypes.sizeof(nbody_lib.NbConfig) == 72
    assert cfg.j_split == 0
    assert ctypes.sizeof(nbody_lib.NbTuning) == 80


@pytest.mark.parametrize("field,value", [("dt_max", 0.1), ("dt_max", -1.0),
                                         ("precision", 7), ("precision", -1),
                                         ("eta_start", 0.0), ("j_split", 3), ("j_split", 16)])
def test_create_rejects_bad_config_before_touching_the_gpu(nbody_lib, field, value):
    cfg = nbody_lib.nb_config_init()
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    st = nbody_lib.load().nb_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st == nbody_lib.NB_EINVAL and h.value is None


def test_precision_enum_matches_header(nbody_lib):
    """The binding's precision names carry the values nbody.h declares."""
    with open(os.path.join(ROOT, "include", "nbody.h")) as fh:
        text = fh.read()
    body = re.search(r"typedef enum nb_precision \{(.*?)\} nb_precision;", text, re.S).group(1)
    declared = {k: int(v) for k, v in re.findall(r"(NB_\w+)\s*=\s*(\d+)", body)}
    bound = {f"NB_{name.upper()}": val for name, val in nbody_lib.PRECISIONS.items()}
    assert declared == bound


def test_null_context_calls_fail_cleanly(nbody_lib):
    lib = nbody_lib.load()
    assert lib.nb_predict(None, 0.0) == nbody_lib.NB_EINVAL
    assert lib.nb_destroy(None) == nbody_lib.NB_OK
    assert lib.nb_num_particles(None) == 0
    assert nbody_lib.nb_status_string(nbody_lib.NB_EDTMIN) == "NB_EDTMIN"
