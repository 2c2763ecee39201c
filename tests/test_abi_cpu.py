"""CPU checks of the boundary: the CUDA library builds for sm_103a, loads, and exports
every entry point that include/salec.h declares; host-only calls validate arguments."""
import ctypes as C
import os
import re

import pytest

from paper_2403_04267_gb300 import salec, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(salec_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = salec.load()
    names = declared()
    assert "salec_step" in names and "salec_mlp_train_step" in names and len(names) >= 40
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(salec.EXPORTS) | {"salec_launches_per_step"}


def test_state_bytes_and_argument_checks():
    L = salec.load()
    spec = W.plain_fp64_100()
    g = salec.make_grid(spec["grid"], 1)
    n = C.c_size_t()
    assert L.salec_state_bytes(C.byref(g), 0, C.byref(n)) == salec.SALEC_OK
    nc, nv = 100 * 100, 101 * 101
    assert n.value > 16 * nc + 16 * nv           # at least (f, rho) and v
    assert n.value % 256 == 0
    bad = salec.make_grid(dict(spec["grid"], pml_r=100), 1)
    assert L.salec_state_bytes(C.byref(bad), 0, C.byref(n)) == salec.SALEC_EINVAL
    assert L.salec_state_bytes(C.byref(g), 7, C.byref(n)) == salec.SALEC_EINVAL
    # create refuses a null or too small buffer before touching the device
    h = C.c_void_p()
    assert L.salec_create(C.byref(g), 0, None, 0, None, C.byref(h)) == salec.SALEC_ENOMEM


def test_graft_build_entry():
    import __graft_entry__ as ge
    ge.build()
