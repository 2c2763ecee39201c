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


def test_host_checks_of_the_batch_modes_and_the_ensemble_group():
    """The entry points added for the persistent batch, the rest-tile switch and the
    ensemble group refuse null or out-of-range arguments on the host, before any CUDA call."""
    L = salec.load()
    assert L.salec_batch_set_persistent(None, 1) == salec.SALEC_EINVAL
    assert L.salec_batch_expire_next_barrier(None) == salec.SALEC_EINVAL
    assert L.salec_set_rest_copy(None, 0) == salec.SALEC_EINVAL
    h = C.c_void_p()
    assert L.salec_mlp_group_create(None, 2, None, C.byref(h)) == salec.SALEC_EINVAL
    one = (C.c_void_p * 1)(None)
    assert L.salec_mlp_group_create(one, 1, None, C.byref(h)) == salec.SALEC_EINVAL      # a null member
    fake = (C.c_void_p * 9)(*[C.c_void_p(16 * (k + 1)) for k in range(9)])
    assert L.salec_mlp_group_create(fake, 9, None, C.byref(h)) == salec.SALEC_EINVAL     # more than 8
    rep = (C.c_void_p * 2)(C.c_void_p(16), C.c_void_p(16))
    assert L.salec_mlp_group_create(rep, 2, None, C.byref(h)) == salec.SALEC_EINVAL      # a repeated member
    assert L.salec_mlp_train_group(None, None, None, 1, 1, None, 0.9, 0.999, 1e-8) == salec.SALEC_EINVAL
