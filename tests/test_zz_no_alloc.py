"""The allocation-free Courant step against the one salec_step computes.

salec_courant_dt_noalloc serves callers that cannot allocate or lend device memory (an
external memory manager owns every allocation, or they only see another program's field
pointers): it keeps its scratch in fixed file-scope device memory.  Here the fields of a
running simulation are copied into plain torch device tensors (standing in for such a
caller's buffers), the step size is computed from them with no allocation by the
library, and compared with the step salec_step then takes from the same state, on two
calls in a row (the scratch is shared and reused).  This file is collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_04267_gb300 import salec, workloads as W

TOL = 1e-9


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _fields(sim, nmat):
    fr = [_dev(np.stack([sim.get(f"f{m}"), sim.get(f"rho{m}")], axis=-1)) for m in range(nmat)]
    I = _dev(sim.get("I"))
    v = _dev(np.stack([sim.get("vr"), sim.get("vz")], axis=-1))
    return fr, I, v


@pytest.mark.parametrize("spec", [W.plain_fp64_100(),
                                  W.impact(120, 90, 25.0, W.basalt(strength=True), W.iron(), 6, 12e3, 60, 10,
                                           gravity=1.62)], ids=["hydro_1mat", "strength_2mat"])
def test_noalloc_courant_step_matches_salec_step(spec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    nmat = len(spec["materials"])
    sim = salec.Sim(spec)
    sim.step(25)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        dt_prev = sim.scalars()["dt"]
        fr, I, v = _fields(sim, nmat)
        torch.cuda.synchronize()
        dt_free = salec.courant_dt_noalloc(spec, [t.data_ptr() for t in fr], I.data_ptr(), v.data_ptr(),
                                           dt_prev, stream)
        sim.step(1)
        dt_step = sim.scalars()["dt"]
        assert abs(dt_free - dt_step) <= TOL * dt_step, (dt_free, dt_step)
        sim.step(7)


def test_noalloc_rejects_grids_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spec = W.scaled_plain(100)
    spec = dict(spec, grid=dict(spec["grid"], nr=8192, nz=8192))
    with pytest.raises(salec.SalecError) as ei:
        salec.courant_dt_noalloc(spec, [0], 0, 0, 1.0, 0)
    assert ei.value.status == salec.SALEC_EINVAL
    assert "fixed scratch" in str(ei.value)
