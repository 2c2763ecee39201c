"""The allocation-free Courant step against the one salec_step computes.

salec_courant_dt_noalloc serves callers that cannot allocate or lend device memory (an
external memory manager owns every allocation, or they only see another program's field
pointers): it keeps its scratch in fixed file-scope device memory.  Here the fields of a
running simulation are copied into plain torch device tensors (standing in for such a
caller's buffers), the step size is computed from them with no allocation by the
library, and compared with the step salec_step then takes from the same state, on two
calls in a row (the scratch is shared and reused), also on a grid of exactly the largest
size the scratch holds; a NaN velocity and a step below dt_min are reported as the
failures salec_step's status word reports.  This file is collected last."""
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


def test_noalloc_at_the_scratch_limit_matches_salec_step():
    """4096 x 4096 cells: 65536 blocks of 32 x 8, every slot of the fixed scratch in the
    last block's reduction."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    spec = W.scaled_plain(4096, radius_cells=100)
    sim = salec.Sim(spec)
    sim.step(3)
    dt_prev = sim.scalars()["dt"]
    fr, I, v = _fields(sim, 1)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    dt_free = salec.courant_dt_noalloc(spec, [t.data_ptr() for t in fr], I.data_ptr(), v.data_ptr(), dt_prev, stream)
    sim.step(1)
    dt_step = sim.scalars()["dt"]
    assert abs(dt_free - dt_step) <= TOL * dt_step, (dt_free, dt_step)


def test_noalloc_reports_nan_and_a_collapsed_step():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    spec = W.plain_fp64_100()
    sim = salec.Sim(spec)
    sim.step(5)
    dt_prev = sim.scalars()["dt"]
    fr, I, v = _fields(sim, 1)
    stream = torch.cuda.current_stream().cuda_stream
    ptrs = [t.data_ptr() for t in fr]
    # a step below dt_min
    tight = dict(spec, grid=dict(spec["grid"], dt_min=1.0))
    with pytest.raises(salec.SalecError) as ei:
        salec.courant_dt_noalloc(tight, ptrs, I.data_ptr(), v.data_ptr(), dt_prev, stream)
    assert ei.value.status == salec.SALEC_EUNSTABLE and "dt_min" in str(ei.value)
    # a NaN vertex velocity under the projectile: salec_step flags it in its status word
    # (bit 2), the allocation-free call returns SALEC_EUNSTABLE
    vr = sim.get("vr")
    vr[70, 3] = np.nan
    v[70, 3, 0] = float("nan")
    torch.cuda.synchronize()
    with pytest.raises(salec.SalecError) as ei:
        salec.courant_dt_noalloc(spec, ptrs, I.data_ptr(), v.data_ptr(), dt_prev, stream)
    assert ei.value.status == salec.SALEC_EUNSTABLE and "NaN" in str(ei.value)
    sim.set("vr", vr)
    sim.step(1)
    assert sim.scalars()["status"] & 2
    # the next call, on clean fields, succeeds: the flag does not outlive its call
    fr, I, v = _fields(salec.Sim(spec), 1)
    torch.cuda.synchronize()
    assert salec.courant_dt_noalloc(spec, [t.data_ptr() for t in fr], I.data_ptr(), v.data_ptr(), 1.0, stream) > 0.0


def test_noalloc_rejects_more_block_rows_than_a_launch_takes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spec = W.scaled_plain(100)
    spec = dict(spec, grid=dict(spec["grid"], nr=32, nz=65536 * 8))
    with pytest.raises(salec.SalecError) as ei:
        salec.courant_dt_noalloc(spec, [0], 0, 0, 1.0, 0)
    assert ei.value.status == salec.SALEC_EINVAL
    assert "65535" in str(ei.value)
