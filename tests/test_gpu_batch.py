"""Batched runs and the block-shape autotuner.

A batch advances independent runs of uneven sizes with one set of launches per step; each
run keeps its own time step and end time.  Every block of a batched launch executes the
same source code as the single-run kernels, but the compiler may contract a multiply-add
differently in the two kernels, so a batched run agrees with the same run stepped alone to
rounding: after 30 steps of an impact the FP64 fields differ in the last bits (measured
< 3e-14 of each field's largest value), the FP32-mix fields are identical.  The bar is a
normwise difference of 1e-12 (FP64) and 1e-5 (FP32-mix) per field; the autotuner changes
only speed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle_cases as OC
from paper_2403_04267_gb300 import salec, workloads as W

FIELDS = ("f0", "f1", "rho0", "rho1", "I", "srr", "szz", "srz", "D", "pmax", "vr", "vz",
          "phi1_b", "psi1z_r", "phi2r_b")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    salec.load()


def _specs(n_runs, seed0=100):
    out = []
    for k in range(n_runs):
        d = W.batched_draw(seed0 + k)
        d["n"] = 40 + 17 * k            # small uneven grids
        d["radius_cells"] = 3 + k % 4
        spec = W.batched_run(d)
        spec["grid"]["pml_r"] = spec["grid"]["pml_b"] = 6
        out.append(spec)
    return out


TOL = {"fp64": 1e-12, "fp32mix": 1e-5}


def _alone(spec, precision):
    """A run stepped by itself with the phase kernels, whose per-cell code the batch runs."""
    s = salec.Sim(spec, precision=precision)
    s.step_form = "phases"
    return s


def _same(a, b, precision):
    sa, sb = a.scalars(), b.scalars()
    bad = []
    for f in FIELDS:
        x, y = a.get(f), b.get(f)
        d = np.max(np.abs(x - y)) if x.size else 0.0
        scale = np.max(np.abs(y)) if y.size else 0.0
        if d > TOL[precision] * scale:
            k = np.unravel_index(np.argmax(np.abs(x - y)), x.shape)
            bad.append(f"{f}: max {d:.3e} of {scale:.3e} at {k}")
    assert not bad, "; ".join(bad)
    assert sa["nstep"] == sb["nstep"]
    assert abs(sa["t"] - sb["t"]) <= TOL[precision] * sb["t"]


@pytest.mark.parametrize("precision", ["fp64", "fp32mix"])
def test_batch_equals_runs_alone(precision):
    specs = _specs(5)
    alone = [_alone(s, precision) for s in specs]
    for s in alone:
        s.step(30)
    runs = [salec.Sim(s, precision=precision) for s in specs]
    b = salec.Batch(runs)
    b.step(30)
    for a, r in zip(alone, runs):
        _same(a, r, precision)


def test_end_times_graph_replay_and_autotune():
    specs = _specs(4, seed0=200)
    runs = [salec.Sim(s, precision="fp32mix") for s in specs]
    ref = [_alone(s, "fp32mix") for s in specs]
    # end times reached after different step counts
    probe = [_alone(s, "fp32mix") for s in specs]
    t_end = []
    for k, p in enumerate(probe):
        p.step(20 + 7 * k)
        sc = p.scalars()
        t_end.append(sc["t"] - 0.5 * sc["dt"])    # reached at exactly that step
    for r, te in zip(runs, t_end):
        r.set_end_time(te)
    b = salec.Batch(runs)
    shapes = b.autotune(trial_steps=1)          # 7 candidates x 2 steps = 14 steps of every run
    assert len(shapes) == 6
    steps, done = b.run(chunk=8, max_steps=400)
    assert done == len(runs)
    polled = b.poll()
    for k, (r, p) in enumerate(zip(runs, probe)):
        sc = r.scalars()
        assert sc["t"] >= t_end[k]
        assert sc["nstep"] == p.scalars()["nstep"]    # stopped at the step that reached t_end
        assert polled[k, 0] == sc["t"]
    # the same runs stepped alone, default shapes, to the same step counts
    for r, p, q in zip(runs, probe, ref):
        q.step(p.scalars()["nstep"])
        _same(r, q, "fp32mix")


def test_single_run_autotune_keeps_fields():
    spec = W.full_fp64_800()
    spec = dict(spec, grid=dict(spec["grid"], nr=200, nz=160))
    spec["layers"][0]["zhi"] = 100 * 25.0
    spec["projectile"]["zc"] = 100 * 25.0 + spec["projectile"]["radius"]
    a = salec.Sim(spec)
    b = salec.Sim(spec)
    shapes = a.autotune(trial_steps=2)          # 7 x 3 = 21 steps
    assert len(shapes) == 6 and all(x % 32 == 0 for x, _ in shapes)
    b.step(21)
    _same(a, b, "fp64")


def test_finished_runs_leave_and_rejoin_the_batch():
    """After a run reaches its end time the batch drops it from its work lists; moving its
    end time later brings it back on the next salec_batch_run, and it continues exactly as
    the same run stepped alone."""
    specs = _specs(3, seed0=300)
    runs = [salec.Sim(s, precision="fp32mix") for s in specs]
    probe = _alone(specs[0], "fp32mix")
    probe.step(12)
    t12 = probe.scalars()["t"]
    probe.step(10)
    sc = probe.scalars()
    runs[0].set_end_time(t12 - 1e-12)
    for r in runs[1:]:
        r.set_end_time(1e9)
    b = salec.Batch(runs)
    b.run(chunk=4, max_steps=40)
    assert runs[0].scalars()["nstep"] == 12
    runs[0].set_end_time(sc["t"] - 0.5 * sc["dt"])
    steps, done = b.run(chunk=4, max_steps=40)
    assert runs[0].scalars()["nstep"] == 22
    _same(runs[0], probe, "fp32mix")
