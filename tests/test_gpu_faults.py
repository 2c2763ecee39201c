"""Failure detection, tested with failures made on the host (no GPU fault): a NaN vertex
velocity and, separately, a negative density are written into a run through
salec_set_field.  The run's status word must carry the bit the oracle sets for the same
injection (2: NaN, 1: non-positive volume or density), salec_get_scalars must return
SALEC_EUNSTABLE, and in a batch of three the damaged run must stop while the other two stay
equal to the same runs stepped alone (the batch executes the phase kernels' per-cell code:
bitwise in the mixed form, to the last bits in FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2403_04267_gb300 import salec, workloads as W

FIELDS = ("f0", "f1", "rho0", "rho1", "I", "srr", "szz", "srz", "D", "pmax", "vr", "vz")
TOL = {"fp64": 1e-12, "fp32mix": 0.0}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    salec.load()


def _spec(k=0):
    return W.impact(60 + 8 * k, 50, 10.0, W.basalt(strength=True), W.iron(), 4, 9e3 + 1e3 * k, 30, 6, gravity=1.62)


def _nan_velocity(sim):
    vz = sim.get("vz")
    vz[20, 5] = np.nan                       # a vertex inside the target
    sim.set("vz", vz)


def _negative_density(sim):
    rho = sim.get("rho0")
    rho[20, 5] = -rho[20, 5]                 # a full target cell
    sim.set("rho0", rho)


@pytest.mark.parametrize("inject,bit", [(_nan_velocity, 2), (_negative_density, 1)], ids=["nan", "negative_density"])
@pytest.mark.parametrize("form", ["phases", "fused"])
def test_injected_failure_sets_the_oracles_status_bit(inject, bit, form):
    spec = _spec()
    g = salec.Sim(spec)
    g.step_form = form
    r = O.OracleSim(spec)
    g.step(5)
    r.step(5)
    inject(g)
    inject(r)
    g.step(1)
    r.step(1)
    sg, so = g.scalars(), r.scalars()
    # the injected failure's bit in both (a NaN also makes the oracle's volume test, a
    # comparison that NaN fails, set bit 1 in the cells it reaches)
    assert so["status"] & bit and sg["status"] & bit
    with pytest.raises(salec.SalecError) as ei:
        g.scalars(check=True)
    assert ei.value.status == salec.SALEC_EUNSTABLE


def _same(a, b, precision):
    for f in FIELDS:
        x, y = a.get(f), b.get(f)
        d = float(np.max(np.abs(x - y))) if x.size else 0.0
        scale = float(np.max(np.abs(y))) if y.size else 0.0
        assert d <= TOL[precision] * scale, f"{f}: {d:.3e} of {scale:.3e}"
    assert a.scalars()["nstep"] == b.scalars()["nstep"]


@pytest.mark.parametrize("precision", ["fp64", "fp32mix"])
@pytest.mark.parametrize("inject,bit,stop_after", [(_nan_velocity, 2, 0), (_negative_density, 1, 1)],
                         ids=["nan", "negative_density"])
def test_a_failed_run_stops_while_the_batch_continues(precision, inject, bit, stop_after):
    """A NaN velocity is caught by the Courant pass of the next step, which the run then
    does not take; a negative density by that step's Lagrangian phase, after which the run
    takes no further step."""
    specs = [_spec(k) for k in range(3)]
    runs, alone = [], []
    for sp in specs:
        for lst in (runs, alone):
            s = salec.Sim(sp, precision=precision)
            s.step_form = "phases"
            s.step(5)
            lst.append(s)
    inject(runs[1])
    b = salec.Batch(runs)
    b.step(12)
    polled = b.poll()
    assert int(polled[1, 3]) & bit
    assert int(polled[1, 2]) == 5 + stop_after
    assert int(polled[0, 3]) == 0 and int(polled[2, 3]) == 0
    for k in (0, 2):
        alone[k].step(12)
        _same(runs[k], alone[k], precision)
