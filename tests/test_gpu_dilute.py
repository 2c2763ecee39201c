"""Hot vapour below the equation of state's density floor on the GPU: a slab at 1e-16 rho0
in vacuum against the oracle (FP64 bar), and, in both precisions, moving exactly like the
same slab at 1e-10 rho0 (in the dilute limit p = a rho I, so the motion does not depend on
the density scale; a pressure left at its floor value would move it 1e4 times faster)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle_cases as OC
from oracle import oracle as O
from paper_2403_04267_gb300 import salec


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    salec.load()


@pytest.mark.parametrize("steps", [1, 10])
def test_dilute_slab_matches_oracle(steps):
    spec = OC.dilute_slab_spec(1e-16)
    g, r = salec.Sim(spec), O.OracleSim(spec)
    g.step(steps)
    r.step(steps)
    vscale = np.max(np.abs(r.get("vz")))
    assert vscale > 0.0
    for name, scale in (("vz", vscale), ("vr", vscale), ("f0", 1.0), ("I", np.max(r.get("I"))),
                        ("rho0", np.max(r.get("rho0")))):
        a, b = g.get(name), r.get(name)
        assert np.max(np.abs(a - b)) <= 1e-9 * scale, name
    sg, so = g.scalars(), r.scalars()
    assert sg["status"] == so["status"] == 0 and sg["nstep"] == so["nstep"]
    assert abs(sg["t"] - so["t"]) <= 1e-12 * so["t"]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32mix", 1e-4)])
def test_dilute_slab_motion_is_scale_free(precision, tol):
    hi = salec.Sim(OC.dilute_slab_spec(1e-10), precision=precision)
    lo = salec.Sim(OC.dilute_slab_spec(1e-16), precision=precision)
    hi.step(10)
    lo.step(10)
    vscale = np.max(np.abs(hi.get("vz")))
    for name, scale in (("vz", vscale), ("f0", 1.0), ("I", np.max(hi.get("I")))):
        a, b = lo.get(name), hi.get(name)
        assert np.max(np.abs(a - b)) <= tol * scale, (name, np.max(np.abs(a - b)) / scale)
    assert lo.scalars()["status"] == hi.scalars()["status"] == 0
