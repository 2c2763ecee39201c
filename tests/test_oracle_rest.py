"""Pins: exact preservation of rest states.  A uniform ideal gas at 1e5 Pa in a closed
box stays bitwise at rest (the corner forces of a uniform pressure cancel exactly,
including the axisymmetric hoop part).  A Tillotson column in discrete hydrostatic
equilibrium under gravity stays at rest to |v|/c <= 1e-12 for 200 steps."""
import numpy as np

import oracle_cases as OC
from oracle import oracle as O


def test_uniform_gas_box_is_bitwise_at_rest():
    s = O.OracleSim(OC.gas_box_spec(37, 29))
    rho0, I0 = s.get("rho0").copy(), s.get("I").copy()
    s.step(200)
    assert np.all(s.get("vr") == 0.0) and np.all(s.get("vz") == 0.0)
    assert np.array_equal(s.get("rho0"), rho0) and np.array_equal(s.get("I"), I0)
    assert s.scalars()["status"] == 0


def test_hydrostatic_column_stays_at_rest():
    s = O.OracleSim(OC.hydrostatic_spec(6, 40))
    p = s.get("p")
    assert p[0, 0] > p[10, 0] > p[25, 0] > 0.0          # lithostatic gradient
    s.step(200)
    v = np.hypot(s.get("vr"), s.get("vz")).max()
    assert v / np.sqrt(26.7e9 / 2700.0) <= 1e-12
