"""Pins: conservation sums.  With no PML, no clean-up threshold and before any wave or
ejecta reaches a boundary: total mass is constant to round-off, z-momentum (the walls
and the hoop term exert no net z-force inside) to 1e-13 relative, and kinetic plus
internal energy to 1e-12 relative, because the Lagrangian work is compatible with the
corner forces and every kinetic-energy deficit is returned as heat.  With clean-up on,
mass on the grid + outflow + discarded mass is exact throughout."""
import numpy as np

from oracle import oracle as O
from paper_2403_04267_gb300 import workloads as W


def _spec(f_min):
    w = W.impact(48, 48, 10.0, W.basalt(strength=True), W.iron(), 4, 8e3, 30, 0)
    w["grid"]["f_min"] = f_min
    w["grid"]["bc_top"] = "wall" if f_min == 0.0 else "outflow"
    return w


def test_mass_momentum_energy_conserved():
    s = O.OracleSim(_spec(0.0))
    c0 = s.conservation()
    s.step(40)
    c1 = s.conservation()
    sc = s.scalars()
    assert abs(c1["mass"] / c0["mass"] - 1) < 1e-14
    assert abs(c1["zmom"] / c0["zmom"] - 1) < 1e-13
    e0, e1 = c0["ke"] + c0["ie"], c1["ke"] + c1["ie"]
    assert abs(e1 / e0 - 1) < 1e-12
    assert c1["ie"] > 0.1 * e0      # a real impact: much of the energy is now heat


def test_mass_bookkeeping_with_cleanup():
    s = O.OracleSim(_spec(1e-6))
    c0 = s.conservation()
    s.step(60)
    c1 = s.conservation()
    sc = s.scalars()
    total = c1["mass"] + sc["mass_out"] + sc["mass_discarded"]
    assert abs(total / c0["mass"] - 1) < 1e-14
