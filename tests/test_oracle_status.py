"""Pins of the failure status word (bit 1: a present material with a non-positive
Lagrangian volume or density; bit 2: a NaN Courant candidate, energy or velocity; bit 4: a
step below dt_min) on host-injected states: a gas box at rest with one cell's density
negative, one vertex velocity NaN, or dt_min above the Courant step."""
import numpy as np

import oracle_cases as OC
from oracle import oracle as O


def _box():
    return O.OracleSim(OC.gas_box_spec(6, 5))


def test_clean_box_reports_nothing():
    s = _box()
    s.step(3)
    assert s.scalars()["status"] == 0


def test_negative_density_sets_bit_1():
    s = _box()
    rho = s.get("rho0")
    rho[2, 3] = -rho[2, 3]
    s.set("rho0", rho)
    s.step(1)
    assert s.scalars()["status"] & 1


def test_nan_velocity_sets_bit_2():
    """The Courant pass of the step keeps a NaN vertex speed (a maximum that drops NaN
    would report the state only once the NaN reached a volume)."""
    s = _box()
    vz = s.get("vz")
    vz[2, 3] = np.nan
    s.set("vz", vz)
    s.phase0()
    assert s.scalars()["status"] == 2


def test_step_below_dt_min_sets_bit_4():
    spec = OC.gas_box_spec(6, 5)
    spec["grid"]["dt_min"] = 1.0
    s = O.OracleSim(spec)
    s.step(1)
    assert s.scalars()["status"] == 4
