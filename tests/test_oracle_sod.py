"""Pin: Sod's shock tube along z in a narrow free-slip column (ideal gas, gamma = 1.4).
Checks the exact solver against the tabulated star state, then the oracle's density
against the exact solution: L1 error below 2 % at 400 cells and decreasing under
refinement; the solution is r-independent and v_r stays at round-off."""
import numpy as np
import pytest

import exact_riemann as ER
import oracle_cases as OC
from oracle import oracle as O


def _golden():
    vals = {}
    with open(__file__.replace("test_oracle_sod.py", "golden/sod_star_state.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_exact_solver_matches_tabulated_star_state():
    g = _golden()
    p, u = ER.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    assert abs(p - g["p_star"]) < 1e-5 and abs(u - g["u_star"]) < 1e-5
    x = np.array([0.5 + 0.5 * u * 0.2 / 0.2 * 0.2, 0.5 + 1.2 * u * 0.2])
    r = ER.sample(np.array([0.5 + 0.5 * u * 0.2]), 0.2, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    assert abs(r[0, 0] - g["rho_star_left"]) < 1e-4
    r = ER.sample(np.array([0.5 + 1.1 * u * 0.2]), 0.2, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    assert abs(r[0, 0] - g["rho_star_right"]) < 1e-4


def _run(nz):
    s = O.OracleSim(OC.sod_spec(nz))
    while s.scalars()["t"] < 0.2 - 1e-12:
        s.step(1)
    t = s.scalars()["t"]
    rho = s.get("rho0")
    z = (np.arange(nz) + 0.5) / nz
    ex = ER.sample(z, t, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    err = np.abs(rho[:, 0] - ex[0]).sum() / nz / (ex[0].sum() / nz)
    return s, err


def test_sod_converges_and_stays_one_dimensional():
    errs = {}
    for nz in (100, 200, 400):
        s, errs[nz] = _run(nz)
    assert errs[400] < 0.02
    assert errs[400] < errs[200] < errs[100]
    rho = s.get("rho0")
    assert np.abs(rho - rho[:, :1]).max() <= 1e-12 * rho.max()
    assert np.abs(s.get("vr")).max() <= 1e-12
