"""Pins of the artificial viscosity q and of the running peak over-pressure (phase 0).

Viscosity (reading R3: q = rho_bar (c_Q L^2 (div v)^2 - c_L L c div v) in compression, 0 in
expansion, c_Q = 1, c_L = 0.25, L the cell size).  A homologous contraction
v = -k (r, z - z0) has div v = -3k exactly in cylindrical coordinates
((1/r) d(r v_r)/dr = -2k, dv_z/dz = -k), and the finite-volume divergence of a cell,
(r_{i+1} u_R - r_i u_L) / (r_c dr) + (u_T - u_B) / dz, reproduces it exactly for any
column (r_{i+1}^2 - r_i^2 = 2 r_c dr): so every cell, the one on the axis included, must
carry the same q.  Its two terms are separated by their scaling in k (quadratic: the
von Neumann-Richtmyer term; linear: the Landshoff term), so swapped constants, a dropped
term or a planar (unweighted) radial divergence each fail.

Peak over-pressure (Sect. 4, the decay of the peak pressure with distance):
pmax = max over time of p_bar - p0(z), p_bar = sum f_m p_m / Phi the pressure of the
matter in the cell, p0 the reference (initial) pressure of its row.  Pins: a half-empty
gas cell at three times the reference pressure has an over-pressure of exactly twice the
reference (the void does not dilute it, and it is measured from p0, not from 0); a
column in hydrostatic equilibrium keeps pmax = 0; behind a planar Tillotson shock pmax
is the Rankine-Hugoniot pressure, ahead of it nothing above round-off.
"""
import numpy as np

import oracle_cases as OC
from oracle import oracle as O
from paper_2403_04267_gb300 import workloads as W
from test_oracle_rh import _rh

GAMMA, RHO, P_REF = 1.4, 1.2, 1e5


def _gas_block(nr=6, nz=5, dx=1.0, spacing=None, **gkw):
    gas = W.ideal_gas(GAMMA, rho0=RHO)
    g = W.grid(nr, nz, dx, bc_top="wall", **gkw)
    if spacing is not None:
        g["dr"], g["dz"] = spacing
    zs = W.positions(spacing[1])[-1] if spacing is not None else nz * dx
    spec = {"grid": g, "materials": [gas], "projectile": None,
            "layers": [dict(mat=0, zlo=0.0, zhi=zs, rho=RHO, I0=P_REF / ((GAMMA - 1) * RHO), vz=0.0)]}
    return O.OracleSim(spec), spec


def _homologous(s, spec, k):
    """Vertex velocities v = -k (r, z - z0) of a uniform contraction (k > 0) or dilation."""
    g = spec["grid"]
    nr, nz = g["nr"], g["nz"]
    rv = np.asarray(W.positions(g["dr"])) if "dr" in g else np.arange(nr + 1) * g["dx"]
    zv = np.asarray(W.positions(g["dz"])) if "dz" in g else np.arange(nz + 1) * g["dx"]
    s.set("vr", np.broadcast_to(-k * rv[None, :], (nz + 1, nr + 1)))
    s.set("vz", np.broadcast_to(-k * (zv[:, None] - 0.5 * zv[-1]), (nz + 1, nr + 1)))
    return rv, zv


def _q(s, spec, k):
    """q of every cell (P_total - p with Phi = 1) under the homologous field of rate k."""
    _homologous(s, spec, k)
    s.phase0()
    return s.get("P_total") - s.get("p")


def test_viscosity_of_a_homologous_contraction_is_uniform_and_splits_into_its_two_terms():
    s, spec = _gas_block()
    c = np.sqrt(GAMMA * P_REF / RHO)              # ideal-gas sound speed
    dx, k = 1.0, 10.0
    q1, q2 = _q(s, spec, k), _q(s, spec, 2 * k)
    # one value in every cell (the axis column included): div v = -3k everywhere
    assert np.ptp(q1) <= 1e-12 * q1.max() and np.ptp(q2) <= 1e-12 * q2.max()
    du = 3 * k * dx                               # velocity jump across a cell, L |div v|
    # quadratic term from q(2k) - 2 q(k), linear from 4 q(k) - q(2k)
    quad = (q2 - 2 * q1).mean() / 2
    lin = (4 * q1 - q2).mean() / 2
    assert abs(quad / (1.0 * RHO * du * du) - 1) < 1e-12          # c_Q rho (L div)^2
    assert abs(lin / (0.25 * RHO * c * du) - 1) < 1e-12           # c_L rho c L |div|


def test_viscosity_is_zero_in_expansion_and_scales_with_its_constants():
    s, spec = _gas_block()
    assert np.all(_q(s, spec, -10.0) == 0.0)      # dilation: no viscous pressure
    c = np.sqrt(GAMMA * P_REF / RHO)
    # only the quadratic term (c_L = 0): q = c_Q rho du^2 with du = 3 k L, any cell size
    for dx in (0.5, 2.0):
        s, spec = _gas_block(dx=dx, av_cq=2.0, av_cl=0.0)
        q = _q(s, spec, 4.0)
        assert np.allclose(q, 2.0 * RHO * (12.0 * dx) ** 2, rtol=1e-12, atol=0)
    # only the linear term (c_Q = 0): q = c_L rho c du
    s, spec = _gas_block(av_cq=0.0, av_cl=0.5)
    assert np.allclose(_q(s, spec, 4.0), 0.5 * RHO * c * 12.0, rtol=1e-12, atol=0)


def test_viscosity_length_on_a_stretched_grid_is_the_smaller_side():
    """On cells of unequal sides the length is min(dr, dz); the contraction still has
    div v = -3k in every cell."""
    dr = [0.5, 0.7, 1.1, 1.6, 0.9]
    dz = [1.3, 0.4, 0.8, 1.0]
    s, spec = _gas_block(nr=len(dr), nz=len(dz), spacing=(dr, dz), av_cq=1.0, av_cl=0.0)
    k = 3.0
    q = _q(s, spec, k)
    L = np.minimum(np.asarray(dr)[None, :], np.asarray(dz)[:, None])
    assert np.allclose(q, RHO * (3 * k * L) ** 2, rtol=1e-12, atol=0)


def test_peak_overpressure_of_a_half_empty_cell_is_measured_from_the_reference():
    s, spec = _gas_block(nr=4, nz=3)
    assert np.all(s.get("pmax") == 0.0)
    s.set("f0", np.full((3, 4), 0.5))
    s.set("I", np.full((3, 4), 3 * P_REF / ((GAMMA - 1) * RHO)))
    s.phase0()
    # the matter's own pressure is 3 p_ref; the reference row pressure p_ref
    assert np.allclose(s.get("pmax"), 2 * P_REF, rtol=1e-13, atol=0)
    # a later, lower pressure leaves the running maximum alone
    s.set("I", np.full((3, 4), 1.5 * P_REF / ((GAMMA - 1) * RHO)))
    s.phase0()
    assert np.allclose(s.get("pmax"), 2 * P_REF, rtol=1e-13, atol=0)


def test_peak_overpressure_stays_zero_in_hydrostatic_equilibrium():
    s = O.OracleSim(OC.hydrostatic_spec(6, 40))
    assert s.get("p")[0, 0] > 3e6                 # a loaded column (30 rows of basalt): p0 far from 0
    s.step(200)
    assert np.abs(s.get("pmax")).max() <= 1e-9 * s.get("p").max()


def test_peak_overpressure_behind_a_tillotson_shock_is_the_hugoniot_pressure():
    U, rho1, p1, I1 = _rh()
    nz, L = 200, 400.0
    dx = L / nz
    s = O.OracleSim(OC.rh_spec(nz))
    while s.scalars()["t"] < 0.045:
        s.step(1)
    t = s.scalars()["t"]
    pmax = s.get("pmax")[:, 0]
    z = (np.arange(nz) + 0.5) * dx
    zs = U * t                                    # shock position
    behind = (z > 0.2 * zs) & (z < 0.8 * zs)
    assert abs(pmax[behind].mean() / p1 - 1) < 0.01
    assert np.all(np.abs(pmax[behind] / p1 - 1) < 0.03)
    # not yet reached: nothing beyond round-off (the column still moves at u_p, compressed
    # by nothing but the rarefaction's precursor from the outflow top)
    ahead = z > zs + 10 * dx
    assert ahead.sum() > 20 and np.abs(pmax[ahead]).max() <= 1e-9 * p1
