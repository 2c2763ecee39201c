"""Pins: exact preservation of rest states.  A uniform ideal gas at 1e5 Pa in a closed
box stays bitwise at rest (the corner forces of a uniform pressure cancel exactly,
including the axisymmetric hoop part).  A Tillotson column in discrete hydrostatic
equilibrium under gravity stays at rest to |v|/c <= 1e-12 for 200 steps."""
import numpy as np

import oracle_cases as OC
from oracle import oracle as O
from paper_2403_04267_gb300 import workloads as W


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


def _lithostatic_ode(spec, z_eval):
    """Pressure of the layered column from dp/dz = -rho(p) g, integrated down from the
    surface (p = 0) layer by layer with scipy; rho(p) inverts the cold Tillotson curve
    p = A mu + B mu^2 of the layer's material (rho = rho0 (1 + mu))."""
    from scipy.integrate import solve_ivp
    g = spec["grid"]["gravity"]
    out = np.full(len(z_eval), np.nan)
    p_top = 0.0
    for lay in sorted(spec["layers"], key=lambda d: -d["zhi"]):
        m = spec["materials"][lay["mat"]]
        A, B, r0 = m["A"], m["B"], m["rho0"]

        def rhs(z, p, A=A, B=B, r0=r0):
            mu = 2.0 * p[0] / (A + np.sqrt(A * A + 4.0 * B * p[0]))
            return [r0 * (1.0 + mu) * g]          # d p / d(depth)

        zs = z_eval[(z_eval >= lay["zlo"]) & (z_eval < lay["zhi"])]
        depth = np.sort(lay["zhi"] - zs)
        sol = solve_ivp(rhs, (0.0, lay["zhi"] - lay["zlo"]), [p_top], t_eval=depth, rtol=1e-12, atol=1e-3)
        for d, p in zip(sol.t, sol.y[0]):
            out[np.argmin(np.abs(z_eval - (lay["zhi"] - d)))] = p
        p_top = solve_ivp(rhs, (0.0, lay["zhi"] - lay["zlo"]), [p_top], rtol=1e-12, atol=1e-3).y[0, -1]
    return out


def test_stacked_layers_carry_the_overburden_and_stay_at_rest():
    """Sediment over crust over mantle (the paper's Sect. 4 column, 400 m cells) under
    Earth gravity: each layer starts from the weight of the layers above it.  Pin: the cell
    pressures equal the lithostatic pressure of the compressible column, integrated as an
    ODE across the density jumps at the interfaces.  The discrete balance weighs each half
    cell at its centre's density, so the surface and each interface add a first-order term
    g dx/2 times the density change across that half cell (about 700 Pa at the surface
    here, 1.3e-4 of the top row's pressure); inside a layer it is second-order.  Bound:
    2e-4 relative.  A layer that ignored its overburden would be off by the whole weight
    above it (order 1).  Then the column stays at rest."""
    spec = W.layered_impact(6, 60, 400.0, 50, 7, 20, 3, 12e3, 0)
    spec["projectile"] = None
    s = O.OracleSim(spec)
    dx = spec["grid"]["dx"]
    zc = (np.arange(60) + 0.5) * dx
    ref = _lithostatic_ode(spec, zc)
    p = s.get("p")[:, 0]
    filled = zc < 50 * dx
    assert np.all(p[~filled] == 0.0)
    assert np.max(np.abs(p[filled] / ref[filled] - 1.0)) < 2e-4
    # the crust's top row (row 42) carries the 7 sediment rows above it
    assert p[42] > 7 * dx * 9.81 * 2710.0
    s.step(200)
    c = np.sqrt(130e9 / 3320.0)
    v = np.hypot(s.get("vr"), s.get("vz")).max()
    assert v / c <= 1e-12
    assert s.scalars()["status"] == 0
