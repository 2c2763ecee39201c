"""Pin: planar Tillotson shock.  Basalt moving at 2 km/s onto the no-slip bottom wall
drives a shock up the column; the plateau behind it must satisfy the Rankine-Hugoniot
jump conditions rho0 (U + u) = rho1 U, p1 = rho0 (U + u) u, I1 = p1 (1/rho0 - 1/rho1)/2
with p1 = p(rho1, I1), solved here by bisection on the shock speed U."""
import numpy as np

import oracle_cases as OC
from oracle import oracle as O
from paper_2403_04267_gb300 import workloads as W


def _rh(up=2000.0):
    bas = W.basalt()
    rho0 = bas["rho0"]

    def resid(U):
        rho1 = rho0 * (U + up) / U
        p1 = rho0 * (U + up) * up
        I1 = 0.5 * p1 * (1 / rho0 - 1 / rho1)
        return O.eos(bas, rho1, I1)[0] - p1, rho1, p1, I1

    lo, hi = 500.0, 30000.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if resid(mid)[0] > 0:
            lo = mid
        else:
            hi = mid
    U = 0.5 * (lo + hi)
    return (U,) + resid(U)[1:]


def test_tillotson_shock_jump():
    U, rho1, p1, I1 = _rh()
    nz, L = 200, 400.0
    dx = L / nz
    s = O.OracleSim(OC.rh_spec(nz))
    while s.scalars()["t"] < 0.045:
        s.step(1)
    t = s.scalars()["t"]
    rho = s.get("rho0")[:, 0]
    p = s.get("p")[:, 0]
    I = s.get("I")[:, 0]
    z = (np.arange(nz) + 0.5) * dx
    half = 0.5 * (2700.0 + rho1)
    k = np.where(rho > half)[0].max()
    zs = z[k] + (rho[k] - half) / (rho[k] - rho[k + 1]) * dx
    assert abs(zs / t / U - 1) < 0.02
    sel = (z > 0.2 * zs) & (z < 0.7 * zs)
    assert abs(rho[sel].mean() / rho1 - 1) < 0.01
    assert abs(p[sel].mean() / p1 - 1) < 0.01
    assert abs(I[sel].mean() / I1 - 1) < 0.01
