"""Pins of the crater read-out: a synthetic paraboloid bowl written as volume fractions
that vary linearly across the surface; the 1/2-crossing interpolated between cell
centres recovers the bowl exactly at every column."""
import numpy as np

from oracle import oracle as O
from paper_2403_04267_gb300 import workloads as W


def test_paraboloid_bowl():
    nr, nz, dx = 40, 60, 10.0
    spec = {"grid": W.grid(nr, nz, dx), "materials": [W.basalt()], "projectile": None,
            "layers": [dict(mat=0, zlo=0.0, zhi=400.0)]}
    s = O.OracleSim(spec)
    rc = (np.arange(nr) + 0.5) * dx
    zs, depth, radius = 400.0, 120.0, 200.0
    h = np.where(rc < radius, zs - depth * (1 - (rc / radius) ** 2), zs)
    zc = (np.arange(nz) + 0.5) * dx
    # phi = 1/2 - (z - h)/(2 dx) clipped to [0, 1]: linear across the surface
    phi = np.clip(0.5 - (zc[:, None] - h[None, :]) / (2 * dx), 0.0, 1.0)
    s.set("f0", phi)
    s.set("rho0", np.where(phi > 0, 2700.0, 0.0))
    got = s.surface_heights()
    assert np.allclose(got, h, rtol=0, atol=1e-9)
    d, D, prof = O.crater_metrics(got, dx, zs, 64, nr * dx)
    assert abs(d - (zs - h[0])) < 1e-9
    assert abs(D - 2 * radius) <= dx + 1e-9     # rim regained within one cell
