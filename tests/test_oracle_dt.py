"""Pin: the Courant step on a 2 x 2 ideal-gas grid, computed by hand from Eq. 14 with the
cell's largest vertex speed and c^2 = gamma (gamma - 1) I."""
import math

import numpy as np

from oracle import oracle as O
from paper_2403_04267_gb300 import workloads as W


def test_dt_two_by_two():
    g = W.grid(2, 2, 0.5, bc_top="wall", cfl=0.4, dt_init=1e30, av_cq=0.0, av_cl=0.0)
    gas = W.ideal_gas(1.4)
    spec = {"grid": g, "materials": [gas], "projectile": None,
            "layers": [dict(mat=0, zlo=0.0, zhi=1.0, rho=1.0, I0=1.0, vz=0.0)]}
    s = O.OracleSim(spec)
    I = np.array([[1.0, 4.0], [9.0, 2.0]])
    s.set("I", I)
    vr = np.zeros((3, 3)); vz = np.zeros((3, 3))
    vr[1, 1] = 3.0; vz[1, 1] = 4.0          # centre vertex: |v| = 5
    vz[2, 1] = 0.0
    s.set("vr", vr); s.set("vz", vz)
    s.step(1)
    c = np.sqrt(1.4 * 0.4 * I)
    cand = 0.5 / (5.0 + c)                  # every cell touches the centre vertex
    assert math.isclose(s.scalars()["dt"], 0.4 * cand.min(), rel_tol=1e-15)
    # growth limit
    g2 = dict(g, dt_init=1e-5)
    s2 = O.OracleSim(dict(spec, grid=g2))
    s2.step(1)
    assert math.isclose(s2.scalars()["dt"], 1.2e-5, rel_tol=1e-15)
