"""Pins of the set-up: the r-weighted sub-sampled sphere has the volume 2 R^3 / 3 per
radian, and the layer fills exactly its rows."""
import numpy as np

from oracle import oracle as O
from paper_2403_04267_gb300 import workloads as W


def test_sphere_volume_and_layer():
    w = W.impact(60, 60, 10.0, W.basalt(), W.iron(), 12, 10e3, 30, 0)
    s = O.OracleSim(w)
    nr, dx = 60, 10.0
    V = (np.arange(nr) + 0.5) * dx * dx * dx
    vol = (s.get("f1") * V[None, :]).sum()
    R = 12 * dx
    assert abs(vol / (2 * R ** 3 / 3) - 1) < 2e-3
    f0 = s.get("f0")
    assert np.all(f0[:30] == 1.0) and np.all(f0[30:] == 0.0)
    # projectile moves down, target rests
    vz = s.get("vz")
    assert vz.min() == -10e3 and np.all(vz[:30] == 0.0)
