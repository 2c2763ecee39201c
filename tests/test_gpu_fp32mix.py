"""The mixed-precision form (FP32 fields and stencils; FP64 specific internal energy,
Courant reduction and conservation sums) against the FP64 oracle.  FP32 rounds every
field to 6e-8 and the impact problem amplifies input perturbations by ~1e5 in the bulk
(the oracle's own response to 1e-15 perturbations, see gpu_util.py), so this form is not
held to field parity: it is held to the crater depth, crater diameter and peak-pressure
decay of the FP64 oracle within 2 %, to exact rest states, and to the conservation laws
at FP32 resolution."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle_cases as OC
from oracle import oracle as O
from paper_2403_04267_gb300 import salec, workloads as W


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    salec.load()


def _run_to(sim, t_end, max_steps=20000):
    n = 0
    while sim.scalars()["t"] < t_end and n < max_steps:
        sim.step(1)
        n += 1
    return n


def _peak_decay(pmax, dx, z_surface, nbins):
    """Max over cells of the peak over-pressure in distance bins from the impact point
    (on the axis at the surface)."""
    nz, nr = pmax.shape
    rc = (np.arange(nr) + 0.5) * dx
    zc = (np.arange(nz) + 0.5) * dx
    dist = np.hypot(rc[None, :], zc[:, None] - z_surface)
    edges = np.linspace(0, dist.max(), nbins + 1)
    out = np.zeros(nbins)
    for k in range(nbins):
        sel = (dist >= edges[k]) & (dist < edges[k + 1])
        out[k] = pmax[sel].max() if sel.any() else 0.0
    return out


def test_fp32mix_crater_and_peak_pressure_within_2_percent():
    spec = W.scaled_plain(160, radius_cells=8)
    t_end = 0.08
    g = salec.Sim(spec, precision="fp32mix")
    r = O.OracleSim(spec)
    _run_to(g, t_end)
    while r.scalars()["t"] < g.scalars()["t"]:
        r.step(1)
    assert g.scalars()["status"] == 0
    zs = spec["z_surface"]
    dx = spec["grid"]["dx"]
    cg = g.crater(zs, 64)
    d, D, prof = O.crater_metrics(r.surface_heights(), dx, zs, 64, (160 - 16) * dx)
    assert d > 5 * dx and D > 10 * dx                 # a real crater has formed
    assert abs(cg["depth"] / d - 1) < 0.02, (cg["depth"], d)
    assert abs(cg["diameter"] / D - 1) < 0.02, (cg["diameter"], D)
    pg = _peak_decay(g.get("pmax"), dx, zs, 12)
    pr = _peak_decay(r.get("pmax"), dx, zs, 12)
    sel = pr > 1e-3 * pr.max()
    assert np.all(np.abs(pg[sel] / pr[sel] - 1) < 0.02), (pg, pr)


def test_fp32mix_rest_states():
    g = salec.Sim(OC.gas_box_spec(37, 29), precision="fp32mix")
    rho, I = g.get("rho0"), g.get("I")
    g.step(200)
    assert np.all(g.get("vr") == 0.0) and np.all(g.get("vz") == 0.0)
    assert np.array_equal(g.get("rho0"), rho) and np.array_equal(g.get("I"), I)
    h = salec.Sim(OC.hydrostatic_spec(40, 120), precision="fp32mix")
    h.step(200)
    v = np.hypot(h.get("vr"), h.get("vz")).max()
    assert v / math.sqrt(26.7e9 / 2700.0) <= 1e-5      # FP32 rounding of the balance


def test_fp32mix_conservation_at_fp32_resolution():
    """Closed box, clean-up on (the mixed form requires f_min >= 1e-7): mass on the grid plus
    removed mass, z-momentum and KE + IE are kept to FP32 resolution over 40 steps."""
    spec = W.impact(48, 48, 10.0, W.basalt(strength=True), W.iron(), 4, 8e3, 30, 0)
    spec["grid"]["bc_top"] = "wall"
    g = salec.Sim(spec, precision="fp32mix")
    c0 = g.conservation()
    g.step(40)
    c1 = g.conservation()
    sc = g.scalars()
    assert sc["status"] == 0
    assert abs((c1["mass"] + sc["mass_discarded"]) / c0["mass"] - 1) < 1e-5
    assert abs(c1["zmom"] / c0["zmom"] - 1) < 1e-3
    assert abs((c1["ke"] + c1["ie"]) / (c0["ke"] + c0["ie"]) - 1) < 1e-3


def test_fp32mix_rejects_a_zero_cleanup_threshold():
    spec = W.plain_fp64_100()
    spec["grid"]["f_min"] = 0.0
    with pytest.raises(salec.SalecError):
        salec.Sim(spec, precision="fp32mix")
