"""Non-uniform grids on the GPU (the paper's extension zones, Table 2): the CUDA path
against the oracle on stretched grids, exact rest states in both precisions, and the
paper's own grid (a 462 x 462 zone of 400 m cells, 20 extension cells growing by 1.05 to
1061 m, 30 PML cells) with its layered target."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import gpu_util as U
import oracle_cases as OC
from oracle import oracle as O
from paper_2403_04267_gb300 import salec, workloads as W

TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    salec.load()


def _check(g, r, spec, tol=TOL, sensitivity=None):
    U.assert_parity(g, r, spec, tol=tol, sensitivity=sensitivity, status_zero=True)


def _parity_run(spec, n1, n2):
    g, r = salec.Sim(spec), O.OracleSim(spec)
    g.step(n1)
    r.step(n1)
    _check(g, r, spec)
    r2 = U.perturbed(O.OracleSim(spec))
    r2.step(n1)
    for s in (g, r, r2):
        s.step(n2)
    sens = U.sensitivity(r, r2, spec)
    _check(g, r, spec, sensitivity=sens)
    return g, r


def test_stretched_hydro_impact_against_oracle():
    """The 100 x 100 physics on a 40-cell core with 8 extension cells growing by 1.05 and
    8 strip cells: every field within the FP64 bar after 1 step and after 150 more."""
    spec = W.stretched_impact(40, 10.0, 8, 8, W.basalt(), None, 3, 10e3, 12)
    g, r = _parity_run(spec, 1, 150)
    cg = g.crater(spec["z_surface"], 32)
    h = r.surface_heights()
    rc = np.asarray(W.positions(spec["grid"]["dr"]))
    rc = 0.5 * (rc[:-1] + rc[1:])
    d, D, prof = O.crater_metrics(h, 10.0, spec["z_surface"], 32, W.positions(spec["grid"]["dr"])[-9], rc=rc)
    assert np.allclose(cg["heights"], h, rtol=0, atol=1e-6)
    assert abs(cg["depth"] - d) < 1e-6 and abs(cg["diameter"] - D) < 1e-6
    assert np.allclose(cg["profile"], prof, rtol=0, atol=1e-6)


def test_stretched_layered_target_against_oracle():
    """Three layers with Table 1 strength under gravity on a stretched grid: 1 step within
    the FP64 bar, 60 more within it or 100 x the oracle's own response to a 1e-15 input
    perturbation."""
    _parity_run(OC.stretched_layered_spec(), 1, 60)


@pytest.mark.parametrize("precision", ["fp64", "fp32mix"])
def test_gas_box_on_a_random_grid_is_bitwise_at_rest(precision):
    rng = np.random.default_rng(1)
    spec = OC.gas_box_spec(23, 19)
    dr, dz = list(rng.uniform(0.5, 2.0, 23)), list(rng.uniform(0.5, 2.0, 19))
    spec["grid"] = dict(spec["grid"], dr=dr, dz=dz)
    spec["layers"][0]["zhi"] = 2.0 * W.positions(dz)[-1]
    g = salec.Sim(spec, precision=precision)
    rho0 = g.get("rho0").copy()
    g.step(200)
    assert np.all(g.get("vr") == 0.0) and np.all(g.get("vz") == 0.0)
    assert np.array_equal(g.get("rho0"), rho0)


@pytest.mark.parametrize("precision,mass_tol", [("fp64", 1e-10), ("fp32mix", 1e-4)])
def test_paper_grid_layered_impact_runs(precision, mass_tol):
    """The paper's grid and target (512 x 532 cells), 1500 steps: no failure, the crater
    opens, and the mass balance closes (grid + top outflow + clean-up - strip damping)."""
    spec = W.chicxulub_stretched()
    g = salec.Sim(spec, precision=precision)
    c0 = g.conservation()
    g.step(1500)
    sc = g.scalars()
    assert sc["status"] == 0, sc
    c1 = g.conservation()
    acc = c1["mass"] + sc["mass_out"] + sc["mass_discarded"] - sc["mass_pml"]
    cr = g.crater(spec["z_surface"], 64)
    print(precision, "t", sc["t"], "mass", c0["mass"], "accounted", acc, "crater", cr["depth"], cr["diameter"])
    assert abs(acc / c0["mass"] - 1.0) < mass_tol
    assert cr["depth"] > 2 * 400.0
