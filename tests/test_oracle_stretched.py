"""Pins of the non-uniform grid (the paper's extension zones, Table 2: cells growing by a
constant factor away from a high-resolution zone).  Facts fixed outside the oracle: the
cells of a cylinder of radius R and height H hold R^2 H / 2 of volume per radian; a
sub-sampled sphere holds 2 R^3 / 3 whatever cells cut it; a uniform gas at rest stays
exactly at rest on any grid; a hydrostatic column on stretched rows stays at rest and
carries the weight of the compressible column above it; Sod's shock tube on a stretched
column follows the exact Riemann solution; the Courant step takes each cell's smaller
side; and the stretched strip cells still absorb the wave that reflects from the bottom
without them."""
import math

import numpy as np

import exact_riemann as ER
import oracle_cases as OC
from oracle import oracle as O
from paper_2403_04267_gb300 import workloads as W


def _stretched(nr, nz, seed=0):
    rng = np.random.default_rng(seed)
    return list(rng.uniform(0.5, 2.0, nr)), list(rng.uniform(0.5, 2.0, nz))


def test_extension_sizes_follow_the_table():
    """Table 2: 20 extension cells growing by 1.05 from 400 m reach the 1061 m maximum."""
    s = W.stretched_sizes(3, 400.0, 0, 20, 1.05, 1061.0, 0, 2)
    assert s[:3] == [400.0] * 3
    assert all(abs(s[3 + k] - 400.0 * 1.05 ** (k + 1)) < 1e-9 for k in range(19))
    assert s[22] == 1061.0 and s[23:] == [1061.0, 1061.0]
    lo = W.stretched_sizes(2, 1.0, 3, 0, 2.0)
    assert lo == [8.0, 4.0, 2.0, 1.0, 1.0]


def test_uniform_gas_box_on_a_random_grid_is_bitwise_at_rest():
    spec = OC.gas_box_spec(23, 19)
    dr, dz = _stretched(23, 19, 1)
    spec["grid"] = dict(spec["grid"], dr=dr, dz=dz)
    spec["layers"][0]["zhi"] = 2.0 * float(np.sum(dz))     # past the top: every row full
    s = O.OracleSim(spec)
    rho0, I0 = s.get("rho0").copy(), s.get("I").copy()
    s.step(200)
    assert np.all(s.get("vr") == 0.0) and np.all(s.get("vz") == 0.0)
    assert np.array_equal(s.get("rho0"), rho0) and np.array_equal(s.get("I"), I0)


def test_cell_volumes_fill_the_cylinder():
    dr, dz = _stretched(17, 13, 2)
    R, H = W.positions(dr)[-1], W.positions(dz)[-1]
    g = dict(W.grid(17, 13, 1.0, bc_top="wall"), dr=dr, dz=dz)
    gas = W.ideal_gas(1.4, rho0=3.0)
    spec = {"grid": g, "materials": [gas], "projectile": None,
            "layers": [dict(mat=0, zlo=0.0, zhi=H, rho=3.0, I0=1.0, vz=0.0)]}
    s = O.OracleSim(spec)
    assert math.isclose(s.conservation()["mass"], 3.0 * R * R * H / 2.0, rel_tol=1e-13)
    # a layer boundary inside a row fills that row's fraction
    spec["layers"] = [dict(mat=0, zlo=0.0, zhi=0.5 * H, rho=3.0, I0=1.0, vz=0.0)]
    s = O.OracleSim(spec)
    assert math.isclose(s.conservation()["mass"], 3.0 * R * R * H / 4.0, rel_tol=1e-13)


def test_sphere_volume_across_growing_cells():
    """A sphere of radius 12 over a zone of 6 unit cells and cells growing by 1.2 beyond
    it: the r-weighted sub-samples still give 2 R^3 / 3 per radian."""
    dr = W.stretched_sizes(6, 1.0, 0, 12, 1.2)
    dz = W.stretched_sizes(10, 1.0, 12, 12, 1.2)
    zc = W.positions(dz)[17]
    g = dict(W.grid(len(dr), len(dz), 1.0), dr=dr, dz=dz)
    gas = W.ideal_gas(1.4, rho0=1.0)
    spec = {"grid": g, "materials": [gas, dict(gas)], "layers": [],
            "projectile": dict(mat=1, radius=12.0, zc=zc, vz=0.0, rho=2.0, I0=1.0)}
    s = O.OracleSim(spec)
    vol = s.conservation()["mass"] / 2.0
    assert abs(vol / (2 * 12.0 ** 3 / 3) - 1) < 3e-3


def _ode_pressure(spec, zc):
    """dp/d(depth) = rho(p) g from the surface, rho(p) inverting p = A mu + B mu^2."""
    from scipy.integrate import solve_ivp
    m = spec["materials"][0]
    A, B, r0, g = m["A"], m["B"], m["rho0"], spec["grid"]["gravity"]
    zs = spec["layers"][0]["zhi"]

    def rhs(_, p):
        mu = 2.0 * p[0] / (A + np.sqrt(A * A + 4.0 * B * p[0]))
        return [r0 * (1.0 + mu) * g]

    depth = zs - zc
    order = np.argsort(depth)
    sol = solve_ivp(rhs, (0.0, depth.max()), [0.0], t_eval=depth[order], rtol=1e-12, atol=1e-3)
    out = np.empty_like(depth)
    out[order] = sol.y[0]
    return out


def test_hydrostatic_column_on_stretched_rows():
    """A basalt column under lunar gravity whose rows grow by 1.1 toward the bottom (12
    extension rows below 20 rows of 25 m): the set-up balances each vertex between rows
    of different heights, the pressures follow the compressible lithostatic ODE (the
    discrete balance weighs each half cell at its centre density: a first-order term at
    the surface, 1e-4 relative here), and the column stays at rest for 200 steps."""
    dz = W.stretched_sizes(24, 25.0, 12, 0, 1.1)
    spec = OC.hydrostatic_spec(6, len(dz), dx=25.0)
    zs = W.positions(dz)[28]
    spec["layers"][0]["zhi"] = zs
    spec["grid"] = dict(spec["grid"], dr=[25.0] * 6, dz=dz)
    s = O.OracleSim(spec)
    zv = np.concatenate([[0.0], np.cumsum(dz)])
    zc = 0.5 * (zv[:-1] + zv[1:])
    p = s.get("p")[:28, 0]
    ref = _ode_pressure(spec, zc[:28])
    assert np.max(np.abs(p / ref - 1.0)) < 2e-4
    s.step(200)
    v = np.hypot(s.get("vr"), s.get("vz")).max()
    assert v / np.sqrt(26.7e9 / 2700.0) <= 1e-12


def _sod_stretched(n_half, f):
    """Sod's tube on [0, 1] with cells growing by f from both ends toward the middle (the
    diaphragm at z = 1/2 lies on a row boundary)."""
    half = f ** np.arange(n_half)
    half = half / half.sum() * 0.5
    dz = np.concatenate([half, half[::-1]])
    spec = OC.sod_spec(2 * n_half)
    z_mid = W.positions(dz)[n_half]
    spec["grid"] = dict(spec["grid"], dr=[1.0 / (2 * n_half)] * 3, dz=list(dz))
    spec["layers"][0]["zhi"] = z_mid
    spec["layers"][1]["zlo"] = z_mid
    spec["layers"][1]["zhi"] = 2.0 * W.positions(dz)[-1]
    return spec, dz


def test_sod_on_a_stretched_column():
    """Cells from 0.0031 to 0.0069 (factor 1.008 over 100 cells each way): the density
    stays within 2.5 % (L1, cell-size weighted) of the exact solution at t = 0.2, no worse
    than 1.5 times the uniform 200-cell error, and the flow stays one-dimensional."""
    spec, dz = _sod_stretched(100, 1.008)
    s = O.OracleSim(spec)
    while s.scalars()["t"] < 0.2 - 1e-12:
        s.step(1)
    t = s.scalars()["t"]
    zv = np.concatenate([[0.0], np.cumsum(dz)])
    z = 0.5 * (zv[:-1] + zv[1:])
    ex = ER.sample(z, t, zv[100], 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)[0]
    rho = s.get("rho0")
    err = np.sum(np.abs(rho[:, 0] - ex) * dz) / np.sum(ex * dz)
    u = O.OracleSim(OC.sod_spec(200))
    while u.scalars()["t"] < 0.2 - 1e-12:
        u.step(1)
    zu = (np.arange(200) + 0.5) / 200
    exu = ER.sample(zu, u.scalars()["t"], 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)[0]
    err_u = np.sum(np.abs(u.get("rho0")[:, 0] - exu)) / np.sum(exu)
    print("stretched", err, "uniform", err_u)
    assert err < 0.025 and err < 1.5 * err_u
    assert np.abs(rho - rho[:, :1]).max() <= 1e-12 * rho.max()
    assert np.abs(s.get("vr")).max() <= 1e-12


def test_dt_takes_the_smaller_side():
    """2 x 2 ideal gas with cells 0.5 wide and 0.2 / 0.7 high: Eq. 14 with L = min(dr, dz)."""
    g = dict(W.grid(2, 2, 0.5, bc_top="wall", cfl=0.4, dt_init=1e30, av_cq=0.0, av_cl=0.0),
             dr=[0.5, 0.5], dz=[0.2, 0.7])
    gas = W.ideal_gas(1.4)
    spec = {"grid": g, "materials": [gas], "projectile": None,
            "layers": [dict(mat=0, zlo=0.0, zhi=0.9, rho=1.0, I0=1.0, vz=0.0)]}
    s = O.OracleSim(spec)
    I = np.array([[1.0, 4.0], [9.0, 2.0]])
    s.set("I", I)
    vr = np.zeros((3, 3)); vz = np.zeros((3, 3))
    vr[1, 1] = 3.0; vz[1, 1] = 4.0
    s.set("vr", vr); s.set("vz", vz)
    s.step(1)
    c = np.sqrt(1.4 * 0.4 * I)
    L = np.array([[0.2, 0.2], [0.5, 0.5]])
    assert math.isclose(s.scalars()["dt"], 0.4 * (L / (5.0 + c)).min(), rel_tol=1e-15)


def _axis_band_history(spec, t_end):
    s = O.OracleSim(spec)
    p0 = s.get("p").copy()
    out = []
    while s.scalars()["t"] < t_end:
        s.step(10)
        sc = s.scalars()
        assert sc["status"] == 0
        dp = np.abs(s.get("p") - p0)[30:60]
        out.append((sc["t"], dp[:, :8].max(), dp[:, 40:60].max()))
    return np.array(out)


def _peak(h, t0, t1, col):
    sel = (h[:, 0] >= t0) & (h[:, 0] <= t1)
    assert sel.sum() >= 3
    return h[sel, col].max()


def test_stretched_strips_absorb_the_bottom_reflection():
    """The 100 x 100 physics (10 m cells, basalt, 10 km/s) on an 80-cell core with 10
    extension cells growing by 1.05 and 16 strip cells of the largest size on the right
    and at the bottom.  With the strips' damping off the wave comes back from the bottom
    wall through the stretched cells: about 0.4 GPa on the axis and 0.5 GPa in the band of
    columns 40-59 at 0.37-0.50 s (rows 30-59); with the damping on, less than a fifth of it
    on the axis and a tenth in the band.  Before the reflection the two runs agree."""
    spec = W.stretched_impact(80, 10.0, 10, 16, W.basalt(), None, 4, 10e3, 24)
    off = dict(spec, grid=dict(spec["grid"], pml_r=0, pml_b=0))
    h0, h1 = _axis_band_history(off, 0.5), _axis_band_history(spec, 0.5)
    assert abs(_peak(h0, 0.0, 0.2, 1) / _peak(h1, 0.0, 0.2, 1) - 1.0) < 1e-2
    a0, a1 = _peak(h0, 0.37, 0.47, 1), _peak(h1, 0.37, 0.47, 1)
    b0, b1 = _peak(h0, 0.40, 0.50, 2), _peak(h1, 0.40, 0.50, 2)
    print(f"axis {a0:.3e} vs {a1:.3e}; band {b0:.3e} vs {b1:.3e}")
    assert a0 > 2e8 and a0 > 5.0 * a1
    assert b0 > 10.0 * b1
