"""Small synthetic set-ups shared by the oracle pins and the GPU parity tests (parameter
dictionaries only; no arithmetic of the method)."""
from __future__ import annotations

import numpy as np

from paper_2403_04267_gb300 import workloads as W


def sod_spec(nz: int, nr: int = 3) -> dict:
    dx = 1.0 / nz
    g = W.grid(nr, nz, dx, bc_top="wall")
    gas = W.ideal_gas(1.4)
    return {"grid": g, "materials": [gas], "projectile": None, "layers": [
        dict(mat=0, zlo=0.0, zhi=0.5, rho=1.0, I0=1.0 / (0.4 * 1.0), vz=0.0),
        dict(mat=0, zlo=0.5, zhi=1.0, rho=0.125, I0=0.1 / (0.4 * 0.125), vz=0.0)]}


def rh_spec(nz: int, up: float = 2000.0, length: float = 400.0) -> dict:
    bas = dict(W.basalt(), p_t=-1e12)
    g = W.grid(3, nz, length / nz, bc_top="outflow")
    return {"grid": g, "materials": [bas], "projectile": None,
            "layers": [dict(mat=0, zlo=0.0, zhi=length, rho=2700.0, I0=0.0, vz=-up)]}


def gas_box_spec(nr: int, nz: int, p: float = 1e5) -> dict:
    gas = W.ideal_gas(1.4, rho0=1.2)
    g = W.grid(nr, nz, 1.0, bc_top="wall")
    return {"grid": g, "materials": [gas], "projectile": None,
            "layers": [dict(mat=0, zlo=0.0, zhi=float(nz), rho=1.2, I0=p / (0.4 * 1.2), vz=0.0)]}


def hydrostatic_spec(nr: int, nz: int, dx: float = 25.0, g: float = 1.62) -> dict:
    bas = W.basalt(strength=True)
    gr = W.grid(nr, nz, dx, gravity=g, bc_top="outflow")
    return {"grid": gr, "materials": [bas], "projectile": None,
            "layers": [dict(mat=0, zlo=0.0, zhi=0.75 * nz * dx, rho=0.0, I0=0.0, vz=0.0)]}


def plane_wave_spec(nz: int, pml_b: int, av: bool = False, dx: float = 10.0) -> dict:
    bas = dict(W.basalt(), p_t=-1e12)
    kw = {} if av else dict(av_cq=0.0, av_cl=0.0)
    g = W.grid(2, nz, dx, bc_top="wall", pml_b=pml_b, pml_R=0.01, **kw)
    return {"grid": g, "materials": [bas], "projectile": None,
            "layers": [dict(mat=0, zlo=0.0, zhi=nz * dx, rho=2700.0, I0=0.0, vz=0.0)]}


def plane_wave_fields(nz: int, dx: float = 10.0, U: float = 1.0, width: float = 20.0,
                      centre: float = 0.6):
    """Density and vertex z-velocity of a Gaussian pulse travelling down (linear acoustics
    of basalt: rho' = rho0 U g / c, v_z = -U g)."""
    bas = W.basalt()
    c = np.sqrt(bas["A"] / bas["rho0"])
    zc = centre * nz * dx
    zcell = (np.arange(nz) + 0.5) * dx
    zv = np.arange(nz + 1) * dx
    gc = np.exp(-((zcell - zc) / (width * dx / 2)) ** 2)
    gv = np.exp(-((zv - zc) / (width * dx / 2)) ** 2)
    rho = bas["rho0"] * (1 + U * gc / c)
    vz = -U * gv
    vz[0] = 0.0
    vz[-1] = 0.0
    return rho, vz, c


def random_impact_spec(seed: int, nr: int, nz: int, nmat: int = 2, strength: bool = True,
                       pml: int = 4, gravity: float = 1.62) -> dict:
    """Small impact with ragged sizes used as a brute-force edge case."""
    rng = np.random.default_rng(seed)
    tgt = W.basalt(strength=strength, cohesion=float(rng.uniform(1e6, 1e8)),
                   friction=float(rng.uniform(0.4, 0.8)))
    proj = W.iron() if nmat == 2 else None
    surface = max(2, int(0.6 * nz))
    rad = float(rng.uniform(1.5, max(1.6, min(nr, nz) / 5)))
    v = float(rng.uniform(3e3, 15e3))
    w = W.impact(nr, nz, 20.0, tgt, proj, rad, v, surface, pml, gravity=gravity)
    w["grid"]["pml_r"] = min(pml, nr - 1)
    w["grid"]["pml_b"] = min(pml, nz - 1)
    return w


def axis_focus_spec(n: int, pml: int) -> dict:
    """The 100 x 100 impact's physics (10 m cells, basalt half-space with its surface at
    70 % of the height, a 10 km/s projectile of radius n/20 cells) on an n x n grid with
    reflecting walls (free-slip right, no-slip bottom), with or without PML strips of
    `pml` cells: the setting of the paper's reflected-wave anomaly (Sect. 5)."""
    return W.impact(n, n, 10.0, W.basalt(), None, 5 * n / 100, 10e3, int(0.7 * n), pml)


def axis_anomaly_history(sim, n: int, t_end: float, every: int = 10):
    """(t, axis, band) every `every` steps up to t_end: the largest |p - p(0)| in the
    cells within 0.08 n of the axis, and in the band of columns 0.40 n .. 0.55 n, both
    between 0.15 n and 0.55 n above the bottom (below the crater, above the strip)."""
    p0 = sim.get("p").copy()
    j0, j1 = int(0.15 * n), int(0.55 * n)
    out = []
    while sim.scalars()["t"] < t_end:
        sim.step(every)
        sc = sim.scalars()
        assert sc["status"] == 0, sc
        dp = np.abs(sim.get("p") - p0)[j0:j1]
        out.append((sc["t"], dp[:, :int(0.08 * n)].max(), dp[:, int(0.40 * n):int(0.55 * n)].max()))
    return np.array(out)


def stretched_layered_spec(n_core: int = 40, ext: int = 8, pml: int = 8) -> dict:
    """The three-layer target under Earth gravity on a stretched grid: n_core x n_core
    cells of 400 m, `ext` extension cells growing by 1.05 on the right, bottom and top,
    `pml` strip cells of the largest size outside the right and bottom; 3 sediment and 12
    crust rows below the surface (10 core rows below the top of the zone), mantle below; a
    dunite sphere of radius 3 cells at 12 km/s."""
    dx = 400.0
    dr = W.stretched_sizes(n_core, dx, 0, ext, 1.05, None, 0, pml)
    dz = W.stretched_sizes(n_core, dx, ext, ext, 1.05, None, pml, 0)
    zv = W.positions(dz)
    ks = pml + ext + n_core - 10
    g = W.grid(len(dr), len(dz), dx, pml_r=pml, pml_b=pml, gravity=9.81, pml_alpha=0.1)
    g["dr"], g["dz"] = dr, dz
    return {"grid": g, "materials": [W.calcite(), W.granite(), W.dunite()],
            "layers": [dict(mat=0, zlo=zv[ks - 3], zhi=zv[ks], rho=0.0, I0=0.0, vz=0.0),
                       dict(mat=1, zlo=zv[ks - 15], zhi=zv[ks - 3], rho=0.0, I0=0.0, vz=0.0),
                       dict(mat=2, zlo=0.0, zhi=zv[ks - 15], rho=0.0, I0=0.0, vz=0.0)],
            "projectile": dict(mat=2, radius=3 * dx, zc=zv[ks] + 3 * dx, vz=-12e3, rho=0.0, I0=0.0),
            "z_surface": zv[ks]}


def dilute_slab_spec(eta: float, nr: int = 8, nz: int = 48, dx: float = 10.0) -> dict:
    """A slab of hot basalt vapour (density eta rho0, specific energy 2 E_cv, at rest) in
    vacuum: rows 20-25 of a column with an open top and no gravity."""
    bas = W.basalt()
    g = W.grid(nr, nz, dx, bc_top="outflow")
    return {"grid": g, "materials": [bas], "projectile": None,
            "layers": [dict(mat=0, zlo=20 * dx, zhi=26 * dx, rho=eta * bas["rho0"],
                            I0=2.0 * bas["Ecv"], vz=0.0)]}
