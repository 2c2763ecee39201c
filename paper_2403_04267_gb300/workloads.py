"""Seeded synthetic workloads: parameter dictionaries only.

This module is the one place that both the CUDA path and the CPU oracle take their
inputs from.  It holds no arithmetic of the method: it only states material constants,
grid sizes, projectile placement and the counter-based random draws of the batched
impact distribution.  Each builder returns a plain dictionary
    {"grid": {...}, "materials": [...], "layers": [...], "projectile": {...} | None}
with SI units throughout (m, kg/m^3, Pa, J/kg, m/s).
"""
from __future__ import annotations

import math

# --- materials -----------------------------------------------------------------------

def basalt(strength: bool = False, cohesion: float = 10e6, friction: float = 0.6,
           limit: float = 2.5e9) -> dict:
    """Basalt-like Tillotson material (the constants the impact configurations name).
    The shear modulus follows from Poisson's ratio 0.25 with bulk modulus K = A, G = 0.6 A.
    With strength: Collins-type yield, cohesion -> Y_i0, friction -> mu_i = mu_d,
    limiting strength -> Y_im = Y_dm, damaged cohesion Y_d0 = 0.01 MPa (Table 1 of the
    paper lists 0.01 MPa for every rock); tensile limit -Y_i0."""
    m = dict(eos="tillotson", rho0=2700.0, A=26.7e9, B=26.7e9, E0=487e6, a=0.5, b=1.5,
             alpha=5.0, beta=5.0, Eiv=4.72e6, Ecv=18.2e6, gamma=0.0, strength="none",
             p_t=0.0)
    if strength:
        m.update(strength="collins", Yi0=cohesion, mui=friction, Yim=limit, Yd0=0.01e6,
                 mud=friction, Ydm=limit, G=0.6 * m["A"], eps_fb=1e-4, B_dam=1e-11, p_bd=3e8,
                 p_t=-cohesion)
    return m


def iron() -> dict:
    """Iron-like Tillotson projectile, rho0 = 7800 kg/m^3 as the configuration states.
    The remaining constants are the commonly tabulated Tillotson iron set (Tillotson 1962,
    as reprinted by Melosh 1989): A = 128 GPa, B = 105 GPa, E0 = 9.5 MJ/kg, a = 0.5,
    b = 1.5, alpha = beta = 5, E_iv = 2.4 MJ/kg, E_cv = 8.67 MJ/kg.  Hydrodynamic."""
    return dict(eos="tillotson", rho0=7800.0, A=128e9, B=105e9, E0=9.5e6, a=0.5, b=1.5,
                alpha=5.0, beta=5.0, Eiv=2.4e6, Ecv=8.67e6, gamma=0.0, strength="none", p_t=0.0)


def _layer_rock(rho0: float, A: float, strength: bool, Yi0: float, mui: float, Yim: float,
                mud: float, **eos) -> dict:
    """A rock of the layered target.  Strength: Table 1 of the paper (cohesion, friction and
    limiting strength, intact and damaged; damaged cohesion 0.01 MPa).  Equation of state:
    the paper gives none for these rocks, so the Tillotson constants are synthetic stand-ins:
    the rock's density, A = B set per rock, the other constants basalt's unless given.
    Shear modulus 0.6 A (Poisson's ratio 0.25)."""
    m = dict(basalt(), rho0=rho0, A=A, B=A)
    m.update(eos)
    if strength:
        m.update(strength="collins", Yi0=Yi0, mui=mui, Yim=Yim, Yd0=0.01e6, mud=mud, Ydm=Yim,
                 G=0.6 * A, eps_fb=1e-4, B_dam=1e-11, p_bd=3e8, p_t=-Yi0)
    return m


def calcite(strength: bool = True) -> dict:
    """Sediment layer: 2710 kg/m^3, A = B = 20 GPa; Table 1: 5 MPa, 1.0 / 0.4, 0.5 GPa."""
    return _layer_rock(2710.0, 20e9, strength, 5e6, 1.0, 0.5e9, 0.4)


def granite(strength: bool = True) -> dict:
    """Crust layer: the commonly tabulated Tillotson granite (2680 kg/m^3, A = B = 18 GPa,
    E0 = 16 MJ/kg, b = 1.3, E_iv = 3.5 MJ/kg, E_cv = 18 MJ/kg); Table 1: 10 MPa,
    2.0 / 0.6, 2.5 GPa."""
    return _layer_rock(2680.0, 18e9, strength, 10e6, 2.0, 2.5e9, 0.6, E0=16e6, b=1.3, Eiv=3.5e6, Ecv=18e6)


def dunite(strength: bool = True) -> dict:
    """Mantle layer (and projectile): 3320 kg/m^3, A = B = 130 GPa; Table 1: 10 MPa,
    1.2 / 0.6, 3.5 GPa."""
    return _layer_rock(3320.0, 130e9, strength, 10e6, 1.2, 3.5e9, 0.6)


def ideal_gas(gamma: float = 1.4, rho0: float = 1.0) -> dict:
    return dict(eos="ideal_gas", rho0=rho0, gamma=gamma, A=0.0, B=0.0, E0=1.0, a=0.0, b=0.0,
                alpha=0.0, beta=0.0, Eiv=0.0, Ecv=1.0, strength="none", p_t=0.0)


# --- grid ----------------------------------------------------------------------------

def grid(nr: int, nz: int, dx: float, **kw) -> dict:
    g = dict(nr=int(nr), nz=int(nz), dx=float(dx), pml_r=0, pml_b=0, pml_R=0.01, pml_c=0.0, pml_alpha=0.0,
             gravity=0.0, cfl=0.4, dt_init=1e30, dt_max=1e30, dt_growth=1.2, dt_min=0.0,
             av_cq=1.0, av_cl=0.25, f_min=1e-6, bc_top="outflow", bc_bottom="noslip")
    g.update(kw)
    return g


def impact(nr: int, nz: int, dx: float, target: dict, projectile_mat: dict | None,
           radius_cells: float, v_imp: float, surface_row: int, pml: int, gravity: float = 0.0,
           **gkw) -> dict:
    """Half-space target with its surface at row `surface_row`; a sphere of radius
    `radius_cells` cells on the axis, tangent to the surface, moving down at `v_imp`.
    By default the PML auxiliaries relax at 0.1 c / delta (complex-frequency-shifted
    stretch): runs to tens of seconds in a strong target otherwise drift.  pml_alpha=0.0
    gives the paper's layer."""
    gkw.setdefault("pml_alpha", 0.1)
    mats = [target] if projectile_mat is None else [target, projectile_mat]
    pmat = 0 if projectile_mat is None else 1
    zs = surface_row * dx
    R = radius_cells * dx
    return {
        "grid": grid(nr, nz, dx, pml_r=pml, pml_b=pml, gravity=gravity, **gkw),
        "materials": mats,
        "layers": [dict(mat=0, zlo=0.0, zhi=zs, rho=0.0, I0=0.0, vz=0.0)],
        "projectile": dict(mat=pmat, radius=R, zc=zs + R, vz=-abs(v_imp), rho=0.0, I0=0.0),
        "z_surface": zs,
    }


def layered_impact(nr: int, nz: int, dx: float, surface_row: int, sediment_rows: int,
                   crust_rows: int, radius_cells: float, v_imp: float, pml: int,
                   gravity: float = 9.81, strength: bool = True, **gkw) -> dict:
    """The paper's three-layer target (Sect. 4): sediment (calcite) over crust (granite)
    over mantle (dunite), each in hydrostatic equilibrium under its overburden, hit
    vertically by a dunite sphere on the axis (materials 0, 1, 2; the projectile shares
    the mantle's material).  Layer boundaries lie on row boundaries."""
    gkw.setdefault("pml_alpha", 0.1)
    z_s = surface_row * dx
    z_c = (surface_row - sediment_rows) * dx
    z_m = (surface_row - sediment_rows - crust_rows) * dx
    R = radius_cells * dx
    layers = [dict(mat=0, zlo=z_c, zhi=z_s, rho=0.0, I0=0.0, vz=0.0),
              dict(mat=1, zlo=max(z_m, 0.0), zhi=z_c, rho=0.0, I0=0.0, vz=0.0)]
    if z_m > 0.0:
        layers.append(dict(mat=2, zlo=0.0, zhi=z_m, rho=0.0, I0=0.0, vz=0.0))
    return {
        "grid": grid(nr, nz, dx, pml_r=pml, pml_b=pml, gravity=gravity, **gkw),
        "materials": [calcite(strength), granite(strength), dunite(strength)],
        "layers": layers,
        "projectile": dict(mat=2, radius=R, zc=z_s + R, vz=-abs(v_imp), rho=0.0, I0=0.0),
        "z_surface": z_s,
    }


def chicxulub_like(n: int = 462) -> dict:
    """The paper's verification geometry at its 400 m resolution (Sect. 4, Tables 1-2):
    2.8 km of sediment (7 rows), 30 km of crust (75 rows), mantle below; a 14.4 km dunite
    projectile (radius 18 cells); PML 30 on the right and bottom; n x n cells with the
    surface 30 rows below the top.  The impact speed (12 km/s) is not given by the paper."""
    w = layered_impact(n, n, 400.0, n - 30, 7, 75, 18, 12e3, 30)
    w["name"] = f"chicxulub_like_{n}x{n}"
    return w


def stretched_sizes(n_core: int, dx: float, n_low: int = 0, n_high: int = 0, factor: float = 1.05,
                    max_dx: float | None = None, pad_low: int = 0, pad_high: int = 0) -> list:
    """Cell sizes along one axis, low end first: pad_low cells at the largest extension
    size, n_low cells growing toward the low end, n_core cells of dx, n_high cells growing
    toward the high end, pad_high cells at the largest size.  Extension cell k (1, 2, ...
    outward) is dx factor^k, capped at max_dx (Table 2 of the paper: factor 1.05 from
    400 m up to 1061 m)."""
    def grow(n):
        out, s = [], dx
        for _ in range(n):
            s = s * factor
            if max_dx is not None and s > max_dx:
                s = max_dx
            out.append(s)
        return out
    lo, hi = grow(n_low), grow(n_high)
    big_lo = lo[-1] if lo else dx
    big_hi = hi[-1] if hi else dx
    return [big_lo] * pad_low + lo[::-1] + [dx] * n_core + hi + [big_hi] * pad_high


def positions(sizes) -> list:
    """Vertex positions 0, s0, s0 + s1, ... summed one by one in order, as the library and
    the oracle sum them (so that a height taken from here lies exactly on a row boundary)."""
    out = [0.0]
    for v in sizes:
        out.append(out[-1] + float(v))
    return out


def stretched_impact(n_core: int, dx: float, n_ext: int, pml: int, target: dict, projectile_mat: dict | None,
                     radius_cells: float, v_imp: float, surface_from_top: int, gravity: float = 0.0,
                     factor: float = 1.05, max_dx: float | None = None, **gkw) -> dict:
    """A half-space impact on the paper's kind of grid: an n_core x n_core zone of dx cells
    at the axis, extension zones of n_ext growing cells on the right, at the bottom and at
    the top, and PML strips of `pml` cells of the largest size outside the right and
    bottom extensions.  The surface lies surface_from_top core rows below the top of the
    core zone; the projectile sits on the axis, tangent to it."""
    gkw.setdefault("pml_alpha", 0.1)
    dr = stretched_sizes(n_core, dx, 0, n_ext, factor, max_dx, 0, pml)
    dz = stretched_sizes(n_core, dx, n_ext, n_ext, factor, max_dx, pml, 0)
    zs = positions(dz)[pml + n_ext + n_core - surface_from_top]
    mats = [target] if projectile_mat is None else [target, projectile_mat]
    R = radius_cells * dx
    g = grid(len(dr), len(dz), dx, pml_r=pml, pml_b=pml, gravity=gravity, **gkw)
    g["dr"], g["dz"] = dr, dz
    return {
        "grid": g,
        "materials": mats,
        "layers": [dict(mat=0, zlo=0.0, zhi=zs, rho=0.0, I0=0.0, vz=0.0)],
        "projectile": dict(mat=0 if projectile_mat is None else 1, radius=R, zc=zs + R, vz=-abs(v_imp),
                           rho=0.0, I0=0.0),
        "z_surface": zs,
    }


def chicxulub_stretched(n_core: int = 462) -> dict:
    """The paper's verification grid (Table 2, SALEc-2D+PML): a high-resolution zone of
    n_core x n_core cells of 400 m, extension zones of 20 cells growing by 1.05 (to
    1061 m) on the right, bottom and top, PML strips of 30 cells of 1061 m outside the
    right and bottom extensions (reading: the strips lie beyond the extension zones, which
    gives the same 231 km radial extent as the 50 extension cells of the runs without
    PML).  The three-layer target of Sect. 4 with its surface 30 core rows below the top
    of the zone; a 14.4 km dunite projectile at 12 km/s (the speed is not given)."""
    dx, ext, pml = 400.0, 20, 30
    dr = stretched_sizes(n_core, dx, 0, ext, 1.05, 1061.0, 0, pml)
    dz = stretched_sizes(n_core, dx, ext, ext, 1.05, 1061.0, pml, 0)
    zv = positions(dz)
    ks = pml + ext + n_core - 30                 # the surface row boundary
    zs, z_c, z_m = zv[ks], zv[ks - 7], zv[ks - 82]
    g = grid(len(dr), len(dz), dx, pml_r=pml, pml_b=pml, gravity=9.81, pml_alpha=0.1)
    g["dr"], g["dz"] = dr, dz
    return {
        "name": f"chicxulub_stretched_{len(dr)}x{len(dz)}",
        "grid": g,
        "materials": [calcite(), granite(), dunite()],
        "layers": [dict(mat=0, zlo=z_c, zhi=zs, rho=0.0, I0=0.0, vz=0.0),
                   dict(mat=1, zlo=z_m, zhi=z_c, rho=0.0, I0=0.0, vz=0.0),
                   dict(mat=2, zlo=0.0, zhi=z_m, rho=0.0, I0=0.0, vz=0.0)],
        "projectile": dict(mat=2, radius=18 * dx, zc=zs + 18 * dx, vz=-12e3, rho=0.0, I0=0.0),
        "z_surface": zs,
    }


# --- the five configurations -------------------------------------------------------------

def plain_fp64_100() -> dict:
    """100 x 100 cells of 10 m, basalt half-space (surface at row 70), hydrodynamic,
    projectile radius 5 cells at 10 km/s, PML 16 on the right and bottom, no gravity,
    CFL 0.4; 200 steps.  The paper's own layer (stretch 1 + i d / omega, no relaxation of
    the auxiliaries): a hydrodynamic target leaves no static stress for them to integrate."""
    w = impact(100, 100, 10.0, basalt(), None, 5, 10e3, 70, 16, pml_alpha=0.0)
    w["name"] = "plain_fp64_100x100"
    w["steps"] = 200
    return w


def full_fp64_800() -> dict:
    """800 x 800 cells of 25 m, iron projectile (radius 20 cells, 15 km/s) into basalt
    with Collins strength and damage, gravity 1.62 m/s^2, PML 40; run to 20 s."""
    w = impact(800, 800, 25.0, basalt(strength=True), iron(), 20, 15e3, 560, 40, gravity=1.62)
    w["name"] = "full_fp64_800x800"
    w["t_end"] = 20.0
    return w


def large_4000() -> dict:
    """4000 x 4000 cells, the 100x100 configuration's physics (10 m cells, basalt,
    hydrodynamic, PML 16 of the paper's unrelaxed form, surface at 70 % of the height),
    projectile radius 100 cells; 2000 steps."""
    w = impact(4000, 4000, 10.0, basalt(), None, 100, 10e3, 2800, 16, pml_alpha=0.0)
    w["name"] = "large_4000x4000"
    w["steps"] = 2000
    return w


def scaled_plain(n: int, radius_cells: float = None) -> dict:
    """The 100x100 configuration's physics on an n x n grid (surface at 70 %, the paper's
    unrelaxed PML)."""
    rc = radius_cells if radius_cells is not None else max(2.0, n / 40.0)
    w = impact(n, n, 10.0, basalt(), None, rc, 10e3, int(round(0.7 * n)), 16, pml_alpha=0.0)
    w["name"] = f"plain_{n}x{n}"
    return w


# --- counter-based draws for the batched distribution (SplitMix64) -------------------------

_MASK = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) of a 64-bit counter."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def uniform01(seed: int, field: int) -> float:
    """53-bit uniform draw in [0, 1) for (seed, field)."""
    return (splitmix64((seed << 8) | field) >> 11) * (1.0 / (1 << 53))


def batched_draw(seed: int) -> dict:
    """One impact of the batched distribution: square grid U{200..800} cells, projectile
    radius U{8..32} cells, velocity U(6, 20) km/s, cohesion log-uniform on 1..100 MPa,
    friction U(0.4, 0.8), projectile basalt or iron with probability 1/2.  Cells of 25 m,
    PML 40, gravity 1.62, surface at 70 % of the height."""
    n = 200 + int(uniform01(seed, 0) * 601)
    rad = 8 + int(uniform01(seed, 1) * 25)
    v = 6e3 + 14e3 * uniform01(seed, 2)
    coh = math.exp(math.log(1e6) + (math.log(100e6) - math.log(1e6)) * uniform01(seed, 3))
    fr = 0.4 + 0.4 * uniform01(seed, 4)
    dense = uniform01(seed, 5) < 0.5
    return dict(seed=seed, n=n, radius_cells=rad, v_imp=v, cohesion=coh, friction=fr,
                projectile="iron" if dense else "basalt")


def batched_run(draw: dict, n_override: int | None = None) -> dict:
    n = n_override or draw["n"]
    tgt = basalt(strength=True, cohesion=draw["cohesion"], friction=draw["friction"])
    proj = iron() if draw["projectile"] == "iron" else basalt()
    # dt_min: a healthy run of this family never steps below ~1e-4 s (25 m cells, speeds
    # below 40 km/s); 1e-6 s flags a failed run so that a batch stops it
    w = impact(n, n, 25.0, tgt, proj, draw["radius_cells"], draw["v_imp"], int(round(0.7 * n)),
               40, gravity=1.62, dt_min=1e-6)
    w["name"] = f"batched_seed{draw['seed']}"
    w["t_end"] = 20.0
    return w


# --- surrogate network initial parameters -------------------------------------------------

def mlp_init(seed: int, dims=(5, 256, 256, 256, 256, 66), gain: float = 1.0):
    """Flat parameter vector (per layer W row-major, then b), weights and biases uniform on
    +-gain/sqrt(n_in), from a seeded generator."""
    import numpy as np
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(dims) - 1):
        ni, no = dims[l], dims[l + 1]
        s = gain / math.sqrt(ni)
        parts.append(rng.uniform(-s, s, no * ni))
        parts.append(rng.uniform(-s, s, no))
    return np.concatenate(parts)
