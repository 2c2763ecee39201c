"""Helpers of the GPU parity tests.

Parity is measured in the relative max-norm ||a - b||_inf / ||b||_inf (b = oracle) on:
 - the conserved variables of every cell and vertex: material volume V f_m, material
   mass V f_m rho_m, energy M I, stress and damage content V Phi (s, D), vertex momentum
   m_v v;
 - the intensive fields (rho_m, I, s, D, peak over-pressure, v) where material is present
   (cells with Phi >= 1e-3, vertices touching such a cell).
In cells at the edge of the clean-up threshold (Phi ~ f_min = 1e-6) the intensive fields
are ratios of round-off-sized contents: the oracle run against itself with inputs
perturbed by 1e-15 already differs there by ~1e-7 after 200 steps, while the two
quantities above stay near 1e-10.  The unmasked intensive norms are reported too.
PML auxiliaries are compared against a floor equal to their size for a 1e-4 relative
fluctuation of the strip (they are round-off noise while no wave has reached the strip).
"""
from __future__ import annotations

import math

import numpy as np

PML_B = ["phi1_b", "phi3_b", "psi2_b", "phi2r_b", "phi2z_b", "psi1r_b", "psi1z_b"]
PML_R = ["phi1_r", "phi3_r", "psi2_r", "phi2r_r", "phi2z_r", "psi1r_r", "psi1z_r"]
PRESENT = 1e-3


def rel_err(a, b, floor=0.0):
    den = max(float(np.abs(b).max()) if b.size else 0.0, floor)
    if den == 0.0:
        return float(np.abs(a).max()) if a.size else 0.0
    return float(np.abs(a - b).max()) / den


def _scales(spec):
    mats = spec["materials"]
    g = spec["grid"]
    dx = g["dx"]
    rho0 = max(m["rho0"] for m in mats)
    A = max([m.get("A", 0.0) for m in mats] + [1e-300])
    c2 = max([m["A"] / m["rho0"] for m in mats if m.get("eos", "tillotson") == "tillotson"] + [1e-300])
    c = math.sqrt(c2)
    Mmax = rho0 * (g["nr"] - 0.5) * dx ** 3
    width = max(g.get("pml_r", 0), g.get("pml_b", 0), 1)
    dmax = 1.5 * c / (width * dx) * math.log(1.0 / g.get("pml_R", 0.01))
    return dict(c=c, c2=c2, A=A, rho0=rho0, M=Mmax, dmax=dmax)


def _vol(spec):
    g = spec["grid"]
    return (np.arange(g["nr"]) + 0.5) * g["dx"] ** 3


def _vertex_sum(cellf):
    nz, nr = cellf.shape
    out = np.zeros((nz + 1, nr + 1))
    for a, b in ((0, 0), (0, 1), (1, 0), (1, 1)):
        out[a:a + nz, b:b + nr] += 0.25 * cellf
    return out


def parity(gpu, ref, spec, fields=None):
    """Per-quantity relative max-norm differences; the gated ones, then 'info:' extras."""
    nm = len(spec["materials"])
    strength = any(m.get("strength", "none") != "none" for m in spec["materials"])
    V = _vol(spec)[None, :]
    S = _scales(spec)
    # velocity and energy scales also from the reference state itself (ideal-gas runs have
    # no Tillotson sound speed)
    vref = max(float(np.abs(ref.get("vr")).max()), float(np.abs(ref.get("vz")).max()))
    S["c"] = max(S["c"], vref)
    S["c2"] = max(S["c2"], float(np.abs(ref.get("I")).max()), S["c"] ** 2)
    out = {}
    G = {}
    R = {}

    def get(name):
        if name not in G:
            G[name] = gpu.get(name)
            R[name] = ref.get(name)
        return G[name], R[name]

    phi_r = sum(get(f"f{m}")[1] for m in range(nm))
    M_g = sum(get(f"f{m}")[0] * get(f"rho{m}")[0] for m in range(nm)) * V
    M_r = sum(get(f"f{m}")[1] * get(f"rho{m}")[1] for m in range(nm)) * V
    cell_mask = phi_r >= PRESENT
    vert_mask = _vertex_sum(cell_mask.astype(float)) > 0
    for m in range(nm):
        fg, fr = get(f"f{m}")
        rg, rr = get(f"rho{m}")
        out[f"volume{m}"] = rel_err(fg * V, fr * V)
        out[f"mass{m}"] = rel_err(fg * rg * V, fr * rr * V)
        present = fr >= PRESENT
        out[f"rho{m}|present"] = rel_err(rg[present], rr[present], S["rho0"]) if present.any() else 0.0
        out[f"info:rho{m}"] = rel_err(rg, rr)
    Ig, Ir = get("I")
    out["energy"] = rel_err(M_g * Ig, M_r * Ir)
    out["I|present"] = rel_err(Ig[cell_mask], Ir[cell_mask], S["c2"] * 1e-4) if cell_mask.any() else 0.0
    out["info:I"] = rel_err(Ig, Ir)
    pg, pr = get("pmax")
    out["pmax|present"] = rel_err(pg[cell_mask], pr[cell_mask], S["A"] * 1e-4) if cell_mask.any() else 0.0
    if strength:
        for k in ("srr", "szz", "srz", "D"):
            a, b = get(k)
            fl = 1.0 if k == "D" else S["A"] * 1e-4
            out[f"{k}*volume"] = rel_err(a * phi_r * V, b * phi_r * V, fl * 1e-4 * float(V.max()))
            out[f"{k}|present"] = rel_err(a[cell_mask], b[cell_mask], fl) if cell_mask.any() else 0.0
    mv_r = _vertex_sum(M_r)
    for k in ("vr", "vz"):
        a, b = get(k)
        out[f"momentum_{k[1]}"] = rel_err(mv_r * a, mv_r * b, S["c"] * 1e-4 * S["M"])
        out[f"{k}|present"] = rel_err(a[vert_mask], b[vert_mask], S["c"] * 1e-4) if vert_mask.any() else 0.0
        out[f"info:{k}"] = rel_err(a, b)
    aux = []
    if spec["grid"].get("pml_b", 0) > 0:
        aux += PML_B
    if spec["grid"].get("pml_r", 0) > 0:
        aux += PML_R
    for k in aux:
        a, b = get(k)
        if k.startswith("phi1"):
            fl = S["dmax"] * S["M"] * 1e-4
        elif k.startswith(("phi3", "psi2")):
            fl = S["dmax"] * S["M"] * S["c2"] * 1e-4
        else:
            fl = S["dmax"] * S["M"] * S["c"] * 1e-4
        out[k] = rel_err(a, b, fl)
    return out


def gated(report):
    return {k: v for k, v in report.items() if not k.startswith("info:")}


# the largest bound a sensitivity-relaxed comparison may apply: beyond it the problem's
# own round-off response would hide a real difference
RELAXED_CAP = 1e-6


def assert_parity(g, r, spec, tol=1e-9, sensitivity=None, status_zero=False):
    """Every gated quantity of `parity` within tol, the step count and status equal, t and
    dt within tol.  With `sensitivity` (the oracle against itself after a 1e-15 input
    perturbation, same steps) a quantity may instead be within 100 times the problem's own
    response to that perturbation, never more than RELAXED_CAP.  The bound applied to each
    quantity is printed beside its difference."""
    rep = parity(g, r, spec)
    errs = gated(rep)

    def bound_of(k):
        if sensitivity is None:
            return tol
        b = max(tol, 100.0 * sensitivity.get(k, 0.0))
        assert b <= RELAXED_CAP, f"{k}: the relaxed bound {b:.1e} exceeds {RELAXED_CAP:.0e}"
        return b

    print({k: f"{v:.1e}" for k, v in rep.items() if k.startswith("info:")})
    print({k: f"{e:.1e} <= {bound_of(k):.1e}" for k, e in errs.items()})
    for k, e in errs.items():
        bound = bound_of(k)
        assert e <= bound, f"{k}: {e:.3e} > {bound:.1e} (all: { {kk: f'{v:.1e}' for kk, v in rep.items()} })"
    sg, so = g.scalars(), r.scalars()
    assert sg["nstep"] == so["nstep"]
    assert sg["status"] == so["status"]
    if status_zero:
        assert so["status"] == 0
    for k in ("t", "dt"):
        bound = bound_of(k)
        print(f"{k}: {abs(sg[k] - so[k]) / max(so[k], 1e-300):.1e} <= {bound:.1e}")
        assert abs(sg[k] - so[k]) <= bound * max(so[k], 1e-300), k
    return errs


def sensitivity(r, r2, spec):
    """The oracle's own response (run r2, perturbed at set-up, against r): the gated
    quantities and the relative t, dt differences."""
    sens = gated(parity(r2, r, spec))
    s2, s1 = r2.scalars(), r.scalars()
    sens.update({k: abs(s2[k] - s1[k]) / s1[k] for k in ("t", "dt")})
    return sens


def perturbed(sim, rel=1e-15, seed=0):
    """Multiply the density, energy and velocity fields of an oracle run by 1 + rel * noise
    (an input perturbation at round-off level, used to measure the problem's own
    sensitivity)."""
    rng = np.random.default_rng(seed)
    names = [n for n in ("rho0", "rho1", "rho2", "I", "vr", "vz")]
    for n in names:
        try:
            x = sim.get(n)
        except KeyError:
            continue
        sim.set(n, x * (1 + rel * rng.standard_normal(x.shape)))
    return sim


def worst(errs):
    k = max(errs, key=errs.get)
    return k, errs[k]
