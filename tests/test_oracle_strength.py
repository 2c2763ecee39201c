"""Pins of the oracle's Collins yield surface and elasto-plastic stress update."""
import math

import numpy as np

from oracle import oracle as O
from paper_2403_04267_gb300 import workloads as W

M = W.basalt(strength=True)


def test_yield_limits():
    assert math.isclose(O.yield_strength(M, 0.0, 0.0), M["Yi0"], rel_tol=1e-15)
    assert math.isclose(O.yield_strength(M, 1e15, 0.0), M["Yim"], rel_tol=1e-4)
    # negative pressure is treated as zero
    assert O.yield_strength(M, -1e9, 0.0) == O.yield_strength(M, 0.0, 0.0)
    for p in (0.0, 1e8, 1e9, 1e10):
        Yd = min(M["Yd0"] + M["mud"] * p, M["Ydm"])
        assert math.isclose(O.yield_strength(M, p, 1.0), Yd, rel_tol=1e-14)
    # small-p slope of the intact surface is the friction coefficient
    h = 1e3
    s = (O.yield_strength(M, h, 0.0) - M["Yi0"]) / h
    assert math.isclose(s, M["mui"], rel_tol=1e-5)
    # linear in D between the two surfaces
    p = 5e8
    Yi, Yd = O.yield_strength(M, p, 0.0), O.yield_strength(M, p, 1.0)
    assert math.isclose(O.yield_strength(M, p, 0.3), 0.7 * Yi + 0.3 * Yd, rel_tol=1e-14)


def test_elastic_slope_is_2G():
    G, e, dt = M["G"], 1e-3, 1e-6
    sv = O.stress_update([0, 0, 0, 0], [0, 0, 0, e, 0], G, 1e12, 0.0, dt)
    assert math.isclose(sv[2], 2 * G * e * dt, rel_tol=1e-14)
    # uniaxial-strain deviator: s_rr = 2G (2/3) e dt, s_zz = s_tt = -2G (1/3) e dt
    sv = O.stress_update([0, 0, 0, 0], [e, 0, 0, 0, 0], G, 1e12, 0.0, dt)
    assert math.isclose(sv[0], 2 * G * (2 / 3) * e * dt, rel_tol=1e-14)
    assert math.isclose(sv[1], -2 * G * (1 / 3) * e * dt, rel_tol=1e-14)


def test_pure_shear_yield_plateau_plastic_strain_and_damage():
    G, e, dt, Y = M["G"], 1e-2, 1e-6, 1e7
    eps_f = 1e-3
    sv = np.zeros(4)
    steps_elastic = int(Y / (2 * G * e * dt))
    n = steps_elastic + 2000
    D_hist = []
    for _ in range(n):
        sv = O.stress_update(sv, [0, 0, 0, e, 0], G, Y, 1.0 / eps_f, dt)
        D_hist.append(sv[3])
    # plateau: sqrt(J2) = |s_rz| = Y
    assert math.isclose(abs(sv[2]), Y, rel_tol=1e-12)
    # von Mises equivalent plastic strain of shear e_rz: (2/sqrt(3)) e dt per plastic step
    plastic_steps = n - steps_elastic - 1
    expected_D = min(1.0, plastic_steps * (2 / math.sqrt(3)) * e * dt / eps_f)
    assert abs(sv[3] - expected_D) <= 2 * (2 / math.sqrt(3)) * e * dt / eps_f + 1e-12
    assert max(D_hist) <= 1.0


def test_rotation_is_objective():
    # pure spin: s(t) = R s0 R^T with R = exp(W t), W = [[0, w], [-w, 0]]
    w, dt, n = 1.0, 1e-4, 5000
    s0 = np.array([3.0, -1.0, 0.5])   # s_rr, s_zz, s_rz
    sv = np.array([s0[0], s0[1], s0[2], 0.0])
    for _ in range(n):
        sv = O.stress_update(sv, [0, 0, 0, 0, w], 1.0, 1e12, 0.0, dt)
    t = n * dt
    R = np.array([[math.cos(w * t), math.sin(w * t)], [-math.sin(w * t), math.cos(w * t)]])
    S0 = np.array([[s0[0], s0[2]], [s0[2], s0[1]]])
    S = R @ S0 @ R.T
    assert np.allclose([sv[0], sv[1], sv[2]], [S[0, 0], S[1, 1], S[0, 1]], atol=5e-3)
    # J2 preserved (up to the explicit scheme's O(dt) drift)
    J2 = lambda a, b, c: 0.5 * (a * a + b * b + (a + b) ** 2) + c * c
    assert math.isclose(J2(sv[0], sv[1], sv[2]), J2(*s0), rel_tol=1e-3)


def test_no_strength_zeroes_the_deviator():
    sv = O.stress_update([1.0, 2.0, 3.0, 0.4], [1, 1, 1, 1, 1], 0.0, 1e7, 1.0, 1e-3)
    assert list(sv) == [0.0, 0.0, 0.0, 0.4]


def test_thermal_softening_factor():
    """Collins et al. (2004) soften the yield strength by tanh(xi (T_m/T - 1)), xi = 1.2,
    to zero at melting.  Reading: T_m/T = E_iv/I (no temperature in the state).  At
    I = E_iv/2 the factor is tanh(1.2); it vanishes continuously at E_iv and stays zero above;
    at I = 0 the strength is untouched."""
    from paper_2403_04267_gb300 import workloads as W
    m = W.basalt(strength=True)
    for p, D in ((0.0, 0.0), (2e8, 0.3), (5e9, 1.0)):
        Y0 = O.yield_strength(m, p, D)
        assert O.yield_strength(m, p, D, 0.0) == Y0
        assert math.isclose(O.yield_strength(m, p, D, 0.5 * m["Eiv"]), Y0 * math.tanh(1.2), rel_tol=1e-14)
        assert O.yield_strength(m, p, D, m["Eiv"]) == 0.0
        assert O.yield_strength(m, p, D, 10 * m["Eiv"]) == 0.0
        assert O.yield_strength(m, p, D, m["Eiv"] * (1 - 1e-9)) < 1e-8 * Y0
        assert O.yield_strength(m, p, D, 1e-6 * m["Eiv"]) == Y0 * math.tanh(1.2 * (1e6 - 1.0))


def test_expansion_weakening_of_strength_and_tension():
    """Reading: rock expanded below half its reference density is fragmented (no shear
    strength, no tension); between rho0/2 and rho0 both scale with w = 2 rho/rho0 - 1."""
    from paper_2403_04267_gb300 import workloads as W
    coh = 5e6
    m = W.basalt(strength=True, cohesion=coh)
    rho0 = m["rho0"]
    for p, D in ((0.0, 0.0), (1e8, 0.5)):
        Y0 = O.yield_strength(m, p, D)
        assert O.yield_strength(m, p, D, 0.0, 1.2 * rho0) == Y0
        assert math.isclose(O.yield_strength(m, p, D, 0.0, 0.75 * rho0), 0.5 * Y0, rel_tol=1e-14)
        assert O.yield_strength(m, p, D, 0.0, 0.5 * rho0) == 0.0
        assert O.yield_strength(m, p, D, 0.0, 1e-7 * rho0) == 0.0
    # tension cut-off in a cell: (1 - D) p_t w with p_t = -cohesion
    spec = {"grid": W.grid(4, 4, 10.0), "materials": [m],
            "layers": [dict(mat=0, zlo=0.0, zhi=40.0, rho=0.0, I0=0.0, vz=0.0)], "projectile": None}
    s = O.OracleSim(spec)
    rho = s.get("rho0")
    rho[0, :] = 0.75 * rho0      # Tillotson p = A mu + B mu^2 = -5 GPa before the cut-off
    rho[1, :] = 0.4 * rho0
    rho[2, :] = 1.0 * rho0
    s.set("rho0", rho)
    p = s.get("p")
    assert np.allclose(p[0], -0.5 * coh, rtol=1e-14)
    assert np.all(p[1] == 0.0)
    assert np.all(p[2] == 0.0)
