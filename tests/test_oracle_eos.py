"""Pins of the oracle's equations of state (Tillotson 1962; ideal gas) against limits,
continuity and derivative identities that any correct implementation must satisfy."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_04267_gb300 import workloads as W

BAS = W.basalt()
IRON = W.iron()


@pytest.mark.parametrize("m", [BAS, IRON])
def test_reference_state_has_zero_pressure_and_bulk_sound_speed(m):
    p, c2 = O.eos(m, m["rho0"], 0.0)
    assert p == 0.0
    # bulk modulus at the reference state is A: c^2 = A / rho0
    assert math.isclose(c2, m["A"] / m["rho0"], rel_tol=1e-14)


@pytest.mark.parametrize("m", [BAS, IRON])
def test_cold_compression_curve_is_quadratic_in_mu(m):
    # p(rho0 (1 + mu), 0) is A mu + B mu^2: first derivative A at mu = 0, second 2B
    h = 1e-3
    ps = [O.eos(m, m["rho0"] * (1 + k * h), 0.0)[0] for k in (0, 1, 2, 3)]
    d1 = (-3 * ps[0] + 4 * ps[1] - ps[2]) / (2 * h)
    d2 = (ps[1] - 2 * ps[2] + ps[3]) / h ** 2
    assert math.isclose(d1, m["A"], rel_tol=1e-5)
    assert math.isclose(d2, 2 * m["B"], rel_tol=1e-5)


@pytest.mark.parametrize("m", [BAS, IRON])
def test_grueneisen_limits(m):
    rho0 = m["rho0"]
    # low energy at rho0: (1/rho) dp/dI -> a + b ; at I = E0: a + b/2 ; very hot: -> a
    for I, gam in ((1.0, m["a"] + m["b"]), (m["E0"], m["a"] + m["b"] / 2)):
        p, _ = O.eos(m, rho0, I)
        assert math.isclose(p / (rho0 * I), gam, rel_tol=1e-6)
    p, _ = O.eos(m, rho0, 1e6 * m["E0"])
    assert math.isclose(p / (rho0 * 1e6 * m["E0"]), m["a"], rel_tol=1e-5)


@pytest.mark.parametrize("m", [BAS, IRON])
def test_expanded_branch_tends_to_ideal_gas(m):
    # rho -> 0 at I >= E_cv: the exponentials vanish and p -> a rho I
    rho, I = 1e-3 * m["rho0"], 2 * m["Ecv"]
    p, _ = O.eos(m, rho, I)
    assert math.isclose(p, m["a"] * rho * I, rel_tol=1e-10)


@pytest.mark.parametrize("m", [BAS, IRON])
def test_continuity_at_rho0_and_at_blend_ends(m):
    eps = 1e-9
    for I in (m["Ecv"] * 1.5, m["Ecv"] * 3):
        pa, _ = O.eos(m, m["rho0"] * (1 + eps), I)
        pb, _ = O.eos(m, m["rho0"] * (1 - eps), I)
        assert abs(pa - pb) <= 1e-6 * abs(pa)
    for rho in (0.9 * m["rho0"], 0.5 * m["rho0"]):
        for Ie in (m["Eiv"], m["Ecv"]):
            pa, _ = O.eos(m, rho, Ie * (1 + 1e-10))
            pb, _ = O.eos(m, rho, Ie * (1 - 1e-10))
            assert abs(pa - pb) <= 1e-6 * max(abs(pa), m["A"] * 1e-6)


def _fd_c2(m, rho, I):
    hr, hI = 1e-6 * rho, 1e-6 * max(I, 1e3)
    pr = (O.eos(m, rho + hr, I)[0] - O.eos(m, rho - hr, I)[0]) / (2 * hr)
    pI = (O.eos(m, rho, I + hI)[0] - O.eos(m, rho, I - hI)[0]) / (2 * hI)
    p = O.eos(m, rho, I)[0]
    return pr + p / rho ** 2 * pI


@pytest.mark.parametrize("m", [BAS, IRON])
@pytest.mark.parametrize("eta,Ifac", [(1.3, 0.5), (1.05, 3.0), (0.9, 0.3), (0.95, 2.0), (0.8, 5.0), (0.6, 1.2)])
def test_sound_speed_matches_central_differences(m, eta, Ifac):
    rho = eta * m["rho0"]
    I = Ifac * m["Ecv"] if Ifac > 1 else Ifac * m["Eiv"] * 2
    _, c2 = O.eos(m, rho, I)
    ref = _fd_c2(m, rho, I)
    floor = 0.01 * m["A"] / m["rho0"]
    assert math.isclose(c2, max(ref, floor), rel_tol=1e-6)


def test_ideal_gas_textbook():
    g = W.ideal_gas(1.4)
    p, c2 = O.eos(g, 2.0, 3.0)
    assert math.isclose(p, 0.4 * 2.0 * 3.0, rel_tol=1e-15)
    assert math.isclose(c2, 1.4 * p / 2.0, rel_tol=1e-15)


def _branch_c2(m, rho, I, branch):
    """c^2 of one Tillotson branch at (rho, I): the same material with the blend moved out
    of the way (the branch formulas do not involve E_iv, E_cv), each branch pinned above by
    central differences."""
    mm = dict(m)
    if branch == "compressed":
        mm.update(Eiv=10.0 * I, Ecv=20.0 * I)     # I <= E_iv: compressed formula
    else:
        mm.update(Eiv=0.25 * I, Ecv=0.5 * I)      # I >= E_cv: expanded formula
    return O.eos(mm, rho, I)[1]


@pytest.mark.parametrize("m", [BAS, IRON])
@pytest.mark.parametrize("eta", [0.9, 0.5, 1e-2, 1e-4])
def test_blend_sound_speed_is_blend_of_branch_sound_speeds(m, eta):
    """Reading of the hybrid region: c^2 = ((I - E_iv) c_e^2 + (E_cv - I) c_c^2) / (E_cv - E_iv),
    floored like everywhere else; continuous at both blend ends, and bounded by the branch
    values even far below rho0, where the derivative of the blended pressure is not (for
    iron, A != B, it reaches c ~ 1e5 m/s at rho ~ 1e-4 rho0)."""
    rho = eta * m["rho0"]
    floor = 0.01 * m["A"] / m["rho0"]
    for f in (0.1, 0.5, 0.9, 1 - 1e-6):
        I = m["Eiv"] + f * (m["Ecv"] - m["Eiv"])
        ce2, cc2 = _branch_c2(m, rho, I, "expanded"), _branch_c2(m, rho, I, "compressed")
        _, c2 = O.eos(m, rho, I)
        raw_e = ce2 if ce2 > floor else None
        raw_c = cc2 if cc2 > floor else None
        if raw_e is not None and raw_c is not None:
            assert math.isclose(c2, max(f * ce2 + (1 - f) * cc2, floor), rel_tol=1e-9)
        assert c2 <= max(ce2, cc2, floor) * (1 + 1e-12)
    for Ie in (m["Eiv"], m["Ecv"]):
        ca = O.eos(m, rho, Ie * (1 + 1e-10))[1]
        cb = O.eos(m, rho, Ie * (1 - 1e-10))[1]
        assert abs(ca - cb) <= 1e-6 * max(ca, cb)


@pytest.mark.parametrize("m", [BAS, IRON])
def test_density_floor(m):
    """Reading: the Tillotson form is evaluated at no less than rho_f = 1e-12 rho0, where it
    is in its dilute limit: c^2 -> a (1 + a) I (pinned above) no longer depends on rho, and
    p -> a rho I is proportional to it, so below rho_f the pressure at rho_f is scaled back
    by rho / rho_f.  Far below the floor the hot state's pressure is the closed form a rho I
    (a pressure left at its rho_f value would be 1e8 times that at 1e-20 rho0 and would
    accelerate a near-empty cell without bound); the cold state keeps its sign (tension,
    clipped by the caller); an empty cell has none."""
    I = 2 * m["Ecv"]
    lo = O.eos(m, 1e-12 * m["rho0"], I)
    assert math.isclose(lo[1], m["a"] * (1 + m["a"]) * I, rel_tol=1e-9)
    for eta in (1e-13, 1e-16, 1e-20):
        rho = eta * m["rho0"]
        p, c2 = O.eos(m, rho, I)
        assert c2 == lo[1]
        assert math.isclose(p, m["a"] * rho * I, rel_tol=1e-12)
    assert O.eos(m, 0.0, I) == (0.0, lo[1])
    pc_lo, _ = O.eos(m, 1e-12 * m["rho0"], 0.5 * m["Eiv"])
    pc, _ = O.eos(m, 1e-16 * m["rho0"], 0.5 * m["Eiv"])
    assert pc_lo < 0.0 and math.isclose(pc, pc_lo * 1e-4, rel_tol=1e-12)