"""The fused step form: one tile kernel per cycle that stages a tile and a 3-cell halo in
shared memory and runs every phase on it, writing the rewritten fields to a second copy.

FP64 fused steps are held to the oracle at the FP64 bar (1e-9 relative max-norm of every
gated quantity, gpu_util.py), as the phase kernels are: the plain 100 x 100 impact on the
paper's PML, the full method on 800 x 800, ragged random grids, the Sod and
Rankine-Hugoniot columns, the plane and 2-D PML pulses, and stretched and layered grids.
Against the phase kernels (same arithmetic per cell and vertex, compiled in another
kernel, so a multiply-add may contract differently) a fused run agrees to rounding: 1e-13
after one step and 1e-12 after 30 in FP64; 1e-6 and 1e-3 in the mixed form, whose single
rounding differences the impact amplifies.  Exact properties: rest states
stay bitwise at rest; results do not depend on how the steps are grouped into calls (CUDA
graph chunks, odd step counts that leave the current fields in the second copy), on
checkpoints taken at either copy, or on a batch stepping a run in between."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import gpu_util as U
import oracle_cases as OC
from oracle import oracle as O
from paper_2403_04267_gb300 import salec, workloads as W

TOL = 1e-9
FIELDS = ("f0", "f1", "rho0", "rho1", "I", "srr", "szz", "srz", "D", "pmax", "vr", "vz")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    salec.load()


def _fused(spec, precision="fp64"):
    g = salec.Sim(spec, precision=precision)
    g.step_form = "fused"
    assert g.step_form == "fused" and g.launches_per_step() == 3
    return g


def _fields(sim, spec):
    nm = len(spec["materials"])
    names = [f for f in FIELDS if not f[-1].isdigit() or int(f[-1]) < nm]
    if not any(m.get("strength", "none") != "none" for m in spec["materials"]):
        names = [f for f in names if f not in ("srr", "szz", "srz", "D")]
    aux = (U.PML_B if spec["grid"].get("pml_b", 0) else []) + (U.PML_R if spec["grid"].get("pml_r", 0) else [])
    return names + aux


def _assert_close(a, b, spec, tol):
    worst = 0.0
    for name in _fields(a, spec):
        x, y = a.get(name), b.get(name)
        den = float(np.abs(y).max())
        e = float(np.abs(x - y).max()) / den if den > 0 else float(np.abs(x).max())
        worst = max(worst, e)
        assert e <= tol, f"{name}: {e:.3e} > {tol:.0e}"
    return worst


def _assert_equal(a, b, spec):
    for name in _fields(a, spec):
        assert np.array_equal(a.get(name), b.get(name)), name
    sa, sb = a.scalars(), b.scalars()
    assert sa["t"] == sb["t"] and sa["dt"] == sb["dt"] and sa["nstep"] == sb["nstep"]


def test_fused_fp64_plain_100x100_against_oracle():
    spec = W.plain_fp64_100()
    g, r = _fused(spec), O.OracleSim(spec)
    g.step(1)
    r.step(1)
    U.assert_parity(g, r, spec)
    g.step(199)
    r.step(199)
    U.assert_parity(g, r, spec)


def test_fused_fp64_full_method_800x800_against_oracle():
    spec = W.full_fp64_800()
    g, r = _fused(spec), O.OracleSim(spec)
    g.step(20)
    r.step(20)
    U.assert_parity(g, r, spec)


@pytest.mark.parametrize("seed,nr,nz,nmat,strength", [
    (1, 3, 3, 1, False), (2, 17, 13, 2, True), (3, 33, 9, 2, True), (4, 9, 41, 1, True),
    (5, 40, 40, 2, False), (6, 65, 31, 2, True), (7, 70, 45, 1, False)])
def test_fused_fp64_random_ragged_grids(seed, nr, nz, nmat, strength):
    """Tiles cut the grid at every position of a ragged edge; the yielding cells' bar is
    1e-9 or 100 x the oracle's own response to a 1e-15 perturbation (at most 1e-6)."""
    spec = OC.random_impact_spec(seed, nr, nz, nmat=nmat, strength=strength, pml=max(1, min(nr, nz) // 3))
    g, r = _fused(spec), O.OracleSim(spec)
    g.step(1)
    r.step(1)
    U.assert_parity(g, r, spec)
    r2 = U.perturbed(O.OracleSim(spec))
    r2.step(1)
    g.step(59)
    r.step(59)
    r2.step(59)
    U.assert_parity(g, r, spec, sensitivity=U.sensitivity(r, r2, spec))


def test_fused_fp64_sod_rh_and_pml_waves():
    for spec, n in ((OC.sod_spec(200), 150), (OC.rh_spec(200), 200)):
        g, r = _fused(spec), O.OracleSim(spec)
        g.step(n)
        r.step(n)
        U.assert_parity(g, r, spec)
    # a 2-D pulse inside both strips with non-zero auxiliaries everywhere
    base = OC.plane_wave_spec(60, 12)
    spec = dict(base, grid=dict(base["grid"], nr=48, pml_r=12, bc_bottom="freeslip"))
    g, r = _fused(spec), O.OracleSim(spec)
    rng = np.random.default_rng(7)
    rho = 2700.0 * (1 + 1e-4 * rng.standard_normal((60, 48)))
    vr = 0.1 * rng.standard_normal((61, 49))
    vz = 0.1 * rng.standard_normal((61, 49))
    aux = {n: 1e3 * rng.standard_normal((60, 48) if n[:4] in ("phi1", "phi3", "psi2") else (61, 49))
           for n in U.PML_B + U.PML_R}
    for n, a in aux.items():
        cell = a.shape == (60, 48)
        if n.endswith("_b"):
            a[12:, :] = 0.0
        elif cell:
            a[:, :36] = 0.0
        else:
            a[:, :37] = 0.0
    for s in (g, r):
        s.set("rho0", rho)
        s.set("vr", vr)
        s.set("vz", vz)
        for n, a in aux.items():
            s.set(n, a)
    g.step(80)
    r.step(80)
    U.assert_parity(g, r, spec)


def test_fused_fp64_stretched_and_layered_grids():
    """Non-uniform cells (Table 2's growing extension zones) and the three-layer target under
    gravity: the per-column and per-row geometry of the non-uniform form."""
    for spec, n in ((W.stretched_impact(40, 10.0, 8, 8, W.basalt(), None, 3, 10e3, 12), 60),
                    (OC.stretched_layered_spec(), 40),
                    (W.layered_impact(60, 70, 400.0, 55, 4, 20, 4, 12e3, 8), 30)):
        g, r = _fused(spec), O.OracleSim(spec)
        g.step(n)
        r.step(n)
        r2 = U.perturbed(O.OracleSim(spec))
        r2.step(n)
        U.assert_parity(g, r, spec, sensitivity=U.sensitivity(r, r2, spec))


@pytest.mark.parametrize("precision,tol1,tol30", [("fp64", 1e-13, 1e-12), ("fp32mix", 1e-6, 1e-3)])
def test_fused_matches_phase_kernels(precision, tol1, tol30):
    """After one step (a wrong halo or tile edge would show at order 1 there) and after 30.
    In FP32 a multiply-add contracted differently rounds one field value by an ulp (6e-8)
    now and then, and the impact amplifies such differences by up to ~1e5 in 30 steps."""
    for spec in (W.impact(90, 70, 10.0, W.basalt(strength=True), W.iron(), 6, 12e3, 45, 10, gravity=1.62),
                 W.scaled_plain(130, radius_cells=6)):
        a = _fused(spec, precision)
        b = salec.Sim(spec, precision=precision)
        b.step_form = "phases"
        a.step(1)
        b.step(1)
        w1 = _assert_close(a, b, spec, tol1)
        a.step(29)
        b.step(29)
        w30 = _assert_close(a, b, spec, tol30)
        print(f"{precision} {spec.get('name', 'impact')}: fused vs phases {w1:.1e} after 1 step, {w30:.1e} after 30")
        sa, sb = a.scalars(), b.scalars()
        assert sa["nstep"] == sb["nstep"] == 30 and sa["status"] == sb["status"] == 0
        assert abs(sa["t"] / sb["t"] - 1) <= tol30
        # the tallies (outflow, strip damping, clean-up) agree to rounding on the scale of the
        # grid's mass (which near-empty cells cross the clean-up threshold is round-off)
        mass = b.conservation()["mass"]
        for k in ("mass_out", "mass_pml", "mass_discarded"):
            assert abs(sa[k] - sb[k]) <= tol30 * 1e-3 * mass, k


@pytest.mark.parametrize("precision", ["fp64", "fp32mix"])
@pytest.mark.parametrize("n", [200, 203])
def test_rest_tiles_copy_what_the_quiescent_path_writes(precision, n):
    """A tile found quiescent in the step before, with its eight neighbours, is copied by
    the rest-tile kernel instead of going through the tile kernel; so is one that the
    Courant-rate pass before the first step (and again after a host write) found quiescent
    with its fields in the quiescent path's form.  Against the same steps taken with the
    copy switched off (every tile then goes through the tile kernel's own quiescence test
    and path): bitwise the same fields, time and dt, the tallies to rounding, on a grid the
    tiles divide and on a ragged one."""
    spec = W.scaled_plain(n, radius_cells=5)
    a = _fused(spec, precision)
    a.step(1)
    q1, tiles = a.fused_queue()
    print(f"{precision} {n}x{n}: {q1} of {tiles} tiles through the whole cycle in the first step")
    assert 0 < q1 < tiles
    a.step(33)
    a.set("vz", a.get("vz"))       # a host write: the rate pass flags the tiles again
    a.step(1)
    assert 0 < a.fused_queue()[0] < tiles
    a.step(35)
    queued = a.fused_queue()[0]
    print(f"{precision} {n}x{n}: {queued} of {tiles} tiles through the whole cycle after 70 steps")
    assert 0 < queued < tiles
    b = _fused(spec, precision)
    b.set_rest_copy(False)
    for _ in range(70):
        b.step(1)
        assert b.fused_queue() == (tiles, tiles)
    _assert_equal(a, b, spec)
    # the tallies are sums of the CTAs' atomic additions, in the order the CTAs take their
    # tiles from the queue: equal to rounding
    sa, sb = a.scalars(), b.scalars()
    for k in ("mass_out", "mass_pml", "mass_discarded", "zmom_out"):
        assert abs(sa[k] - sb[k]) <= 1e-12 * abs(sb[k]), k


@pytest.mark.parametrize("nr,nz,pml", [(200, 200, 16), (256, 192, 0), (202, 160, 16), (230, 176, 0)])
def test_rest_copy_beside_the_tile_kernel_matches_the_rest_tile_kernel(nr, nz, pml):
    """FP64, one hydrodynamic material, nr even: the copy kernel that runs beside the tile
    kernel (bulk tensor copies of the tiles at rest, on a second stream) against the
    rest-tile kernel that runs before the tile kernel, and against no copy at all: bitwise
    the same fields, time and dt after 60 steps (a graph chunk included), the tallies to
    rounding.  The 32 x 16 tiles divide the grid in neither direction, in both (without
    absorbing strips, so the last tile column is at rest too: the grid's last vertex row and
    column fall just outside the copied vertex boxes), in z only, and in r only."""
    spec = W.impact(nr, nz, 10.0, W.basalt(), None, 4, 10e3, int(0.7 * nz), pml, pml_alpha=0.0)
    runs = {}
    for mode in (2, 1, 0):
        g = _fused(spec)
        g.set_rest_copy(mode)
        assert g.launches_per_step() == (4 if mode == 2 else 3)
        g.step(1)
        q, tiles = g.fused_queue()
        assert (0 < q < tiles) if mode else q == tiles
        g.set_kernel_timing(True)
        g.step(2)
        names = set(g.kernel_times()[0])
        g.set_kernel_timing(False)
        assert names == ({"k_rest_copy", "k_step_fused"} if mode == 2 else {"k_rest_tiles", "k_step_fused"})
        g.step(57)
        runs[mode] = g
    print(f"{nr}x{nz} pml {pml}: {runs[2].fused_queue()} queued / tiles after 60 steps")
    for mode in (1, 0):
        _assert_equal(runs[2], runs[mode], spec)
        sa, sb = runs[2].scalars(), runs[mode].scalars()
        for k in ("mass_out", "mass_pml", "mass_discarded", "zmom_out"):
            assert abs(sa[k] - sb[k]) <= 1e-12 * abs(sb[k]), k
    with pytest.raises(salec.SalecError):
        runs[2].set_rest_copy(3)


def test_rest_copy_beside_falls_back_where_the_form_does_not_allow_it():
    """Odd nr (the energy's rows would not start on 16-byte boundaries), the mixed form and
    two materials: the tiles at rest are copied by the rest-tile kernel, with the same
    results as no copy."""
    cases = [(W.impact(201, 160, 10.0, W.basalt(), None, 4, 10e3, 112, 0, pml_alpha=0.0), "fp64"),
             (W.impact(200, 160, 10.0, W.basalt(), None, 4, 10e3, 112, 0, pml_alpha=0.0), "fp32mix"),
             (W.impact(200, 160, 10.0, W.basalt(), W.iron(), 4, 10e3, 112, 0, pml_alpha=0.0), "fp64")]
    for spec, precision in cases:
        a, b = _fused(spec, precision), _fused(spec, precision)
        a.set_rest_copy(2)
        b.set_rest_copy(0)
        assert a.launches_per_step() == 3
        a.step(40)
        b.step(40)
        assert 0 < a.fused_queue()[0] < a.fused_queue()[1]
        _assert_equal(a, b, spec)


@pytest.mark.parametrize("precision", ["fp64", "fp32mix"])
def test_fused_rest_states_are_exact(precision):
    spec = OC.gas_box_spec(37, 29)
    g = _fused(spec, precision)
    rho, I = g.get("rho0"), g.get("I")
    g.step(201)
    assert np.all(g.get("vr") == 0.0) and np.all(g.get("vz") == 0.0)
    assert np.array_equal(g.get("rho0"), rho) and np.array_equal(g.get("I"), I)
    g = _fused(OC.hydrostatic_spec(40, 120), precision)
    g.step(200)
    v = np.hypot(g.get("vr"), g.get("vz")).max()
    assert v / np.sqrt(26.7e9 / 2700.0) <= (1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "fp32mix"])
def test_fused_steps_do_not_depend_on_their_grouping(precision):
    """200 steps as one call (CUDA-graph chunks), as 200 single calls, and as 105 + 95 with a
    checkpoint taken after the odd count (current fields in the second copy) and restored
    into a fresh run: bitwise the same."""
    spec = W.impact(80, 80, 10.0, W.basalt(strength=True), W.iron(), 6, 12e3, 50, 10, gravity=1.62)
    a = _fused(spec, precision)
    a.step(200)
    b = _fused(spec, precision)
    for _ in range(200):
        b.step(1)
    c = _fused(spec, precision)
    c.step(105)
    snap = c.get_state()
    c.step(95)
    d = _fused(spec, precision)
    d.set_state(snap)
    d.step(95)
    for x in (b, c, d):
        _assert_equal(a, x, spec)
    # a field read at an odd step count and written back changes nothing
    e = _fused(spec, precision)
    e.step(33)
    e.set("vz", e.get("vz"))
    e.step(167)
    _assert_equal(a, e, spec)


def test_fused_form_switches_and_batches():
    """Switching the form in the middle of a run, and a batch stepping a run that was last
    stepped fused at an odd count, continue from the current fields."""
    spec = W.impact(70, 60, 10.0, W.basalt(strength=True), W.iron(), 5, 10e3, 40, 8, gravity=1.62)
    ref = salec.Sim(spec)
    ref.step_form = "phases"
    ref.step(60)
    a = salec.Sim(spec)
    a.step_form = "phases"
    a.step(20)
    a.step_form = "fused"
    a.step(21)
    a.step_form = "phases"
    a.step(19)
    # rounding differences between the two forms' kernels grow in yielding cells (1e-13 after
    # 30 steps, a few 1e-12 after 60); continuing from the wrong copy would differ at order 1
    _assert_close(a, ref, spec, 1e-10)
    b = _fused(spec)
    b.step(21)
    batch = salec.Batch([b])
    batch.step(19)
    b.step(20)
    assert b.scalars()["nstep"] == 60
    _assert_close(b, ref, spec, 1e-10)


def test_fused_fp32mix_impact_conserves_and_stays_healthy():
    """The mixed form stepped fused on the 4000 x 4000 physics at 400 x 400: no failure,
    mass bookkeeping (grid + top outflow + strip damping + clean-up) conserved to FP32
    resolution, the same crater depth as the phase kernels within 0.1 %."""
    spec = W.scaled_plain(400, radius_cells=10)
    a = _fused(spec, "fp32mix")
    b = salec.Sim(spec, precision="fp32mix")
    b.step_form = "phases"
    m0 = a.conservation()["mass"]
    a.step(600)
    b.step(600)
    sa = a.scalars()
    assert sa["status"] == 0
    m1 = a.conservation()["mass"]
    # the strips' damping tally is the mass they added (negative: removed)
    assert abs((m1 + sa["mass_out"] + sa["mass_discarded"] - sa["mass_pml"]) / m0 - 1) < 1e-5
    ca, cb = a.crater(spec["z_surface"], 64), b.crater(spec["z_surface"], 64)
    assert abs(ca["depth"] - cb["depth"]) <= 1e-3 * abs(cb["depth"]) + 1e-3
