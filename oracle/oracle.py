"""ctypes front end of the serial FP64 CPU oracle (oracle/salec_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and bench.py's
cpu_baseline / ``--impl reference`` leg may import this module.  It shares no code with
the CUDA library and never imports the product package: it takes plain dictionaries of
parameters (the seeded workload builders produce them) and returns numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "salec_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# field codes (same meaning as the C enum in salec_oracle.c)
FIELDS = {
    "f0": 0, "f1": 1, "f2": 2, "rho0": 3, "rho1": 4, "rho2": 5, "I": 6, "srr": 7, "szz": 8,
    "srz": 9, "D": 10, "pmax": 11, "vr": 12, "vz": 13, "p": 14, "P_total": 15,
    "phi1_b": 20, "phi3_b": 21, "psi2_b": 22, "phi1_r": 23, "phi3_r": 24, "psi2_r": 25,
    "phi2r_b": 30, "phi2z_b": 31, "psi1r_b": 32, "psi1z_b": 33,
    "phi2r_r": 34, "phi2z_r": 35, "psi1r_r": 36, "psi1z_r": 37,
}
VERTEX_FIELDS = {"vr", "vz", "phi2r_b", "phi2z_b", "psi1r_b", "psi1z_b",
                 "phi2r_r", "phi2z_r", "psi1r_r", "psi1z_r"}


class Material(C.Structure):
    _fields_ = [
        ("eos", C.c_int), ("rho0", C.c_double),
        ("A", C.c_double), ("B", C.c_double), ("E0", C.c_double), ("a", C.c_double),
        ("b", C.c_double), ("alpha", C.c_double), ("beta", C.c_double), ("Eiv", C.c_double),
        ("Ecv", C.c_double), ("gamma", C.c_double),
        ("strength", C.c_int),
        ("Yi0", C.c_double), ("mui", C.c_double), ("Yim", C.c_double), ("Yd0", C.c_double),
        ("mud", C.c_double), ("Ydm", C.c_double), ("G", C.c_double),
        ("eps_fb", C.c_double), ("B_dam", C.c_double), ("p_bd", C.c_double), ("p_t", C.c_double),
    ]


class Grid(C.Structure):
    _fields_ = [
        ("nr", C.c_int), ("nz", C.c_int), ("nmat", C.c_int), ("dx", C.c_double),
        ("pml_r", C.c_int), ("pml_b", C.c_int), ("pml_R", C.c_double), ("pml_c", C.c_double), ("pml_alpha", C.c_double),
        ("gravity", C.c_double), ("cfl", C.c_double), ("dt_init", C.c_double),
        ("dt_max", C.c_double), ("dt_growth", C.c_double), ("dt_min", C.c_double),
        ("av_cq", C.c_double), ("av_cl", C.c_double), ("f_min", C.c_double),
        ("bc_top", C.c_int), ("bc_bottom", C.c_int),
    ]


_EOS = {"tillotson": 0, "ideal_gas": 1}
_STR = {"none": 0, "collins": 1}
_TOP = {"outflow": 0, "wall": 1}
_BOTTOM = {"noslip": 0, "freeslip": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off: no contraction of a*b+c)."""
    global _lib
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                                   "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
            _lib = None
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        D = C.POINTER(C.c_double)
        L.orc_create.restype = P
        L.orc_create.argtypes = [C.POINTER(Grid), C.POINTER(Material)]
        L.orc_destroy.argtypes = [P]
        L.orc_add_layer.argtypes = [P, C.c_int] + [C.c_double] * 5
        L.orc_set_spacing.argtypes = [P, D, D]
        L.orc_place_projectile.argtypes = [P, C.c_int] + [C.c_double] * 5
        L.orc_finalize.argtypes = [P]
        L.orc_step.argtypes = [P, C.c_int]
        L.orc_phase0.argtypes = [P]
        L.orc_get_field.argtypes = [P, C.c_int, D, C.c_long]
        L.orc_set_field.argtypes = [P, C.c_int, D, C.c_long]
        L.orc_scalars.argtypes = [P, D]
        L.orc_set_time.argtypes = [P, C.c_double, C.c_double]
        L.orc_conservation.argtypes = [P, D]
        L.orc_surface_heights.argtypes = [P, D]
        L.orc_eos.argtypes = [C.POINTER(Material), C.c_double, C.c_double, D, D]
        L.orc_yield.restype = C.c_double
        L.orc_yield.argtypes = [C.POINTER(Material), C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_stress_update.argtypes = [D, D, C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_pml_profile.restype = C.c_double
        L.orc_pml_profile.argtypes = [C.c_double] * 5
        _lib = L
    return _lib


def make_material(d: dict) -> Material:
    m = Material()
    for name, _ in Material._fields_:
        if name == "eos":
            m.eos = _EOS[d.get("eos", "tillotson")]
        elif name == "strength":
            m.strength = _STR[d.get("strength", "none")]
        else:
            setattr(m, name, float(d.get(name, 0.0)))
    return m


def make_grid(d: dict) -> Grid:
    g = Grid()
    for name, ctype in Grid._fields_:
        if name == "bc_top":
            g.bc_top = _TOP[d.get("bc_top", "outflow")]
        elif name == "bc_bottom":
            g.bc_bottom = _BOTTOM[d.get("bc_bottom", "noslip")]
        elif ctype is C.c_int:
            setattr(g, name, int(d[name]) if name in ("nr", "nz", "nmat") else int(d.get(name, 0)))
        else:
            setattr(g, name, float(d[name]) if name == "dx" else float(d.get(name, 0.0)))
    return g


def eos(material: dict, rho: float, I: float):
    """Unclipped pressure and squared sound speed of one material at (rho, I)."""
    p, c2 = C.c_double(), C.c_double()
    m = make_material(material)
    lib().orc_eos(C.byref(m), rho, I, C.byref(p), C.byref(c2))
    return p.value, c2.value


def yield_strength(material: dict, p: float, D: float, I: float = 0.0, rho: float | None = None) -> float:
    m = make_material(material)
    return lib().orc_yield(C.byref(m), p, D, I, material["rho0"] if rho is None else rho)


def stress_update(s4, rates5, G: float, Y: float, inv_epsf: float, dt: float):
    """One elasto-plastic update of (s_rr, s_zz, s_rz, D) with rates (e_rr, e_zz, e_tt, e_rz, omega)."""
    sv = np.ascontiguousarray(s4, dtype=np.float64).copy()
    rt = np.ascontiguousarray(rates5, dtype=np.float64)
    lib().orc_stress_update(sv.ctypes.data_as(C.POINTER(C.c_double)), rt.ctypes.data_as(C.POINTER(C.c_double)),
                            G, Y, inv_epsf, dt)
    return sv


def pml_profile(c: float, width: float, dx: float, y: float, R: float) -> float:
    return lib().orc_pml_profile(c, width, dx, y, R)


class OracleSim:
    """One simulation held by the oracle.  ``spec`` is a workload dictionary:
    {"grid": {...}, "materials": [...], "layers": [...], "projectile": {...} | None}."""

    def __init__(self, spec: dict):
        L = lib()
        self.spec = spec
        self.grid = dict(spec["grid"])
        mats = spec["materials"]
        self.grid["nmat"] = len(mats)
        g = make_grid(self.grid)
        arr = (Material * len(mats))(*[make_material(m) for m in mats])
        self._h = L.orc_create(C.byref(g), arr)
        if not self._h:
            raise ValueError("oracle rejected the grid")
        self.nr, self.nz = self.grid["nr"], self.grid["nz"]
        if self.grid.get("dr") is not None or self.grid.get("dz") is not None:
            dr = np.ascontiguousarray(self.grid.get("dr", [self.grid["dx"]] * self.nr), dtype=np.float64)
            dz = np.ascontiguousarray(self.grid.get("dz", [self.grid["dx"]] * self.nz), dtype=np.float64)
            if dr.shape != (self.nr,) or dz.shape != (self.nz,):
                raise ValueError("spacing arrays must have nr and nz entries")
            self._dr, self._dz = dr, dz
            rc = L.orc_set_spacing(self._h, dr.ctypes.data_as(C.POINTER(C.c_double)),
                                   dz.ctypes.data_as(C.POINTER(C.c_double)))
            if rc:
                raise ValueError(f"oracle rejected the spacing ({rc})")
        for lay in spec.get("layers", []):
            rc = L.orc_add_layer(self._h, lay["mat"], lay["zlo"], lay["zhi"], lay.get("rho", 0.0),
                                 lay.get("I0", 0.0), lay.get("vz", 0.0))
            if rc:
                raise ValueError(f"oracle rejected layer {lay} ({rc})")
        pj = spec.get("projectile")
        if pj:
            rc = L.orc_place_projectile(self._h, pj["mat"], pj["radius"], pj["zc"], pj["vz"],
                                        pj.get("rho", 0.0), pj.get("I0", 0.0))
            if rc:
                raise ValueError("oracle rejected the projectile")
        rc = L.orc_finalize(self._h)
        if rc:
            raise ValueError(f"oracle finalize failed ({rc})")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def step(self, n: int) -> int:
        return lib().orc_step(self._h, int(n))

    def phase0(self) -> int:
        """Phase 0 alone on the current state (EoS, artificial viscosity, peak
        over-pressure, Courant step) without advancing; afterwards ``get("P_total")`` is the
        total isotropic pressure p_hat + Phi q it formed."""
        return lib().orc_phase0(self._h)

    def _shape(self, name):
        return (self.nz + 1, self.nr + 1) if name in VERTEX_FIELDS else (self.nz, self.nr)

    def get(self, name: str) -> np.ndarray:
        shp = self._shape(name)
        out = np.zeros(shp, dtype=np.float64)
        rc = lib().orc_get_field(self._h, FIELDS[name], out.ctypes.data_as(C.POINTER(C.c_double)), out.size)
        if rc:
            raise KeyError(name)
        return out

    def set(self, name: str, values) -> None:
        arr = np.ascontiguousarray(values, dtype=np.float64).reshape(self._shape(name))
        rc = lib().orc_set_field(self._h, FIELDS[name], arr.ctypes.data_as(C.POINTER(C.c_double)), arr.size)
        if rc:
            raise KeyError(name)

    def scalars(self) -> dict:
        out = np.zeros(10)
        lib().orc_scalars(self._h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return {"t": out[0], "dt": out[1], "nstep": int(out[2]), "status": int(out[3]),
                "mass_out": out[4], "mass_discarded": out[5], "mass_pml": out[6], "zmom_out": out[7],
                "ke_lag": out[8], "ie_lag": out[9]}

    def set_time(self, t: float, dt_prev: float) -> None:
        lib().orc_set_time(self._h, t, dt_prev)

    def conservation(self) -> dict:
        out = np.zeros(4)
        lib().orc_conservation(self._h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return {"mass": out[0], "zmom": out[1], "ke": out[2], "ie": out[3]}

    def surface_heights(self) -> np.ndarray:
        out = np.zeros(self.nr)
        lib().orc_surface_heights(self._h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out


def crater_metrics(h: np.ndarray, dx: float, z_surface: float, npts: int, r_extent: float, rc=None):
    """Crater read-out from column surface heights h: depth on the axis (z_surface - h[0]);
    diameter = twice the first radius beyond the deepest column where the surface, linearly
    interpolated between column centres, regains z_surface (twice the last centre if it
    never does, 0 if there is no depression); depth profile z_surface - h sampled at
    r_k = (k + 1/2) r_extent / npts.  Column centres rc: (i + 1/2) dx unless given."""
    nr = h.size
    rc = (np.arange(nr) + 0.5) * dx if rc is None else np.asarray(rc, dtype=np.float64)
    depth_profile = z_surface - h
    depth = float(depth_profile[0])
    kmin = int(np.argmax(depth_profile))
    diameter = 0.0
    if depth_profile[kmin] > 0.0:
        diameter = 2.0 * float(rc[-1])
        for i in range(kmin, nr - 1):
            if h[i] < z_surface <= h[i + 1]:
                diameter = 2.0 * float(rc[i] + (z_surface - h[i]) / (h[i + 1] - h[i]) * (rc[i + 1] - rc[i]))
                break
    rk = (np.arange(npts) + 0.5) * r_extent / npts
    prof = np.interp(rk, rc, depth_profile)
    return depth, diameter, prof
