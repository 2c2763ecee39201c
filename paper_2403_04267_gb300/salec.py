"""Python binding of the C ABI in include/salec.h (ctypes; argument marshalling only).

Every step of the time step runs in the CUDA library ``_build/libsalec.so``; this module
only converts arguments.  PyTorch provides the device buffer and the stream.  If the
library cannot be loaded the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SALEC_OK, SALEC_EINVAL, SALEC_ENOMEM, SALEC_ECUDA, SALEC_EORDER, SALEC_EUNSTABLE, SALEC_ETIMEOUT = range(7)
SALEC_FP64 = 0
SALEC_FP32MIX = 1
SALEC_STEP_PHASES, SALEC_STEP_FUSED = 0, 1
PRECISIONS = {"fp64": SALEC_FP64, "fp32mix": SALEC_FP32MIX}
_STATUS = {0: "SALEC_OK", 1: "SALEC_EINVAL", 2: "SALEC_ENOMEM", 3: "SALEC_ECUDA", 4: "SALEC_EORDER",
           5: "SALEC_EUNSTABLE", 6: "SALEC_ETIMEOUT"}

FIELDS = {
    "f0": 0, "f1": 1, "f2": 2, "rho0": 3, "rho1": 4, "rho2": 5, "I": 6, "srr": 7, "szz": 8,
    "srz": 9, "D": 10, "pmax": 11, "vr": 12, "vz": 13, "p": 14,
    "phi1_b": 20, "phi3_b": 21, "psi2_b": 22, "phi1_r": 23, "phi3_r": 24, "psi2_r": 25,
    "phi2r_b": 30, "phi2z_b": 31, "psi1r_b": 32, "psi1z_b": 33,
    "phi2r_r": 34, "phi2z_r": 35, "psi1r_r": 36, "psi1z_r": 37,
}
VERTEX_FIELDS = {"vr", "vz", "phi2r_b", "phi2z_b", "psi1r_b", "psi1z_b",
                 "phi2r_r", "phi2z_r", "psi1r_r", "psi1z_r"}


class salec_grid(C.Structure):
    _fields_ = [
        ("nr", C.c_int), ("nz", C.c_int), ("nmat", C.c_int), ("dx", C.c_double),
        ("pml_right", C.c_int), ("pml_bottom", C.c_int), ("pml_R", C.c_double), ("pml_c", C.c_double), ("pml_alpha", C.c_double),
        ("gravity", C.c_double), ("cfl", C.c_double), ("dt_init", C.c_double), ("dt_max", C.c_double),
        ("dt_growth", C.c_double), ("dt_min", C.c_double), ("av_cq", C.c_double), ("av_cl", C.c_double),
        ("f_min", C.c_double), ("bc_top", C.c_int), ("bc_bottom", C.c_int),
    ]


class salec_material(C.Structure):
    _fields_ = [
        ("eos", C.c_int), ("rho0", C.c_double),
        ("A", C.c_double), ("B", C.c_double), ("E0", C.c_double), ("a", C.c_double), ("b", C.c_double),
        ("alpha", C.c_double), ("beta", C.c_double), ("Eiv", C.c_double), ("Ecv", C.c_double),
        ("gamma", C.c_double), ("strength", C.c_int),
        ("Yi0", C.c_double), ("mui", C.c_double), ("Yim", C.c_double), ("Yd0", C.c_double),
        ("mud", C.c_double), ("Ydm", C.c_double), ("G", C.c_double),
        ("eps_fb", C.c_double), ("B_dam", C.c_double), ("p_bd", C.c_double), ("p_t", C.c_double),
    ]


_lib = None
EXPORTS = ["salec_state_bytes", "salec_create", "salec_set_material", "salec_set_spacing", "salec_add_layer",
           "salec_place_projectile", "salec_finalize", "salec_step", "salec_get_scalars",
           "salec_set_time", "salec_get_field", "salec_set_field", "salec_crater_profile",
           "salec_conservation", "salec_checkpoint_bytes", "salec_get_state", "salec_set_state", "salec_state_changed",
           "salec_launches_per_step", "salec_set_kernel_timing", "salec_kernel_times",
           "salec_kernel_name", "salec_step_kernel_name", "salec_set_step_form", "salec_get_step_form",
           "salec_fused_queue", "salec_set_rest_copy",
           "salec_courant_dt_noalloc", "salec_last_error", "salec_destroy",
           "salec_set_end_time", "salec_set_block_shapes", "salec_get_block_shapes", "salec_autotune",
           "salec_batch_bytes", "salec_batch_create", "salec_batch_step", "salec_batch_run", "salec_batch_poll",
           "salec_batch_autotune", "salec_batch_set_persistent", "salec_batch_expire_next_barrier",
           "salec_batch_last_error", "salec_batch_destroy",
           "salec_mlp_n_params", "salec_mlp_bytes", "salec_mlp_create", "salec_mlp_set_params",
           "salec_mlp_get_params", "salec_mlp_forward", "salec_mlp_gradient", "salec_mlp_train_step",
           "salec_mlp_train", "salec_mlp_group_create", "salec_mlp_train_group", "salec_mlp_group_last_error",
           "salec_mlp_group_destroy",
           "salec_mlp_check", "salec_gemm_bf16", "salec_mlp_last_error", "salec_mlp_destroy"]


def load(build: bool = True):
    """Load (building first if needed) the CUDA library and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library missing: {path}")
    L = C.CDLL(path)
    P, D, Z, I = C.c_void_p, C.c_double, C.c_size_t, C.c_int
    PD = C.POINTER(C.c_double)
    sig = {
        "salec_state_bytes": (I, [C.POINTER(salec_grid), I, C.POINTER(C.c_size_t)]),
        "salec_create": (I, [C.POINTER(salec_grid), I, P, Z, P, C.POINTER(P)]),
        "salec_set_material": (I, [P, I, C.POINTER(salec_material)]),
        "salec_add_layer": (I, [P, I, D, D, D, D, D]),
        "salec_set_spacing": (I, [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "salec_place_projectile": (I, [P, I, D, D, D, D, D]),
        "salec_finalize": (I, [P]),
        "salec_step": (I, [P, I]),
        "salec_get_scalars": (I, [P, PD]),
        "salec_set_time": (I, [P, D, D]),
        "salec_get_field": (I, [P, I, PD, Z]),
        "salec_set_field": (I, [P, I, PD, Z]),
        "salec_crater_profile": (I, [P, D, I, PD, PD, PD, PD]),
        "salec_conservation": (I, [P, PD]),
        "salec_checkpoint_bytes": (I, [P, C.POINTER(C.c_size_t)]),
        "salec_get_state": (I, [P, P, Z]),
        "salec_set_state": (I, [P, P, Z]),
        "salec_state_changed": (I, [P]),
        "salec_launches_per_step": (I, [P]),
        "salec_set_kernel_timing": (I, [P, I]),
        "salec_kernel_times": (I, [P, PD, I, C.POINTER(C.c_int)]),
        "salec_kernel_name": (C.c_char_p, [I]),
        "salec_step_kernel_name": (C.c_char_p, [P, I]),
        "salec_fused_queue": (I, [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "salec_set_step_form": (I, [P, I]),
        "salec_set_rest_copy": (I, [P, I]),
        "salec_get_step_form": (I, [P]),
        "salec_courant_dt_noalloc": (I, [C.POINTER(salec_grid), C.POINTER(salec_material), C.POINTER(C.c_void_p),
                                         P, P, P, D, PD, P]),
        "salec_last_error": (C.c_char_p, [P]),
        "salec_set_end_time": (I, [P, D]),
        "salec_set_block_shapes": (I, [P, C.POINTER(C.c_int)]),
        "salec_get_block_shapes": (I, [P, C.POINTER(C.c_int)]),
        "salec_autotune": (I, [P, I, C.POINTER(C.c_int)]),
        "salec_batch_bytes": (I, [C.POINTER(P), I, C.POINTER(C.c_size_t)]),
        "salec_batch_create": (I, [C.POINTER(P), I, P, Z, P, C.POINTER(P)]),
        "salec_batch_step": (I, [P, I]),
        "salec_batch_run": (I, [P, I, C.c_long, C.POINTER(C.c_long), C.POINTER(C.c_int)]),
        "salec_batch_poll": (I, [P, PD]),
        "salec_batch_autotune": (I, [P, I, C.POINTER(C.c_int)]),
        "salec_batch_set_persistent": (I, [P, I]),
        "salec_batch_expire_next_barrier": (I, [P]),
        "salec_batch_last_error": (C.c_char_p, [P]),
        "salec_batch_destroy": (None, [P]),
        "salec_destroy": (None, [P]),
        "salec_mlp_n_params": (I, []),
        "salec_mlp_bytes": (I, [I, C.POINTER(C.c_size_t)]),
        "salec_mlp_create": (I, [I, P, Z, P, C.POINTER(P)]),
        "salec_mlp_set_params": (I, [P, P]),
        "salec_mlp_get_params": (I, [P, P]),
        "salec_mlp_forward": (I, [P, P, I, P]),
        "salec_mlp_gradient": (I, [P, P, P, I, P, PD]),
        "salec_mlp_train_step": (I, [P, P, P, I, C.c_float, C.c_float, C.c_float, C.c_float, P]),
        "salec_mlp_train": (I, [P, P, P, I, I, P, C.c_float, C.c_float, C.c_float, P]),
        "salec_mlp_group_create": (I, [C.POINTER(P), I, P, C.POINTER(P)]),
        "salec_mlp_train_group": (I, [P, P, P, I, I, P, C.c_float, C.c_float, C.c_float]),
        "salec_mlp_group_last_error": (C.c_char_p, [P]),
        "salec_mlp_group_destroy": (None, [P]),
        "salec_mlp_check": (I, [P]),
        "salec_gemm_bf16": (I, [I, I, I, P, C.c_long, C.c_long, P, C.c_long, C.c_long, P, C.c_long, P]),
        "salec_mlp_last_error": (C.c_char_p, [P]),
        "salec_mlp_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class SalecError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_EOS = {"tillotson": 0, "ideal_gas": 1}
_STR = {"none": 0, "collins": 1}
_TOP = {"outflow": 0, "wall": 1}
_BOTTOM = {"noslip": 0, "freeslip": 1}


def make_grid(d: dict, nmat: int) -> salec_grid:
    g = salec_grid()
    g.nr, g.nz, g.nmat, g.dx = int(d["nr"]), int(d["nz"]), int(nmat), float(d["dx"])
    g.pml_right, g.pml_bottom = int(d.get("pml_r", 0)), int(d.get("pml_b", 0))
    for k in ("pml_R", "pml_c", "pml_alpha", "gravity", "cfl", "dt_init", "dt_max", "dt_growth", "dt_min",
              "av_cq", "av_cl", "f_min"):
        setattr(g, k, float(d.get(k, 0.0)))
    g.bc_top = _TOP[d.get("bc_top", "outflow")]
    g.bc_bottom = _BOTTOM[d.get("bc_bottom", "noslip")]
    return g


def make_material(d: dict) -> salec_material:
    m = salec_material()
    for name, _ in salec_material._fields_:
        if name == "eos":
            m.eos = _EOS[d.get("eos", "tillotson")]
        elif name == "strength":
            m.strength = _STR[d.get("strength", "none")]
        else:
            setattr(m, name, float(d.get(name, 0.0)))
    return m


class Sim:
    """One simulation on the current CUDA device.  ``spec`` is a workload dictionary
    (see workloads.py); ``precision`` is "fp64" or "fp32mix" (FP32 fields and stencils,
    FP64 specific internal energy, Courant reduction and sums).  The device state is one
    torch uint8 tensor owned here."""

    def __init__(self, spec: dict, device=None, stream=None, precision: str = "fp64"):
        import torch
        L = load()
        self.spec = spec
        self.precision = PRECISIONS[precision]
        self.nmat = len(spec["materials"])
        self.grid = make_grid(spec["grid"], self.nmat)
        self.nr, self.nz = self.grid.nr, self.grid.nz
        nb = C.c_size_t()
        self._check(L.salec_state_bytes(C.byref(self.grid), self.precision, C.byref(nb)), None)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.state = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        self._check(L.salec_create(C.byref(self.grid), self.precision, C.c_void_p(self.state.data_ptr()), nb.value,
                                   C.c_void_p(self.stream.cuda_stream), C.byref(h)), None)
        self._h = h
        for k, m in enumerate(spec["materials"]):
            mm = make_material(m)
            self._check(L.salec_set_material(h, k, C.byref(mm)))
        gd = spec["grid"]
        if gd.get("dr") is not None or gd.get("dz") is not None:
            dr = np.ascontiguousarray(gd.get("dr", [gd["dx"]] * self.nr), dtype=np.float64)
            dz = np.ascontiguousarray(gd.get("dz", [gd["dx"]] * self.nz), dtype=np.float64)
            if dr.shape != (self.nr,) or dz.shape != (self.nz,):
                raise ValueError("spacing arrays must have nr and nz entries")
            self._check(L.salec_set_spacing(h, dr.ctypes.data_as(C.POINTER(C.c_double)),
                                            dz.ctypes.data_as(C.POINTER(C.c_double))))
            self.rc = np.cumsum(dr) - 0.5 * dr
        for lay in spec.get("layers", []):
            self._check(L.salec_add_layer(h, int(lay["mat"]), float(lay["zlo"]), float(lay["zhi"]),
                                          float(lay.get("rho", 0.0)), float(lay.get("I0", 0.0)),
                                          float(lay.get("vz", 0.0))))
        pj = spec.get("projectile")
        if pj:
            self._check(L.salec_place_projectile(h, int(pj["mat"]), float(pj["radius"]), float(pj["zc"]),
                                                 float(pj["vz"]), float(pj.get("rho", 0.0)),
                                                 float(pj.get("I0", 0.0))))
        self._check(L.salec_finalize(h))

    def _check(self, st, h="self"):
        if st != SALEC_OK:
            hh = self._h if h == "self" else None
            msg = load().salec_last_error(hh).decode() if hh else ""
            raise SalecError(st, msg)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            load().salec_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def step(self, n: int) -> None:
        self._check(load().salec_step(self._h, int(n)))

    def scalars(self, check: bool = False) -> dict:
        out = np.zeros(8)
        st = load().salec_get_scalars(self._h, out.ctypes.data_as(C.POINTER(C.c_double)))
        if st not in (SALEC_OK, SALEC_EUNSTABLE) or (check and st != SALEC_OK):
            self._check(st)
        return {"t": out[0], "dt": out[1], "nstep": int(out[2]), "status": int(out[3]),
                "mass_out": out[4], "mass_discarded": out[5], "mass_pml": out[6], "zmom_out": out[7]}

    def set_time(self, t: float, dt_prev: float) -> None:
        self._check(load().salec_set_time(self._h, float(t), float(dt_prev)))

    def _shape(self, name):
        return (self.nz + 1, self.nr + 1) if name in VERTEX_FIELDS else (self.nz, self.nr)

    def get(self, name: str) -> np.ndarray:
        out = np.zeros(self._shape(name))
        self._check(load().salec_get_field(self._h, FIELDS[name], out.ctypes.data_as(C.POINTER(C.c_double)), out.size))
        return out

    def set(self, name: str, values) -> None:
        arr = np.ascontiguousarray(values, dtype=np.float64).reshape(self._shape(name))
        self._check(load().salec_set_field(self._h, FIELDS[name], arr.ctypes.data_as(C.POINTER(C.c_double)), arr.size))

    def conservation(self) -> dict:
        out = np.zeros(4)
        self._check(load().salec_conservation(self._h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return {"mass": out[0], "zmom": out[1], "ke": out[2], "ie": out[3]}

    def crater(self, z_surface: float, npts: int = 64):
        prof = np.zeros(max(npts, 1))
        h = np.zeros(self.nr)
        d, D = C.c_double(), C.c_double()
        self._check(load().salec_crater_profile(self._h, float(z_surface), int(npts),
                                                prof.ctypes.data_as(C.POINTER(C.c_double)),
                                                h.ctypes.data_as(C.POINTER(C.c_double)), C.byref(d), C.byref(D)))
        return {"depth": d.value, "diameter": D.value, "profile": prof[:npts], "heights": h}

    def surface_heights(self) -> np.ndarray:
        return self.crater(0.0, 0)["heights"]

    def checkpoint_bytes(self) -> int:
        n = C.c_size_t()
        self._check(load().salec_checkpoint_bytes(self._h, C.byref(n)))
        return n.value

    def get_state(self) -> np.ndarray:
        buf = np.zeros(self.checkpoint_bytes(), dtype=np.uint8)
        self._check(load().salec_get_state(self._h, C.c_void_p(buf.ctypes.data), buf.size))
        return buf

    def set_state(self, buf) -> None:
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(load().salec_set_state(self._h, C.c_void_p(b.ctypes.data), b.size))

    def state_changed(self) -> None:
        """Declare that the checkpoint range of ``state`` was written directly (a device
        copy of an earlier image): the next step starts from it."""
        self._check(load().salec_state_changed(self._h))

    def launches_per_step(self) -> int:
        return load().salec_launches_per_step(self._h)

    def set_end_time(self, t_end: float) -> None:
        self._check(load().salec_set_end_time(self._h, float(t_end)))

    def block_shapes(self) -> list:
        a = (C.c_int * 12)()
        self._check(load().salec_get_block_shapes(self._h, a))
        return [(a[2 * k], a[2 * k + 1]) for k in range(6)]

    def set_block_shapes(self, shapes) -> None:
        a = (C.c_int * 12)(*[int(v) for xy in shapes for v in xy])
        self._check(load().salec_set_block_shapes(self._h, a))

    def autotune(self, trial_steps: int = 5) -> list:
        a = (C.c_int * 12)()
        self._check(load().salec_autotune(self._h, int(trial_steps), a))
        return [(a[2 * k], a[2 * k + 1]) for k in range(6)]

    def set_kernel_timing(self, on: bool) -> None:
        self._check(load().salec_set_kernel_timing(self._h, 1 if on else 0))

    def kernel_times(self) -> tuple[dict, int]:
        """Mean per-kernel duration (ms) over the steps recorded since the last read."""
        n = 6
        out = np.zeros(n)
        steps = C.c_int()
        self._check(load().salec_kernel_times(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), n, C.byref(steps)))
        names = [load().salec_step_kernel_name(self._h, k).decode() for k in range(n)]
        return {nm: float(out[k]) for k, nm in enumerate(names) if nm}, steps.value

    def fused_queue(self) -> tuple[int, int]:
        """(tiles the last fused step ran through the whole cycle, tiles of the grid); the
        others it copied as at rest.  (0, 0) before a fused step."""
        q, t = C.c_int(), C.c_int()
        self._check(load().salec_fused_queue(self._h, C.byref(q), C.byref(t)))
        return q.value, t.value

    def set_rest_copy(self, mode) -> None:
        """Fused form, tiles at rest: 0 (or False) run every tile through the tile kernel;
        1 (or True, the default) copy them with the rest-tile kernel before the tile kernel;
        2 copy them beside the tile kernel where the form allows it, else as 1.  The results
        are the same bit for bit."""
        m = 1 if mode is True else 0 if mode is False else int(mode)
        self._check(load().salec_set_rest_copy(self._h, m))

    @property
    def step_form(self) -> str:
        """"fused" (one tile kernel per step after the Courant kernel) or "phases" (six
        whole-grid kernels and the Courant kernel)."""
        return {SALEC_STEP_PHASES: "phases", SALEC_STEP_FUSED: "fused"}[load().salec_get_step_form(self._h)]

    @step_form.setter
    def step_form(self, form: str) -> None:
        self._check(load().salec_set_step_form(self._h, {"phases": SALEC_STEP_PHASES, "fused": SALEC_STEP_FUSED}[form]))


def run_logged(sim, steps: int, every: int, path: str, z_surface: float | None = None) -> list:
    """Advance `sim` by `steps` steps in calls of `every` steps; after each call append one
    JSON line to `path` (and to the returned list): the step count, time, the last dt and the
    status word, the conservation sums (mass, z-momentum, kinetic and internal energy), the
    tallies (mass out through the top, removed by clean-up, added by the strips' damping,
    z-momentum out), the largest peak over-pressure, and with `z_surface` the crater depth
    and diameter.  The dt history and the crater's growth of a run, as a log.  A run whose
    status reports a failure stops logging after the line that shows it."""
    import json
    every = max(int(every), 1)
    out = []
    done = 0
    with open(path, "a") as fh:
        while done < steps:
            n = min(every, steps - done)
            sim.step(n)
            done += n
            sc = sim.scalars()
            rec = {"step": int(sc["nstep"]), "t": float(sc["t"]), "dt": float(sc["dt"]), "status": int(sc["status"]),
                   "tallies": {k: float(sc[k]) for k in ("mass_out", "mass_discarded", "mass_pml", "zmom_out")},
                   "sums": {k: float(v) for k, v in sim.conservation().items()},
                   "pmax": float(np.max(sim.get("pmax")))}
            if z_surface is not None:
                cr = sim.crater(z_surface, 64)
                rec["crater"] = {"depth": float(cr["depth"]), "diameter": float(cr["diameter"])}
            fh.write(json.dumps(rec) + "\n")
            out.append(rec)
            if rec["status"] != 0:
                break
    return out


def courant_dt_noalloc(spec: dict, fr_ptrs, I_ptr: int, v_ptr: int, dt_prev: float, stream_ptr: int,
                       D_ptr: int | None = None) -> float:
    """Courant time step of a state held in caller device buffers, with no allocation
    (see salec_courant_dt_noalloc in include/salec.h).  Pointers are raw device addresses."""
    L = load()
    nm = len(spec["materials"])
    g = make_grid(spec["grid"], nm)
    mats = (salec_material * nm)(*[make_material(m) for m in spec["materials"]])
    frs = (C.c_void_p * nm)(*[C.c_void_p(int(p)) for p in fr_ptrs])
    out = C.c_double()
    st = L.salec_courant_dt_noalloc(C.byref(g), mats, frs, C.c_void_p(int(I_ptr)),
                                    C.c_void_p(int(D_ptr)) if D_ptr else None, C.c_void_p(int(v_ptr)),
                                    float(dt_prev), C.byref(out), C.c_void_p(int(stream_ptr)))
    if st != SALEC_OK:
        raise SalecError(st, L.salec_last_error(None).decode())
    return out.value


class Batch:
    """Independent runs advanced together (one set of launches per step, per-run dt and end
    time, CUDA-graph-captured chunks).  ``sims`` are finalized Sim objects of one precision
    and material class on the current device."""

    def __init__(self, sims, stream=None):
        import torch
        L = load()
        self.sims = list(sims)
        n = len(self.sims)
        self._arr = (C.c_void_p * n)(*[s.handle for s in self.sims])
        nb = C.c_size_t()
        st = L.salec_batch_bytes(self._arr, n, C.byref(nb))
        if st != SALEC_OK:
            raise SalecError(st, "runs cannot be batched together")
        dev = self.sims[0].device
        self.buf = torch.empty(nb.value, dtype=torch.uint8, device=dev)
        # graph capture needs a created stream; the runs' own work must be finished first
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        torch.cuda.synchronize(dev)
        h = C.c_void_p()
        st = L.salec_batch_create(self._arr, n, C.c_void_p(self.buf.data_ptr()), nb.value,
                                  C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != SALEC_OK:
            raise SalecError(st, "batch create failed")
        self._h = h

    def _check(self, st):
        if st != SALEC_OK:
            raise SalecError(st, load().salec_batch_last_error(self._h).decode())

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            load().salec_batch_destroy(h)
            self._h = None

    def step(self, n: int) -> None:
        """n batched steps; returns after they finished (the runs' fields are then safe to
        read on any stream).  In persistent mode a grid-barrier wait that ran out raises
        SalecError (SALEC_ETIMEOUT)."""
        self._check(load().salec_batch_step(self._h, int(n)))
        self.stream.synchronize()
        if self.persistent:
            self.poll()

    @property
    def persistent(self) -> bool:
        """Persistent mode: one cooperative launch per step call or run chunk (grid-wide
        barriers between the phases) instead of six launches and a Courant kernel per step."""
        return getattr(self, "_persistent", False)

    @persistent.setter
    def persistent(self, on: bool) -> None:
        self._check(load().salec_batch_set_persistent(self._h, 1 if on else 0))
        self._persistent = bool(on)

    def expire_next_barrier(self) -> None:
        """Failure-detection test: the next persistent step call's first grid barrier never
        completes, its waits run out (2 s) and step() raises SalecError (SALEC_ETIMEOUT)."""
        self._check(load().salec_batch_expire_next_barrier(self._h))

    def run(self, chunk: int = 50, max_steps: int = 10 ** 9):
        steps, done = C.c_long(), C.c_int()
        self._check(load().salec_batch_run(self._h, int(chunk), int(max_steps), C.byref(steps), C.byref(done)))
        return steps.value, done.value

    def poll(self) -> np.ndarray:
        out = np.zeros(5 * len(self.sims))
        self._check(load().salec_batch_poll(self._h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out.reshape(-1, 5)

    def autotune(self, trial_steps: int = 3) -> list:
        a = (C.c_int * 12)()
        self._check(load().salec_batch_autotune(self._h, int(trial_steps), a))
        return [(a[2 * k], a[2 * k + 1]) for k in range(6)]
