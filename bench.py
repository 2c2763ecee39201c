#!/usr/bin/env python
"""Headline benchmark: cell-updates/s of the explicit ALE step of SALEc-2D on GB300.

Workload (default): the 4000 x 4000 single-run configuration (10 m cells, basalt
Tillotson half-space, hydrodynamic, projectile radius 100 cells at 10 km/s, PML 16 right
and bottom, no gravity), FP64: W warm-up steps from t = 0, then K timed steps that continue
the run (default K = 2000, the configuration's run length).  One "step" is one full cycle of the hot path (EoS + artificial viscosity +
Courant min-reduction, Lagrangian momentum/energy/strength, PML, donor-cell remap,
momentum remap, heat) over all 16e6 cells.  The state (~1.3 GB) is larger than L2, so no
flush is needed between steps.

Output: one JSON line:
  value      cell-updates/s, device-timed (CUDA events on the library's stream), state
             resident in HBM; N GPUs run N independent replicas (weak scaling)
  e2e        the same metric through the C ABI with host buffers: the initial state is
             copied from pinned host memory, every step reads its scalars (t, dt, status)
             back, and the final pressure field is copied to the host
  roofline   the dominant kernel against its bound: the FP64 pipe for the FP64 form,
             HBM bandwidth for the mixed form
  cpu_baseline  the serial FP64 oracle on the host cores, on a bounded sample
``--impl reference`` times the oracle itself (the reference arm of this repository).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per ALE step (FP64 vs FP32, % HBM roofline); batched runs/hour"
UNIT = "cell-updates/s"

# FP64 issue rate of the part: 2 DFMA per clock per SM (its nominal 1.25 TFLOP/s at
# 152 SMs and 2.07 GHz); the bench reads the SM count from the device and the clock from
# nvidia-smi, and measures an FP64 GEMM (cuBLAS) as the attainable peak.
DFMA_PER_CLK_PER_SM = 2


def fp64_peaks(sm_max_mhz):
    """(nominal TFLOP/s from the device's SM count and maximum clock, measured TFLOP/s of a
    4096^3 FP64 GEMM, best of 5 by CUDA events)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    nominal = sms * DFMA_PER_CLK_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    n = 4096
    a = torch.rand((n, n), dtype=torch.float64, device="cuda")
    b = torch.rand((n, n), dtype=torch.float64, device="cuda")
    c = a @ b
    best = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(5):
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    del a, b, c
    return sms, nominal, best

# Algorithmic bytes per cell-update of each kernel (one material, hydrodynamic): the fields
# each kernel must read and write once, e = element bytes (8 FP64, 4 mixed), energies 8.
def kernel_bytes_per_cell(e: int) -> dict:
    return {
        "k_phase0": 2 * e + 8 + 2 * e + 2 * e + 2 * e + 2 * e,    # (f,rho) I v pmax(rw) -> (P,M) (pbar,phi)
        "k_phase1": 2 * e + 2 * e + 2 * e + 2 * e + e + e,        # (P,M) phi v -> vL mv dK
        "k_phase2": 2 * e + 2 * e + 2 * e + 8 + 2 * e + e + 8,    # vL (P,M) (pbar,phi) I -> (fL,rhoL) VL IL
        "k_phase3a": 2 * e + 2 * e + e + 8 + 2 * e + 8 + e + e,   # vL (fL,rhoL) VL IL -> (f,rho) I dMR dMZ
        "k_phase3b": e + e + 2 * e + e + e + 2 * e + e,           # dMR dMZ vL mv dK -> v kheat
        "k_phase3c": 2 * e + e + 8 + 8,                           # (f,rho) kheat I(rw)
        # the fused cycle reads and writes the persistent state once (plus the Courant kernel)
        "k_step_fused": step_bytes_per_cell(e),
        # a tile at rest: (f, rho), I and the EoS cache (p, c^2) read and written, vertices
        # written (at rest): the same count as the state's
        "k_rest_tiles": 2 * (2 * e + 8 + 2 * e) + 2 * e,
        # the same tiles moved by the copy kernel that runs beside the tile kernel
        "k_rest_copy": 2 * (2 * e + 8 + 2 * e) + 2 * e,
    }


# the fused form's kernels that copy the tiles at rest (before the tile kernel, or beside it)
REST_KERNELS = ("k_rest_tiles", "k_rest_copy")


# persistent state read once and written once per step (one material, hydrodynamic):
# (f, rho), I, pmax, v
def step_bytes_per_cell(e: int) -> int:
    return 2 * (2 * e + 8 + e + 2 * e)


def _load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"])
    except Exception:
        return 2070.0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload(name):
    from paper_2403_04267_gb300 import workloads as W
    return {"large_4000": W.large_4000, "full_800": W.full_fp64_800, "plain_100": W.plain_fp64_100,
            "plain_2000": lambda: W.scaled_plain(2000, radius_cells=50)}[name]()


def _cpu_baseline(spec, steps):
    """The oracle as it stands, serial, on `steps` steps of the full workload from t = 0."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    s = O.OracleSim(spec)
    t1 = time.perf_counter()
    s.step(steps)
    t2 = time.perf_counter()
    cells = spec["grid"]["nr"] * spec["grid"]["nz"]
    return {"value": cells * steps / (t2 - t1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} steps of the full {spec['grid']['nr']}x{spec['grid']['nz']} workload from t=0 "
                      f"(serial C, -O2; set-up {t1 - t0:.1f} s excluded)", "seconds": round(t2 - t1, 2)}


def shard(n_units: int, rank: int, ws: int) -> list:
    """The units (runs, seeds) rank `rank` of `ws` processes: r, r + ws, r + 2 ws, ...  No
    unit is shared, none is left out, and no data-path exchange is needed."""
    return list(range(rank, n_units, ws))


def job_reduce(vals_max, vals_sum, device="cpu"):
    """Whole-job figures over ranks: the max of times, the sum of counts (one all_reduce each;
    a no-op in a single process)."""
    import torch
    import torch.distributed as dist
    mx = torch.tensor(list(vals_max), dtype=torch.float64, device=device)
    sm = torch.tensor(list(vals_sum), dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx.tolist(), sm.tolist()


def batch_failures(polled, specs, half_diameters, cavity_in_strip=None) -> list:
    """Counts of a batch's outcomes, in the order [non-positive volume or density, NaN, step
    below dt_min, failed runs with an iron projectile, with a basalt one, runs whose crater
    rim reached the absorbing strip, failed runs whose transient cavity had reached an
    absorbing strip, failed runs whose cavity had not].  `polled` rows are (t, dt, steps,
    status, t_end); `half_diameters` holds each run's crater half-width in metres (None for
    a failed run); `cavity_in_strip[k]` tells whether run k, where it stopped, has emptied
    strip cells below its initial surface (None: not examined).  A run counts once per
    status bit it carries."""
    import numpy as np
    st = np.asarray(polled)[:, 3].astype(np.int64)
    failed = st != 0
    iron = np.array([sp["materials"][-1]["rho0"] > 5000.0 for sp in specs], dtype=bool)
    at_pml = sum(1 for sp, h in zip(specs, half_diameters)
                 if h is not None and h >= (sp["grid"]["nr"] - sp["grid"]["pml_r"]) * sp["grid"]["dx"])
    cav = [bool(c) for c in (cavity_in_strip or [None] * len(specs))]
    in_strip = sum(1 for k in range(len(specs)) if failed[k] and cav[k])
    return [int(((st & 1) != 0).sum()), int(((st & 2) != 0).sum()), int(((st & 4) != 0).sum()),
            int((failed & iron).sum()), int((failed & ~iron).sum()), int(at_pml),
            int(in_strip), int(failed.sum()) - int(in_strip)]


def cavity_in_strip(phi, spec, density_ratio=None) -> bool:
    """Whether a cavity has reached an absorbing strip: a strip cell (bottom rows < pml_b,
    right columns >= nr - pml_r) below the initial surface holds less than half matter, or
    its matter has been torn open to below 1 % of its reference density (density_ratio:
    sum f_m rho_m / sum f_m rho0_m per cell, where matter is present).  The strips damp
    deviations from the initial state and are written for small ones (Sect. 3); a run whose
    cavity reaches them is outside that regime."""
    import numpy as np
    g = spec["grid"]
    nr, nz, pb, pr = g["nr"], g["nz"], g.get("pml_b", 0), g.get("pml_r", 0)
    ks = int(round(spec["z_surface"] / g["dx"]))
    strip = np.zeros((nz, nr), dtype=bool)
    strip[:pb, :] = True
    strip[:, nr - pr:] = True
    strip[ks:, :] = False
    hole = np.asarray(phi) < 0.5
    if density_ratio is not None:
        hole |= np.asarray(density_ratio) < 0.01
    return bool(hole[strip].any())


def density_ratio(sim, spec):
    """Per cell sum f_m rho_m / sum f_m rho0_m (1 where no matter is present)."""
    import numpy as np
    num, den = 0.0, 0.0
    for m, mat in enumerate(spec["materials"]):
        f = sim.get(f"f{m}")
        num = num + f * sim.get(f"rho{m}")
        den = den + f * mat["rho0"]
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), 1.0)


def _batched(args, rank, ws):
    """Batched impacts of the seeded distribution (rank r takes seeds r, r + ws, ...), FP32-mix,
    each to t_end: one batch, autotuned block shapes, CUDA-graph chunks.  A run whose status
    reports a failure (a non-positive volume or density, a NaN, or a step below dt_min) stops
    where it failed, counts as finished and is listed by cause.  runs/hour over the
    whole job; the plain FP64 solver, one run at a time, on the first few draws that finished
    cleanly gives the reference runs/hour and the crater depth and diameter that the batch
    is checked against (the FP64 GPU solver matches the FP64 oracle to 1e-9 and stands in
    for it here)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2403_04267_gb300 import salec, workloads as W
    seeds = shard(args.batch_runs, rank, ws)
    specs = [W.batched_run(W.batched_draw(sd)) for sd in seeds]
    for sp in specs:
        sp["t_end"] = args.batch_t_end
    t0 = time.perf_counter()
    sims = [salec.Sim(sp, precision="fp32mix") for sp in specs]
    for sm in sims:
        sm.set_end_time(args.batch_t_end)
    batch = salec.Batch(sims)
    setup_s = time.perf_counter() - t0
    cells = sum(sp["grid"]["nr"] * sp["grid"]["nz"] for sp in specs)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    shapes = batch.autotune(trial_steps=2)
    steps, done = 0, 0
    while done < len(sims) and time.perf_counter() - t0 < args.batch_max_s:
        s1, done = batch.run(chunk=50, max_steps=2000)
        steps += s1
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    polled = batch.poll()
    failed = polled[:, 3] != 0
    finished = (polled[:, 0] >= polled[:, 4]) | failed
    completed = (polled[:, 0] >= polled[:, 4]) & ~failed
    cell_updates = float(sum(polled[k, 2] * specs[k]["grid"]["nr"] * specs[k]["grid"]["nz"] for k in range(len(specs))))
    st = polled[:, 3].astype(np.int64)
    # read after the timed region: each clean run's crater half-width, for the strip flag,
    # and where each failed run stopped, whether its cavity had reached a strip
    half = [None if failed[k] else 0.5 * sims[k].crater(sp["z_surface"], 64)["diameter"]
            for k, sp in enumerate(specs)]
    cav = [cavity_in_strip(sum(sims[k].get(f"f{m}") for m in range(len(sp["materials"]))), sp,
                           density_ratio(sims[k], sp)) if failed[k] else None
           for k, sp in enumerate(specs)]
    causes = batch_failures(polled, specs, half, cav)
    (tmax,), (nfin, nfail, ncomp, *causes) = job_reduce(
        [wall], [int(finished.sum()), int(failed.sum()), int(completed.sum())] + causes, "cuda")
    nfin, nfail, ncomp = int(nfin), int(nfail), int(ncomp)
    out = {"runs": args.batch_runs, "t_end_s": args.batch_t_end, "precision": "FP32-mix",
           "runs_finished": nfin, "runs_failed": nfail, "runs_completed": ncomp, "complete": nfin == args.batch_runs,
           "wall_s": round(tmax, 2),
           # runs that reached t_end without a failure, per hour of the whole batch's wall time
           "runs_per_hour": ncomp * 3600.0 / tmax if nfin == args.batch_runs else None,
           "cell_updates_per_s": cell_updates / wall, "batch_steps": int(steps), "cells_per_step": cells,
           "setup_s": round(setup_s, 1), "block_shapes": shapes, "runs_per_rank": len(specs),
           "crater_reached_pml": int(causes[5]),
           "failures": {"volume_or_density": int(causes[0]), "nan": int(causes[1]), "dt_min": int(causes[2]),
                        "iron_projectile": int(causes[3]), "basalt_projectile": int(causes[4]),
                        "cavity_in_strip": int(causes[6]), "unexplained": int(causes[7]),
                        "rank0_first": [{"seed": int(seeds[k]), "n": specs[k]["grid"]["nr"], "status": int(st[k]),
                                         "t_s": round(float(polled[k, 0]), 3), "steps": int(polled[k, 2]),
                                         "cavity_in_strip": cav[k]}
                                        for k in np.where(failed)[0][:16]]}}
    # reference: the plain FP64 solver, one run at a time, on the first draws that finished cleanly
    ok = [k for k in range(len(specs)) if finished[k] and not failed[k]][:args.batch_ref_runs]
    if ok:
        errs_d, errs_D, t_ref, nref = [], [], 0.0, 0
        t_start = time.perf_counter()
        for k in ok:
            if time.perf_counter() - t_start > args.batch_ref_max_s:
                break
            sp = specs[k]
            ref = salec.Sim(sp, precision="fp64")
            ref.set_end_time(args.batch_t_end)
            one = salec.Batch([ref])            # one run: stops at the step that reaches t_end
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            one.run(chunk=50, max_steps=400000)
            torch.cuda.synchronize()
            t_ref += time.perf_counter() - t1
            if ref.scalars()["status"] != 0:
                continue
            nref += 1
            a, b = sims[k].crater(sp["z_surface"], 64), ref.crater(sp["z_surface"], 64)
            errs_d.append(abs(a["depth"] / b["depth"] - 1) if b["depth"] else 0.0)
            errs_D.append(abs(a["diameter"] / b["diameter"] - 1) if b["diameter"] else 0.0)
            del one, ref
        if nref:
            out["fp64_single_run_runs_per_hour"] = nref * 3600.0 / t_ref
            out["fp64_reference_runs"] = nref
            if out["runs_per_hour"]:
                out["speedup_vs_fp64_runs_per_hour"] = out["runs_per_hour"] / out["fp64_single_run_runs_per_hour"]
            out["crater_rel_err_vs_fp64"] = {"depth_max": max(errs_d), "diameter_max": max(errs_D),
                                             "depth_mean": float(np.mean(errs_d)),
                                             "diameter_mean": float(np.mean(errs_D))}
    del batch, sims
    torch.cuda.empty_cache()
    return out


def _batch_modes(args):
    """The two batched launch forms on the same runs: graph replays of six kernels and a
    Courant kernel per step (the default), against one persistent cooperative launch per
    chunk with grid-wide barriers between the phases.  Each form steps fresh copies of the
    runs from t = 0, after one untimed chunk, with its own autotuned block shapes; ms per
    batched step over the timed chunks, by CUDA events on the batch stream.  Two cases: the
    batched workload's full draw (every run active, large work per phase) and 16 runs of
    200 x 200 cells (little work per phase: launch and barrier costs show)."""
    import torch
    from paper_2403_04267_gb300 import salec, workloads as W
    out = {}
    cases = [("full_draw", args.batch_runs, None), ("small_16x200", 16, 200)]
    for name, nruns, n in cases:
        specs = []
        for sd in range(nruns):
            d = W.batched_draw(sd)
            if n:
                d["n"] = n
            specs.append(W.batched_run(d))
        res = {"runs": nruns, "cells_per_step": sum(sp["grid"]["nr"] * sp["grid"]["nz"] for sp in specs)}
        chunk, chunks = 25, 8 if n is None else 40
        for mode in ("graph", "persistent"):
            sims = [salec.Sim(sp, precision="fp32mix") for sp in specs]
            b = salec.Batch(sims)
            if mode == "persistent":
                b.persistent = True
            shapes = b.autotune(trial_steps=2)
            b.run(chunk=chunk, max_steps=chunk)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(b.stream)
            for _ in range(chunks):
                b.run(chunk=chunk, max_steps=chunk)
            e1.record(b.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / (chunk * chunks)
            res[mode] = {"ms_per_step": round(ms, 4), "block_shapes": shapes[:1] if mode == "persistent" else shapes,
                         "launches_per_step": 7 if mode == "graph" else round(1.0 / chunk, 3)}
            del b, sims
            torch.cuda.empty_cache()
        res["persistent_over_graph"] = round(res["persistent"]["ms_per_step"] / res["graph"]["ms_per_step"], 3)
        out[name] = res
    out["note"] = ("ms per batched step (every active run advances one step), FP32-mix, strength, two materials, "
                   "gravity; each chunk ends with a poll of the runs' scalars in both forms")
    return out


def _mlp_step_probe(batch: int, steps: int) -> int:
    """One network's training steps on seeded random inputs and targets of the surrogate's
    shape, one salec_mlp_train_step call each: `steps` untimed, then `steps` timed by CUDA
    events on the network's stream."""
    import numpy as np
    import torch
    from paper_2403_04267_gb300 import surrogate as S, workloads as W
    torch.cuda.set_device(0)
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.uniform(-1, 1, (batch, S.N_IN)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.uniform(0, 1, (batch, S.N_OUT)).astype(np.float32)).cuda()
    net = S.MLP(batch)
    net.set_params(W.mlp_init(1).astype(np.float32))
    torch.cuda.synchronize()
    for _ in range(steps):
        net.train_step(X, T, 1e-4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(net.stream)
    for _ in range(steps):
        net.train_step(X, T, 1e-4)
    e1.record(net.stream)
    torch.cuda.synchronize()
    net.check()
    ms = e0.elapsed_time(e1) / steps
    fwd = 2.0 * sum(a * b for a, b in zip(S.DIMS[:-1], S.DIMS[1:]))
    print(json.dumps({"mlp_step_probe": {"batch": batch, "steps": steps, "ms_per_step": ms,
                                         "tflops": 3.0 * fwd * batch / (ms * 1e-3) / 1e12}}))
    return 0


def _surrogate(args):
    """The crater surrogate: an ensemble of MLPs trained on the GPU by the library's own
    tcgen05 kernels on the batched solver's 400 x 400 runs (4096 training draws, 256
    held-out), gated by ensemble spread with the solver as fallback.  Reports runs/hour on
    the held-out draws with and without the surrogate (the solver's cost measured here: the
    plain FP64 solver, one run at a time, on held-out draws), the accepted predictions'
    errors, and the tensor throughput of training and of large-batch inference."""
    import numpy as np
    import torch
    from paper_2403_04267_gb300 import salec, surrogate as S, workloads as W
    path = os.path.join(ROOT, "paper_2403_04267_gb300", "data", "surrogate_400.npz")
    if not os.path.exists(path):
        return {"unavailable": "training data file missing (python -m paper_2403_04267_gb300.surrogate generate)"}
    D = np.load(path)
    ok_tr = D["train_status"] == 0
    ok_ho = D["heldout_status"] == 0
    X, T = D["train_X"][ok_tr], D["train_T"][ok_tr]
    nv = max(len(X) // 10, 16)
    Xf, Tf, Xv, Tv = X[:-nv], T[:-nv], X[-nv:], T[-nv:]
    Xh, Th = D["heldout_X"][ok_ho], D["heldout_T"][ok_ho]
    seeds_h = D["heldout_seeds"][ok_ho]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ens = S.Ensemble(Xf, Tf, members=args.sur_members, steps=args.sur_steps)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    tau = S.calibrate_gate(ens, Xv, Tv, target=args.sur_gate_target)
    # the solver's cost per held-out run: plain FP64, one run at a time, to 20 s, timed on
    # the first draws that it completes (a failed run stops early and is not a run's cost;
    # at most four times as many draws are tried)
    t_sol, nsol, nfail, errs = 0.0, 0, 0, []
    for k in range(min(4 * args.sur_solver_runs, len(seeds_h))):
        if nsol == args.sur_solver_runs:
            break
        sp = W.batched_run(W.batched_draw(int(seeds_h[k])), int(D["heldout_n"]))
        ref = salec.Sim(sp, precision="fp64")
        ref.set_end_time(20.0)
        one = salec.Batch([ref])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        one.run(chunk=50, max_steps=400000)
        torch.cuda.synchronize()
        dt_run = time.perf_counter() - t1
        if ref.scalars()["status"] != 0:
            nfail += 1
        else:
            t_sol += dt_run
            nsol += 1
            c = ref.crater(sp["z_surface"], 64)
            errs.append(abs(c["diameter"] / (1000.0 * float(Th[k, S.N_PROFILE + 1])) - 1.0))
        del one, ref
    fwd = 2.0 * sum(a * b for a, b in zip(S.DIMS[:-1], S.DIMS[1:]))        # flops per sample
    out = {"train_draws": int(ok_tr.sum()), "heldout_draws": int(ok_ho.sum()),
           "failed_runs_excluded": int((~ok_tr).sum() + (~ok_ho).sum()),
           "members": args.sur_members, "train_steps": args.sur_steps, "train_s": round(t_train, 2),
           # the whole ensemble's training (groups of two members, each group's step one set of
           # launches, groups on their own streams, 25-step graph replays; wall time including
           # set-up): forward + backward = 3 forward passes per sample and step
           "train_tflops_ensemble": round(3.0 * fwd * len(Xf) * args.sur_members * args.sur_steps / t_train / 1e12, 2),
           "fp64_solver_runs": nsol, "fp64_solver_failed": nfail}
    if nsol:
        rep = S.gain_report(ens, tau, Xh, Th, t_sol / nsol)
        out.update(rep)
        # the same with the batched FP32-mix solver as the fallback, at the cost per run it
        # had when it generated the training data (batches of 1024 runs of 400 x 400 to 20 s)
        s_batch = float(D["train_wall_s"]) / len(D["train_status"])
        rb = S.gain_report(ens, tau, Xh, Th, s_batch)
        out["batched_fallback"] = {"solver_s_per_run": s_batch, "runs_per_hour_solver": rb["runs_per_hour_solver"],
                                   "runs_per_hour_with_surrogate": rb["runs_per_hour_with_surrogate"]}
        # the gate's trade-off: stricter validation targets accept fewer draws, more accurately
        sweep = []
        for target in (0.9, 0.95, 0.96, 0.97, 0.99):
            tt = S.calibrate_gate(ens, Xv, Tv, target=target)
            r1 = S.gain_report(ens, tt, Xh, Th, t_sol / nsol)
            r2 = S.gain_report(ens, tt, Xh, Th, s_batch)
            sweep.append({"target": target, "accepted": r1["accepted"], "accepted_within_tol": r1["accepted_within_tol"],
                          "runs_per_hour_fp64_fallback": r1["runs_per_hour_with_surrogate"],
                          "runs_per_hour_batched_fallback": r2["runs_per_hour_with_surrogate"]})
        out["gate_sweep"] = sweep
        out["fp64_vs_dataset_diameter_err_max"] = max(errs)
    # tensor throughput: one training step at the full training batch, and inference on
    # a large batch of draws
    net = ens.nets[0]
    Xd = torch.from_numpy(np.ascontiguousarray(Xf, dtype=np.float32)).cuda()
    Td = torch.from_numpy(np.ascontiguousarray(Tf, dtype=np.float32)).cuda()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()                 # the inputs, before the network's stream reads them
    for _ in range(3):
        net.train_step(Xd, Td, 0.0)
    ev0.record(net.stream)                   # the events on the stream the steps run on
    for _ in range(20):
        net.train_step(Xd, Td, 0.0)
    ev1.record(net.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / 20
    out["train_step_ms"] = ms
    out["train_tflops_single_step"] = 3.0 * fwd * len(Xf) / (ms * 1e-3) / 1e12
    big = S.MLP(args.sur_infer_batch)
    big.set_params(net.get_params())
    Xb = torch.rand((args.sur_infer_batch, S.N_IN), device="cuda") * 2 - 1
    Yb = torch.empty((args.sur_infer_batch, S.N_OUT), device="cuda")
    for _ in range(3):
        big.forward(Xb, Yb)
    ev0.record()
    for _ in range(10):
        big.forward(Xb, Yb)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / 10
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak = float(json.load(fh)["bf16_tflops"])
    except Exception:
        peak = 1900.0
    ach = fwd * args.sur_infer_batch / (ms * 1e-3) / 1e12
    out["inference"] = {"batch": args.sur_infer_batch, "ms": ms, "draws_per_s": args.sur_infer_batch / (ms * 1e-3)}
    out["roofline"] = {"bound": "tensor", "kernel": "k_mlp_forward_pp", "unit": "TFLOP/s", "achieved": ach,
                       "peak": peak, "peak_kind": "measured bf16 burst", "frac": ach / peak,
                       "note": "whole forward pass (input conversion + the five layers in one kernel) at the inference batch"}
    big.check()
    net.check()
    return out


def _layered(args):
    """The paper's verification run set-up (Sect. 4, Tables 1-2): its grid -- a 462 x 462
    zone of 400 m cells, 20 extension cells growing by 1.05 to 1061 m on the right, bottom
    and top, 30 PML cells outside (512 x 532 cells) -- and its target, sediment / crust /
    mantle in hydrostatic equilibrium under Earth gravity with Table 1 strength, hit by a
    14.4 km dunite projectile.  Device-timed steps from the start of the impact in both
    precisions (the state fits in L2 at this size)."""
    import torch
    from paper_2403_04267_gb300 import salec, workloads as W
    spec = W.chicxulub_stretched()
    cells = spec["grid"]["nr"] * spec["grid"]["nz"]
    out = {"workload": spec["name"], "cells": cells, "steps": args.layered_steps, "l2": "state fits in L2"}
    for prec in ("fp64", "fp32mix"):
        sim = salec.Sim(spec, precision=prec)
        sim.step(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(args.layered_steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        sc = sim.scalars()
        cr = sim.crater(spec["z_surface"], 64)
        out[prec] = {"value": cells * args.layered_steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.layered_steps,
                     "sim_time_s": sc["t"], "status": sc["status"], "crater_depth_m": cr["depth"],
                     "crater_diameter_m": cr["diameter"], "gpu_launches": sim.launches_per_step() * args.layered_steps}
        del sim
        torch.cuda.empty_cache()
    return out


def peak_decay(pmax, rc, zc, z_surface, bin_width, nbins):
    """Peak over-pressure against distance from the impact point (on the axis at the
    surface), Sect. 4 of the paper: the largest recorded over-pressure of the cells in each
    distance bin of width bin_width."""
    import numpy as np
    dist = np.hypot(np.asarray(rc)[None, :], np.asarray(zc)[:, None] - z_surface)
    k = np.minimum((dist / bin_width).astype(np.int64), nbins)
    out = np.zeros(nbins + 1)
    np.maximum.at(out, k.ravel(), np.asarray(pmax).ravel())
    return out[:nbins]


def decay_errors(p32, p64, floor=0.01):
    """Relative errors of a peak-pressure decay curve against the FP64 one, over the bins
    whose FP64 peak is at least `floor` of the largest."""
    import numpy as np
    p32, p64 = np.asarray(p32), np.asarray(p64)
    sel = p64 >= floor * p64.max()
    e = np.abs(p32[sel] / p64[sel] - 1.0)
    return {"bins": int(sel.sum()), "max": float(e.max()) if e.size else None, "mean": float(e.mean()) if e.size else None}


def _fp32_accuracy(args):
    """The mixed form's error against FP64 on the 4000 x 4000 physics (basalt, hydrodynamic,
    10 m cells, 10 km/s) at 400 x 400 with a 10-cell projectile, run until a crater has
    formed (t = 0.6 s, the simulated time of the large run's 2000 steps, and t = 2 s): crater
    depth and diameter, and the peak-pressure decay with distance.  The FP64 GPU solver,
    which matches the FP64 oracle to 1e-9, stands in for the oracle."""
    import numpy as np
    from paper_2403_04267_gb300 import salec, workloads as W
    spec = W.scaled_plain(400, radius_cells=10)
    g = spec["grid"]
    rc = (np.arange(g["nr"]) + 0.5) * g["dx"]
    zc = (np.arange(g["nz"]) + 0.5) * g["dx"]
    sims = {p: salec.Sim(spec, precision=p) for p in ("fp64", "fp32mix")}
    out = {"workload": "4000x4000 physics at 400x400, projectile radius 10 cells", "reference": "FP64 GPU solver",
           "fp32_form": sims["fp32mix"].step_form}
    for t_end in (0.6, 2.0):
        res = {}
        for p, sim in sims.items():
            while sim.scalars()["t"] < t_end and sim.scalars()["status"] == 0:
                sim.step(10)
            sc = sim.scalars()
            res[p] = (sim.crater(spec["z_surface"], 64), peak_decay(sim.get("pmax"), rc, zc, spec["z_surface"], g["dx"], 300), sc)
        c32, c64 = res["fp32mix"][0], res["fp64"][0]
        out[f"t={t_end}s"] = {
            "t_fp64": res["fp64"][2]["t"], "t_fp32mix": res["fp32mix"][2]["t"],
            "status": [res["fp64"][2]["status"], res["fp32mix"][2]["status"]],
            "depth_m": [c32["depth"], c64["depth"]], "diameter_m": [c32["diameter"], c64["diameter"]],
            "depth_rel_err": abs(c32["depth"] / c64["depth"] - 1) if c64["depth"] else None,
            "diameter_rel_err": abs(c32["diameter"] / c64["diameter"] - 1) if c64["diameter"] else None,
            "peak_pressure_decay_rel_err": decay_errors(res["fp32mix"][1], res["fp64"][1])}
    del sims
    return out


def _active(args, hbm_peak):
    """Throughput on a grid most of which moves: the 4000 x 4000 physics at 1600 x 1600
    (state above L2 in both forms) with a 200-cell projectile, advanced 3000 steps before
    the timed ones (the large run's first steps time an almost resting grid).  Both
    precisions, each in its default step form; the fraction of moving vertices is stated."""
    import numpy as np
    import torch
    from paper_2403_04267_gb300 import salec, workloads as W
    spec = W.scaled_plain(1600, radius_cells=200)
    cells = spec["grid"]["nr"] * spec["grid"]["nz"]
    out = {"workload": "4000x4000 physics at 1600x1600, projectile radius 200 cells, after 3000 steps",
           "cells": cells, "steps": args.active_steps}
    for prec in ("fp64", "fp32mix"):
        sim = salec.Sim(spec, precision=prec)
        sim.step(3000)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(args.active_steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.active_steps
        sc = sim.scalars()
        moving = float((np.hypot(sim.get("vr"), sim.get("vz")) > 1.0).mean())
        r = {"form": sim.step_form, "value": cells / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "sim_time_s": sc["t"],
             "status": sc["status"], "moving_vertex_fraction": round(moving, 3)}
        if sim.step_form == "fused":
            q, t = sim.fused_queue()
            r["tiles_queued_last_step"] = [q, t]
        if prec == "fp32mix":
            gbs = step_bytes_per_cell(4) * cells / (ms * 1e-3) / 1e9
            r["step_hbm"] = {"achieved_gbs": round(gbs, 1), "peak_gbs": hbm_peak, "frac": round(gbs / hbm_peak, 4),
                             "bytes_per_cell": step_bytes_per_cell(4)}
        out[prec] = r
        del sim
        torch.cuda.empty_cache()
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2403_04267_gb300 import workloads as W
    spec = _workload(args.workload)
    # each reference step: one oracle step of the same physics on a bounded window so the
    # whole --steps/--warmup run stays within minutes (per-step budget ~0.06 s)
    n = 400
    sample = W.scaled_plain(n, radius_cells=10) if args.workload == "large_4000" else spec
    s = O.OracleSim(sample)
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    cells = sample["grid"]["nr"] * sample["grid"]["nz"]
    value = cells * args.steps / dt
    desc = (f"serial FP64 oracle, {args.steps} steps of the same physics on a {sample['grid']['nr']}x"
            f"{sample['grid']['nz']} grid per step (bounded sample of the {args.workload} workload)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_4000", choices=["large_4000", "full_800", "plain_100", "plain_2000"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "fp32mix"])
    ap.add_argument("--form", default="default", choices=["default", "phases", "fused"],
                    help="step form of the timed runs (default: the library's choice)")
    ap.add_argument("--rest-copy", type=int, default=None, choices=[0, 1, 2],
                    help="fused form: how the tiles at rest are copied (salec_set_rest_copy; "
                         "default: the library's choice)")
    ap.add_argument("--batch-runs", type=int, default=256)
    ap.add_argument("--batch-t-end", type=float, default=20.0)
    ap.add_argument("--batch-ref-runs", type=int, default=16)
    ap.add_argument("--batch-max-s", type=float, default=900.0)
    ap.add_argument("--batch-ref-max-s", type=float, default=300.0)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-layered", action="store_true")
    ap.add_argument("--layered-steps", type=int, default=1000)
    ap.add_argument("--active-steps", type=int, default=100)
    ap.add_argument("--no-active", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--sur-members", type=int, default=8)
    ap.add_argument("--sur-steps", type=int, default=12000)
    ap.add_argument("--sur-solver-runs", type=int, default=8)
    ap.add_argument("--sur-infer-batch", type=int, default=65536)
    ap.add_argument("--sur-gate-target", type=float, default=0.97)
    ap.add_argument("--mlp-step-probe", type=int, nargs=2, metavar=("BATCH", "STEPS"), default=None,
                    help="only time one surrogate network's training steps (salec_mlp_train_step) at BATCH random "
                         "samples: STEPS untimed, then STEPS timed; one JSON line (a profiling aid)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.mlp_step_probe:
        return _mlp_step_probe(*args.mlp_step_probe)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2403_04267_gb300 import salec

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    spec = _workload(args.workload)
    cells = spec["grid"]["nr"] * spec["grid"]["nz"]

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def measure(precision, with_e2e, form=None):
        """Device-timed K steps that continue the run after its W warm-up steps (steps W + 1
        to W + K of the workload), with live per-kernel events; then optionally K steps from
        t = 0 end to end through the C ABI (initial state copied from the host)."""
        sim = salec.Sim(spec, precision=precision)
        form = form or (None if args.form == "default" else args.form)
        if form:
            sim.step_form = form
        if args.rest_copy is not None:
            sim.set_rest_copy(args.rest_copy)
        stream = sim.stream
        nbytes = sim.checkpoint_bytes()
        init = sim.state[:nbytes].clone()          # device copy of the initial state

        def restore():
            sim.state[:nbytes].copy_(init)
            torch.cuda.synchronize()
            sim.state_changed()

        sim.step(args.warmup)
        torch.cuda.synchronize()
        snap = sim.get_state() if sim.step_form == "fused" else None    # host copy of the timed steps' start
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sim.set_kernel_timing(True)
        barrier()
        with ClockSampler(local) as clk:
            e0.record(stream)
            sim.step(args.steps)
            e1.record(stream)
            barrier()
        ms = e0.elapsed_time(e1)
        ktimes, _ = sim.kernel_times()
        sim.set_kernel_timing(False)
        sc = sim.scalars()
        queue = None
        if sim.step_form == "fused":
            # the same K steps again, untimed, one call each: how many tiles each step ran
            # through the whole cycle (the others the rest-tile kernel copied)
            sim.set_state(snap)
            qs = []
            for _ in range(args.steps):
                sim.step(1)
                qs.append(sim.fused_queue()[0])
            tiles = sim.fused_queue()[1]
            queue = {"tiles": tiles, "queued_mean": float(np.mean(qs)), "queued_first": qs[0], "queued_last": qs[-1],
                     "note": "steps W + 1 .. W + K; the replay restarts from a host copy, so its first step "
                             "follows a Courant-rate pass"}
        ms_max = ms
        if ws > 1:
            t = torch.tensor([ms], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_max = float(t.item())
        out = {"value": ws * cells * args.steps / (ms_max * 1e-3), "ms": ms, "ms_max": ms_max, "ktimes": ktimes,
               "scalars": sc, "clocks": clk.summary(),
               "launches": sim.launches_per_step() * args.steps,
               "form": sim.step_form, "pmax": sim.get("pmax"), "queue": queue}
        if with_e2e:
            host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
            host.copy_(init.cpu())
            p_host = np.zeros((spec["grid"]["nz"], spec["grid"]["nr"]))
            restore()
            barrier()
            t0 = time.perf_counter()
            sim.set_state(host.numpy())
            for _ in range(args.steps):
                sim.step(1)
                sim.scalars()
            p_host[:] = sim.get("p")
            torch.cuda.synchronize()
            t_e2e = time.perf_counter() - t0
            if ws > 1:
                t = torch.tensor([t_e2e], device="cuda", dtype=torch.float64)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                t_e2e = float(t.item())
            out["e2e"] = {"value": ws * cells * args.steps / t_e2e, "unit": UNIT,
                          "h2d_bytes_per_step": nbytes / args.steps,
                          "d2h_bytes_per_step": 64 + p_host.nbytes / args.steps,
                          "note": "initial state H2D once from pinned memory (amortised over the steps), "
                                  "per-step scalar read-back, final pressure field D2H"}
        del sim, init
        torch.cuda.empty_cache()
        return out

    hbm_peak, peak_kind = _load_peaks()

    def roofline(res, e, dom=None):
        kt = res["ktimes"]
        dom = dom or max(kt, key=kt.get)
        kb = kernel_bytes_per_cell(e)
        # cells one launch processes: every cell for a phase kernel; in the fused form the
        # cells of the tiles at rest (rest-tile kernel) or of the queued tiles (tile kernel),
        # averaged over the K steps
        units = float(cells)
        q = res.get("queue")
        if q:
            qf = q["queued_mean"] / q["tiles"]
            units = cells * (1.0 - qf if dom in REST_KERNELS else qf)
        gbs = kb[dom] * units / (kt[dom] * 1e-3) / 1e9
        roof = {"kernel": dom, "hbm": {"achieved_gbs": round(gbs, 1), "peak_gbs": hbm_peak, "peak_kind": peak_kind,
                                       "frac": round(gbs / hbm_peak, 4), "bytes_per_cell": kb[dom],
                                       "cells_per_launch": round(units)}}
        return roof, dom

    res64 = measure("fp64", not args.no_e2e) if args.precision in ("both", "fp64") else None
    # the FP64 form's other step form beside the library's choice
    res64o = measure("fp64", False, "phases" if res64["form"] == "fused" else "fused") \
        if res64 is not None and args.form == "default" else None
    res32 = measure("fp32mix", not args.no_e2e and args.precision == "fp32mix") if args.precision in ("both", "fp32mix") else None
    # the mixed form's other step form beside the library's choice
    res32f = measure("fp32mix", False, "phases" if res32 is not None and res32["form"] == "fused" else "fused") \
        if args.precision == "both" and args.form == "default" else None
    if rank != 0:
        dist.destroy_process_group()
        return 0

    main_res = res64 if res64 is not None else res32
    e_main = 8 if res64 is not None else 4
    prec_main = "fp64" if res64 is not None else "fp32mix"
    roof_hbm, dom = roofline(main_res, e_main)

    def hbm_roof(r, d, prec):
        h = r["hbm"]
        tr, trk = _traffic(d, prec, args)
        return {"bound": "hbm", "kernel": d, "unit": "GB/s", "achieved": h["achieved_gbs"], "peak": hbm_peak,
                "frac": h["frac"], "peak_kind": peak_kind, "bytes_per_cell": h["bytes_per_cell"],
                "cells_per_launch": h["cells_per_launch"], "traffic": tr, "traffic_kind": trk}

    fp64_alu = None
    if res64 is not None:
        clk = main_res["clocks"].get("sm_max_mhz") or _sm_max_mhz()
        sms, fp64_nominal, fp64_gemm = fp64_peaks(clk)

        def alu_roof(d):
            kt = main_res["ktimes"][d]
            if d in _FUSED_FULL_SIZE.get("fp64", {}) and d not in _COUNTERS_STALE["fp64"] and \
                    _FUSED_FULL_SIZE["fp64"][d].get("flops"):
                full = _FUSED_FULL_SIZE["fp64"][d] if (args.workload, args.steps, args.warmup) == _FULL_SIZE_CASE else {}
                flops = full.get("flops")
                ach = flops / (kt * 1e-3) / 1e12 if flops else None
                per = {"flops_per_launch": flops, "flops_kind": "ncu FP64 instruction counts of the same 20 launches "
                       "(large_4000, after 5 warm-up steps), mean per launch" if flops else "not captured for this workload / K / W"}
            else:
                stale = d in _COUNTERS_STALE["fp64"]
                flops = None if stale else _FLOPS_PER_CELL.get(d)
                ach = flops * cells / (kt * 1e-3) / 1e12 if flops else None
                per = {"flops_per_cell": flops, "counters_stale": stale}
            tr, trk = _traffic(d, "fp64", args, "k_rest_copy" in main_res["ktimes"])
            return {"bound": "alu", "kernel": d, "unit": "TFLOP/s", "peak": round(fp64_gemm, 4),
                    "peak_kind": "measured FP64 GEMM (cuBLAS, 4096^3) on this GPU",
                    "peak_nominal": round(fp64_nominal, 4),
                    "peak_nominal_kind": f"{sms} SMs (device) x {DFMA_PER_CLK_PER_SM} DFMA/clk x 2 flop x {clk:.0f} MHz",
                    "achieved": round(ach, 4) if ach else None, "frac": round(ach / fp64_gemm, 4) if ach else None,
                    "frac_of_nominal": round(ach / fp64_nominal, 4) if ach else None, **per,
                    "traffic": tr, "traffic_kind": trk, "fp64_pipe_busy": _FP64_PIPE_BUSY.get(d),
                    "note": "flops count 2 per DFMA and 1 per DADD/DMUL; the FP64 pipe issues every FP64 "
                            "instruction at the DFMA rate, and fp64_pipe_busy (ncu, 2000x2000) is its occupancy"}

        rest_k = next((k for k in REST_KERNELS if k in main_res["ktimes"]), None)
        if dom in REST_KERNELS:
            # the tiles at rest dominate: a copy of the state, held to HBM
            roof = hbm_roof(roof_hbm, dom, "fp64")
            if "k_step_fused" in main_res["ktimes"]:
                fp64_alu = alu_roof("k_step_fused")
        else:
            roof = alu_roof(dom)
            roof["hbm"] = roof_hbm["hbm"]
        if rest_k is not None and dom != rest_k:
            rr, _ = roofline(main_res, e_main, rest_k)
            line_rest = hbm_roof(rr, rest_k, "fp64")
        else:
            line_rest = None
    else:
        roof = hbm_roof(roof_hbm, dom, "fp32mix")
        line_rest = None
    ms = main_res["ms"]
    sc = main_res["scalars"]
    line = {
        "metric": METRIC, "value": main_res["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_res["ms_max"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if res64 is not None else "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload + " " + spec["name"], "grid": f"{spec['grid']['nr']}x{spec['grid']['nz']}",
                   "cells": cells, "precision": "FP64" if res64 is not None else "FP32-mix",
                   "l2": "state > L2 (no flush)", "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "sim_time_s": sc["t"], "status": sc["status"]},
        "gpu_launches": main_res["launches"],
        "kernel_ms": {k: round(v, 4) for k, v in main_res["ktimes"].items()},
        "step_hbm_frac": round(step_bytes_per_cell(e_main) * cells / (ms / args.steps * 1e-3) / 1e9 / hbm_peak, 4),
        "roofline": roof, "clocks": main_res["clocks"], "e2e": main_res.get("e2e"), "step_form": main_res["form"],
    }
    if fp64_alu is not None:
        line["roofline_fp64_pipe"] = fp64_alu
    if line_rest is not None:
        line["roofline_rest_tiles"] = line_rest
    if main_res.get("queue"):
        line["fused_queue"] = main_res["queue"]
    if res64o is not None:
        line["other_form"] = {"form": res64o["form"], "value": res64o["value"], "unit": UNIT,
                              "ms_per_step": res64o["ms_max"] / args.steps,
                              "kernel_ms": {k: round(v, 4) for k, v in res64o["ktimes"].items()},
                              "gpu_launches": res64o["launches"], "status": res64o["scalars"]["status"]}
    if res64 is not None and res32 is not None:
        r32, d32 = roofline(res32, 4)
        # the peak-pressure decay of the two forms over the same K steps (Sect. 4)
        g = spec["grid"]
        rc = (np.arange(g["nr"]) + 0.5) * g["dx"]
        zc = (np.arange(g["nz"]) + 0.5) * g["dx"]
        dec = decay_errors(peak_decay(res32["pmax"], rc, zc, spec["z_surface"], g["dx"], 400),
                           peak_decay(res64["pmax"], rc, zc, spec["z_surface"], g["dx"], 400))
        line["fp32_mix"] = {
            "value": res32["value"], "unit": UNIT, "ms_per_step": res32["ms_max"] / args.steps,
            "speedup_vs_fp64": res32["value"] / res64["value"], "step_form": res32["form"],
            "kernel_ms": {k: round(v, 4) for k, v in res32["ktimes"].items()},
            "roofline": hbm_roof(r32, d32, "fp32mix"), "fused_queue": res32.get("queue"),
            "step_hbm_frac": round(step_bytes_per_cell(4) * cells / (res32["ms"] / args.steps * 1e-3) / 1e9 / hbm_peak, 4),
            "peak_pressure_decay_vs_fp64_same_steps": dec,
            "gpu_launches": res32["launches"], "clocks": res32["clocks"], "status": res32["scalars"]["status"]}
        if res32f is not None:
            rf, df = roofline(res32f, 4)
            line["fp32_mix"]["other_form"] = {"form": res32f["form"],
                "value": res32f["value"], "unit": UNIT, "ms_per_step": res32f["ms_max"] / args.steps,
                "kernel_ms": {k: round(v, 4) for k, v in res32f["ktimes"].items()},
                "roofline": hbm_roof(rf, df, "fp32mix"),
                "step_hbm_frac": round(step_bytes_per_cell(4) * cells / (res32f["ms"] / args.steps * 1e-3) / 1e9 / hbm_peak, 4),
                "gpu_launches": res32f["launches"], "status": res32f["scalars"]["status"]}
        if not args.no_accuracy and ws == 1:
            line["fp32_mix"]["accuracy"] = _fp32_accuracy(args)
    if not args.no_active and ws == 1:
        line["active_grid"] = _active(args, hbm_peak)
    if not args.no_layered and ws == 1:
        line["layered"] = _layered(args)
    if not args.no_batch and args.batch_runs > 0:
        line["batched"] = _batched(args, rank, ws)
        if ws == 1:
            line["batched"]["launch_forms"] = _batch_modes(args)
    if not args.no_surrogate and ws == 1:
        line["surrogate"] = _surrogate(args)
    if ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = _cpu_baseline(spec, args.cpu_steps)
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


# FP64 operations per cell (2 DFMA + DADD + DMUL) issued by each phase kernel of the FP64
# form, and DRAM bytes per cell of each phase kernel, from ncu (one kernel, one launch: the
# first timed step of the 4000 x 4000 physics at 2000 x 2000, radius 50 cells; profiles/).
_FLOPS_PER_CELL: dict = {"k_phase0": 85.1, "k_phase1": 37.7, "k_phase2": 27.4, "k_phase3a": 51.4, "k_phase3b": 50.1, "k_phase3c": 4.8}
_TRAFFIC_PER_CELL: dict = {"k_phase0": 57.7, "k_phase1": 72.2, "k_phase2": 75.3, "k_phase3a": 78.5, "k_phase3b": 62.8, "k_phase3c": 22.1}
_TRAFFIC_PER_CELL_FP32MIX: dict = {"k_phase0": 27.7, "k_phase1": 30.8, "k_phase2": 40.1, "k_phase3a": 42.3, "k_phase3b": 29.6, "k_phase3c": 10.8}
# fraction of the FP64 pipe's issue slots each FP64-form kernel keeps busy (ncu,
# sm__pipe_fp64_cycles_active, 2000 x 2000, the fused kernels at the second timed step)
_FP64_PIPE_BUSY: dict = {"k_phase0": 0.847, "k_phase1": 0.847, "k_phase2": 0.845, "k_phase3a": 0.847, "k_phase3b": 0.841,
                         "k_phase3c": 0.783, "k_step_fused": 0.735, "k_rest_tiles": 0.180}
# The fused form's two kernels on the headline workload (4000 x 4000, K = 20 timed steps after
# W = 5 warm-up steps): DRAM read + write bytes and FP64 operations per launch, the mean over
# the 20 launches of the timed region from one-pass ncu captures of the same command
# (profiles/).  The rest flags make these launches depend on the step sequence, so they hold
# for that case only.
_FULL_SIZE_CASE = ("large_4000", 20, 5)
_FUSED_FULL_SIZE: dict = {
    "fp64": {"k_rest_tiles": {"traffic": 1.43016e9}, "k_step_fused": {"traffic": 4.2122e7, "flops": 1.14608e8}},
    "fp32mix": {"k_rest_tiles": {"traffic": 8.0653e8}, "k_step_fused": {"traffic": 2.6158e7}},
}
# kernels changed since their counters were taken: neither DRAM traffic nor flop rates are
# reported for them until the next capture
_COUNTERS_STALE: dict = {"fp64": set(), "fp32mix": set()}
# Beside the copy kernel (salec_set_rest_copy mode 2) the FP64 tile kernel is another
# instantiation (120 registers, the same arithmetic) sharing the SMs with the copies: its
# FP64 operation count carries over, the DRAM traffic of the capture above does not.


def _traffic(kernel: str, prec: str, args, beside: bool = False):
    """DRAM bytes per launch of a kernel from ncu, and what they were measured on; None
    where no capture applies (beside: the step copied its tiles at rest beside the tile
    kernel)."""
    if kernel in _COUNTERS_STALE[prec]:
        return None, "counters stale"
    if beside and kernel == "k_step_fused":
        return None, "runs beside the copy kernel: not captured"
    if kernel in _FUSED_FULL_SIZE[prec]:
        if (args.workload, args.steps, args.warmup) != _FULL_SIZE_CASE:
            return None, "not captured for this workload / K"
        return _FUSED_FULL_SIZE[prec][kernel]["traffic"], "ncu, the same 20 launches, mean per launch"
    table = _TRAFFIC_PER_CELL if prec == "fp64" else _TRAFFIC_PER_CELL_FP32MIX
    if kernel not in table:
        return None, "no capture"
    g = _workload(args.workload)["grid"]
    return table[kernel] * g["nr"] * g["nz"], "ncu bytes per cell (one launch, 2000x2000) x the cells"


if __name__ == "__main__":
    sys.exit(main())
