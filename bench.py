#!/usr/bin/env python3
"""Benchmark of the FDTD-Bath hot path: cell-updates/s and fraction of HBM roofline.

Workload (default): the 3D slab cavity, 256^3 cells, periodic x/y, 16-cell CPML in z,
8-cell Drude mirrors around a 64-plane Lorentz-Bath layer with N_b = 8, Ex plane source
with a seeded transverse phase, one flux monitor (256 DFT frequencies) and the energy
box -- FP32 state and arithmetic (the FP64 path is measured beside it).  One "step" is
one full FDTD-Bath time step of the whole grid (fields, CPML, source, Lorentz/Drude/
Lorentz-Bath ADE with the bath modes, DFT and energy partial sums).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the only other place this file runs
``oracle/``) on the same workload, one oracle step of the full grid per timed step.
Under torchrun (N > 1) every rank advances its own replica (weak scaling) and rank 0
prints the JSON line; the reference arm runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2505_23963_gb300 import workloads as wl  # noqa: E402

METRIC = "Lorentz-Bath FDTD cell-updates/s (3D slab cavity 256^3, N_b=8)"
UNIT = "cell-updates/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(prob: dict, esz: int, bath_bytes: float | None = None,
                      sigma_map: bool = False) -> float:
    """Bytes per launch with every state word read once and written once: E, H (6 words
    per cell), +4 CPML memories in the absorber planes, +3 x (2 reads + 1 write) of P in
    Drude/Lorentz planes and additionally +3 x 3 N_b words for the bath modes (two levels
    read, one written) in Lorentz-Bath planes.  Coefficient tables are not counted.
    bath_bytes overrides the bytes per bath mode and component (bf16 value/increment pairs
    read and written: 8); sigma_map adds the read of a per-cell sigma(r) in every Drude,
    Lorentz and Lorentz-Bath cell."""
    nx, ny, nz = prob["n"]
    pml = prob.get("pml", 0)
    words = np.full(nz, 12.0)
    words[:pml] += 8
    words[nz - pml:] += 8
    for m in prob["materials"]:
        lo, hi = m["z"]
        if m["kind"] in ("lorentz", "drude"):
            words[lo:hi] += 9
        elif m["kind"] == "lorentz_bath":
            nb = len(m["bath_frequencies"])
            words[lo:hi] += 9 + (9 * nb if bath_bytes is None else 3 * nb * bath_bytes / esz)
        if sigma_map and m["kind"] != "vacuum":
            words[lo:hi] += 1
    return float(words.sum()) * nx * ny * esz


def algorithmic_bytes_te(prob: dict, esz: int = 4) -> dict:
    """Bytes per step of the differentiation form's y-invariant TE grid (E_y, H_x, H_z, the y
    polarization and bath modes), every word once per kernel that touches it:
      forward: E_y, H_x, H_z read and written (6 words per cell), +2 x 2 CPML memories in the
      absorber planes, +3 words of P_y (two levels read, one written) in Drude / Lorentz planes,
      +3 + 3 N_b in Lorentz-Bath planes;
      record (reverse sweep, recomputed forward steps): the differentiated layer's E_y, P_y of two
      levels and two levels of its bath modes written, 3 + 2 N_b words per layer cell;
      adjoint (adjoint_k1 + adjoint_k2): H_bar_x, H_bar_z read and E_bar_y read and written in k1,
      E_bar_y read and H_bar_x, H_bar_z read and written in k2 (9 words per cell), +5 in the
      absorber planes (the CPML adjoints), +4 P-adjoint words in Drude / Lorentz planes, in the
      differentiated Lorentz-Bath layer also 4 N_b bath-adjoint words and the 3 + 2 N_b recorded
      values read."""
    nx, ny, nz = prob["n"]
    pml = prob.get("pml", 0)
    fwd = np.full(nz, 6.0)
    adj = np.full(nz, 9.0)
    fwd[:pml] += 4
    fwd[nz - pml:] += 4
    adj[:pml] += 5
    adj[nz - pml:] += 5
    rec = 0.0
    for m in prob["materials"]:
        lo, hi = m["z"]
        nb = len(m.get("bath_frequencies", ()))
        if m["kind"] in ("lorentz", "drude"):
            fwd[lo:hi] += 3
            adj[lo:hi] += 4
        elif m["kind"] == "lorentz_bath":
            fwd[lo:hi] += 3 + 3 * nb
            adj[lo:hi] += 4 + 4 * nb + 3 + 2 * nb
            rec += (3 + 2 * nb) * (hi - lo)
    w = float(nx * ny * esz)
    return {"forward": float(fwd.sum()) * w, "record": rec * w, "adjoint": float(adj.sum()) * w}


def algorithmic_flops_fp64(prob: dict, instructions: bool = False) -> float:
    """Floating-point operations per step of the FP64 path, which evaluates the literal updates
    (Eq. FDTD-1D with Eq. 1a,b in 3D, Eq. Pz_1D_Lorentz / Pz_update-LB, Eq. Yzj_finite_difference),
    one operation per multiply or add, counted per cell from those expressions: the H update 15 (six differences, three scaled subtractions), the E update 15
    (six differences, three curl subtractions, three scaled additions), +8 per CPML memory pair
    on each side; Drude / Lorentz planes +8 per component (D, E = (D - P)/eps, P update); a
    Lorentz-Bath plane with N_b modes 51 N_b + 112 (per component 5 N_b for the bath sum, 12 N_b
    for the mode updates and their energy, 27 for D, E, P and the P energy), energy-box planes
    +7 for the field energy.
    instructions=True counts FP64 instructions instead: the bath recursion runs with fused
    multiply-adds (per mode and component the bath sum's 5 operations in 3 instructions, the mode
    update and its energy term's 12 in 8), everything else uncontracted, one instruction per
    operation: 33 N_b + 112 per Lorentz-Bath cell."""
    nx, ny, nz = prob["n"]
    pml = prob.get("pml", 0)
    f = np.full(nz, 30.0)
    f[:pml] += 16
    f[nz - pml:] += 16
    lo_b, hi_b = prob.get("energy_box", (0, 0))
    for m in prob["materials"]:
        lo, hi = m["z"]
        if m["kind"] in ("lorentz", "drude"):
            f[lo:hi] += 24
        elif m["kind"] == "lorentz_bath":
            f[lo:hi] = (33 if instructions else 51) * len(m["bath_frequencies"]) + 112
    f[lo_b:hi_b] += 7
    return float(f.sum()) * nx * ny


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int = 0):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def spectrum_is_finite(fb, sim) -> bool:
    """Whether the run's spectra are finite (the library reports NaN / Inf as an error code)."""
    try:
        sim.dft(0)
    except fb.FdtdBathError as e:
        if e.code != fb.ERR_NONFINITE:
            raise
        return False
    return True


def max_over_ranks(x: float, device=None) -> float:
    """The largest of the ranks' values of x (the slowest replica sets the job's time); x itself
    without a process group.  The reduction runs on the rank's GPU under NCCL, on the host under
    gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: float, world_size: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas: the units every rank processed over the
    slowest rank's time."""
    return world_size * units_per_rank / seconds


def oracle_sample(prob: dict, ny_sample: int) -> dict:
    """A bounded sample of the workload for the CPU oracle: the full x and z extent (every
    plane type in its true proportion) over the first ny_sample rows of y."""
    nx, ny, nz = prob["n"]
    smp = dict(prob, n=(nx, ny_sample, nz))
    smp["sources"] = [dict(s, phase=None if s.get("phase") is None else s["phase"][:ny_sample])
                      for s in prob["sources"]]
    return smp


def oracle_rate(prob: dict, min_seconds: float = 10.0, max_steps: int = 4000, ny_sample: int = 16):
    """Cell-updates/s of the FP64 CPU oracle on a bounded sample (see oracle_sample)."""
    from oracle import oracle as O
    smp = oracle_sample(prob, ny_sample)
    sim = O.OracleSim(smp)
    sim.step(1)                       # first touch of the arrays, untimed
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and (time.perf_counter() - t0) < min_seconds:
        sim.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    sim.close()
    nx, ny, nz = smp["n"]
    return nx * ny * nz * steps / dt, dt, steps, smp


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    prob = wl.slab_3d(steps=args.steps)
    smp = oracle_sample(prob, args.ref_ny)
    cores = host_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    from oracle import oracle as O
    sim = O.OracleSim(smp)
    for _ in range(max(args.warmup, 0)):
        sim.step(1)
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    nx, ny, nz = smp["n"]
    value = nx * ny * nz * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded workload generator)",
        "config": {"workload": prob["name"], "grid": list(prob["n"]), "num_bath": 8,
                   "precision": 64, "timed": f"oracle steps of a {nx}x{ny}x{nz} sample (all z planes)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
                         "kind": "oracle",
                         "sample": f"{args.steps} oracle steps of the {nx}x{ny}x{nz} sample of the 256^3 workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def form_precision(fb, stream, torch):
    """Precision form: the 512 x 512 x 384 workload (N_b = 16, Rabi 0.1) in FP32 and in FP32 with
    bf16-stored bath modes (throughput, roofline), and both against the FP64 GPU path on the 64^3
    crop (field, spectrum and polariton-peak errors)."""
    from paper_2505_23963_gb300 import analysis
    hbm, _ = peaks()
    prob = wl.precision_3d(steps=40)
    cells = float(np.prod(prob["n"]))
    out = {"workload": prob["name"]}
    for tag, bs in (("fp32", 0), ("bf16_bath", 1)):
        with torch.cuda.stream(stream):
            sim = fb.Simulation(prob, precision=32, stream=stream, bath_storage=bs, energy_capacity=64)
        sim.step(3)
        sim.sync()
        k = 20
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        sim.step(k)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / k
        byts = algorithmic_bytes(prob, 4, None if bs == 0 else 8.0)
        out[tag] = {"value": cells / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                    "bytes_per_cell": byts / cells, "achieved_GBs": byts / (ms * 1e-3) / 1e9,
                    "frac_hbm": byts / (ms * 1e-3) / 1e9 / hbm,
                    "bath_kernel": "plain3d Lorentz-Bath form" if sim.bath_plain_kernel() else "step3d"}
        if bs:
            # against 6 B per mode and component (a bf16 value of each of two levels read, one
            # written): the bf16 pair layout moves 8 (value and increment read and written)
            b6 = algorithmic_bytes(prob, 4, 6.0)
            out[tag].update({"bytes_per_cell_6B_per_mode": b6 / cells,
                             "frac_hbm_6B_per_mode": b6 / (ms * 1e-3) / 1e9 / hbm,
                             "pair_layout_extra_bytes_per_cell": (byts - b6) / cells})
        sim.close()
    crop = wl.precision_crop()
    runs = {}
    for tag, prec, bs in (("fp64", 64, 0), ("fp32", 32, 0), ("bf16_bath", 32, 1)):
        sim = fb.Simulation(crop, precision=prec, bath_storage=bs, energy=False)
        sim.step(crop["steps"])
        spec = sim.dft(0)
        runs[tag] = (np.asarray(sim.get("E", comp=0), np.float64), spec,
                     analysis.spectral_peaks(crop["monitors"][0]["freqs"], np.abs(spec[:, 0]) ** 2, 2))
        sim.close()
    E0, S0, P0 = runs["fp64"]
    for tag in ("fp32", "bf16_bath"):
        E, S, P = runs[tag]
        out[tag]["crop_errors_vs_fp64"] = {
            "E": float(np.linalg.norm(E - E0) / np.linalg.norm(E0)),
            "spectrum": float(np.linalg.norm(S - S0) / np.linalg.norm(S0)),
            "peaks": float(np.max(np.abs(P - P0) / P0))}
    return out


def many_bath_slab(fb, nxy: int = 256, steps: int = 40) -> dict:
    """nxy x nxy x 160 slab cavity (resolution 32, CPML 16 | 40 | Drude 8 | Lorentz-Bath 32 |
    Drude 8 | 40 | CPML 16) whose layer carries the paper's Fig. 2 bath: N_b = 100 modes of
    Table I's Lorentzian form over nu0 +/- 0.2 (fdtdbath_bath_form), bath damping 4e-4,
    dephasing 0.0396, gamma0 = 4e-4, sigma = 2e-2."""
    f, g, k = fb.bath_form("lorentzian", 1.0, 4e-4, 100, 0.4, 4e-4, 0.0396)
    prob = wl.slab_cavity(nxy, nxy, (16, 40, 8, 32, 8, 40), 32.0, num_bath=8, sigma=2e-2,
                          steps=steps, name=f"slab3d_{nxy}x{nxy}x160_nb100")
    mats = list(prob["materials"])
    mats[1] = dict(mats[1], gamma=4e-4, bath_frequencies=f, bath_gammas=g, bath_couplings=k)
    return dict(prob, materials=mats)


def form_many_bath(fb, stream, torch):
    """N_b = 100 (the paper's Fig. 2 bath) on the 256 x 256 x 160 slab, FP32: above 32 modes the
    step kernel streams the bath modes twice per step (bath sum, then update); the algorithmic
    bytes count every state word once, so the roofline fraction shows what the second pass
    costs."""
    hbm, _ = peaks()
    prob = many_bath_slab(fb)
    cells = float(np.prod(prob["n"]))
    with torch.cuda.stream(stream):
        sim = fb.Simulation(prob, precision=32, stream=stream, energy_capacity=64)
    sim.step(3)
    sim.sync()
    k = 20
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    sim.step(k)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / k
    finite = spectrum_is_finite(fb, sim)
    sim.close()
    byts = algorithmic_bytes(prob, 4)
    return {"workload": prob["name"], "value": cells / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms, "bytes_per_cell": byts / cells,
            "achieved_GBs": byts / (ms * 1e-3) / 1e9, "frac_hbm": byts / (ms * 1e-3) / 1e9 / hbm,
            "finite": finite}


def form_sigma_map(fb, stream, torch):
    """Per-cell oscillator strength sigma(r) on the 256^3 slab cavity (N_b = 8, FP32): the
    Lorentz-Bath layer patterned by fdtdbath_sigma_box -- a 128 x 128-cell square of twice the
    layer's sigma whose edges cut cells in half (sub-pixel averaged) -- so every cell of the
    dispersive layers reads its own sigma (one more word per such cell), on the same plain-plane
    kernels as the headline step."""
    hbm, _ = peaks()
    prob = wl.slab_3d(steps=0)
    cells = float(np.prod(prob["n"]))
    lb = next(m for m in prob["materials"] if m["kind"] == "lorentz_bath")
    with torch.cuda.stream(stream):
        sim = fb.Simulation(prob, precision=32, stream=stream, energy_capacity=64)
    sim.sigma_box((63.5, 63.5, lb["z"][0]), (191.5, 191.5, lb["z"][1]), 2.0 * lb["sigma"])
    assert sim.sigma_map()
    sim_plain = sim.plain_kernel() and sim.bath_plain_kernel()
    sim.step(3)
    sim.sync()
    k = 20
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    sim.step(k)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / k
    finite = spectrum_is_finite(fb, sim)
    sim.close()
    byts = algorithmic_bytes(prob, 4, sigma_map=True)
    return {"workload": prob["name"] + "_sigma_box", "value": cells / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms, "bytes_per_cell": byts / cells,
            "kernel": "plain3d_kernel (bath-free and Lorentz-Bath forms)" if sim_plain else "step3d_kernel",
            "achieved_GBs": byts / (ms * 1e-3) / 1e9, "frac_hbm": byts / (ms * 1e-3) / 1e9 / hbm,
            "finite": finite}


def form_temporal_blocking(fb, stream, torch):
    """Two steps per pass (temporal blocking) on the 256^3 slab cavity's flux normalization run
    (its layers removed: 16-cell CPML at both ends, vacuum, the phased plane source, the flux
    monitor and the energy box; FP32): the two-steps-per-pass kernel against single steps of the
    plain-plane kernel on the same grid.  The algorithmic bytes count every state word once per
    step, as for the other forms, so a kernel that moves the state once per two steps can exceed
    the copy bandwidth (frac_hbm above 1); the DRAM traffic of one two-step launch is recorded
    beside it when a capture of the current source exists."""
    import hashlib
    hbm, _ = peaks()
    prob = wl.vacuum_of(wl.slab_3d(steps=0))
    cells = float(np.prod(prob["n"]))
    byts = algorithmic_bytes(prob, 4)
    out = {"workload": prob["name"], "unit": UNIT, "bytes_per_cell": byts / cells}
    k = 40
    for label, flag in (("two_step", "1"), ("single_step", "0")):
        old = os.environ.get("FDTDBATH_TB")
        if flag is None:
            os.environ.pop("FDTDBATH_TB", None)
        else:
            os.environ["FDTDBATH_TB"] = flag
        try:
            with torch.cuda.stream(stream):
                sim = fb.Simulation(prob, precision=32, stream=stream, energy_capacity=64)
        finally:
            if old is None:
                os.environ.pop("FDTDBATH_TB", None)
            else:
                os.environ["FDTDBATH_TB"] = old
        active = sim.tb2_kernel()
        sim.step(5)   # odd: the H half-step stays pending, so the timed steps run in pairs
        sim.sync()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        sim.step(k)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / k
        finite = spectrum_is_finite(fb, sim)
        sim.close()
        out[label] = {"kernel": ("tb2_kernel<float> (one launch per two steps)" if active else
                                 "plain3d_kernel<float> (one launch per step)"),
                      "value": cells / (ms * 1e-3), "ms_per_step": ms,
                      "achieved_GBs": byts / (ms * 1e-3) / 1e9,
                      "frac_hbm": byts / (ms * 1e-3) / 1e9 / hbm, "finite": finite}
    out["value"] = out["two_step"]["value"]
    out["speedup"] = out["single_step"]["ms_per_step"] / out["two_step"]["ms_per_step"]
    traffic = None
    prof = os.path.join(ROOT, "profiles", "tb2_f32_vacuum256_traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                rec = json.load(f)
            with open(os.path.join(ROOT, "paper_2505_23963_gb300", "csrc", "tb2.cuh"), "rb") as f:
                cur = hashlib.sha256(f.read()).hexdigest()[:16]
            if rec.get("source_sha256_16") == cur:
                traffic = rec.get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    out["dram_bytes_per_two_step_launch"] = traffic
    out["algorithmic_bytes_per_two_steps"] = 2 * byts
    return out


def form_cavity_1d(fb, stream, torch):
    """The plain method on the 1D Fabry-Perot cavity (Nz = 2000, N_b = 16, 500 DFT frequencies,
    energy every step), 20000 steps on the persistent 1D kernel in FP64 and FP32: steps/s and
    cell-updates/s.  On-chip and latency-bound: the state stays in registers for a whole call."""
    steps = 20000
    prob = wl.cavity_1d(steps=steps)
    nz = prob["n"][2]
    out = {"workload": prob["name"], "steps": steps}
    for prec in (64, 32):
        with torch.cuda.stream(stream):
            sim = fb.Simulation(prob, precision=prec, stream=stream, energy_capacity=steps + 208)
        sim.step(200)
        sim.sync()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        sim.step(steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        out[f"fp{prec}"] = {"value": nz * steps / (ms * 1e-3), "unit": UNIT,
                            "steps_per_s": steps / (ms * 1e-3), "us_per_step": 1e3 * ms / steps,
                            "finite": spectrum_is_finite(fb, sim)}
        sim.close()
    return out


# FP32 ALU peak derived from the part's unit counts: 152 SMs x 128 FP32 lanes x 2 flops per FMA
# x 2.07 GHz maximum SM clock (no measured FP32 figure exists for this machine)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def batch_flops_per_step(probs) -> float:
    """Algorithmic flops of one step of a batch of 1D cavities (an FMA counts 2): per cell 6 for
    the E and H half-steps, +8 in CPML cells (both memories), +8 for a Lorentz / Drude
    polarization, +10 N_b + 8 for a Lorentz-Bath polarization with its N_b bath modes.  Energy
    sums are not counted."""
    total = 0.0
    for p in probs:
        nz, pml = p["n"][2], int(p.get("pml", 0))
        total += 6.0 * nz + 8.0 * 2 * pml
        for m in p["materials"]:
            n = m["z"][1] - m["z"][0]
            nb = len(m.get("bath_frequencies", ()))
            if m["kind"] == "lorentz_bath" and nb > 0:
                total += (10.0 * nb + 8.0) * n
            elif m["kind"] in ("lorentz", "drude", "lorentz_bath"):
                total += 8.0 * n
    return total


def form_batch(fb, torch):
    """Batching form: 64 independent 1D cavities (lengths 1000-8000, Rabi 0.01-0.2, N_b in
    {4, 8, 16, 32}), 50000 FP32 steps in persistent launches replayed from CUDA graphs, energy every
    10 steps; per-cavity relaxation rate and bath share; the plain FP64 GPU path's time for the
    same cell-updates, measured on one cavity and scaled."""
    from paper_2505_23963_gb300 import analysis
    steps = 50000
    probs = wl.batch_sweep(steps=steps)
    cells = float(sum(p["n"][2] for p in probs))
    b = fb.Batch(probs, precision=32, energy_every=10)
    t0 = time.perf_counter()
    C, T, tuned = b.autotune(200)
    tune_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    b.sync()
    secs = time.perf_counter() - t0
    dtr = 10 * probs[0]["courant"] / probs[0]["resolution"]
    gam, share = [], []
    for i, p in enumerate(probs):
        tr = b.trace(i)
        t0p = 2 * p["sources"][0]["t0"]
        gam.append(analysis.relaxation_rate(tr, dtr, t0p))
        share.append(analysis.bath_share(tr, dtr, t0p))
    shape = b.shape()
    b.close()
    # the plain FP64 path on one cavity of the sweep
    ref = probs[int(np.argsort([p["n"][2] for p in probs])[len(probs) // 2])]
    sim = fb.Simulation(ref, precision=64, energy_capacity=2100)
    sim.step(100)
    sim.sync()
    t0 = time.perf_counter()
    sim.step(2000)
    sim.sync()
    rate64 = ref["n"][2] * 2000 / (time.perf_counter() - t0)
    sim.close()
    g = np.asarray(gam)
    flops = batch_flops_per_step(probs)
    return {"workload": "batch sweep: 64 cavities x 50000 steps", "value": cells * steps / secs,
            "unit": UNIT, "seconds": secs, "steps": steps, "cells": cells,
            "launch_shape": {"cluster_ctas": C, "threads": T, **shape}, "autotune_s": tune_s,
            "gamma_pol": {"min": float(np.nanmin(g)), "median": float(np.nanmedian(g)),
                          "max": float(np.nanmax(g))},
            "bath_share": {"min": float(np.nanmin(share)), "median": float(np.nanmedian(share)),
                           "max": float(np.nanmax(share))},
            "plain_fp64_path": {"value": rate64, "unit": UNIT,
                                "seconds_for_same_work": cells * steps / rate64},
            # on-chip and bound by issue and latency, not by arithmetic: the FP32 rate against
            # the derived ALU peak shows how far
            "roofline": {"bound": "alu", "achieved": flops * steps / secs / 1e12,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": flops * steps / secs / 1e12 / FP32_PEAK_TFLOPS,
                         "peak_kind": "derived (152 SMs x 128 FP32 lanes x 2 x 2.07 GHz)",
                         "flops_per_step": flops}}


def form_adjoint(fb, torch):
    """Differentiation form: 2D TE cavity 2048 x 2048 (N_b = 8), 8000 FP32 steps with checkpoints
    every 256, loss = sum (T - T*)^2 over 128 frequencies; gradient w.r.t. sigma, gamma and the 8
    couplings through torch.autograd (forward and backward wall times); the target T* is the
    transmission at the seeded perturbed parameters."""
    from paper_2505_23963_gb300 import adjoint as adj
    prob = wl.adjoint_2d(steps=8000)
    n = prob["steps"]
    cells = float(np.prod(prob["n"]))
    p0 = adj.layer_params(prob, 1)
    s = fb.Simulation(wl.vacuum_of(prob), precision=32, energy=False)
    s.step(n)
    fv = np.real(_flux(s.dft(0)))
    s.close()
    s = fb.Simulation(adj.with_params(prob, 1, wl.adjoint_target_params(p0)), precision=32, energy=False)
    s.step(n)
    target = _flux(s.dft(0)) / fv
    s.close()
    x = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = adj.transmission_loss(x, prob, 1, fv, target, n, 256, 32)
    torch.cuda.synchronize()
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    L.backward()
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    g = x.grad.numpy()
    # memory roofline of both sweeps (algorithmic bytes as counted in algorithmic_bytes_te; the
    # reverse sweep recomputes every forward step with recording, then runs the adjoint kernels)
    hbm, _ = peaks()
    bt = algorithmic_bytes_te(prob)
    fwd_gbs = bt["forward"] * n / tf / 1e9
    rev_gbs = (bt["forward"] + bt["record"] + bt["adjoint"]) * n / tb / 1e9
    roof = {"bound": "hbm", "unit": "GB/s", "peak": hbm,
            "forward": {"bytes_per_step": bt["forward"], "achieved": fwd_gbs, "frac": fwd_gbs / hbm},
            "reverse": {"bytes_per_step": bt["forward"] + bt["record"] + bt["adjoint"],
                        "achieved": rev_gbs, "frac": rev_gbs / hbm}}
    return {"workload": prob["name"], "steps": n, "checkpoint_every": 256,
            "forward_s": tf, "backward_s": tb, "roofline": roof,
            "value": cells * n / (tf + tb), "unit": UNIT + " (forward + reverse sweep)",
            "loss": float(L.detach()), "grad_finite": bool(np.all(np.isfinite(g))),
            "grad": [float(v) for v in g]}


def profile_form(name: str) -> int:
    """Short runs of one form for profiler captures: the 64-cavity batch for 64 steps in the shape
    the autotuner picks for it (C = 4, 896 threads), 16 steps of the 2048^2 differentiation form forward and
    reverse (checkpoints every 8 steps: about 2 GB of device memory), 8 steps of the N_b = 100
    slab at 128 x 128 (about 1.5 GB), 8 steps of the N_b = 16 precision workload at 128 x 128 x
    384 (about 1.3 GB), or 8 steps of the 256^3 slab with the sigma box of the sigma_map form
    (about 1.7 GB), 9 steps of the 256^3 flux normalization run (about 1 GB; the two-step
    kernel), or the temporal-blocking form itself."""
    import torch
    from paper_2505_23963_gb300 import fdtdbath as fb
    torch.cuda.set_device(0)
    if name == "manybath":
        sim = fb.Simulation(many_bath_slab(fb, nxy=128, steps=8), precision=32, energy_capacity=16)
        sim.step(8)
        sim.sync()
        print(json.dumps({"form": "manybath", "steps": 8}), flush=True)
        sim.close()
        return 0
    if name == "precision":
        prob = wl.precision_3d(steps=8)
        prob = dict(prob, n=(128, 128, prob["n"][2]), name="precision3d_128x128x384_nb16")
        prob["sources"] = [dict(q, phase=q["phase"][:128, :128]) for q in prob["sources"]]
        sim = fb.Simulation(prob, precision=32, energy_capacity=16)
        sim.step(8)
        sim.sync()
        print(json.dumps({"form": "precision", "steps": 8, "bath_form": sim.bath_plain_kernel()}), flush=True)
        sim.close()
        return 0
    if name == "sigma":
        prob = wl.slab_3d(steps=8)
        lb = next(m for m in prob["materials"] if m["kind"] == "lorentz_bath")
        sim = fb.Simulation(prob, precision=32, energy_capacity=16)
        sim.sigma_box((63.5, 63.5, lb["z"][0]), (191.5, 191.5, lb["z"][1]), 2.0 * lb["sigma"])
        sim.step(8)
        sim.sync()
        print(json.dumps({"form": "sigma", "steps": 8, "plain": sim.plain_kernel(),
                          "bath_form": sim.bath_plain_kernel()}), flush=True)
        sim.close()
        return 0
    if name == "tb2":
        # the 256^3 flux normalization run: one single step, then four two-step launches
        os.environ["FDTDBATH_TB"] = "1"
        sim = fb.Simulation(wl.vacuum_of(wl.slab_3d(steps=9)), precision=32, energy_capacity=16)
        sim.step(9)
        sim.sync()
        print(json.dumps({"form": "tb2", "steps": 9, "two_step": sim.tb2_kernel()}), flush=True)
        sim.close()
        return 0
    if name == "tb2_form":
        stream = torch.cuda.Stream()
        print(json.dumps({"form": "temporal_blocking",
                          **form_temporal_blocking(fb, stream, torch)}), flush=True)
        return 0
    if name == "batch":
        b = fb.Batch(wl.batch_sweep(steps=64), precision=32, energy_every=10, cluster_ctas=4,
                     block_threads=896, use_graph=False)
        b.step(64)
        b.sync()
        print(json.dumps({"form": "batch", "steps": 64, **b.shape()}), flush=True)
        b.close()
        return 0
    from paper_2505_23963_gb300 import adjoint as adj
    prob = wl.adjoint_2d(steps=16)
    p0 = adj.layer_params(prob, 1)
    x = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    nf = len(prob["monitors"][0]["freqs"])
    L = adj.transmission_loss(x, prob, 1, np.ones(nf), np.zeros(nf), 16, 8, 32)
    L.backward()
    print(json.dumps({"form": "adjoint", "steps": 16, "grad_finite": bool(np.all(np.isfinite(x.grad.numpy())))}),
          flush=True)
    return 0


def _flux(spec):
    return np.real(spec[:, 0] * np.conj(spec[:, 3]) - spec[:, 1] * np.conj(spec[:, 2]))


def run_ours(args):
    import torch
    from paper_2505_23963_gb300 import fdtdbath as fb

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local if ws > 1 else 0
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    prob = wl.slab_3d(steps=args.warmup + args.steps)
    if args.grid:
        gx, gy = (int(v) for v in args.grid.split(","))
        prob = dict(prob, n=(gx, gy, prob["n"][2]), name=f"slab3d_{gx}x{gy}x256_nb8")
        prob["sources"] = [dict(s, phase=s["phase"][:gy, :gx]) for s in prob["sources"]]
    nx, ny, nz = prob["n"]
    cells = nx * ny * nz

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed_run(precision: int, steps: int, warmup: int, sample_clocks: bool):
        with torch.cuda.stream(stream):
            sim = fb.Simulation(prob, precision=precision, stream=stream,
                                energy_capacity=warmup + steps + 8)
        sim.step(warmup)
        sim.sync()
        l0 = sim.launches()
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(dev) if sample_clocks else None
        if clk:
            clk.__enter__()
            time.sleep(0.5)
        ev0.record(stream)
        sim.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        if clk:
            clk.__exit__(None, None, None)
        barrier()
        ms = ev0.elapsed_time(ev1)
        launches = sim.launches() - l0
        # kernel-only duration: events around each single-step call (one step-kernel launch)
        kev = []
        nk = min(steps, 20)
        for _ in range(nk):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(1)
            b.record(stream)
            kev.append((a, b))
        torch.cuda.synchronize()
        kms = float(np.mean([a.elapsed_time(b) for a, b in kev]))
        finite = spectrum_is_finite(fb, sim)
        sim.close()
        return ms, launches, kms, finite, (clk.summary() if clk else None)

    # ---- FP32 headline ----
    ms32, launches, kms32, ok32, clocks = timed_run(32, args.steps, args.warmup, not args.quick)
    ms32 = max_over_ranks(ms32, f"cuda:{dev}")
    value = replica_rate(cells * args.steps, ws, ms32 * 1e-3)
    if args.quick:
        # profiling mode: the FP32 step only, no FP64 / end-to-end / CPU legs
        if rank == 0:
            print(json.dumps({"mode": "quick", "workload": prob["name"], "value": value,
                              "unit": UNIT, "ms_per_step": ms32 / args.steps,
                              "kernel_ms": kms32, "finite": ok32}), flush=True)
        return 0
    # ---- FP64 beside it (fewer steps: FP64 arithmetic is slow on this part) ----
    k64 = max(3, min(args.steps, 20))
    ms64, _, kms64, ok64, _ = timed_run(64, k64, 3, False)
    ms64 = max_over_ranks(ms64, f"cuda:{dev}")
    value64 = replica_rate(cells * k64, ws, ms64 * 1e-3)

    # ---- FP64 roofline: FP64 instruction issue (the measured FMA rate / 2 instructions per
    # second) against the memory roofline of the same step ----
    fma64 = fb.measure_fma_rate(64, dev, 5)
    flops64 = algorithmic_flops_fp64(prob)
    instr64 = algorithmic_flops_fp64(prob, instructions=True)
    step64 = ms64 / k64 * 1e-3
    hbm_gbs, _ = peaks()
    peak64 = fma64 / 2.0 * flops64 / instr64   # flop rate at one FP64 instruction per FMA slot
    alu_frac = flops64 / step64 / peak64
    hbm_frac64 = algorithmic_bytes(prob, 8) / step64 / 1e9 / hbm_gbs
    roof64 = {"bound": "alu" if alu_frac >= hbm_frac64 else "hbm",
              "achieved": flops64 / step64 / 1e12, "peak": peak64 / 1e12, "unit": "TFLOP/s",
              "frac": alu_frac, "flops_per_step": flops64, "fp64_instructions_per_step": instr64,
              "fma_rate_tflops": fma64 / 1e12,
              "peak_kind": "measured FP64 FMA rate / 2 instructions per second x the step's flops per "
                           "FP64 instruction (fused multiply-adds in the bath recursion only)",
              "hbm_frac": hbm_frac64}

    # ---- end to end through the C ABI with host buffers (create .. dft/energy .. destroy) ----
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = fb.Simulation(prob, precision=32, stream=stream, energy_capacity=args.steps + 8)
    sim.step(args.steps)
    spec = sim.dft(0)
    tr = sim.trace()
    sim.close()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, f"cuda:{dev}")
    e2e_value = replica_rate(cells * args.steps, ws, e2e_s)
    h2d = (prob["sources"][0]["phase"].size * 8 + prob["monitors"][0]["freqs"].size * 8
           + sum(3 * 8 * len(m.get("bath_frequencies", [])) for m in prob["materials"]))
    d2h = spec.size * 16 + tr.size * 8

    # ---- roofline of the step kernel ----
    hbm, peak_kind = peaks()
    bytes32 = algorithmic_bytes(prob, 4)
    # one step = the launch pair of the plain-plane kernel (the bath-free chunks on a side stream
    # beside its Lorentz-Bath form over the bath chunks on the simulation's stream, joined back into
    # it); its average duration over the timed region comes from the events on the simulation's
    # stream (plus one reduce + DFT per 256 steps)
    step_ms = ms32 / args.steps
    achieved = bytes32 / (step_ms * 1e-3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "plain3d_f32_slab3d_traffic.json")
    if os.path.exists(prof) and not args.grid:
        try:
            import hashlib
            with open(prof) as f:
                rec = json.load(f)
            with open(os.path.join(ROOT, "paper_2505_23963_gb300", "csrc", "plain3d.cuh"), "rb") as f:
                cur = hashlib.sha256(f.read()).hexdigest()[:16]
            # counters describe the kernel they were taken on: none once it has changed
            traffic = rec.get("dram_bytes_per_step") if rec.get("source_sha256_16") == cur else None
        except Exception:
            traffic = None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = host_cores()
        os.environ["OMP_NUM_THREADS"] = str(cores)
        rate, secs, nst, smp = oracle_rate(prob)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{nst} FP64 oracle steps of a {smp['n'][0]}x{smp['n'][1]}x{smp['n'][2]} "
                         f"sample (full x, z; 16 of 256 y rows) of the workload, {secs:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded workload generator; no dataset)",
        "config": {"workload": prob["name"], "grid": [nx, ny, nz], "num_bath": 8,
                   "precision": 32, "l2": "state 1.6 GB > 129 MB L2 (no flush needed)",
                   "parallelism": f"replicas x{ws}"},
        "fp64": {"value": value64, "unit": UNIT, "steps": k64, "ms_per_step": ms64 / k64,
                 "kernel_ms": kms64, "finite": ok64, "roofline": roof64},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "plain3d_kernel<float> (launch pair of one step: bath-free chunks, "
                               "Lorentz-Bath form)", "kernel_ms": step_ms,
                     "kernel_ms_single_call": kms32,
                     "algorithmic_bytes_per_launch": bytes32},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "finite": ok32,
    }
    if ws == 1 and not args.no_forms:
        forms = {}
        for name, fn in (("precision", lambda: form_precision(fb, stream, torch)),
                         ("many_bath", lambda: form_many_bath(fb, stream, torch)),
                         ("sigma_map", lambda: form_sigma_map(fb, stream, torch)),
                         ("temporal_blocking", lambda: form_temporal_blocking(fb, stream, torch)),
                         ("batch", lambda: form_batch(fb, torch)),
                         ("adjoint", lambda: form_adjoint(fb, torch)),
                         ("cavity_1d", lambda: form_cavity_1d(fb, stream, torch))):
            try:
                forms[name] = fn()
            except Exception as exc:   # reported, not hidden: the line says which form failed
                forms[name] = {"error": f"{type(exc).__name__}: {exc}"}
        line["forms"] = forms
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-ny", type=int, default=8, help="y rows of the reference arm's sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the precision / batching / differentiation forms")
    ap.add_argument("--quick", action="store_true",
                    help="FP32 step timing only (for profiler captures)")
    ap.add_argument("--grid", default="", help="override nx,ny of the workload (profiling)")
    ap.add_argument("--profile-form", default="", choices=["", "batch", "adjoint", "manybath", "precision", "sigma", "tb2", "tb2_form"],
                    help="run a short version of one form only (for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_form:
        return profile_form(args.profile_form)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
