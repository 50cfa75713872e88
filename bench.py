#!/usr/bin/env python3
"""Throughput of the boosted-frame PIC step on GB300.

Workload: the plasma buncher (128 x 128 x 512 Yee grid, transverse PML, longitudinal moving
window, boost 20, 4,194,304 beam electrons of lab gamma 400, cold lab-static plasma of
1e15 cm^-3 at 8 particles per cell with frozen neutralising ions, TSC shape).  One step =
tile sort (every 8 steps) + gather + push + Esirkepov deposit of every species + FDTD with
CPML + window shift / plasma injection when due.  Metric: pushed macroparticle-steps per
second (beam + plasma electrons; frozen ions are deposited every step but not counted).

Default (--impl gbpic): the CUDA path through the C-ABI, timed with CUDA events on the
context's stream over exactly K steps after W warm-up steps, barrier + synchronize on both
sides, max over ranks.  N > 1 ranks run independent replicas (weak scaling).  The JSON line
also carries the roofline of the dominant kernel (from the library's per-launch CUDA-event
trace), the FP64 oracle timed on the host cores on a bounded sample (cpu_baseline), the
end-to-end figure through the C-ABI with host buffers (e2e), clocks sampled during the timed
region and the number of kernels launched.

--impl reference: the FP64 CPU oracle, as it stands, on a bounded sample of the same workload
(the only other place this script runs the oracle).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+deposit+FDTD) FP32 vs FP64 at tol; adjoint/fwd ratio"
UNIT = "particle-steps/s"
HBM_FALLBACK = 6800.0
# algorithmic bytes (FP32 storage) of the particle kernel: per pushed particle r+w of cell 4 +
# offset 12 + momentum 12 (56 B; the weight, read with the momentum, is reported apart); per
# frozen particle r+w of cell + offset; per cell, once per step, E,B read by the gather (24) and J
# written by the deposit (12)
BYTES_PUSHED = 56.0
BYTES_WEIGHT = 4.0
BYTES_FROZEN = 32.0
BYTES_CELL_PUSH = 36.0
# DRAM bytes (read + write) of the particle kernel per step of the plasma buncher 128x128x512 (its
# two launches: plasma electrons and beam): one-pass ncu capture of dram__bytes_read.sum and
# dram__bytes_write.sum on the half-length grid 128x128x256 (plasma launch 2.24 GB for 30.38M
# electrons, beam launch 0.110 GB for 2.10M), scaled by the particles each launch pushes at full
# size (61.36M and 4.19M).
TRAFFIC_PUSH_BUNCHER_STEP = 4.74e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(os.environ.get("GBPIC_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_vacuum(steps, warmup, seed=1):
    """FP64 oracle on the whole vacuum-undulator workload (32 x 32 x 64, 65,536 beam, CIC)."""
    import oracle
    from paper_2411_04703_gb300 import workloads as W
    oracle.build()
    w = W.vacuum_undulator(seed=seed)
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
    o.set_external(w.undulator.K, w.undulator.lambda_u)
    sb = o.add_species(-1.0, 1.0)
    x, u, wt = W.sample_beam(w)
    o.load(sb, x, u, wt, frame=0, origin=w.beam.origin, match_undulator=True)
    if warmup:
        o.step(warmup)
    n0 = o.count(sb)
    t0 = time.perf_counter()
    o.step(steps)
    t = time.perf_counter() - t0
    value = 0.5 * (n0 + o.count(sb)) * steps / t
    sample = f"FP64 oracle, the whole vacuum-undulator workload ({n0} beam, CIC), {steps} steps, single thread"
    return value, t, sample


def oracle_sample_ensemble(steps, warmup, seed=4):
    """FP64 oracle on a bounded sample of the batched ensemble: run 0 on a 32 x 32 x 64 sub-box
    (same cells, K, plasma density and particles per cell; beam scaled with the volume)."""
    import oracle
    from paper_2411_04703_gb300 import workloads as W
    oracle.build()
    e = W.batched_ensemble(seed=seed)
    w = W.ensemble_run(e, 0)
    w.grid = (32, 32, 64)
    w.plasma = W.dataclasses.replace(w.plasma, xrange=(0, 32, 0, 32))
    w.beam.n = max(1000, e.n_beam[0] // 8)
    w.beam.origin = (16.0, 16.0, 32.0)
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
    o.set_external(w.undulator.K, w.undulator.lambda_u)
    se = o.add_species(-1.0, 1.0)
    si = o.add_species(1.0, 1836.15267343, frozen=True)
    sb = o.add_species(-1.0, 1.0)
    p = w.plasma
    o.set_plasma(se, si, p.ppc, p.xrange, p.z_nodes, p.n_nodes)
    x, u, wt = W.sample_beam(w)
    o.load(sb, x, u, wt, frame=0, origin=w.beam.origin, match_undulator=True)
    if warmup:
        o.step(warmup)
    n0 = o.count(se) + o.count(sb)
    t0 = time.perf_counter()
    o.step(steps)
    t = time.perf_counter() - t0
    n1 = o.count(se) + o.count(sb)
    value = 0.5 * (n0 + n1) * steps / t
    sample = (f"FP64 oracle, run 0 of the ensemble on a 32x32x64 sub-box (4 ppc plasma + frozen ions, "
              f"{o.count(sb)} beam), {steps} steps after {warmup} warm-up, single thread")
    return value, t, sample


def oracle_sample_long(steps, warmup, seed=3):
    """FP64 oracle on a bounded sample of the long undulator: a 32 x 32 x 128 sub-box (same cells,
    undulator and ramp, PML) with the beam scaled to the sub-box's volume."""
    import oracle
    from paper_2411_04703_gb300 import workloads as W
    oracle.build()
    # the bunch inside the field, as in the timed GPU steps (which follow its entry)
    w = W.long_undulator(grid=(32, 32, 128), n_beam=65536, seed=seed, z_start=0.0)
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order)
    un = w.undulator
    o.set_external(un.K, un.lambda_u, un.phase, un.z_start, un.ramp, kind=un.kind)
    sb = o.add_species(-1.0, 1.0)
    x, u, wt = W.sample_beam(w)
    o.load(sb, x, u, wt, frame=0, origin=w.beam.origin, match_undulator=un.match)
    if warmup:
        o.step(warmup)
    n0 = o.count(sb)
    t0 = time.perf_counter()
    o.step(steps)
    t = time.perf_counter() - t0
    value = 0.5 * (n0 + o.count(sb)) * steps / t
    sample = (f"FP64 oracle, 32x32x128 sub-box of the long undulator ({n0} beam inside the field, TSC, PML), {steps} steps, "
              f"single thread")
    return value, t, sample


def oracle_sample(steps, warmup, seed=2):
    """FP64 oracle on a bounded sample of the workload: a 32 x 32 x 128 sub-box with the same
    cells, plasma density, particles per cell, beam density, boundaries and window."""
    import oracle
    from paper_2411_04703_gb300 import workloads as W
    oracle.build()
    w = W.plasma_buncher(grid=(32, 32, 128), n_beam=65536, seed=seed)
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order,
                   moving_window=w.moving_window, window_v=w.window_v)
    se = o.add_species(-1.0, 1.0)
    si = o.add_species(1.0, 1836.15267343, frozen=True)
    sb = o.add_species(-1.0, 1.0)
    p = w.plasma
    o.set_plasma(se, si, p.ppc, p.xrange, p.z_nodes, p.n_nodes)
    x, u, wt = W.sample_beam(w)
    o.load(sb, x, u, wt, frame=0, origin=w.beam.origin)
    if warmup:
        o.step(warmup)
    n0 = o.count(se) + o.count(sb)
    t0 = time.perf_counter()
    o.step(steps)
    t = time.perf_counter() - t0
    n1 = o.count(se) + o.count(sb)
    value = 0.5 * (n0 + n1) * steps / t
    sample = (f"FP64 oracle, 32x32x128 sub-box of the plasma buncher (8 ppc plasma + frozen ions, "
              f"{o.count(sb)} beam), {steps} steps after {warmup} warm-up, single thread")
    return value, t, sample


def cpu_info():
    """Host core count and CPU model (lscpu), for the CPU baseline."""
    n = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                v = line.split(":", 1)[1].strip()
                if v and v != "-" and not v.isdigit():
                    model = v
                    break
    except Exception:
        pass
    return n, model


def oracle_buncher_sim(seed=2, grid=(32, 32, 128), n_beam=65536, threads=1):
    import oracle
    from paper_2411_04703_gb300 import workloads as W
    oracle.build()
    w = W.plasma_buncher(grid=grid, n_beam=n_beam, seed=seed)
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order,
                   moving_window=w.moving_window, window_v=w.window_v)
    used = o.set_threads(threads)
    se = o.add_species(-1.0, 1.0)
    si = o.add_species(1.0, 1836.15267343, frozen=True)
    sb = o.add_species(-1.0, 1.0)
    p = w.plasma
    o.set_plasma(se, si, p.ppc, p.xrange, p.z_nodes, p.n_nodes)
    x, u, wt = W.sample_beam(w)
    o.load(sb, x, u, wt, frame=0, origin=w.beam.origin)
    return o, (se, sb), used


def oracle_sample_threads(steps, threads):
    """The oracle's particle loop on `threads` host threads (private J per thread), same sub-box as
    oracle_sample: the all-core CPU figure."""
    o, (se, sb), used = oracle_buncher_sim(threads=threads)
    n0 = o.count(se) + o.count(sb)
    t0 = time.perf_counter()
    o.step(steps)
    t = time.perf_counter() - t0
    n1 = o.count(se) + o.count(sb)
    return 0.5 * (n0 + n1) * steps / t, t, used


def _rel(g, r):
    import numpy as np
    den = float(np.max(np.abs(r)))
    return float(np.max(np.abs(g - r)) / den) if den > 0 else float(np.max(np.abs(g)))


def _species_err(sim, sid, o, osid):
    """Momentum error of matching particles (by id), max over components of max|du| / max|u_ref|."""
    import numpy as np
    P = sim.get_particles(sid)
    X, U, Wt, ids = o.particles(osid)
    common, ga, oa = np.intersect1d(P["id"], ids, return_indices=True)
    Ug = P["u"][ga].astype(np.float64)
    Uo = U[oa]
    return {"matched": int(len(common)), "only_gpu": int(len(P["id"]) - len(common)),
            "only_oracle": int(len(ids) - len(common)),
            "u_rel_err": max(_rel(Ug[:, c], Uo[:, c]) for c in range(3)) if len(common) else 0.0}


def fp32_vs_fp64(device, threads):
    """Error of the FP32 CUDA path against the FP64 oracle, per result, on cases the oracle finishes
    in seconds.  Both sides start from the same seeded lab-frame beam and plasma (each transforms
    them itself).  (1) The reduced plasma buncher (28x26x52, TSC, PML, moving window): relative
    field and momentum errors after 1 and 20 steps.  (2) The whole vacuum-undulator run (32x32x64,
    65,536 beam, CIC, 200 steps): the long-run diagnostics in the boosted frame and the lab."""
    import numpy as np
    import oracle
    from paper_2411_04703_gb300 import api, workloads as W
    oracle.build()
    names = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz"]
    out = {"definition": "max|gpu - oracle| / max|oracle| per field component (over the grid) and per "
                         "momentum component (over matched particles); diagnostics |d_gpu - d_ref| / |d_ref|"}
    w = W.mini_plasma()
    x, u, wt = W.sample_beam(w)
    sim, ids = api.from_workload(w, device=device, beam_arrays=(x, u, wt))
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order,
                   moving_window=w.moving_window, window_v=w.window_v)
    o.set_threads(threads)
    oid = {"plasma_e": o.add_species(-1.0, 1.0), "plasma_i": o.add_species(1.0, 1836.15267343, frozen=True)}
    oid["beam"] = o.add_species(-1.0, 1.0)
    p = w.plasma
    o.set_plasma(oid["plasma_e"], oid["plasma_i"], p.ppc, p.xrange, p.z_nodes, p.n_nodes)
    o.load(oid["beam"], x, u, wt, frame=0, origin=w.beam.origin)
    done = 0
    for n in (1, 20):
        sim.step(n - done)
        sim.sync()
        o.step(n - done)
        done = n
        f = {names[c]: _rel(sim.get_field(c).astype(np.float64), o.field(c)) for c in range(9)}
        sp = {k: _species_err(sim, ids[k], o, oid[k]) for k in ("beam", "plasma_e")}
        out[f"{w.name}, {n} step(s)"] = {"fields": f, "species": sp}
    sim.close()
    del sim, o
    w = W.vacuum_undulator()
    x, u, wt = W.sample_beam(w)
    sim, ids = api.from_workload(w, device=device, beam_arrays=(x, u, wt))
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
    o.set_threads(threads)
    o.set_external(w.undulator.K, w.undulator.lambda_u)
    sb = o.add_species(-1.0, 1.0)
    o.load(sb, x, u, wt, frame=0, origin=w.beam.origin, match_undulator=True)
    sim.step(w.steps)
    sim.sync()
    o.step(w.steps)
    un = w.undulator
    k_lab = api.resonant_wavenumber(un.lambda_u, un.K, w.beam.gamma)
    k_rrf = api.rrf_resonant_wavenumber(w)
    diag = {}
    for frame, oframe, k, tag in [(api.PIC_FRAME_BOOSTED, 0, k_rrf, "boosted"), (api.PIC_FRAME_LAB, 1, k_lab, "lab")]:
        mg = sim.get_moments(ids["beam"], frame, k_bunch=k)
        mo = o.moments(sb, frame=oframe, k=k)
        for key in ("bunching", "emit_nx", "emit_ny", "rel_energy_spread"):
            diag[f"{key} ({tag})"] = {"gpu": mg[key], "oracle": mo[key],
                                      "rel_err": abs(mg[key] - mo[key]) / max(abs(mo[key]), 1e-300)}
    out[f"{w.name}, whole run ({w.steps} steps)"] = diag
    sim.close()
    return out


def run_steps(sim, ids, w, workload, steps, diag):
    """The workload's steps; the long undulator takes its FP64 back-transformed bunching
    diagnostic every 100 steps among them (each one a host round trip), appended to diag."""
    if workload != "long_undulator":
        sim.step(steps)
        return
    from paper_2411_04703_gb300 import api
    un = w.undulator
    k_lab = api.resonant_wavenumber(un.lambda_u, un.K, w.beam.gamma)
    done = 0
    while done < steps:
        nxt = min(steps, done + 100 - (done % 100))
        sim.step(nxt - done)
        done = nxt
        if done % 100 == 0:
            diag.append(sim.get_moments(ids["beam"], api.PIC_FRAME_LAB, k_bunch=k_lab)["bunching"])


def entry_steps(w):
    """Steps until the undulator entrance, moving at -beta_R in the RRF, has passed the bunch's
    3-sigma tail (moving at the bunch's RRF velocity until it enters) and its ramp with it."""
    gR, gB = w.gamma_R, w.beam.gamma
    bR, bB = math.sqrt(1.0 - 1.0 / gR ** 2), math.sqrt(1.0 - 1.0 / gB ** 2)
    v_b = (bB - bR) / (1.0 - bB * bR)                      # RRF velocity before the entrance
    sig = w.beam.sigma_z * gB / (gR * gB * (1.0 - bR * bB))  # RRF bunch length (Eq. Belon)
    un = w.undulator
    z_tail = w.beam.origin[2] * w.d[2] - 3.0 * sig
    gap = (un.z_start + max(un.ramp, 0.0)) / gR - z_tail
    return max(0, int(math.ceil(gap / ((bR + v_b) * w.dt))))


def adjoint_block(device, steps=100, every=50):
    """Adjoint/forward cost of the differentiated run (64x64x256, 2M beam + 4 ppc plasma, CIC):
    `steps` forward steps recording checkpoints every `every`, then pic_backward (segment
    recompute with per-step records + the adjoint sweep), both timed with CUDA events."""
    import torch
    from paper_2411_04703_gb300 import api, workloads as W
    w = W.adjoint_workload()
    sim, ids = api.from_workload(w, device=device)
    sim.step(3)
    sim.sync()
    sim.checkpoint(every)
    stream = sim.stream
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    g = sim.backward(ids["beam"], api.rrf_resonant_wavenumber(w))
    e2.record(stream)
    torch.cuda.synchronize()
    fwd, bwd = e0.elapsed_time(e1), e1.elapsed_time(e2)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return {"workload": w.name, "steps": steps, "checkpoint_every": every,
            "forward_ms_per_step": fwd / steps, "backward_ms_per_step": bwd / steps, "ratio": bwd / fwd,
            "includes": "backward = segment recompute with per-step records + adjoint sweep",
            "loss": g["loss"], "dL_dK": g["dL_dK"]}


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores (its particle loop on
    all of them), each step a step of the 32x32x128 sub-box of the plasma buncher."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from paper_2411_04703_gb300 import workloads as W
    full = W.plasma_buncher()            # the workload the default arm measures (its config)
    steps = args.steps
    ncores, model = cpu_info()
    o, (se, sb), used = oracle_buncher_sim(threads=ncores)
    if args.warmup:
        o.step(args.warmup)
    n0 = o.count(se) + o.count(sb)
    t0 = time.perf_counter()
    o.step(steps)
    t = time.perf_counter() - t0
    n1 = o.count(se) + o.count(sb)
    value = 0.5 * (n0 + n1) * steps / t
    sample = (f"FP64 oracle, 32x32x128 sub-box of the plasma buncher (8 ppc plasma + frozen ions, "
              f"{o.count(sb)} beam), {steps} steps after {args.warmup} warm-up, particle loop on {used} host "
              f"thread(s) (OpenMP, a private J per thread)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": full.name, "grid": [32, 32, 128], "target_grid": list(full.grid), "shape": "TSC",
                   "boundaries": "transverse CPML 10 cells, moving window", "sample": sample,
                   "note": "value is per particle-step on the 32x32x128 sub-box (same cells, densities, "
                           "particles per cell, boundaries and window), not a run of the full grid"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                         "cpu_model": model, "nproc": ncores},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def aggregate(psteps, ms, world, device="cpu"):
    """Whole-job figures of independent replicas: particle-steps summed over ranks, timed
    milliseconds maxed over ranks (the slowest rank bounds the job)."""
    if world <= 1:
        return float(psteps), float(ms)
    import torch
    import torch.distributed as dist
    a = torch.tensor([float(psteps)], dtype=torch.float64, device=device)
    b = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    dist.all_reduce(b, op=dist.ReduceOp.MAX)
    return float(a[0]), float(b[0])


def run_adjoint(args):
    """Adjoint/forward cost on the differentiated run (64x64x256, 2M beam + 4 ppc plasma, CIC):
    K forward steps recording checkpoints every 50, then pic_backward (segment recompute + the
    adjoint sweep); the line's value is the forward's pushed particle-steps/s, and "adjoint" gives
    the backward's time per step and the adjoint/forward ratio."""
    import torch
    from paper_2411_04703_gb300 import api, workloads as W
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    w = W.adjoint_workload(seed=5 + rank)
    sim, ids = api.from_workload(w, device=local)
    if args.warmup:
        sim.step(args.warmup)
    sim.sync()
    n0 = sim.get_count(ids["beam"]) + sim.get_count(ids["plasma_e"])
    sim.checkpoint(50)
    stream = sim.stream
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    sim.sync()
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    k_rrf = api.rrf_resonant_wavenumber(w)
    t0 = time.perf_counter()
    g = sim.backward(ids["beam"], k_rrf)
    torch.cuda.synchronize()
    bwd_ms = 1000.0 * (time.perf_counter() - t0)
    clk = clocks.stop()
    value = n0 * args.steps / (fwd_ms / 1000.0)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": fwd_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.grid), "beam": w.beam.n, "plasma_electrons": int(n0 - w.beam.n),
                       "shape": "CIC", "boundaries": "periodic", "checkpoint_every": 50,
                       "l2": "inputs larger than L2 (particle state ~0.5 GB, checkpoints and records ~15 GB)"},
            "adjoint": {"forward_ms_per_step": fwd_ms / args.steps, "backward_ms_per_step": bwd_ms / args.steps,
                        "ratio": bwd_ms / fwd_ms, "includes": "segment recompute with per-step records, adjoint sweep",
                        "loss": g["loss"], "dL_dK": g["dL_dK"],
                        "dL_dprofile_norm": float(sum(v * v for v in g["dL_dprofile"]) ** 0.5)},
            "clocks": clk,
        }
        print(json.dumps(line))
    return 0


def run_gbpic(args):
    import torch
    import torch.distributed as dist
    from paper_2411_04703_gb300 import api, workloads as W

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    ens = None
    tuned = None
    pre_steps = 0
    if args.workload == "vacuum":
        # the vacuum undulator 32x32x64, 65,536 beam electrons, CIC: small enough to be bound by
        # launches, so its step sequence runs as a replayed CUDA graph
        w = W.vacuum_undulator(seed=1 + rank)
        if args.sort_every:
            w.sort_every = args.sort_every
        beam = W.sample_beam(w)
        sim, ids = api.from_workload(w, device=local, beam_arrays=beam)
        if args.autotune and not args.sort_every:
            w.sort_every = tuned = sim.autotune(16)     # the trials advance this periodic run
        ncell_total = w.ncell
        boundaries = "periodic"
        l2 = "L2-resident (fields 2.4 MB, particles 2 MB): launch-bound, timed as a CUDA graph"
    elif args.workload == "long_undulator":
        # the long undulator 256x256x1024: 33.5M beam electrons of lab gamma 2000 at rest on average
        # in a frame of gamma_R = gamma / sqrt(1 + K^2/2), TSC, PML on every face, entrance ramp;
        # the FP64 lab-frame bunching is taken every 100 steps inside the timed steps
        if args.grid:
            # a reduced grid keeps the bunch's peak density (sigma_r is 6 cells, sigma_z 1/12 of
            # the z extent): the beam count scales with nz only
            grid = tuple(int(v) for v in args.grid.split(","))
            nb = args.beam or int(round(33554432 * grid[2] / 1024))
            w = W.long_undulator(grid=grid, n_beam=nb, seed=3 + rank,
                                 name=f"long undulator {grid[0]}x{grid[1]}x{grid[2]} (reduced), {nb} beam, TSC")
        else:
            w = W.long_undulator(seed=3 + rank)
        if args.sort_every:
            w.sort_every = args.sort_every
        beam = W.sample_beam(w)
        sim, ids = api.from_workload(w, device=local, beam_arrays=beam)
        # the bunch starts in front of the undulator; the timed steps are those of the run inside
        # it, so the entrance first sweeps over the whole bunch (3 sigma tail) and its ramp
        pre_steps = entry_steps(w)
        sim.step(pre_steps)
        sim.sync()
        if args.autotune and not args.sort_every:
            t0_steps = sim.get_time()[0]
            w.sort_every = tuned = sim.autotune(16)     # trials inside the undulator, after the entry
            pre_steps += sim.get_time()[0] - t0_steps
        ncell_total = w.ncell
        boundaries = "CPML 10 cells on every face, static window"
        l2 = ("inputs larger than L2 (beam state ~2 GB, fields and CPML ~5.6 GB)" if not args.grid else
              "reduced case for profiling captures")
    elif args.workload == "ensemble":
        # batched sweep: 64 runs of 64x64x128 stacked in one context (one launch per kernel)
        import numpy as np
        ens = W.batched_ensemble(runs=args.runs, seed=4 + rank,
                                 name=f"batched ensemble {args.runs} x (64x64x128), K and density sweep, TSC")
        w = ens.base
        parts = [W.sample_beam(W.ensemble_run(ens, r)) for r in range(ens.runs)]
        beam = (np.concatenate([q[0] for q in parts], axis=1), np.concatenate([q[1] for q in parts], axis=1),
                np.concatenate([q[2] for q in parts]))
        if args.sort_every:
            ens.base.sort_every = args.sort_every
        elif not args.no_autotune:
            # the autotuner's trials advance a run: tune tile and cadence on a throwaway copy,
            # measure a fresh one
            tmp, _ = api.from_ensemble(ens, device=local)
            tile, tuned = tmp.autotune_tiles(((8, 8, 8), (8, 8, 4), (8, 4, 4), (4, 4, 4)), 16)
            ens.base.tile, ens.base.sort_every = tuple(tile), tuned
            tmp.close()
            del tmp
            torch.cuda.empty_cache()
        sim, ids = api.from_ensemble(ens, device=local)
        ncell_total = w.ncell * ens.runs
        boundaries = "periodic (each run)"
        l2 = (f"inputs larger than L2 (particle state ~{8 * ens.runs / 64:.1f} GB, fields "
              f"{0.4 * ens.runs / 64:.2f} GB)")
    else:
        grid = tuple(int(v) for v in (args.grid or "128,128,512").split(","))
        if args.workload == "buncher2d":
            # the paper's 2-D geometry (x-z, ny = 1): 1024 x 2048 cells, 4 ppc, 1M beam
            w = W.plasma_buncher_2d(seed=6 + rank)
        else:
            nb = args.beam or int(round(4194304 * (grid[0] * grid[1] * grid[2]) / (128 * 128 * 512)))
            w = W.plasma_buncher(grid=grid, n_beam=nb, seed=2 + rank)
            if grid != (128, 128, 512):
                w.name = f"plasma buncher {grid[0]}x{grid[1]}x{grid[2]} (reduced), {nb} beam + 8 ppc plasma, TSC"
        beam = W.sample_beam(w)
        if args.tile:
            w.tile = tuple(int(v) for v in args.tile.split(","))
        if args.sort_every:
            w.sort_every = args.sort_every
        elif args.autotune:
            tmp, _ = api.from_workload(w, device=local, beam_arrays=beam)
            w.sort_every = tuned = tmp.autotune(16)
            tmp.close()
            del tmp
            torch.cuda.empty_cache()
        sim, ids = api.from_workload(w, device=local, beam_arrays=beam)
        ncell_total = w.ncell
        boundaries = "transverse CPML 10 cells, moving window" + (" (2-D: x PML, y uniform)" if args.workload == "buncher2d" else "")
        l2 = ("inputs larger than L2 (particle state ~0.6 GB, fields 0.05 GB)" if args.workload == "buncher2d"
              else "inputs larger than L2 (particle state ~9 GB, fields 0.3 GB)" if grid == (128, 128, 512)
              else "reduced case for profiling captures")
    # periodic workloads replay their steps as CUDA graphs (tracing would turn that off): their
    # kernel-class composition comes from a traced pass after the timed region
    graphs = args.workload in ("vacuum", "ensemble")
    sim.trace_enable(not graphs)
    if args.warmup:
        sim.step(args.warmup)
    sim.sync()
    sim.trace_read()
    pushed = [ids[k] for k in ("beam", "plasma_e") if k in ids]
    n0 = sum(sim.get_count(s) for s in pushed)
    frozen0 = sim.get_count(ids["plasma_i"]) if "plasma_i" in ids else 0
    stream = sim.stream
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    shifts0 = sim.get_time()[1]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    diag = []
    e0.record(stream)
    run_steps(sim, ids, w, args.workload, args.steps, diag)
    e1.record(stream)
    sim.sync()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    shifts_timed = sim.get_time()[1] - shifts0
    ms = e0.elapsed_time(e1)
    n1 = sum(sim.get_count(s) for s in pushed)
    frozen1 = sim.get_count(ids["plasma_i"]) if "plasma_i" in ids else 0
    kernels_timed = None
    if graphs:
        kernels_timed = sim.trace_read()["kernels"]
        sim.trace_enable(True)
        sim.step(args.steps)
        sim.sync()
    tr = sim.trace_read()
    psteps = 0.5 * (n0 + n1) * args.steps
    psteps_all, ms_max = aggregate(psteps, ms, world, dev)
    value = psteps_all / (ms_max / 1000.0)

    # roofline of the dominant kernel class (live CUDA-event trace of the timed region): the
    # algorithmic bytes of one step's launches of that class over their CUDA-event time per step
    hbm, peak_kind = peaks()
    ncell = ncell_total
    n_beam = sim.get_count(ids["beam"])
    n_e = 0.5 * (n0 + n1) - n_beam
    classes = tr["ms"]
    steps_traced = args.steps      # the traced pass (the timed region, or the pass after it) has K steps
    dom = max(("push", "push_frozen", "fields", "sort"), key=lambda k: classes[k])
    shape = "CIC" if w.order == 1 else "TSC"
    launches = tr["events"][dom]
    if dom == "push":
        # one launch per mobile species per step; the grid term (E, B read once, J written once)
        # is counted once per step, not once per species launch
        bytes_step = (n_e + n_beam) * BYTES_PUSHED + ncell * BYTES_CELL_PUSH
        units = {"pushed_particles": int(round(n_e + n_beam)), "cells": int(ncell),
                 "bytes_per_pushed_particle": BYTES_PUSHED, "bytes_per_cell": BYTES_CELL_PUSH,
                 "weight_read_bytes_not_counted": BYTES_WEIGHT * (n_e + n_beam)}
    elif dom == "push_frozen":
        bytes_step = 0.5 * (frozen0 + frozen1) * BYTES_FROZEN + ncell * 12.0
        units = {"frozen_particles": int(0.5 * (frozen0 + frozen1)), "cells": int(ncell)}
    elif dom == "fields":
        bytes_step = ncell * (36.0 + 48.0 + 36.0)
        units = {"cells": int(ncell), "bytes_per_cell": 120.0}
    else:
        bytes_step = 3 * (n0 + frozen0) * 36.0
        units = {"particles": int(n0 + frozen0)}
    ms_step = classes[dom] / steps_traced
    achieved = bytes_step / (ms_step / 1000.0) / 1e9
    traffic = None
    if dom == "push" and args.workload == "buncher" and w.grid == (128, 128, 512):
        traffic = TRAFFIC_PUSH_BUNCHER_STEP
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic,
                "kernel": {"push": f"k_push<{shape}, mobile> (" + " + ".join(k for k in ("beam", "plasma_e") if k in ids) + ")",
                           "push_frozen": f"k_lattice / k_push<{shape}, frozen> (ions)", "fields": "k_fdtd_b/e",
                           "sort": "tile sort"}[dom],
                "per": "step (all launches of the kernel in one step)",
                "launches_per_step": launches / max(steps_traced, 1),
                "avg_launch_ms": classes[dom] / max(launches, 1),
                "ms_per_step": ms_step,
                "algorithmic_bytes_per_step": bytes_step,
                "units": units,
                "peak_kind": f"{peak_kind} (hbm_gbs)",
                "time_share": {k: v / max(sum(classes.values()), 1e-9) for k, v in classes.items() if v > 0}}
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # end to end through the C-ABI with host buffers: beam H2D from pinned memory, K steps,
    # moments D2H, on a fresh context (allocation and plasma fill are set-up, not timed)
    e2e = None
    if not args.no_e2e:
        x, u, wt = beam
        xh = torch.from_numpy(x).pin_memory()
        uh = torch.from_numpy(u).pin_memory()
        wh = torch.from_numpy(wt).pin_memory()
        if ens is not None:
            sim2, ids2 = api.from_ensemble(ens, device=local, beam=False)
        else:
            sim2, ids2 = api.from_workload(w, device=local, beam=False)
        sim2.sync()
        barrier()
        torch.cuda.synchronize()
        ne_plasma0 = sim2.get_count(ids2["plasma_e"]) if "plasma_e" in ids2 else 0
        t0 = time.perf_counter()
        b = w.beam
        match = bool(w.undulator is not None and w.undulator.match)
        if ens is not None:
            sb = sim2.load_species_batch(b.q, b.m, ens.n_beam, xh, uh, wh, frame=api.PIC_FRAME_LAB,
                                         origin=b.origin, match_undulator=match)
        else:
            sb = sim2.load_species(b.q, b.m, xh, uh, wh, frame=api.PIC_FRAME_LAB, origin=b.origin,
                                   match_undulator=match)
        # the long undulator's job includes its bunch's entry into the undulator (steps the
        # device-timed region leaves before its warm-up)
        ids2["beam"] = sb
        sim2.step(pre_steps)
        run_steps(sim2, ids2, w, args.workload, args.steps, [])
        mom = sim2.get_moments(sb, api.PIC_FRAME_LAB, k_bunch=0.0)
        t_e2e = time.perf_counter() - t0
        # particle counts for the metric, read outside the timed region
        ne0 = sim2.get_count(sb) + ne_plasma0
        ne1 = int(mom["count"]) + (sim2.get_count(ids2["plasma_e"]) if "plasma_e" in ids2 else 0)
        barrier()
        h2d = (xh.numel() + uh.numel() + wh.numel()) * 8
        n_e2e = pre_steps + args.steps
        e2e = {"value": 0.5 * (ne0 + ne1) * n_e2e * world / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": h2d / n_e2e, "d2h_bytes_per_step": 8 * 20 / n_e2e,
               "seconds": t_e2e, "steps": n_e2e}
        sim2.close()
        del sim2
        torch.cuda.empty_cache()

    adjoint = None
    if rank == 0 and world == 1 and args.workload == "buncher" and not args.no_adjoint:
        adjoint = adjoint_block(local)

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ncores, model = cpu_info()
        if args.workload == "vacuum":
            cv, ct, sample = oracle_sample_vacuum(20, 0)
        elif ens is not None:
            cv, ct, sample = oracle_sample_ensemble(2, 0)
        elif args.workload == "long_undulator":
            cv, ct, sample = oracle_sample_long(10, 0)
        else:
            cv, ct, sample = oracle_sample(3, 0)
        cpu = {"value": cv, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
               "cpu_model": model, "nproc": ncores}
        if args.workload == "buncher":
            av, at, used = oracle_sample_threads(10, ncores)
            cpu["all_cores"] = {"value": av, "unit": UNIT, "cores": used, "seconds": at,
                                "sample": "the same sub-box, 10 steps, the particle loop on all host cores "
                                          "(OpenMP, a private J per thread)"}
            # the FP32 path's error against the FP64 oracle, per result (this leg is where bench.py
            # runs the oracle)
            accuracy = fp32_vs_fp64(local, ncores)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.grid), "beam": int(n_beam),
                       "plasma_electrons": int(n_e), "frozen_ions": int(0.5 * (frozen0 + frozen1)),
                       "plasma_fill": (f"the lattice fills every cell that the transverse absorbing layers and "
                                       f"the shape's margins leave ({w.plasma.ppc[0] * w.plasma.ppc[1] * w.plasma.ppc[2]}"
                                       f" per cell there), not the whole grid" if w.plasma is not None else None),
                       "shape": shape, "boundaries": boundaries,
                       "tile": list(w.tile), "sort_every": tuned if tuned else w.sort_every,
                       "sort_every_from": "autotuner" if tuned else "workload",
                       "tile_from": "autotuner" if (tuned and ens is not None) else "workload",
                       "l2": l2,
                       "window_shifts_in_timed_region": int(shifts_timed),
                       "lab_bunching_every_100_steps": diag if diag else None,
                       "steps_before_warmup": int(pre_steps),
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "fp32_vs_fp64": accuracy, "adjoint": adjoint,
            "gpu_launches": int(kernels_timed if kernels_timed is not None else tr["kernels"]),
            "cuda_graphs": bool(graphs),
            "fallback_deposits": int(tr.get("fallback", 0)),
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gbpic", "reference"], default="gbpic")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle leg (CPU timing and the FP32-vs-FP64 accuracy block)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward block")
    ap.add_argument("--grid", default="",
                    help="grid of the plasma buncher (default 128,128,512) or the long undulator (default "
                         "256,256,1024); a smaller one, e.g. 64,64,128, for profiling captures")
    ap.add_argument("--beam", type=int, default=0, help="beam macroparticles (0: scaled with the grid)")
    ap.add_argument("--sort-every", type=int, default=0, help="steps between tile sorts (0: the workload's)")
    ap.add_argument("--tile", default="", help="buncher: tile size in cells, e.g. 8,4,4 (default: the workload's)")
    ap.add_argument("--runs", type=int, default=64, help="ensemble runs (the batched sweep has 64)")
    ap.add_argument("--no-autotune", action="store_true", help="ensemble: keep the workload's sort cadence")
    ap.add_argument("--autotune", action="store_true",
                    help="buncher, vacuum, long undulator: pick the sort cadence with the autotuner "
                         "(the default keeps the workload's 8)")
    ap.add_argument("--workload", choices=["buncher", "buncher2d", "long_undulator", "ensemble", "vacuum", "adjoint"],
                    default="buncher",
                    help="buncher: the plasma buncher 128x128x512 (default); ensemble: the batched sweep "
                         "of 64 runs of 64x64x128 in one context")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        raise SystemExit("need --steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    return run_gbpic(args)


if __name__ == "__main__":
    sys.exit(main())
