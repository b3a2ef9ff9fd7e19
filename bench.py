#!/usr/bin/env python
"""Benchmark of the fused IB-LBM-FEM time step on one GB300 per rank.

Workload (config 2 of the paper-shaped set-ups): 128^3 D3Q19 lattice, tau = 1,
wall-driven simple shear (shear rate 1e-3), one capsule of radius 16 on the
5120-face icosphere, Skalak C = 1, reduced shear rate G = 0.0125, 4-point delta,
FP32 populations.  One step = membrane forces + spreading, collide-and-stream,
interpolation + advection, and the FP64 capsule reductions behind the Taylor
deformation recorded on the device.  All of it runs in the library's CUDA
kernels through the C ABI.

Metric: MLUPS (lattice cell updates per second / 1e6) of the whole step,
summed over ranks (independent replicas, weak scaling).  Also reported: the
collide-and-stream kernel against the measured HBM bandwidth (152 algorithmic
bytes per FP32 cell update), membrane nodes/s, an end-to-end figure through
host buffers, the CPU oracle as a baseline, and SM clocks sampled during the
timed region.

`--impl reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fused IB-LBM step MLUPS & % HBM roofline; adjoint/forward time at 1e-4 rel error"
BYTES_PER_CELL = {"fp32": 152, "fp16": 76, "fp64": 304}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20000)
    p.add_argument("--warmup", type=int, default=200)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["config1", "config2", "config3", "config4", "config5",
                                          "convergence35", "convergence70", "convergence140"],
                   default="config2")
    p.add_argument("--delta", type=int, default=4, help="stencil of config 2 and the convergence workloads")
    p.add_argument("--G", type=float, default=0.0125, help="config 2 only")
    p.add_argument("--precision", default=None, help="override the workload's storage precision")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-budget-s", type=float, default=20.0)
    p.add_argument("--profile-steps", type=int, default=500)
    p.add_argument("--no-adjoint", action="store_true", help="skip the config-5 adjoint timing")
    p.add_argument("--record-every", type=int, default=1,
                   help="steps between device records of the capsule reductions (sub-step 6)")
    p.add_argument("--equilibrium", type=int, default=2, choices=[1, 2],
                   help="2: Eq. (equilibrium); 1: the linearised equilibrium of Sec. IV.A")
    p.add_argument("--integrator", type=int, default=0, choices=[0, 1],
                   help="node advection: 0 Euler, 1 Adams-Bashforth")
    p.add_argument("--interp-mode", type=int, default=-1, choices=[-1, 0, 1],
                   help="interpolation: -1 automatic, 0 gather at the stencil cells, 1 cell velocities first")
    p.add_argument("--launch-overlap", type=int, default=-1, choices=[-1, 0, 1],
                   help="step kernels with programmatic dependent launch: 1 on, 0 off, -1 automatic")
    p.add_argument("--deterministic-spreading", action="store_true",
                   help="force density summed in 64-bit fixed point (bit-reproducible steps)")
    p.add_argument("--collide-staging", type=int, default=-1, choices=[-1, 0, 1],
                   help="collide populations staged in shared memory by bulk copies: 1 on, 0 off, -1 automatic")
    p.add_argument("--adjoint-only", action="store_true",
                   help="only the config-5 adjoint timing, printed as {\"adjoint\": ...}")
    p.add_argument("--adjoint-steps", type=int, default=None,
                   help="steps of the adjoint timing (default: the workload's 2000)")
    return p.parse_args()


def _workload(a):
    from paper_1004_2416_gb300 import workloads as W

    if a.workload == "config3":
        cases = W.config3_cases()
        if a.precision:
            for c in cases:
                c.precision = a.precision
        return Batch(cases)
    if a.workload == "config1":
        case = W.config1()
    elif a.workload == "config4":
        case = W.config4()
    elif a.workload == "config5":
        case = W.config5()
    elif a.workload.startswith("convergence"):
        # the coupled-convergence series of Sec. IV.C (phi from --delta, default 4)
        case = W.convergence_case(int(a.workload[len("convergence"):]), a.delta)
    else:
        case = W.config2(G=a.G, delta=a.delta)
    if a.precision:
        case.precision = a.precision
    return case


class Batch:
    """The 64 independent runs of config 3, advanced as one batch."""

    def __init__(self, cases):
        self.cases = cases
        self.name = f"config3-batch-{len(cases)}runs-24..64^3-fp32-phi3"
        self.precision = cases[0].precision
        self.delta = 3
        self.tau = 1.0
        self.capsules = [c.capsules[0] for c in cases]
        self.ncell = sum(c.ncell for c in cases)
        self.n_nodes = sum(c.n_nodes for c in cases)
        self.shape = cases[0].shape
        self.u_wall = cases[0].u_wall


def _make_sim(case, stream):
    from paper_1004_2416_gb300 import Sim

    if isinstance(case, Batch):
        sim = Sim.batch([(*c.shape, c.tau, c.u_wall) for c in case.cases], precision=case.precision,
                        delta_points=case.delta, stream=stream)
        for k, c in enumerate(case.cases):
            for cap in c.capsules:
                cid = sim.add_capsule_icosphere_in_run(k, cap.center, cap.radius, cap.subdivisions)
                sim.set_skalak(cap.k_s, cap.C, cid)
        sim.init_fluid(1)
        sim.autotune_tiles(5)
        return sim
    nx, ny, nz = case.shape
    sim = Sim(nx, ny, nz, tau=case.tau, precision=case.precision, delta_points=case.delta, stream=stream)
    sim.set_shear_walls(case.u_wall)
    for c in case.capsules:
        cid = sim.add_capsule_icosphere(c.center, c.radius, c.subdivisions)
        sim.set_skalak(c.k_s, c.C, cid)
    sim.init_fluid(1)
    return sim


def _config(case, a):
    if isinstance(case, Batch):
        sizes = sorted({c.shape[0] for c in case.cases})
        return {"workload": case.name, "runs": len(case.cases), "box_sides": sizes, "cells": case.ncell,
                "capsules": len(case.capsules), "membrane_nodes": case.n_nodes,
                "faces_per_capsule": "320 (r <= 4) or 1280", "delta_points": 3,
                "reduced_shear_rate_G": "log-uniform in [0.003, 0.1], seed 3", "tau": 1.0,
                "storage": f"{case.precision} deviations from rest equilibrium",
                "step": "forces+spread, persistent batched collide-stream, interpolate+advect, "
                        "FP64 Taylor reductions recorded",
                "l2": f"inputs larger than L2: two population buffers of "
                      f"{case.ncell * BYTES_PER_CELL[case.precision] / 2 / 1e6:.0f} MB each",
                "parallelism": "replicas (one independent batch per rank)"}
    c = case.capsules[0]
    return {
        "workload": case.name,
        "lattice": list(case.shape),
        "cells": case.ncell,
        "capsules": len(case.capsules),
        "membrane_nodes": case.n_nodes,
        "faces": 20 * 4 ** c.subdivisions,
        "radius": c.radius,
        "delta_points": case.delta,
        "reduced_shear_rate_G": round(c.radius * (case.tau - 0.5) / 3.0 * 2.0 * case.u_wall / case.shape[2] / c.k_s, 6),
        "k_s": c.k_s,
        "u_wall": case.u_wall,
        "tau": case.tau,
        "storage": f"{case.precision} deviations from rest equilibrium",
        "step": "forces+spread, collide-stream, interpolate+advect, FP64 Taylor reductions recorded",
        "record_every": a.record_every,
        "equilibrium": "second order, Eq. (equilibrium)" if a.equilibrium == 2 else "linearised, Sec. IV.A",
        "advection": "Euler" if a.integrator == 0 else "Adams-Bashforth",
        "spreading": "64-bit fixed point (deterministic)" if a.deterministic_spreading else "float atomics",
        "l2": f"inputs larger than L2: two population buffers of {19 * case.ncell * BYTES_PER_CELL[case.precision] // 38 / 1e6:.0f} MB each",
        "parallelism": "replicas (one independent simulation per rank)",
    }


# ---- distributed plumbing ------------------------------------------------------

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_mlups(world_size: int, cells_per_rank: int, steps: int, ms_max: float) -> float:
    """Whole-job throughput of independent replicas (weak scaling): every rank
    advanced its own lattice of cells_per_rank cells by `steps` steps, and the
    slowest rank's time (ms_max, the max over ranks) is the job's time."""
    return world_size * cells_per_rank * steps / (ms_max * 1e-3) / 1e6


class _Group:
    def __init__(self, backend):
        self.ws, self.rank, self.local = _dist()
        self.pg = None
        if self.ws > 1:
            import torch.distributed as dist

            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---- clocks -------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.p = None
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if not self.p:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(self.REASONS, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _gpu_index(local: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [v for v in vis.split(",") if v.strip()]
    if parts and local < len(parts) and parts[local].strip().isdigit():
        return int(parts[local])
    return local


# ---- roofline helpers --------------------------------------------------------------------

def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _kernel_source_hash() -> str:
    """Hash of the sources that define the collide-and-stream kernels."""
    h = hashlib.sha256()
    for f in ("lbm.cu", "device_common.cuh"):
        with open(os.path.join(ROOT, "paper_1004_2416_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(workload: str, precision: str):
    """DRAM bytes per collide-and-stream launch from the committed ncu summary,
    or None when the summary is absent or was taken on other kernel source."""
    path = os.path.join(ROOT, "profiles", f"collide_stream_{workload}_{precision}.txt")
    try:
        kv = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != _kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


# ---- CPU oracle ------------------------------------------------------------------------------

def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_run(case, budget_s: float, max_steps: int, a=None, threads: int = 1):
    """Times the FP64 oracle on the full workload: one untimed step, then as many
    timed steps as fit in the budget (at least one, at most max_steps), with the
    method variants of the run's arguments, its whole-lattice loops on
    `threads` host threads (results do not depend on the count)."""
    import oracle as O

    O.build()
    O.set_threads(threads)
    nx, ny, nz = case.shape
    o = O.Sim(nx, ny, nz, case.tau, case.delta, case.u_wall)
    for c in case.capsules:
        X0, tri = O.icosphere(c.subdivisions, c.radius, c.center)
        o.add_capsule(X0, tri, c.k_s, c.C * c.k_s)
    if a is not None:
        o.set_equilibrium(getattr(a, "equilibrium", 2))
        o.set_integrator(getattr(a, "integrator", 0))
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    n = int(max(1, min(max_steps, budget_s // max(t1, 1e-9))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    o.close()
    O.set_threads(1)
    return n, dt


def _cpu_leg(case, a, budget_s, threads):
    """(MLUPS, sample text) of the oracle on `threads` host threads."""
    if isinstance(case, Batch):
        cells_done, dt = 0, 0.0
        for c in case.cases:
            n, t = _oracle_run(c, budget_s / len(case.cases), a.steps, a, threads)
            cells_done += c.ncell * n
            dt += t
        return cells_done / dt / 1e6, (f"every run of the batch stepped by the FP64 oracle for a bounded "
                                       f"number of steps each, {dt:.1f} s in total")
    n, dt = _oracle_run(case, budget_s, a.steps, a, threads)
    return case.ncell * n / dt / 1e6, (f"{n} full FP64 oracle steps of the same workload after one untimed "
                                       f"step, {dt:.1f} s")


def _cpu_baseline(case, a):
    """The oracle as it stands, timed on the host's cores: all of them (the
    reported value) and one (beside it)."""
    cores = _host_cores()
    v_all, s_all = _cpu_leg(case, a, a.cpu_budget_s, cores)
    v_one, s_one = _cpu_leg(case, a, a.cpu_budget_s, 1)
    return {"value": round(v_all, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{s_all}; whole-lattice loops on {cores} OpenMP threads, spreading, membrane forces "
                      f"and reductions serial",
            "cpu_model": _cpu_model(), "nproc": os.cpu_count(),
            "single_core": {"value": round(v_one, 4), "unit": "MLUPS", "cores": 1, "sample": s_one}}


# ---- adjoint timing (config 5) ---------------------------------------------------------------------

def _adjoint_timing(stream, steps=None):
    """Config 5 (64^3, FP32, one 1280-face capsule, phi3): 2000 steps forward with
    checkpoints every 100 steps, then the reverse sweep for dD/dk_s, dD/du_wall and
    dD/dX0; host wall-clock times of both, each ending in a synchronisation.  The
    gradient is compared with the FP64 oracle's central differences when the
    reference file is present and the run has the workload's full length."""
    import importlib.util

    import numpy as np
    import torch

    from paper_1004_2416_gb300 import workloads as W

    case = W.config5()
    n_steps = case.steps if steps is None else max(100, 100 * (steps // 100))
    sim = _make_sim(case, stream)
    X0 = sim.get_nodes()
    sim.adjoint_forward(200, 100)  # warm-up: kernels, graphs and reverse-sweep buffers
    sim.adjoint_backward(0)

    def reset():
        sim.init_fluid(1)
        sim.set_nodes(X0)
        torch.cuda.synchronize()

    reset()
    t0 = time.perf_counter()
    sim.step(n_steps)
    sim.sync()
    plain = time.perf_counter() - t0
    reset()
    t0 = time.perf_counter()
    sim.adjoint_forward(n_steps, 100)
    fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = sim.adjoint_backward(0)
    bwd = time.perf_counter() - t0
    out = {"workload": case.name, "steps": n_steps, "checkpoint_every": 100,
           "plain_forward_ms": round(plain * 1e3, 2), "forward_with_checkpoints_ms": round(fwd * 1e3, 2),
           "backward_ms": round(bwd * 1e3, 2), "backward_over_forward": round(bwd / plain, 3),
           "D": r["D"], "dD_dks": r["dD_dks"], "dD_duw": r["dD_duw"],
           "dD_dG": r["dD_duw"] * case.capsules[0].k_s * case.shape[2] / (2.0 * (case.tau - 0.5) / 3.0 * case.capsules[0].radius)}
    path = os.path.join(ROOT, "tests", "golden", "adjoint_fd_config5.json")
    if os.path.exists(path) and n_steps == case.steps:
        with open(path) as fh:
            fd = json.load(fh)
        spec = importlib.util.spec_from_file_location("mkfd", os.path.join(ROOT, "tests", "golden", "make_adjoint_fd.py"))
        mk = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mk)
        g = r["dD_dX0"] + r["dD_dx0"]
        dirs = mk.directions(len(g), fd["n_directions"], fd["directions_seed"])
        gn = float(np.linalg.norm(g))
        out["vs_oracle_fd"] = {
            "dD_dks_rel": abs(r["dD_dks"] - fd["dD_dks"]) / abs(fd["dD_dks"]),
            "dD_duw_rel": abs(r["dD_duw"] - fd["dD_duw"]) / abs(fd["dD_duw"]),
            "dD_dX0_directions_err_over_norm": [abs(float(np.sum(g * d)) - b) / gn
                                                for d, b in zip(dirs, fd["dD_dX0_along"])],
            "D_rel": abs(r["D"] - fd["D"]) / abs(fd["D"]),
        }
    sim.close()
    return out


# ---- our arm ------------------------------------------------------------------------------------

def run_ours(a):
    import numpy as np
    import torch

    from paper_1004_2416_gb300 import iblbm as B

    grp = _Group("nccl")
    torch.cuda.set_device(grp.local)
    if a.adjoint_only:
        out = _adjoint_timing(torch.cuda.Stream(), a.adjoint_steps)
        grp.close()
        if grp.rank == 0:
            print(json.dumps({"adjoint": out}), flush=True)
        return
    case = _workload(a)
    batch = isinstance(case, Batch)
    stream = torch.cuda.Stream()
    sim = _make_sim(case, stream)
    sim.set_interp_mode(a.interp_mode)
    sim.set_launch_overlap(a.launch_overlap)
    if not batch:
        sim.set_collide_staging(a.collide_staging)
        if a.deterministic_spreading:
            sim.set_deterministic_spreading(True)
    sim.set_equilibrium(a.equilibrium)
    sim.set_integrator(a.integrator)
    batch = isinstance(case, Batch)
    sim.set_taylor_recording(a.record_every, ring=(a.steps + a.warmup) // max(1, a.record_every) + 4096)
    # the captured step graphs carry event nodes around each kernel group, so
    # the kernel times below come from the timed steps themselves
    sim.set_kernel_timing(True)

    sim.step(a.warmup)
    # capture (not run) the graphs of the timed call, so the timed region
    # holds graph launches only
    sim.prepare_steps(a.steps)
    sim.sync()
    sim.kernel_times()  # forget the warm-up's timings
    torch.cuda.synchronize()
    sampler = ClockSampler(_gpu_index(grp.local))
    time.sleep(0.3)
    grp.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    launches0 = sim.info().kernel_launches
    start.record(stream)
    sim.step(a.steps)
    end.record(stream)
    launches = sim.info().kernel_launches - launches0  # the library's own count of its kernels
    end.synchronize()
    torch.cuda.synchronize()
    grp.barrier()
    clocks = sampler.stop()
    ms = start.elapsed_time(end)
    sim.sync()  # raises on any device-side error of the timed region
    live = sim.kernel_times()  # kernel groups of the timed steps (last replay of each graph)
    ms_max = grp.max(ms)
    cells = case.ncell
    value = aggregate_mlups(grp.ws, cells, a.steps, ms_max)
    nodes_per_s = grp.ws * case.n_nodes * a.steps / (ms_max * 1e-3)
    steps_rec, rec = sim.taylor_records(0, max_records=1)
    D_last = float(rec[-1][0]) if len(rec) else None
    final_shape = None
    if not batch and case.capsules:
        # diagnostics of capsule 0 after the timed steps (host side, untimed)
        T = sim.taylor(0)
        fit = B.ellipsoid_fit(sim.get_nodes(0), [T["c_x"], T["c_y"], T["c_z"]])
        q = sim.mesh_quality(0)
        final_shape = {"D": T["D"], "theta": T["theta"], "D_ellipsoid_fit": fit["D"],
                       "theta_ellipsoid_fit": fit["theta"], "face_area_dev_mean": q["dA_mean"],
                       "face_area_dev_std": q["dA_std"], "volume_drift": q["dV"]}

    # the Taylor record's device time, which runs on a side stream in the
    # timed steps: profile mode (kernels launched one by one, the record on
    # the main stream between events)
    prof = sim.profile_kernels(a.profile_steps)
    sim.sync()
    peak, peak_kind = _peaks()
    algo_bytes = BYTES_PER_CELL[case.precision] * cells
    k_ms = live["collide_stream"]
    achieved = algo_bytes / (k_ms * 1e-3) / 1e9
    traffic = _ncu_traffic(a.workload, case.precision)
    step_ms = ms_max / a.steps
    roofline = {"kernel": sim.collide_kernel(), "bound": "hbm", "achieved": round(achieved, 1),
                "peak": peak, "peak_kind": f"{peak_kind} copy bandwidth", "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": algo_bytes, "kernel_ms": round(k_ms, 5),
                "kernel_ms_from": f"CUDA events in the timed step graphs, on a branch forked from the "
                                  f"launching stream after the kernel before and after this one (the last "
                                  f"replay of each graph: {live['steps']} steps)",
                "kernel_ms_profile_mode": round(prof["collide_stream"], 5),
                # the whole step against the same peak: algorithmic bytes of the
                # collide (the only HBM-sized traffic of a step) over ms_per_step
                "whole_step_frac": round(algo_bytes / (step_ms * 1e-3) / 1e9 / peak, 4),
                "dram_frac": (round(traffic / (k_ms * 1e-3) / 1e9 / peak, 4) if traffic else None)}

    # end to end through the C ABI with pinned host buffers: the state is
    # uploaded, then every step is enqueued with an asynchronous read-back of
    # all node positions and the capsule reductions into pinned host memory
    # (two alternating buffers), and the run ends when the stream has
    # delivered the last step's results
    e2e = None
    if not a.no_e2e and not batch:
        nx, ny, nz = case.shape
        n_caps = len(case.capsules)
        f_host = torch.empty(19 * cells, dtype=torch.float64, pin_memory=True).numpy().reshape(19, nz, ny, nx)
        x_host = torch.empty(case.n_nodes * 3, dtype=torch.float64, pin_memory=True).numpy().reshape(-1, 3)
        out_nodes = [torch.empty(case.n_nodes * 3, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        out_sums = [torch.empty(n_caps * 12, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        f_host[...] = sim.get_populations()
        x_host[...] = sim.get_nodes()
        import ctypes

        h = sim.handle
        k_e2e = a.steps
        sim.set_taylor_recording(0, 1)  # the read-back reduces the capsules of every step itself
        sim.set_kernel_timing(False)  # a user's steps carry no timing events
        p_nodes = [ctypes.c_void_p(b.ctypes.data) for b in out_nodes]
        p_sums = [ctypes.c_void_p(b.ctypes.data) for b in out_sums]
        # capture the one-step graphs of both buffer parities and make the
        # read-back's device buffers exist (untimed; the timed region uploads
        # the state again)
        for k in range(2):
            B.iblbm_step(h, 1)
            B.iblbm_read_async(h, p_nodes[k], p_sums[k])
        sim.sync()
        grp.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.set_populations(f_host)
        sim.set_nodes(x_host)
        for k in range(k_e2e):
            rc = B.iblbm_step(h, 1)
            rc = rc or B.iblbm_read_async(h, p_nodes[k & 1], p_sums[k & 1])
            if rc:
                raise B.IblbmError(rc, B.iblbm_last_error(h).decode())
        rc = B.iblbm_sync(h)
        if rc:
            raise B.IblbmError(rc, B.iblbm_last_error(h).decode())
        dt = time.perf_counter() - t0
        dt_max = grp.max(dt)
        last = (k_e2e - 1) & 1
        D_last = B.taylor_from_sums(out_sums[last][:12])["D"]
        D_now = sim.taylor(0)["D"]
        if not abs(D_last - D_now) <= 1e-12 * max(1.0, abs(D_now)):
            raise RuntimeError(f"asynchronous read-back gave D = {D_last}, the getter {D_now}")
        e2e = {"value": round(grp.ws * cells * k_e2e / dt_max / 1e6, 2), "unit": "MLUPS",
               "steps": k_e2e,
               "h2d_bytes_per_step": int((19 * cells * 8 + case.n_nodes * 24) / k_e2e),
               "d2h_bytes_per_step": case.n_nodes * 24 + n_caps * 12 * 8,
               "note": "timed region: upload of the state from pinned host memory, then per step "
                       "iblbm_step(1) + iblbm_read_async of all node positions and the capsule reductions "
                       "into pinned host memory (two alternating buffers), then iblbm_sync"}

    cpu = None
    if grp.rank == 0 and grp.ws == 1 and not a.no_cpu_baseline:
        cpu = _cpu_baseline(case, a)

    adjoint = None
    if grp.rank == 0 and not a.no_adjoint and a.workload == "config2":
        adjoint = _adjoint_timing(stream, a.adjoint_steps)

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": grp.ws,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms_max / a.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if case.precision == "fp32" else ("f16-storage/f32" if case.precision == "fp16" else "f64"),
        "data": "synthetic", "config": _config(case, a),
        "membrane_nodes_per_s": round(nodes_per_s, 1),
        "kernel_ms_per_step": {"force_spread": round(live["force_spread"], 5),
                               "collide_stream": round(live["collide_stream"], 5),
                               "interp_advect": round(live["interp_advect"], 5),
                               "taylor_record_profile_mode": round(prof["taylor"], 5),
                               "note": "first three: CUDA event nodes in the timed step graphs; their sum "
                                       "is the main stream's step minus graph and join gaps; the Taylor "
                                       "record runs beside them on a side stream (its time here from "
                                       "profile mode, kernels launched one by one)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": int(launches),
        "final_D": D_last,
        "final_shape": final_shape,
        "adjoint": adjoint,
    }
    sim.close()
    grp.close()
    if grp.rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    case = _workload(a)
    w = min(a.warmup, 1)
    cores = _host_cores()
    n, dt = _oracle_run(case, max(a.cpu_budget_s, 30.0), a.steps, a, cores)
    value = case.ncell * n / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS", "n_gpus": ws,
        "steps": n, "warmup": w, "ms_per_step": round(dt / n * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(case, a),
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{n} full FP64 oracle steps of the workload (of {a.steps} requested; "
                                   f"an oracle step of 2.1 M cells takes a fraction of a second on all "
                                   f"cores), after 1 untimed step; whole-lattice loops on {cores} OpenMP "
                                   f"threads, spreading, membrane forces and reductions serial",
                         "cpu_model": _cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
