"""Throughput benchmark of the fused Bingham LBM step on GB300.

Workload: 3D square duct, D3Q27, 256 (x, streamwise, periodic) x 128 x 128
cells with solid rows y = 0 and z = 0 (127 x 127 fluid cross-section,
4,129,024 fluid cells), body force along x, Bn = 2 (a-posteriori, mapped to
the yield stress through the Mosolov-Miasnikov duct formula), nu_p = 0.1,
FP32 population storage, started from rest.  One bench "step" is one pass of
the whole hot path for BOTH Bingham models, each on its own copy of the duct
(PR with m = 1e6 and IR): one check interval of 100 lattice time steps, 99
plain fused stream-and-collide steps and one check step that also computes
the flow rate and the residual (with its FP64 finaliser).  The metric is
MLUPS: fluid-cell updates per second (all_cell_mlups counts the solid cells
too).

Timing: W untimed warm-up steps, then K timed steps bracketed by a barrier and
cudaDeviceSynchronize, measured with CUDA events on the solvers' stream (the
IR phase and the PR phase each have their own events, which gives each
kernel's average launch duration).  The populations (2 x 905 MB) are far
larger than L2, so no flush is needed between steps.

Also reported, outside the timed region: the porous box of the porous-medium
workload (256^3, D3Q19, FP32 and FP16 storage, both models) with its own
roofline, the precision workload's 512x192x192 duct and 512^3 porous box
(D3Q27, FP32 and FP16; the box in the compact layout), the
same metric end to end through the C ABI with host buffers, and the
continuous-batching server on a Poisson stream of independent solves run to
steady state.

--impl reference times the FP64 CPU oracle (the correctness reference) on
the host cores, on a bounded sample of the same duct, one sample per step.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D3Q27 Bingham MLUPS and % HBM roofline; served solves/s, p50/p99 latency"
NX, NY, NZ = 256, 128, 128
LATTICE = "D3Q27"
STORAGE = "F32"
STORAGE_CTYPE = {"F32": "float", "F64": "double", "F16": "__half", "BF16": "__nv_bfloat16"}
STORAGE_DTYPE = {"F32": "f32", "F64": "f64", "F16": "f16 storage / f32 arithmetic",
                 "BF16": "bf16 storage / f32 arithmetic"}
NU_P = 0.1
BN = 2.0
M_PR = 1e6
CHECK_EVERY = 100     # lattice steps per check step; one bench step = one check interval
SAMPLE_NX = 4          # x-extent of the oracle's sample of the duct (periodic along x)
POROUS = 0             # > 0: a porous box of this side replaces the duct


def workload_params():
    from paper_1610_01388_gb300 import workloads as W
    if POROUS:
        prm = W.porous_params(nu_p=NU_P, d_mean=16.0, g=2e-5, bn=BN)
        return prm["g"], prm["sigma_y"]
    prm = W.duct_params(H=NY - 1, nu_p=NU_P, u_newton=0.02, bn=BN)
    return prm["g"], prm["sigma_y"]


def workload_config(extra=None):
    q = {"D3Q15": 15, "D3Q19": 19}.get(LATTICE, 27)
    pop_mb = 2 * q * NX * NY * NZ * {"F64": 8, "F32": 4}.get(STORAGE, 2) / 1e6
    cfg = {"workload": f"square duct {LATTICE} {NX}x{NY}x{NZ} ({NY - 1}x{NZ - 1} fluid "
                       "cross-section), "
                       f"PR (m={M_PR:g}) + IR per step, Bn={BN:g}, nu_p={NU_P}, {STORAGE} populations, "
                       f"check step every {CHECK_EVERY}",
           "bench_step": f"{CHECK_EVERY} lattice time steps of each model: {CHECK_EVERY - 1} plain "
                         "fused steps + 1 check step (flow rate, residual, FP64 finaliser)",
           "lattice": LATTICE, "nx": NX, "ny": NY, "nz": NZ, "models": ["PR", "IR"],
           "storage": STORAGE,
           "l2": f"inputs {'larger' if pop_mb > 129 else 'smaller'} than L2 (populations per model: "
                 f"{pop_mb:.0f} MB)"}
    if POROUS:
        cfg.update({"workload": f"porous box {LATTICE} {POROUS}^3 (random non-overlapping spheres, "
                                "radius 6-10, porosity 0.7, seed 1), "
                                f"PR (m={M_PR:g}) + IR per step, Bn={BN:g}, nu_p={NU_P}, "
                                f"{STORAGE} populations, check step every {CHECK_EVERY}",
                    "nx": POROUS, "ny": POROUS, "nz": POROUS})
    if extra:
        cfg.update(extra)
    return cfg


def workload_mask(nx=None):
    """The bench's geometry: the square duct, or the porous box of --porous
    (its first nx x-layers when nx is given)."""
    from paper_1610_01388_gb300 import workloads as W
    if POROUS:
        m = W.porous_mask(POROUS, porosity=0.7, r_min=6.0, r_max=10.0, seed=1)[0]
        return np.ascontiguousarray(m[:, :, :nx]) if nx else m
    return W.duct_mask(nx or NX, NY, NZ)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# step kernels, from ncu captures of this script (the commands are in the
# profiles/ summaries).  NCU_TRAFFIC: the 256x128x128 D3Q27 duct, keyed by
# storage, model, block size and cells per thread.  NCU_TRAFFIC_POROUS: the
# porous box of the porous record (256^3, D3Q19, 256 threads), keyed by
# layout, storage and model.  Both are valid only
# for the device-code sources they were captured with (KERNEL_FINGERPRINT)
# and are reported as null once any of those sources changes.
NCU_TRAFFIC_POROUS = {
    ('compact', 'F16', 'IR'): 1017978014, ('compact', 'F16', 'PR'): 1113269616,
    ('compact', 'F32', 'IR'): 1903769109, ('compact', 'F32', 'PR'): 1998954998,
    ('dense', 'F16', 'IR'): 1249633474, ('dense', 'F16', 'PR'): 1377774772,
    ('dense', 'F32', 'IR'): 2433578501, ('dense', 'F32', 'PR'): 2559411298,
}
NCU_TRAFFIC = {
    ('F16', 'IR', 128, 1): 420014114, ('F16', 'IR', 128, 2): 419242511, ('F16', 'IR', 256, 1): 419807719, ('F16', 'IR', 256, 2): 420148489, ('F16', 'IR', 512, 1): 420246713,
    ('F16', 'PR', 128, 1): 451687740, ('F16', 'PR', 128, 2): 450993049, ('F16', 'PR', 256, 1): 451128599, ('F16', 'PR', 256, 2): 451178877, ('F16', 'PR', 512, 1): 451255470,
    ('F32', 'IR', 128, 1): 855939396, ('F32', 'IR', 128, 2): 855419924, ('F32', 'IR', 256, 1): 855652990, ('F32', 'IR', 256, 2): 857036609, ('F32', 'IR', 512, 1): 857513376,
    ('F32', 'PR', 128, 1): 889867913, ('F32', 'PR', 128, 2): 889934811, ('F32', 'PR', 256, 1): 889658765, ('F32', 'PR', 256, 2): 890827582, ('F32', 'PR', 512, 1): 890181304,
}
KERNEL_FINGERPRINT = "49211dcd9ff1d162"
KERNEL_SOURCES = ("kernels.cuh", "lattice.cuh", "lbm_internal.h", "fastdiv.h", "kern_d3q27.cu",
                  "kern_d3q19.cu")


def kernel_fingerprint():
    """SHA-256 of the device-code sources without comments and blank space
    (a comment edit does not change what was captured)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1610_01388_gb300", "csrc", name)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(storage, model, block, cpt, override=None, workload="duct", layout="dense"):
    if override is not None:
        return override
    if KERNEL_FINGERPRINT is None or kernel_fingerprint() != KERNEL_FINGERPRINT:
        return None
    if workload == "porous":
        return NCU_TRAFFIC_POROUS.get((layout, storage, model))
    if POROUS or (LATTICE, NX, NY, NZ) != ("D3Q27", 256, 128, 128):
        return None
    return NCU_TRAFFIC.get((storage, model, block, cpt))


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --- distributed plumbing -----------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value, backend_device=None):
    """Max of a float over ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=backend_device if backend_device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def aggregate(updates_per_rank, max_seconds, world_size):
    """Whole-job MLUPS: every rank processes the same number of updates."""
    return updates_per_rank * world_size / max_seconds / 1e6


# --- clocks --------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)], stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(parts)
                except Exception:
                    pass
        os.unlink(self.path)
        if not rows:
            return None
        sm = []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        smax = None
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# --- our arm ----------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1610_01388_gb300 import _build, lbm
    from paper_1610_01388_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if not os.path.exists(lbm.LIB_PATH):
        _build.build()
    dev = torch.device("cuda", local)
    g, sy = workload_params()
    mask = workload_mask()
    nfluid = int((mask == 0).sum())

    # the project's autotuner picks the step kernel's block size for this
    # problem class (outside the timed region)
    tuned = {}
    if not args.no_tune:
        from paper_1610_01388_gb300 import autotune
        for model in ("IR", "PR"):
            best, times = autotune.tune(LATTICE, model, STORAGE, mask.size, steps=200, mask=mask)
            tuned[model] = {"block": best[0], "cells_per_thread": best[1],
                            "us_per_step": {f"{b}x{c}": round(t * 1e6, 2)
                                            for (b, c), t in times.items()}}

    solvers = {}
    for model in ("IR", "PR"):
        solvers[model] = lbm.Solver(LATTICE, mask, model=model, storage=STORAGE, mu_p=NU_P,
                                    sigma_y=sy, m=M_PR, g=(g, 0.0, 0.0),
                                    check_every=CHECK_EVERY, use_torch=True)
    stream = torch.cuda.current_stream(dev)

    # warm-up (also captures the CUDA graphs)
    for model in ("IR", "PR"):
        solvers[model].step(args.warmup * CHECK_EVERY)
    torch.cuda.synchronize(dev)

    K = args.steps                 # bench steps
    NL = K * CHECK_EVERY           # lattice time steps per model
    # events between bench steps: IR's K bench steps, then PR's
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K + 1)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ev[0].record(stream)
    for m, model in enumerate(("IR", "PR")):
        for k in range(K):
            solvers[model].step(CHECK_EVERY)
            ev[m * K + k + 1].record(stream)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    barrier()
    clk = clocks.stop()
    ms_ir = ev[0].elapsed_time(ev[K])
    ms_pr = ev[K].elapsed_time(ev[2 * K])
    # per bench step (both models): the IR and the PR part of step k
    step_ms = [ev[k].elapsed_time(ev[k + 1]) + ev[K + k].elapsed_time(ev[K + k + 1])
               for k in range(K)]
    ms_total = ms_ir + ms_pr
    max_s = reduce_max(ms_total / 1e3, dev if ws > 1 else None)
    value = aggregate(2.0 * nfluid * NL, max_s, ws)

    # residual sanity (the run must stay finite)
    for model in ("IR", "PR"):
        solvers[model].residual()

    info_ir = solvers["IR"].info
    info_pr = solvers["PR"].info
    peak, peak_kind = measured_hbm_peak()
    launches_per_model = NL + NL // CHECK_EVERY   # step kernels + check-step finalisers
    per = {}
    for model, ms, inf in (("IR", ms_ir, info_ir), ("PR", ms_pr, info_pr)):
        t_launch = ms / 1e3 / NL
        gbs = inf.bytes_per_fluid_update * nfluid / t_launch / 1e9
        per[model] = {"bytes_per_update": inf.bytes_per_fluid_update, "launch_us": t_launch * 1e6,
                      "achieved_gbs": gbs, "frac": gbs / peak,
                      "mlups": nfluid / t_launch / 1e6}
    dom = "PR" if ms_pr >= ms_ir else "IR"
    roof = {"bound": "hbm",
            "kernel": (f"{'k_step2' if tuned.get(dom, {}).get('cells_per_thread', 1) == 2 else 'k_step'}"
                       f"<{LATTICE},{dom},{STORAGE_CTYPE[STORAGE]}> (dominant by time)"),
            "achieved": round(per[dom]["achieved_gbs"], 1), "peak": peak,
            "peak_kind": f"{peak_kind} (copy bandwidth)", "unit": "GB/s",
            "frac": round(per[dom]["frac"], 4),
            "bytes_per_fluid_update": per[dom]["bytes_per_update"],
            "fluid_cells_per_launch": nfluid,
            "traffic": ncu_traffic(STORAGE, dom, tuned.get(dom, {}).get("block", 256),
                                   tuned.get(dom, {}).get("cells_per_thread", 1), args.traffic),
            "per_model": {k: {kk: round(vv, 4) if isinstance(vv, float) else vv
                              for kk, vv in v.items()} for k, v in per.items()}}
    for s in solvers.values():
        s.close()
    del solvers
    torch.cuda.synchronize(dev)

    e2e = run_e2e(args, mask, nfluid, g, sy, dev)
    steady = run_steady(args, mask, nfluid, g, sy) if args.steady else None
    porous = run_porous_record(args) if (args.porous_record > 0 and not POROUS) else None
    precision = (run_precision_record(args)
                 if (args.precision_steps > 0 and not POROUS and LATTICE == "D3Q27") else None)
    serving = None
    if args.serve_requests > 0:
        serving = {"form": "served FP16-offset storage (stochastic rounding) vs FP32, batched; "
                           "mixed: FP16 with the near-jammed porous requests (a-priori Bn >= 1) "
                           "in FP32",
                   "budget_gb": 120, "rate_per_s": args.serve_rate,
                   "steady_state": (f"{args.serve_criterion} criterion: "
                                    + ("relative change of the mean velocity vector"
                                       if args.serve_criterion == "flow" else "field residual")
                                    + f" between check steps {args.serve_check_every} steps "
                                      f"apart < {args.serve_tolerance:g}"),
                   "step_cap": args.serve_max_steps,
                   "mix": SERVE_MIX_FULL if args.serve_full else SERVE_MIX,
                   "plain_fp32_single_domain_mlups": round(value, 1),
                   "runs": [run_serving(args, st) for st in args.serve_storage.split(",")]}
    cpu = run_cpu_baseline(args) if (rank == 0 and ws == 1 and not args.no_cpu) else None
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws,
                "steps": K, "warmup": args.warmup, "ms_per_step": round(max_s * 1e3 / K, 5),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": STORAGE_DTYPE[STORAGE], "data": "synthetic",
                "config": workload_config({"per_rank": "independent duct pair per GPU",
                                           "fluid_cells": nfluid, "autotuned": tuned}),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "porous": porous,
                "precision": precision,
                "serving": serving, "time_to_steady": steady,
                "ms_per_step_median": round(statistics.median(step_ms), 5),
                "ms_per_step_spread": [round(min(step_ms), 5), round(max(step_ms), 5)],
                "gpu_launches": 2 * launches_per_model, "clocks": clk,
                "all_cell_mlups": round(value * mask.size / nfluid, 1),
                "wall_s_timed_region": round(t1 - t0, 4)}
        print(json.dumps(line), flush=True)
    if ws > 1 and dist.is_initialized():
        dist.destroy_process_group()


def run_steady(args, mask, nfluid, g, sy):
    """Time to steady state of the start-up flow (both models, from rest):
    check every 1000 steps, steady when the residual between consecutive
    checks, sqrt(sum |u - u_prev|^2 / sum |u|^2), falls below the tolerance."""
    import torch
    from paper_1610_01388_gb300 import lbm
    out = {"tolerance": args.steady_tol, "check_every": 1000, "step_cap": args.steady_cap}
    for model in ("IR", "PR"):
        s = lbm.Solver(LATTICE, mask, model=model, storage=STORAGE, mu_p=NU_P, sigma_y=sy,
                       m=M_PR, g=(g, 0.0, 0.0), check_every=1000, use_torch=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, r = 0, -1.0
        while steps < args.steady_cap:
            s.step(1000)
            steps += 1000
            r, _, _ = s.residual()
            if 0.0 <= r < args.steady_tol:
                break
        dt = time.perf_counter() - t0
        out[model] = {"steps": steps, "seconds": round(dt, 3), "residual": r,
                      "steady": bool(0.0 <= r < args.steady_tol),
                      "flow_rate_x": s.flowrate(0), "mlups": round(nfluid * steps / dt / 1e6, 1)}
        s.close()
    return out


def run_e2e(args, mask, nfluid, g, sy, dev):
    """The same metric through the public C ABI with host buffers: per model a
    solve = lbm_create from the host mask (H2D), lbm_step(K), lbm_fields to
    host (D2H of rho and u), lbm_destroy; all inside the timed region."""
    import torch
    from paper_1610_01388_gb300 import lbm
    K = (args.e2e_steps if args.e2e_steps > 0 else args.steps) * CHECK_EVERY   # lattice steps
    # pinned host buffers for the read-back
    rho = torch.empty(mask.size, dtype=torch.float64, pin_memory=True).numpy()
    u = torch.empty((3, mask.size), dtype=torch.float64, pin_memory=True).numpy()
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for model in ("IR", "PR"):
        p = lbm.lbm_params_default(model=model, storage=STORAGE, mu_p=NU_P, sigma_y=sy, m=M_PR,
                                   g=(g, 0.0, 0.0), check_every=CHECK_EVERY)
        h = lbm.lbm_create(LATTICE, mask, p)
        lbm.lbm_step(h, K)
        lib = lbm.library()
        import ctypes
        vp = ctypes.c_void_p
        lbm._check(lib.lbm_fields(h, vp(rho.ctypes.data), vp(u[0].ctypes.data),
                                  vp(u[1].ctypes.data), vp(u[2].ctypes.data)))
        lbm.lbm_destroy(h)
    t1 = time.perf_counter()
    ws, _, _ = dist_env()
    max_s = reduce_max(t1 - t0, dev if ws > 1 else None)
    nb = K // CHECK_EVERY                                      # bench steps
    return {"value": round(aggregate(2.0 * nfluid * K, max_s, ws), 1), "unit": "MLUPS",
            "h2d_bytes_per_step": round(2 * mask.size / nb, 3),
            "d2h_bytes_per_step": round(2 * 4 * 8 * mask.size / nb, 3),
            "steps": nb, "lattice_steps": K,
            "what": "per model: lbm_create (host mask H2D) + lbm_step(lattice steps) + "
                    "lbm_fields (rho,u D2H into pinned host memory) + lbm_destroy, inside the "
                    "timed region"}


def run_precision_record(args):
    """The precision workload's duct outside the timed region: D3Q27,
    512 x 192 x 192 (191 x 191 fluid), Bn = 2, both models, FP32 and FP16
    offset storage, each on the launch shape the tuner picks for it on this
    geometry, timed with CUDA events over args.precision_steps lattice steps
    after one check interval.  The FP16 velocity field is compared with the
    FP32 one at the same step count (both from rest)."""
    import torch
    from paper_1610_01388_gb300 import autotune, lbm
    from paper_1610_01388_gb300 import workloads as W
    nx, ny, nz = 512, 192, 192
    mask = W.duct_mask(nx, ny, nz)
    nfluid = int((mask == 0).sum())
    prm = W.duct_params(H=ny - 1, nu_p=NU_P, u_newton=0.02, bn=BN)
    peak, kind = measured_hbm_peak()
    st = torch.cuda.current_stream()
    out, u_of = {}, {}
    n = CHECK_EVERY + args.precision_steps
    for storage in ("F32", "F16"):
        for model in ("IR", "PR"):
            shape = (256, 1)
            if not args.no_tune:
                shape, _ = autotune.tune("D3Q27", model, storage, mask.size, steps=100, mask=mask)
            s = lbm.Solver("D3Q27", mask, model=model, storage=storage, mu_p=NU_P,
                           sigma_y=prm["sigma_y"], m=M_PR, g=(prm["g"], 0.0, 0.0),
                           check_every=CHECK_EVERY, use_torch=True)
            s.step(CHECK_EVERY)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            s.step(args.precision_steps)
            e1.record(st)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3 / args.precision_steps
            b = s.info.bytes_per_fluid_update
            _, u_of[(storage, model)] = s.fields()
            s.close()
            gbs = b * nfluid / t / 1e9
            out[f"{model}/{storage}"] = {
                "kernel": f"k_step<D3Q27,{model},{STORAGE_CTYPE[storage]}>",
                "shape": f"{shape[0]}x{shape[1]}", "launch_us": round(t * 1e6, 2),
                "mlups": round(nfluid / t / 1e6, 1), "bytes_per_fluid_update": b,
                "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
    fl = mask == 0
    diff = {}
    for model in ("IR", "PR"):
        a, r = u_of[("F16", model)][:, fl], u_of[("F32", model)][:, fl]
        diff[model] = float(np.linalg.norm(a - r) / np.linalg.norm(r))
    rec = {"workload": f"square duct D3Q27 {nx}x{ny}x{nz} ({ny - 1}x{nz - 1} fluid), Bn={BN:g}, "
                       f"nu_p={NU_P}, PR m={M_PR:g}, from rest",
           "fluid_cells": nfluid, "lattice_steps": n, "peak_gbs": peak,
           "peak_kind": f"{kind} (copy bandwidth)", "kernels": out,
           "rel_l2_u_f16_vs_f32_at_equal_steps": diff}
    if args.precision_porous > 0:
        rec["porous"] = run_precision_porous(args)
    return rec


PRECISION_POROUS_BN = 0.5


def run_precision_porous(args):
    """The precision workload's porous box: args.precision_porous^3 cells of
    random non-overlapping spheres (radius 6-10, target porosity 0.6, seed 1;
    random sequential addition jams above it, so the packing stops after
    2e6 candidates, near porosity 0.67), D3Q27, both models, FP32 and FP16
    offset storage in the compact layout, timed as the duct is.  Bn = 0.5 a
    priori: at the porous record's Bn = 2 this box is near-jammed, where FP16
    storage does not resolve the flow.  The FP16 velocity field is compared
    with the FP32 one at the same step count on the device."""
    import torch
    from paper_1610_01388_gb300 import lbm
    from paper_1610_01388_gb300 import workloads as W
    side = args.precision_porous
    mask, info = W.porous_mask(side, porosity=0.6, r_min=6.0, r_max=10.0, seed=1,
                               max_attempts=2_000_000)
    fl = torch.from_numpy(mask.reshape(-1) == 0).cuda()
    nfluid = int(fl.sum())
    prm = W.porous_params(nu_p=NU_P, d_mean=16.0, g=2e-5, bn=PRECISION_POROUS_BN)
    peak, kind = measured_hbm_peak()
    st = torch.cuda.current_stream()
    out, diff, u32 = {}, {}, {}
    for storage in ("F32", "F16"):
        for model in ("IR", "PR"):
            s = lbm.Solver("D3Q27", mask, model=model, storage=storage, mu_p=NU_P,
                           sigma_y=prm["sigma_y"], m=M_PR, g=(prm["g"], 0.0, 0.0),
                           check_every=CHECK_EVERY, use_torch=True, layout="compact")
            s.step(CHECK_EVERY)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            s.step(args.precision_steps)
            e1.record(st)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3 / args.precision_steps
            b = s.info.bytes_per_fluid_update
            u = torch.empty((3, mask.size), dtype=torch.float64, device="cuda")
            lbm.lbm_fields_device(s.h, 0, u[0].data_ptr(), u[1].data_ptr(), u[2].data_ptr())
            torch.cuda.synchronize()
            s.close()
            u = u[:, fl]
            if storage == "F32":
                u32[model] = u
            else:
                r = u32.pop(model)
                diff[model] = float(torch.linalg.norm(u - r) / torch.linalg.norm(r))
            del u
            gbs = b * nfluid / t / 1e9
            name = "k_step_compact_loop" if (model == "IR" and storage == "F16") else "k_step_compact"
            out[f"{model}/{storage}"] = {
                "kernel": f"{name}<D3Q27,{model},{STORAGE_CTYPE[storage]}>",
                "launch_us": round(t * 1e6, 2), "mlups": round(nfluid / t / 1e6, 1),
                "bytes_per_fluid_update": b, "achieved_gbs": round(gbs, 1),
                "frac": round(gbs / peak, 4)}
    return {"workload": f"porous box D3Q27 {side}^3 (random non-overlapping spheres, radius "
                        f"6-10, porosity {info['porosity']:.3f}, seed 1, 2e6 candidates), "
                        f"Bn={PRECISION_POROUS_BN:g} a priori, nu_p={NU_P}, PR m={M_PR:g}, "
                        f"compact layout, from rest",
            "fluid_cells": nfluid, "cells": int(mask.size),
            "lattice_steps": CHECK_EVERY + args.precision_steps, "kernels": out,
            "rel_l2_u_f16_vs_f32_at_equal_steps": diff}


def run_porous_record(args):
    """The porous-medium workload outside the timed region: a 256^3 periodic
    box of random non-overlapping spheres (radius 6-10, porosity 0.7, seed 1),
    D3Q19, both models, FP32 and FP16 storage, each timed with CUDA events
    over args.porous_steps lattice steps after one check interval of warm-up.
    The compact layout (fluid cells only) is the porous path; the dense
    layout is timed beside it.  The dense layout keeps every cell, so an
    aligned group of 8 cells (one 32-byte sector of a plane) with any fluid
    cell moves all 8 cells' populations: touched_over_fluid is that floor of
    its traffic relative to the algorithmic (fluid-cell) bytes."""
    import torch
    from paper_1610_01388_gb300 import lbm
    from paper_1610_01388_gb300 import workloads as W
    side = args.porous_record
    mask, info = W.porous_mask(side, porosity=0.7, r_min=6.0, r_max=10.0, seed=1)
    flat = (mask.reshape(-1) == 0).astype(np.int64)
    nfluid = int(flat.sum())
    group = np.arange(flat.size) // 8
    fluid_per_group = np.bincount(group, weights=flat)
    cells_per_group = np.bincount(group)
    touched = int(cells_per_group[fluid_per_group > 0].sum())
    prm = W.porous_params(nu_p=NU_P, d_mean=16.0, g=2e-5, bn=BN)
    peak, kind = measured_hbm_peak()
    st = torch.cuda.current_stream()
    kernels = {"compact": {}, "dense": {}}
    for layout in ("compact", "dense"):
        for storage in ("F32", "F16"):
            for model in ("IR", "PR"):
                s = lbm.Solver("D3Q19", mask, model=model, storage=storage, mu_p=NU_P,
                               sigma_y=prm["sigma_y"], m=M_PR, g=(prm["g"], 0.0, 0.0),
                               check_every=CHECK_EVERY, use_torch=True, layout=layout)
                s.step(CHECK_EVERY)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(st)
                s.step(args.porous_steps)
                e1.record(st)
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / 1e3 / args.porous_steps
                b = s.info.bytes_per_fluid_update
                s.residual()
                s.close()
                gbs = b * nfluid / t / 1e9
                name = "k_step_compact" if layout == "compact" else "k_step"
                k = {"kernel": f"{name}<D3Q19,{model},{STORAGE_CTYPE[storage]}>",
                     "launch_us": round(t * 1e6, 2), "mlups": round(nfluid / t / 1e6, 1),
                     "bytes_per_fluid_update": b, "achieved_gbs": round(gbs, 1),
                     "frac": round(gbs / peak, 4),
                     "traffic": ncu_traffic(storage, model, 256, 1, None, workload="porous",
                                            layout=layout)}
                if layout == "dense":
                    k["frac_of_touched"] = round(gbs * touched / nfluid / peak, 4)
                kernels[layout][f"{model}/{storage}"] = k
    roof = {}
    comp = kernels["compact"]
    for storage in ("F32", "F16"):
        dom = max(("IR", "PR"), key=lambda m: comp[f"{m}/{storage}"]["launch_us"])
        k = comp[f"{dom}/{storage}"]
        roof[storage] = {"bound": "hbm", "kernel": k["kernel"] + " (dominant by time)",
                         "achieved": k["achieved_gbs"], "peak": peak,
                         "peak_kind": f"{kind} (copy bandwidth)", "unit": "GB/s",
                         "frac": k["frac"], "traffic": k["traffic"],
                         "bytes_per_fluid_update": k["bytes_per_fluid_update"],
                         "fluid_cells_per_launch": nfluid}
    return {"workload": f"porous box D3Q19 {side}^3 (random non-overlapping spheres, radius "
                        f"6-10, porosity {info['porosity']:.3f}, seed 1), Bn={BN:g} a priori, "
                        f"nu_p={NU_P}, PR m={M_PR:g}; 256 threads per block, check step every "
                        f"{CHECK_EVERY}",
            "layout": "compact (fluid cells only, LBM_FLAG_COMPACT); dense timed beside it",
            "fluid_cells": nfluid, "cells": int(flat.size),
            "touched_over_fluid": round(touched / nfluid, 4),
            "lattice_steps_timed": args.porous_steps, "roofline": roof,
            "kernels": kernels["compact"], "dense": kernels["dense"]}


# --- serving ----------------------------------------------------------------------

SERVE_MIX = ("D2Q9 channels 128 x (17..65), D3Q19/D3Q27 ducts 32 x (17..49)^2, "
             "D3Q19/D3Q27 porous boxes (24..48)^3 porosity 0.7 radius 3-5; Bn U[0.1,10]; PR/IR")
SERVE_MIX_FULL = ("D2Q9 channels 4 x (17..257), D3Q19/D3Q27 ducts 64 x (33..193)^2, "
                  "D3Q19/D3Q27 porous boxes (64..256)^3 (sides in steps of 16, 2 seeded "
                  "geometries per side) porosity 0.7 radius 6-10; Bn U[0.1,10]; PR/IR")


def _serve_sizes(args):
    if args.serve_full:
        return dict(duct_sides=(32, 192), porous_sides=(64, 256), porous_radius=(6.0, 10.0),
                    porous_pool=2)
    # a mix whose solves reach steady state within the bench's minutes: the
    # slowest mode of a channel or duct of width H decays over ~H^2 / nu steps
    return dict(channel_widths=(16, 64), channel_length=128, duct_sides=(16, 48),
                duct_length=32, porous_sides=(24, 48), porous_radius=(3.0, 5.0))


def _route(storage, req):
    """Storage of a request.  "mixed": FP16, except the porous boxes with an
    a-priori Bn of 1 or more, which run in FP32: those flows are nearly
    jammed, and the stress their populations carry makes FP16's rounding
    noise as large as their velocity."""
    if storage != "mixed":
        return storage
    if req is None:
        return "F16"
    return "F32" if (req["kind"] == "porous" and req["bn"] >= 1.0) else "F16"


def run_serving(args, storage):
    """A Poisson stream of independent solves (channels, ducts, porous boxes;
    Bn uniform in [0.1, 10]; PR or IR) through the continuous-batching server
    under a 120 GB budget: requests are submitted at their arrival times while
    the server steps everything admitted in chunks of args.serve_chunk steps
    (check every 100) and retires each solve at steady state (the criterion
    of --serve-criterion between consecutive check steps below the
    tolerance) or at the step cap.  Latency = completion - arrival; time to
    steady state is that latency for the converged requests.  Accuracy: a
    sample of the served requests (the first two of each kind) is solved
    again on the plain FP32 single-domain path (lbm_step) for the same number
    of steps, and the relative L2 difference of the velocity fields is
    reported."""
    from paper_1610_01388_gb300 import lbm
    from paper_1610_01388_gb300 import workloads as W
    reqs = W.serving_requests(n=args.serve_requests, rate=args.serve_rate, seed=7,
                              storage=_route(storage, None), max_steps=args.serve_max_steps,
                              tolerance=args.serve_tolerance, criterion=args.serve_criterion,
                              **_serve_sizes(args))
    for r in reqs:
        r["storage"] = _route(storage, r)
    sample = []
    for kind in ("channel", "duct", "porous"):
        sample += [i for i, r in enumerate(reqs) if r["kind"] == kind][:4]
    schedule = None
    if not args.no_tune:
        # the batch schedule, tuned on a mix drawn from the same generator
        # (another seed), outside the timed region
        from paper_1610_01388_gb300 import autotune
        tune_mix = W.serving_requests(n=48, rate=args.serve_rate, seed=8,
                                      storage=_route(storage, None),
                                      max_steps=args.serve_max_steps,
                                      tolerance=args.serve_tolerance, **_serve_sizes(args))
        for r in tune_mix:
            r["storage"] = _route(storage, r)
        mix = [(r["lattice"], r["mask"], dict(model=r["model"], storage=r["storage"],
                                              mu_p=r["mu_p"], sigma_y=r["sigma_y"], m=r["m"],
                                              g=r["g"])) for r in tune_mix]
        tuned = autotune.tune_batch(mix)
        schedule = {k: v for k, v in tuned.items() if k != "tried"}
        schedule["us_per_step_untuned"] = round(tuned["tried"]["base"] * 1e6, 1)
        schedule["seconds_per_step"] = round(schedule["seconds_per_step"] * 1e6, 1)
        schedule["us_per_step"] = schedule.pop("seconds_per_step")
    srv = lbm.Server(120 * (1 << 30), check_every=args.serve_check_every)
    t0 = srv.now()
    ids = []
    k = 0
    while True:
        now = srv.now() - t0
        while k < len(reqs) and reqs[k]["arrival"] <= now:
            r = reqs[k]
            ids.append(srv.submit(r["lattice"], r["mask"], tolerance=r["tolerance"],
                                  max_steps=r["max_steps"], criterion=r["criterion"],
                                  keep_fields=k in sample, model=r["model"],
                                  storage=r["storage"], mu_p=r["mu_p"], sigma_y=r["sigma_y"],
                                  m=r["m"], g=r["g"]))
            k += 1
        q, running, _ = srv.pending()
        if q == 0 and running == 0:
            if k == len(reqs):
                break
            time.sleep(max(0.0, reqs[k]["arrival"] - (srv.now() - t0)))
            continue
        srv.advance(args.serve_chunk)
    res = [srv.result(i) for i in ids]
    served_u = {i: srv.fields(ids[i], reqs[i]["mask"].shape if reqs[i]["mask"].ndim == 3
                              else (1,) + reqs[i]["mask"].shape)[1] for i in sample}
    srv.close()
    acc = []
    for i in sample:
        r = reqs[i]
        ref = lbm.Solver(r["lattice"], r["mask"], model=r["model"], storage="F32", mu_p=r["mu_p"],
                         sigma_y=r["sigma_y"], m=r["m"], g=r["g"],
                         check_every=args.serve_check_every)
        ref.step(res[i].steps)
        _, uref = ref.fields()
        ref.close()
        fl = (r["mask"] if r["mask"].ndim == 3 else r["mask"][None]) == 0
        a, b = served_u[i][:, fl], uref.reshape(served_u[i].shape)[:, fl]
        acc.append({"kind": r["kind"], "lattice": r["lattice"], "model": r["model"],
                    "bn": round(r["bn"], 2), "steps": int(res[i].steps),
                    "u_rms": float(np.linalg.norm(b) / np.sqrt(b.shape[1])),
                    "rel_l2_u_vs_fp32_single_domain": float(np.linalg.norm(a - b) / np.linalg.norm(b))})
    lat = np.array([r.t_done - r.t_submit for r in res])
    conv = np.array([r.state == lbm.LBM_REQ_CONVERGED for r in res])
    upd = sum(r.fluid_cells * r.steps for r in res)
    span = max(r.t_done for r in res) - min(r.t_submit for r in res)
    tts = lat[conv]
    errs = [a["rel_l2_u_vs_fp32_single_domain"] for a in acc]
    kinds = np.array([r["kind"] for r in reqs])
    bar = 1e-5 if storage in ("F32", "F64") else 1e-3
    by_kind = {}
    for kind in ("channel", "duct", "porous"):
        sel = kinds == kind
        ek = [a["rel_l2_u_vs_fp32_single_domain"] for a in acc if a["kind"] == kind]
        by_kind[kind] = {"requests": int(sel.sum()), "converged": int(conv[sel].sum()),
                         "sampled": len(ek), "sampled_within_bar": int(sum(e <= bar for e in ek)),
                         "max_rel_l2_u": max(ek) if ek else None}
    return {"storage": storage, "requests": len(res), "served_solves_per_s": round(len(res) / span, 3),
            "converged_fraction": round(float(conv.mean()), 4),
            "steps_to_steady_p50": int(np.percentile([r.steps for r, c in zip(res, conv) if c], 50))
            if conv.any() else None,
            "accuracy": {"max_rel_l2_u_vs_fp32_single_domain": max(errs) if errs else None,
                         "bar": bar, "by_kind": by_kind, "requests": acc},
            "latency_p50_s": round(float(np.percentile(lat, 50)), 4),
            "latency_p99_s": round(float(np.percentile(lat, 99)), 4),
            "time_to_steady_p50_s": round(float(np.percentile(tts, 50)), 4) if tts.size else None,
            "time_to_steady_p99_s": round(float(np.percentile(tts, 99)), 4) if tts.size else None,
            "converged": int(conv.sum()),
            "capped": int(sum(r.state == lbm.LBM_REQ_CAPPED for r in res)),
            "failed": int(sum(r.state == lbm.LBM_REQ_FAILED for r in res)),
            "aggregate_mlups": round(upd / span / 1e6, 1), "makespan_s": round(span, 3),
            "batch_schedule": schedule}


# --- oracle arms ------------------------------------------------------------------

def _oracle_sample_step(states):
    for st in states:
        st.step(1)


def _oracle_states():
    import oracle
    from paper_1610_01388_gb300 import workloads as W
    g, sy = workload_params()
    mask = workload_mask(SAMPLE_NX)
    states = []
    for model in ("IR", "PR"):
        p = oracle.params(model=model, nu_p=NU_P, sigma_y=sy, m=M_PR, g=(g, 0, 0))
        states.append(oracle.State(LATTICE, p, mask, nthreads=0))
    return states, int((mask == 0).sum())


def run_cpu_baseline(args):
    """The oracle as it stands on the host cores: a bounded sample (a
    4-cell-long slab of the same duct, both models, periodic along x) stepped
    for about args.cpu_seconds seconds."""
    import oracle
    states, nf = _oracle_states()
    _oracle_sample_step(states)
    n = 0
    t0 = time.perf_counter()
    while True:
        _oracle_sample_step(states)
        n += 1
        if time.perf_counter() - t0 > args.cpu_seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": round(2.0 * nf * n / dt / 1e6, 4), "unit": "MLUPS",
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{SAMPLE_NX}x{NY}x{NZ} slab of the {'porous box' if POROUS else 'duct'} (both models, {nf} fluid cells "
                      f"each), {n} steps in {dt:.1f} s, FP64"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    states, nf = _oracle_states()
    for _ in range(args.warmup):
        _oracle_sample_step(states)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_sample_step(states)
    dt = time.perf_counter() - t0
    value = 2.0 * nf * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": round(value, 4), "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3 / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_config({"sample": f"{SAMPLE_NX}x{NY}x{NZ} slab per step"}),
            "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS",
                             "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{SAMPLE_NX}x{NY}x{NZ} slab of the {'porous box' if POROUS else 'duct'}, both models, "
                                       "one time step each per bench step"},
            "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    global NX, NY, NZ, LATTICE, STORAGE, POROUS
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20,
                    help=f"timed bench steps ({CHECK_EVERY} lattice steps of each model each)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the block-size autotuner")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests in the serving leg (0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=150.0, help="Poisson arrival rate, 1/s")
    ap.add_argument("--serve-max-steps", type=int, default=200_000)
    ap.add_argument("--serve-tolerance", type=float, default=1e-5)
    ap.add_argument("--serve-criterion", choices=["flow", "residual"], default="flow")
    ap.add_argument("--serve-check-every", type=int, default=1000,
                    help="steps between the check steps the steady-state test compares")
    ap.add_argument("--serve-chunk", type=int, default=1000,
                    help="steps per server advance (a multiple of the check interval)")
    ap.add_argument("--porous-record", type=int, default=256, metavar="SIDE",
                    help="side of the porous box timed beside the duct (0 skips it)")
    ap.add_argument("--porous-steps", type=int, default=500)
    ap.add_argument("--precision-steps", type=int, default=500,
                    help="lattice steps timed on the precision workload's duct (0 skips it)")
    ap.add_argument("--precision-porous", type=int, default=512, metavar="SIDE",
                    help="side of the precision workload's porous box (0 skips it)")
    ap.add_argument("--serve-storage", default="F16,F32,mixed",
                    help="storage forms served, comma-separated, in order (mixed: FP16, with "
                         "FP32 for the near-jammed porous requests)")
    ap.add_argument("--serve-full", action="store_true",
                    help="serve the full-size mix (ducts to 192^2, porous boxes to 256^3) "
                         "instead of the scaled-down one")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel, if captured")
    ap.add_argument("--nx", type=int, default=NX, help="duct length (other workloads)")
    ap.add_argument("--ny", type=int, default=NY, help="duct cross-section (profiling runs)")
    ap.add_argument("--lattice", default=LATTICE, choices=["D3Q15", "D3Q19", "D3Q27"])
    ap.add_argument("--storage", default=STORAGE, choices=["F32", "F64", "F16", "BF16"])
    ap.add_argument("--nz", type=int, default=NZ)
    ap.add_argument("--porous", type=int, default=0, metavar="SIDE",
                    help="time a porous box of SIDE^3 cells (spheres of radius 6-10, porosity "
                         "0.7, seed 1) instead of the duct")
    ap.add_argument("--steady", action="store_true",
                    help="also run both models from rest to steady state and report the time")
    ap.add_argument("--steady-tol", type=float, default=1e-6)
    ap.add_argument("--steady-cap", type=int, default=2_000_000)
    args = ap.parse_args(argv)
    NX, NY, NZ = args.nx, args.ny, args.nz
    LATTICE, STORAGE = args.lattice, args.storage
    POROUS = args.porous
    if POROUS:
        NX = NY = NZ = POROUS
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.serve_chunk < args.serve_check_every or args.serve_chunk % args.serve_check_every:
        ap.error("--serve-chunk must be a positive multiple of --serve-check-every")
    world = os.environ.get("WORLD_SIZE")
    if world is not None and int(world) != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}", file=sys.stderr)
        sys.exit(2)
    if world is None and args.gpus > 1:
        # one process per GPU: relaunch under torch.distributed.run
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        argv_full = sys.argv[1:] if argv is None else list(argv)
        os.execvp(sys.executable, [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                                   f"--nproc-per-node={args.gpus}", "--master-addr=127.0.0.1",
                                   f"--master-port={port}", os.path.abspath(__file__), *argv_full])
    if not set(args.serve_storage.split(",")) <= {"F32", "F64", "F16", "BF16", "mixed"}:
        ap.error("--serve-storage takes F32, F64, F16, BF16, mixed, comma-separated")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
