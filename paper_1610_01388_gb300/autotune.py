"""Autotuner for the step kernel's launch shape.

For a (lattice, model, storage, size class) it builds a synthetic square duct
with about 2**size_class cells, times every candidate shape (128, 256 or 512
threads per block at one cell per thread; 128 or 256 at two cells per
thread, FP32 arithmetic only) for a few hundred steps with CUDA events on
the solver's stream (after a warm-up that also captures the CUDA graphs),
takes the fastest, and writes it into the library's tuning table
(lbm_tuning_set_shape).  Results are cached in a JSON file keyed by the GPU
name so later processes skip the measurement (``load``).  All timing goes
through the C ABI.  The block size changes only the launch; two cells per
thread run the same collision in packed two-wide FP32 instructions (equal to
FP32 round-off).
"""
from __future__ import annotations

import json
import math
import os

from . import lbm
from . import workloads as W

# launch shapes (threads per block, cells per thread)
CANDIDATES = ((128, 1), (256, 1), (512, 1), (128, 2), (256, 2))


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _duct_for(lattice, cells):
    if lattice == "D2Q9":
        ny = max(8, int(math.sqrt(cells)))
        nx = max(4, cells // ny)
        return W.channel_mask(nx, ny)
    side = max(8, int(round((cells / 2) ** (1 / 3))))
    return W.duct_mask(max(4, cells // (side * side)), side, side)


def measure(lattice, model, storage, size_class, steps=300, warmup=70, mask=None):
    """Average step time (s) of every candidate launch shape, on `mask` when
    given (the workload's own geometry), else on a duct of the size class.
    The geometry matters beyond its size: it decides, among others, whether
    the 16-bit PR step runs its copy-through form (mixed warps), so a duct
    whose rows do not fill whole warps can rank the shapes differently from
    one whose rows do."""
    import torch
    cells = 1 << size_class
    if mask is None:
        mask = _duct_for(lattice, cells)
    out = {}
    for block, cpt in CANDIDATES:
        if cpt == 2 and storage == "F64":
            continue
        lbm.lbm_tuning_set_shape(lattice, model, storage, size_class, block, cpt)
        s = lbm.Solver(lattice, mask, model=model, storage=storage, mu_p=0.1, sigma_y=1e-6,
                       m=1e6, g=(1e-6, 0.0, 0.0), use_torch=True)
        s.step(warmup)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        out[(block, cpt)] = e0.elapsed_time(e1) / 1e3 / steps
        s.close()
    return out


def tune(lattice, model, storage, cells, cache=None, steps=300, mask=None):
    """Tune the size class of `cells` (on `mask`, the workload's geometry,
    when given); returns (best (block, cells per thread), {(block, cells per
    thread): seconds})."""
    _, cls = lbm.lbm_tuning_get(lattice, model, storage, cells)
    times = measure(lattice, model, storage, cls, steps=steps, mask=mask)
    best = min(times, key=times.get)
    lbm.lbm_tuning_set_shape(lattice, model, storage, cls, *best)
    if cache:
        data = _read(cache)
        data.setdefault(_gpu_name(), {})[f"{lattice}/{model}/{storage}/{cls}"] = {
            "block": best[0], "cells_per_thread": best[1],
            "seconds_per_step": {f"{b}x{c}": t for (b, c), t in times.items()}}
        with open(cache, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
    return best, times


def _read(path):
    if path and os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def load(cache):
    """Apply cached decisions for this GPU; returns how many were applied."""
    n = 0
    for key, v in _read(cache).get(_gpu_name(), {}).items():
        if key == "batch":
            continue
        lat, model, storage, cls = key.split("/")
        lbm.lbm_tuning_set_shape(lat, model, storage, int(cls), int(v["block"]),
                                 int(v.get("cells_per_thread", 1)))
        n += 1
    return n


# --- batch schedule -------------------------------------------------------------

BATCH_CTAS = (0, 1, 2, 4, 8)
# plain-step tile shapes (threads per CTA, cells per thread), the default first
BATCH_TILES = ((256, 1), (128, 1), (512, 1), (128, 2), (256, 2))


def measure_batch(mix, steps=160, warmup=32, budget=64 << 30):
    """Wall time (s) per step of a batch holding every domain of `mix`
    ((lattice, mask, params) tuples), graphs captured during the warm-up; the
    time includes the host's launch work, which is what small domains pay."""
    import time
    b = lbm.Batch(budget, check_every=1 << 30)
    ids = [b.add(lat, mask, **prm) for lat, mask, prm in mix]
    b.step(warmup)
    b.status(ids[0])
    t0 = time.perf_counter()
    b.step(steps)
    b.status(ids[0])
    dt = (time.perf_counter() - t0) / steps
    b.close()
    return dt


def _group_key(lat, prm):
    return (lat, prm.get("model", "IR"), prm.get("storage", "F32"))


def tune_batch(mix, steps=160, cache=None):
    """Coordinate search over the batch schedule on `mix`: group concurrency
    first (with one CTA per tile), then, group by group, the CTAs per SM of a
    persistent grid, then the plain-step tile shape (threads per CTA x cells
    per thread) for the group's size class (floor(log2) of its domains' mean
    cell count).  Leaves the fastest schedule set; returns it with the
    measured seconds per step of every candidate tried, and records the
    choices in the JSON file `cache` under the GPU's name and
    "lattice/model/storage/size class" keys (``load_batch`` applies them)."""
    keys = sorted({_group_key(lat, prm) for lat, _, prm in mix})
    for lat, model, storage in keys:
        lbm.lbm_tuning_set_batch(lat, model, storage, 0)
    lbm.lbm_tuning_set_batch_concurrency(False)
    tried = {"base": measure_batch(mix, steps)}
    best = tried["base"]
    lbm.lbm_tuning_set_batch_concurrency(True)
    tried["concurrent"] = measure_batch(mix, steps)
    concurrent = tried["concurrent"] < best
    best = min(best, tried["concurrent"])
    lbm.lbm_tuning_set_batch_concurrency(concurrent)
    ctas = {}
    for key in keys:
        ctas[key] = 0
        for c in BATCH_CTAS[1:]:
            lbm.lbm_tuning_set_batch(*key, c)
            t = measure_batch(mix, steps)
            tried[f"{'/'.join(key)}:{c}"] = t
            if t < best:
                best, ctas[key] = t, c
        lbm.lbm_tuning_set_batch(*key, ctas[key])
    tiles = {}
    for key in keys:
        lat, model, storage = key
        sizes = [mask.size for l, mask, prm in mix if _group_key(l, prm) == key]
        _, _, cls = lbm.lbm_tuning_get_batch_tile(lat, model, storage, sum(sizes) // len(sizes))
        shape = BATCH_TILES[0]
        if storage != "F64":
            for cand in BATCH_TILES[1:]:
                lbm.lbm_tuning_set_batch_tile(lat, model, storage, cls, *cand)
                t = measure_batch(mix, steps)
                tried[f"{'/'.join(key)}:tile{cand[0]}x{cand[1]}"] = t
                if t < best:
                    best, shape = t, cand
        lbm.lbm_tuning_set_batch_tile(lat, model, storage, cls, *shape)
        tiles[key] = (shape, cls)
    if cache:
        data = _read(cache)
        ent = data.setdefault(_gpu_name(), {}).setdefault("batch", {})
        ent["concurrent"] = bool(concurrent)
        for key in keys:
            (th, cpt), cls = tiles[key]
            ent[f"{'/'.join(key)}/{cls}"] = {"ctas_per_sm": ctas[key], "threads": th,
                                             "cells_per_thread": cpt}
        with open(cache, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
    return {"concurrent": concurrent, "ctas_per_sm": {"/".join(k): v for k, v in ctas.items()},
            "tile": {f"{'/'.join(k)}/{cls}": f"{th}x{cpt}" for k, ((th, cpt), cls) in tiles.items()},
            "seconds_per_step": best, "tried": tried}


def load_batch(cache):
    """Apply cached batch schedules for this GPU; returns how many group
    entries were applied."""
    ent = _read(cache).get(_gpu_name(), {}).get("batch", {})
    n = 0
    for key, v in ent.items():
        if key == "concurrent":
            lbm.lbm_tuning_set_batch_concurrency(bool(v))
            continue
        lat, model, storage, cls = key.split("/")
        lbm.lbm_tuning_set_batch(lat, model, storage, int(v["ctas_per_sm"]))
        lbm.lbm_tuning_set_batch_tile(lat, model, storage, int(cls), int(v["threads"]),
                                      int(v["cells_per_thread"]))
        n += 1
    return n
