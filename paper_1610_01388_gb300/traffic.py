"""Sector-level DRAM traffic of one fused step on a given geometry.

The step kernels keep every cell of the box in the population planes (the
dense layout), so on a porous geometry the 32-byte sectors a launch touches
carry solid cells too.  This module counts those sectors on the host for
FP32 or FP64 storage (one value per cell and plane):

* reads: per plane j, the sectors holding the values pulled from it (a fluid
  cell's fluid neighbour at x - c_j; the cell itself when the neighbour in
  direction opp(j) is solid, the halfway bounce-back), plus, with the
  copy-through, the own values of the solid cells in aligned groups of 8
  consecutive cells that hold fluid cells (the kernels' copy rule);
* fills: per plane, the written sectors that the stores cover only in part
  (such a sector is read before it is written);
* writes: per plane, every sector a store touches;
* links: the 4-byte link word of every cell.

Each sector is counted once per launch (L2 catches the reuse between
neighbouring warps).  `compact_traffic` counts the same for the compact
(fluid-only) layout.  On a 160^3 D3Q27 porous box the total matched an ncu
capture of the FP32 IR step to 1 % (copy groups of 32 cells, the kernels'
rule at the time).
"""
from __future__ import annotations

import numpy as np

from . import lbm

SECTOR = 32


def _geometry(mask, lattice, value_bytes, read_bytes):
    if value_bytes not in (4, 8):
        raise ValueError("value_bytes must be 4 (FP32) or 8 (FP64)")
    if read_bytes not in (32, 64):
        raise ValueError("read_bytes must be 32 or 64")
    m = np.asarray(mask)
    if m.ndim == 2:
        m = m[None]
    nz, ny, nx = m.shape
    n = m.size
    solid = m.reshape(-1) != 0
    c, w = lbm.lbm_lattice_info(lattice)
    q = len(w)
    c = np.asarray(c).reshape(q, -1)
    if c.shape[1] == 2:
        c = np.concatenate([c, np.zeros((q, 1), c.dtype)], axis=1)
    opp = [int(np.flatnonzero((c == -c[i]).all(1))[0]) for i in range(q)]
    idx = np.arange(n)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    src = [((x - c[i, 0]) % nx) + nx * (((y - c[i, 1]) % ny) + ny * ((z - c[i, 2]) % nz))
           for i in range(q)]
    return n, solid, q, opp, idx, src


def sector_traffic(mask: np.ndarray, lattice: str, value_bytes: int = 4,
                   copy_through: bool = True, group: int = 8, read_bytes: int = 32) -> dict:
    """Bytes one step moves on `mask` ((nz, ny, nx) or (ny, nx), 1 = solid,
    periodic), split into reads, fills, writes and link words, next to the
    algorithmic bytes (fluid cells x (2 Q value_bytes + 1)).  Populations
    only: the PR tau field and the check-step snapshot are not counted.
    `group`: cells per copy-through group (8 in the kernels).  `read_bytes`:
    the unit a read fetches from DRAM, a 32-byte sector or a 64-byte pair of
    sectors (writes stay per sector)."""
    n, solid, q, opp, idx, src = _geometry(mask, lattice, value_bytes, read_bytes)
    fluid = ~solid
    per = SECTOR // value_bytes
    per_read = read_bytes // value_bytes
    group_has_fluid = np.bincount(idx // group, weights=fluid.astype(np.int64)) > 0
    copy = solid & group_has_fluid[idx // group] if copy_through else np.zeros(n, bool)
    writers = fluid | copy
    cnt = np.bincount(idx[writers] // per, minlength=(n + per - 1) // per)
    touched = int((cnt > 0).sum())
    partial = int(((cnt > 0) & (cnt < per)).sum())
    reads = 0
    for j in range(q):
        parts = [src[j][fluid & ~solid[src[j]]], idx[fluid & solid[src[opp[j]]]], idx[copy]]
        reads += len(np.unique(np.concatenate(parts) // per_read))
    out = {"reads": reads * read_bytes, "fills": partial * q * SECTOR,
           "writes": touched * q * SECTOR, "links": 4 * n}
    out["total"] = sum(out.values())
    out["algorithmic"] = int(fluid.sum()) * (2 * q * value_bytes + 1)
    out["ratio"] = out["total"] / out["algorithmic"] if out["algorithmic"] else float("nan")
    return out


def compact_traffic(mask: np.ndarray, lattice: str, value_bytes: int = 4,
                    read_bytes: int = 32) -> dict:
    """The same count for the compact layout (LBM_FLAG_COMPACT): the planes
    hold the fluid cells in cell-index order, one slot each, so every plane
    is written whole; plane j is read at the slots of the cells pulled from
    (the fluid sources x - c_j) and at a cell's own slot where population
    opp(j) bounces back.  `maps` are each slot's cell index and link word
    (4 + 4 bytes, read whole) and the rank words read at the fluid sources
    (4 bytes per cell of the box, counted by access unit)."""
    n, solid, q, opp, idx, src = _geometry(mask, lattice, value_bytes, read_bytes)
    fluid = ~solid
    nf = int(fluid.sum())
    slot = np.full(n, -1, np.int64)
    slot[fluid] = np.arange(nf)
    per_read = read_bytes // value_bytes
    reads = 0
    rank_cells = []
    for j in range(q):
        pulled = fluid & fluid[src[j]]
        parts = [slot[src[j][pulled]], slot[fluid & solid[src[opp[j]]]]]
        reads += len(np.unique(np.concatenate(parts) // per_read))
        if j:                                    # population 0 is the cell's own
            rank_cells.append(src[j][pulled])
    rank_units = len(np.unique(np.concatenate(rank_cells) // (read_bytes // 4))) if rank_cells else 0
    whole = lambda b: -(-b // SECTOR) * SECTOR   # bytes rounded up to whole sectors
    out = {"reads": reads * read_bytes, "writes": q * whole(nf * value_bytes),
           "maps": 2 * whole(4 * nf) + rank_units * read_bytes}
    out["total"] = sum(out.values())
    out["algorithmic"] = nf * (2 * q * value_bytes + 1)
    out["ratio"] = out["total"] / out["algorithmic"] if out["algorithmic"] else float("nan")
    return out
