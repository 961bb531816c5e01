"""Seeded synthetic inputs: solid masks, random populations and workload
parameters for the Bingham LBM solver.

This module holds input generators only (geometry, random numbers, the
mapping of a requested Bingham number to a yield stress through the
*continuum* closed forms of the flows).  It contains none of the lattice
Boltzmann method's arithmetic; both the CUDA path and the CPU oracle receive
what it produces.

Geometry conventions (all masks are uint8, 1 = solid, shape (nz, ny, nx),
x fastest):

* plane channel (Sec. 4.3 geometry in 2D): row y = 0 solid, periodic in x and
  y, so the single solid row is the wall on both sides and the channel has
  ny - 1 fluid rows (odd ny - 1 puts a node on the centre line);
* square duct (Sec. 4.3): rows y = 0 and z = 0 solid, periodic wrap, flow
  along x; the fluid cross-section is (ny - 1) x (nz - 1);
* porous medium: random sequential addition of non-overlapping spheres in a
  periodic box (minimum-image distance), radius uniform in [r_min, r_max],
  stopping once the voxel porosity (fraction of cells whose centre is outside
  every sphere) reaches the target;
* cylinder array (Sec. 4.5): one cylinder of diameter D in an L x L periodic
  cell.
"""
from __future__ import annotations

import math

import numpy as np


def channel_mask(nx: int = 4, ny: int = 64) -> np.ndarray:
    m = np.zeros((1, ny, nx), np.uint8)
    m[0, 0, :] = 1
    return m


def duct_mask(nx: int, ny: int, nz: int) -> np.ndarray:
    m = np.zeros((nz, ny, nx), np.uint8)
    m[:, 0, :] = 1
    m[0, :, :] = 1
    return m


def periodic_box_mask(nx: int, ny: int, nz: int) -> np.ndarray:
    return np.zeros((nz, ny, nx), np.uint8)


def cylinder_mask(L: int = 80, D: float = 32.0, shift: float = 0.0) -> np.ndarray:
    """2D periodic cell with one cylinder; cell centres inside are solid."""
    y, x = np.mgrid[0:L, 0:L].astype(np.float64)
    c = (L - 1) / 2.0 + shift
    inside = (x - c) ** 2 + (y - (L - 1) / 2.0) ** 2 <= (D / 2.0) ** 2
    return inside.astype(np.uint8)[None, :, :]


def porous_mask(n: int | tuple = 64, porosity: float = 0.7, r_min: float = 6.0,
                r_max: float = 10.0, seed: int = 1, max_attempts: int = 10_000_000):
    """Random non-overlapping spheres in a periodic box (random sequential
    addition).

    Candidates (centre uniform in the box, radius uniform in [r_min, r_max])
    are drawn in chunks of 256 from numpy's PCG64 seeded with `seed` and taken
    in order: a candidate is kept if it overlaps no sphere kept before it
    (periodic minimum-image distance below the sum of the radii), and painted
    into the mask (a cell is solid if its centre lies inside a sphere).  The
    packing stops once the solid fraction reaches 1 - porosity, or at the
    first chunk boundary after max_attempts candidates (jamming).

    Returns (mask, info) with info = {"porosity", "spheres", "attempts",
    "reached"}.  Overlap tests look only at the 27 neighbouring bins of edge
    >= 2 r_max when the box holds at least 3 bins per axis, which gives the
    same accept / reject decisions as testing every kept sphere.
    """
    nx, ny, nz = (n, n, n) if isinstance(n, int) else n
    rng = np.random.Generator(np.random.PCG64(seed))
    mask = np.zeros((nz, ny, nx), np.uint8)
    box = np.array([nx, ny, nz], np.float64)
    total = nx * ny * nz
    target_solid = (1.0 - porosity) * total
    nb = np.floor(box / (2.0 * r_max)).astype(int)
    binned = bool(np.all(nb >= 3))
    edge = box / np.maximum(nb, 1)
    cap = int(np.ceil((float(edge.max()) / (2.0 * r_min) + 1.0) ** 3)) + 1
    grid = np.full((nb[0], nb[1], nb[2], cap), -1, np.int64) if binned else None
    fill = np.zeros((nb[0], nb[1], nb[2]), np.int64) if binned else None
    offs = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)])
    centres = np.zeros((0, 3), np.float64)
    radii = np.zeros(0, np.float64)
    solid = 0
    attempts = 0
    chunk, group = 256, 16

    def hits_kept(cand, rad):
        """Candidates (m, 3) overlapping a sphere kept before this group."""
        if len(radii) == 0:
            return np.zeros(len(rad), bool)
        if not binned:
            d = centres[None, :, :] - cand[:, None, :]
            d -= box * np.round(d / box)
            return np.any(np.sqrt(np.sum(d * d, axis=2)) < radii[None, :] + rad[:, None], axis=1)
        b = np.minimum((cand / edge).astype(int), nb - 1)
        nbins = (b[:, None, :] + offs[None, :, :]) % nb              # (m, 27, 3)
        top = int(fill.max())
        idx = grid[nbins[..., 0], nbins[..., 1], nbins[..., 2], :top].reshape(len(rad), -1)
        valid = idx >= 0
        j = np.where(valid, idx, 0)
        d = centres[j] - cand[:, None, :]
        d -= box * np.round(d / box)
        dist = np.sqrt(np.sum(d * d, axis=2))
        return np.any(valid & (dist < radii[j] + rad[:, None]), axis=1)

    done = False
    while not done and solid < target_solid and attempts < max_attempts:
        cs, rs = [], []
        for _ in range(group):
            cs.append(rng.random((chunk, 3)) * box)
            rs.append(r_min + (r_max - r_min) * rng.random(chunk))
        cand, rad = np.concatenate(cs), np.concatenate(rs)
        # chunks are taken while fewer than max_attempts candidates were drawn
        limit = len(rad)
        for ci in range(1, group):
            if attempts + ci * chunk >= max_attempts:
                limit, done = ci * chunk, True
                break
        rejected = hits_kept(cand[:limit], rad[:limit])
        new_c, new_r = [], []
        stop = None
        for k in np.flatnonzero(~rejected):
            if new_r:
                d = np.asarray(new_c) - cand[k]
                d -= box * np.round(d / box)
                if np.any(np.sqrt(np.sum(d * d, axis=1)) < np.asarray(new_r) + rad[k]):
                    continue
            new_c.append(cand[k])
            new_r.append(rad[k])
            solid += _paint_sphere(mask, cand[k], rad[k])
            if solid >= target_solid:
                stop = int(k)
                break
        if stop is not None:
            attempts += stop + 1
            done = True
        else:
            attempts += limit
        if new_r:
            first = len(radii)
            centres = np.vstack([centres, np.asarray(new_c)])
            radii = np.concatenate([radii, np.asarray(new_r)])
            if binned:
                for s_idx in range(first, len(radii)):
                    bx, by, bz = np.minimum((centres[s_idx] / edge).astype(int), nb - 1)
                    if fill[bx, by, bz] >= cap:
                        raise RuntimeError("sphere bin overflow")
                    grid[bx, by, bz, fill[bx, by, bz]] = s_idx
                    fill[bx, by, bz] += 1
    info = {"porosity": 1.0 - mask.sum() / total, "spheres": int(len(radii)),
            "attempts": attempts, "reached": bool(solid >= target_solid)}
    return mask, info


def _paint_sphere(mask, c, r):
    nz, ny, nx = mask.shape
    lo = np.floor(c - r).astype(int)
    hi = np.ceil(c + r).astype(int)
    xs = np.arange(lo[0], hi[0] + 1)
    ys = np.arange(lo[1], hi[1] + 1)
    zs = np.arange(lo[2], hi[2] + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    inside = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r
    zi, yi, xi = Z[inside] % nz, Y[inside] % ny, X[inside] % nx
    before = int(mask[zi, yi, xi].sum())
    mask[zi, yi, xi] = 1
    return int(inside.sum()) - before


def random_populations(weights: np.ndarray, ncells: int, amplitude: float = 0.05,
                       seed: int = 0) -> np.ndarray:
    """f[i, n] = w_i (1 + amplitude * r), r uniform in [-1, 1): a seeded
    perturbation of the rest state.  `weights` is passed in by the caller."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.uniform(-1.0, 1.0, size=(len(weights), ncells))
    return np.asarray(weights, np.float64)[:, None] * (1.0 + amplitude * r)


def permutation(c_from: np.ndarray, c_to: np.ndarray) -> np.ndarray:
    """Index map p with c_to[p[k]] == c_from[k]: population k of one velocity
    order sits at p[k] in the other."""
    lookup = {tuple(int(v) for v in c): k for k, c in enumerate(c_to)}
    return np.array([lookup[tuple(int(v) for v in c)] for c in c_from], np.int64)


# --- workload parameters ---------------------------------------------------

def channel_bn_to_xi(bn: float) -> float:
    """Plane Bingham-Poiseuille flow: invert Bn = sigma_y H / (mu_p U_mean)
    for xi = y_0 / h, using U_mean = (g h^2 / 3 nu)(1 - 3 xi/2 + xi^3/2) and
    sigma_y = xi rho g h, which give Bn = 6 xi / (1 - 1.5 xi + 0.5 xi^3)."""
    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        val = 6.0 * mid / (1.0 - 1.5 * mid + 0.5 * mid ** 3)
        if val < bn:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def channel_params(H: int = 63, nu_p: float = 0.1, u_newton: float = 0.01, bn: float = 1.0):
    """Body force for a Newtonian centre-line speed u_newton and the yield
    stress for the requested Bingham number (rho = 1)."""
    h = H / 2.0
    g = 2.0 * nu_p * u_newton / (h * h)
    xi = channel_bn_to_xi(bn) if bn > 0 else 0.0
    return {"g": g, "sigma_y": xi * g * h, "xi": xi, "h": h, "nu_p": nu_p}


BI_CR = 4.0 / (2.0 + math.sqrt(math.pi))
C_MAX = 1.178741652


def duct_bn_to_bi(bn: float) -> float:
    """Square duct: map an a-posteriori Bn = sigma_y H / (mu_p U_max) to the
    a-priori Bi = 4 sigma_y / (rho g H) through the Mosolov-Miasnikov form
    U_max = g c_max H^2 / (16 mu_p) (1 - Bi/Bi_cr)^2 (eq. U_max_square;
    about 2 % off for Bi > 0, which only shifts the realised Bn)."""
    # Bn = (Bi g H^2 / 4) / (g c_max H^2 / 16 (1 - Bi/Bi_cr)^2) = 4 Bi / (c_max (1 - Bi/Bi_cr)^2)
    lo, hi = 0.0, BI_CR * (1 - 1e-12)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        val = 4.0 * mid / (C_MAX * (1.0 - mid / BI_CR) ** 2)
        if val < bn:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def duct_params(H: int = 127, nu_p: float = 0.1, u_newton: float = 0.02, bn: float = 2.0):
    """Body force for a Newtonian centre-line speed u_newton in a square duct of
    side H, and the yield stress for the requested Bn (rho = 1)."""
    g = 16.0 * nu_p * u_newton / (C_MAX * H * H)
    bi = duct_bn_to_bi(bn) if bn > 0 else 0.0
    return {"g": g, "sigma_y": bi * g * H / 4.0, "bi": bi, "nu_p": nu_p}


def porous_params(nu_p: float = 0.1, d_mean: float = 16.0, g: float = 2e-5, bn: float = 1.0):
    """Porous box: a-priori Bn = 4 sigma_y / (rho g d_mean)."""
    return {"g": g, "sigma_y": bn * g * d_mean / 4.0, "nu_p": nu_p}


_POROUS_POOL: dict = {}


def _pooled_porous(side: int, seed: int, r_min: float, r_max: float):
    key = (side, seed, r_min, r_max)
    if key not in _POROUS_POOL:
        _POROUS_POOL[key] = porous_mask(side, porosity=0.7, r_min=r_min, r_max=r_max, seed=seed)[0]
    return _POROUS_POOL[key]


def serving_requests(n: int = 200, rate: float = 40.0, seed: int = 7, storage: str = "F16",
                     channel_widths=(16, 256), duct_sides=(32, 96), duct_length: int = 64,
                     porous_sides=(32, 64), max_steps: int = 2000, tolerance: float = 1e-4,
                     porous_radius=(4.0, 6.0), porous_pool: int = 0, criterion: str = "flow",
                     channel_length: int = 4):
    """Poisson stream of independent solves: 2D channels (D2Q9, channel_length
    x width, periodic along the length),
    square ducts (D3Q19/D3Q27, side x side x length) and porous boxes
    (D3Q19/D3Q27, random spheres of radius U[porous_radius], porosity 0.7),
    Bingham number uniform in [0.1, 10], model PR or IR with equal
    probability.  Returns a list of dicts with the arrival time (s) and
    everything a solver needs.

    porous_pool = 0 draws a fresh geometry per porous request.  porous_pool =
    P > 0 rounds each box side to a multiple of 16 and draws its geometry from
    P seeds per side, generated once per process (a 256^3 box takes seconds
    on the host, which a stream of thousands of requests cannot pay each
    time); Bingham number and model are still drawn per request."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for k in range(n):
        t += rng.exponential(1.0 / rate)
        kind = rng.integers(3)
        bn = float(rng.uniform(0.1, 10.0))
        model = "PR" if rng.integers(2) == 0 else "IR"
        if kind == 0:
            w = int(rng.integers(channel_widths[0], channel_widths[1] + 1))
            mask = channel_mask(channel_length, w + 1)
            p = channel_params(H=w, nu_p=0.1, u_newton=0.02, bn=bn)
            lat, g = "D2Q9", (p["g"], 0.0, 0.0)
        elif kind == 1:
            s = int(rng.integers(duct_sides[0], duct_sides[1] + 1))
            mask = duct_mask(duct_length, s + 1, s + 1)
            p = duct_params(H=s, nu_p=0.1, u_newton=0.02, bn=min(bn, 8.0))
            lat, g = ("D3Q19" if rng.integers(2) == 0 else "D3Q27"), (p["g"], 0.0, 0.0)
        else:
            s = int(rng.integers(porous_sides[0], porous_sides[1] + 1))
            if porous_pool > 0:
                s = min(max(16 * round(s / 16), porous_sides[0]), porous_sides[1])
                mask = _pooled_porous(s, int(rng.integers(porous_pool)) + 1, *porous_radius)
            else:
                mask, _ = porous_mask(s, porosity=0.7, r_min=porous_radius[0],
                                      r_max=porous_radius[1], seed=int(rng.integers(1 << 30)))
            p = porous_params(nu_p=0.1, d_mean=10.0, g=2e-5, bn=bn)
            lat, g = ("D3Q19" if rng.integers(2) == 0 else "D3Q27"), (p["g"], 0.0, 0.0)
        out.append({"arrival": t, "lattice": lat, "mask": mask, "model": model,
                    "storage": storage, "mu_p": 0.1, "sigma_y": p["sigma_y"], "m": 1e6,
                    "g": g, "tolerance": tolerance, "max_steps": max_steps,
                    "criterion": criterion, "kind": ("channel", "duct", "porous")[kind],
                    "bn": bn})
    return out
