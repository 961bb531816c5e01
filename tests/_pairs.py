"""Helpers that run the same seeded problem on the CUDA path (through the C
ABI binding) and on the FP64 oracle, and compare them.

The two sides use different velocity orders; populations are mapped by
matching velocity vectors (workloads.permutation)."""
import numpy as np

import oracle
from paper_1610_01388_gb300 import lbm
from paper_1610_01388_gb300 import workloads as W

LAT_Q = {"D2Q9": 9, "D3Q15": 15, "D3Q19": 19, "D3Q27": 27}


def perm_gpu_to_oracle(lat):
    c_gpu, _ = lbm.lbm_lattice_info(lat)
    c_orc, _, _ = oracle.lattice_info(lat)
    return W.permutation(c_gpu, c_orc)     # c_orc[p[k]] == c_gpu[k]


def gpu_to_oracle(lat, f_gpu):
    p = perm_gpu_to_oracle(lat)
    Q = f_gpu.shape[0]
    f = np.empty((Q, f_gpu[0].size), np.float64)
    f[p] = f_gpu.reshape(Q, -1)
    return f


def oracle_to_gpu(lat, f_orc):
    p = perm_gpu_to_oracle(lat)
    return np.ascontiguousarray(f_orc[p])


def make_pair(lat, mask, model="IR", storage="F32", nu_p=0.1, sigma_y=0.0, m=0.0, g=(0, 0, 0),
              magic=0.25, gammadot_c=1e-8, check_every=0, flags=0, use_torch=False, nthreads=0,
              newton=0, layout="dense"):
    mask = np.ascontiguousarray(mask, np.uint8)
    if mask.ndim == 2:
        mask = mask[None]
    s = lbm.Solver(lat, mask, model=model, storage=storage, mu_p=nu_p, sigma_y=sigma_y, m=m,
                   gammadot_c=gammadot_c, g=g, magic=magic, check_every=check_every,
                   flags=flags, newton_iters=newton, use_torch=use_torch, layout=layout)
    p = oracle.params(model=model, nu_p=nu_p, sigma_y=sigma_y, m=m, gdot_c=gammadot_c, g=g,
                      magic=magic, burnett_x=bool(flags & lbm.LBM_FLAG_BURNETT_X), newton=newton)
    o = oracle.State(lat, p, mask, nthreads=nthreads)
    return s, o


def set_both(lat, s, o, f_orc, tau=None):
    """Same full-f state on both sides (f_orc in oracle order, shape (Q, N))."""
    o.f = np.ascontiguousarray(f_orc, np.float64)
    s.set_populations(oracle_to_gpu(lat, o.f))
    if tau is not None:
        o.tau = np.ascontiguousarray(tau, np.float64).reshape(-1)
        s.set_tau(o.tau)


def rel_l2_u(s, o):
    _, ug = s.fields()
    _, uo = o.fields()
    fl = (o.mask == 0)
    a, b = ug[:, fl], uo[:, fl]
    den = np.sqrt(np.sum(b * b))
    return float(np.sqrt(np.sum((a - b) ** 2)) / den) if den > 0 else float(np.sqrt(np.sum(a * a)))


def pulled_inputs(c, mask, cells, gather):
    """Streamed inputs of `cells` in the library's velocity order, (n, Q):
    f_i(x - c_i) with periodic wrap, or the cell's own f_opp(i)(x) where x - c_i
    is solid (eq. 8 with halfway bounce-back).  gather(idx) returns the (Q, m)
    populations of the cells idx, library order."""
    Q = len(c)
    opp = np.array([next(j for j in range(Q) if np.array_equal(c[j], -c[i])) for i in range(Q)])
    nz, ny, nx = mask.shape
    flat = mask.reshape(-1)
    z, y, x = cells // (nx * ny), (cells // nx) % ny, cells % nx
    nb = (((z[:, None] - c[None, :, 2]) % nz) * ny + (y[:, None] - c[None, :, 1]) % ny) * nx \
        + (x[:, None] - c[None, :, 0]) % nx
    probe = np.unique(np.concatenate([cells, nb.reshape(-1)]))
    fp = gather(probe)
    icell = np.searchsorted(probe, cells)
    inb = np.searchsorted(probe, nb)
    fin = np.empty((cells.size, Q))
    for i in range(Q):
        solid = flat[nb[:, i]] != 0
        fin[:, i] = np.where(solid, fp[opp[i], icell], fp[i, inb[:, i]])
    return fin


def oracle_collide_cells(lat, p, fin, tau_old):
    """Oracle single-cell collisions of pulled inputs (n, Q, library order);
    returns ((Q, n) post-collision populations in library order, (n,) tau)."""
    po = perm_gpu_to_oracle(lat)           # oracle direction of library direction k
    n, Q = fin.shape
    out = np.empty((Q, n))
    tau = np.empty(n)
    fo_in = np.empty(Q)
    for k in range(n):
        fo_in[po] = fin[k]
        fo, tn, _ = oracle.collide(lat, p, fo_in, tau_old=float(tau_old[k]))
        out[:, k] = fo[po]
        tau[k] = tn
    return out, tau
