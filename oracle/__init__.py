"""FP64 CPU oracle for the Bingham LBM step: ctypes wrapper around oracle.c.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA path (``paper_1610_01388_gb300``) and imports
nothing from it.

The C file follows the paper's equations step by step (see its header for the
equation list and the readings taken where the printed text is garbled).  This
module adds only argument marshalling, the A/B time loop's Python entry, and
the flow-rate / residual diagnostics written out from their definitions:

* flow rate along axis a: Q_a = (1/L_a) * sum over fluid cells of u_real,a
  (volumetric flow through a cross-section, Sec. 4.5: Q / L^2 = U_avg);
* residual: sqrt(sum |u - u_prev|^2 / sum |u|^2) over fluid cells.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q15, D3Q19, D3Q27 = 0, 1, 2, 3
PR, IR = 0, 1
LATTICES = {"D2Q9": D2Q9, "D3Q15": D3Q15, "D3Q19": D3Q19, "D3Q27": D3Q27}
MODELS = {"PR": PR, "IR": IR}
DIAG_N = 44


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int),
        ("nu_p", ctypes.c_double),
        ("sigma_y", ctypes.c_double),
        ("m", ctypes.c_double),
        ("gdot_c", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("magic", ctypes.c_double),
        ("burnett_x", ctypes.c_int),
        ("newton", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
        vp = ctypes.c_void_p
        lib.orc_lattice_info.argtypes = [i, P(i), P(i), vp, vp]
        lib.orc_opposite.argtypes = [i, vp]
        lib.orc_feq.argtypes = [i, d, vp, vp]
        lib.orc_pr_nu_app.argtypes = [P(OrcParams), d, d]
        lib.orc_pr_nu_app.restype = d
        lib.orc_collide.argtypes = [i, P(OrcParams), vp, d, vp, vp, vp]
        lib.orc_step.argtypes = [i, P(OrcParams), i, i, i, vp, vp, vp, vp, vp, i]
        lib.orc_run.argtypes = [i, P(OrcParams), i, i, i, vp, vp, vp, i64, i]
        lib.orc_fields.argtypes = [i, P(OrcParams), i, i, i, vp, vp, vp, vp]
        lib.orc_step_cells.argtypes = [i, P(OrcParams), i, i, i, vp, vp, vp, i64, vp, vp, vp]
        lib.orc_num_threads.restype = i
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _lat(lattice):
    return LATTICES[lattice] if isinstance(lattice, str) else int(lattice)


def params(model="IR", nu_p=0.1, sigma_y=0.0, m=0.0, gdot_c=1e-8, g=(0.0, 0.0, 0.0),
           magic=0.25, burnett_x=False, newton=0) -> OrcParams:
    p = OrcParams()
    p.model = MODELS[model] if isinstance(model, str) else int(model)
    p.nu_p, p.sigma_y, p.m, p.gdot_c, p.magic = nu_p, sigma_y, m, gdot_c, magic
    p.burnett_x = 1 if burnett_x else 0
    p.newton = int(newton)
    gg = list(g) + [0.0] * (3 - len(g))
    p.g = (ctypes.c_double * 3)(*gg)
    return p


def lattice_info(lattice):
    """(c [Q,3] int, w [Q] float64, opp [Q] int) in the oracle's own order."""
    lib = _load()
    Q, D = ctypes.c_int(), ctypes.c_int()
    lib.orc_lattice_info(_lat(lattice), ctypes.byref(Q), ctypes.byref(D), None, None)
    c = np.zeros((Q.value, 3), np.int32)
    w = np.zeros(Q.value, np.float64)
    opp = np.zeros(Q.value, np.int32)
    lib.orc_lattice_info(_lat(lattice), ctypes.byref(Q), ctypes.byref(D), _ptr(c), _ptr(w))
    lib.orc_opposite(_lat(lattice), _ptr(opp))
    return c, w, opp


def dims(lattice):
    lib = _load()
    Q, D = ctypes.c_int(), ctypes.c_int()
    lib.orc_lattice_info(_lat(lattice), ctypes.byref(Q), ctypes.byref(D), None, None)
    return Q.value, D.value


def feq(lattice, rho, u):
    Q, _ = dims(lattice)
    out = np.zeros(Q, np.float64)
    uu = np.ascontiguousarray(list(u) + [0.0] * (3 - len(u)), dtype=np.float64)
    _load().orc_feq(_lat(lattice), float(rho), _ptr(uu), _ptr(out))
    return out


def pr_nu_app(p: OrcParams, gdot, rho=1.0):
    return _load().orc_pr_nu_app(ctypes.byref(p), float(gdot), float(rho))


def collide(lattice, p: OrcParams, fin, tau_old=0.0):
    """Collide one cell; returns (fout, tau_new, diag dict)."""
    Q, _ = dims(lattice)
    fin = np.ascontiguousarray(fin, np.float64)
    assert fin.shape == (Q,)
    fout = np.zeros(Q, np.float64)
    tn = ctypes.c_double()
    dg = np.zeros(DIAG_N, np.float64)
    _load().orc_collide(_lat(lattice), ctypes.byref(p), _ptr(fin), float(tau_old), _ptr(fout),
                        ctypes.byref(tn), _ptr(dg))
    diag = {
        "rho": dg[0], "u": dg[1:4].copy(), "T": dg[4:13].reshape(3, 3).copy(),
        "s": dg[13:22].reshape(3, 3).copy(), "sigma": dg[22:31].reshape(3, 3).copy(),
        "A": dg[31:40].reshape(3, 3).copy(), "gdot": dg[40], "nu_app": dg[41],
        "tau_new": dg[42], "yielded": bool(dg[43]),
    }
    return fout, tn.value, diag


class State:
    """Oracle state of one domain: full FP64 populations f[Q, N] (oracle order)
    and, for PR, the per-cell relaxation time."""

    def __init__(self, lattice, p: OrcParams, mask: np.ndarray, nthreads: int = 0):
        self.lat = _lat(lattice)
        self.p = p
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        if mask.ndim == 2:
            mask = mask[None, :, :]
        self.nz, self.ny, self.nx = mask.shape
        self.mask = mask
        self.N = mask.size
        self.Q, self.D = dims(lattice)
        self.nthreads = nthreads
        c, w, opp = lattice_info(lattice)
        self.c, self.w, self.opp = c, w, opp
        # rest state: f_i = w_i (rho = 1, u = 0)
        self.f = np.ascontiguousarray(np.repeat(w[:, None], self.N, axis=1))
        nu0 = p.nu_p + p.m * p.sigma_y
        self.tau = np.full(self.N, 0.5 + 3.0 * nu0, np.float64)

    def step(self, n=1):
        rc = _load().orc_run(self.lat, ctypes.byref(self.p), self.nx, self.ny, self.nz,
                             _ptr(self.mask), _ptr(self.f), _ptr(self.tau), int(n),
                             int(self.nthreads))
        if rc != 0:
            raise RuntimeError(f"orc_run failed: {rc}")

    def fields(self):
        """rho [nz,ny,nx], u [3,nz,ny,nx] (u_real; zeros on solid cells)."""
        rho = np.zeros(self.N, np.float64)
        u = np.zeros(3 * self.N, np.float64)
        rc = _load().orc_fields(self.lat, ctypes.byref(self.p), self.nx, self.ny, self.nz,
                                _ptr(self.mask), _ptr(self.f), _ptr(rho), _ptr(u))
        if rc != 0:
            raise RuntimeError("orc_fields failed")
        shp = (self.nz, self.ny, self.nx)
        return rho.reshape(shp), u.reshape((3,) + shp)

    def flowrate(self, axis=0):
        _, u = self.fields()
        L = (self.nx, self.ny, self.nz)[axis]
        return float(np.sum(u[axis][self.mask == 0])) / L

    def total_mass(self):
        fl = self.mask.reshape(-1) == 0
        return float(np.sum(self.f[:, fl]))

    def step_cells(self, cells):
        """Post-collision populations of the listed cells, [len(cells), Q]."""
        cells = np.ascontiguousarray(cells, np.int64)
        out = np.zeros((len(cells), self.Q), np.float64)
        tout = np.zeros(len(cells), np.float64)
        rc = _load().orc_step_cells(self.lat, ctypes.byref(self.p), self.nx, self.ny, self.nz,
                                    _ptr(self.mask), _ptr(self.f), _ptr(self.tau), len(cells),
                                    _ptr(cells), _ptr(out), _ptr(tout))
        if rc != 0:
            raise RuntimeError("orc_step_cells failed")
        return out, tout


def residual(u, u_prev, fluid):
    """sqrt(sum |u - u_prev|^2 / sum |u|^2) over fluid cells."""
    du = (u - u_prev)[:, fluid]
    uu = u[:, fluid]
    return float(np.sqrt(np.sum(du * du) / np.sum(uu * uu)))


def num_threads():
    return _load().orc_num_threads()
