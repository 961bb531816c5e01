"""Thin Python binding of the C ABI in include/bingham_lbm.h (ctypes).

Functions carry the C names and do argument marshalling only; every step of
the solver runs in libbingham_lbm.so's CUDA kernels.  There is no CPU
fallback: if the library is missing or fails to load, every call raises.
PyTorch, when used, only supplies device memory (the workspace tensor) and
the CUDA stream handle.

Array conventions: masks and fields are numpy arrays shaped (nz, ny, nx)
(x fastest, matching the C layout); populations are (Q, nz, ny, nx) full
FP64 values in the library's velocity order (``lbm_lattice_info``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbingham_lbm.so")

LBM_D2Q9, LBM_D3Q15, LBM_D3Q19, LBM_D3Q27 = 0, 1, 2, 3
LBM_MODEL_PR, LBM_MODEL_IR = 0, 1
LBM_F64, LBM_F32, LBM_F16_OFS, LBM_BF16_OFS = 0, 1, 2, 3
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_EBUSY, \
    LBM_EUNSUPPORTED = range(8)
LBM_FLAG_BURNETT_X = 0x1
LBM_FLAG_Z_GHOSTS = 0x2
LBM_FLAG_COMPACT = 0x4

LATTICES = {"D2Q9": LBM_D2Q9, "D3Q15": LBM_D3Q15, "D3Q19": LBM_D3Q19, "D3Q27": LBM_D3Q27}
MODELS = {"PR": LBM_MODEL_PR, "IR": LBM_MODEL_IR}
STORAGES = {"F64": LBM_F64, "F32": LBM_F32, "F16": LBM_F16_OFS, "BF16": LBM_BF16_OFS}
EXPORTED = ["lbm_params_default", "lbm_lattice_info", "lbm_workspace_bytes", "lbm_create",
            "lbm_create_with_workspace", "lbm_step", "lbm_sync", "lbm_fields", "lbm_fields_device",
            "lbm_flowrate", "lbm_totals", "lbm_residual", "lbm_set_populations",
            "lbm_get_populations", "lbm_set_tau", "lbm_get_tau", "lbm_get_info", "lbm_destroy",
            "lbm_last_error", "lbm_status_string", "lbm_flowrate_noalloc",
            "lbm_batch_create", "lbm_batch_add", "lbm_batch_remove", "lbm_batch_step",
            "lbm_batch_domain_status", "lbm_batch_solver", "lbm_batch_usage", "lbm_batch_destroy",
            "lbm_server_create", "lbm_server_submit", "lbm_server_advance", "lbm_server_result",
            "lbm_server_fields", "lbm_server_pending", "lbm_server_now", "lbm_server_destroy",
            "lbm_tuning_set", "lbm_tuning_get", "lbm_tuning_clear", "lbm_set_wait_limit",
            "lbm_get_wait_limit", "lbm_get_populations_cells", "lbm_tuning_set_shape",
            "lbm_tuning_get_shape", "lbm_tuning_set_batch", "lbm_tuning_get_batch",
            "lbm_tuning_set_batch_concurrency", "lbm_tuning_get_batch_concurrency",
            "lbm_tuning_set_batch_tile", "lbm_tuning_get_batch_tile",
            "lbm_halo_bytes", "lbm_halo_pack", "lbm_halo_unpack", "lbm_set_hash_offset",
            "lbm_check_sums", "lbm_step_cells", "lbm_step_commit",
            "lbm_workspace_bytes_for_mask"]
LBM_REQ_QUEUED, LBM_REQ_RUNNING, LBM_REQ_CONVERGED, LBM_REQ_CAPPED, LBM_REQ_FAILED = range(5)
LBM_STEADY_FLOW, LBM_STEADY_RESIDUAL = 0, 1


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"[{status}] {msg}")
        self.status = status


class lbm_params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("mu_p", ctypes.c_double), ("sigma_y", ctypes.c_double),
                ("m", ctypes.c_double), ("gammadot_c", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("magic", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("newton_iters", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class lbm_info(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int32), ("Q", ctypes.c_int32), ("D", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("cells", ctypes.c_int64), ("fluid_cells", ctypes.c_int64),
                ("steps_done", ctypes.c_int64), ("model", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("bytes_per_fluid_update", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t)]


class lbm_domain_status(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("checks", ctypes.c_int64),
                ("residual", ctypes.c_double), ("flow", ctypes.c_double * 3),
                ("nonfinite", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("flow_change", ctypes.c_double)]


class lbm_request(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("solid_mask", ctypes.c_void_p), ("params", lbm_params),
                ("tolerance", ctypes.c_double), ("max_steps", ctypes.c_int64),
                ("keep_fields", ctypes.c_int32), ("criterion", ctypes.c_int32)]


class lbm_result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("pad", ctypes.c_int32), ("steps", ctypes.c_int64),
                ("fluid_cells", ctypes.c_int64), ("residual", ctypes.c_double),
                ("flow_x", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def library():
    """Load libbingham_lbm.so (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise LbmError(LBM_EUNSUPPORTED,
                           f"CUDA library not built: {LIB_PATH} is missing "
                           "(run __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        P, vp = ctypes.POINTER, ctypes.c_void_p
        i32, i64, d, sz = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        sig = {
            "lbm_params_default": [P(lbm_params)],
            "lbm_lattice_info": [i32, P(i32), P(i32), vp, vp],
            "lbm_workspace_bytes": [i32, i32, i32, i32, P(lbm_params), P(sz)],
            "lbm_workspace_bytes_for_mask": [i32, i32, i32, i32, vp, P(lbm_params), P(sz)],
            "lbm_create": [P(vp), i32, i32, i32, i32, vp, P(lbm_params), vp],
            "lbm_create_with_workspace": [P(vp), i32, i32, i32, i32, vp, P(lbm_params), vp, vp, sz],
            "lbm_step": [vp, i64],
            "lbm_sync": [vp],
            "lbm_fields": [vp, vp, vp, vp, vp],
            "lbm_fields_device": [vp, vp, vp, vp, vp],
            "lbm_flowrate": [vp, i32, P(d)],
            "lbm_totals": [vp, P(d), vp],
            "lbm_residual": [vp, P(d), P(i64), P(d)],
            "lbm_set_populations": [vp, vp],
            "lbm_get_populations": [vp, vp],
            "lbm_set_tau": [vp, vp],
            "lbm_get_tau": [vp, vp],
            "lbm_get_info": [vp, P(lbm_info)],
            "lbm_flowrate_noalloc": [vp, i32, vp],
            "lbm_batch_create": [P(vp), sz, i32, vp],
            "lbm_batch_add": [vp, i32, i32, i32, i32, vp, P(lbm_params), P(i64)],
            "lbm_batch_remove": [vp, i64],
            "lbm_batch_step": [vp, i64],
            "lbm_batch_domain_status": [vp, i64, P(lbm_domain_status)],
            "lbm_batch_solver": [vp, i64, P(vp)],
            "lbm_batch_usage": [vp, P(sz), P(i64), P(i64)],
            "lbm_server_create": [P(vp), sz, i32, vp],
            "lbm_server_submit": [vp, P(lbm_request), P(i64)],
            "lbm_server_advance": [vp, i64, P(i32)],
            "lbm_server_result": [vp, i64, P(lbm_result)],
            "lbm_server_fields": [vp, i64, vp, vp, vp, vp],
            "lbm_server_pending": [vp, P(i64), P(i64), P(sz)],
            "lbm_server_now": [vp, P(d)],
            "lbm_tuning_set": [i32, i32, i32, i32, i32],
            "lbm_tuning_get": [i32, i32, i32, i64, P(i32), P(i32)],
            "lbm_tuning_clear": [],
            "lbm_tuning_set_shape": [i32, i32, i32, i32, i32, i32],
            "lbm_tuning_get_shape": [i32, i32, i32, i64, P(i32), P(i32), P(i32)],
            "lbm_set_wait_limit": [ctypes.c_double],
            "lbm_get_populations_cells": [vp, vp, i64, vp],
            "lbm_tuning_set_batch": [i32, i32, i32, i32],
            "lbm_tuning_get_batch": [i32, i32, i32, P(i32)],
            "lbm_tuning_set_batch_concurrency": [i32],
            "lbm_tuning_get_batch_concurrency": [P(i32)],
            "lbm_tuning_set_batch_tile": [i32, i32, i32, i32, i32, i32],
            "lbm_halo_bytes": [vp, P(sz)],
            "lbm_halo_pack": [vp, i32, vp],
            "lbm_halo_unpack": [vp, i32, vp],
            "lbm_set_hash_offset": [vp, i64],
            "lbm_check_sums": [vp, vp, P(d), P(d)],
            "lbm_step_cells": [vp, i64, i64],
            "lbm_step_commit": [vp],
            "lbm_tuning_get_batch_tile": [i32, i32, i32, i64, P(i32), P(i32), P(i32)],
            "lbm_get_wait_limit": [P(d)],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        for name in ("lbm_destroy", "lbm_batch_destroy", "lbm_server_destroy"):
            getattr(lib, name).argtypes = [vp]
            getattr(lib, name).restype = None
        lib.lbm_last_error.restype = ctypes.c_char_p
        lib.lbm_status_string.restype = ctypes.c_char_p
        lib.lbm_status_string.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _check(st):
    if st != LBM_OK:
        msg = library().lbm_last_error().decode(errors="replace")
        raise LbmError(st, msg)


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _lat(x):
    return LATTICES[x] if isinstance(x, str) else int(x)


# --- C-named functions ------------------------------------------------------

def lbm_params_default(**kw) -> lbm_params:
    p = lbm_params()
    _check(library().lbm_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if k == "g":
            gg = list(v) + [0.0] * (3 - len(v))
            p.g = (ctypes.c_double * 3)(*gg)
        elif k == "model":
            p.model = MODELS[v] if isinstance(v, str) else int(v)
        elif k == "storage":
            p.storage = STORAGES[v] if isinstance(v, str) else int(v)
        else:
            setattr(p, k, v)
    return p


def lbm_lattice_info(lat):
    lib = library()
    Q, D = ctypes.c_int(), ctypes.c_int()
    _check(lib.lbm_lattice_info(_lat(lat), ctypes.byref(Q), ctypes.byref(D), None, None))
    c = np.zeros((Q.value, 3), np.int32)
    w = np.zeros(Q.value, np.float64)
    _check(lib.lbm_lattice_info(_lat(lat), ctypes.byref(Q), ctypes.byref(D), _ptr(c), _ptr(w)))
    return c, w


def lbm_workspace_bytes(lat, nx, ny, nz, params) -> int:
    b = ctypes.c_size_t()
    _check(library().lbm_workspace_bytes(_lat(lat), nx, ny, nz, ctypes.byref(params),
                                         ctypes.byref(b)))
    return b.value


def lbm_workspace_bytes_for_mask(lat, mask, params) -> int:
    """mask: uint8 (nz, ny, nx) or (ny, nx)."""
    mask = np.ascontiguousarray(mask, np.uint8)
    if mask.ndim == 2:
        mask = mask[None]
    nz, ny, nx = mask.shape
    b = ctypes.c_size_t()
    _check(library().lbm_workspace_bytes_for_mask(_lat(lat), nx, ny, nz, _ptr(mask),
                                                  ctypes.byref(params), ctypes.byref(b)))
    return b.value


def lbm_create(lat, mask, params, stream=None, workspace=None):
    """mask: uint8 (nz, ny, nx) or (ny, nx); stream: int handle or None;
    workspace: (device pointer, bytes) or None."""
    mask = np.ascontiguousarray(mask, np.uint8)
    if mask.ndim == 2:
        mask = mask[None]
    nz, ny, nx = mask.shape
    h = ctypes.c_void_p()
    lib = library()
    if workspace is None:
        _check(lib.lbm_create(ctypes.byref(h), _lat(lat), nx, ny, nz, _ptr(mask),
                              ctypes.byref(params), ctypes.c_void_p(stream or 0)))
    else:
        ptr, nbytes = workspace
        _check(lib.lbm_create_with_workspace(ctypes.byref(h), _lat(lat), nx, ny, nz, _ptr(mask),
                                             ctypes.byref(params), ctypes.c_void_p(stream or 0),
                                             ctypes.c_void_p(ptr), nbytes))
    return h


def lbm_step(h, n):
    _check(library().lbm_step(h, int(n)))


def lbm_sync(h):
    _check(library().lbm_sync(h))


def lbm_get_info(h) -> lbm_info:
    i = lbm_info()
    _check(library().lbm_get_info(h, ctypes.byref(i)))
    return i


def lbm_fields(h):
    inf = lbm_get_info(h)
    n = inf.cells
    rho = np.empty(n, np.float64)
    u = np.empty((3, n), np.float64)
    _check(library().lbm_fields(h, _ptr(rho), _ptr(u[0]), _ptr(u[1]), _ptr(u[2])))
    shp = (inf.nz, inf.ny, inf.nx)
    return rho.reshape(shp), u.reshape((3,) + shp)


def lbm_fields_device(h, rho_ptr, ux_ptr, uy_ptr, uz_ptr):
    vp = ctypes.c_void_p
    _check(library().lbm_fields_device(h, vp(rho_ptr), vp(ux_ptr), vp(uy_ptr), vp(uz_ptr)))


def lbm_flowrate(h, axis=0) -> float:
    q = ctypes.c_double()
    _check(library().lbm_flowrate(h, int(axis), ctypes.byref(q)))
    return q.value


def lbm_flowrate_noalloc(h, axis, q_device_ptr):
    """Flow rate written to a caller-owned device double; allocates nothing and
    does not synchronise (see the header for the shared static scratch)."""
    _check(library().lbm_flowrate_noalloc(h, int(axis), ctypes.c_void_p(q_device_ptr)))


def lbm_totals(h):
    m = ctypes.c_double()
    j = np.zeros(3, np.float64)
    _check(library().lbm_totals(h, ctypes.byref(m), _ptr(j)))
    return m.value, j


def lbm_residual(h):
    """(residual, step index, flow rate along x) of the last check step.
    Raises LbmError(LBM_ENONFINITE) if that check step saw a non-finite density."""
    r, s, q = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    _check(library().lbm_residual(h, ctypes.byref(r), ctypes.byref(s), ctypes.byref(q)))
    return r.value, s.value, q.value


def lbm_set_populations(h, f):
    f = np.ascontiguousarray(f, np.float64)
    inf = lbm_get_info(h)
    if f.size != inf.Q * inf.cells:
        raise LbmError(LBM_EINVAL, f"populations must have {inf.Q * inf.cells} values")
    _check(library().lbm_set_populations(h, _ptr(f)))


def lbm_get_populations(h):
    inf = lbm_get_info(h)
    f = np.empty((inf.Q, inf.nz, inf.ny, inf.nx), np.float64)
    _check(library().lbm_get_populations(h, _ptr(f)))
    return f


def lbm_set_tau(h, tau):
    tau = np.ascontiguousarray(tau, np.float64)
    _check(library().lbm_set_tau(h, _ptr(tau)))


def lbm_get_tau(h):
    inf = lbm_get_info(h)
    t = np.empty((inf.nz, inf.ny, inf.nx), np.float64)
    _check(library().lbm_get_tau(h, _ptr(t)))
    return t


def lbm_destroy(h):
    if h:
        library().lbm_destroy(h)


def _mdl(x):
    return MODELS[x] if isinstance(x, str) else int(x)


def _sto(x):
    return STORAGES[x] if isinstance(x, str) else int(x)


def lbm_tuning_set(lat, model, storage, size_class, block):
    _check(library().lbm_tuning_set(_lat(lat), _mdl(model), _sto(storage), int(size_class),
                                    int(block)))


def lbm_tuning_get(lat, model, storage, cells):
    """(block, size class) the library uses for a problem of `cells` cells."""
    b, c = ctypes.c_int32(), ctypes.c_int32()
    _check(library().lbm_tuning_get(_lat(lat), _mdl(model), _sto(storage), int(cells),
                                    ctypes.byref(b), ctypes.byref(c)))
    return b.value, c.value


def lbm_tuning_clear():
    _check(library().lbm_tuning_clear())


def lbm_tuning_set_shape(lat, model, storage, size_class, block, cells_per_thread):
    _check(library().lbm_tuning_set_shape(_lat(lat), _mdl(model), _sto(storage), int(size_class),
                                          int(block), int(cells_per_thread)))


def lbm_tuning_get_shape(lat, model, storage, cells):
    """(block, cells per thread, size class) the library uses for `cells` cells."""
    b, c, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(library().lbm_tuning_get_shape(_lat(lat), _mdl(model), _sto(storage), int(cells),
                                          ctypes.byref(b), ctypes.byref(c), ctypes.byref(k)))
    return b.value, c.value, k.value


def lbm_tuning_set_batch(lat, model, storage, ctas_per_sm):
    _check(library().lbm_tuning_set_batch(_lat(lat), _mdl(model), _sto(storage),
                                          int(ctas_per_sm)))


def lbm_tuning_get_batch(lat, model, storage) -> int:
    v = ctypes.c_int32()
    _check(library().lbm_tuning_get_batch(_lat(lat), _mdl(model), _sto(storage),
                                          ctypes.byref(v)))
    return v.value


def lbm_tuning_set_batch_tile(lat, model, storage, size_class, threads, cells_per_thread):
    _check(library().lbm_tuning_set_batch_tile(_lat(lat), _mdl(model), _sto(storage),
                                               int(size_class), int(threads),
                                               int(cells_per_thread)))


def lbm_tuning_get_batch_tile(lat, model, storage, mean_cells):
    """(threads, cells per thread, size class) a group of this mean size runs."""
    t, c, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(library().lbm_tuning_get_batch_tile(_lat(lat), _mdl(model), _sto(storage),
                                               int(mean_cells), ctypes.byref(t), ctypes.byref(c),
                                               ctypes.byref(k)))
    return t.value, c.value, k.value


def lbm_tuning_set_batch_concurrency(on):
    _check(library().lbm_tuning_set_batch_concurrency(1 if on else 0))


def lbm_tuning_get_batch_concurrency() -> bool:
    v = ctypes.c_int32()
    _check(library().lbm_tuning_get_batch_concurrency(ctypes.byref(v)))
    return bool(v.value)


def lbm_get_populations_cells(h, cells, Q):
    """(Q, n) FP64 populations of the listed cells, library velocity order."""
    cells = np.ascontiguousarray(cells, np.int64)
    out = np.zeros((Q, cells.size), np.float64)
    _check(library().lbm_get_populations_cells(h, _ptr(cells), cells.size, _ptr(out)))
    return out


def lbm_halo_bytes(h) -> int:
    b = ctypes.c_size_t()
    _check(library().lbm_halo_bytes(h, ctypes.byref(b)))
    return b.value


def lbm_halo_pack(h, side, buf_ptr):
    _check(library().lbm_halo_pack(h, int(side), ctypes.c_void_p(buf_ptr)))


def lbm_halo_unpack(h, side, buf_ptr):
    _check(library().lbm_halo_unpack(h, int(side), ctypes.c_void_p(buf_ptr)))


def lbm_set_hash_offset(h, offset):
    _check(library().lbm_set_hash_offset(h, int(offset)))


def lbm_check_sums(h):
    """(usum[3], du2, u2) of the last check step."""
    us = (ctypes.c_double * 3)()
    du2, u2 = ctypes.c_double(), ctypes.c_double()
    _check(library().lbm_check_sums(h, us, ctypes.byref(du2), ctypes.byref(u2)))
    return np.array(list(us)), du2.value, u2.value


def lbm_step_cells(h, cell_begin, cell_end):
    _check(library().lbm_step_cells(h, int(cell_begin), int(cell_end)))


def lbm_step_commit(h):
    _check(library().lbm_step_commit(h))


def lbm_set_wait_limit(seconds):
    _check(library().lbm_set_wait_limit(float(seconds)))


def lbm_get_wait_limit() -> float:
    v = ctypes.c_double()
    _check(library().lbm_get_wait_limit(ctypes.byref(v)))
    return v.value


# --- convenience wrapper ----------------------------------------------------

class Solver:
    """One domain on the current CUDA device.

    With ``use_torch=True`` the device memory is a torch uint8 tensor (kept
    alive by this object) and work goes to torch's current stream; otherwise
    the library allocates with cudaMalloc and uses the legacy default stream.
    """

    def __init__(self, lattice, mask, model="IR", storage="F32", mu_p=0.1, sigma_y=0.0, m=0.0,
                 gammadot_c=1e-8, g=(0.0, 0.0, 0.0), magic=0.25, check_every=0, flags=0,
                 newton_iters=0, use_torch=False, stream=None, layout="dense"):
        """layout: "dense" (every cell held) or "compact" (fluid cells only,
        LBM_FLAG_COMPACT)."""
        if layout not in ("dense", "compact"):
            raise ValueError(f"layout must be 'dense' or 'compact' (got {layout!r})")
        if layout == "compact":
            flags |= LBM_FLAG_COMPACT
        self.lattice = lattice
        self.params = lbm_params_default(model=model, storage=storage, mu_p=mu_p,
                                         sigma_y=sigma_y, m=m, gammadot_c=gammadot_c, g=g,
                                         magic=magic, check_every=check_every, flags=flags,
                                         newton_iters=newton_iters)
        mask = np.ascontiguousarray(mask, np.uint8)
        if mask.ndim == 2:
            mask = mask[None]
        self.mask = mask
        self._ws = None
        ws = None
        if use_torch:
            import torch
            nb = lbm_workspace_bytes_for_mask(lattice, mask, self.params)
            self._ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
            ws = (self._ws.data_ptr(), nb)
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
        self.h = lbm_create(lattice, mask, self.params, stream=stream, workspace=ws)
        self.info = lbm_get_info(self.h)

    def step(self, n=1):
        lbm_step(self.h, n)

    def sync(self):
        lbm_sync(self.h)

    def fields(self):
        return lbm_fields(self.h)

    def flowrate(self, axis=0):
        return lbm_flowrate(self.h, axis)

    def totals(self):
        return lbm_totals(self.h)

    def residual(self):
        return lbm_residual(self.h)

    def set_populations(self, f):
        lbm_set_populations(self.h, f)

    def get_populations(self):
        return lbm_get_populations(self.h)

    def set_tau(self, t):
        lbm_set_tau(self.h, t)

    def get_tau(self):
        return lbm_get_tau(self.h)

    @property
    def steps_done(self):
        return lbm_get_info(self.h).steps_done

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# --- batched stepping ---------------------------------------------------------

class Batch:
    """Many resident domains stepped together (lbm_batch_*)."""

    def __init__(self, budget_bytes, check_every=100, stream=None):
        self.h = ctypes.c_void_p()
        _check(library().lbm_batch_create(ctypes.byref(self.h), int(budget_bytes),
                                          int(check_every), ctypes.c_void_p(stream or 0)))

    def add(self, lattice, mask, **params):
        mask = np.ascontiguousarray(mask, np.uint8)
        if mask.ndim == 2:
            mask = mask[None]
        nz, ny, nx = mask.shape
        p = lbm_params_default(**params)
        i = ctypes.c_int64()
        _check(library().lbm_batch_add(self.h, _lat(lattice), nx, ny, nz, _ptr(mask),
                                       ctypes.byref(p), ctypes.byref(i)))
        return i.value

    def try_add(self, lattice, mask, **params):
        """Domain id, or None if the budget is exhausted (LBM_EBUSY)."""
        try:
            return self.add(lattice, mask, **params)
        except LbmError as e:
            if e.status == LBM_EBUSY:
                return None
            raise

    def remove(self, dom):
        _check(library().lbm_batch_remove(self.h, int(dom)))

    def step(self, n):
        _check(library().lbm_batch_step(self.h, int(n)))

    def status(self, dom):
        st = lbm_domain_status()
        _check(library().lbm_batch_domain_status(self.h, int(dom), ctypes.byref(st)))
        return st

    def solver(self, dom):
        """Borrowed lbm_solver handle (for lbm_fields, lbm_flowrate, ...)."""
        s = ctypes.c_void_p()
        _check(library().lbm_batch_solver(self.h, int(dom), ctypes.byref(s)))
        return s

    def usage(self):
        b, d, c = ctypes.c_size_t(), ctypes.c_int64(), ctypes.c_int64()
        _check(library().lbm_batch_usage(self.h, ctypes.byref(b), ctypes.byref(d),
                                         ctypes.byref(c)))
        return b.value, d.value, c.value

    def close(self):
        if getattr(self, "h", None):
            library().lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- serving ----------------------------------------------------------------------

class Server:
    """Continuous-batching server of independent solves (lbm_server_*)."""

    def __init__(self, budget_bytes, check_every=100, stream=None):
        self.h = ctypes.c_void_p()
        _check(library().lbm_server_create(ctypes.byref(self.h), int(budget_bytes),
                                           int(check_every), ctypes.c_void_p(stream or 0)))

    def submit(self, lattice, mask, tolerance=1e-6, max_steps=100000, keep_fields=False,
               criterion="flow", **params):
        """criterion "flow": relative change of the mean velocity vector per
        check interval below tolerance; "residual": the field residual."""
        mask = np.ascontiguousarray(mask, np.uint8)
        if mask.ndim == 2:
            mask = mask[None]
        nz, ny, nx = mask.shape
        r = lbm_request()
        r.lattice, r.nx, r.ny, r.nz = _lat(lattice), nx, ny, nz
        r.solid_mask = mask.ctypes.data
        r.params = lbm_params_default(**params)
        r.tolerance = float(tolerance)
        r.max_steps = int(max_steps)
        r.keep_fields = 1 if keep_fields else 0
        r.criterion = {"flow": LBM_STEADY_FLOW, "residual": LBM_STEADY_RESIDUAL}[criterion]
        i = ctypes.c_int64()
        _check(library().lbm_server_submit(self.h, ctypes.byref(r), ctypes.byref(i)))
        return i.value

    def advance(self, nsteps):
        c = ctypes.c_int32()
        _check(library().lbm_server_advance(self.h, int(nsteps), ctypes.byref(c)))
        return c.value

    def result(self, rid):
        r = lbm_result()
        _check(library().lbm_server_result(self.h, int(rid), ctypes.byref(r)))
        return r

    def fields(self, rid, shape):
        n = int(np.prod(shape))
        out = np.empty((4, n), np.float64)
        _check(library().lbm_server_fields(self.h, int(rid), _ptr(out[0]), _ptr(out[1]),
                                           _ptr(out[2]), _ptr(out[3])))
        return out[0].reshape(shape), out[1:].reshape((3,) + tuple(shape))

    def pending(self):
        q, r, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        _check(library().lbm_server_pending(self.h, ctypes.byref(q), ctypes.byref(r),
                                            ctypes.byref(b)))
        return q.value, r.value, b.value

    def now(self):
        t = ctypes.c_double()
        _check(library().lbm_server_now(self.h, ctypes.byref(t)))
        return t.value

    def close(self):
        if getattr(self, "h", None):
            library().lbm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
