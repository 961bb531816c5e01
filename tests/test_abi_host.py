"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every symbol include/bingham_lbm.h declares; the GPU path's own
velocity tables satisfy the lattice identities; argument validation rejects
bad input before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1610_01388_gb300 import _build
from paper_1610_01388_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    yield


def _declared():
    txt = open(os.path.join(ROOT, "include", "bingham_lbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = lbm.library()
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(lbm.EXPORTED) <= set(names)


LATS = {"D2Q9": (9, 2), "D3Q15": (15, 3), "D3Q19": (19, 3), "D3Q27": (27, 3)}


@pytest.mark.parametrize("lat", list(LATS))
def test_gpu_lattice_tables(lat):
    c, w = lbm.lbm_lattice_info(lat)
    Q, D = LATS[lat]
    assert c.shape == (Q, 3)
    assert len({tuple(v) for v in c}) == Q
    assert tuple(c[0]) == (0, 0, 0)
    for i in range(1, Q, 2):          # opposite pairs are adjacent
        assert np.array_equal(c[i + 1], -c[i]) and w[i] == w[i + 1]
    cf = c.astype(np.float64)
    d = np.zeros((3, 3))
    d[:D, :D] = np.eye(D)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(cf.T @ w, 0)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, cf, cf), d / 3, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, cf, cf, cf, cf)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(m4, iso, atol=1e-16)


def test_params_default():
    p = lbm.lbm_params_default()
    assert p.model == lbm.LBM_MODEL_IR and p.storage == lbm.LBM_F32
    assert p.mu_p == 0.1 and p.gammadot_c == 1e-8 and p.magic == 0.25 and p.check_every == 0
    assert p.newton_iters == 0 and p.reserved == 0


def _create_status(lat, mask, **kw):
    lib = lbm.library()
    p = lbm.lbm_params_default(**kw)
    mask = np.ascontiguousarray(mask, np.uint8)
    if mask.ndim == 2:
        mask = mask[None]
    nz, ny, nx = mask.shape
    h = ctypes.c_void_p()
    st = lib.lbm_create(ctypes.byref(h), lbm.LATTICES[lat], nx, ny, nz,
                        ctypes.c_void_p(mask.ctypes.data), ctypes.byref(p), None)
    if st == lbm.LBM_OK:
        lib.lbm_destroy(h)
    return st, lib.lbm_last_error().decode()


@pytest.mark.parametrize("lat,mask,kw,expect", [
    ("D2Q9", np.zeros((2, 4, 4)), {}, "nz == 1"),
    ("D3Q19", np.ones((2, 2, 2)), {}, "no fluid"),
    ("D3Q19", np.zeros((2, 2, 2)), {"mu_p": 0.0}, "mu_p"),
    ("D3Q19", np.zeros((2, 2, 2)), {"mu_p": float("nan")}, "mu_p"),
    ("D3Q19", np.zeros((2, 2, 2)), {"sigma_y": -1.0}, "sigma_y"),
    ("D3Q19", np.zeros((2, 2, 2)), {"model": "PR", "gammadot_c": 0.0}, "gammadot_c"),
    ("D3Q19", np.zeros((2, 2, 2)), {"model": "PR", "m": -1.0}, "m must"),
    ("D3Q19", np.zeros((2, 2, 2)), {"model": "PR", "magic": 0.0}, "magic"),
    ("D2Q9", np.zeros((1, 4, 4)), {"g": (0, 0, 1e-6)}, "g[2]"),
    ("D3Q19", np.zeros((2, 2, 2)), {"check_every": -1}, "check_every"),
    ("D3Q19", np.zeros((2, 2, 2)), {"flags": 0x80}, "flags"),
    ("D3Q19", np.zeros((2, 2, 2)), {"model": "PR", "newton_iters": -1}, "newton_iters"),
    ("D3Q19", np.zeros((2, 2, 2)), {"model": "PR", "newton_iters": 65}, "newton_iters"),
    ("D3Q19", np.zeros((2, 2, 2)), {"reserved": 1}, "reserved"),
    ("D3Q19", np.zeros((2, 2, 2)), {"flags": 0x2}, "ghost planes"),            # nz < 3
    ("D2Q9", np.zeros((1, 4, 4)), {"flags": 0x2}, "ghost planes"),
    # ghost planes are not stepped: a slab whose interior is all solid has no fluid
    ("D3Q19", np.concatenate([np.zeros((1, 2, 2)), np.ones((1, 2, 2)), np.zeros((1, 2, 2))]),
     {"flags": 0x2}, "no fluid"),
    # the compact layout holds no ghost planes
    ("D3Q19", np.zeros((4, 2, 2)), {"flags": 0x2 | 0x4}, "dense layout"),
    ("D3Q19", np.ones((2, 2, 2)), {"flags": 0x4}, "no fluid"),
])
def test_create_rejects_invalid_arguments(lat, mask, kw, expect):
    st, msg = _create_status(lat, mask, **kw)
    assert st == lbm.LBM_EINVAL
    assert expect in msg


def test_halo_calls_reject_null_handle():
    lib = lbm.library()
    b = ctypes.c_size_t()
    assert lib.lbm_halo_bytes(None, ctypes.byref(b)) == lbm.LBM_EINVAL
    assert lib.lbm_halo_pack(None, 0, None) == lbm.LBM_EINVAL
    assert lib.lbm_halo_unpack(None, 1, None) == lbm.LBM_EINVAL
    assert lib.lbm_set_hash_offset(None, 5) == lbm.LBM_EINVAL
    assert lib.lbm_check_sums(None, None, None, None) == lbm.LBM_EINVAL
    assert lib.lbm_step_cells(None, 0, 1) == lbm.LBM_EINVAL
    assert lib.lbm_step_commit(None) == lbm.LBM_EINVAL


def test_create_rejects_empty_and_oversized_extents():
    lib = lbm.library()
    p = lbm.lbm_params_default()
    h = ctypes.c_void_p()
    m = np.zeros(1, np.uint8)
    assert lib.lbm_create(ctypes.byref(h), 1, 0, 1, 1, ctypes.c_void_p(m.ctypes.data),
                          ctypes.byref(p), None) == lbm.LBM_EINVAL
    b = ctypes.c_size_t()
    assert lib.lbm_workspace_bytes(3, 2048, 2048, 1024, ctypes.byref(p),
                                   ctypes.byref(b)) == lbm.LBM_EINVAL
    assert lib.lbm_create(ctypes.byref(h), 1, 4, 4, 4, None, ctypes.byref(p),
                          None) == lbm.LBM_EINVAL


def test_workspace_bytes_cover_the_layout():
    p = lbm.lbm_params_default(model="PR", check_every=10)
    n = lbm.lbm_workspace_bytes("D3Q27", 256, 128, 128, p)
    cells = 256 * 128 * 128
    # two population buffers, links, tau, 3-component snapshot, mask
    assert n >= 2 * 27 * 4 * cells + 4 * cells + 4 * cells + 12 * cells + cells
    p64 = lbm.lbm_params_default(model="IR", storage="F64")
    assert lbm.lbm_workspace_bytes("D3Q27", 256, 128, 128, p64) >= 2 * 27 * 8 * cells


def test_workspace_bytes_for_mask_size_the_compact_layout():
    """The mask-aware size is exact: equal to the maskless one for the dense
    layout, and for the compact one the fluid cells' planes plus the two slot
    maps (cell index per slot, slot per cell), below the maskless bound."""
    mask = np.ones((16, 16, 64), np.uint8)
    mask[:, :, :16] = 0                                # 4096 fluid cells of 16384
    for model in ("PR", "IR"):
        for storage in ("F32", "F16", "F64"):
            d = lbm.lbm_params_default(model=model, storage=storage, check_every=10)
            c = lbm.lbm_params_default(model=model, storage=storage, check_every=10,
                                       flags=lbm.LBM_FLAG_COMPACT)
            dense = lbm.lbm_workspace_bytes_for_mask("D3Q19", mask, d)
            assert dense == lbm.lbm_workspace_bytes("D3Q19", 64, 16, 16, d)
            comp = lbm.lbm_workspace_bytes_for_mask("D3Q19", mask, c)
            bound = lbm.lbm_workspace_bytes("D3Q19", 64, 16, 16, c)
            sb = {"F32": 4, "F16": 2, "F64": 8}[storage]
            rs = 8 if storage == "F64" else 4
            per_slot = 2 * 19 * sb + 4 + 4 + 3 * rs + (rs if model == "PR" else 0)
            assert comp >= 4096 * per_slot + 16384 * (1 + 4)
            assert comp < dense < bound
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_bytes_for_mask("D3Q19", np.ones((2, 2, 2), np.uint8),
                                         lbm.lbm_params_default())


def test_tuning_table_host_logic():
    lbm.lbm_tuning_clear()
    assert lbm.lbm_tuning_get("D3Q27", "IR", "F32", 4_194_304) == (256, 22)
    assert lbm.lbm_tuning_get("D2Q9", "PR", "F16", 1) == (256, 0)
    lbm.lbm_tuning_set("D3Q27", "IR", "F32", 22, 512)
    assert lbm.lbm_tuning_get("D3Q27", "IR", "F32", 5_000_000) == (512, 22)
    assert lbm.lbm_tuning_get("D3Q27", "PR", "F32", 5_000_000)[0] == 256   # other key
    assert lbm.lbm_tuning_get("D3Q27", "IR", "F32", 9_000_000)[0] == 256   # other class
    lib = lbm.library()
    assert lib.lbm_tuning_set(3, 1, 1, 22, 300) == lbm.LBM_EINVAL
    assert lib.lbm_tuning_set(3, 1, 9, 22, 256) == lbm.LBM_EINVAL
    assert lib.lbm_tuning_set(9, 1, 1, 22, 256) == lbm.LBM_EINVAL
    lbm.lbm_tuning_clear()
    assert lbm.lbm_tuning_get("D3Q27", "IR", "F32", 5_000_000)[0] == 256


def test_tuning_shape_host_logic():
    lbm.lbm_tuning_clear()
    assert lbm.lbm_tuning_get_shape("D3Q27", "PR", "F32", 4_194_304) == (256, 1, 22)
    lbm.lbm_tuning_set_shape("D3Q27", "PR", "F32", 22, 128, 2)
    assert lbm.lbm_tuning_get_shape("D3Q27", "PR", "F32", 5_000_000) == (128, 2, 22)
    assert lbm.lbm_tuning_get("D3Q27", "PR", "F32", 5_000_000) == (128, 22)
    lbm.lbm_tuning_set("D3Q27", "PR", "F32", 22, 512)          # plain set: one cell per thread
    assert lbm.lbm_tuning_get_shape("D3Q27", "PR", "F32", 5_000_000) == (512, 1, 22)
    lib = lbm.library()
    assert lib.lbm_tuning_set_shape(3, 0, 1, 22, 512, 2) == lbm.LBM_EINVAL    # 512 x 2
    assert lib.lbm_tuning_set_shape(3, 0, 0, 22, 128, 2) == lbm.LBM_EINVAL    # F64
    assert lib.lbm_tuning_set_shape(3, 0, 1, 22, 128, 3) == lbm.LBM_EINVAL
    lbm.lbm_tuning_set_shape("D2Q9", "IR", "F16", 10, 256, 2)
    assert lbm.lbm_tuning_get_shape("D2Q9", "IR", "F16", 1500) == (256, 2, 10)
    lbm.lbm_tuning_clear()
    assert lbm.lbm_tuning_get_shape("D2Q9", "IR", "F16", 1500) == (256, 1, 10)


def test_batch_schedule_host_logic():
    lbm.lbm_tuning_clear()
    assert lbm.lbm_tuning_get_batch("D3Q27", "PR", "F16") == 0
    assert lbm.lbm_tuning_get_batch_concurrency() is False
    lbm.lbm_tuning_set_batch("D3Q27", "PR", "F16", 4)
    lbm.lbm_tuning_set_batch_concurrency(True)
    assert lbm.lbm_tuning_get_batch("D3Q27", "PR", "F16") == 4
    assert lbm.lbm_tuning_get_batch("D3Q27", "IR", "F16") == 0      # other key
    assert lbm.lbm_tuning_get_batch_concurrency() is True
    lib = lbm.library()
    assert lib.lbm_tuning_set_batch(3, 0, 2, 33) == lbm.LBM_EINVAL
    assert lib.lbm_tuning_set_batch(3, 0, 2, -1) == lbm.LBM_EINVAL
    assert lib.lbm_tuning_set_batch(7, 0, 2, 1) == lbm.LBM_EINVAL
    assert lib.lbm_tuning_set_batch(3, 5, 2, 1) == lbm.LBM_EINVAL
    assert lib.lbm_tuning_set_batch_concurrency(2) == lbm.LBM_EINVAL
    lbm.lbm_tuning_clear()
    assert lbm.lbm_tuning_get_batch("D3Q27", "PR", "F16") == 0
    assert lbm.lbm_tuning_get_batch_concurrency() is False


def test_batch_tile_table_host_logic():
    """Plain-step tile shape per (lattice, model, storage, size class), with
    the nearest class of the same group standing in for a missing one."""
    lbm.lbm_tuning_clear()
    assert lbm.lbm_tuning_get_batch_tile("D3Q19", "PR", "F16", 100_000) == (256, 1, 16)
    lbm.lbm_tuning_set_batch_tile("D3Q19", "PR", "F16", 16, 128, 2)
    lbm.lbm_tuning_set_batch_tile("D3Q19", "PR", "F16", 20, 512, 1)
    assert lbm.lbm_tuning_get_batch_tile("D3Q19", "PR", "F16", 70_000) == (128, 2, 16)
    assert lbm.lbm_tuning_get_batch_tile("D3Q19", "PR", "F16", 3_000) == (128, 2, 11)   # nearest: 16
    assert lbm.lbm_tuning_get_batch_tile("D3Q19", "PR", "F16", 2_000_000) == (512, 1, 20)
    assert lbm.lbm_tuning_get_batch_tile("D3Q19", "IR", "F16", 70_000) == (256, 1, 16)  # other key
    assert lbm.lbm_tuning_get_batch_tile("D3Q27", "PR", "F16", 70_000) == (256, 1, 16)
    lib = lbm.library()
    assert lib.lbm_tuning_set_batch_tile(2, 0, 2, 16, 512, 2) == lbm.LBM_EINVAL   # 512 x 2
    assert lib.lbm_tuning_set_batch_tile(2, 0, 2, 16, 64, 1) == lbm.LBM_EINVAL
    assert lib.lbm_tuning_set_batch_tile(2, 0, 2, 16, 256, 3) == lbm.LBM_EINVAL
    assert lib.lbm_tuning_set_batch_tile(2, 0, 0, 16, 128, 1) == lbm.LBM_EINVAL   # F64: 256 x 1 only
    assert lib.lbm_tuning_set_batch_tile(2, 0, 0, 16, 256, 1) == lbm.LBM_OK
    assert lib.lbm_tuning_set_batch_tile(2, 0, 2, 63, 256, 1) == lbm.LBM_EINVAL
    assert lib.lbm_tuning_set_batch_tile(9, 0, 2, 16, 256, 1) == lbm.LBM_EINVAL
    lbm.lbm_tuning_clear()
    assert lbm.lbm_tuning_get_batch_tile("D3Q19", "PR", "F16", 70_000) == (256, 1, 16)


def test_wait_limit_host_logic():
    assert lbm.lbm_get_wait_limit() == 0.0
    lbm.lbm_set_wait_limit(2.5)
    assert lbm.lbm_get_wait_limit() == 2.5
    lib = lbm.library()
    for bad in (-1.0, float("nan"), float("inf")):
        assert lib.lbm_set_wait_limit(bad) == lbm.LBM_EINVAL
    assert lbm.lbm_get_wait_limit() == 2.5
    assert lib.lbm_get_wait_limit(None) == lbm.LBM_EINVAL
    lbm.lbm_set_wait_limit(0.0)
    assert lib.lbm_status_string(lbm.LBM_ETIMEOUT) == b"timeout"


def test_null_handle_is_rejected():
    lib = lbm.library()
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_sync(None) == lbm.LBM_EINVAL
    lib.lbm_destroy(None)   # no-op
    assert lib.lbm_status_string(lbm.LBM_ECUDA) == b"CUDA error"
