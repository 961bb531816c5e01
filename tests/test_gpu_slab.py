"""One domain split into z-slabs on the GPU (paper_1610_01388_gb300.slab):
two or three slabs in one process, their face populations exchanged through
lbm_halo_pack / lbm_halo_unpack before every step.  A step reads only the
nearest neighbours (eq. 8), so the slabs' populations must equal the
undivided solver's bit for bit (same per-cell arithmetic; the 16-bit form
draws the same stochastic-rounding bits through the hash offset), and the
flow rate and residual combined from the slabs must equal the undivided
ones to round-off of their summation order (the check step's warp and block
sums run in the arithmetic type, FP32 for the FP32 and 16-bit forms)."""
import numpy as np
import pytest

from paper_1610_01388_gb300 import lbm, slab
from paper_1610_01388_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lat,model,storage,nslabs", [
    ("D3Q19", "PR", "F64", 2), ("D3Q27", "IR", "F32", 3), ("D3Q19", "PR", "F16", 2),
    ("D3Q15", "PR", "F32", 2), ("D3Q27", "PR", "BF16", 3),
])
def test_slabs_match_undivided_domain(lat, model, storage, nslabs):
    mask, _ = W.porous_mask(32, porosity=0.7, r_min=3.0, r_max=5.0, seed=8)
    prm = dict(model=model, storage=storage, mu_p=0.1, sigma_y=2e-6, m=1e6,
               g=(2e-5, 2e-6, -3e-6), check_every=50)
    dom = slab.gpu_slab_domain(lat, mask, nslabs, **prm)
    ref = lbm.Solver(lat, mask, use_torch=True, **prm)
    n = 130                                   # two check steps, then 30 more steps
    dom.step(n)
    ref.step(n)
    f_ref = ref.get_populations()
    for (z0, nl, _), s in zip(slab.split_z(mask, nslabs), dom.ring.slabs):
        assert np.array_equal(s.populations(), f_ref[:, z0:z0 + nl]), (z0, nl)
    for a in range(3):
        q = ref.flowrate(a)
        assert abs(dom.flowrate(a) - q) <= 1e-12 * abs(q) + 1e-18, a
    r_ref, at, _ = ref.residual()
    assert at == 100
    # FP32 warp and block sums in the check step, grouped by slab (FP64 for F64)
    assert abs(dom.residual() - r_ref) <= (1e-12 if storage == "F64" else 1e-6) * r_ref
    _, u = dom.fields()
    _, u_ref = ref.fields()
    assert np.array_equal(u, u_ref)
    for s in dom.ring.slabs:
        s.close()
    ref.close()


def test_halo_calls_reject_solvers_without_ghosts():
    import torch
    s = lbm.Solver("D3Q19", W.duct_mask(8, 6, 6), use_torch=True)
    lib = lbm.library()
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    assert lib.lbm_halo_pack(s.h, 1, buf.data_ptr()) == lbm.LBM_EINVAL
    s.close()
    g = lbm.Solver("D3Q19", W.duct_mask(8, 6, 6), flags=lbm.LBM_FLAG_Z_GHOSTS, use_torch=True)
    assert lib.lbm_halo_pack(g.h, 2, buf.data_ptr()) == lbm.LBM_EINVAL
    assert lib.lbm_halo_unpack(g.h, 0, None) == lbm.LBM_EINVAL
    assert lbm.lbm_halo_bytes(g.h) == 5 * 8 * 6 * 4        # D3Q19: 5 crossing populations, FP32
    g.close()


@pytest.mark.parametrize("nslabs", [6, 3])
def test_thin_slabs(nslabs):
    """Slabs one and two planes deep (no inner planes; both planes next to a
    face) still match the undivided domain bit for bit, with check steps."""
    mask, _ = W.porous_mask((24, 20, 6), porosity=0.7, r_min=2.0, r_max=3.0, seed=4)   # nx, ny, nz
    prm = dict(model="IR", storage="F32", mu_p=0.1, sigma_y=2e-6, g=(2e-5, 1e-6, 3e-6),
               check_every=7)
    dom = slab.gpu_slab_domain("D3Q27", mask, nslabs, **prm)
    ref = lbm.Solver("D3Q27", mask, use_torch=True, **prm)
    dom.step(30)
    ref.step(30)
    f_ref = ref.get_populations()
    for (z0, nl, _), s in zip(slab.split_z(mask, nslabs), dom.ring.slabs):
        assert np.array_equal(s.populations(), f_ref[:, z0:z0 + nl])
    # the check step sums warps and blocks in FP32 (FP64 per-block partials):
    # other slab boundaries group those sums differently
    assert abs(dom.residual() - ref.residual()[0]) <= 1e-6 * ref.residual()[0]
    for s in dom.ring.slabs:
        s.close()
    ref.close()


@pytest.mark.parametrize("storage,model,newton", [("F32", "PR", 0), ("F16", "PR", 0),
                                                  ("F64", "IR", 0), ("BF16", "IR", 0),
                                                  ("F64", "PR", 3)])
def test_step_in_parts_equals_whole_step(storage, model, newton):
    """A plain step taken as three cell ranges (cut anywhere, not at warp or
    plane boundaries) plus the commit equals lbm_step(1) bit for bit, the
    16-bit forms' stochastic rounding included; check steps are refused."""
    mask, _ = W.porous_mask(24, porosity=0.7, r_min=3.0, r_max=4.0, seed=5)
    prm = dict(model=model, storage=storage, mu_p=0.1, sigma_y=2e-6, m=1e6, g=(2e-5, 0.0, 0.0),
               check_every=10, newton_iters=newton)
    a = lbm.Solver("D3Q19", mask, use_torch=True, **prm)
    b = lbm.Solver("D3Q19", mask, use_torch=True, **prm)
    n = mask.size
    cuts = [0, 1237, 8191, n]
    for step in range(1, 26):
        a.step(1)
        if step % 10 == 0:
            with pytest.raises(lbm.LbmError):
                lbm.lbm_step_cells(b.h, 0, n)
            with pytest.raises(lbm.LbmError):
                lbm.lbm_step_commit(b.h)
            b.step(1)
        else:
            for c0, c1 in zip(cuts[:-1], cuts[1:]):
                lbm.lbm_step_cells(b.h, c0, c1)
            lbm.lbm_step_commit(b.h)
    assert np.array_equal(a.get_populations(), b.get_populations())
    if model == "PR":
        assert np.array_equal(a.get_tau(), b.get_tau())
    assert a.residual() == b.residual()
    lib = lbm.library()
    assert lib.lbm_step_cells(b.h, -1, 5) == lbm.LBM_EINVAL
    assert lib.lbm_step_cells(b.h, 10, 5) == lbm.LBM_EINVAL
    assert lib.lbm_step_cells(b.h, 0, n + 1) == lbm.LBM_EINVAL
    a.close()
    b.close()


def test_rank_ring_on_one_nccl_rank():
    """The rank form of the decomposition on this GPU as a one-rank NCCL
    group: the slab's faces come back to itself (periodic), its sums go
    through an NCCL allreduce of device tensors, and it must equal the
    undivided solver bit for bit."""
    import os
    import socket
    import torch
    import torch.distributed as dist
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        mask, _ = W.porous_mask(24, porosity=0.7, r_min=3.0, r_max=4.0, seed=9)
        prm = dict(model="PR", storage="F32", mu_p=0.1, sigma_y=2e-6, m=1e6, g=(2e-5, 0.0, 0.0),
                   check_every=20)
        dom = slab.gpu_rank_slab("D3Q19", mask, **prm)
        ref = lbm.Solver("D3Q19", mask, use_torch=True, **prm)
        dom.step(50)
        ref.step(50)
        s = dom.ring.slabs[0]
        assert np.array_equal(s.populations(), ref.get_populations())
        assert abs(dom.flowrate(0) - ref.flowrate(0)) <= 1e-12 * abs(ref.flowrate(0))
        assert abs(dom.residual() - ref.residual()[0]) <= 1e-6 * ref.residual()[0]
        s.close()
        ref.close()
    finally:
        dist.destroy_process_group()
