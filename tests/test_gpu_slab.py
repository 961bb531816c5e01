"""One domain split into z-slabs on the GPU (paper_1610_01388_gb300.slab):
two or three slabs in one process, their face populations exchanged through
lbm_halo_pack / lbm_halo_unpack before every step.  A step reads only the
nearest neighbours (eq. 8), so the slabs' populations must equal the
undivided solver's bit for bit (same per-cell arithmetic; the 16-bit form
draws the same stochastic-rounding bits through the hash offset), and the
flow rate and residual combined from the slabs must equal the undivided
ones to round-off of their summation order."""
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
    assert abs(dom.residual() - r_ref) <= 1e-10 * r_ref
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
