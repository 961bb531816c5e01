"""The allocation-free flow-rate entry point, lbm_flowrate_noalloc.

It serves callers that must not allocate device memory at query time (a
serving loop that has handed its whole memory budget out up front, a caller
with its own device-memory pool, a latency-critical loop where cudaMalloc's
possible device synchronisation is not acceptable).  It reuses the flow-rate
reduction kernel with its block partials in a static device array of the
library.  This file is collected last so that a failure here cannot stop the
other tests of a -x run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1610_01388_gb300 import lbm
from paper_1610_01388_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _solver(lat, mask, model, storage="F32", layout="dense"):
    g = (2e-5, -4e-6, 0.0 if lat == "D2Q9" else 3e-6)
    return lbm.Solver(lat, mask, model=model, storage=storage, mu_p=0.08, sigma_y=1e-5, m=1e5,
                      g=g, layout=layout)


# The reduction runs at most 1216 blocks of 256 cells and strides over the
# rest, so domains above 311,296 cells (the bench duct, the porous box) take
# the grid-stride loop and fill every partial of the static array.
# (compact layout: the reduction strides over the fluid slots; 96^3 holds
# 875,520 of them)
@pytest.mark.parametrize("lat,shape,model,storage,layout", [
    ("D3Q19", (13, 17, 40), "IR", "F32", "dense"),
    ("D3Q27", (9, 11, 300), "PR", "F32", "dense"),
    ("D2Q9", (1, 64, 4), "IR", "F32", "dense"),
    ("D3Q27", (128, 128, 256), "PR", "F32", "dense"),
    ("D3Q19", (96, 96, 96), "IR", "F16", "dense"),
    ("D3Q19", (96, 96, 96), "PR", "F32", "compact"),
])
def test_noalloc_flowrate_matches_flowrate_on_two_calls(lat, shape, model, storage, layout):
    import torch
    mask = np.zeros(shape, np.uint8)
    mask[:, 0, :] = 1
    if shape[0] > 1:
        mask[0, :, :] = 1
    s = _solver(lat, mask, model, storage, layout)
    q_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call, steps in enumerate((37, 64)):
        s.step(steps)
        want = [s.flowrate(a) for a in range(3)]          # existing entry point (syncs)
        for a in range(3):
            lbm.lbm_flowrate_noalloc(s.h, a, q_dev.data_ptr() + 8 * a)
        s.sync()
        stream.synchronize()
        got = q_dev.cpu().numpy()[:3]
        for a in range(3):
            assert abs(got[a] - want[a]) <= 1e-12 * max(abs(want[a]), 1e-30), (call, a, got, want)
        assert abs(want[0]) > 0
    s.close()


def test_noalloc_rejects_bad_arguments():
    import torch
    mask = W.duct_mask(8, 6, 6)
    s = _solver("D3Q19", mask, "IR")
    lib = lbm.library()
    q_dev = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert lib.lbm_flowrate_noalloc(s.h, 3, ctypes.c_void_p(q_dev.data_ptr())) == lbm.LBM_EINVAL
    assert lib.lbm_flowrate_noalloc(s.h, 0, None) == lbm.LBM_EINVAL
    assert lib.lbm_flowrate_noalloc(s.h, 0, ctypes.c_void_p(q_dev.data_ptr() + 4)) == lbm.LBM_EINVAL
    assert lib.lbm_flowrate_noalloc(None, 0, ctypes.c_void_p(q_dev.data_ptr())) == lbm.LBM_EINVAL
    s.close()
