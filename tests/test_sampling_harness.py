"""Host check of the sampled-step harness the full-size GPU tests use: the
test-side pull streaming (pulled_inputs) followed by the oracle's single-cell
collision reproduces the oracle's own full step for the sampled cells, for
both models, on a duct with walls and a porous box (periodic wrap, solid
neighbours, corners)."""
import numpy as np
import pytest

import oracle
from paper_1610_01388_gb300 import lbm
from paper_1610_01388_gb300 import workloads as W

from _pairs import oracle_collide_cells, perm_gpu_to_oracle, pulled_inputs


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("model", ["PR", "IR"])
def test_pulled_inputs_and_single_cell_collision_equal_a_full_step(lat, model):
    if lat == "D2Q9":
        mask = W.channel_mask(5, 12)
    elif lat == "D3Q19":
        mask, _ = W.porous_mask(12, porosity=0.7, r_min=2, r_max=3, seed=4)
    else:
        mask = W.duct_mask(6, 7, 5)
    p = oracle.params(model=model, nu_p=0.08, sigma_y=2e-5, m=1e5, g=(2e-5, 1e-6, 0.0))
    o = oracle.State(lat, p, mask)
    o.f = np.ascontiguousarray(W.random_populations(o.w, o.N, amplitude=0.02, seed=9))
    o.tau = 0.6 + np.random.default_rng(3).random(o.N)
    c, _ = lbm.lbm_lattice_info(lat)
    po = perm_gpu_to_oracle(lat)
    cells = np.flatnonzero(mask.reshape(-1) == 0)
    fin = pulled_inputs(c, mask, cells, lambda idx: o.f[po][:, idx])
    got, got_tau = oracle_collide_cells(lat, p, fin, o.tau[cells])
    want, want_tau = o.step_cells(cells)          # oracle order, (n, Q)
    assert np.array_equal(got.T, want[:, po])
    if model == "PR":
        assert np.array_equal(got_tau, want_tau)
