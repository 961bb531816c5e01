"""Parity at the full workload sizes, in the launch configuration bench.py
times (FP32, CUDA-graph replay of long step runs), on sampled cells.

The GPU state after n steps is read back (FP32 offsets -> FP64 full f); the
oracle computes one more step for a sample of cells from exactly that state
(its per-population FP64 collision); the GPU takes the same step and the two
are compared cell by cell.  Whole-domain invariants (mass) are checked too.
"""
import numpy as np
import pytest

from paper_1610_01388_gb300 import lbm
from paper_1610_01388_gb300 import workloads as W

from _pairs import gpu_to_oracle, make_pair, perm_gpu_to_oracle

pytestmark = pytest.mark.gpu


def _sample(mask, n, seed):
    rng = np.random.default_rng(seed)
    flat = mask.reshape(-1)
    fluid = np.flatnonzero(flat == 0)
    pick = rng.choice(fluid, size=min(n, fluid.size), replace=False)
    # every fluid cell of a few wall-adjacent and wrap rows as well
    nz, ny, nx = mask.shape
    extra = []
    for z, y in ((1, 1), (1, ny - 1), (nz - 1, 1), (nz // 2, ny // 2), (nz - 1, ny - 1)):
        if 0 <= z < nz and 0 <= y < ny:
            row = z * ny * nx + y * nx + np.arange(nx)
            extra.append(row[flat[row] == 0])
    return np.unique(np.concatenate([pick] + extra)).astype(np.int64)


def _sampled_step_parity(lat, mask, model, steps, **kw):
    s, o = make_pair(lat, mask, model=model, storage="F32", check_every=100, **kw)
    s.step(steps)                                  # graph replay path
    m0, _ = s.totals()
    f_state = gpu_to_oracle(lat, s.get_populations())
    o.f = np.ascontiguousarray(f_state)
    if model == "PR":
        o.tau = np.ascontiguousarray(s.get_tau().reshape(-1))
    cells = _sample(mask, 4000, seed=steps)
    want, want_tau = o.step_cells(cells)           # oracle: one step of the sampled cells
    s.step(1)
    got_all = gpu_to_oracle(lat, s.get_populations())
    got = got_all[:, cells].T
    scale = np.max(np.abs(want - o.w[None, :]))
    err = np.max(np.abs(got - want)) / scale
    assert err < 1e-5, (lat, model, err)
    if model == "PR":
        got_tau = s.get_tau().reshape(-1)[cells]
        assert np.max(np.abs(got_tau - want_tau) / want_tau) < 1e-5
    m1, _ = s.totals()
    assert abs(m1 - m0) / m0 < 1e-6
    s.close()
    return err


@pytest.mark.parametrize("lat", ["D3Q27", "D3Q19"])
@pytest.mark.parametrize("model", ["PR", "IR"])
def test_fullsize_square_duct(lat, model):
    """Square duct 256 x 128 x 128 (127 x 127 fluid), Bn = 2, from rest."""
    prm = W.duct_params(H=127, nu_p=0.1, u_newton=0.02, bn=2.0)
    mask = W.duct_mask(256, 128, 128)
    _sampled_step_parity(lat, mask, model, 300, nu_p=0.1, sigma_y=prm["sigma_y"], m=1e6,
                         g=(prm["g"], 0.0, 0.0))


@pytest.mark.parametrize("model", ["PR", "IR"])
@pytest.mark.parametrize("block", [128, 256])
def test_fullsize_square_duct_two_cells_per_thread(model, block):
    """The bench duct (D3Q27, 256 x 128 x 128) with plain steps at two cells
    per thread, a launch shape the autotuner may pick for the bench."""
    prm = W.duct_params(H=127, nu_p=0.1, u_newton=0.02, bn=2.0)
    mask = W.duct_mask(256, 128, 128)
    lbm.lbm_tuning_clear()
    try:
        _, _, cls = lbm.lbm_tuning_get_shape("D3Q27", model, "F32", mask.size)
        lbm.lbm_tuning_set_shape("D3Q27", model, "F32", cls, block, 2)
        _sampled_step_parity("D3Q27", mask, model, 300, nu_p=0.1, sigma_y=prm["sigma_y"], m=1e6,
                             g=(prm["g"], 0.0, 0.0))
    finally:
        lbm.lbm_tuning_clear()


@pytest.mark.parametrize("model", ["PR", "IR"])
def test_fullsize_porous_d3q19(model):
    """Porous box 256^3, random non-overlapping spheres r in [6, 10], porosity
    0.7, seed 1, body-force driven."""
    mask, info = W.porous_mask(256, porosity=0.7, r_min=6, r_max=10, seed=1)
    assert info["reached"]
    _sampled_step_parity("D3Q19", mask, model, 200, nu_p=0.1, sigma_y=2e-6, m=1e6,
                         g=(2e-6, 0.0, 0.0))


@pytest.mark.parametrize("model,block", [("PR", 128), ("IR", 256)])
def test_fullsize_duct_whole_field_equal_steps(model, block):
    """The bench duct itself (D3Q27, 256 x 128 x 128, 127 x 127 fluid, FP32,
    Bn = 2, m = 1e6, check step every 100, the block size the bench's tuner
    picks for the model, CUDA-graph replay), 200 steps from rest on the GPU
    and in the FP64 oracle: relative L2 of u_real over the whole field within
    1e-5, and the flow rate within 1e-5."""
    from _pairs import rel_l2_u
    prm = W.duct_params(H=127, nu_p=0.1, u_newton=0.02, bn=2.0)
    mask = W.duct_mask(256, 128, 128)
    lbm.lbm_tuning_clear()
    try:
        _, _, cls = lbm.lbm_tuning_get_shape("D3Q27", model, "F32", mask.size)
        lbm.lbm_tuning_set_shape("D3Q27", model, "F32", cls, block, 1)
        s, o = make_pair("D3Q27", mask, model=model, storage="F32", check_every=100, nu_p=0.1,
                         sigma_y=prm["sigma_y"], m=1e6, g=(prm["g"], 0.0, 0.0))
        s.step(200)
        o.step(200)
        err = rel_l2_u(s, o)
        print(f"duct 256x128x128 D3Q27 {model} F32, 200 steps: rel L2 u {err:.3e}")
        assert err <= 1e-5
        qo = o.flowrate(0)
        assert abs(s.flowrate(0) - qo) <= 1e-5 * abs(qo)
        s.close()
    finally:
        lbm.lbm_tuning_clear()


@pytest.mark.parametrize("model", ["PR", "IR"])
def test_fullsize_fp16_duct_whole_field_equal_steps(model):
    """FP16 offset storage on the precision workload's duct cross-section
    (D3Q27, 191 x 191 fluid, periodic along x, here 16 cells long so the FP64
    oracle runs it in about a minute), Bn = 2, 1500 steps from rest on both
    sides: relative L2 of u_real over the whole field within 1e-3."""
    from _pairs import rel_l2_u
    prm = W.duct_params(H=191, nu_p=0.1, u_newton=0.02, bn=2.0)
    mask = W.duct_mask(16, 192, 192)
    s, o = make_pair("D3Q27", mask, model=model, storage="F16", check_every=100, nu_p=0.1,
                     sigma_y=prm["sigma_y"], m=1e6, g=(prm["g"], 0.0, 0.0))
    s.step(1500)
    o.step(1500)
    err = rel_l2_u(s, o)
    print(f"duct 16x192x192 D3Q27 {model} F16, 1500 steps: rel L2 u {err:.3e}")
    assert err <= 1e-3
    s.close()


def test_fullsize_channel_fp64_20k_steps():
    """Channel 4 x 64, D2Q9, FP64, 20k steps from rest, both models: the whole
    field against the oracle at equal step count."""
    from _pairs import rel_l2_u
    prm = W.channel_params(H=63, nu_p=0.1, u_newton=0.01, bn=1.0)
    for model in ("PR", "IR"):
        s, o = make_pair("D2Q9", W.channel_mask(4, 64), model=model, storage="F64",
                         sigma_y=prm["sigma_y"], m=1e4, g=(prm["g"], 0, 0))
        s.step(20000)
        o.step(20000)
        assert rel_l2_u(s, o) < 1e-11
        s.close()


def _ulp16(x, storage):
    """Spacing of the 16-bit format at |x| (FP16: 10 fraction bits, normal
    from 2^-14; BF16: 7 fraction bits)."""
    frac, emin = (10, -14) if storage == "F16" else (7, -126)
    e = np.floor(np.log2(np.maximum(np.abs(x), 2.0 ** emin)))
    return 2.0 ** (e - frac)


def _units(f, w, storage):
    """Populations in the stored unit: 2^14 (f - w) / w for FP16, (f - w) / w
    for BF16 (the forms the storage documents)."""
    return (f - w[:, None]) / w[:, None] * (16384.0 if storage == "F16" else 1.0)


def _reduced_precision_sampled_step(lat, mask, model, storage, steps, nsample, **kw):
    """One step of sampled cells at full size for 16-bit storage.  The GPU
    state after `steps` steps is probed cell by cell (lbm_get_populations_cells);
    the test streams it itself (pulled_inputs: eq. 8 with halfway bounce-back)
    and the oracle's FP64 single-cell collision gives the post-collision
    values.  The GPU's next stored values must be within one 16-bit spacing of
    them (the stochastic rounding picks one of the two neighbours of its FP32
    result), plus FP32 round-off."""
    import oracle
    from _pairs import oracle_collide_cells, pulled_inputs
    # no full oracle state: at 512^3 its FP64 populations alone are 29 GB
    s = lbm.Solver(lat, mask, model=model, storage=storage, mu_p=kw["nu_p"], sigma_y=kw["sigma_y"],
                   m=kw["m"], g=kw["g"], check_every=100)
    p = oracle.params(model=model, nu_p=kw["nu_p"], sigma_y=kw["sigma_y"], m=kw["m"], g=kw["g"])
    s.step(steps)
    c, w = lbm.lbm_lattice_info(lat)
    cells = _sample(mask, nsample, seed=steps)
    fin = pulled_inputs(c, mask, cells, lambda idx: lbm.lbm_get_populations_cells(s.h, idx, len(w)))
    tau_old = s.get_tau().reshape(-1)[cells] if model == "PR" else np.zeros(cells.size)
    want, want_tau = oracle_collide_cells(lat, p, fin, tau_old)
    s.step(1)
    got = lbm.lbm_get_populations_cells(s.h, cells, len(w))
    xw, xg = _units(want, w, storage), _units(got, w, storage)
    tol = _ulp16(np.maximum(np.abs(xw), np.abs(xg)), storage) + 1e-5 * np.max(np.abs(xw), axis=0)
    assert np.all(np.abs(xg - xw) <= tol), (lat, model, storage, np.max(np.abs(xg - xw) / tol))
    if model == "PR":
        got_tau = s.get_tau().reshape(-1)[cells]
        assert np.max(np.abs(got_tau - want_tau) / want_tau) < 1e-5
    s.close()


@pytest.mark.parametrize("storage", ["F16", "BF16"])
@pytest.mark.parametrize("model", ["PR", "IR"])
def test_fullsize_precision_duct_d3q27(storage, model):
    """Precision workload: square duct 512 x 192 x 192 (191 x 191 fluid), D3Q27,
    16-bit offset storage, Bn = 2, from rest."""
    prm = W.duct_params(H=191, nu_p=0.1, u_newton=0.02, bn=2.0)
    mask = W.duct_mask(512, 192, 192)
    _reduced_precision_sampled_step("D3Q27", mask, model, storage, 300, 3000, nu_p=0.1,
                                    sigma_y=prm["sigma_y"], m=1e6, g=(prm["g"], 0.0, 0.0))


_POROUS512 = {}


def _porous512():
    """Precision workload's porous box: 512^3, spheres r in [6, 10], target
    porosity 0.6, seed 1.  Random sequential addition jams above 0.6; the
    packing stops at 2e6 candidates (porosity ~0.67, asserted below 0.7)."""
    if "m" not in _POROUS512:
        mask, info = W.porous_mask(512, porosity=0.6, r_min=6, r_max=10, seed=1,
                                   max_attempts=2_000_000)
        assert 0.6 <= info["porosity"] < 0.7
        _POROUS512["m"] = mask
    return _POROUS512["m"]


@pytest.mark.parametrize("storage", ["F16", "BF16"])
@pytest.mark.parametrize("model", ["PR", "IR"])
def test_fullsize_precision_porous512_d3q27(storage, model):
    """Precision workload: 512^3 porous box, D3Q27, 16-bit offset storage,
    body-force driven from rest."""
    _reduced_precision_sampled_step("D3Q27", _porous512(), model, storage, 200, 3000, nu_p=0.1,
                                    sigma_y=2e-6, m=1e6, g=(2e-6, 0.0, 0.0))
