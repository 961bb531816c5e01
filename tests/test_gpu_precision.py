"""Reduced-precision storage (FP16 / BF16 offsets, FP32 arithmetic,
stochastic rounding on store) against the FP64 oracle.

The reduced-precision form is FP16: relative L2 velocity error <= 1e-3 at
equal step count on the precision-form geometries (square duct and porous
box, D3Q27) at sizes the oracle runs in seconds (test_*_velocity_error).
BF16 keeps 8 significant bits (8x coarser than FP16) and lands at
1.4-1.7e-3 on these flows: it does NOT meet the 1e-3 bar and is offered only
as a storage option that fails it.  Its own tests (test_bf16_*_error_level)
hold it at its measured level, <= 2.5e-3, so that a regression still fails;
they are not the bar.  Single collisions agree with the oracle up to the
storage quantum of the outputs.
"""
import numpy as np
import pytest

import oracle
from paper_1610_01388_gb300 import lbm
from paper_1610_01388_gb300 import workloads as W

from _pairs import gpu_to_oracle, make_pair, oracle_to_gpu, rel_l2_u, set_both

pytestmark = pytest.mark.gpu

# relative rounding bound of (f - w) / w: round-to-nearest on upload (set
# populations), stochastic rounding (up to one ulp) on every kernel store
QUANTUM = {"F16": 2.0 ** -11, "BF16": 2.0 ** -8}
QUANTUM_SR = {"F16": 2.0 ** -10, "BF16": 2.0 ** -7}


@pytest.mark.parametrize("storage", ["F16", "BF16"])
@pytest.mark.parametrize("model", ["PR", "IR"])
@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
def test_single_cell_quantised(lat, model, storage):
    mask = np.zeros((1, 1, 1), np.uint8)
    g = (3e-5, -1e-5, 0.0 if lat == "D2Q9" else 2e-5)
    s, o = make_pair(lat, mask, model=model, storage=storage, nu_p=0.05, sigma_y=2e-4, m=1e4, g=g)
    f0 = W.random_populations(o.w, 1, amplitude=0.05, seed=11)
    s.set_populations(oracle_to_gpu(lat, f0))
    fq = gpu_to_oracle(lat, s.get_populations())       # the stored (quantised) state
    rel_in = np.max(np.abs((fq - f0) / o.w[:, None]))
    assert rel_in <= QUANTUM[storage] * 0.05 * 1.01 + 1e-12   # |(f-w)/w| <= 0.05 here
    o.f = np.ascontiguousarray(fq)
    if model == "PR":
        tau0 = np.array([0.5 + 3 * (0.05 + 1e4 * 2e-4)])
        s.set_tau(tau0)
        o.tau = tau0.copy()
    s.step(1)
    o.step(1)
    got = gpu_to_oracle(lat, s.get_populations())
    off = np.abs((o.f - o.w[:, None]) / o.w[:, None])
    err = np.abs((got - o.f) / o.w[:, None])
    assert np.all(err <= QUANTUM_SR[storage] * off + 2e-6), np.max(err - QUANTUM_SR[storage] * off)


def _duct_case(storage, model, steps=2000):
    mask = W.duct_mask(16, 25, 25)
    s, o = make_pair("D3Q27", mask, model=model, storage=storage, nu_p=0.05, sigma_y=4e-6,
                     m=1e6, g=(2e-5, 0.0, 0.0))
    s.step(steps)
    o.step(steps)
    err = rel_l2_u(s, o)
    s.close()
    return err


def _porous_case(storage, model, steps=600):
    mask, info = W.porous_mask(40, porosity=0.6, r_min=4, r_max=6, seed=5)
    s, o = make_pair("D3Q27", mask, model=model, storage=storage, nu_p=0.05, sigma_y=2e-6,
                     m=1e6, g=(5e-5, 0.0, 0.0), nthreads=0)
    s.step(steps)
    o.step(steps)
    err = rel_l2_u(s, o)
    s.close()
    return err


BAR = 1e-3                 # the reduced-precision bar (FP16)
BF16_LEVEL = 2.5e-3        # BF16's measured level, held against regressions; fails BAR


def _two_cells(storage, model):
    mask_cells = 16 * 25 * 25
    lbm.lbm_tuning_clear()
    try:
        _, _, cls = lbm.lbm_tuning_get_shape("D3Q27", model, storage, mask_cells)
        lbm.lbm_tuning_set_shape("D3Q27", model, storage, cls, 128, 2)
        return _duct_case(storage, model)
    finally:
        lbm.lbm_tuning_clear()


@pytest.mark.parametrize("model", ["PR", "IR"])
def test_duct_velocity_error(model):
    err = _duct_case("F16", model)
    print(f"duct D3Q27 {model} F16: rel L2 u error {err:.3e}")
    assert err <= BAR


@pytest.mark.parametrize("model", ["PR", "IR"])
def test_porous_velocity_error(model):
    err = _porous_case("F16", model)
    print(f"porous D3Q27 {model} F16: rel L2 u error {err:.3e}")
    assert err <= BAR


@pytest.mark.parametrize("model", ["PR", "IR"])
def test_duct_velocity_error_two_cells_per_thread(model):
    """The same bar with plain steps at two cells per thread (packed FP32
    collision of both cells)."""
    err = _two_cells("F16", model)
    print(f"duct D3Q27 {model} F16 2 cells/thread: rel L2 u error {err:.3e}")
    assert err <= BAR


@pytest.mark.parametrize("case", ["duct", "porous", "duct_two_cells"])
@pytest.mark.parametrize("model", ["PR", "IR"])
def test_bf16_velocity_error_level(case, model):
    """BF16 does not meet the 1e-3 bar; this holds it at its measured level."""
    err = {"duct": lambda: _duct_case("BF16", model), "porous": lambda: _porous_case("BF16", model),
           "duct_two_cells": lambda: _two_cells("BF16", model)}[case]()
    print(f"{case} D3Q27 {model} BF16: rel L2 u error {err:.3e} (bar 1e-3 not met)")
    assert err <= BF16_LEVEL
