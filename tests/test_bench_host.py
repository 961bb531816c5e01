"""bench.py's host-side workload selection, run on CPU: the duct and the
porous box, the oracle's sample slab, and when a recorded traffic figure
may be reported."""
import numpy as np

import bench
from paper_1610_01388_gb300 import workloads as W


def test_duct_workload_is_the_default(monkeypatch):
    monkeypatch.setattr(bench, "POROUS", 0)
    monkeypatch.setattr(bench, "NX", 16)
    monkeypatch.setattr(bench, "NY", 8)
    monkeypatch.setattr(bench, "NZ", 6)
    m = bench.workload_mask()
    assert np.array_equal(m, W.duct_mask(16, 8, 6))
    assert np.array_equal(bench.workload_mask(4), W.duct_mask(4, 8, 6))
    cfg = bench.workload_config()
    assert cfg["workload"].startswith("square duct") and "smaller than L2" in cfg["l2"]


def test_porous_workload_and_its_sample_slab(monkeypatch):
    monkeypatch.setattr(bench, "POROUS", 32)
    monkeypatch.setattr(bench, "NX", 32)
    monkeypatch.setattr(bench, "NY", 32)
    monkeypatch.setattr(bench, "NZ", 32)
    m = bench.workload_mask()
    want, info = W.porous_mask(32, porosity=0.7, r_min=6.0, r_max=10.0, seed=1)
    assert np.array_equal(m, want) and m.shape == (32, 32, 32)
    slab = bench.workload_mask(4)
    assert slab.shape == (32, 32, 4) and slab.flags["C_CONTIGUOUS"]
    assert np.array_equal(slab, want[:, :, :4])
    cfg = bench.workload_config()
    assert cfg["workload"].startswith("porous box") and cfg["nx"] == 32
    g, sy = bench.workload_params()
    p = W.porous_params(nu_p=bench.NU_P, d_mean=16.0, g=2e-5, bn=bench.BN)
    assert (g, sy) == (p["g"], p["sigma_y"])


def test_recorded_traffic_only_for_the_captured_workload(monkeypatch):
    monkeypatch.setattr(bench, "POROUS", 0)
    monkeypatch.setattr(bench, "LATTICE", "D3Q27")
    monkeypatch.setattr(bench, "NX", 256)
    monkeypatch.setattr(bench, "NY", 128)
    monkeypatch.setattr(bench, "NZ", 128)
    key = ("F32", "PR", 256, 1)
    monkeypatch.setattr(bench, "KERNEL_FINGERPRINT", bench.kernel_fingerprint())
    assert bench.ncu_traffic(*key) == bench.NCU_TRAFFIC[key]
    assert bench.ncu_traffic(*key, override=123) == 123
    # another workload, or device code changed since the capture: no figure
    monkeypatch.setattr(bench, "POROUS", 160)
    assert bench.ncu_traffic(*key) is None
    monkeypatch.setattr(bench, "POROUS", 0)
    monkeypatch.setattr(bench, "KERNEL_FINGERPRINT", "0" * 16)
    assert bench.ncu_traffic(*key) is None


def test_mixed_storage_routes_near_jammed_porous_requests_to_fp32():
    reqs = W.serving_requests(n=60, rate=1e9, seed=7, storage="F16", channel_widths=(16, 20),
                              duct_sides=(16, 18), duct_length=8, porous_sides=(24, 24),
                              porous_radius=(3.0, 4.0))
    got = [bench._route("mixed", r) for r in reqs]
    for r, st in zip(reqs, got):
        want = "F32" if (r["kind"] == "porous" and r["bn"] >= 1.0) else "F16"
        assert st == want
    assert "F32" in got and "F16" in got
    assert bench._route("mixed", None) == "F16"
    assert bench._route("F32", reqs[0]) == "F32"


def test_gpus_must_match_world_size(monkeypatch, capsys):
    import pytest
    monkeypatch.setenv("WORLD_SIZE", "2")
    with pytest.raises(SystemExit) as e:
        bench.main(["--gpus", "4"])
    assert e.value.code == 2
    assert "WORLD_SIZE=2" in capsys.readouterr().err
