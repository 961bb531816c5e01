"""Seeded input generators: determinism and the geometric properties they promise."""
import numpy as np

from paper_1610_01388_gb300 import workloads as W


def test_channel_and_duct_masks():
    m = W.channel_mask(4, 64)
    assert m.shape == (1, 64, 4) and m[0, 0].all() and m[0, 1:].sum() == 0
    d = W.duct_mask(8, 6, 5)
    assert d.shape == (5, 6, 8)
    assert d[:, 0, :].all() and d[0, :, :].all() and d[1:, 1:, :].sum() == 0


def test_porous_generator_is_seeded_and_non_overlapping():
    m1, i1 = W.porous_mask(48, porosity=0.7, seed=3)
    m2, i2 = W.porous_mask(48, porosity=0.7, seed=3)
    m3, _ = W.porous_mask(48, porosity=0.7, seed=4)
    assert np.array_equal(m1, m2) and not np.array_equal(m1, m3)
    assert i1["reached"] and abs(i1["porosity"] - 0.7) < 0.02
    assert i1["porosity"] == 1.0 - m1.mean()


def test_bn_maps_invert_their_definitions():
    for bn in (0.1, 1.0, 10.0):
        xi = W.channel_bn_to_xi(bn)
        assert abs(6 * xi / (1 - 1.5 * xi + 0.5 * xi ** 3) - bn) < 1e-10
    for bn in (0.5, 2.0, 8.0):
        bi = W.duct_bn_to_bi(bn)
        assert abs(4 * bi / (W.C_MAX * (1 - bi / W.BI_CR) ** 2) - bn) < 1e-9
    assert abs(W.duct_bn_to_bi(0.5) - 0.11670) < 1e-4


def test_permutation_maps_velocity_orders():
    c1 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0]])
    c2 = np.array([[-1, 0, 0], [0, 0, 0], [1, 0, 0]])
    p = W.permutation(c1, c2)
    assert np.array_equal(c2[p], c1)


def test_serving_stream_is_seeded_and_in_range():
    a = W.serving_requests(n=40, rate=50.0, seed=11, duct_sides=(32, 48), porous_sides=(32, 40))
    b = W.serving_requests(n=40, rate=50.0, seed=11, duct_sides=(32, 48), porous_sides=(32, 40))
    assert [r["arrival"] for r in a] == [r["arrival"] for r in b]
    assert all(np.array_equal(x["mask"], y["mask"]) for x, y in zip(a, b))
    t = [r["arrival"] for r in a]
    assert all(t1 > t0 for t0, t1 in zip(t, t[1:]))
    for r in a:
        assert 0.1 <= r["bn"] <= 10.0 and r["model"] in ("PR", "IR")
        if r["kind"] == "channel":
            assert r["lattice"] == "D2Q9" and 17 <= r["mask"].shape[1] <= 257
        elif r["kind"] == "duct":
            assert r["lattice"] in ("D3Q19", "D3Q27") and 33 <= r["mask"].shape[1] <= 49
        else:
            assert r["lattice"] in ("D3Q19", "D3Q27") and 32 <= r["mask"].shape[0] <= 40


def test_serving_stream_pools_porous_geometry():
    reqs = W.serving_requests(n=60, rate=50.0, seed=5, porous_sides=(32, 64), porous_pool=2)
    porous = [r for r in reqs if r["kind"] == "porous"]
    assert porous
    shapes = {r["mask"].shape[0] for r in porous}
    assert all(s % 16 == 0 and 32 <= s <= 64 for s in shapes)
    # at most pool-size distinct geometries per side, each generated once
    for s in shapes:
        ids = {id(r["mask"]) for r in porous if r["mask"].shape[0] == s}
        assert 1 <= len(ids) <= 2
    # the Bingham number and model are still drawn per request
    assert len({r["bn"] for r in porous}) == len(porous)
