"""The sector-level traffic count, on geometries whose counts are known by
hand."""
import numpy as np
import pytest

from paper_1610_01388_gb300 import lbm, traffic, workloads as W


def _q(lat):
    return len(lbm.lbm_lattice_info(lat)[1])


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
def test_all_fluid_box_moves_every_sector_once(lat):
    shape = (16, 8) if lat == "D2Q9" else (4, 6, 16)
    m = np.zeros(shape, np.uint8)
    n, q = m.size, _q(lat)
    r = traffic.sector_traffic(m, lat)
    assert r["fills"] == 0
    assert r["reads"] == r["writes"] == q * n * 4
    assert r["links"] == 4 * n and r["algorithmic"] == n * (8 * q + 1)


def test_duct_rows_are_whole_so_no_fills():
    m = W.duct_mask(32, 9, 7)
    r = traffic.sector_traffic(m, "D3Q27", copy_through=False)
    fluid_rows = int((m[:, :, 0] == 0).sum())
    assert r["fills"] == 0
    assert r["writes"] == 27 * fluid_rows * 32 * 4
    # the bounce-back reads fall in the cell's own sectors, already counted
    assert r["reads"] == r["writes"]


@pytest.mark.parametrize("fp64", [False, True])
def test_one_solid_cell_costs_one_fill_per_plane(fp64):
    m = np.zeros((2, 2, 32), np.uint8)
    m[1, 1, 3] = 1
    vb = 8 if fp64 else 4
    per = 32 // vb
    r = traffic.sector_traffic(m, "D3Q19", value_bytes=vb, copy_through=False)
    assert r["fills"] == 19 * 32
    assert r["writes"] == 19 * (m.size // per) * 32
    # with the copy-through the solid cell writes its own value back
    rc = traffic.sector_traffic(m, "D3Q19", value_bytes=vb, copy_through=True)
    assert rc["fills"] == 0 and rc["writes"] == r["writes"]


def test_copy_through_moves_only_groups_with_fluid():
    """One fluid cell in a row of 32 solid ones: its group of 8 cells is one
    sector per plane, copied through whole; the other three groups of the
    warp are not touched.  Counting by warps of 32 would move all four."""
    m = np.ones((3, 3, 32), np.uint8)
    m[1, 1, 11] = 0
    r = traffic.sector_traffic(m, "D3Q19")
    assert r["fills"] == 0 and r["writes"] == 19 * 32
    rw = traffic.sector_traffic(m, "D3Q19", group=32)
    assert rw["fills"] == 0 and rw["writes"] == 4 * 19 * 32


def test_copy_through_leaves_no_partial_sector_and_skips_solid_warps():
    m, _ = W.porous_mask(32, porosity=0.7, r_min=3.0, r_max=5.0, seed=4)
    r0 = traffic.sector_traffic(m, "D3Q19", copy_through=False)
    r1 = traffic.sector_traffic(m, "D3Q19", copy_through=True)
    assert r0["fills"] > 0 and r1["fills"] == 0
    # copy lanes add their own sectors: never fewer reads or writes
    assert r1["reads"] >= r0["reads"] and r1["writes"] >= r0["writes"]
    # a warp of solid cells only moves nothing but its link words
    solid_box = np.ones((2, 2, 64), np.uint8)
    rs = traffic.sector_traffic(solid_box, "D3Q19")
    assert rs["reads"] == rs["writes"] == rs["fills"] == 0 and rs["links"] == 4 * 256
