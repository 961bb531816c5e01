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


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
def test_compact_all_fluid_box_adds_only_the_maps(lat):
    """No solid cell: slots are cells, so the compact layout moves what the
    dense one does, plus the slot map (4 bytes per cell; its link words
    replace the dense ones) and the rank words (4 per cell)."""
    shape = (16, 8) if lat == "D2Q9" else (4, 6, 16)
    m = np.zeros(shape, np.uint8)
    n, q = m.size, _q(lat)
    d = traffic.sector_traffic(m, lat)
    c = traffic.compact_traffic(m, lat)
    assert c["reads"] == c["writes"] == q * n * 4
    assert c["maps"] == 12 * n
    assert c["total"] == d["total"] + 8 * n
    # whole 64-byte pairs are read in full: no change
    assert traffic.compact_traffic(m, lat, read_bytes=64)["total"] == c["total"]


def test_compact_single_fluid_cell_reads_only_its_own_slot():
    """One fluid cell among solid ones: every population but the rest one
    bounces back, so each plane is read and written at the cell's own slot
    (one sector each), and no rank word is read."""
    m = np.ones((3, 3, 32), np.uint8)
    m[1, 1, 11] = 0
    c = traffic.compact_traffic(m, "D3Q19")
    assert c["reads"] == c["writes"] == 19 * 32
    assert c["maps"] == 2 * 32
    assert c["algorithmic"] == 2 * 19 * 4 + 1


def test_compact_moves_fewer_bytes_than_dense_on_a_porous_box():
    """Porosity 0.7: the dense layout moves the solid cells that share an
    access with fluid ones, the compact one only its maps on top of the
    fluid cells' bytes; 64-byte reads widen the gap."""
    m, _ = W.porous_mask(32, porosity=0.7, r_min=3.0, r_max=5.0, seed=4)
    for rb in (32, 64):
        d = traffic.sector_traffic(m, "D3Q19", read_bytes=rb)
        c = traffic.compact_traffic(m, "D3Q19", read_bytes=rb)
        assert c["ratio"] < d["ratio"]
        assert c["reads"] <= d["reads"] and c["writes"] < d["writes"]
    assert (traffic.sector_traffic(m, "D3Q19", read_bytes=64)["reads"]
            >= traffic.sector_traffic(m, "D3Q19")["reads"])
