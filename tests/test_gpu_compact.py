"""The compact layout (LBM_FLAG_COMPACT): the planes hold the fluid cells
only, one slot each, and one thread steps one slot.  The pull (eq. 8 with
halfway bounce-back) and the collision are the dense layout's source, but the
two kernels are compiled apart, and the compiler may contract multiply-adds
differently in each: on every fluid cell the populations, the velocity
field, the PR relaxation time, the flow rate, totals and residual must agree
with the dense solver to round-off of the arithmetic type (measured: 0 to
3e-7 relative in FP32 after 30 steps, 1e-14 in FP64; a one-ulp difference
can move a 16-bit rounding by one step), and the layout must match the FP64
oracle at the dense layout's bars.  Solid cells hold nothing and read back
as the rest state."""
import numpy as np
import pytest

from paper_1610_01388_gb300 import lbm
from paper_1610_01388_gb300 import workloads as W
from _pairs import make_pair, rel_l2_u

pytestmark = pytest.mark.gpu

BURNETT = lbm.LBM_FLAG_BURNETT_X


def _disks_2d(nx, ny, n, r, seed):
    """Periodic random disks (may overlap): a 2D porous geometry."""
    rng = np.random.Generator(np.random.PCG64(seed))
    y, x = np.mgrid[0:ny, 0:nx]
    mask = np.zeros((ny, nx), np.uint8)
    for cx, cy in zip(rng.uniform(0, nx, n), rng.uniform(0, ny, n)):
        dx = np.minimum(np.abs(x - cx), nx - np.abs(x - cx))
        dy = np.minimum(np.abs(y - cy), ny - np.abs(y - cy))
        mask[dx * dx + dy * dy < r * r] = 1
    return mask


def _mask(lat):
    if lat == "D2Q9":
        return _disks_2d(45, 37, 12, 3.5, seed=3)
    return W.porous_mask((24, 20, 16), porosity=0.7, r_min=2.0, r_max=4.0, seed=6)[0]


def _pair(lat, mask, **prm):
    d = lbm.Solver(lat, mask, use_torch=True, **prm)
    c = lbm.Solver(lat, mask, use_torch=True, layout="compact", **prm)
    return d, c


# population / velocity / flow-rate bar (relative), and the residual's
TOL = {"F64": (1e-12, 1e-9), "F32": (1e-5, 1e-3), "F16": (2e-3, 5e-2), "BF16": (1e-2, 2e-1)}


def _rel(a, b, scale):
    return float(np.max(np.abs(a - b)) / scale)


@pytest.mark.parametrize("lat,model,storage,newton,flags", [
    ("D3Q19", "PR", "F32", 0, 0), ("D3Q19", "IR", "F32", 0, 0),
    ("D3Q19", "PR", "F16", 0, 0), ("D3Q19", "IR", "F16", 0, 0),
    ("D3Q27", "PR", "F32", 0, 0), ("D3Q27", "IR", "BF16", 0, 0),
    ("D3Q15", "PR", "F64", 0, 0), ("D3Q15", "IR", "F32", 0, BURNETT),
    ("D2Q9", "PR", "F32", 0, 0), ("D2Q9", "IR", "F64", 0, 0),
    ("D3Q19", "PR", "F32", 3, 0), ("D3Q27", "PR", "F64", 2, BURNETT),
])
def test_compact_matches_dense(lat, model, storage, newton, flags):
    mask = _mask(lat)
    g = (2e-5, 1e-6, 0.0) if lat == "D2Q9" else (2e-5, 1e-6, -2e-6)
    prm = dict(model=model, storage=storage, mu_p=0.1, sigma_y=2e-6, m=1e6, g=g,
               check_every=7, flags=flags, newton_iters=newton)
    tol, rtol = TOL[storage]
    d, c = _pair(lat, mask, **prm)
    _, w = lbm.lbm_lattice_info(lat)
    f0 = W.random_populations(w, mask.size, amplitude=0.02, seed=11)
    d.set_populations(f0)
    c.set_populations(f0)
    d.step(30)                                  # four check steps, two after the last
    c.step(30)
    fluid = mask.reshape(-1) == 0
    fd = d.get_populations().reshape(len(w), -1)
    fc = c.get_populations().reshape(len(w), -1)
    scale = np.max(np.abs(fd[:, fluid] - w[:, None]))
    assert _rel(fc[:, fluid], fd[:, fluid], scale) <= tol
    assert np.array_equal(fc[:, ~fluid], np.broadcast_to(w[:, None], fc[:, ~fluid].shape))
    rd, ud = d.fields()
    rc, uc = c.fields()
    assert _rel(uc, ud, np.max(np.abs(ud))) <= tol
    assert _rel(rc, rd, 1.0) <= tol * scale
    if model == "PR":
        td, tc = d.get_tau().reshape(-1), c.get_tau().reshape(-1)
        assert _rel(tc[fluid], td[fluid], np.max(td[fluid])) <= tol
        t0 = 0.5 + 3.0 * (0.1 + 1e6 * 2e-6)
        assert np.all(tc[~fluid] == (t0 if storage == "F64" else float(np.float32(t0))))
    ext = mask.shape[::-1] + (1,) * (3 - mask.ndim)          # nx, ny, nz
    for a in range(3 if lat != "D2Q9" else 2):
        q = d.flowrate(a)
        assert abs(c.flowrate(a) - q) <= tol * np.sum(np.abs(ud[a])) / ext[a] + 1e-18, a
    md, pd = d.totals()
    mc, pc = c.totals()
    assert abs(mc - md) <= tol * scale * fluid.sum()
    assert np.allclose(pc, pd, rtol=0, atol=tol * scale * fluid.sum())
    rd_, atd, _ = d.residual()
    rc_, atc, _ = c.residual()
    assert atd == atc == 28
    assert abs(rc_ - rd_) <= rtol * rd_
    d.close()
    c.close()


@pytest.mark.parametrize("lat,model,storage,bar", [
    ("D3Q19", "IR", "F64", 1e-10), ("D3Q19", "PR", "F64", 1e-10),
    ("D3Q27", "PR", "F32", 1e-5), ("D3Q15", "IR", "F32", 1e-5),
])
def test_compact_matches_oracle(lat, model, storage, bar):
    """A 40^3 sample of the porous-medium generator (spheres of radius 3-6,
    porosity 0.7), 300 steps from rest: the velocity field at equal step
    count and the flow rate against the FP64 oracle."""
    mask, _ = W.porous_mask(40, porosity=0.7, r_min=3.0, r_max=6.0, seed=2)
    s, o = make_pair(lat, mask, model=model, storage=storage, sigma_y=2e-6, m=1e6,
                     g=(2e-5, 0, 0), use_torch=True, layout="compact")
    s.step(300)
    o.step(300)
    assert rel_l2_u(s, o) < bar
    q = o.flowrate(0)
    assert abs(s.flowrate(0) - q) < bar * abs(q)
    s.close()


def test_compact_probes_and_uploads():
    """Populations of listed cells (solid ones read as w_i), an upload that
    drops the solid cells, tau transfers through the slot map."""
    lat = "D3Q19"
    mask = _mask(lat)
    _, w = lbm.lbm_lattice_info(lat)
    c = lbm.Solver(lat, mask, model="PR", storage="F64", mu_p=0.1, sigma_y=1e-6, m=1e5,
                   layout="compact", use_torch=True)
    n = mask.size
    f = W.random_populations(w, n, amplitude=0.05, seed=4)
    c.set_populations(f)
    fluid = mask.reshape(-1) == 0
    got = c.get_populations().reshape(len(w), -1)
    assert np.array_equal(got[:, fluid], f[:, fluid])
    assert np.array_equal(got[:, ~fluid], np.broadcast_to(w[:, None], got[:, ~fluid].shape))
    rng = np.random.Generator(np.random.PCG64(1))
    cells = rng.choice(n, 300, replace=False).astype(np.int64)
    assert (~fluid[cells]).any() and fluid[cells].any()
    probe = lbm.lbm_get_populations_cells(c.h, cells, len(w))
    assert np.array_equal(probe, got[:, cells])
    tau = rng.uniform(0.6, 1.4, n)
    c.set_tau(tau)
    back = c.get_tau().reshape(-1)
    assert np.array_equal(back[fluid], tau[fluid])
    assert np.all(back[~fluid] == 0.5 + 3.0 * (0.1 + 1e5 * 1e-6))
    c.close()


def test_compact_refusals():
    """Steps in parts need the dense planes; batches and the server take
    whole dense domains."""
    mask = _mask("D3Q19")
    c = lbm.Solver("D3Q19", mask, layout="compact", use_torch=True)
    for call in (lambda: lbm.lbm_step_cells(c.h, 0, 10), lambda: lbm.lbm_step_commit(c.h)):
        with pytest.raises(lbm.LbmError) as e:
            call()
        assert e.value.status == lbm.LBM_EINVAL
    c.close()
    b = lbm.Batch(1 << 30, check_every=10)
    with pytest.raises(lbm.LbmError) as e:
        b.add("D3Q19", mask, flags=lbm.LBM_FLAG_COMPACT)
    assert e.value.status == lbm.LBM_EINVAL
    b.close()
    srv = lbm.Server(1 << 30, check_every=10)
    for flags in (lbm.LBM_FLAG_COMPACT, lbm.LBM_FLAG_Z_GHOSTS):
        with pytest.raises(lbm.LbmError) as e:
            srv.submit("D3Q19", mask, flags=flags)
        assert e.value.status == lbm.LBM_EINVAL
    srv.close()


@pytest.mark.parametrize("storage", ["F16", "BF16"])
@pytest.mark.parametrize("layout", ["dense", "compact"])
def test_totals_of_16bit_storage(storage, layout):
    """Mass and momentum of the stored state, against FP64 sums of the
    populations read back: the 16-bit forms interleave each opposite pair,
    so element n of population i > 0 sits at 2 n past its plane's base."""
    lat = "D3Q27"
    mask = _mask(lat)
    c_, w = lbm.lbm_lattice_info(lat)
    s = lbm.Solver(lat, mask, storage=storage, layout=layout, use_torch=True)
    s.set_populations(W.random_populations(w, mask.size, amplitude=0.3, seed=9))
    f = s.get_populations().reshape(len(w), -1)[:, mask.reshape(-1) == 0]
    mass, mom = s.totals()
    df = f - w[:, None]
    scale = np.abs(df).sum()
    assert abs((mass - f.shape[1]) - df.sum()) <= 1e-6 * scale
    want = np.asarray(c_, np.float64).reshape(-1, 3).T @ df.sum(axis=1)
    assert np.allclose(mom, want, rtol=0, atol=1e-6 * scale)
    s.close()
