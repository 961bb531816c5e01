"""The z-slab decomposition's host logic (paper_1610_01388_gb300.slab) on
CPU: the split with its ghost rows, and the exchange between gloo ranks.

The rank exchange is driven with a stepper backed by the FP64 oracle (test
code: each rank steps its slab's planes, ghost rows included, and the ring
fills the ghost planes before every step).  A step reads only the nearest
neighbours (eq. 8), so after n steps every interior plane must equal the
undivided domain's oracle run bit for bit, and the flow rate summed over the
ranks must equal the undivided one."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1610_01388_gb300 import slab
from paper_1610_01388_gb300 import workloads as W


def test_split_z_sizes_and_ghost_rows():
    mask = (np.arange(11)[:, None, None] * np.ones((1, 3, 4), np.uint8)).astype(np.uint8)
    parts = slab.split_z(mask, 3)
    assert [p[1] for p in parts] == [4, 4, 3]
    assert [p[0] for p in parts] == [0, 4, 8]
    for z0, nl, m in parts:
        assert m.shape == (nl + 2, 3, 4)
        rows = [int(r[0, 0]) for r in m]
        assert rows == [(z0 - 1) % 11] + list(range(z0, z0 + nl)) + [(z0 + nl) % 11]
    assert slab.split_z(mask, 1)[0][2][0, 0, 0] == 10          # periodic: plane below 0 is 10
    with pytest.raises(ValueError):
        slab.split_z(mask, 12)


class OracleSlab:
    """Stepper over the oracle for one slab (planes 0 and -1 are the ghosts)."""

    def __init__(self, lattice, slab_mask, params):
        import oracle
        self.st = oracle.State(lattice, params, slab_mask)
        self.nzg, self.ny, self.nx = slab_mask.shape
        self.nz_local = self.nzg - 2
        c = self.st.c
        self.up = np.flatnonzero(c[:, 2] == 1)
        self.down = np.flatnonzero(c[:, 2] == -1)
        self.nxy = self.nx * self.ny

    def _plane(self, z):
        return slice(z * self.nxy, (z + 1) * self.nxy)

    def pack(self, side):
        import torch
        pops, z = (self.up, self.nzg - 2) if side == 1 else (self.down, 1)
        return torch.from_numpy(np.ascontiguousarray(self.st.f[pops][:, self._plane(z)]))

    def empty_face(self):
        import torch
        return torch.empty((len(self.up), self.nxy), dtype=torch.float64)

    def unpack(self, side, buf):
        pops, z = (self.up, 0) if side == 0 else (self.down, self.nzg - 1)
        f = self.st.f
        f[np.ix_(pops, np.arange(self._plane(z).start, self._plane(z).stop))] = buf.numpy()

    def step(self, n=1):
        self.st.step(n)

    def flow_sums(self):
        _, u = self.st.fields()
        fl = self.st.mask[1:-1] == 0
        return np.array([u[a][1:-1][fl].sum() for a in range(3)])

    def interior(self):
        return self.st.f[:, self.nxy:-self.nxy]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    import oracle
    mask, _ = W.porous_mask(12, porosity=0.7, r_min=2.0, r_max=3.0, seed=6)
    p = dict(nu_p=0.1, sigma_y=2e-5, m=1e5, g=(2e-5, 3e-6, -4e-6))
    return mask, p


def _worker(rank, world, port, model, lattice, nsteps, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mask, p = _case()
    z0, nl, m = slab.split_z(mask, world)[rank]
    o = OracleSlab(lattice, m, oracle.params(model=model, **p))
    ring = slab.RankRing(o)
    nz, ny, nx = mask.shape
    dom = slab.SlabDomain(ring, nz, nx, ny)
    dom.step(nsteps)
    q.put((rank, z0, nl, o.interior().copy(), dom.flowrate(0), dom.flowrate(2)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,model,lattice", [(2, "PR", "D3Q19"), (3, "IR", "D3Q27"),
                                                 (2, "IR", "D3Q15")])
def test_rank_ring_matches_undivided_oracle(world, model, lattice):
    import oracle
    nsteps = 25
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, model, lattice, nsteps, q))
          for r in range(world)]
    for p in ps:
        p.start()
    out = sorted((q.get(timeout=180) for _ in ps), key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    mask, prm = _case()
    ref = oracle.State(lattice, oracle.params(model=model, **prm), mask)
    ref.step(nsteps)
    nxy = mask.shape[1] * mask.shape[2]
    for rank, z0, nl, f, qx, qz in out:
        want = ref.f[:, z0 * nxy:(z0 + nl) * nxy]
        assert np.array_equal(f, want), (rank, np.max(np.abs(f - want)))
        assert qx == pytest.approx(ref.flowrate(0), rel=1e-12, abs=1e-18)
        assert qz == pytest.approx(ref.flowrate(2), rel=1e-12, abs=1e-18)


def test_rank_ring_catches_a_swapped_face():
    """The same exchange with the faces crossed (downward populations into
    the lower ghost plane) no longer matches the undivided run: the pin above
    would catch a wrong face, sign or neighbour."""
    import oracle
    mask, prm = _case()
    p = oracle.params(model="IR", **prm)
    parts = slab.split_z(mask, 2)
    slabs = [OracleSlab("D3Q19", m, p) for _, _, m in parts]

    class Crossed(slab.LocalRing):
        def exchange(self):
            up = [s.pack(1) for s in self.slabs]
            down = [s.pack(0) for s in self.slabs]
            for k, s in enumerate(self.slabs):
                s.unpack(0, down[(k - 1) % 2])
                s.unpack(1, up[(k + 1) % 2])

    good = [OracleSlab("D3Q19", m, p) for _, _, m in parts]
    nz, ny, nx = mask.shape
    slab.SlabDomain(slab.LocalRing(good), nz, nx, ny).step(10)
    slab.SlabDomain(Crossed(slabs), nz, nx, ny).step(10)
    ref = oracle.State("D3Q19", p, mask)
    ref.step(10)
    nxy = mask.shape[1] * mask.shape[2]
    assert np.array_equal(good[0].interior(), ref.f[:, :parts[0][1] * nxy])
    assert not np.array_equal(slabs[0].interior(), ref.f[:, :parts[0][1] * nxy])
