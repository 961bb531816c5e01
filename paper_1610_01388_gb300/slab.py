"""One lattice Boltzmann domain split into z-slabs.

A time step reads only the nearest neighbours of each cell (the streaming of
eq. 8), so a domain periodic in z splits into slabs of consecutive z-planes
that need, before every step, one plane of populations from each neighbour:
the populations with c_z = +1 of the lower neighbour's last plane and those
with c_z = -1 of the upper neighbour's first plane.  Each slab is a solver
over its own planes plus one ghost plane on each side (LBM_FLAG_Z_GHOSTS):
the ghost planes are never stepped and carry the neighbours' mask rows, so
halfway bounce-back across a slab face is the whole domain's.  With the
exchange done before every step the slabs hold exactly the populations of
the undivided domain.

The pieces:
  split_z        the slab extents and their masks with ghost rows;
  GpuSlab        one slab on the GPU through the C ABI (pack / unpack of
                 the face populations, one step, the check-step sums);
  LocalRing      every slab in this process: faces move by reference;
  RankRing       one slab per rank of a torch.distributed process group:
                 faces travel by point-to-point send / receive (NCCL between
                 GPUs, gloo between CPU processes) to the ranks above and
                 below, periodic in z;
  SlabDomain     steps the slabs with the exchange and combines their flow
                 rates and residuals.
The rings and SlabDomain use only a stepper's pack(side), unpack(side, buf),
empty_face(), step(), sums() and flow_sums(), so any stepper with that
interface is decomposed the same way; a stepper that also takes a step in
parts (step_inner, step_faces, next_is_check) gets the exchange overlapped
with the update of its inner planes.
"""
from __future__ import annotations

import numpy as np

from . import lbm


def split_z(mask: np.ndarray, nslabs: int):
    """[(z0, nz_local, slab_mask)]: nslabs runs of consecutive z-planes whose
    sizes differ by at most one, each slab's mask with the plane below its
    first plane and the plane above its last one as ghost rows (periodic)."""
    mask = np.ascontiguousarray(mask, np.uint8)
    nz = mask.shape[0]
    if not 1 <= nslabs <= nz:
        raise ValueError(f"nslabs must be in 1..{nz}")
    out = []
    z0 = 0
    for k in range(nslabs):
        nl = nz // nslabs + (1 if k < nz % nslabs else 0)
        rows = [(z0 - 1) % nz] + list(range(z0, z0 + nl)) + [(z0 + nl) % nz]
        out.append((z0, nl, np.ascontiguousarray(mask[rows])))
        z0 += nl
    return out


class GpuSlab:
    """One z-slab as a solver with ghost planes (C ABI).  pack(1) returns the
    last interior plane's c_z = +1 populations, pack(0) the first interior
    plane's c_z = -1 populations, as a device tensor of stored values;
    unpack(0, buf) writes a lower neighbour's pack(1) into the lower ghost
    plane, unpack(1, buf) an upper neighbour's pack(0) into the upper one."""

    def __init__(self, lattice, slab_mask, z0, flags=0, **params):
        import torch
        nzg, ny, nx = slab_mask.shape
        self.nz_local = nzg - 2
        self.nx, self.ny = nx, ny
        self.solver = lbm.Solver(lattice, slab_mask, flags=flags | lbm.LBM_FLAG_Z_GHOSTS,
                                 use_torch=True, **params)
        # global index of local cell n is n + (z0 - 1) nx ny
        lbm.lbm_set_hash_offset(self.solver.h, (z0 - 1) * nx * ny)
        nbytes = lbm.lbm_halo_bytes(self.solver.h)
        self._out = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]

    def pack(self, side):
        buf = self._out[side]
        lbm.lbm_halo_pack(self.solver.h, side, buf.data_ptr())
        return buf

    def empty_face(self):
        import torch
        return torch.empty_like(self._out[0])

    def unpack(self, side, buf):
        lbm.lbm_halo_unpack(self.solver.h, side, buf.data_ptr())

    def step(self, n=1):
        self.solver.step(n)

    def next_is_check(self):
        k = self.solver.params.check_every
        return k > 0 and (lbm.lbm_get_info(self.solver.h).steps_done + 1) % k == 0

    def step_inner(self):
        """The planes that read no ghost value (interior planes 2..nz_local-1)."""
        nxy = self.nx * self.ny
        if self.nz_local > 2:
            lbm.lbm_step_cells(self.solver.h, 2 * nxy, self.nz_local * nxy)

    def step_faces(self):
        """The two interior planes next to the faces, then the buffer flip."""
        nxy = self.nx * self.ny
        lbm.lbm_step_cells(self.solver.h, nxy, 2 * nxy)
        if self.nz_local > 1:
            lbm.lbm_step_cells(self.solver.h, self.nz_local * nxy, (self.nz_local + 1) * nxy)
        lbm.lbm_step_commit(self.solver.h)

    def sync(self):
        self.solver.sync()

    def sums(self):
        """(sum of u_real [3], sum |u - u_prev|^2, sum |u|^2) of the last check step."""
        return lbm.lbm_check_sums(self.solver.h)

    def flow_sums(self):
        """Current sums of u_real over the slab's fluid cells, per axis."""
        L = (self.nx, self.ny, self.nz_local + 2)
        return np.array([self.solver.flowrate(a) * L[a] for a in range(3)])

    def fields(self):
        """rho, u of the interior planes."""
        rho, u = self.solver.fields()
        return rho[1:-1], u[:, 1:-1]

    def populations(self):
        """Full FP64 populations of the interior planes, (Q, nz_local, ny, nx)."""
        f = self.solver.get_populations()
        return f[:, 1:-1]

    def close(self):
        self.solver.close()


class LocalRing:
    """All slabs in this process, slab k above slab k - 1 (periodic)."""

    def __init__(self, slabs):
        self.slabs = list(slabs)

    def exchange(self):
        self.exchange_begin()
        self.exchange_end()

    def exchange_begin(self):
        self._faces = ([s.pack(1) for s in self.slabs], [s.pack(0) for s in self.slabs])

    def exchange_end(self):
        up, down = self._faces
        n = len(self.slabs)
        for k, s in enumerate(self.slabs):
            s.unpack(0, up[(k - 1) % n])     # the lower neighbour's upward populations
            s.unpack(1, down[(k + 1) % n])   # the upper neighbour's downward populations

    def allreduce(self, values):
        return values


class RankRing:
    """One slab per rank: rank r's slab lies above rank r - 1's (periodic).
    Each exchange sends this slab's upward face to rank r + 1 and its
    downward face to rank r - 1, and receives the matching faces from them
    (tags 0 up, 1 down; with two ranks both neighbours are the same rank and
    the tags keep the faces apart)."""

    def __init__(self, slab, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.slab = slab
        self.slabs = [slab]
        self._recv = [slab.empty_face(), slab.empty_face()]

    def exchange(self):
        self.exchange_begin()
        self.exchange_end()

    def exchange_begin(self):
        """Pack both faces and start their transfer (returns at once)."""
        up, down = self.slab.pack(1), self.slab.pack(0)
        self._reqs = None
        if self.world == 1:
            self._local = (up, down)
            return
        d = self.dist
        above, below = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        peer = (lambda r: d.get_global_rank(self.group, r)) if self.group is not None else (lambda r: r)
        self._sync_device()
        # one group of point-to-point operations: NCCL runs separately issued
        # sends and receives in order on its stream, so two ranks that both
        # send first would wait on each other
        ops = [d.P2POp(d.isend, up, peer(above), self.group, 0),
               d.P2POp(d.irecv, self._recv[0], peer(below), self.group, 0),
               d.P2POp(d.isend, down, peer(below), self.group, 1),
               d.P2POp(d.irecv, self._recv[1], peer(above), self.group, 1)]
        self._reqs = d.batch_isend_irecv(ops)

    def exchange_end(self):
        """Wait for the faces and write them into the ghost planes."""
        if self._reqs is None:
            up, down = self._local
            self.slab.unpack(0, up)
            self.slab.unpack(1, down)
            return
        for r in self._reqs:
            r.wait()
        self._reqs = None
        self.slab.unpack(0, self._recv[0])
        self.slab.unpack(1, self._recv[1])

    def _sync_device(self):
        # the packs run on the solver's stream; the transport reads the buffers
        sync = getattr(self.slab, "sync", None)
        if sync is not None:
            sync()

    def allreduce(self, values):
        import torch
        # on the faces' device: NCCL reduces device tensors, gloo host ones
        t = torch.as_tensor(np.asarray(values, np.float64), device=self._recv[0].device)
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()


class SlabDomain:
    """A domain of global extent (nz, ny, nx) stepped as z-slabs.  Every step
    exchanges the faces, then steps each slab once; check steps (every
    check_every-th step of every slab) give combined flow rates and the
    residual."""

    def __init__(self, ring, nz, nx, ny):
        self.ring = ring
        self.nz, self.ny, self.nx = nz, ny, nx

    def step(self, n=1):
        """n steps.  A plain step, when every slab can take one in parts,
        overlaps the face exchange with the update of the planes that read
        no ghost value; a check step exchanges first and steps whole."""
        for _ in range(int(n)):
            slabs = self.ring.slabs
            if all(hasattr(s, "step_inner") and not s.next_is_check() for s in slabs):
                self.ring.exchange_begin()
                for s in slabs:
                    s.step_inner()
                self.ring.exchange_end()
                for s in slabs:
                    s.step_faces()
            else:
                self.ring.exchange()
                for s in slabs:
                    s.step(1)

    def check_sums(self):
        """(sum of u_real [3], sum |u - u_prev|^2, sum |u|^2) over the whole
        domain at the last check step."""
        tot = np.zeros(5)
        for s in self.ring.slabs:
            us, du2, u2 = s.sums()
            tot += np.concatenate([us, [du2, u2]])
        tot = self.ring.allreduce(tot)
        return tot[:3], tot[3], tot[4]

    def residual(self):
        _, du2, u2 = self.check_sums()
        return float(np.sqrt(du2 / u2)) if u2 > 0 else -1.0

    def refresh_ghosts(self):
        """Fill the ghost planes from the current state.  A step leaves them
        holding the faces exchanged before it, and the fields of the planes
        next to a face are moments of populations pulled from them; the
        exchange writes ghost planes only, so repeating it is harmless."""
        self.ring.exchange()

    def fields(self):
        """rho (nz, ny, nx) and u_real (3, nz, ny, nx) of this process's slabs,
        stacked along z (the whole domain for a LocalRing)."""
        self.refresh_ghosts()
        parts = [s.fields() for s in self.ring.slabs]
        return (np.concatenate([r for r, _ in parts], axis=0),
                np.concatenate([u for _, u in parts], axis=1))

    def flowrate(self, axis=0):
        """Q_a = (1/L_a) sum over the domain's fluid cells of u_real,a, now."""
        self.refresh_ghosts()
        tot = np.zeros(3)
        for s in self.ring.slabs:
            tot += s.flow_sums()
        tot = self.ring.allreduce(tot)
        return float(tot[axis] / (self.nx, self.ny, self.nz)[axis])


def gpu_slab_domain(lattice, mask, nslabs, **params):
    """All slabs of `mask` on this process's GPU (a LocalRing)."""
    mask = np.ascontiguousarray(mask, np.uint8)
    nz, ny, nx = mask.shape
    slabs = [GpuSlab(lattice, m, z0, **params) for z0, _, m in split_z(mask, nslabs)]
    return SlabDomain(LocalRing(slabs), nz, nx, ny)


def gpu_rank_slab(lattice, mask, group=None, **params):
    """This rank's slab of `mask` (slab r of the group's world size) in a
    RankRing; every rank passes the same global mask."""
    import torch.distributed as dist
    mask = np.ascontiguousarray(mask, np.uint8)
    nz, ny, nx = mask.shape
    r, w = dist.get_rank(group), dist.get_world_size(group)
    z0, _, m = split_z(mask, w)[r]
    return SlabDomain(RankRing(GpuSlab(lattice, m, z0, **params), group), nz, nx, ny)
