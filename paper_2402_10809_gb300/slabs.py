"""z-slab decomposition of one problem over several contexts (the C ABI's
lbm_slab_bounds, lbm_set_halo, lbm_halo_* calls; argument marshalling only).

A slab owns the z-planes [z0, z1) of the box and is a context on the sub-box
[z0 - h0, z1 + h1) with one halo plane on each side that has a neighbour.
After every time step the populations that a slab pulls across a face (those
whose c_z points into it) are copied from the neighbour's plane next to the
face into the slab's halo plane.  Every cell then computes exactly what it
computes in the unsharded box.

* :class:`SlabSimulation`: all slabs on one device, one stream; the faces are
  exchanged by lbm_halo_exchange.
* :class:`ShardedSimulation`: one slab per process (torch.distributed, NCCL
  between GPUs); each face is packed, sent and received with
  :func:`exchange_faces` and unpacked.
"""

import dataclasses

import numpy as np

from . import lbm as L


def slab_bounds(problem, nslabs):
    """z0 of each slab plus the box's nz, balanced by packed slots."""
    if nslabs > 1 and problem.periodic[2]:
        raise ValueError("a box periodic in z is not sharded into z-slabs")
    grid = L.make_grid(problem.dims, problem.q, "f32", problem.periodic)
    flags = np.ascontiguousarray(problem.flags, dtype=np.uint8)
    return L.lbm_slab_bounds(grid, flags.ctypes.data, nslabs)


def slab_problem(problem, z0, z1):
    """(sub-problem of the slab [z0, z1) with its halo planes, h0, h1)."""
    nz = problem.dims[2]
    h0, h1 = int(z0 > 0), int(z1 < nz)
    a, b = z0 - h0, z1 + h1
    sub = dataclasses.replace(
        problem, name=f"{problem.name}_z{z0}_{z1}", flags=np.ascontiguousarray(problem.flags[a:b]),
        phi=np.ascontiguousarray(problem.phi[a:b]),
        region=None if problem.region is None else np.ascontiguousarray(problem.region[a:b]))
    return sub, h0, h1


def combine_diag(parts):
    """Diagnostics of the box from those of its slabs: sums of mass, kinetic
    energy, region |u| sum, region count and non-finite count; max |u|;
    the omega range."""
    d = np.array(parts, dtype=np.float64)
    out = d.sum(axis=0)
    out[4] = d[:, 4].max()
    out[5] = d[:, 5].min()
    out[6] = d[:, 6].max()
    return out


class SlabSimulation:
    """One problem as ``nslabs`` z-slabs on one device.  With ``concurrent``
    every slab has a stream of its own and lbm_step_slabs lets the slabs step
    at the same time (each face exchanged once its two slabs have stepped);
    otherwise all of them share the current stream and step in turn.  Either
    way the work is ordered against the current stream of the device."""

    def __init__(self, problem, nslabs, storage="f32", device="cuda", concurrent=True):
        import torch

        self.problem = problem
        self.bounds = slab_bounds(problem, nslabs)
        dev = torch.device(device)
        self.stream = torch.cuda.current_stream(dev)
        self.streams = [torch.cuda.Stream(dev) if concurrent else self.stream for _ in range(nslabs)]
        self.sims, self.halo = [], []
        for k in range(nslabs):
            sub, h0, h1 = slab_problem(problem, self.bounds[k], self.bounds[k + 1])
            if concurrent:
                # the set-up on the slab's stream follows the current stream's work
                self.streams[k].wait_stream(self.stream)
            sim = L.Simulation(sub, storage=storage, device=device, stream=self.streams[k])
            L.lbm_set_halo(sim.ctx, h0, h1)
            # the slabs step in turn: they share the persisting L2 (their
            # per-slot words together are the unsharded box's)
            L.lbm_set_l2_group(sim.ctx, id(self))
            self.sims.append(sim)
            self.halo.append((h0, h1))

    def close(self):
        for st in self.streams:
            st.synchronize()  # before the workspaces go back to the allocator
        for s in self.sims:
            s.close()

    @property
    def t(self):
        return self.sims[0].t

    def step(self, n=1):
        L.lbm_step_slabs([s.ctx for s in self.sims], n, self.stream.cuda_stream)

    def moments(self):
        """rho, u, gdot, omega on the dense box (host), from the slabs' interiors."""
        shape = self.problem.flags.shape
        out = dict(rho=np.zeros(shape, np.float32), u=np.zeros((3,) + shape, np.float32),
                   gdot=np.zeros(shape, np.float32), omega=np.zeros(shape, np.float32))
        for k, s in enumerate(self.sims):
            m = s.moments()
            z0, z1 = self.bounds[k], self.bounds[k + 1]
            h0 = self.halo[k][0]
            for key in ("rho", "gdot", "omega"):
                out[key][z0:z1] = m[key][h0:h0 + z1 - z0]
            out["u"][:, z0:z1] = m["u"][:, h0:h0 + z1 - z0]
        return out

    def diag(self, region=None):
        parts = []
        for k, s in enumerate(self.sims):
            if region is None:
                parts.append(s.diag())
            else:
                z0, z1 = self.bounds[k], self.bounds[k + 1]
                h0, h1 = self.halo[k]
                parts.append(s.diag(np.ascontiguousarray(region[z0 - h0:z1 + h1])))
        return combine_diag(parts)


def exchange_faces(dist, rank, world, pack, unpack, send, recv):
    """One exchange of the faces of slab ``rank`` of ``world``: pack the faces
    that have a neighbour (side 0 toward rank - 1, side 1 toward rank + 1),
    post every send and receive together, wait, unpack.  ``pack(side, buf)``
    / ``unpack(side, buf)`` move the populations between the state and the
    message buffers ``send[side]`` / ``recv[side]``."""
    ops = []
    for side, peer in ((0, rank - 1), (1, rank + 1)):
        if 0 <= peer < world:
            pack(side, send[side])
            ops.append(dist.P2POp(dist.isend, send[side], peer))
            ops.append(dist.P2POp(dist.irecv, recv[side], peer))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for side, peer in ((0, rank - 1), (1, rank + 1)):
        if 0 <= peer < world:
            unpack(side, recv[side])


def face_message_elements(flags, q, side, h0, h1):
    """Elements of the message a slab receives on ``side`` (the halo plane's
    slots times the directions crossing the face), from its sub-box flags."""
    nz, ny, nx = flags.shape
    grid = L.make_grid((nx, ny, nz), q, "f32", (0, 0, 0))
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    z = 0 if side == 0 else nz - 1
    _, count = L.lbm_plane_slots(grid, f.ctypes.data, z)
    return (9 if q == 27 else 5) * count


class ShardedSimulation:
    """This process's slab of a problem sharded over the processes of a
    torch.distributed group (one GPU each); faces travel as packed messages."""

    def __init__(self, problem, dist, storage="f32", device="cuda"):
        import torch

        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.bounds = slab_bounds(problem, self.world)
        z0, z1 = self.bounds[self.rank], self.bounds[self.rank + 1]
        sub, h0, h1 = slab_problem(problem, z0, z1)
        self.sim = L.Simulation(sub, storage=storage, device=device)
        L.lbm_set_halo(self.sim.ctx, h0, h1)
        self.halo = (h0, h1)
        dt = torch.float32 if storage == "f32" else torch.float16
        es = 4 if storage == "f32" else 2
        self.send, self.recv = {}, {}
        for side in (0, 1):
            if self.halo[side]:
                nbytes = L.lbm_halo_message_size(self.sim.ctx, side)
                self.send[side] = torch.empty(nbytes // es, dtype=dt, device=self.sim.device)
                self.recv[side] = torch.empty(face_message_elements(sub.flags, problem.q, side, h0, h1), dtype=dt,
                                              device=self.sim.device)

    def close(self):
        self.sim.close()

    def step(self, n=1):
        ctx = self.sim.ctx
        for _ in range(n):
            L.lbm_step(ctx, 1)
            exchange_faces(self.dist, self.rank, self.world,
                           lambda side, buf: L.lbm_halo_pack(ctx, side, buf.data_ptr()),
                           lambda side, buf: L.lbm_halo_unpack(ctx, side, buf.data_ptr()),
                           self.send, self.recv)

    def diag(self, region=None):
        """The box's diagnostics on every rank (FP64 all-gather of the slabs')."""
        import torch

        if region is None:
            d = self.sim.diag()
        else:
            z0, z1 = self.bounds[self.rank], self.bounds[self.rank + 1]
            d = self.sim.diag(np.ascontiguousarray(region[z0 - self.halo[0]:z1 + self.halo[1]]))
        t = torch.tensor(d, dtype=torch.float64, device=self.sim.device)
        parts = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(parts, t)
        return combine_diag([p.cpu().numpy() for p in parts])
