"""Slab decomposition of one lattice along z: the box's z layers are split into
consecutive slabs, each a lattice of its own (lbm_set_slab) with two halo
layers on each side, and one exchange of edge layers per time step.

The paper gives no parallel scheme; this places its step on slabs (Sec. 2:
the pull reads one layer across a cut; Sec. 3: the refill of a node in that
layer averages densities one layer further out, hence two halo layers).
Before every step each slab's halo layers take the neighbouring slabs' own
edge layers (all 27 post-collision populations); after it the slabs' forces
and torques, each summed over the links of its own fluid nodes, are added in
slab order and handed back to every slab's copy of the body, so all copies
move alike.  Own nodes then end every step with the bits of the undivided
lattice while the body's velocity does not depend on the force; a free body
differs by the order in which the link forces are added.

SlabSet keeps all slabs in this process (one device or several, the edge
layers moved by device copies); DistSlab is one slab per rank of a
torch.distributed process group (NCCL between GPUs), the edge layers sent
and received as packed device tensors.  This module is host orchestration
only: every step of the method runs in liblbm.so.
"""
from __future__ import annotations

import numpy as np

from . import binding as _b

HALO = 2


def slab_bounds(nz: int, parts: int, k: int) -> tuple[int, int]:
    """Own z layers [z0, z1) of slab k of parts: consecutive, sizes differing by one."""
    return k * nz // parts, (k + 1) * nz // parts


def slab_rows(nz: int, parts: int, k: int, halo: int = HALO) -> list[int]:
    """The box's z layer of each local layer of slab k (halo layers wrapped)."""
    z0, z1 = slab_bounds(nz, parts, k)
    return [(z0 - halo + j) % nz for j in range(z1 - z0 + 2 * halo)]


def _slab_lattice(shape, nu, storage, faces, parts, k, halo, device, local_z=_b.FACE_PERIODIC, two_phase=False,
                  **kw):
    nx, ny, nz = shape
    if faces[4] != _b.FACE_PERIODIC or faces[5] != _b.FACE_PERIODIC:
        raise ValueError("the split axis z must be periodic")
    z0, z1 = slab_bounds(nz, parts, k)
    if z1 - z0 < halo:
        raise ValueError("slabs thinner than the halo")
    nloc = z1 - z0 + 2 * halo
    # the slab's own z faces (no own node reads across them): periodic by
    # default, so the bulk kernel keeps its all-periodic form where x and y
    # are periodic; walls give the same own nodes
    local_faces = (faces[0], faces[1], faces[2], faces[3], local_z, local_z)
    lat = _b.Lattice((nx, ny, nloc), nu, storage=storage, faces=local_faces, device=device, **kw)
    lat.set_slab(z0 - halo, nz, halo, nloc - halo)
    if two_phase:  # the two-phase step takes the split launch order
        lat.set_launch_order("split")
    return lat


def _fixed_order_sum(parts):
    tot = np.array(parts[0], dtype=np.float64)
    for p in parts[1:]:
        tot = tot + np.asarray(p, dtype=np.float64)
    return tot


class SlabSet:
    """All slabs of one box in this process.  devices: one device for every
    slab, or a list (slab k on devices[k % len]); local_z: the slabs' own z
    face kind (FACE_PERIODIC or FACE_WALL); two_phase: each step as
    lbm_step_interior, the exchange, lbm_step_edges (else the exchange, then
    lbm_step)."""

    def __init__(self, shape, nu, parts, storage="fp32", faces=(0,) * 6, geometry=None, devices=None,
                 halo=HALO, local_z=_b.FACE_PERIODIC, two_phase=False, **kw):
        self.shape = tuple(int(v) for v in shape)
        self.parts, self.halo = int(parts), int(halo)
        self.two_phase = bool(two_phase)
        devs = devices if isinstance(devices, (list, tuple)) else [devices]
        self.slabs = [_slab_lattice(self.shape, nu, storage, faces, self.parts, k, self.halo,
                                    devs[k % len(devs)], local_z=local_z, two_phase=self.two_phase, **kw)
                      for k in range(self.parts)]
        self.launches = 0
        self.body = geometry is not None
        if self.body:
            for lat in self.slabs:
                lat.set_geometry(geometry)

    def init_state(self, rho, u, xi=None, amp: float = 0.0):
        """The whole box's fields (as Lattice.init_state takes them), each slab
        its layers and halos."""
        nz = self.shape[2]
        for k, lat in enumerate(self.slabs):
            rows = slab_rows(nz, self.parts, k, self.halo)
            lat.init_state(rho[rows], u[rows], xi[:, rows] if xi is not None else None, amp)

    def exchange(self):
        """Every slab's halo layers from its neighbours' own edge layers."""
        h = self.halo
        lows = [lat.pack_layers(h, h) for lat in self.slabs]                       # first own layers
        highs = [lat.pack_layers(lat.shape[2] - 2 * h, h) for lat in self.slabs]    # last own layers
        for k, lat in enumerate(self.slabs):
            lat.unpack_layers(0, highs[k - 1].to(lat.device))
            lat.unpack_layers(lat.shape[2] - h, lows[(k + 1) % self.parts].to(lat.device))

    def step(self, n: int = 1):
        """n steps: exchange, step every slab, then the slabs' forces added in
        slab order on the device and handed to every body copy
        (lbm_body_force_to_device, lbm_sum_body_force: no host round trip)."""
        import torch
        self.launches = 0
        for _ in range(n):
            if self.two_phase:
                for lat in self.slabs:
                    lat.step_interior()
                    self.launches += lat.launches()
                self.exchange()
                for lat in self.slabs:
                    lat.step_edges()
                    self.launches += lat.launches()
            else:
                self.exchange()
                for lat in self.slabs:
                    lat.step(1)
                    self.launches += lat.launches()
            if self.body:
                dev0 = self.slabs[0].device
                parts = torch.stack([lat.body_force_to().to(dev0) for lat in self.slabs])
                for lat in self.slabs:
                    lat.sum_body_force(parts.to(lat.device))
                    self.launches += 1
                self._parts = parts

    @property
    def last_force(self) -> np.ndarray:
        """The summed force and torque of the last step (host copy, FP64 6)."""
        return self.slabs[0].body_force_to().cpu().numpy()

    def populations(self) -> np.ndarray:
        """The own layers of every slab assembled into the whole box, decoded
        FP64 (27, nz, ny, nx)."""
        nx, ny, nz = self.shape
        out = np.empty((27, nz, ny, nx))
        h = self.halo
        for k, lat in enumerate(self.slabs):
            z0, z1 = slab_bounds(nz, self.parts, k)
            out[:, z0:z1] = lat.populations()[:, h:h + z1 - z0]
        return out

    def close(self):
        for lat in self.slabs:
            lat.close()


class DistSlab:
    """This rank's slab of one box split over the ranks of the default
    torch.distributed process group (one slab per rank, ranks in z order):
    edge layers by send/recv of packed device tensors, the force and torque
    records all-gathered and added in rank order on the device.  Every
    operation is enqueued on the lattice's stream (the collectives wait on it
    and it on them), so a step needs no host synchronisation.  two_phase (the
    default): the transfers are enqueued first and the bulk of the own layers
    that read no halo layer runs beside them (lbm_step_interior), the rest of
    the step after them (lbm_step_edges).  lattice: an object with the
    Lattice methods used here in place of a new slab lattice (the exchange and
    the force hand-over run on it unchanged)."""

    def __init__(self, shape, nu, storage="fp32", faces=(0,) * 6, geometry=None, device=None, halo=HALO,
                 lattice=None, two_phase=True, **kw):
        import torch.distributed as dist
        self.dist = dist
        if dist.is_available() and dist.is_initialized():
            self.world, self.rank = dist.get_world_size(), dist.get_rank()
        else:
            self.world, self.rank = 1, 0
        if self.world < 2:
            raise ValueError("DistSlab needs a process group of two or more ranks (one GPU: SlabSet)")
        self.shape = tuple(int(v) for v in shape)
        self.halo = int(halo)
        self.two_phase = bool(two_phase)
        self.lat = lattice if lattice is not None else \
            _slab_lattice(self.shape, nu, storage, faces, self.world, self.rank, self.halo, device,
                          two_phase=self.two_phase, **kw)
        self.body = geometry is not None
        if self.body and lattice is None:
            self.lat.set_geometry(geometry)
        self.z0, self.z1 = slab_bounds(self.shape[2], self.world, self.rank)
        self.launches = 0

    def init_state(self, rho, u, xi=None, amp: float = 0.0):
        rows = slab_rows(self.shape[2], self.world, self.rank, self.halo)
        self.lat.init_state(rho[rows], u[rows], xi[:, rows] if xi is not None else None, amp)

    def _on_stream(self):
        import contextlib

        import torch
        stream = getattr(self.lat, "stream", None)
        return torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext()

    def exchange(self, between=None):
        """Halo layers from the neighbouring ranks' own edge layers: rank r
        sends its first own layers down to r - 1 and its last up to r + 1
        (periodic in rank order).  between: called once the transfers are
        enqueued, before the lattice's stream waits for them."""
        lat, h = self.lat, self.halo
        nloc = lat.shape[2]
        lo_out, hi_out = lat.pack_layers(h, h), lat.pack_layers(nloc - 2 * h, h)
        import torch
        staged = self._host_staged()
        if staged:  # a host-only backend: the layers travel through host memory
            lo_out, hi_out = lo_out.cpu(), hi_out.cpu()
        lower, upper = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        lo_in, hi_in = torch.empty_like(lo_out), torch.empty_like(hi_out)
        with self._on_stream():
            ops = [self.dist.P2POp(self.dist.isend, lo_out, lower),
                   self.dist.P2POp(self.dist.isend, hi_out, upper),
                   self.dist.P2POp(self.dist.irecv, hi_in, upper),
                   self.dist.P2POp(self.dist.irecv, lo_in, lower)]
            works = self.dist.batch_isend_irecv(ops)
            if between is not None:
                between()
            for r in works:
                r.wait()
        if staged:
            lo_in, hi_in = lo_in.to(lat.device), hi_in.to(lat.device)
        lat.unpack_layers(0, lo_in)
        lat.unpack_layers(nloc - h, hi_in)

    def _host_staged(self) -> bool:
        """A CUDA lattice in a group whose backend moves host memory only
        (gloo): exchanges and gathers go through host copies."""
        dev = getattr(self.lat, "device", None)
        return dev is not None and dev.type == "cuda" and self.dist.get_backend() != "nccl"

    def hand_over_force(self):
        """Every rank's force and torque record gathered and added in rank
        order into this rank's body copy (all copies get the same bits)."""
        import torch
        mine = self.lat.body_force_to()
        staged = self._host_staged()
        if staged:
            mine = mine.cpu()
        parts = [torch.empty_like(mine) for _ in range(self.world)]
        with self._on_stream():
            self.dist.all_gather(parts, mine)
        all_parts = torch.stack(parts)
        self.lat.sum_body_force(all_parts.to(self.lat.device) if staged else all_parts)

    def step(self, n: int = 1):
        """n steps: exchange and step (two-phase: the interior layers beside
        the transfers), then the force hand-over."""
        self.launches = 0
        for _ in range(n):
            if self.two_phase:
                self.exchange(between=self.lat.step_interior)
                self.launches += self.lat.launches()
                self.lat.step_edges()
            else:
                self.exchange()
                self.lat.step(1)
            self.launches += self.lat.launches()
            if self.body:
                self.hand_over_force()
                self.launches += 1

    @property
    def last_force(self) -> np.ndarray:
        return self.lat.body_force_to().cpu().numpy()

    def close(self):
        self.lat.close()
