"""Slab decomposition of the FP64 oracle along z over CPU ranks
(torch.distributed, gloo): the CPU prototype of splitting one box over
several devices, one exchange step per time step (arXiv 1608.04658 gives no
parallel scheme; this follows its step, Sec. 2 streaming, Sec. 3 boundary and
refill, Sec. 4.1 momentum exchange).

TEST INFRASTRUCTURE ONLY: the tests are its only callers.

Each rank owns the z layers [z0, z1) of a box periodic in z and keeps two
halo layers on each side: a local oracle box of (z1 - z0) + 4 layers whose
own z faces are walls, which no owned node reads, placed as a slab of the
whole box (`Oracle.set_z_frame`) so that the sphere's geometry, nearest
image and centre wrap are computed from the same numbers as in the whole
box.  Before every step the ranks swap edge layers, all 27 post-collision
populations per node: the first two owned layers go to the rank below (its
upper halo) and the last two to the rank above (its lower halo).  One layer
feeds the pulls of the owned edge nodes, the Grad boundary's neighbour
velocities and finite-difference gradient, and the refill's neighbour
densities; the second makes the refill of a node in the first halo layer,
which owned nodes then pull from, the one of the undivided box.  A boundary
link belongs to the rank that owns its fluid node: each rank sums the force
and torque over its own layers, and the ranks gather the six sums and add
them in rank order, so every rank holds the same bits.  The body is
replicated: each rank hands the gathered force to its own copy before the
next step's Euler update, so all copies move alike.  Owned nodes end each
step bitwise equal to the undivided oracle while the body's velocity does
not depend on the force (a fixed velocity); a free body differs from the
undivided run by the order in which the link forces are added.  The sphere
is the supported body.
"""
from __future__ import annotations

import numpy as np

from . import FACE_PERIODIC, FACE_WALL, Oracle, lattice, sphere_body

HALO = 2


def slab_bounds(nz: int, world: int, rank: int) -> tuple[int, int]:
    """Owned z layers [z0, z1) of rank: consecutive, sizes differing by one."""
    return rank * nz // world, (rank + 1) * nz // world


def _exchange(f, world, rank, halo):
    """Fills the halo layers of the local state f (27, nloc, ny, nx) from the
    neighbouring ranks' edge layers (periodic ring of ranks)."""
    import torch
    import torch.distributed as dist
    nloc = f.shape[1]
    lo_out = torch.from_numpy(np.ascontiguousarray(f[:, halo:2 * halo]))
    hi_out = torch.from_numpy(np.ascontiguousarray(f[:, nloc - 2 * halo:nloc - halo]))
    if world == 1:
        lo_in, hi_in = hi_out, lo_out
    else:
        lower, upper = (rank - 1) % world, (rank + 1) % world
        lo_in, hi_in = torch.empty_like(lo_out), torch.empty_like(hi_out)
        reqs = [dist.isend(lo_out, lower, tag=0), dist.isend(hi_out, upper, tag=1),
                dist.irecv(hi_in, upper, tag=0), dist.irecv(lo_in, lower, tag=1)]
        for r in reqs:
            r.wait()
    f[:, :halo] = lo_in.numpy()
    f[:, nloc - halo:] = hi_in.numpy()


def _fixed_order_sum(v: np.ndarray, world: int) -> np.ndarray:
    """Sum of v over the ranks, added in rank order (the same bits on every
    rank, whatever the collective's own reduction order)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return v.copy()
    t = torch.from_numpy(np.ascontiguousarray(v))
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    tot = parts[0].clone()
    for p in parts[1:]:
        tot += p
    return tot.numpy()


def decomposed_run(shape, nu, faces, sphere, fields, amp, steps, world=None, rank=None, halo=HALO,
                   after_step=None):
    """Runs `steps` steps of a sphere problem on this rank's slab.

    shape (nx, ny, nz) with faces periodic in z; sphere = keyword arguments of
    `oracle.sphere_body`; fields = (rho, u, xi) of the whole box as synth
    builds them.  Returns (z0, z1, f, forces, body): f (27, z1 - z0, ny, nx)
    the owned post-collision populations, forces the per-step (F, M) summed
    over all ranks, shape (steps, 6), body the final (X, U).  halo: layers
    kept on each side (two are needed; one, for tests, leaves the refill of
    the first halo layer short of neighbours).  after_step(k), if given, is
    called after step k (tests use it to end a rank between steps)."""
    if world is None:
        import torch.distributed as dist
        world, rank = dist.get_world_size(), dist.get_rank()
    nx, ny, nz = shape
    if faces[4] != FACE_PERIODIC or faces[5] != FACE_PERIODIC:
        raise ValueError("the split axis z must be periodic")
    z0, z1 = slab_bounds(nz, world, rank)
    if z1 - z0 < halo:
        raise ValueError("slabs thinner than the halo")
    nloc = z1 - z0 + 2 * halo
    off = z0 - halo  # global z of local layer 0
    zidx = [(off + k) % nz for k in range(nloc)]
    local_faces = (faces[0], faces[1], faces[2], faces[3], FACE_WALL, FACE_WALL)
    o = Oracle((nx, ny, nloc), nu=nu, faces=local_faces, body=sphere_body(**sphere))
    o.set_z_frame(off, nz)
    rho, u, xi = fields
    o.init_state(rho[zidx], u[zidx], xi[:, zidx] if xi is not None else None, amp)
    o.set_owned_z(halo, nloc - halo)
    forces = []
    for k in range(steps):
        f = o.get_f()
        _exchange(f, world, rank, halo)
        o.set_f(f)
        o.step(1)
        b = o.body
        fm = _fixed_order_sum(np.array(list(b.F) + list(b.M)), world)
        for a in range(3):
            b.F[a], b.M[a] = fm[a], fm[3 + a]
        o.body = b  # the gathered force drives the next Euler update
        forces.append(fm)
        if after_step is not None:
            after_step(k)
    b = o.body
    return z0, z1, o.get_f()[:, halo:nloc - halo].copy(), np.array(forces), (list(b.X), list(b.U))


def _exchange_crossing(f, world, rank, up, dn):
    """The reduced exchange of a bodiless step: one halo layer per side,
    holding only the populations that cross into the slab (c_z = +1 into
    the lower halo from the rank below, c_z = -1 into the upper halo from the
    rank above); every other halo value is set to NaN, so a pull of one shows
    in the result.  Returns the bytes this rank sent."""
    import torch
    import torch.distributed as dist
    nloc = f.shape[1]
    lo_out = torch.from_numpy(np.ascontiguousarray(f[dn, 1]))          # my bottom row, c_z = -1
    hi_out = torch.from_numpy(np.ascontiguousarray(f[up, nloc - 2]))   # my top row, c_z = +1
    if world == 1:
        from_upper, from_lower = lo_out, hi_out
    else:
        lower, upper = (rank - 1) % world, (rank + 1) % world
        from_upper, from_lower = torch.empty_like(lo_out), torch.empty_like(hi_out)
        reqs = [dist.isend(lo_out, lower, tag=0), dist.isend(hi_out, upper, tag=1),
                dist.irecv(from_upper, upper, tag=0), dist.irecv(from_lower, lower, tag=1)]
        for r in reqs:
            r.wait()
    f[:, 0] = np.nan
    f[:, nloc - 1] = np.nan
    f[up, 0] = from_lower.numpy()
    f[dn, nloc - 1] = from_upper.numpy()
    return lo_out.numel() * 8 + hi_out.numel() * 8


def decomposed_run_crossing(shape, nu, faces, fields, amp, steps, world=None, rank=None):
    """A bodiless run on this rank's slab with the reduced exchange
    (_exchange_crossing): one halo layer of the nine crossing populations per
    side instead of two layers of all 27.  Returns (z0, z1, f, bytes sent per
    step): f the owned post-collision populations."""
    if world is None:
        import torch.distributed as dist
        world, rank = dist.get_world_size(), dist.get_rank()
    nx, ny, nz = shape
    if faces[4] != FACE_PERIODIC or faces[5] != FACE_PERIODIC:
        raise ValueError("the split axis z must be periodic")
    z0, z1 = slab_bounds(nz, world, rank)
    nloc = z1 - z0 + 2
    zidx = [(z0 - 1 + k) % nz for k in range(nloc)]
    local_faces = (faces[0], faces[1], faces[2], faces[3], FACE_WALL, FACE_WALL)
    o = Oracle((nx, ny, nloc), nu=nu, faces=local_faces)
    rho, u, xi = fields
    o.init_state(rho[zidx], u[zidx], xi[:, zidx] if xi is not None else None, amp)
    c, _ = lattice()
    up, dn = np.nonzero(c[:, 2] == 1)[0], np.nonzero(c[:, 2] == -1)[0]
    sent = 0
    for _ in range(steps):
        f = o.get_f()
        sent = _exchange_crossing(f, world, rank, up, dn)
        o.set_f(f)
        o.step(1)
    return z0, z1, o.get_f()[:, 1:nloc - 1].copy(), sent
