"""Slab decomposition of the FP64 oracle along z over CPU ranks
(torch.distributed, gloo): the CPU prototype of splitting one box over
several devices, one exchange step per time step (arXiv 1608.04658 gives no
parallel scheme; this follows its step, Sec. 2 streaming, Sec. 3 boundary and
refill, Sec. 4.1 momentum exchange).

TEST INFRASTRUCTURE ONLY: the tests are its only callers.

Each rank owns the z layers [z0, z1) of a box periodic in z and keeps two
halo layers on each side: a local oracle box of (z1 - z0) + 4 layers whose
own z faces are walls, which no owned node reads.  Before every step the
ranks swap edge layers, all 27 post-collision populations per node: the
first two owned layers go to the rank below (its upper halo) and the last two
to the rank above (its lower halo).  One layer feeds the pulls of the owned
edge nodes, the Grad boundary's neighbour velocities and finite-difference
gradient, and the refill's neighbour densities; the second makes the refill
of a node in the first halo layer, which owned nodes then pull from, the one
of the undivided box.  Owned nodes therefore end each step bitwise equal to
the single-rank oracle.  The body is replicated on every rank; its force and
torque are the owned-layer sums gathered from all ranks and added in rank
order, the same on every rank.

Supported body: a sphere moving with a fixed velocity in x and y (free with a
mass large enough that the force leaves its velocity unchanged), whose centre
z is a dyadic number: it is shifted by whole layers into each local frame,
which is exact only then, and a free body's Euler update would need the
gathered force inside the oracle's own step.
"""
from __future__ import annotations

import numpy as np

from . import FACE_PERIODIC, FACE_WALL, Oracle, sphere_body

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


def decomposed_run(shape, nu, faces, X, R, U, fields, amp, steps, world=None, rank=None, halo=HALO):
    """Runs `steps` steps of the sphere problem on this rank's slab.

    shape (nx, ny, nz) with faces periodic in z; X, R, U the sphere (U[2] = 0,
    X[2] dyadic); fields = (rho, u, xi) of the whole box as synth builds them.
    Returns (z0, z1, f, forces): f (27, z1 - z0, ny, nx) the owned
    post-collision populations, forces the per-step (F, M) summed over all
    ranks, shape (steps, 6).  halo: layers kept on each side (two are needed; one, for
    tests, leaves the refill of the first halo layer short of neighbours)."""
    if world is None:
        import torch.distributed as dist
        world, rank = dist.get_world_size(), dist.get_rank()
    nx, ny, nz = shape
    if faces[4] != FACE_PERIODIC or faces[5] != FACE_PERIODIC:
        raise ValueError("the split axis z must be periodic")
    if U[2] != 0.0 or float(X[2]) * 1024.0 != int(float(X[2]) * 1024.0):
        raise ValueError("the sphere must move in x and y only and have a dyadic centre z")
    z0, z1 = slab_bounds(nz, world, rank)
    if z1 - z0 < halo:
        raise ValueError("slabs thinner than the halo")
    nloc = z1 - z0 + 2 * halo
    off = z0 - halo  # global z of local layer 0
    zidx = [(off + k) % nz for k in range(nloc)]
    # the image of the centre nearest the slab, in the local frame
    zc = 0.5 * (z0 + z1 - 1)
    xz = float(X[2]) + nz * round((zc - float(X[2])) / nz) - off
    body = sphere_body((X[0], X[1], xz), R, U=U, free=True, g=(0.0, 0.0, 0.0), mass=1e30)
    local_faces = (faces[0], faces[1], faces[2], faces[3], FACE_WALL, FACE_WALL)
    o = Oracle((nx, ny, nloc), nu=nu, faces=local_faces, body=body)
    rho, u, xi = fields
    o.init_state(rho[zidx], u[zidx], xi[:, zidx] if xi is not None else None, amp)
    o.set_owned_z(halo, nloc - halo)
    forces = []
    for _ in range(steps):
        f = o.get_f()
        _exchange(f, world, rank, halo)
        o.set_f(f)
        o.step(1)
        b = o.body
        forces.append(_fixed_order_sum(np.array(list(b.F) + list(b.M)), world))
    return z0, z1, o.get_f()[:, halo:nloc - halo].copy(), np.array(forces)
