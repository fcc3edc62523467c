"""The adjoint of the slab decomposition along z on CPU ranks: the halo
exchange of every forward step, run in reverse.

TEST INFRASTRUCTURE ONLY.  Only the test suite may import this module.  It
splits the differentiable restatement of the bodiless step (``tape.Box``) over
``torch.distributed`` ranks (gloo) like ``slab.py`` splits the C oracle: each
rank owns consecutive z layers of a box periodic in z and holds one halo layer
on each side (a bodiless pull reaches one layer).

Forward, per step: the halo layers are filled from the neighbours' edge
layers (a copy), then the local slab takes the step; only the owned layers'
results are kept.  The objective is J = sum lambda_T . f_T over the owned
layers of every rank.

Reverse, per step from the last: each rank forms the vector-Jacobian product
of its slab's step with its owned adjoint lambda^{t+1} (zero on the halo
rows), which yields adjoint contributions on its owned layers and on its two
halo layers; the halo contributions belong to the neighbours' edge layers
that the forward exchange copied there, so they are sent back and added to
those layers (the adjoint of a copy is an accumulation).  The owned adjoint
after the first step is dJ/df_0 on the rank's layers.
"""
from __future__ import annotations

import numpy as np
import torch

from .tape import Box

HALO = 1


def slab_bounds(nz: int, world: int, rank: int) -> tuple[int, int]:
    """Owned z layers [z0, z1) of rank: consecutive, sizes differing by one."""
    return rank * nz // world, (rank + 1) * nz // world


def _ring_exchange(lo_out: torch.Tensor, hi_out: torch.Tensor, world: int, rank: int):
    """Sends lo_out to the rank below and hi_out to the rank above (a periodic
    ring); returns what arrives from above and from below."""
    import torch.distributed as dist
    if world == 1:
        return lo_out.clone(), hi_out.clone()
    lower, upper = (rank - 1) % world, (rank + 1) % world
    from_upper, from_lower = torch.empty_like(lo_out), torch.empty_like(hi_out)
    reqs = [dist.isend(lo_out.contiguous(), lower, tag=0), dist.isend(hi_out.contiguous(), upper, tag=1),
            dist.irecv(from_upper, upper, tag=0), dist.irecv(from_lower, lower, tag=1)]
    for r in reqs:
        r.wait()
    return from_upper, from_lower


def _fill_halo(f: torch.Tensor, world: int, rank: int) -> torch.Tensor:
    """Local state (27, nloc + 2, ny, nx) with its halo rows from the
    neighbours' edge layers."""
    from_upper, from_lower = _ring_exchange(f[:, HALO:2 * HALO], f[:, -2 * HALO:-HALO], world, rank)
    out = f.clone()
    out[:, :HALO] = from_lower
    out[:, -HALO:] = from_upper
    return out


def decomposed_gradient(shape, beta, f0: np.ndarray, lam_T: np.ndarray, steps: int, world: int, rank: int,
                        faces=(0, 0, 0, 0, 0, 0)):
    """(J of this rank's layers, dJ/df_0 on this rank's owned layers) for J =
    sum lambda_T . f_T after `steps` steps, the box split along z over the
    ranks.  faces: x and y faces as tape.Box takes them; z must be periodic.
    f0, lam_T: whole-box arrays (27, nz, ny, nx)."""
    assert faces[4] == 0 and faces[5] == 0, "the split axis must be periodic"
    nx, ny, nz = shape
    z0, z1 = slab_bounds(nz, world, rank)
    nloc = z1 - z0
    # the slab with one halo row each side; the local box is periodic in z
    # (the halo rows make the owned layers' pulls those of the whole box)
    box = Box((nx, ny, nloc + 2 * HALO), faces=tuple(faces[:4]) + (0, 0))
    idx = [(z - HALO) % nz for z in range(z0, z1 + 2 * HALO)]
    f = torch.tensor(np.ascontiguousarray(f0[:, idx]), dtype=torch.float64)
    states = []
    for _ in range(steps):
        f = _fill_halo(f, world, rank)
        states.append(f)
        f = box.step(f, beta).detach()
    lam = torch.zeros_like(f)
    lam[:, HALO:-HALO] = torch.tensor(np.ascontiguousarray(lam_T[:, z0:z1]), dtype=torch.float64)
    J = float((lam[:, HALO:-HALO] * f[:, HALO:-HALO]).sum())
    for t in range(steps - 1, -1, -1):
        x = states[t].clone().requires_grad_(True)
        (g,) = torch.autograd.grad(box.step(x, beta), x, grad_outputs=lam)
        # the halo rows' adjoint goes back to the layers they were copied from
        from_upper, from_lower = _ring_exchange(g[:, :HALO], g[:, -HALO:], world, rank)
        lam = torch.zeros_like(g)
        lam[:, HALO:-HALO] = g[:, HALO:-HALO]
        lam[:, -2 * HALO:-HALO] += from_upper
        lam[:, HALO:2 * HALO] += from_lower
    return J, lam[:, HALO:-HALO].numpy()
