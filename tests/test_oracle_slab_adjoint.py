"""The adjoint of the slab decomposition on CPU ranks (gloo, world sizes 1, 2
and 3; oracle/slab_adjoint.py): the forward halo exchange run in reverse
gives, on every rank's owned layers, the gradient of J = lambda_T . f_T with
respect to the initial state that the undivided autograd tape gives, and the
ranks' J add up to the undivided J.  A wrong direction of the reversed
exchange, or dropping it, fails by O(1) of the gradient at the cuts."""
import multiprocessing as mp
import os
import queue
import socket
import time

import numpy as np
import pytest
import torch

import synth

BETA = 0.8
STEPS = 4


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs(shape):
    rho, u, xi = synth.parity_fields(shape, 6)
    from oracle import tape
    f0 = (tape.equilibrium(torch.tensor(rho), torch.tensor(u).permute(3, 0, 1, 2)).numpy()
          + 1e-3 * tape.W_NP[:, None, None, None] * xi)
    lam = np.random.default_rng(6).normal(size=f0.shape)
    return f0, lam


def _rank(rank, world, port, shape, faces, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    from oracle.slab_adjoint import decomposed_gradient
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f0, lam = _inputs(shape)
        q.put((rank, decomposed_gradient(shape, BETA, f0, lam, STEPS, world, rank, faces=faces)))
    finally:
        dist.destroy_process_group()


def _decomposed(world, shape, faces):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, shape, faces, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    deadline = time.monotonic() + 300
    try:
        while len(got) < world:
            try:
                rank, out = q.get(timeout=2)
                got[rank] = out
            except queue.Empty:
                dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
                assert not dead and time.monotonic() < deadline, f"ranks failed: exit codes {dead}"
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert all(p.exitcode == 0 for p in procs)
    return [got[r] for r in range(world)]


def _undivided(shape, faces):
    from oracle import tape
    f0, lam = _inputs(shape)
    box = tape.Box(shape, faces=faces)
    x = torch.tensor(f0, requires_grad=True)
    f = x
    for _ in range(STEPS):
        f = box.step(f, BETA)
    J = (torch.tensor(lam) * f).sum()
    J.backward()
    return float(J.detach()), x.grad.numpy()


@pytest.mark.parametrize("world,shape,faces", [(1, (8, 6, 7), (0,) * 6), (2, (8, 6, 10), (0,) * 6),
                                               (3, (8, 6, 11), (1, 1, 0, 0, 0, 0))])
def test_slab_adjoint_reproduces_the_undivided_gradient(world, shape, faces):
    from oracle.slab_adjoint import slab_bounds
    J_ref, g_ref = _undivided(shape, faces)
    parts = _decomposed(world, shape, faces)
    J = sum(p[0] for p in parts)
    g = np.concatenate([p[1] for p in parts], axis=1)
    assert [p[1].shape[1] for p in parts] == [slab_bounds(shape[2], world, r)[1] - slab_bounds(shape[2], world, r)[0]
                                             for r in range(world)]
    assert J == pytest.approx(J_ref, rel=1e-13)
    assert np.abs(g - g_ref).max() <= 1e-12 * np.abs(g_ref).max()
