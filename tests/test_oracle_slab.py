"""The slab decomposition of the oracle along z on CPU ranks (gloo, world
sizes 2 and 3): owned populations bitwise equal to the undivided oracle, and
the force and torque summed over ranks equal to its sums up to the order of
addition.  A moving sphere straddles a cut, so boundary nodes, links and
refilled nodes lie on both sides of it."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import synth

NU = 0.05
FACES = (1, 1, 0, 0, 0, 0)  # walls in x, periodic y and z (the split axis)
R = 3.2
U = (0.35, -0.15, 0.0)
AMP = 1e-3


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, shape, X, steps, halo, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    from oracle.slab import decomposed_run
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = decomposed_run(shape, NU, FACES, X, R, U, synth.parity_fields(shape, 4), AMP, steps, halo=halo)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _decomposed(world, shape, X, steps, halo=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, shape, X, steps, halo, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return [got[r] for r in range(world)]


def _undivided(orc, shape, X, steps):
    o = orc.Oracle(shape, nu=NU, faces=FACES, body=orc.sphere_body(X, R, U=U, free=True, g=(0, 0, 0), mass=1e30))
    o.init_state(*synth.parity_fields(shape, 4), AMP)
    fm = []
    for _ in range(steps):
        o.step(1)
        fm.append(list(o.body.F) + list(o.body.M))
    return o, o.get_f(), np.array(fm)


@pytest.mark.parametrize("world,shape,X", [(2, (14, 12, 20), (6.3, 5.7, 10.375)),
                                           (3, (14, 12, 21), (6.3, 5.7, 13.875))])
def test_slab_ranks_reproduce_the_undivided_oracle(orc, world, shape, X):
    pytest.importorskip("torch.distributed")
    steps = 4
    o, f, fm = _undivided(orc, shape, X, steps)
    c = o.counters()
    assert c["refill"] > 0 and c["boundary"] > 0
    parts = _decomposed(world, shape, X, steps)
    cuts = [z0 for z0, _, _, _ in parts[1:]]
    solid = o.solid()
    # the body's links and refills reach both sides of a cut
    assert any(solid[z - 1].any() and solid[z].any() for z in cuts)
    for z0, z1, fr, forces in parts:
        assert np.array_equal(fr, f[:, z0:z1])
        # the same gathered sums on every rank
        assert np.array_equal(forces, parts[0][3])
    scale = np.abs(fm).max()
    assert np.abs(parts[0][3] - fm).max() <= 1e-13 * scale


def test_one_halo_layer_is_not_enough_once_a_halo_node_is_refilled(orc):
    """With one halo layer a refilled node in it averages fewer neighbours
    than in the undivided box, and an owned node pulls the difference."""
    pytest.importorskip("torch.distributed")
    shape, X, steps = (14, 12, 20), (6.3, 5.7, 10.375), 4
    _, f, _ = _undivided(orc, shape, X, steps)
    parts = _decomposed(2, shape, X, steps, halo=1)
    assert any(not np.array_equal(fr, f[:, z0:z1]) for z0, z1, fr, _ in parts)
