"""The slab decomposition of the oracle along z on CPU ranks (gloo, world
sizes 2 and 3): owned populations bitwise equal to the undivided oracle, and
the force and torque summed over ranks equal to its sums up to the order of
addition.  A moving sphere straddles a cut, so boundary nodes, links and
refilled nodes lie on both sides of it."""
import multiprocessing as mp
import os
import queue
import socket
import time

import numpy as np
import pytest

import synth

NU = 0.05
FACES = (1, 1, 0, 0, 0, 0)  # walls in x, periodic y and z (the split axis)
AMP = 1e-3


def _carried(X):
    """Sphere carried at a fixed velocity (free, with a mass so large that
    the force leaves its velocity unchanged), moving across z layers."""
    return dict(X=X, R=3.2, U=(0.35, -0.15, 0.3), free=True, g=(0.0, 0.0, 0.0), mass=1e30)


def _sedimenting(X):
    """Free sphere, 1.5 times the fluid density, falling along -z."""
    return dict(X=X, R=3.2, U=(0.02, 0.0, -0.25), free=True, rho_ratio=1.5, g=(0.0, 0.0, -0.01))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, shape, sphere, steps, halo, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    from oracle.slab import decomposed_run
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = decomposed_run(shape, NU, FACES, sphere, synth.parity_fields(shape, 4), AMP, steps, halo=halo)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _decomposed(world, shape, sphere, steps, halo=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, shape, sphere, steps, halo, q)) for r in range(world)]
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


def _undivided(orc, shape, sphere, steps):
    o = orc.Oracle(shape, nu=NU, faces=FACES, body=orc.sphere_body(**sphere))
    o.init_state(*synth.parity_fields(shape, 4), AMP)
    fm = []
    cut_solid = []
    for _ in range(steps):
        o.step(1)
        fm.append(list(o.body.F) + list(o.body.M))
        cut_solid.append(o.solid())
    return o, o.get_f(), np.array(fm), cut_solid


def _straddles(solids, cuts):
    """The body has solid nodes on both sides of some cut at some step, so
    its links and refills reach both ranks there."""
    return any(s[z - 1].any() and s[z].any() for s in solids for z in cuts)


@pytest.mark.parametrize("world,shape,X", [(2, (14, 12, 20), (6.3, 5.7, 8.9)),
                                           (3, (14, 12, 21), (6.3, 5.7, 12.6))])
def test_slab_ranks_reproduce_the_undivided_oracle(orc, world, shape, X):
    """Sphere carried across the cut at a fixed velocity: owned populations
    bitwise equal, force and torque equal up to the order of addition."""
    pytest.importorskip("torch.distributed")
    steps = 5
    sphere = _carried(X)
    o, f, fm, solids = _undivided(orc, shape, sphere, steps)
    c = o.counters()
    assert c["refill"] > 0 and c["boundary"] > 0
    parts = _decomposed(world, shape, sphere, steps)
    assert _straddles(solids, [p[0] for p in parts[1:]])
    for z0, z1, fr, forces, body in parts:
        assert np.array_equal(fr, f[:, z0:z1])
        # the same gathered sums and the same body on every rank
        assert np.array_equal(forces, parts[0][3])
        assert body == parts[0][4]
    assert np.abs(parts[0][3] - fm).max() <= 1e-13 * np.abs(fm).max()
    assert parts[0][4] == (list(o.body.X), list(o.body.U))


def test_slab_ranks_move_a_free_sphere_with_the_gathered_force(orc):
    """Free sedimenting sphere crossing the cut: every rank's copy of the body
    takes the Euler update of the gathered force, so all copies agree bit for
    bit, and the run differs from the undivided oracle only through the order
    in which the link forces are added."""
    pytest.importorskip("torch.distributed")
    shape, steps = (14, 12, 20), 6
    sphere = _sedimenting((6.3, 5.7, 11.4))
    o, f, fm, solids = _undivided(orc, shape, sphere, steps)
    parts = _decomposed(2, shape, sphere, steps)
    assert _straddles(solids, [parts[1][0]])
    X, U = parts[0][4]
    assert all(p[4] == parts[0][4] for p in parts)
    assert np.abs(np.array(U) - np.array(o.body.U)).max() < 1e-15
    assert np.abs(np.array(X) - np.array(o.body.X)).max() < 1e-13
    # the body really moved with the force: U differs from its force-free value
    U_free = np.array(sphere["U"]) + steps * (1 - 1 / 1.5) * np.array(sphere["g"])
    assert np.abs(np.array(U) - U_free).max() > 1e-4
    for z0, z1, fr, _, _ in parts:
        assert np.abs(fr - f[:, z0:z1]).max() < 1e-13
    assert np.abs(parts[0][3] - fm).max() <= 1e-12 * np.abs(fm).max()


def test_one_halo_layer_is_not_enough_once_a_halo_node_is_refilled(orc):
    """With one halo layer a refilled node in it averages fewer neighbours
    than in the undivided box, and an owned node pulls the difference."""
    pytest.importorskip("torch.distributed")
    shape, steps = (14, 12, 20), 5
    sphere = _carried((6.3, 5.7, 8.9))
    _, f, _, _ = _undivided(orc, shape, sphere, steps)
    parts = _decomposed(2, shape, sphere, steps, halo=1)
    assert any(not np.array_equal(fr, f[:, z0:z1]) for z0, z1, fr, _, _ in parts)


def _rank_that_dies(rank, port, shape, q):
    """Rank 1 ends its process after step 2, between steps; rank 0 reports
    what its next exchange raises."""
    import datetime

    os.environ.update(RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    from oracle.slab import decomposed_run
    dist.init_process_group("gloo", rank=rank, world_size=2, timeout=datetime.timedelta(seconds=20))

    def die(k):
        if rank == 1 and k == 2:
            os._exit(3)

    try:
        decomposed_run(shape, NU, FACES, _carried((6.3, 5.7, 8.9)), synth.parity_fields(shape, 4), AMP, 6,
                       after_step=die)
        q.put((rank, "finished"))
    except RuntimeError as e:
        q.put((rank, "error: " + str(e)[:200]))


def test_a_rank_that_leaves_makes_its_peer_fail_not_hang(orc):
    """A rank that exits between steps: its peer's next halo exchange ends
    with an error (closed connection or the process group's timeout) instead
    of waiting forever; the failure is made on the host, no device involved."""
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_that_dies, args=(r, port, (14, 12, 20), q)) for r in range(2)]
    for p in procs:
        p.start()
    rank, msg = q.get(timeout=120)
    assert rank == 0 and msg.startswith("error"), msg
    for p in procs:
        p.join(timeout=60)
    assert procs[1].exitcode == 3
    assert procs[0].exitcode == 0


def test_whole_box_frame_changes_nothing(orc):
    """The slab frame of the whole box (origin 0, period nz) gives the same bits
    as no frame, for a free sphere that crosses the periodic seam in z."""
    shape = (16, 14, 18)

    def run(frame):
        o = orc.Oracle(shape, nu=0.02, faces=FACES, body=orc.sphere_body((7.3, 6.6, 17.1), 3.1, U=(0.05, -0.02, 0.3),
                                                                          free=True, g=(0, 0, -1e-3)))
        if frame:
            o.set_z_frame(0, shape[2])
        o.init_state(*synth.parity_fields(shape, 2), AMP)
        o.step(6)
        return o.get_f(), list(o.body.F), list(o.body.X)

    a, b = run(False), run(True)
    assert a[2][2] < 3.0  # the centre wrapped through z = 0
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and a[2] == b[2]


def _crossing_rank(rank, world, port, shape, steps, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    from oracle.slab import decomposed_run_crossing
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, decomposed_run_crossing(shape, NU, FACES, synth.parity_fields(shape, 5), AMP, steps)))
    finally:
        dist.destroy_process_group()


def _crossing(world, shape, steps):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_crossing_rank, args=(r, world, port, shape, steps, q)) for r in range(world)]
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


@pytest.mark.parametrize("world,shape", [(2, (14, 12, 20)), (3, (14, 12, 21))])
def test_bodiless_slabs_need_only_the_crossing_populations(orc, world, shape):
    """Without a body near a cut one halo layer of the nine populations that
    cross it (c_z = +-1) is enough: every other halo value is NaN, and the
    owned populations still equal the undivided oracle's bit for bit after 6
    steps, for a sixth of the bytes of the two-layer exchange of all 27."""
    steps = 6
    o = orc.Oracle(shape, nu=NU, faces=FACES)
    o.init_state(*synth.parity_fields(shape, 5), AMP)
    o.step(steps)
    ref = o.get_f()
    parts = _crossing(world, shape, steps)
    for z0, z1, f, sent in parts:
        assert np.isfinite(f).all()
        assert np.array_equal(f, ref[:, z0:z1])
        nx, ny = shape[0], shape[1]
        assert sent == 2 * 9 * nx * ny * 8 and 6 * sent == 2 * 2 * 27 * nx * ny * 8
