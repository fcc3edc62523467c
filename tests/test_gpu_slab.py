"""Slab decomposition on the GPU: one box split along z into slab lattices
(lbm_set_slab) that exchange two edge layers per side before every step
(lbm_pack_layers / lbm_unpack_layers, device copies in one process) and add
their own links' forces in slab order (lbm_set_body_force).  Own nodes must
end every step with the bits of the undivided lattice when the body's
velocity does not depend on the force, and differ from it by the order of
the force additions when it does.  A sphere straddles the cuts, so boundary
nodes, links and refilled nodes lie on both sides of them."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

NU = 0.05
FACES = (1, 1, 0, 0, 0, 0)  # walls in x, periodic y and z (the split axis)
AMP = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_04658_gb300 as lbm
    lbm.build()
    lbm.lib()


def _undivided(lbm, shape, storage, geom, steps, faces=FACES):
    lat = lbm.Lattice(shape, NU, storage=storage, faces=faces)
    if geom is not None:
        lat.set_geometry(geom)
    lat.init_state(*synth.parity_fields(shape, 4), AMP)
    forces = []
    for _ in range(steps):
        lat.step(1)
        if geom is not None:
            b = lat.body()
            forces.append(np.concatenate([b["F"], b["M"]]))
    return lat, np.array(forces)


def _split(lbm, shape, storage, geom, steps, parts, faces=FACES, local_z=None, two_phase=False):
    from paper_1608_04658_gb300.slab import SlabSet
    ss = SlabSet(shape, NU, parts, storage=storage, faces=faces, geometry=geom,
                 local_z=lbm.FACE_PERIODIC if local_z is None else local_z, two_phase=two_phase)
    rho, u, xi = synth.parity_fields(shape, 4)
    ss.init_state(rho, u, xi, AMP)
    forces = []
    for _ in range(steps):
        ss.step(1)
        if geom is not None:
            forces.append(ss.last_force.copy())
    return ss, np.array(forces)


def _straddles(lat, cuts):
    """The body's solid nodes lie on both sides of a cut."""
    solid = (lat.flags.cpu().numpy() & 1).astype(bool)
    zs = np.nonzero(solid.any(axis=(1, 2)))[0]
    return any(zs.min() < c <= zs.max() for c in cuts)


def _fluid(lat, ss):
    """Fluid nodes at the last step; the slabs' own layers carry the same
    solid marks as the whole box.  (Solid nodes keep a stale state that no
    fluid node reads, so only fluid nodes are compared.)"""
    from paper_1608_04658_gb300.slab import slab_bounds
    whole = (lat.flags.cpu().numpy() & 1).astype(bool)
    nz = lat.shape[2]
    for k, s in enumerate(ss.slabs):
        z0, z1 = slab_bounds(nz, ss.parts, k)
        own = (s.flags.cpu().numpy() & 1).astype(bool)[ss.halo:ss.halo + z1 - z0]
        assert np.array_equal(own, whole[z0:z1])
    return ~whole


@pytest.mark.parametrize("storage,local_z,two_phase", [("fp32", "periodic", False), ("fp16", "periodic", False),
                                                       ("fp32", "wall", False), ("fp32", "periodic", True),
                                                       ("fp16", "periodic", True)])
@pytest.mark.parametrize("parts,shape,X", [(2, (14, 12, 20), (6.3, 5.7, 9.1)),
                                           (3, (14, 12, 21), (6.3, 5.7, 13.4))])
def test_slabs_reproduce_the_undivided_lattice_bitwise(storage, local_z, two_phase, parts, shape, X):
    """Sphere carried across a cut at a fixed velocity (free, with a mass so
    large that the force leaves its velocity unchanged): the own layers of
    every slab equal the undivided lattice bit for bit, the slab-ordered sum
    of the forces equals the undivided force up to the order of addition.
    The slabs' own z faces (periodic or walls) are never read by own nodes.
    two_phase: each slab step as lbm_step_interior, the exchange,
    lbm_step_edges."""
    import paper_1608_04658_gb300 as lbm
    from paper_1608_04658_gb300.slab import slab_bounds
    geom = lbm.sphere(X, 3.2, U=(0.35, -0.15, 0.3), free=True, mass=1e30)
    steps = 5
    lat, fm = _undivided(lbm, shape, storage, geom, steps)
    assert lat.body()["n_boundary"] > 0
    ss, fs = _split(lbm, shape, storage, geom, steps, parts,
                    local_z=lbm.FACE_WALL if local_z == "wall" else lbm.FACE_PERIODIC, two_phase=two_phase)
    cuts = [slab_bounds(shape[2], parts, k)[0] for k in range(1, parts)]
    assert _straddles(lat, cuts)
    fluid = _fluid(lat, ss)
    f = lat.populations()[:, fluid]
    g = ss.populations()[:, fluid]
    assert np.array_equal(g, f)
    assert np.abs(fs - fm).max() <= 1e-12 * np.abs(fm).max()
    bodies = [s.body() for s in ss.slabs]
    for b in bodies:
        assert np.array_equal(b["X"], bodies[0]["X"]) and np.array_equal(b["U"], bodies[0]["U"])
    assert np.array_equal(bodies[0]["X"], lat.body()["X"])
    ss.close()


@pytest.mark.parametrize("two_phase", [False, True])
def test_slabs_move_a_free_sphere_with_the_summed_force(two_phase):
    """Free sedimenting sphere crossing the cut: every slab's copy of the body
    takes the Euler update of the slab-ordered force sum, so the copies agree
    bit for bit and differ from the undivided run only by rounding."""
    import paper_1608_04658_gb300 as lbm
    shape, steps = (14, 12, 20), 6
    geom = lbm.sphere((6.3, 5.7, 11.4), 3.2, U=(0.02, 0.0, -0.25), free=True, rho_ratio=1.5, g=(0.0, 0.0, -0.01))
    lat, fm = _undivided(lbm, shape, "fp32", geom, steps)
    ss, fs = _split(lbm, shape, "fp32", geom, steps, 2, two_phase=two_phase)
    bodies = [s.body() for s in ss.slabs]
    assert np.array_equal(bodies[0]["U"], bodies[1]["U"]) and np.array_equal(bodies[0]["X"], bodies[1]["X"])
    b0 = lat.body()
    assert np.abs(np.array(bodies[0]["U"]) - np.array(b0["U"])).max() < 1e-14
    assert np.abs(np.array(bodies[0]["X"]) - np.array(b0["X"])).max() < 1e-13
    # the body moved with the force, not only with gravity
    U_free = np.array([0.02, 0.0, -0.25]) + steps * (1 - 1 / 1.5) * np.array([0.0, 0.0, -0.01])
    assert np.abs(np.array(b0["U"]) - U_free).max() > 1e-4
    fluid = _fluid(lat, ss)
    assert np.abs(ss.populations()[:, fluid] - lat.populations()[:, fluid]).max() < 1e-6
    assert np.abs(fs - fm).max() <= 1e-9 * np.abs(fm).max()
    ss.close()


@pytest.mark.parametrize("storage,free,two_phase", [("fp32", 1, False), ("fp16", 1, False), ("fp32", 7, False),
                                                    ("fp32", 1, True), ("fp32", 7, True)])
def test_deforming_swimmer_over_slabs(storage, free, two_phase):
    """The triangulated swimmer (Sec. 4.3, deforming, refilled nodes every
    step; free along x in its head frame, or free in x, y and yaw in its
    centre-of-mass frame) across the cut of two slabs: each slab places the
    mesh in its own z frame.  The solid marks of the own layers equal the
    whole box's, the body copies agree bit for bit, and the state differs from
    the undivided run by rounding (the pose in the slab frame, the force
    summed in another order)."""
    import paper_1608_04658_gb300 as lbm
    shape, steps = (64, 32, 20), 6
    rest, tris = synth.swimmer_mesh(32.0, 40, 24)
    geom = lbm.swimmer((20.137 if free == 1 else 36.137, 16.371, 10.293), rest, tris, 32.0, 0.125, 32.0, 160.0,
                       free=free, mass=synth.swimmer_volume(32.0), U=(-0.004, 0.0, 0.0), t0=5.0)
    faces = (0,) * 6
    lat, fm = _undivided(lbm, shape, storage, geom, steps, faces=faces)
    ss, fs = _split(lbm, shape, storage, geom, steps, 2, faces=faces, two_phase=two_phase)
    assert _straddles(lat, [10])
    assert lat.body()["n_uncovered"] > 0
    fluid = _fluid(lat, ss)
    tol = {"fp32": 2e-6, "fp16": 2e-3}[storage]
    f, g = lat.populations()[:, fluid], ss.populations()[:, fluid]
    assert (np.abs(g - f) / np.abs(f)).max() <= tol
    bodies = [s.body() for s in ss.slabs]
    assert np.array_equal(bodies[0]["X"], bodies[1]["X"]) and np.array_equal(bodies[0]["U"], bodies[1]["U"])
    assert np.abs(np.array(bodies[0]["X"]) - np.array(lat.body()["X"])).max() < 1e-9
    assert np.abs(fs - fm).max() <= 1e-3 * np.abs(fm).max()
    ss.close()


@pytest.mark.parametrize("storage,two_phase,nz", [("fp32", False, 24), ("fp16", False, 24), ("fp32", True, 24),
                                                  ("fp16", True, 24), ("fp32", True, 8), ("fp32", True, 12)])
def test_bodiless_periodic_box_over_slabs(storage, two_phase, nz):
    """Periodic box without a body (rows of 64 nodes: the two-node kernel's
    all-periodic form in both the whole box and the slabs): 4 slabs, bitwise
    equal to the undivided box; with the two-phase step also slabs of 2 and
    3 own layers (no interior layer, one)."""
    import paper_1608_04658_gb300 as lbm
    shape = (64, 10, nz)
    lat, _ = _undivided(lbm, shape, storage, None, 6, faces=(0,) * 6)
    ss, _ = _split(lbm, shape, storage, None, 6, 4, faces=(0,) * 6, two_phase=two_phase)
    assert np.array_equal(ss.populations(), lat.populations())
    ss.close()


def test_slab_arguments_are_checked():
    import paper_1608_04658_gb300 as lbm
    for zf in ((0, 0, 0, 0, 3, 3), (0, 0, 0, 0, 2, 2), (0, 0, 0, 0, 1, 3)):
        lat = lbm.Lattice((8, 8, 8), NU, faces=zf)
        with pytest.raises(lbm.LbmError):
            lat.set_slab(-2, 12, 2, 6)  # z faces: both walls or both periodic
    lat = lbm.Lattice((8, 8, 8), NU, faces=(0, 0, 0, 0, 1, 1))
    with pytest.raises(lbm.LbmError):
        lat.set_slab(-2, 12, 6, 2)  # empty own range
    lat.set_slab(-2, 12, 2, 6)
    with pytest.raises(lbm.LbmError):
        # the next image of a sphere this large (12 layers away) reaches the
        # layers that own nodes read, (12 - 2R) / 2 <= 3
        lat.set_geometry(lbm.sphere((4.0, 4.0, 5.0), 3.0))
    lat.set_geometry(lbm.sphere((4.0, 4.0, 5.0), 2.9))
    with pytest.raises(lbm.LbmError):
        lat.pack_layers(7, 2)
    # the two-phase step: only on a slab, and no plain step while one is open
    whole = lbm.Lattice((8, 8, 8), NU, faces=(0,) * 6)
    whole.init_state(*synth.uniform_fields((8, 8, 8)))
    with pytest.raises(lbm.LbmError):
        whole.step_interior()
    lat.init_state(*synth.uniform_fields((8, 8, 8)))
    lat.set_launch_order("split")
    lat.step_interior()
    with pytest.raises(lbm.LbmError):
        lat.step(1)
    with pytest.raises(lbm.LbmError):
        lat.step_interior()
    lat.step_edges()
    lat.step(1)


def _dist_rank(rank, world, port, shape, storage, steps, q):
    """One rank of a gloo group on this GPU: its slab's own fluid layers and
    the summed force after the steps (the group moves host memory only, so
    the ranks' kernels never wait on one another)."""
    import os
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import paper_1608_04658_gb300 as lbm
    from paper_1608_04658_gb300.slab import DistSlab
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        geom = lbm.sphere((6.3, 5.7, 9.1), 3.2, U=(0.35, -0.15, 0.3), free=True, mass=1e30)
        ds = DistSlab(shape, NU, storage=storage, faces=FACES, geometry=geom, device="cuda:0")
        rho, u, xi = synth.parity_fields(shape, 4)
        ds.init_state(rho, u, xi, AMP)
        ds.step(steps)
        f = ds.lat.populations()[:, ds.halo:ds.halo + ds.z1 - ds.z0]
        solid = (ds.lat.flags.cpu().numpy() & 1).astype(bool)[ds.halo:ds.halo + ds.z1 - ds.z0]
        q.put((rank, f, solid, ds.last_force, ds.z0, ds.z1))
        ds.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_dist_slab_ranks_reproduce_the_undivided_lattice(storage):
    """DistSlab end to end on the GPU: two ranks (processes) of a gloo group,
    each with its slab on this GPU and the two-phase step, the edge layers and
    force records staged through host memory.  Own fluid nodes equal the
    undivided lattice bit for bit; the summed force equals its force up to
    the order of addition."""
    import multiprocessing as mp
    import queue
    import socket
    import time

    import paper_1608_04658_gb300 as lbm
    shape, steps, world = (14, 12, 20), 5, 2
    geom = lbm.sphere((6.3, 5.7, 9.1), 3.2, U=(0.35, -0.15, 0.3), free=True, mass=1e30)
    lat, fm = _undivided(lbm, shape, storage, geom, steps)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_dist_rank, args=(r, world, port, shape, storage, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, deadline = {}, time.monotonic() + 240
    try:
        while len(got) < world:
            try:
                out = q.get(timeout=2)
                got[out[0]] = out[1:]
            except queue.Empty:
                dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
                assert not dead and time.monotonic() < deadline, f"ranks failed: exit codes {dead}"
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    whole = lat.populations()
    wsolid = (lat.flags.cpu().numpy() & 1).astype(bool)
    for r in range(world):
        f, solid, force, z0, z1 = got[r]
        assert np.array_equal(solid, wsolid[z0:z1])
        fluid = ~solid
        assert np.array_equal(f[:, fluid], whole[:, z0:z1][:, fluid])
        assert np.abs(force - fm[-1]).max() <= 1e-12 * np.abs(fm[-1]).max()
    assert np.array_equal(got[0][2], got[1][2])
