"""The host side of the GPU slab split (paper_1608_04658_gb300.slab.DistSlab)
on CPU ranks (gloo, world sizes 2 and 3): a stand-in lattice holds each
rank's layers of one known box in plain tensors, so that the exchange of edge
layers and the rank-ordered force hand-over run through DistSlab unchanged
without a GPU.  After one exchange every local layer must hold the box's layer
it stands for (halo layers wrapped around the periodic z axis), and every
rank's body copy the same force: the records added in rank order."""
import multiprocessing as mp
import os
import queue
import socket
import time

import numpy as np
import pytest

Q = 27


def _box(shape):
    nx, ny, nz = shape
    return np.arange(Q * nz * ny * nx, dtype=np.float32).reshape(Q, nz, ny, nx)


def _force(rank):
    """A rank's own force and torque record: values whose sum depends on the
    order of addition."""
    base = np.array([1.0, 1e-17, -3.0, 0.1, 0.2, 0.3])
    return base * (1 + rank) + np.array([1e16, 1.0, 0.0, 0.0, 0.0, 0.0]) * (-1) ** rank


class _Lattice:
    """Stand-in for paper_1608_04658_gb300.Lattice: the slab's layers (with
    halo layers set to NaN), layer copies and a force record."""

    def __init__(self, shape, layers, rank):
        import torch
        nx, ny, nz = shape
        self.shape = (nx, ny, layers.shape[1])
        self.state = torch.from_numpy(layers.copy())
        self.F = torch.from_numpy(_force(rank))
        self.summed = None
        self.device = torch.device("cpu")
        self.calls = []

    def pack_layers(self, z0, n):
        self.calls.append("pack")
        return self.state[:, z0:z0 + n].clone()

    def unpack_layers(self, z0, src):
        self.calls.append("unpack")
        self.state[:, z0:z0 + src.shape[1]] = src

    def step(self, n=1):
        self.calls.append("step")

    def step_interior(self):
        self.calls.append("interior")

    def step_edges(self):
        self.calls.append("edges")

    def launches(self):
        return 0

    def body_force_to(self, out=None):
        return self.F.clone()

    def sum_body_force(self, parts):
        assert parts.shape[1] == 6
        tot = parts[0].clone()
        for k in range(1, parts.shape[0]):
            tot = tot + parts[k]
        self.F = tot
        self.summed = parts.shape[0]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, shape, two_phase, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    from paper_1608_04658_gb300.slab import DistSlab, slab_rows
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        box = _box(shape)
        rows = slab_rows(shape[2], world, rank)
        layers = box[:, rows].copy()
        layers[:, :2] = np.nan
        layers[:, -2:] = np.nan
        ds = DistSlab(shape, 0.05, faces=(0,) * 6, geometry=object(), lattice=_Lattice(shape, layers, rank),
                      two_phase=two_phase)
        ds.step(1)
        q.put((rank, ds.lat.state.numpy(), rows, ds.last_force, ds.lat.summed, ds.launches, ds.lat.calls))
    finally:
        dist.destroy_process_group()


def _run(world, shape, two_phase):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, shape, two_phase, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    deadline = time.monotonic() + 240
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
    assert all(p.exitcode == 0 for p in procs)
    return [got[r] for r in range(world)]


@pytest.mark.parametrize("two_phase", [True, False])
@pytest.mark.parametrize("world,shape", [(2, (6, 4, 10)), (3, (6, 4, 13))])
def test_dist_slab_exchange_and_force_hand_over(world, shape, two_phase):
    """Two-phase: the interior layers' launch is enqueued once the transfers
    are (between the packs and the unpacks), the edges after the unpacks."""
    box = _box(shape)
    out = _run(world, shape, two_phase)
    expected = _force(0)
    for r in range(1, world):
        expected = expected + _force(r)
    if world >= 3:   # the order matters for these records: reversed, other bits
        rev = _force(world - 1)
        for r in reversed(range(world - 1)):
            rev = rev + _force(r)
        assert not np.array_equal(expected, rev)
    calls = ["pack", "pack", "interior", "unpack", "unpack", "edges"] if two_phase else \
        ["pack", "pack", "unpack", "unpack", "step"]
    for state, rows, force, summed, launches, seen in out:
        assert np.array_equal(state, box[:, rows])   # halo layers refilled, own layers kept
        assert np.array_equal(force, expected)
        assert summed == world and launches == 1
        assert seen == calls
