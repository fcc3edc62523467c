"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank runs
an independent replica and rank 0 reports the slowest rank's time."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.dist_barrier(w)
    q.put((rank, bench.dist_max(1.5 + rank, w)))
    dist.destroy_process_group()


def test_dist_max_over_two_gloo_ranks():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 2.5), (1, 2.5)]


def test_ncu_traffic_only_for_the_profiled_workload():
    """The committed DRAM traffic per bulk launch belongs to one workload; any
    other box (another size, the Taylor-Green box) reports none."""
    import bench
    sphere = bench.workload(None, "sphere")["name"]
    for other in (bench.workload("384", "tgv")["name"], bench.workload("128,128,64", "sphere")["name"]):
        assert bench.ncu_traffic("fp32", other) is None
        assert bench.ncu_traffic("fp16", other) is None
    for st in ("fp32", "fp16"):
        v = bench.ncu_traffic(st, sphere)
        # None once the kernel sources changed after the capture
        assert v is None or v > 0.5 * bench.BYTES_PER_NODE[st] * 128 * 128 * 256


def test_all_cores_oracle_baseline_runs_replicas(orc):
    """The all-cores CPU baseline starts independent oracle replicas in
    spawned processes and reports their aggregate node updates."""
    import bench
    wl = bench.workload("16", "tgv")
    r = bench.cpu_baseline_all_cores(wl, nsteps=2, procs=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["unit"] == "GLUPS"
    assert r["value"] > 0 and r["seconds"] > 0
    assert "2 independent replicas" in r["sample"]
