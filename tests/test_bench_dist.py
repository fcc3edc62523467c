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


def _bench(args, env_extra):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", *args], cwd=root, env=env, capture_output=True, text=True,
                          timeout=600)


def test_reference_arm_prints_one_line_on_rank_zero_only(orc):
    """The reference arm (the FP64 oracle on host cores): rank 0 prints one
    JSON line with the contract's keys; another rank prints nothing and exits
    0 without work."""
    import json
    r1 = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    # the sphere box keeps this CPU test short; the swimmer's sample is checked below
    r0 = _bench(["--impl", "reference", "--workload", "sphere", "--steps", "2", "--warmup", "1"],
                {"RANK": "0", "WORLD_SIZE": "1"})
    assert r0.returncode == 0, r0.stderr[-2000:]
    lines = [s for s in r0.stdout.splitlines() if s.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GLUPS"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "sedimenting_sphere_128x128x256_D16"
    assert d["steps"] == 2 and d["warmup"] == 1 and 1 <= d["config"]["processes"] <= 2


def test_headline_workload_and_its_oracle_sample():
    """The main line measures the largest configuration, the swimmer in
    768x256x256; the oracle's sample of it is a periodic crop holding the whole
    body with the same mesh, kinematics and viscosity."""
    import bench
    args = bench.parse_args([])
    assert args.workload == "swimmer" and args.second_workload == "sphere"
    wl = bench.workload(None, "swimmer")
    assert wl["shape"] == (768, 256, 256)
    smp, n, desc = bench.cpu_sample(wl)
    assert smp["shape"] == (176, 64, 32) and n == 1 and "crop" in desc
    for k in ("L", "period", "amp", "wavelength", "nu", "mass", "faces"):
        assert smp[k] == wl[k], k
    assert (smp["rest"] == wl["rest"]).all() and (smp["tris"] == wl["tris"]).all()
    # the body (head at X, length L along +x, tail amplitude 0.125 L, half
    # width 0.04 L, half height 0.08 L) stays two nodes clear of every face
    X, L = smp["X"], smp["L"]
    nx, ny, nz = smp["shape"]
    assert X[0] - 2 > 0 and X[0] + L + 2 < nx
    assert X[1] - 0.165 * L - 2 > 0 and X[1] + 0.165 * L + 2 < ny
    assert X[2] - 0.08 * L - 2 > 0 and X[2] + 0.08 * L + 2 < nz


def test_clock_sampler_reads_the_timed_window_and_its_throttle_reasons(tmp_path):
    """The bench's clock record: samples inside the timed windows (with a
    0.15 s margin) give the median SM clock, the maximum clock and every
    throttle reason reported Active there; malformed lines are skipped."""
    import datetime

    import bench

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    t0 = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def row(dt, mhz, hw="Not Active", cap="Not Active"):
        ts = (t0 + datetime.timedelta(seconds=dt)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, 900.5, 0x0, {hw}, Not Active, Not Active, {cap}\n"

    path = tmp_path / "clocks.csv"
    path.write_text(row(0.0, 1200, hw="Active") + "garbage line\n" + row(1.0, 2070) + row(1.1, 2040, cap="Active")
                    + row(1.2, 2070) + row(3.0, 900, hw="Active"))
    s = bench.ClockSampler(0)
    s.path, s.proc, s.fh = str(path), _Proc(), open(os.devnull, "w")
    base = t0.timestamp()
    s.mark(base + 0.95, base + 1.25)
    c = s.stop()
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3,
                 "in_timed_region": True}
    # no window marked: every sample counts, and the slowdowns outside show up
    s = bench.ClockSampler(0)
    s.path, s.proc, s.fh = str(path), _Proc(), open(os.devnull, "w")
    c = s.stop()
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"] and c["samples"] == 5 and not c["in_timed_region"]


def test_hbm_peak_comes_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    import json

    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6680.2, "bf16_tflops": 1930.3}))
    assert bench.measured_hbm_peak() == (6680.2, "measured (hbm_gbs)")
    (tmp_path / "MEASURED_PEAKS.json").write_text("not json")
    assert bench.measured_hbm_peak()[1] == "fallback"


def test_refined_node_counts_match_the_levels_masks():
    """The node updates the refinement lines count per coarse step equal the
    nodes the refined step updates, counted from the masks of what each level
    computes (coarse: all but the block's inside; fine: the interior, twice),
    for a closed block and for one spanning the periodic z axis."""
    import numpy as np

    import bench
    for shape, lo, hi in (((64, 32, 16), (16, 8, 2), (47, 23, 13)), ((64, 48, 4), (8, 8, 0), (55, 39, 4))):
        full = [l == 0 and h == n for l, h, n in zip(lo, hi, shape)]
        inside = np.ones(shape[::-1], dtype=bool)
        sl = [slice(None) if f else slice(l + 1, h) for l, h, f in zip(lo, hi, full)]
        mask = np.zeros(shape[::-1], dtype=bool)
        mask[sl[2], sl[1], sl[0]] = True
        coarse = int((inside & ~mask).sum())
        fshape = [2 * n if f else 2 * (h - l) + 2 for l, h, n, f in zip(lo, hi, shape, full)]
        fmask = np.zeros(fshape[::-1], dtype=bool)
        fsl = [slice(None) if f else slice(1, 2 * (h - l)) for l, h, f in zip(lo, hi, full)]
        fmask[fsl[2], fsl[1], fsl[0]] = True
        fine = int(fmask.sum())
        assert bench.refined_counts(shape, lo, hi) == (coarse, fine, coarse + 2 * fine)


def test_refined_cpu_baseline_line_is_well_formed():
    """The refinement lines' oracle baseline runs the refined oracle on its
    bounded crops (closed block; spanning block with the airfoil) and reports
    node updates per second in the GPU line's unit."""
    import bench
    import synth
    for wl, body in ((synth.refined_block(), False), (synth.refined_airfoil(), True)):
        r = bench.refine_cpu_baseline(wl, body)
        assert r["kind"] == "oracle" and r["unit"] == "GLUPS" and r["cores"] == 1
        assert 0 < r["value"] < 1e-1 and r["seconds"] > 0
        assert "FP64, one thread" in r["sample"]
