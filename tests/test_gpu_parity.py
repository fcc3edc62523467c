"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, element by element (arXiv 1608.04658, Secs. 2-4.1).

Bars (max relative error of full populations over fluid nodes): 1e-12 for
FP64 storage, 2e-6 for FP32, 2e-3 for FP16/BF16 after 10 steps; the one BF16
case above that bar is marked as an expected failure with its measured error."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import TOL, fluid_mask, random_fields, rel_err, run_pair

pytestmark = pytest.mark.gpu
STORAGES = ["fp64", "fp32", "fp16", "bf16"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_04658_gb300 as lbm
    lbm.build()
    lbm.lib()


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("shape", [(150, 6, 5), (24, 20, 17), (1, 64, 1), (3, 3, 3), (64, 3, 2), (192, 5, 3)])
def test_periodic_random_state(storage, shape):
    """Rough random fields on periodic boxes: 150 = 128 + 22 nodes per row (two
    x-blocks with a ragged tail), a non-power-of-two box, a one-node-wide
    column (every pull wraps), the smallest cube, and rows of 64 and 192 nodes
    (the two-node kernel with one and two blocks per row, the second ragged)."""
    fields = random_fields(shape, 1)
    for steps in (1, 10):
        lat, orc = run_pair(shape, 0.01, storage, fields, steps)
        err = rel_err(lat.populations(), orc.get_f())
        assert err <= TOL[storage], (storage, steps, err)


_PIPE_FACES = [(0,) * 6, (2, 3, 1, 1, 0, 0), (1, 1, 2, 2, 3, 3)]


@pytest.mark.parametrize("storage,faces", [(st, f) for st in ("fp32", "fp16") for f in _PIPE_FACES]
                         + [("bf16", _PIPE_FACES[0])])
def test_two_node_kernel_faces(storage, faces):
    """The two-node bulk kernel on a 128x64x64 box (several blocks per row,
    more blocks than fit on the GPU at once) with each kind of face: periodic;
    equilibrium inflow x-, outflow x+, walls y; walls x (folded into the
    outer nodes' addresses), equilibrium y (the x-face nodes of those rows
    gathered again), outflow z."""
    shape = (128, 64, 64)
    lat, orc = run_pair(shape, 0.02, storage, random_fields(shape, 23), 10, faces=faces, u_face=(0.04, 0.0, 0.01))
    assert rel_err(lat.populations(), orc.get_f()) <= TOL[storage], faces


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_lbgk_mode(storage):
    shape = (40, 9, 7)
    lat, orc = run_pair(shape, 0.02, storage, random_fields(shape, 2), 10, gamma_mode=2)
    assert rel_err(lat.populations(), orc.get_f()) <= TOL[storage]


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16"])
def test_exact_stabilizer(storage):
    """Exact stabilizer (root of Eq. gamma_min by safeguarded Newton on the
    GPU) vs the oracle's bisection root: rough random state on a periodic box
    and a moving sphere with refill, 10 steps."""
    import paper_1608_04658_gb300 as lbm
    shape = (12, 10, 9)
    lat, orc = run_pair(shape, 0.01, storage, random_fields(shape, 17), 10, gamma_mode=lbm.GAMMA_EXACT)
    assert rel_err(lat.populations(), orc.get_f()) <= TOL[storage]
    shape = (16, 14, 12)
    geom = lbm.sphere((7.3, 6.6, 5.8), 3.1, U=(0.05, -0.03, 0.02))
    rho, u, xi = synth.parity_fields(shape, 19)
    lat, orc = run_pair(shape, 0.02, storage, (rho, 0.3 * u, xi, 1e-3), 10, geom=geom,
                        gamma_mode=lbm.GAMMA_EXACT)
    mask = fluid_mask(lat, orc)
    assert rel_err(lat.populations(), orc.get_f(), mask) <= TOL[storage]


def test_taylor_green_32_re1600_fp64_100_steps():
    """Plain method, periodic 32^3 Taylor-Green vortex, u0 = 0.05, Re = 1600,
    100 steps: FP64 parity, mass and momentum conservation, energy decay."""
    wl = synth.tgv_periodic(32)
    rho, u = synth.taylor_green_fields(wl["shape"], wl["u0"])
    lat, orc = run_pair(wl["shape"], wl["nu"], "fp64", (rho, u, None, 0.0), 100)
    assert rel_err(lat.populations(), orc.get_f()) <= TOL["fp64"]
    T = lat.totals()
    To = orc.totals()
    assert abs(T[0] - To[0]) < 1e-12 * To[0]
    assert np.abs(T[1:4]).max() < 1e-11
    assert T[4] == pytest.approx(To[4], rel=1e-11)


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_taylor_green_storage_forms(storage):
    wl = synth.tgv_periodic(32)
    rho, u = synth.taylor_green_fields(wl["shape"], wl["u0"])
    lat, orc = run_pair(wl["shape"], wl["nu"], storage, (rho, u, None, 0.0), 10)
    assert rel_err(lat.populations(), orc.get_f()) <= TOL[storage]


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16"])
def test_box_faces(storage):
    """Equilibrium inflow at x-, outflow at x+, walls at y+-, periodic z; and
    walls on x with equilibrium y faces and outflow z faces."""
    shape = (24, 12, 10)
    for faces in [(2, 3, 1, 1, 0, 0), (1, 1, 2, 2, 3, 3)]:
        lat, orc = run_pair(shape, 0.02, storage, random_fields(shape, 3), 10, faces=faces,
                            u_face=(0.04, 0.0, 0.01))
        assert rel_err(lat.populations(), orc.get_f()) <= TOL[storage], faces


@pytest.mark.parametrize("storage", STORAGES)
def test_stationary_sphere(storage):
    """Fixed sphere in a periodic box with a mean flow: Grad boundary, momentum
    exchange."""
    import paper_1608_04658_gb300 as lbm
    shape = (24, 20, 22)
    rho, u, xi = synth.parity_fields(shape, 4)
    fields = (rho, 0.3 * u + np.array([0.03, 0.01, -0.02]), xi, 1e-3)
    geom = lbm.sphere((11.37, 9.61, 10.83), 4.3)
    lat, orc = run_pair(shape, 0.02, storage, fields, 10, geom=geom)
    mask = fluid_mask(lat, orc)
    assert rel_err(lat.populations(), orc.get_f(), mask) <= TOL[storage]
    F, M = lat.forces()
    Fo, Mo = np.array(orc.body.F), np.array(orc.body.M)
    ftol = 1e-10 if storage == "fp64" else (1e-5 if storage == "fp32" else 2e-2)
    assert np.abs(F - Fo).max() <= ftol * np.abs(Fo).max()
    assert np.abs(M - Mo).max() <= ftol * np.abs(Mo).max() + 1e-12
    b = lat.body()
    assert b["n_boundary"] == orc.counters()["boundary"] // 10
    assert b["n_links"] == orc.counters()["links"] // 10


def test_monitor_records_carry_each_steps_force_and_sums(tmp_path):
    """The run monitor's JSON lines, every 2 steps of a fixed sphere: each
    record's force and torque are the oracle's for that step, its mass and
    momentum the oracle's sums over fluid nodes."""
    import json

    from paper_1608_04658_gb300 import monitor
    shape = (24, 20, 22)
    rho, u, xi = synth.parity_fields(shape, 4)
    fields = (rho, 0.3 * u + np.array([0.03, 0.01, -0.02]), xi, 1e-3)
    import paper_1608_04658_gb300 as lbm
    geom = lbm.sphere((11.37, 9.61, 10.83), 4.3)
    lat, orc = run_pair(shape, 0.02, "fp32", fields, 0, geom=geom)
    recs = monitor.run_logged(lat, 6, 2, tmp_path / "run.jsonl")
    assert [json.loads(line) for line in (tmp_path / "run.jsonl").read_text().splitlines()] == recs
    assert [r["step"] for r in recs] == [2, 4, 6]
    for r in recs:
        orc.step(2)
        Fo, Mo = np.array(orc.body.F), np.array(orc.body.M)
        assert np.abs(np.array(r["F"]) - Fo).max() <= 1e-5 * np.abs(Fo).max()
        assert np.abs(np.array(r["M"]) - Mo).max() <= 1e-5 * np.abs(Mo).max() + 1e-12
        T = orc.totals()
        assert abs(r["mass"] - T[0]) <= 1e-6 * T[0]
        assert np.abs(np.array(r["momentum"]) - T[1:4]).max() <= 1e-6 * T[0]
        assert r["status"] == 0 and r["n_links"] > 0


@pytest.mark.parametrize("storage", STORAGES)
def test_moving_free_sphere_with_refill(storage):
    """Free sphere between no-slip x/y walls, periodic z, under gravity: body
    update, moving-wall Grad boundary and refill of uncovered nodes."""
    import paper_1608_04658_gb300 as lbm
    shape = (28, 24, 40)
    faces = (1, 1, 1, 1, 0, 0)
    rho, u, xi = synth.parity_fields(shape, 5)
    fields = (rho, 0.2 * u, xi, 1e-3)
    geom = lbm.sphere((13.71, 11.42, 19.13), 4.6, U=(0.05, -0.03, -0.12), free=True,
                      rho_ratio=1.5, g=(0.0, 0.0, -2e-4))
    lat, orc = run_pair(shape, 0.03, storage, fields, 10, faces=faces, geom=geom)
    mask = fluid_mask(lat, orc)
    assert orc.counters()["refill"] > 10
    assert rel_err(lat.populations(), orc.get_f(), mask) <= TOL[storage]
    b = lat.body()
    ob = orc.body
    # the trajectory integrates the force, whose error follows the storage rounding
    xtol = {"fp64": 1e-13, "fp32": 1e-8, "fp16": 1e-5, "bf16": 1e-4}[storage]
    assert np.abs(b["X"] - np.array(ob.X)).max() < xtol
    assert np.abs(b["U"] - np.array(ob.U)).max() < xtol
    assert b["status"] == 0


def test_couette_planes_fp64():
    """Channel walls at q = 0.3 with the top wall moving: Grad boundary on a
    flat moving wall."""
    import paper_1608_04658_gb300 as lbm
    shape = (3, 20, 4)
    geom = lbm.planes(1.7, 18.3, U_hi=(0.01, 0.0, 0.0))
    lat, orc = run_pair(shape, 1.0 / 6.0, "fp64", (*synth.uniform_fields(shape), None, 0.0), 200, geom=geom)
    mask = fluid_mask(lat, orc)
    assert rel_err(lat.populations(), orc.get_f(), mask) <= TOL["fp64"]


def test_unstable_state_is_reported():
    """A NaN in the initial density (made on the host) sets the device status
    word; lbm_body_forces returns LBM_ERR_UNSTABLE.  No GPU fault is involved."""
    import paper_1608_04658_gb300 as lbm
    shape = (16, 8, 8)
    rho, u = synth.uniform_fields(shape)
    rho[3, 4, 5] = np.nan
    lat = lbm.Lattice(shape, 0.02, storage="fp32")
    lat.init_state(rho, u)
    lat.step(1)
    with pytest.raises(lbm.LbmError) as e:
        lat.forces()
    assert e.value.status == 4


@pytest.mark.parametrize("case", ["fp32", "fp16", "fp64", "bf16", "fp32_exact"])
def test_sedimenting_sphere_full_size_sampled(case):
    """Full-size sedimenting-sphere box (128x128x256, D = 16, x/y walls,
    periodic z) in the launch configuration the benchmark times: one step from
    a seeded random state, compared at every boundary node and at 4000 random
    nodes, which the oracle computes one by one.  fp32_exact: the exact
    stabilizer (root of Eq. gamma_min) on both sides."""
    import paper_1608_04658_gb300 as lbm
    storage = case.split("_")[0]
    gmode = lbm.GAMMA_EXACT if case.endswith("_exact") else lbm.GAMMA_ANALYTIC
    wl = synth.sedimenting_sphere()
    shape = wl["shape"]
    rho, u, xi = synth.parity_fields(shape, 7)
    geom = lbm.sphere(wl["X"], wl["D"] / 2, U=(0.0, 0.0, -0.04), free=True, rho_ratio=wl["rho_ratio"],
                      g=wl["g"])
    lat = lbm.Lattice(shape, wl["nu"], storage=storage, faces=wl["faces"], gamma_mode=gmode)
    lat.set_geometry(geom)
    lat.init_state(rho, u, xi, 1e-3)
    f0 = lat.populations()
    lat.step(1)
    f1 = lat.populations()
    flags = lat.flags.cpu().numpy().reshape(-1)
    orc = oracle.Oracle(shape, nu=wl["nu"], faces=wl["faces"], gamma_mode=gmode,
                        body=oracle.sphere_body(wl["X"], wl["D"] / 2, U=(0.0, 0.0, -0.04), free=True,
                                                rho_ratio=wl["rho_ratio"], g=wl["g"]))
    orc.set_f(f0)  # the decoded stored state is the common input
    rng = np.random.default_rng(7)
    bnodes = np.nonzero(flags & 4)[0]
    assert len(bnodes) > 500
    nodes = np.unique(np.concatenate([bnodes, rng.integers(0, lat.N, 4000),
                                      [0, lat.N - 1, shape[0] - 1]]))
    ref = orc.step_sampled(nodes)
    got = f1.reshape(27, -1)[:, nodes].T
    ok = ~np.isnan(ref[:, 0])
    assert np.array_equal(ok, (flags[nodes] & 1) == 0)
    # one step from the same stored input: FP32 arithmetic and one rounding
    # to storage (BF16: the 2e-3 bar of 16-bit storage; the exact stabilizer:
    # the GPU's FP32 Newton root against the oracle's FP64 bisection root)
    tol = {"fp64": 1e-12, "fp32": 1e-6, "fp16": 1e-3, "bf16": 2e-3, "fp32_exact": 2e-6}[case]
    assert float((np.abs(got[ok] - ref[ok]) / np.abs(ref[ok])).max()) <= tol


def _sampled_after_one_step(lat, nodes):
    """Full populations of the listed nodes after the step, read from the
    device state without decoding the whole lattice."""
    _, W = oracle.lattice()
    g = lat.f.reshape(27, -1)[:, torch.as_tensor(nodes, device=lat.device)].double().cpu().numpy()
    return (g + W[:, None] * lat.rho0).T


def _rough_fields(shape, seed, u_mean=(0.0, 0.0, 0.0)):
    """Seeded random density and velocity (the parity-field ranges) without
    the 27-plane noise array, which would not fit comfortably at full size;
    the steps before the compared one develop the non-equilibrium part."""
    nx, ny, nz = shape
    N = nx * ny * nz
    rho = (1.0 + 0.01 * (2.0 * synth.uniform(seed, 0, N) - 1.0)).reshape(nz, ny, nx)
    u = (0.01 * (2.0 * synth.uniform(seed, 1, 3 * N) - 1.0)).reshape(nz, ny, nx, 3) + np.array(u_mean)
    return rho, u


def _full_size_sampled(lat, orc_body, wl, f_fields, storage, seed):
    lat.step(2)
    f0 = lat.populations()
    lat.step(1)
    flags = lat.flags.cpu().numpy().reshape(-1)
    rng = np.random.default_rng(seed)
    bnodes = np.nonzero(flags & 4)[0]
    unodes = np.nonzero(flags & 8)[0]
    nodes = np.unique(np.concatenate([bnodes, unodes, rng.integers(0, lat.N, 4000), [0, lat.N - 1]]))
    got = _sampled_after_one_step(lat, nodes)
    del lat
    orc = oracle.Oracle(wl["shape"], nu=wl["nu"], faces=wl["faces"], u_face=wl.get("u_face", (0.0, 0.0, 0.0)),
                        body=orc_body)
    orc.set_f(f0)
    del f0
    ref = orc.step_sampled(nodes)
    ok = ~np.isnan(ref[:, 0])
    assert np.array_equal(ok, (flags[nodes] & 1) == 0)
    tol = {"fp64": 1e-12, "fp32": 1e-6, "fp16": 1e-3, "bf16": 2e-3}[storage]
    assert float((np.abs(got[ok] - ref[ok]) / np.abs(ref[ok])).max()) <= tol
    return len(bnodes), len(unodes)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_plunging_airfoil_full_size_sampled(storage):
    """Full-size plunging airfoil (1024x512x64, chord 128, equilibrium inflow,
    outflow, far field) in the benchmark's configuration: after two steps from
    a seeded random state around the inflow, one step compared at every
    boundary and refilled node and at 4000 random nodes computed one by one by
    the oracle."""
    import paper_1608_04658_gb300 as lbm
    wl = synth.plunging_airfoil()
    shape = wl["shape"]
    rho, u = _rough_fields(shape, 11, wl["u_face"])
    geom = (wl["le"], wl["chord"], wl["ca"], wl["sa"], wl["h_amp"], wl["h_omega"], wl["camber_m"],
            wl["camber_p"], wl["thick"], 500.0)
    lat = lbm.Lattice(shape, wl["nu"], storage=storage, faces=wl["faces"], u_face=wl["u_face"])
    lat.set_geometry(lbm.airfoil(*geom))
    lat.init_state(rho, u)
    del rho, u
    # the oracle's body starts at the pose after the two warm-up steps
    geom2 = geom[:-1] + (502.0,)
    nb, nu_ = _full_size_sampled(lat, oracle.airfoil_body(*geom2), wl, None, storage, 11)
    assert nb > 10000


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_anguilliform_swimmer_full_size_sampled(storage):
    """Full-size swimmer (768x256x256, L = 128, 19,200 triangles) in the
    benchmark's launch configuration, held so that its pose after the warm-up
    steps is known to the oracle: one step from a seeded random state,
    compared at every boundary and refilled node and 4000 random nodes."""
    import paper_1608_04658_gb300 as lbm
    wl = synth.anguilliform_swimmer()
    shape = wl["shape"]
    rho, u = _rough_fields(shape, 13)
    lat = lbm.Lattice(shape, wl["nu"], storage=storage, faces=wl["faces"])
    lat.set_geometry(lbm.swimmer(wl["X"], wl["rest"], wl["tris"], wl["L"], wl["amp"], wl["wavelength"],
                                 wl["period"], U=(-0.003, 0.0, 0.0), mass=wl["mass"], t0=700.0))
    lat.init_state(rho, u)
    del rho, u
    # held swimmer (its pose after the warm-up steps is then known exactly)
    body = oracle.mesh_body(wl["X"], wl["rest"], wl["tris"], wl["L"], wl["amp"], wl["wavelength"], wl["period"],
                            U=(-0.003, 0.0, 0.0), mass=wl["mass"], t0=702.0)
    nb, nu_ = _full_size_sampled(lat, body, wl, None, storage, 13)
    assert nb > 5000


@pytest.mark.parametrize("storage", ["fp32", "fp16", "fp64"])
def test_init_from_pinned_host_fields(storage):
    """lbm_init_state reading pinned host fields across the host link gives
    the bits of the same fields in device memory, and lbm_init_state_f32 those
    of the same single-precision values in double; pageable host memory is
    refused (LBM_ERR_ARG) before any kernel runs."""
    import ctypes

    import paper_1608_04658_gb300 as lbm
    shape = (24, 10, 6)
    rho, u, xi = synth.parity_fields(shape, 21)
    a = lbm.Lattice(shape, 0.05, storage=storage)
    a.init_state(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda(), torch.from_numpy(xi).cuda(), 1e-3)
    b = lbm.Lattice(shape, 0.05, storage=storage)
    b.init_state(torch.from_numpy(rho).pin_memory(), torch.from_numpy(u).pin_memory(),
                 torch.from_numpy(xi).pin_memory(), 1e-3)
    assert torch.equal(a.f, b.f)
    # single-precision fields (lbm_init_state_f32): the bits of the same values in double
    r32, u32, x32 = (torch.from_numpy(v.astype(np.float32)) for v in (rho, u, xi))
    c = lbm.Lattice(shape, 0.05, storage=storage)
    c.init_state(r32.pin_memory(), u32.pin_memory(), x32.pin_memory(), 1e-3)
    d = lbm.Lattice(shape, 0.05, storage=storage)
    d.init_state(r32.double().cuda(), u32.double().cuda(), x32.double().cuda(), 1e-3)
    e = lbm.Lattice(shape, 0.05, storage=storage)
    e.init_state(r32.cuda(), u32.cuda(), x32.cuda(), 1e-3)
    assert torch.equal(c.f, d.f) and torch.equal(e.f, d.f)
    r = np.ascontiguousarray(rho)
    v = np.ascontiguousarray(u)
    st = lbm.lib().lbm_init_state(b._ctx, r.ctypes.data_as(ctypes.c_void_p), v.ctypes.data_as(ctypes.c_void_p),
                                  None, 0.0)
    from paper_1608_04658_gb300.binding import LBM_ERR_ARG
    assert st == LBM_ERR_ARG


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_checkpoint_resume_is_bitwise(storage, tmp_path):
    """20 steps straight equal 10 steps + save + load into a fresh context +
    10 steps, bit for bit (populations and body state)."""
    import paper_1608_04658_gb300 as lbm
    shape = (32, 28, 40)
    faces = (1, 1, 1, 1, 0, 0)
    rho, u, xi = synth.parity_fields(shape, 12)
    geom = lbm.sphere((15.4, 13.7, 20.3), 5.2, U=(0.01, 0.0, -0.06), free=True, g=(0.0, 0.0, -2e-4))

    def fresh():
        lat = lbm.Lattice(shape, 0.03, storage=storage, faces=faces)
        lat.set_geometry(geom)
        return lat

    a = fresh()
    a.init_state(rho, 0.2 * u, xi, 1e-3)
    a.step(20)
    b = fresh()
    b.init_state(rho, 0.2 * u, xi, 1e-3)
    b.step(10)
    path = str(tmp_path / "state.lbm")
    b.save(path)
    c = fresh()
    c.load(path)
    c.step(10)
    fa, fc = a.populations(), c.populations()
    fluid = (a.flags.cpu().numpy() & 1) == 0
    assert np.array_equal(fa[:, fluid], fc[:, fluid])
    ba, bc = a.body(), c.body()
    for k in ("X", "U", "F", "M"):
        assert np.array_equal(ba[k], bc[k]), k


def _golden_sphere_re100():
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "sphere_re100.txt")):
        if line.strip() and not line.startswith("#"):
            name, cd, ld = line.split()
            rows[name] = (float(cd), float(ld))
    return rows


@pytest.mark.parametrize("D,u,steps,cd_tol", [(16.0, 0.04, 12000, 0.06), (30.0, 0.02, 24000, 0.03)])
def test_stationary_sphere_drag_and_wake_at_re100(D, u, steps, cd_tol):
    """Sec. 4.1, Table 4: a held sphere in a uniform stream at Re = 100 (box
    8D x 8D x 16D, equilibrium far-field faces at u_inf, zero-gradient outflow,
    FP32 storage).  The momentum-exchange drag coefficient averaged over the
    last 2000 steps is within 6% (D = 16) and 3% (D = 30, the paper's
    resolution) of the paper's C_d = 1.1; at D = 30 the recirculation length
    along the axis behind the sphere is within 0.06 D of the paper's 0.86 D."""
    import paper_1608_04658_gb300 as lbm
    golden = _golden_sphere_re100()
    cd_paper, ld_paper = golden["present"]
    n = int(D)
    shape = (8 * n, 8 * n, 16 * n)
    nu = u * D / 100.0
    faces = (2, 2, 2, 2, 2, 3)
    lat = lbm.Lattice(shape, nu, storage="fp32", faces=faces, u_face=(0.0, 0.0, u))
    X = (shape[0] / 2 - 0.5 + 0.123, shape[1] / 2 - 0.5 + 0.0567, 0.3 * shape[2] + 0.311)
    lat.set_geometry(lbm.sphere(X, D / 2))
    lat.init_state(*synth.uniform_fields(shape, u=(0.0, 0.0, u)))
    lat.step(steps - 2000)
    lat.reset_average()
    lat.step(2000)
    F, _ = lat.forces(averaged=True)
    cd = F[2] / (0.5 * u * u * np.pi * D * D / 4.0)
    print(f"D={D:g}: C_d={cd:.4f} (paper {cd_paper})")
    assert abs(cd - cd_paper) <= cd_tol * cd_paper
    assert abs(F[0]) <= 0.01 * F[2] and abs(F[1]) <= 0.01 * F[2]
    if D < 30:
        return
    # axial velocity on the sphere's axis (bilinear in x, y between node lines),
    # from the stored populations f = g + W rho0
    import torch
    cur = lbm.binding.lib().lbm_current_buffer(lat._ctx)
    g = (lat.f_a if cur == 0 else lat.f_b).double()
    _, W = oracle.lattice()
    c = torch.tensor(oracle.lattice()[0], dtype=torch.float64, device=g.device)
    Wt = torch.tensor(W, dtype=torch.float64, device=g.device)
    x0, y0 = int(np.floor(X[0])), int(np.floor(X[1]))
    fx, fy = X[0] - x0, X[1] - y0
    uz = 0.0
    for dx, wx in ((0, 1 - fx), (1, fx)):
        for dy, wy in ((0, 1 - fy), (1, fy)):
            f = g[:, :, y0 + dy, x0 + dx] + Wt[:, None] * lat.rho0
            uz = uz + wx * wy * ((c[:, 2, None] * f).sum(0) / f.sum(0))
    uz = uz.cpu().numpy()
    z_rear = X[2] + D / 2
    k = int(np.ceil(z_rear))
    while uz[k] >= 0.0:  # first node behind the surface in the reverse flow
        k += 1
    while uz[k + 1] < 0.0:
        k += 1
    z_cross = k + uz[k] / (uz[k] - uz[k + 1])
    ld = (z_cross - z_rear) / D
    print(f"D={D:g}: L/D={ld:.3f} (paper {ld_paper})")
    assert abs(ld - ld_paper) <= 0.06


_LONG_RUN = {}


def _long_run_oracle(wl):
    """The FP64 oracle's mean force over steps 1001-2000 and its velocity at
    step 2000 (about a minute and a half of one host core, run once)."""
    if "r" not in _LONG_RUN:
        shape = wl["shape"]
        orc = oracle.Oracle(shape, nu=wl["nu"], faces=wl["faces"],
                            body=oracle.sphere_body(wl["X"], wl["D"] / 2, free=True, rho_ratio=wl["rho_ratio"],
                                                    g=wl["g"]))
        orc.init_state(*synth.uniform_fields(shape))
        orc.step(1000)
        Fsum = np.zeros(3)
        for _ in range(1000):
            orc.step(1)
            Fsum += np.array(orc.body.F)
        _LONG_RUN["r"] = (Fsum / 1000, np.array(orc.body.U))
    return _LONG_RUN["r"]


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_long_run_drag_matches_the_oracle(storage):
    """The sedimenting sphere of Sec. 4.1 on a reduced box (32x32x64, D = 8,
    solid/fluid density ratio 1.5, x/y walls, periodic z, Re = u_t D / nu =
    100 with gravity from the terminal-velocity balance), started at rest and
    run 2000 steps on the GPU and in the FP64 oracle: the force averaged over
    steps 1001-2000 and the settling velocity at step 2000 agree within 0.5%
    (the long-run drag bar).  The sphere falls about 40 nodes, so its
    boundary links, covered and refilled nodes change every few steps."""
    import paper_1608_04658_gb300 as lbm
    wl = synth.sedimenting_sphere(shape=(32, 32, 64), D=8.0)
    shape = wl["shape"]
    geom = lbm.sphere(wl["X"], wl["D"] / 2, free=True, rho_ratio=wl["rho_ratio"], g=wl["g"])
    lat = lbm.Lattice(shape, wl["nu"], storage=storage, faces=wl["faces"])
    lat.set_geometry(geom)
    lat.init_state(*synth.uniform_fields(shape))
    lat.step(1000)
    lat.reset_average()
    lat.step(1000)
    F, _ = lat.forces(averaged=True)
    U = np.array(lat.body()["U"])
    Fo, Uo = _long_run_oracle(wl)
    drag_err = abs(F[2] - Fo[2]) / abs(Fo[2])
    u_err = abs(U[2] - Uo[2]) / abs(Uo[2])
    print(f"{storage}: drag {F[2]:.6e} vs oracle {Fo[2]:.6e} (rel {drag_err:.2e}), "
          f"U_z {U[2]:.6e} vs {Uo[2]:.6e} (rel {u_err:.2e})")
    assert abs(Uo[2]) > 0.01 and Fo[2] > 0
    assert drag_err <= 5e-3
    assert u_err <= 5e-3


def test_sedimenting_sphere_reaches_terminal_velocity():
    """The benchmark's sedimenting sphere (128x128x256, D = 16, rho_s/rho_f =
    1.5, walls in x and y, periodic z; Sec. 4.1 two-way coupling, Euler
    update of Newton's equations) run from rest: over the last 2000 of 14000
    steps the mean momentum-exchange force balances the buoyancy-corrected
    weight m (1 - rho_f/rho_s) g to 2% (the sphere keeps gaining a little
    speed: along the periodic axis it falls through its own wake), the
    lateral force stays small, and the settling velocity lies within 20% of
    the 0.04 the gravity was set for (by the force balance with C_d = 1.1)."""
    import paper_1608_04658_gb300 as lbm
    wl = synth.sedimenting_sphere()
    lat = lbm.Lattice(wl["shape"], wl["nu"], storage="fp32", faces=wl["faces"])
    lat.set_geometry(lbm.sphere(wl["X"], wl["D"] / 2, free=True, rho_ratio=wl["rho_ratio"], g=wl["g"]))
    lat.init_state(*synth.uniform_fields(wl["shape"]))
    lat.step(12000)
    lat.reset_average()
    lat.step(2000)
    F, _ = lat.forces(averaged=True)
    D, rr, g = wl["D"], wl["rho_ratio"], -wl["g"][2]
    m = rr * np.pi * D ** 3 / 6.0
    weight = m * (1.0 - 1.0 / rr) * g
    u_t = -lat.body()["U"][2]
    print(f"sedimenting: u_t={u_t:.5f} F_z/weight={F[2] / weight:.5f}")
    assert abs(F[2] - weight) <= 2e-2 * weight
    assert abs(F[0]) <= 0.05 * weight and abs(F[1]) <= 0.05 * weight
    assert 0.8 * 0.04 <= u_t <= 1.2 * 0.04
    assert lat.body()["status"] == 0


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("kind", ["sphere", "swimmer"])
def test_launch_orders_agree_bitwise(kind, storage):
    """The split and the sequential launch order of a step (and the automatic
    choice between them after its timed trial steps) give the same
    populations and body state bit for bit.  In the split order the sweep
    box's nodes take the one-node bulk kernel and the others the two-node
    kernel (packed arithmetic); in the sequential order every bulk node takes
    the two-node kernel, so this also checks that the two give the same bits
    (with x walls on the sphere's box)."""
    import paper_1608_04658_gb300 as lbm
    if kind == "sphere":
        shape, faces = (32, 28, 40), (1, 1, 1, 1, 0, 0)
        geom = lbm.sphere((15.4, 13.7, 20.3), 5.2, U=(0.01, 0.0, -0.06), free=True, g=(0.0, 0.0, -2e-4))
    else:
        shape, faces = (64, 32, 20), (0,) * 6
        geom = _swimmer_geom(lbm, U=(-0.004, 0.0, 0.0), free=True, t0=5.0)
    rho, u, xi = synth.parity_fields(shape, 41)
    runs = {}
    for order in ("split", "sequential", "auto"):
        lat = lbm.Lattice(shape, 0.03, storage=storage, faces=faces)
        lat.set_launch_order(order)
        lat.set_geometry(geom)
        lat.init_state(rho, 0.2 * u + np.array([0.01, 0.0, 0.0]), xi, 1e-3)
        lat.step(9)
        lat.body()  # synchronises: the trial steps have run
        lat.step(3)
        runs[order] = (lat.populations(), lat.body(), lat.launch_order())
    assert runs["split"][2] == "split" and runs["sequential"][2] == "sequential"
    assert runs["auto"][2] in ("split", "sequential")
    for order in ("sequential", "auto"):
        assert np.array_equal(runs[order][0], runs["split"][0]), order
        for k in ("X", "U", "F", "M"):
            assert np.array_equal(runs[order][1][k], runs["split"][1][k]), (order, k)
    assert lbm.binding.lib().lbm_set_launch_order(lat._ctx, 7) != 0


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_async_force_records(storage):
    """Force records copied while later steps run (lbm_body_forces_async /
    lbm_body_forces_wait, two records outstanding) equal, bit for bit, the
    synchronous force of the same step in an identical run; a pageable
    record and an unissued ticket are rejected."""
    import ctypes
    import paper_1608_04658_gb300 as lbm
    shape = (32, 28, 40)
    faces = (1, 1, 1, 1, 0, 0)
    rho, u, xi = synth.parity_fields(shape, 31)
    geom = lbm.sphere((15.4, 13.7, 20.3), 5.2, U=(0.01, 0.0, -0.06), free=True, g=(0.0, 0.0, -2e-4))

    def fresh():
        lat = lbm.Lattice(shape, 0.03, storage=storage, faces=faces)
        lat.set_geometry(geom)
        lat.init_state(rho, 0.2 * u, xi, 1e-3)
        return lat

    a, b = fresh(), fresh()
    steps = 20
    sync = []
    for _ in range(steps):
        b.step(1)
        sync.append(b.forces())
    pending, got = [], []
    for _ in range(steps):
        a.step(1)
        pending.append(a.forces_async())
        if len(pending) > 2:
            got.append(a.forces_wait(pending.pop(0)))
    got += [a.forces_wait(t) for t in pending]
    assert len(got) == steps
    for k in range(steps):
        assert np.array_equal(got[k][0], sync[k][0]) and np.array_equal(got[k][1], sync[k][1]), k
    assert np.abs(got[-1][0]).max() > 0
    assert a.body()["t"] == a._rec[(steps - 1) % lbm.binding.RECORD_DEPTH].numpy()[6] == steps
    # a pageable record is refused; so is a ticket not yet issued
    pageable = np.zeros(8)
    t = ctypes.c_int64()
    assert lbm.binding.lib().lbm_body_forces_async(a._ctx, ctypes.c_void_p(pageable.ctypes.data),
                                                   ctypes.byref(t)) != 0
    assert lbm.binding.lib().lbm_body_forces_wait(a._ctx, steps + 5) != 0


# BF16 exceeds the 2e-3 bar of 16-bit storage on this case (3.8e-3 measured
# on GB300: the inflow at 0.05 with rough random fields makes |g|/f close to 1,
# and BF16, with 8 significand bits, rounds each store of g by up to 2^-8 of it);
# every other BF16 case meets the bar.
@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", pytest.param(
    "bf16", marks=pytest.mark.xfail(strict=True, reason="BF16 storage: 3.8e-3 measured against the 2e-3 bar"))])
def test_plunging_airfoil(storage):
    """Plunging cambered airfoil (chord 32, 4 degrees, amplitude 1.6, a fast
    plunge so nodes get uncovered) with equilibrium inflow, outflow and far
    field: airfoil geometry by bisection, prescribed kinematics, refill."""
    import paper_1608_04658_gb300 as lbm
    wl = synth.plunging_airfoil()
    shape = (96, 40, 6)
    rho, u, xi = synth.parity_fields(shape, 13)
    fields = (rho, 0.2 * u + np.array([0.05, 0.0, 0.0]), xi, 1e-3)
    geom = lbm.airfoil((24.37, 20.29), 32.0, wl["ca"], wl["sa"], 1.6, 0.05, wl["camber_m"], wl["camber_p"],
                       wl["thick"], t0=3.0)
    lat, orc = run_pair(shape, 0.02, storage, fields, 10, faces=wl["faces"], geom=geom, u_face=wl["u_face"])
    mask = fluid_mask(lat, orc)
    assert orc.counters()["refill"] > 0
    assert rel_err(lat.populations(), orc.get_f(), mask) <= TOL[storage]
    F, M = lat.forces()
    Fo, Mo = np.array(orc.body.F), np.array(orc.body.M)
    ftol = {"fp64": 1e-10, "fp32": 1e-4, "fp16": 3e-2, "bf16": 3e-2}[storage]
    assert np.abs(F - Fo).max() <= ftol * np.abs(Fo).max()
    assert np.abs(M - Mo).max() <= ftol * np.abs(Mo).max()
    assert lat.body()["X"][1] == pytest.approx(orc.body.X[1], abs=1e-13)


def _swimmer_geom(lat_mod, L=32.0, segments=40, ring=24, X=(20.137, 16.371, 10.293), period=160.0, **kw):
    rest, tris = synth.swimmer_mesh(L, segments, ring)
    return lat_mod.swimmer(X, rest, tris, L, 0.125, L, period, mass=synth.swimmer_volume(L), **kw)


@pytest.mark.parametrize("storage", STORAGES)
def test_anguilliform_swimmer(storage):
    """Deforming triangulated swimmer (L = 32, 40 segments x 24 around, a fast
    undulation so nodes get uncovered every step, free along x) in a periodic
    box: ray-parity solid marks, link search over the triangle cells,
    barycentric wall velocity, refill with the material velocity, Euler step
    of the head along x."""
    import paper_1608_04658_gb300 as lbm
    shape = (64, 32, 20)
    rho, u, xi = synth.parity_fields(shape, 17)
    fields = (rho, 0.2 * u + np.array([0.01, 0.0, 0.0]), xi, 1e-3)
    geom = _swimmer_geom(lbm, U=(-0.004, 0.0, 0.0), free=True, t0=5.0)
    lat, orc = run_pair(shape, 0.02, storage, fields, 10, geom=geom)
    mask = fluid_mask(lat, orc)
    cnt = orc.counters()
    assert cnt["refill"] > 0 and cnt["error"] == 0
    assert rel_err(lat.populations(), orc.get_f(), mask) <= TOL[storage]
    F, M = lat.forces()
    Fo, Mo = np.array(orc.body.F), np.array(orc.body.M)
    ftol = {"fp64": 1e-10, "fp32": 1e-4, "fp16": 3e-2, "bf16": 3e-2}[storage]
    assert np.abs(F - Fo).max() <= ftol * np.abs(Fo).max()
    assert np.abs(M - Mo).max() <= ftol * np.abs(Mo).max()
    b = lat.body()
    if storage == "fp64":
        xtol = 1e-13
    else:
        # explicit Euler (Sec. 4.3) over n steps adds the per-step force
        # error into the head's position at most n(n-1)/2 times
        n = 10
        xtol = 0.5 * n * (n - 1) * ftol * np.abs(Fo).max() / geom.mass
    assert b["X"][0] == pytest.approx(orc.body.X[0], abs=xtol)
    assert b["t"] == orc.body.t == 15.0
    assert b["status"] == 0


@pytest.mark.parametrize("storage", STORAGES)
def test_three_dof_swimmer(storage):
    """Swimmer free in x, y and yaw (Sec. 4.3) in a periodic box: the centre of
    mass frame (pose X + R(psi)(b - c(t)) with the mesh's mass properties by
    the divergence theorem), the rotating wall velocity in the links and the
    refill, and the Euler update of X, U, psi and the angular momentum."""
    import paper_1608_04658_gb300 as lbm
    shape = (64, 40, 20)
    rho, u, xi = synth.parity_fields(shape, 23)
    fields = (rho, 0.2 * u + np.array([0.01, -0.004, 0.0]), xi, 1e-3)
    geom = _swimmer_geom(lbm, X=(33.137, 19.371, 10.293), U=(-0.004, 0.003, 0.0), free=7, t0=5.0, psi=0.21,
                         omega=0.004)
    lat, orc = run_pair(shape, 0.02, storage, fields, 10, geom=geom)
    mask = fluid_mask(lat, orc)
    cnt = orc.counters()
    assert cnt["refill"] > 0 and cnt["error"] == 0
    assert rel_err(lat.populations(), orc.get_f(), mask) <= TOL[storage]
    F, M = lat.forces()
    Fo, Mo = np.array(orc.body.F), np.array(orc.body.M)
    ftol = {"fp64": 1e-10, "fp32": 1e-4, "fp16": 3e-2, "bf16": 3e-2}[storage]
    assert np.abs(F - Fo).max() <= ftol * np.abs(Fo).max()
    assert np.abs(M - Mo).max() <= ftol * np.abs(Mo).max()
    b = lat.body()
    if storage == "fp64":
        xtol = wtol = 1e-13
    else:
        # explicit Euler over n steps sums the per-step force (torque) error
        # at most n(n-1)/2 times into X (psi) and n times into U (omega)
        n = 10
        xtol = 0.5 * n * (n - 1) * ftol * np.abs(Fo).max() / geom.mass
        wtol = 0.5 * n * (n - 1) * ftol * np.abs(Mo).max() / orc.body.Izz
    for a in range(2):
        assert b["X"][a] == pytest.approx(orc.body.X[a], abs=xtol)
        assert b["U"][a] == pytest.approx(orc.body.U[a], abs=xtol)
    assert b["psi"] == pytest.approx(orc.body.psi, abs=wtol)
    assert b["omega"] == pytest.approx(orc.body.omega, abs=wtol)
    assert b["Izz"] == pytest.approx(orc.body.Izz, rel=1e-12)
    assert abs(b["psi"] - 0.21) > 1e-3 and abs(b["omega"] - 0.004) > 1e-3
    assert b["t"] == orc.body.t == 15.0
    assert b["status"] == 0


def test_swimmer_rejects_bad_meshes():
    """Host-side checks of lbm_set_geometry for a mesh: triangle indices out
    of range and a pose too close to a box face are rejected, nothing runs."""
    import paper_1608_04658_gb300 as lbm
    shape = (64, 32, 20)
    lat = lbm.Lattice(shape, 0.02, storage="fp32")
    rest, tris = synth.swimmer_mesh(32.0, 40, 24)
    bad = tris.copy()
    bad[5, 1] = len(rest)
    with pytest.raises(lbm.LbmError):
        lat.set_geometry(lbm.swimmer((20.137, 16.371, 10.293), rest, bad, 32.0, 0.125, 32.0, 160.0))
    with pytest.raises(lbm.LbmError):
        lat.set_geometry(lbm.swimmer((40.137, 16.371, 10.293), rest, tris, 32.0, 0.125, 32.0, 160.0))
    lat.set_geometry(lbm.swimmer((20.137, 16.371, 10.293), rest, tris, 32.0, 0.125, 32.0, 160.0))
