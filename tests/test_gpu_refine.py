"""GPU parity of the two-level block refinement (lbm_refine_*; Sec. 4.2's
two-level grid, readings stated in include/lbm.h and oracle/kbc_oracle.c)
against the oracle's RefinedOracle on the same seeded inputs, element by
element on every node the refined step defines: all coarse nodes but those
more than one layer inside the block's surface, all fine nodes but the pad.

Bars as for the single-level step (tests/parity_util.py): 1e-12 FP64, 2e-6
FP32, 2e-3 16-bit."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import TOL, random_fields, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_04658_gb300 as lbm
    lbm.build()
    lbm.lib()


def run_refined(shape, nu, storage, lo, hi, steps, seed=1, faces=(0,) * 6, u_face=(0.0, 0.0, 0.0),
                gamma_mode=0):
    import paper_1608_04658_gb300 as lbm
    rho, u, xi, amp = random_fields(shape, seed)
    lat = lbm.Lattice(shape, nu, storage=storage, faces=faces, u_face=u_face, gamma_mode=gamma_mode)
    ref = lbm.Refinement(lat, lo, hi)
    frho, fu, fxi, famp = random_fields(ref.fine.shape, seed + 100)
    lat.init_state(rho, u, xi, amp)
    ref.fine.init_state(frho, fu, fxi, famp)
    ref.init()
    ref.step(steps)

    orc = oracle.Oracle(shape, nu=nu, faces=faces, u_face=u_face, gamma_mode=gamma_mode)
    orc.init_state(rho, u, xi, amp)
    ro = oracle.RefinedOracle(orc, lo, hi)
    assert ro.fine.shape == ref.fine.shape
    ro.fine.init_state(frho, fu, fxi, famp)
    ro.init()
    ro.step(steps)
    return lat, ref, orc, ro


def errors(lat, ref, orc, ro):
    ec = rel_err(lat.populations(), orc.get_f(), ro.coarse_valid())
    ef = rel_err(ref.fine.populations(), ro.fine.get_f(), ro.fine_valid())
    return ec, ef


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
def test_refined_step_matches_the_oracle(storage):
    """A 24 x 20 x 18 periodic box with the block [5, 16] x [4, 13] x [3, 12]
    (fine lattice 24 x 20 x 20), rough random states on both levels, 1 and 4
    coarse steps."""
    for steps in (1, 4):
        lat, ref, orc, ro = run_refined((24, 20, 18), 0.02, storage, (5, 4, 3), (16, 13, 12), steps)
        ec, ef = errors(lat, ref, orc, ro)
        assert ec <= TOL[storage] and ef <= TOL[storage], (storage, steps, ec, ef)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_refined_step_with_box_faces_and_the_smallest_block(storage):
    """Coarse faces of every kind (equilibrium inflow x-, outflow x+, walls y,
    periodic z) around a block reaching to one node off them ([1, 14] x [1, 8]
    on a 16 x 10 box), and the smallest block (three cells) in z."""
    lat, ref, orc, ro = run_refined((16, 10, 9), 0.05, storage, (1, 1, 2), (14, 8, 5), 3, seed=5,
                                    faces=(2, 3, 1, 1, 0, 0), u_face=(0.03, 0.0, 0.01))
    ec, ef = errors(lat, ref, orc, ro)
    assert ec <= TOL[storage] and ef <= TOL[storage], (storage, ec, ef)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_refined_step_exact_stabilizer(storage):
    lat, ref, orc, ro = run_refined((20, 16, 14), 0.01, storage, (4, 3, 3), (13, 11, 9), 3, seed=9, gamma_mode=1)
    ec, ef = errors(lat, ref, orc, ro)
    assert ec <= TOL[storage] and ef <= TOL[storage], (storage, ec, ef)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_refined_step_several_tiles(storage):
    """Fine rows of 160 nodes (two 128-node blocks of the bulk launch, the
    second ragged) on a 100 x 36 x 30 coarse box, 3 coarse steps."""
    lat, ref, orc, ro = run_refined((100, 36, 30), 0.01, storage, (10, 6, 5), (89, 21, 16), 3, seed=13)
    assert ref.fine.shape == (160, 32, 24)
    ec, ef = errors(lat, ref, orc, ro)
    assert ec <= TOL[storage] and ef <= TOL[storage], (storage, ec, ef)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_refined_uniform_flow_stays_uniform(storage):
    """Uniform flow is a steady state of both levels and of their coupling."""
    import paper_1608_04658_gb300 as lbm
    U = (0.04, -0.02, 0.03)
    shape = (40, 24, 20)
    lat = lbm.Lattice(shape, 0.01, storage=storage)
    ref = lbm.Refinement(lat, (8, 5, 4), (31, 18, 15))
    lat.init_state(*synth.uniform_fields(shape, U))
    ref.fine.init_state(*synth.uniform_fields(ref.fine.shape, U))
    ref.init()
    ref.step(6)
    fe = oracle.feq(1.0, U)[:, None, None, None]
    vc = np.ones(shape[::-1], dtype=bool)
    vc[6:14, 7:17, 10:30] = False
    vf = np.zeros(ref.fine.shape[::-1], dtype=bool)
    vf[:-1, :-1, :-1] = True
    bar = 1e-14 if storage == "fp64" else 1e-6
    assert rel_err(lat.populations(), np.broadcast_to(fe, (27,) + shape[::-1]), vc) < bar
    assert rel_err(ref.fine.populations(), np.broadcast_to(fe, (27,) + ref.fine.shape[::-1]), vf) < bar


def test_refinement_rejects_mismatched_levels():
    import paper_1608_04658_gb300 as lbm
    from paper_1608_04658_gb300 import binding
    lat = lbm.Lattice((24, 20, 18), 0.02, storage="fp32")
    with pytest.raises(lbm.LbmError) as e:
        lbm.Refinement(lat, (0, 4, 3), (16, 13, 12))  # touches the face
    assert e.value.status == binding.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError):
        lbm.Refinement(lat, (5, 4, 3), (7, 13, 12))   # two cells
    # a fine lattice of the wrong viscosity or size, through the C ABI
    import ctypes as C
    L = lbm.lib()
    r = C.c_void_p()
    lo, hi = (C.c_int32 * 3)(5, 4, 3), (C.c_int32 * 3)(16, 13, 12)
    wrong_nu = lbm.Lattice((24, 20, 20), 0.02, storage="fp32")
    assert L.lbm_refine_create(lat._ctx, wrong_nu._ctx, lo, hi, C.byref(r)) == binding.LBM_ERR_ARG
    wrong_shape = lbm.Lattice((24, 20, 22), 0.04, storage="fp32")
    assert L.lbm_refine_create(lat._ctx, wrong_shape._ctx, lo, hi, C.byref(r)) == binding.LBM_ERR_ARG
    wrong_storage = lbm.Lattice((24, 20, 20), 0.04, storage="fp16")
    assert L.lbm_refine_create(lat._ctx, wrong_storage._ctx, lo, hi, C.byref(r)) == binding.LBM_ERR_ARG
    assert not r.value
    ref = lbm.Refinement(lat, (5, 4, 3), (16, 13, 12))
    with pytest.raises(lbm.LbmError) as e:
        ref.step(1)  # before init
    assert e.value.status == binding.LBM_ERR_STATE
    lat.init_state(*synth.uniform_fields((24, 20, 18)))
    ref.fine.init_state(*synth.uniform_fields(ref.fine.shape))
    ref.init()
    ref.step(1)
    lat.set_geometry(lbm.sphere((3.3, 3.4, 3.6), 1.5))  # a coarse body after the coupling
    with pytest.raises(lbm.LbmError) as e:
        ref.step(1)
    assert e.value.status == binding.LBM_ERR_STATE


def test_refined_block_bench_configuration_keeps_the_free_stream():
    """The refined block workload the bench times (512 x 256 x 64 coarse box
    with equilibrium inflow, outflow and far-field faces; fine block of
    512 x 256 x 96), FP32, through lbm_refine_step: the uniform free stream
    is a steady state, so every defined node of both levels keeps
    f^eq(1, u_inf) to FP32 rounding over 4 coarse steps."""
    import paper_1608_04658_gb300 as lbm
    wl = synth.refined_block()
    U = wl["u_face"]
    lat = lbm.Lattice(wl["shape"], wl["nu"], storage="fp32", faces=wl["faces"], u_face=U)
    ref = lbm.Refinement(lat, wl["lo"], wl["hi"])
    assert ref.fine.shape == wl["fine_shape"]
    lat.init_state(*synth.uniform_fields(wl["shape"], U))
    ref.fine.init_state(*synth.uniform_fields(wl["fine_shape"], U))
    ref.init()
    ref.step(4)
    fe = oracle.feq(1.0, U)
    (x0, y0, z0), (x1, y1, z1) = wl["lo"], wl["hi"]
    fc = lat.populations()
    vc = np.ones(fc.shape[1:], dtype=bool)
    vc[z0 + 2:z1 - 1, y0 + 2:y1 - 1, x0 + 2:x1 - 1] = False
    for i in range(27):
        assert np.abs(fc[i][vc] / fe[i] - 1.0).max() < 1e-6, i
    del fc
    ff = ref.fine.populations()
    for i in range(27):
        assert np.abs(ff[i, :-1, :-1, :-1] / fe[i] - 1.0).max() < 1e-6, i


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16"])
def test_refined_block_with_a_free_sphere(storage):
    """A free sphere (fine units: centre (11.3, 9.4, 9.6), radius 2.6,
    density ratio 2, launched at (0.02, 0.005, 0)) on the fine level of a
    block over [6, 17] x [5, 14]^2 of a 24 x 20 x 20 periodic box, rough
    random states, 6 coarse steps (12 steps of the sphere): populations on
    both levels, the sphere's solid marks, force and velocity against the
    oracle."""
    import paper_1608_04658_gb300 as lbm
    shape, lo, hi, nu = (24, 20, 20), (6, 5, 5), (17, 14, 14), 0.02
    Xf, R, U = (11.3, 9.4, 9.6), 2.6, (0.02, 0.005, 0.0)
    rho, u, xi, amp = random_fields(shape, 31)
    lat = lbm.Lattice(shape, nu, storage=storage)
    ref = lbm.Refinement(lat, lo, hi)
    ref.fine.set_geometry(lbm.sphere(Xf, R, U=U, free=True, rho_ratio=2.0))
    frho, fu, fxi, famp = random_fields(ref.fine.shape, 131)
    lat.init_state(rho, 0.2 * u, xi, amp)
    ref.fine.init_state(frho, 0.2 * fu, fxi, famp)
    ref.init()
    ref.step(6)
    F, _ = ref.fine.forces()
    body = ref.fine.body()

    orc = oracle.Oracle(shape, nu=nu)
    orc.init_state(rho, 0.2 * u, xi, amp)
    ro = oracle.RefinedOracle(orc, lo, hi, fine_body=oracle.sphere_body(Xf, R, U=U, free=True, rho_ratio=2.0))
    ro.fine.init_state(frho, 0.2 * fu, fxi, famp)
    ro.init()
    ro.step(6)
    # the sphere's marks inside the block (the surface and pad carry the
    # fine level's own solid marks)
    inner = np.zeros(ro.fine_valid().shape, dtype=bool)
    inner[1:-2, 1:-2, 1:-2] = True
    solid = (ref.fine.flags.cpu().numpy() & 1).astype(bool) & inner
    assert solid.sum() > 0
    assert np.array_equal(solid, ro.fine.solid().astype(bool) & inner)
    fluid = ro.fine_valid() & ~solid
    assert rel_err(lat.populations(), orc.get_f(), ro.coarse_valid()) <= TOL[storage]
    assert rel_err(ref.fine.populations(), ro.fine.get_f(), fluid) <= TOL[storage]
    Fo, Uo = np.array(ro.fine.body.F), np.array(ro.fine.body.U)
    fbar = {"fp64": 1e-10, "fp32": 1e-5, "fp16": 2e-2}[storage]
    assert np.abs(np.array(F) - Fo).max() <= fbar * np.abs(Fo).max()
    assert np.abs(np.array(body["U"]) - Uo).max() <= fbar * np.abs(Uo).max()


def test_refinement_rejects_an_airfoil_on_the_fine_level():
    import paper_1608_04658_gb300 as lbm
    from paper_1608_04658_gb300 import binding
    lat = lbm.Lattice((24, 20, 20), 0.02, storage="fp32")
    ref = lbm.Refinement(lat, (6, 5, 5), (17, 14, 14))
    wl = synth.plunging_airfoil()
    ref.fine.set_geometry(lbm.airfoil((6.3, 9.1), 8.0, wl["ca"], wl["sa"], 0.0, 0.0, wl["camber_m"],
                                      wl["camber_p"], wl["thick"]))
    lat.init_state(*synth.uniform_fields((24, 20, 20)))
    ref.fine.init_state(*synth.uniform_fields(ref.fine.shape))
    with pytest.raises(lbm.LbmError) as e:
        ref.init()
    assert e.value.status == binding.LBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16"])
def test_spanning_block_matches_the_oracle(storage):
    """A block over [4, 11] x [3, 8] spanning the periodic z axis of a 16 x 12
    x 10 box (fine lattice 16 x 12 x 20, periodic along z, the surface
    interpolation wrapping there), rough random states, 4 coarse steps."""
    lat, ref, orc, ro = run_refined((16, 12, 10), 0.02, storage, (4, 3, 0), (11, 8, 10), 4, seed=17)
    assert ref.full == (False, False, True) and ref.fine.shape == (16, 12, 20)
    ec, ef = errors(lat, ref, orc, ro)
    assert ec <= TOL[storage] and ef <= TOL[storage], (storage, ec, ef)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_refined_plunging_airfoil(storage):
    """The paper's two-level airfoil grid (Sec. 4.2) at small size: a
    plunging cambered airfoil (chord 16 fine nodes) on the fine level of a
    block over [12, 35] x [8, 23] spanning the periodic span of a 48 x 32 x 4
    box with equilibrium inflow, outflow and far field, impulsive start, 6
    coarse steps: both levels' populations, the airfoil's marks and its force
    against the oracle."""
    import math

    import paper_1608_04658_gb300 as lbm
    nu, U = 0.01, (0.05, 0.0, 0.0)
    shape, lo, hi, faces = (48, 32, 4), (12, 8, 0), (35, 23, 4), (2, 3, 2, 2, 0, 0)
    wl = synth.plunging_airfoil()
    chord, le = 16.0, (14.3, 15.2)
    args = (chord, wl["ca"], wl["sa"], 0.05 * chord, 2 * math.pi * 0.01, wl["camber_m"], wl["camber_p"], wl["thick"])
    lat = lbm.Lattice(shape, nu, storage=storage, faces=faces, u_face=U)
    ref = lbm.Refinement(lat, lo, hi)
    ref.fine.set_geometry(lbm.airfoil(le, *args))
    lat.init_state(*synth.uniform_fields(shape, U))
    ref.fine.init_state(*synth.uniform_fields(ref.fine.shape, U))
    ref.init()
    ref.step(6)
    F, _ = ref.fine.forces()

    orc = oracle.Oracle(shape, nu=nu, faces=faces, u_face=U)
    orc.init_state(*synth.uniform_fields(shape, U))
    ro = oracle.RefinedOracle(orc, lo, hi, fine_body=oracle.airfoil_body(le, *args))
    ro.fine.init_state(*synth.uniform_fields(ro.fine.shape, U))
    ro.init()
    ro.step(6)
    inner = np.zeros(ro.fine_valid().shape, dtype=bool)
    inner[:, 1:-2, 1:-2] = True
    solid = (ref.fine.flags.cpu().numpy() & 1).astype(bool) & inner
    assert solid.sum() > 0
    assert np.array_equal(solid, ro.fine.solid().astype(bool) & inner)
    assert rel_err(lat.populations(), orc.get_f(), ro.coarse_valid()) <= TOL[storage]
    assert rel_err(ref.fine.populations(), ro.fine.get_f(), ro.fine_valid() & ~solid) <= TOL[storage]
    Fo = np.array(ro.fine.body.F)
    ftol = 1e-10 if storage == "fp64" else 1e-5
    assert np.abs(np.array(F) - Fo).max() <= ftol * np.abs(Fo).max()


def test_refined_run_resumes_bitwise(tmp_path):
    """Both levels saved with lbm_save and the coupling with lbm_refine_save
    after 3 coarse steps; fresh contexts loaded from the files continue the
    next 3 steps to the same bits on every node the refined step defines."""
    import paper_1608_04658_gb300 as lbm
    shape, lo, hi = (24, 20, 18), (5, 4, 3), (16, 13, 12)
    rho, u, xi, amp = random_fields(shape, 41)
    lat = lbm.Lattice(shape, 0.02, storage="fp32")
    ref = lbm.Refinement(lat, lo, hi)
    frho, fu, fxi, famp = random_fields(ref.fine.shape, 141)
    lat.init_state(rho, u, xi, amp)
    ref.fine.init_state(frho, fu, fxi, famp)
    ref.init()
    ref.step(3)
    pc, pf, pr = (str(tmp_path / n) for n in ("coarse.bin", "fine.bin", "coupling.bin"))
    lat.save(pc)
    ref.fine.save(pf)
    ref.save(pr)
    ref.step(3)
    fc, ff = lat.populations(), ref.fine.populations()

    lat2 = lbm.Lattice(shape, 0.02, storage="fp32")
    ref2 = lbm.Refinement(lat2, lo, hi)
    lat2.load(pc)
    ref2.fine.load(pf)
    ref2.load(pr)
    ref2.step(3)
    vc = np.ones(fc.shape[1:], dtype=bool)
    vc[lo[2] + 2:hi[2] - 1, lo[1] + 2:hi[1] - 1, lo[0] + 2:hi[0] - 1] = False
    assert np.array_equal(lat2.populations()[:, vc], fc[:, vc])
    assert np.array_equal(ref2.fine.populations()[:, :-1, :-1, :-1], ff[:, :-1, :-1, :-1])
    # a coupling of another block refuses the file
    from paper_1608_04658_gb300 import binding
    ref3 = lbm.Refinement(lbm.Lattice(shape, 0.02, storage="fp32"), lo, (15, 13, 12))
    with pytest.raises(lbm.LbmError) as e:
        ref3.load(pr)
    assert e.value.status == binding.LBM_ERR_ARG
