"""GPU adjoint (lbm_adjoint_step) against independent references:
  - the PyTorch FP64 tape (oracle/tape.py) differentiated by autograd, for the
    gradient of a terminal functional with respect to the initial state on
    bodiless boxes (periodic, walls, equilibrium/outflow faces; KBC and LBGK);
  - central finite differences of the GPU forward (dot-product test) with a
    held sphere and with the deforming swimmer (Grad boundary, refill and
    momentum-exchange adjoints);
  - central finite differences of the FP64 oracle for the gradient of the
    swimmer's mean thrust with respect to (wave amplitude, wavelength, period)
    on a 48x24x24 box over 8 steps, and of the airfoil's mean lift with respect
    to the plunge amplitude and frequency, the link set being the same at
    theta +- h.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import tape

pytestmark = pytest.mark.gpu


def _lat(shape, nu, storage="fp64", faces=(0,) * 6, u_face=(0.0, 0.0, 0.0), gamma_mode=0):
    import paper_1608_04658_gb300 as lbm
    return lbm.Lattice(shape, nu, storage=storage, faces=faces, u_face=u_face, gamma_mode=gamma_mode)


@pytest.mark.parametrize("faces,lbgk", [((0,) * 6, False), ((1, 1, 0, 0, 0, 0), False),
                                         ((2, 3, 2, 2, 0, 0), False), ((0,) * 6, True)])
def test_initial_state_gradient_matches_tape(faces, lbgk):
    shape = (8, 7, 6)
    nu, H = 0.02, 3
    u_face = (0.03, 0.0, 0.0)
    lat = _lat(shape, nu, faces=faces, u_face=u_face, gamma_mode=2 if lbgk else 0)
    rho, u, xi = synth.parity_fields(shape, 31)
    lat.init_state(rho, u, xi, 1e-3)
    f0 = lat.populations()
    rng = np.random.default_rng(5)
    lamT = rng.normal(size=(27,) + shape[::-1])
    out = lat.adjoint(H, lambda_T=torch.tensor(lamT, device=lat.device), want_lambda0=True)
    box = tape.Box(shape, faces, u_face=u_face)
    ft = torch.tensor(f0, dtype=torch.float64, requires_grad=True)
    f = ft
    for _ in range(H):
        f = box.step(f, oracle.beta_from_nu(nu), lbgk)
    J = (f * torch.tensor(lamT)).sum()
    J.backward()
    ref = ft.grad.numpy()
    got = out["lambda_0"].cpu().numpy()
    assert out["J"] == pytest.approx(J.item(), rel=1e-12)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def _swimmer_geom(L=24.0, X=(12.137, 12.371, 12.293), theta=(0.125, 24.0, 96.0), segments=48, ring=16,
                  free=False, mass_scale=1.0, U=(0.0, 0.0, 0.0), psi=0.0, omega=0.0):
    import paper_1608_04658_gb300 as lbm
    rest, tris = synth.swimmer_mesh(L, segments, ring)
    a, lam, T = theta
    return lbm.swimmer(X, rest, tris, L, a, lam, T, mass=mass_scale * synth.swimmer_volume(L), free=free, U=U,
                       psi=psi, omega=omega)


def _dot_product_check(shape, geom_fn, storage="fp64", H=4, seed=41):
    lat = _lat(shape, 0.02, storage=storage)
    lat.set_geometry(geom_fn())
    rho, u, xi = synth.parity_fields(shape, seed)
    lat.init_state(rho, 0.3 * u, xi, 1e-3)
    f0 = lat.populations()
    fluid0 = (lat.flags.cpu().numpy() & 1) == 0
    rng = np.random.default_rng(seed)
    _, W = oracle.lattice()
    lamT = rng.normal(size=(27,) + shape[::-1])
    w = np.array([0.7, -1.3, 0.4])
    out = lat.adjoint(H, w, lambda_T=torch.tensor(lamT, device=lat.device), want_lambda0=True)
    lam0 = out["lambda_0"].cpu().numpy()
    delta = rng.normal(size=f0.shape) * W[:, None, None, None] * fluid0[None]
    # central differences at eps and 2 eps combined to cancel their eps^2
    # error (the stabilizer makes J strongly curved: the plain difference at
    # 1e-5 is off by ~1e-7 relative, shrinking as eps^2)
    eps = 1e-4

    def J_at(f):
        l2 = _lat(shape, 0.02, storage=storage)
        l2.set_geometry(geom_fn())
        l2.set_populations(f)
        r = l2.adjoint(H, w, lambda_T=torch.tensor(lamT, device=l2.device))
        b = l2.body()
        l2.close()
        return r["J"], (b["n_boundary"], b["n_links"], b["n_uncovered"])

    fds = []
    for e in (eps, 2 * eps):
        Jp, cp = J_at(f0 + e * delta)
        Jm, cm = J_at(f0 - e * delta)
        assert cp == cm
        fds.append((Jp - Jm) / (2 * e))
    fd = (4 * fds[0] - fds[1]) / 3
    ad = float((lam0 * delta).sum())
    return ad, fd


def test_dot_product_with_held_sphere():
    import paper_1608_04658_gb300 as lbm
    ad, fd = _dot_product_check((14, 13, 12), lambda: lbm.sphere((6.6, 6.3, 5.8), 2.9))
    assert ad == pytest.approx(fd, rel=1e-7)


def test_dot_product_with_free_sphere():
    """A sphere free in x, y and z under gravity (Sec. 4.1, explicit Euler with
    buoyancy) and walls in x and y: the adjoint carries its position and
    velocity backwards (links' q through the centre, u_w = U, refill
    velocity U); initial-state gradient vs central differences."""
    import paper_1608_04658_gb300 as lbm
    ad, fd = _dot_product_check((14, 13, 12), lambda: lbm.sphere((6.6, 6.3, 5.8), 2.9, U=(0.004, -0.003, -0.01),
                                                                  free=True, rho_ratio=1.2, g=(0.0, 0.0, -5e-4)))
    assert ad == pytest.approx(fd, rel=1e-7)


def test_dot_product_with_deforming_swimmer():
    ad, fd = _dot_product_check((48, 24, 24), _swimmer_geom)
    assert ad == pytest.approx(fd, rel=1e-7)


def test_dot_product_with_free_swimmer():
    """The swimmer free along x (Sec. 4.3 Newton equation, explicit Euler):
    the adjoint carries the head's position and velocity backwards, so the
    initial-state gradient includes the force -> velocity -> pose -> flow
    feedback."""
    ad, fd = _dot_product_check((48, 24, 24), lambda: _swimmer_geom(free=True, mass_scale=0.25,
                                                                    U=(-0.01, 0.0, 0.0)))
    assert ad == pytest.approx(fd, rel=1e-7)


def _oracle_thrust(shape, theta, fields, H, w, L=24.0, X=(12.137, 12.371, 12.293), segments=48, ring=16,
                   free=False, mass_scale=1.0, U=(0.0, 0.0, 0.0), psi=0.0, omega=0.0):
    rest, tris = synth.swimmer_mesh(L, segments, ring)
    a, lam, T = theta
    o = oracle.Oracle(shape, nu=0.02, body=oracle.mesh_body(X, rest, tris, L, a, lam, T, U=U, free=free,
                                                           mass=mass_scale * synth.swimmer_volume(L),
                                                           psi=psi, omega=omega))
    rho, u, xi, amp = fields
    o.init_state(rho, u, xi, amp)
    J = 0.0
    counts = []
    for _ in range(H):
        o.step(1)
        J += float(np.dot(w, np.array(o.body.F)))
        counts.append((o.counters()["boundary"], o.counters()["links"], o.counters()["refill"]))
    return J / H, counts, o.solid()


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-6), ("fp32", 1e-4), ("fp16", 2e-5), ("bf16", 3e-4)])
def test_swimmer_thrust_gradient_matches_oracle_fd(storage, tol):
    """Sec. 4.3 kinematics: d(mean thrust)/d(amplitude, wavelength, period)
    from the GPU adjoint vs central differences of the FP64 oracle, in every
    storage form (16-bit: the states and checkpoints in the storage type, the
    adjoint in FP32, the stores' rounding passed through)."""
    shape, H = (48, 24, 24), 8
    theta = np.array([0.125, 24.0, 96.0])
    w = np.array([-1.0, 0.0, 0.0])  # swimming towards -x: thrust = -F_x
    rho, u, xi = synth.parity_fields(shape, 43)
    fields = (rho, 0.2 * u, xi, 1e-3)
    lat = _lat(shape, 0.02, storage=storage)
    lat.set_geometry(_swimmer_geom(theta=tuple(theta)))
    lat.init_state(*fields)
    out = lat.adjoint(H, w)
    J0, _, _ = _oracle_thrust(shape, theta, fields, H, w)
    jrel = {"fp64": 1e-9, "fp32": 1e-6, "fp16": 1e-5, "bf16": 5e-4}[storage]
    print(f"{storage}: J rel err {abs(out['J'] - J0) / abs(J0):.2e}")
    assert out["J"] == pytest.approx(J0, rel=jrel)
    fd = np.zeros(3)
    for k in range(3):
        h = 1e-6 * theta[k]
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        Jp, cp, sp = _oracle_thrust(shape, tp, fields, H, w)
        Jm, cm, sm = _oracle_thrust(shape, tm, fields, H, w)
        assert cp == cm and np.array_equal(sp, sm), "link set changed within the difference step"
        fd[k] = (Jp - Jm) / (2 * h)
    g = out["dJ_dtheta"]
    assert np.all(np.abs(fd) > 0)
    print(f"{storage}: gradient err {np.abs(g - fd).max() / np.abs(fd).max():.2e}")
    assert np.abs(g - fd).max() <= tol * np.abs(fd).max()


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_free_swimmer_thrust_gradient_matches_oracle_fd(storage, tol):
    """As above with the swimmer free along x and a light body (mass a quarter
    of the displaced fluid's), so the kinematics also change the head's path:
    d(mean thrust)/d(theta) from the GPU adjoint, which carries (X0, U0) as
    adjoint state, vs central differences of the FP64 oracle."""
    shape, H = (48, 24, 24), 8
    theta = np.array([0.125, 24.0, 96.0])
    w = np.array([-1.0, 0.0, 0.0])
    kw = dict(free=True, mass_scale=0.25, U=(-0.01, 0.0, 0.0))
    rho, u, xi = synth.parity_fields(shape, 47)
    fields = (rho, 0.2 * u, xi, 1e-3)
    lat = _lat(shape, 0.02, storage=storage)
    lat.set_geometry(_swimmer_geom(theta=tuple(theta), **kw))
    lat.init_state(*fields)
    out = lat.adjoint(H, w)
    b = lat.body()
    J0, _, _ = _oracle_thrust(shape, theta, fields, H, w, **kw)
    assert out["J"] == pytest.approx(J0, rel=1e-9 if storage == "fp64" else 1e-6)
    assert b["X"][0] != 12.137  # the head moved
    fd = np.zeros(3)
    for k in range(3):
        h = 1e-6 * theta[k]
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        Jp, cp, sp = _oracle_thrust(shape, tp, fields, H, w, **kw)
        Jm, cm, sm = _oracle_thrust(shape, tm, fields, H, w, **kw)
        assert cp == cm and np.array_equal(sp, sm), "link set changed within the difference step"
        fd[k] = (Jp - Jm) / (2 * h)
    g = out["dJ_dtheta"]
    assert np.all(np.abs(fd) > 0)
    assert np.abs(g - fd).max() <= tol * np.abs(fd).max()
    # the held swimmer's gradient differs: the feedback through the head's path counts
    held = _lat(shape, 0.02, storage=storage)
    held.set_geometry(_swimmer_geom(theta=tuple(theta), mass_scale=0.25, U=(-0.01, 0.0, 0.0)))
    held.init_state(*fields)
    assert np.abs(held.adjoint(H, w)["dJ_dtheta"] - g).max() > 10 * tol * np.abs(fd).max()


# the swimmer in the centre-of-mass frame: X is its centre of mass
_COM = dict(X=(24.137, 12.371, 12.293), mass_scale=1.0, U=(-0.01, 0.004, 0.0), psi=0.1, omega=0.003)


def test_dot_product_with_three_dof_swimmer():
    """Swimmer free in x, y and yaw (centre-of-mass frame): the adjoint carries
    the centre of mass, its velocity, the yaw angle and the angular momentum
    backwards through the Euler update; initial-state gradient vs central
    differences of the GPU forward."""
    ad, fd = _dot_product_check((48, 24, 24), lambda: _swimmer_geom(free=7, **_COM))
    assert ad == pytest.approx(fd, rel=1e-7)


@pytest.mark.parametrize("free,storage,tol", [(3, "fp64", 1e-6), (4, "fp64", 1e-6), (7, "fp64", 1e-6),
                                              (7, "fp32", 1e-4)])
def test_com_frame_swimmer_thrust_gradient_matches_oracle_fd(free, storage, tol):
    """Mean-thrust gradient of the swimmer free in x and y (3), in yaw (4) or
    in x, y and yaw (7): the pose X + R(psi)(b - c(t)) moves with theta
    through the midline and the centre of mass c and, with yaw free, through
    omega = L / I(theta) (the initial L = I(t0) omega_0 included); GPU adjoint
    vs central differences of the FP64 oracle."""
    shape, H = (48, 24, 24), 8
    theta = np.array([0.125, 24.0, 96.0])
    w = np.array([-1.0, 0.0, 0.0])
    kw = dict(free=free, **_COM)
    rho, u, xi = synth.parity_fields(shape, 53)
    fields = (rho, 0.2 * u, xi, 1e-3)
    lat = _lat(shape, 0.02, storage=storage)
    lat.set_geometry(_swimmer_geom(theta=tuple(theta), **kw))
    lat.init_state(*fields)
    out = lat.adjoint(H, w)
    J0, _, _ = _oracle_thrust(shape, theta, fields, H, w, **kw)
    assert out["J"] == pytest.approx(J0, rel=1e-9 if storage == "fp64" else 1e-6)
    fd = np.zeros(3)
    for k in range(3):
        h = 1e-6 * theta[k]
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        Jp, cp, sp = _oracle_thrust(shape, tp, fields, H, w, **kw)
        Jm, cm, sm = _oracle_thrust(shape, tm, fields, H, w, **kw)
        assert cp == cm and np.array_equal(sp, sm), "link set changed within the difference step"
        fd[k] = (Jp - Jm) / (2 * h)
    g = out["dJ_dtheta"]
    assert np.all(np.abs(fd) > 0)
    assert np.abs(g - fd).max() <= tol * np.abs(fd).max()


def _airfoil_case(theta, t0=3.0):
    wl = synth.plunging_airfoil()
    A, w_ = theta
    args = ((24.37, 20.29), 32.0, wl["ca"], wl["sa"], A, w_, wl["camber_m"], wl["camber_p"], wl["thick"], t0)
    return wl, args


def _oracle_airfoil(shape, theta, fields, H, w):
    wl, args = _airfoil_case(theta)
    o = oracle.Oracle(shape, nu=0.02, faces=wl["faces"], u_face=wl["u_face"], body=oracle.airfoil_body(*args))
    o.init_state(*fields)
    J, counts = 0.0, []
    for _ in range(H):
        o.step(1)
        J += float(np.dot(w, np.array(o.body.F)))
        c = o.counters()
        counts.append((c["boundary"], c["links"], c["refill"]))
    return J / H, counts, o.solid()


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_airfoil_lift_gradient_matches_oracle_fd(storage, tol):
    """Sec. 4.2 plunge: d(mean lift)/d(amplitude, angular frequency) from the
    GPU adjoint vs central differences of the FP64 oracle, with equilibrium
    inflow, outflow and far-field faces and refilled nodes."""
    import paper_1608_04658_gb300 as lbm
    shape, H = (96, 40, 6), 8
    theta = np.array([1.6, 0.05])
    w = np.array([0.0, 1.0, 0.0])
    rho, u, xi = synth.parity_fields(shape, 59)
    fields = (rho, 0.2 * u + np.array([0.05, 0.0, 0.0]), xi, 1e-3)
    wl, args = _airfoil_case(theta)
    lat = _lat(shape, 0.02, storage=storage, faces=wl["faces"], u_face=wl["u_face"])
    lat.set_geometry(lbm.airfoil(*args))
    lat.init_state(*fields)
    out = lat.adjoint(H, w)
    J0, c0, _ = _oracle_airfoil(shape, theta, fields, H, w)
    assert sum(c[2] for c in c0) > 0  # nodes get refilled
    assert out["J"] == pytest.approx(J0, rel=1e-9 if storage == "fp64" else 1e-6)
    fd = np.zeros(2)
    for k in range(2):
        h = 1e-6 * theta[k]
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        Jp, cp, sp = _oracle_airfoil(shape, tp, fields, H, w)
        Jm, cm, sm = _oracle_airfoil(shape, tm, fields, H, w)
        assert cp == cm and np.array_equal(sp, sm), "link set changed within the difference step"
        fd[k] = (Jp - Jm) / (2 * h)
    g = out["dJ_dtheta"][:2]
    assert out["dJ_dtheta"][2] == 0.0
    assert np.abs(g - fd).max() <= tol * np.abs(fd).max()


def test_checkpoint_interval_does_not_change_the_result():
    shape, H = (48, 24, 24), 12
    rho, u, xi = synth.parity_fields(shape, 47)
    res = []
    for K in (1, 4, 12, 0):
        lat = _lat(shape, 0.02)
        lat.set_geometry(_swimmer_geom())
        lat.init_state(rho, 0.2 * u, xi, 1e-3)
        out = lat.adjoint(H, (-1.0, 0.0, 0.0), want_lambda0=True, checkpoint_every=K)
        res.append((out["J"], out["dJ_dtheta"], out["lambda_0"].cpu().numpy(), lat.populations()))
        lat.close()
    for J, g, l0, f in res[1:]:
        assert J == res[0][0]
        assert np.allclose(g, res[0][1], rtol=1e-12, atol=0)
        assert np.abs(l0 - res[0][2]).max() <= 1e-12 * np.abs(res[0][2]).max()
        assert np.array_equal(f, res[0][3])


def test_autograd_function_returns_the_adjoint_gradient():
    import paper_1608_04658_gb300 as lbm
    shape, H = (48, 24, 24), 4
    rho, u, xi = synth.parity_fields(shape, 53)

    def make(theta):
        lat = _lat(shape, 0.02)
        lat.set_geometry(_swimmer_geom(theta=tuple(float(v) for v in theta)))
        lat.init_state(rho, 0.2 * u, xi, 1e-3)
        return lat

    f = lbm.kinematics_objective(make, H, (-1.0, 0.0, 0.0))
    theta = torch.tensor([0.125, 24.0, 96.0], dtype=torch.float64, requires_grad=True)
    J = f(theta)
    J.backward()
    lat = make(theta.detach().numpy())
    ref = lat.adjoint(H, (-1.0, 0.0, 0.0))
    assert J.item() == pytest.approx(ref["J"], rel=1e-13)
    assert np.allclose(theta.grad.numpy(), ref["dJ_dtheta"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_adjoint_near_rest_is_finite(storage):
    """A swimmer starting in fluid at rest: <dh|dh> is tiny at most nodes,
    where the stabilizer's derivative must not underflow to inf/NaN."""
    shape, H = (48, 24, 24), 6
    lat = _lat(shape, 0.02, storage=storage)
    lat.set_geometry(_swimmer_geom())
    lat.init_state(*synth.uniform_fields(shape))
    out = lat.adjoint(H, (-1.0, 0.0, 0.0), want_lambda0=True)
    assert np.isfinite(out["J"]) and np.all(np.isfinite(out["dJ_dtheta"]))
    assert torch.isfinite(out["lambda_0"]).all()
    assert np.abs(out["dJ_dtheta"]).max() > 0


@pytest.mark.parametrize("kind", ["sphere", "swimmer"])
def test_adjoint_launch_orders_agree(kind):
    """The split and the sequential launch order (forward, recomputed segments
    and reversed steps) give the same J, dJ/dtheta and lambda_0 (to the
    rounding of the band buffer's atomic sums)."""
    import paper_1608_04658_gb300 as lbm
    shape = (48, 24, 24) if kind == "swimmer" else (14, 13, 12)
    rho, u, xi = synth.parity_fields(shape, 61)
    outs = {}
    for order in ("split", "sequential"):
        lat = _lat(shape, 0.02, storage="fp64")
        lat.set_launch_order(order)
        if kind == "swimmer":
            lat.set_geometry(_swimmer_geom(free=True, U=(-0.01, 0.0, 0.0)))
        else:
            lat.set_geometry(lbm.sphere((6.6, 6.3, 5.8), 2.9, U=(0.004, -0.003, -0.01), free=True, rho_ratio=1.2,
                                        g=(0.0, 0.0, -5e-4)))
        lat.init_state(rho, 0.3 * u, xi, 1e-3)
        outs[order] = lat.adjoint(6, (-1.0, 0.3, 0.2), want_lambda0=True, checkpoint_every=2)
    a, b = outs["split"], outs["sequential"]
    assert a["J"] == pytest.approx(b["J"], rel=1e-13)
    assert np.allclose(a["dJ_dtheta"], b["dJ_dtheta"], rtol=1e-11, atol=1e-14)
    la, lb = a["lambda_0"].cpu().numpy(), b["lambda_0"].cpu().numpy()
    assert np.abs(la - lb).max() <= 1e-11 * np.abs(la).max()


def test_adjoint_rejects_the_exact_stabilizer():
    import paper_1608_04658_gb300 as lbm
    lat = _lat((12, 12, 12), 0.05, storage="fp32", gamma_mode=lbm.GAMMA_EXACT)
    lat.init_state(*synth.uniform_fields((12, 12, 12)))
    with pytest.raises(lbm.LbmError):
        lat.adjoint(2)
