"""Pins of the oracle's triangulated swimmer (Sec. 4.3): the closed mesh of
elliptic cross sections, the prescribed midline deformation, the ray-parity
solid test, the link fraction and barycentric wall velocity, the momentum
balance and the Euler update along the swimming axis.  Each is checked against
the analytic body, the paper's printed amplitudes or an exact invariant."""
import math

import numpy as np
import pytest

import synth


def _body(orc, L, segments, ring, X, amp=0.0, period=64.0, **kw):
    rest, tris = synth.swimmer_mesh(L, segments, ring)
    return orc.mesh_body(X, rest, tris, L, amp, L, period, mass=synth.swimmer_volume(L), **kw)


def test_synth_mesh_is_closed_and_encloses_the_analytic_volume():
    """Every directed edge appears once and its reverse once (a closed,
    consistently oriented surface); the divergence-theorem volume approaches
    the integral of pi w h (Sec. 4.3 cross sections) from below."""
    L = 128.0
    rest, tris = synth.swimmer_mesh(L)
    assert len(tris) == 19200  # 150 segments x 64 x 2, head fan and tail cap
    edges = {}
    for a, b, c in tris:
        for u, v in ((a, b), (b, c), (c, a)):
            edges[(u, v)] = edges.get((u, v), 0) + 1
    assert max(edges.values()) == 1
    assert all((v, u) in edges for (u, v) in edges)
    P = rest
    vol = np.einsum("ij,ij->i", P[tris[:, 0]], np.cross(P[tris[:, 1]], P[tris[:, 2]])).sum() / 6.0
    ref = synth.swimmer_volume(L)
    assert 0.98 * ref < vol < ref
    # printed half axes: w_h = 0.04 L at s_b = 0.04 L, tail width 0.01 L at 0.95 L,
    # height b = 0.08 L at s = a = 0.51 L
    assert synth.swimmer_half_width(0.04 * L, L) == pytest.approx(0.04 * L)
    assert synth.swimmer_half_width(0.95 * L, L) == pytest.approx(0.01 * L)
    assert synth.swimmer_half_width(L, L) == 0.0
    assert synth.swimmer_half_height(0.51 * L, L) == pytest.approx(0.08 * L)


def test_midline_amplitudes_and_travelling_wave(orc):
    """Sec. 4.3 midline: lateral amplitude 0.125 L at the tail and
    0.125 L * 0.03125/1.03125 at the head; the wave moves one wavelength per
    period towards the tail; the pose repeats after one period."""
    L, T = 40.0, 64.0
    shape = (72, 40, 24)
    X = (16.137, 20.371, 12.293)
    o = orc.Oracle(shape, nu=0.02, body=_body(orc, L, 20, 8, X, amp=0.125, period=T))
    rest = o.body
    n = rest.n_vertices
    head, tail = 0, n - 1
    ys_head, ys_tail, poses = [], [], []
    for k in range(int(T)):
        pos, _ = o.mesh_pose()
        ys_head.append(pos[head, 1] - X[1])
        ys_tail.append(pos[tail, 1] - X[1])
        poses.append(pos.copy())
        o.step_sampled([0])  # advances the pose, state untouched except refill
    assert max(np.abs(ys_tail)) == pytest.approx(0.125 * L, rel=2e-3)
    assert max(np.abs(ys_head)) == pytest.approx(0.125 * L * 0.03125 / 1.03125, rel=2e-3)
    pos, _ = o.mesh_pose()
    assert np.abs(pos - poses[0]).max() < 1e-12
    # travelling wave: y(s, t + T/4) / A(s) = y(s - lambda/4, t) / A(s - lambda/4)
    r, _ = synth.swimmer_mesh(L, 20, 8)
    s = r[:, 0]
    env = 0.125 * L * (s / L + 0.03125) / 1.03125
    ring0 = 1 + 8 * np.arange(20)  # position 0 of each of the 20 rings of 8 vertices
    ss = s[ring0]
    y0 = (poses[0][ring0, 1] - X[1] - r[ring0, 1]) / env[ring0]
    y1 = (poses[int(T // 4)][ring0, 1] - X[1] - r[ring0, 1]) / env[ring0]
    shifted = ss + L / 4
    ok = shifted <= L
    assert np.abs(np.interp(shifted[ok], ss, y1) - y0[ok]).max() < 0.02


@pytest.mark.parametrize("amp,t0", [(0.0, 0.0), (0.125, 9.0)])
def test_ray_parity_solid_test_matches_analytic_body(orc, amp, t0):
    """A node is solid when it lies inside the elliptic cross section of the
    (displaced) centre line at s = x - X0; nodes clearly inside or outside the
    analytic surface (10% margin) are classified by ray parity accordingly,
    and the solid count approaches the analytic volume."""
    L, T = 48.0, 64.0
    shape = (72, 48, 24)
    X = (12.137, 24.371, 12.293)
    body = _body(orc, L, 150, 96, X, amp=amp, period=T, t0=t0)
    o = orc.Oracle(shape, nu=0.02, body=body)
    solid = o.solid().astype(bool)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in shape[::-1]], indexing="ij")
    s = x - X[0]
    w = synth.swimmer_half_width(np.clip(s, 0, L), L)
    h = synth.swimmer_half_height(np.clip(s, 0, L), L)
    ymid = amp * L * (s / L + 0.03125) / 1.03125 * np.sin(2 * np.pi * (s / L - t0 / T))
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = ((y - X[1] - ymid) / w) ** 2 + ((z - X[2]) / h) ** 2
    core = (s > 2.0) & (s < L - 2.0)
    inside = core & (phi < 0.9)
    outside = (s < -0.5) | (s > L + 0.5) | (core & (phi > 1.1))
    assert inside.sum() > 300
    assert solid[inside].all()
    assert not solid[outside].any()
    vol = synth.swimmer_volume(L)
    assert abs(solid.sum() - vol) < 0.05 * vol


def test_link_fraction_and_wall_velocity_on_the_analytic_surface(orc):
    """Straight body translating with U (prescribed): for lateral links
    (c = +-e_y) the wall point lies on the elliptic cross section,
    y_w = Y + w(s) sqrt(1 - (dz/h(s))^2), and the barycentric wall velocity
    of equal vertex velocities is U."""
    L = 48.0
    shape = (64, 32, 24)
    X = (8.137, 16.371, 12.293)
    U = (0.013, -0.004, 0.002)
    o = orc.Oracle(shape, nu=0.02, body=_body(orc, L, 150, 256, X, U=U))
    solid = o.solid().astype(bool)
    c, _ = orc.lattice()
    iy = {+1: int(np.where((c == [0, 1, 0]).all(1))[0][0]), -1: int(np.where((c == [0, -1, 0]).all(1))[0][0])}
    checked = 0
    for xx in range(int(X[0]) + 6, int(X[0] + L) - 6, 3):
        s = xx - X[0]
        w = float(synth.swimmer_half_width(s, L))
        h = float(synth.swimmer_half_height(s, L))
        for zz in range(24):
            dz = zz - X[2]
            if abs(dz) > 0.8 * h:
                continue
            yw = w * math.sqrt(1 - (dz / h) ** 2)
            for sign in (+1, -1):
                # fluid node just outside the wall on this side, solid node inside
                yb = int(math.floor(X[1] + sign * yw)) + (1 if sign > 0 else 0)
                ys = yb - sign
                if solid[zz, yb, xx] or not solid[zz, ys, xx]:
                    continue
                # link from x_b towards x_b - c_i = the solid node
                q, uw = o.mesh_link(xx, yb, zz, iy[sign])
                q_ref = abs(yb - (X[1] + sign * yw))
                assert q == pytest.approx(q_ref, abs=5e-3)
                assert np.abs(uw - U).max() < 1e-15
                checked += 1
    assert checked > 40


def test_vertex_velocity_is_central_difference_of_the_pose(orc):
    """Sec. 4.3 wall velocity by finite differences of the prescribed
    deformation: the vertex velocity at t equals (x(t+1) - x(t-1))/2 of the
    poses the oracle actually takes (prescribed body, no translation)."""
    L, T = 40.0, 32.0
    o = orc.Oracle((72, 40, 24), nu=0.02,
                   body=_body(orc, L, 20, 8, (16.137, 20.371, 12.293), amp=0.125, period=T, ramp=True))
    pos = []
    vel = []
    for _ in range(4):
        p, v = o.mesh_pose()
        pos.append(p)
        vel.append(v)
        o.step_sampled([0])
    for k in (1, 2):
        assert np.abs(vel[k] - 0.5 * (pos[k + 1] - pos[k - 1])).max() < 1e-13
    # ramp: the body starts straight
    rest = synth.swimmer_mesh(L, 20, 8)[0]
    assert np.abs(pos[0][:, 1] - 20.371 - rest[:, 1]).max() < 1e-13


def test_swimmer_momentum_exchange_balances_fluid_momentum(orc):
    """Fixed straight mesh in a periodic box: the fluid's momentum change in
    one step is exactly minus the momentum-exchange force (as for the sphere)."""
    shape = (40, 16, 16)
    o = orc.Oracle(shape, nu=0.05, body=_body(orc, 24.0, 24, 12, (8.137, 8.371, 8.293)))
    rho, u, xi = synth.parity_fields(shape, 9)
    o.init_state(rho, u * 0.5 + 0.02, xi, 1e-3)
    for _ in range(2):
        T0 = o.totals()
        o.step(1)
        T1 = o.totals()
        F = np.array(o.body.F)
        assert np.linalg.norm(F) > 0.01
        assert np.abs(T1[1:4] - T0[1:4] + F).max() < 1e-12 * T0[0]
        assert o.counters()["error"] == 0


def _moment_of_fluid(orc, f, fluid, X):
    """sum over fluid nodes of (x - X) x j(x), j = sum_i c_i f_i, with the
    node offsets taken as they are (no wrap): the disturbance never reaches
    the box faces in the tests below."""
    c, _ = orc.lattice()
    nz, ny, nx = fluid.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.stack([x - X[0], y - X[1], z - X[2]], axis=-1)
    j = np.einsum("ia,izyx->zyxa", c, f)
    return np.cross(r[fluid], j[fluid]).sum(0)


@pytest.mark.parametrize("free", [False, 4])
def test_swimmer_torque_balances_fluid_angular_momentum(orc, free):
    """Straight mesh at rest, held with the head as reference point, or free
    in yaw about its centre of mass with a mass so large that it does not
    turn: streaming keeps each population's moment about any point and the
    collision keeps j, so the change of the fluid's angular momentum about the
    reference point in one step is exactly minus the momentum-exchange torque.
    The disturbance lies within 5 nodes of the body and spreads one node per
    step, so the wrap at the box faces only moves rest-equilibrium
    populations, whose moments cancel."""
    ndimage = pytest.importorskip("scipy.ndimage")
    shape = (48, 24, 24)
    # the head (held) or the centre of mass (free in yaw)
    X = np.array([24.137 if free else 12.137, 12.371, 12.293])
    body = _body(orc, 24.0, 24, 12, X, free=free)
    if free:
        body.mass = 1e30
    o = orc.Oracle(shape, nu=0.05, body=body)
    Xref = np.array(o.body.X)
    assert np.array_equal(Xref, X)
    fluid = o.solid() == 0
    d = ndimage.distance_transform_edt(fluid)  # distance to the nearest solid node
    w = np.clip(5.0 - d, 0.0, 1.0)
    sol = np.argwhere(~fluid)
    for a, n in enumerate(shape[::-1]):
        # 5 nodes of disturbance, 2 steps of spread, and 1 node to spare
        assert sol[:, a].min() >= 8 and sol[:, a].max() <= n - 9
    rho, u, xi = synth.parity_fields(shape, 11, umax=0.08)
    o.init_state(1.0 + w * (rho - 1.0), w[..., None] * u, w[None] * xi, 1e-3)
    L0 = _moment_of_fluid(orc, o.get_f(), fluid, Xref)
    for _ in range(2):
        o.step(1)
        assert np.array_equal(np.array(o.body.X), Xref)
        L1 = _moment_of_fluid(orc, o.get_f(), fluid, Xref)
        M = np.array(o.body.M)
        assert np.linalg.norm(M) > 0.05
        # rounding of the sums over ~10^4 nodes; a wrong arm or sign is O(|M|)
        assert np.abs(L1 - L0 + M).max() < 1e-11 * np.linalg.norm(M) + 1e-12
        assert o.counters()["error"] == 0
        L0 = L1


def test_swimmer_euler_update_along_the_swimming_axis(orc):
    """Newton's equation along x by explicit Euler (Sec. 4.3 with Sec. 4.1's
    scheme): X0 += U0, U0 += F0/m; the lateral and vertical position of the
    centre line stay fixed."""
    shape = (48, 20, 20)
    X0 = np.array([10.137, 10.371, 10.293])
    U0 = 0.01
    m = 7.5
    body = _body(orc, 24.0, 24, 12, X0, amp=0.125, period=32.0, U=(U0, 0, 0), free=True)
    body.mass = m
    o = orc.Oracle(shape, nu=0.05, body=body)
    o.init_state(*synth.uniform_fields(shape, (0.01, 0.0, 0.0)))
    o.step(1)
    b1 = o.body
    assert b1.X[0] == pytest.approx(X0[0] + U0, abs=1e-15)
    assert list(b1.X[1:]) == list(X0[1:])
    assert b1.U[0] == U0
    F1 = b1.F[0]
    o.step(1)
    b2 = o.body
    assert b2.X[0] == pytest.approx(X0[0] + 2 * U0, abs=1e-14)
    assert b2.U[0] == pytest.approx(U0 + F1 / m, abs=1e-16)
    assert b2.t == 2.0


# ---------------------------------------------------------------- three degrees of freedom
def _box_mesh(a, b, c):
    """Closed, outward-oriented triangulation of the box [0,a]x[0,b]x[0,c] in the
    (s, dy, dz) rest format (12 triangles)."""
    V = np.array([[x, y, z] for x in (0, a) for y in (0, b) for z in (0, c)], dtype=float)
    faces = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    T = []
    for q in faces:
        T += [(q[0], q[1], q[2]), (q[0], q[2], q[3])]
    T = np.array(T, dtype=np.int32)
    # orient every triangle outwards (normal away from the centre)
    ctr = V.mean(0)
    for k, (i, j, l) in enumerate(T):
        n = np.cross(V[j] - V[i], V[l] - V[i])
        if np.dot(n, V[i] - ctr) < 0:
            T[k] = (i, l, j)
    return V, T


def test_mesh_mass_properties_of_a_box(orc):
    """Divergence-theorem mass properties (volume, centre of mass, moment of
    inertia about the vertical axis through it) are exact for a polyhedron:
    box a x b x c -> V = abc, c = (a/2, b/2), Izz = V (a^2 + b^2)/12."""
    a, b, c = 3.0, 2.0, 1.5
    V, T = _box_mesh(a, b, c)
    o = orc.Oracle((24, 24, 24), nu=0.05, body=orc.mesh_body((10.1, 10.2, 10.3), V, T, 3.0, 0.0, 3.0, 50.0))
    vol, cx, cy, Izz = o.mesh_mass(0.0)
    assert vol == pytest.approx(a * b * c, rel=1e-14)
    assert cx == pytest.approx(a / 2, rel=1e-14) and cy == pytest.approx(b / 2, rel=1e-14)
    assert Izz == pytest.approx(a * b * c * (a * a + b * b) / 12, rel=1e-13)


def test_swimmer_mass_properties_track_the_deformation(orc):
    """The sheared mesh keeps its volume (the midline only moves rings
    sideways); its centre of mass moves sideways with the mean midline
    displacement weighted by the cross-section areas."""
    L = 48.0
    body = _body(orc, L, 150, 64, (40.0, 24.371, 12.293), amp=0.125, period=64.0)
    o = orc.Oracle((96, 48, 24), nu=0.02, body=body)
    m0 = o.mesh_mass(0.0)
    m1 = o.mesh_mass(17.0)
    assert m1[0] == pytest.approx(m0[0], rel=1e-12)
    assert m0[0] == pytest.approx(synth.swimmer_volume(L), rel=0.02)
    s = np.linspace(0, L, 20001)
    A = np.pi * synth.swimmer_half_width(s, L) * synth.swimmer_half_height(s, L)
    for t, m in ((0.0, m0), (17.0, m1)):
        ym = 0.125 * L * (s / L + 0.03125) / 1.03125 * np.sin(2 * np.pi * (s / L - t / 64.0))
        assert m[2] == pytest.approx(np.trapezoid(A * ym, s) / np.trapezoid(A, s), abs=2e-3 * L)
        assert m[1] == pytest.approx(np.trapezoid(A * s, s) / np.trapezoid(A, s), abs=2e-3 * L)


def test_rotated_pose_matches_the_analytic_body(orc):
    """Centre-of-mass frame with a yaw angle: nodes clearly inside / outside
    the analytic elliptic body rotated by psi about the centre of mass are
    classified accordingly by ray parity."""
    L, psi = 40.0, 0.5
    X = (36.137, 30.371, 12.293)
    body = _body(orc, L, 150, 96, X, free=4, psi=psi)
    o = orc.Oracle((72, 60, 24), nu=0.02, body=body)
    solid = o.solid().astype(bool)
    vol, cx, cy, _ = o.mesh_mass(0.0)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in (24, 60, 72)], indexing="ij")
    rx, ry = x - X[0], y - X[1]
    s = np.cos(psi) * rx + np.sin(psi) * ry + cx
    q = -np.sin(psi) * rx + np.cos(psi) * ry + cy
    w = synth.swimmer_half_width(np.clip(s, 0, L), L)
    h = synth.swimmer_half_height(np.clip(s, 0, L), L)
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = (q / w) ** 2 + ((z - X[2]) / h) ** 2
    core = (s > 2.0) & (s < L - 2.0)
    inside = core & (phi < 0.9)
    outside = (s < -0.7) | (s > L + 0.7) | (core & (phi > 1.1))
    assert inside.sum() > 200
    assert solid[inside].all() and not solid[outside].any()


def test_three_dof_euler_update(orc):
    """Free in x, y and yaw (Sec. 4.3, Euler): X += U, U += F/m on x and y,
    psi += omega, I omega += M_z with I of the new pose; the pose's vertex
    velocities are the central differences of the poses."""
    shape = (64, 48, 24)
    X0 = np.array([30.137, 24.371, 12.293])
    U0 = np.array([0.004, -0.002, 0.0])
    body = _body(orc, 24.0, 48, 16, X0, amp=0.125, period=64.0, U=tuple(U0), free=7, omega=2e-3)
    body.mass = 40.0
    o = orc.Oracle(shape, nu=0.05, body=body)
    rho, u, xi = synth.parity_fields(shape, 23)
    o.init_state(rho, 0.2 * u, xi, 1e-3)
    b0 = o.body
    I0 = b0.Izz
    assert b0.Iw == pytest.approx(I0 * 2e-3, rel=1e-14)
    vol0 = o.mesh_mass(0.0)[0]
    assert I0 == pytest.approx(40.0 / vol0 * o.mesh_mass(0.0)[3], rel=1e-14)
    o.step(1)
    b1 = o.body
    assert np.allclose(b1.X[:2], X0[:2] + U0[:2], atol=1e-14, rtol=0) and b1.X[2] == X0[2]
    assert np.allclose(b1.U[:2], U0[:2], atol=1e-15, rtol=0)   # F of the step before the first is 0
    assert b1.psi == pytest.approx(2e-3, abs=1e-15)
    I1 = 40.0 / vol0 * o.mesh_mass(1.0)[3]
    assert b1.omega == pytest.approx(I0 * 2e-3 / I1, rel=1e-12)
    F1, M1 = np.array(b1.F), np.array(b1.M)
    assert np.abs(F1[:2]).max() > 0 and abs(M1[2]) > 0
    o.step(1)
    b2 = o.body
    assert np.allclose(b2.U[:2], U0[:2] + F1[:2] / 40.0, atol=1e-15, rtol=0)
    assert b2.psi == pytest.approx(2e-3 + b1.omega, abs=1e-15)
    I2 = 40.0 / vol0 * o.mesh_mass(2.0)[3]
    assert b2.omega == pytest.approx((I0 * 2e-3 + M1[2]) / I2, rel=1e-12)


def test_com_frame_vertex_velocity_is_central_difference(orc):
    """Held yaw rate and translation in the centre-of-mass frame: the vertex
    velocity U + omega x r + R (b_dot - c_dot) agrees with the central
    difference of the actual poses to O(omega^2)."""
    body = _body(orc, 24.0, 48, 16, (30.137, 24.371, 12.293), amp=0.125, period=64.0,
                 U=(0.003, 0.001, 0.0), free=7, omega=1e-4)
    body.mass = 1e30   # forces do not change U, omega changes only with I
    o = orc.Oracle((64, 48, 24), nu=0.05, body=body)
    pos, vel = [], []
    for _ in range(3):
        p, v = o.mesh_pose()
        pos.append(p)
        vel.append(v)
        o.step_sampled([0])
    fd = 0.5 * (pos[2] - pos[0])
    assert np.abs(vel[1] - fd).max() < 1e-5
