"""FP64 CPU oracle for the entropic (KBC) D3Q27 step with Grad moving-wall
boundaries and momentum-exchange coupling (arXiv 1608.04658, Secs. 2-4.1).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` are the only callers.  The library under
``paper_1608_04658_gb300`` never imports this package and shares no code with
it; the two meet only through the seeded generators in ``synth``.

The arithmetic lives in ``kbc_oracle.c`` (plain C99, IEEE double, compiled
without fast-math or FMA contraction); this module is ctypes marshalling.
Layout of a population array: numpy ``(27, nz, ny, nx)`` float64, direction
index i = 9(cx+1) + 3(cy+1) + (cz+1).

``slab.py`` runs the same oracle split into z slabs over CPU ranks (the
decomposition of one box over several devices, tests/test_oracle_slab.py);
``slab_adjoint.py`` runs the adjoint of that split, the halo exchange
reversed, on the autograd restatement of the bodiless step
(tests/test_oracle_slab_adjoint.py).

Parity status per function (pins live in tests/test_oracle_*.py):
  feq, kbc_split, collide (all modes), gamma_exact, grad, stream/box faces,
  refill moments, momentum exchange force and torque, Couette with Grad walls, the Grad
  wall targets (target velocity and static + dynamic target density in co-moving flow),
  shear-wave and Taylor-Green viscosity: pinned.
  Two-level block refinement (RefinedOracle; Sec. 4.2's two-level grid, readings in
  kbc_oracle.c): pinned by uniform flow, refined Couette flow and a sound wave against
  the single-level run at the fine resolution (tests/test_oracle_refine.py).
  Sphere refill density average and the sphere's Euler update beyond one step:
  pinned only by invariants (moments of the refilled node, mass accounting).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kbc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

FACE_PERIODIC, FACE_WALL, FACE_EQ, FACE_OUTFLOW = 0, 1, 2, 3
BODY_NONE, BODY_SPHERE, BODY_PLANES, BODY_AIRFOIL, BODY_MESH = 0, 1, 2, 3, 4
MODE_ANALYTIC, MODE_EXACT, MODE_LBGK = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile kbc_oracle.c into oracle/_build/liboracle.so (gcc, -O2, no
    fast-math, no FMA contraction so x86 and Arm hosts agree)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("face", C.c_int * 6), ("gamma_mode", C.c_int), ("pad_", C.c_int),
                ("beta", C.c_double), ("rho0", C.c_double), ("u_face", C.c_double * 3)]


class Body(C.Structure):
    _fields_ = [("kind", C.c_int), ("free_motion", C.c_int),
                ("X", C.c_double * 3), ("U", C.c_double * 3), ("R", C.c_double),
                ("y_lo", C.c_double), ("y_hi", C.c_double),
                ("U_lo", C.c_double * 3), ("U_hi", C.c_double * 3),
                ("mass", C.c_double), ("rho_ratio", C.c_double), ("g", C.c_double * 3),
                ("F", C.c_double * 3), ("M", C.c_double * 3),
                ("chord", C.c_double), ("ca", C.c_double), ("sa", C.c_double),
                ("h_amp", C.c_double), ("h_omega", C.c_double),
                ("camber_m", C.c_double), ("camber_p", C.c_double), ("thick", C.c_double * 5),
                ("y_base", C.c_double), ("t", C.c_double),
                ("mesh_rest", C.POINTER(C.c_double)), ("mesh_tris", C.POINTER(C.c_int)),
                ("n_vertices", C.c_int), ("n_triangles", C.c_int),
                ("length", C.c_double), ("wave_amp", C.c_double), ("wave_length", C.c_double),
                ("wave_period", C.c_double), ("wave_ramp", C.c_int), ("pad2_", C.c_int),
                ("psi", C.c_double), ("omega", C.c_double), ("Iw", C.c_double), ("Izz", C.c_double),
                ("com", C.c_double * 2), ("com_dot", C.c_double * 2)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = C.CDLL(so)
            L.orc_lattice.argtypes = [_I, _D]
            L.orc_feq.argtypes = [C.c_double, _D, _D]
            L.orc_kbc_split.argtypes = [_D, _D, _D, _D]
            L.orc_entropy.argtypes = [_D]
            L.orc_entropy.restype = C.c_double
            L.orc_gamma_residual.argtypes = [_D, _D, _D, C.c_double, C.c_double]
            L.orc_gamma_residual.restype = C.c_double
            L.orc_gamma_exact.argtypes = [_D, _D, _D, C.c_double]
            L.orc_gamma_exact.restype = C.c_double
            L.orc_collide.argtypes = [_D, C.c_double, C.c_int, _D]
            L.orc_collide.restype = C.c_double
            L.orc_grad.argtypes = [C.c_double, _D, _D, _D]
            L.orc_create.argtypes = [C.POINTER(Params), C.POINTER(Body)]
            L.orc_create.restype = C.c_void_p
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_f.argtypes = [C.c_void_p, _D]
            L.orc_get_f.argtypes = [C.c_void_p, _D]
            L.orc_get_solid.argtypes = [C.c_void_p, C.c_void_p]
            L.orc_get_body.argtypes = [C.c_void_p, C.POINTER(Body)]
            L.orc_set_body.argtypes = [C.c_void_p, C.POINTER(Body)]
            L.orc_link.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, _D]
            L.orc_link.restype = C.c_double
            L.orc_set_owned_z.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_set_owned_z.restype = None
            L.orc_set_z_frame.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_set_z_frame.restype = None
            L.orc_counter.argtypes = [C.c_void_p, C.c_int]
            L.orc_counter.restype = C.c_long
            L.orc_init_state.argtypes = [C.c_void_p, _D, _D, C.c_void_p, C.c_double]
            L.orc_step.argtypes = [C.c_void_p, C.c_int]
            L.orc_step.restype = C.c_int
            L.orc_step_sampled.argtypes = [C.c_void_p, C.c_long, C.POINTER(C.c_long), _D]
            L.orc_step_sampled.restype = C.c_int
            L.orc_wall_targets_sampled.argtypes = [C.c_void_p, C.c_long, C.POINTER(C.c_long), _D]
            L.orc_wall_targets_sampled.restype = C.c_int
            L.orc_totals.argtypes = [C.c_void_p, _D]
            L.orc_mesh_pose.argtypes = [C.c_void_p, _D, _D]
            L.orc_mesh_link.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, _D]
            L.orc_mesh_link.restype = C.c_double
            L.orc_mesh_mass.argtypes = [C.c_void_p, C.c_double, _D]
            L.orc_refine_create.argtypes = [C.c_void_p, _I, _I, C.c_void_p]
            L.orc_refine_create.restype = C.c_void_p
            L.orc_refine_fine.argtypes = [C.c_void_p]
            L.orc_refine_fine.restype = C.c_void_p
            L.orc_refine_destroy.argtypes = [C.c_void_p]
            L.orc_refine_destroy.restype = None
            L.orc_refine_init.argtypes = [C.c_void_p]
            L.orc_refine_init.restype = None
            L.orc_refine_step.argtypes = [C.c_void_p, C.c_int]
            L.orc_refine_step.restype = C.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def lattice():
    """(c[27,3] int, W[27]) of the D3Q27 lattice."""
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    lib().orc_lattice(c.ctypes.data_as(_I), _dp(w))
    return c.astype(np.int64), w


def feq(rho: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(27)
    lib().orc_feq(float(rho), _dp(u), _dp(out))
    return out


def kbc_split(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    fe, ds, dh = np.zeros(27), np.zeros(27), np.zeros(27)
    lib().orc_kbc_split(_dp(f), _dp(fe), _dp(ds), _dp(dh))
    return fe, ds, dh


def entropy(f) -> float:
    return lib().orc_entropy(_dp(np.ascontiguousarray(f, dtype=np.float64)))


def gamma_residual(ds, dh, fe, beta, g) -> float:
    return lib().orc_gamma_residual(_dp(np.ascontiguousarray(ds)), _dp(np.ascontiguousarray(dh)),
                                    _dp(np.ascontiguousarray(fe)), float(beta), float(g))


def gamma_exact(ds, dh, fe, beta) -> float:
    return lib().orc_gamma_exact(_dp(np.ascontiguousarray(ds)), _dp(np.ascontiguousarray(dh)),
                                 _dp(np.ascontiguousarray(fe)), float(beta))


def collide(f, beta: float, mode: int = MODE_ANALYTIC):
    """Post-collision populations and the stabilizer used."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(27)
    g = lib().orc_collide(_dp(f), float(beta), int(mode), _dp(out))
    return out, g


def grad(rho: float, u, Pi) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    Pi = np.ascontiguousarray(np.asarray(Pi, dtype=np.float64).reshape(9))
    out = np.zeros(27)
    lib().orc_grad(float(rho), _dp(u), _dp(Pi), _dp(out))
    return out


def beta_from_nu(nu: float) -> float:
    """nu = c_s^2 (1/(2b) - 1/2) with c_s^2 = 1/3 (Sec. 2)."""
    return 1.0 / (6.0 * nu + 1.0)


class Oracle:
    """Whole-lattice oracle state.  ``faces`` = (x-, x+, y-, y+, z-, z+)."""

    def __init__(self, shape, nu=None, beta=None, faces=(0,) * 6, rho0=1.0,
                 u_face=(0.0, 0.0, 0.0), gamma_mode=MODE_ANALYTIC, body=None):
        nx, ny, nz = shape
        self.shape = (nx, ny, nz)
        if beta is None:
            beta = beta_from_nu(nu)
        p = Params()
        p.nx, p.ny, p.nz = nx, ny, nz
        for k in range(6):
            p.face[k] = int(faces[k])
        p.gamma_mode = int(gamma_mode)
        p.beta = float(beta)
        p.rho0 = float(rho0)
        for a in range(3):
            p.u_face[a] = float(u_face[a])
        self.params = p
        b = Body() if body is None else body
        # the mesh arrays a body points to must outlive the context
        self._keep = getattr(b, "_arrays", None)
        self._ctx = lib().orc_create(C.byref(p), C.byref(b))
        if not self._ctx:
            raise MemoryError("oracle allocation failed")
        self.N = nx * ny * nz

    def __del__(self):
        if getattr(self, "_ctx", None) and not getattr(self, "_borrowed", False):
            lib().orc_destroy(self._ctx)
        self._ctx = None

    # state ------------------------------------------------------------
    def set_f(self, f: np.ndarray):
        nx, ny, nz = self.shape
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(27, nz, ny, nx)
        lib().orc_set_f(self._ctx, _dp(f))

    def get_f(self) -> np.ndarray:
        nx, ny, nz = self.shape
        out = np.empty((27, nz, ny, nx))
        lib().orc_get_f(self._ctx, _dp(out))
        return out

    def init_state(self, rho: np.ndarray, u: np.ndarray, xi: np.ndarray | None = None,
                   amp: float = 0.0):
        """f = f^eq(rho, u) + amp * W_i * xi_i.  rho: (nz,ny,nx); u: (nz,ny,nx,3);
        xi: (27,nz,ny,nx) or None."""
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        if xi is None:
            lib().orc_init_state(self._ctx, _dp(rho), _dp(u), None, 0.0)
        else:
            xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1)
            lib().orc_init_state(self._ctx, _dp(rho), _dp(u), xi.ctypes.data_as(C.c_void_p),
                                 float(amp))

    def solid(self) -> np.ndarray:
        nx, ny, nz = self.shape
        out = np.empty((nz, ny, nx), dtype=np.uint8)
        lib().orc_get_solid(self._ctx, out.ctypes.data_as(C.c_void_p))
        return out

    @property
    def body(self) -> Body:
        b = Body()
        lib().orc_get_body(self._ctx, C.byref(b))
        return b

    @body.setter
    def body(self, b: Body):
        lib().orc_set_body(self._ctx, C.byref(b))

    def link(self, x: int, y: int, z: int, i: int):
        """(q, u_w) of the link from fluid node (x, y, z) to the solid node
        (x, y, z) - c_i at the current pose, as the boundary step takes them."""
        uw = np.zeros(3)
        q = lib().orc_link(self._ctx, int(x), int(y), int(z), int(i), _dp(uw))
        return q, uw

    def set_owned_z(self, z_lo: int, z_hi: int):
        """Later steps sum the force and torque over the boundary nodes of the
        z layers [z_lo, z_hi) only (one slab of a decomposed box)."""
        lib().orc_set_owned_z(self._ctx, int(z_lo), int(z_hi))

    def set_z_frame(self, origin: int, period: int):
        """Treats the box as a slab of a box periodic in z with `period`
        layers, layer k at z = (k + origin) mod period, for the sphere's
        geometry and centre wrap (recomputes the current solid marks)."""
        lib().orc_set_z_frame(self._ctx, int(origin), int(period))

    def counters(self):
        L = lib()
        return dict(step=L.orc_counter(self._ctx, 0), boundary=L.orc_counter(self._ctx, 1),
                    links=L.orc_counter(self._ctx, 2), refill=L.orc_counter(self._ctx, 3),
                    error=L.orc_counter(self._ctx, 4))

    # dynamics ---------------------------------------------------------
    def step(self, n: int = 1):
        if lib().orc_step(self._ctx, int(n)) != 0:
            raise MemoryError("oracle step allocation failed")

    def step_sampled(self, nodes) -> np.ndarray:
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        out = np.empty((len(nodes), 27))
        lib().orc_step_sampled(self._ctx, len(nodes), nodes.ctypes.data_as(C.POINTER(C.c_long)),
                               _dp(out))
        return out

    def wall_targets_sampled(self, nodes) -> np.ndarray:
        """Moves to t+1's marks (body update, marks, refill, as a step does)
        and returns per listed node (number of missing directions, static
        density, dynamic density, target density, target velocity x, y, z) of
        the Grad wall boundary (Sec. 3); NaN densities where the node is no
        boundary node.  The state is not advanced."""
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        out = np.empty((len(nodes), 7))
        lib().orc_wall_targets_sampled(self._ctx, len(nodes), nodes.ctypes.data_as(C.POINTER(C.c_long)),
                                       _dp(out))
        return out

    def mesh_pose(self):
        """(positions, velocities) of the mesh vertices, each (n_vertices, 3)."""
        n = self.body.n_vertices
        pos, vel = np.zeros((n, 3)), np.zeros((n, 3))
        lib().orc_mesh_pose(self._ctx, _dp(pos), _dp(vel))
        return pos, vel

    def mesh_mass(self, t: float):
        """(V, cx, cy, Izz) of the mesh at time t in the body frame, unit density."""
        out = np.zeros(4)
        lib().orc_mesh_mass(self._ctx, float(t), _dp(out))
        return out

    def mesh_link(self, x: int, y: int, z: int, i: int):
        """(q, u_w) of the link from node (x, y, z) along -c_i."""
        uw = np.zeros(3)
        q = lib().orc_mesh_link(self._ctx, int(x), int(y), int(z), int(i), _dp(uw))
        return q, uw

    def totals(self) -> np.ndarray:
        """[mass, jx, jy, jz, kinetic energy] over fluid nodes."""
        out = np.zeros(5)
        lib().orc_totals(self._ctx, _dp(out))
        return out


def sphere_body(X, R, U=(0.0, 0.0, 0.0), free=False, rho_ratio=1.5, g=(0.0, 0.0, 0.0),
                mass=None) -> Body:
    b = Body()
    b.kind = BODY_SPHERE
    b.free_motion = 1 if free else 0
    for a in range(3):
        b.X[a], b.U[a], b.g[a] = float(X[a]), float(U[a]), float(g[a])
    b.R = float(R)
    b.rho_ratio = float(rho_ratio)
    # m_s = rho_s * pi D^3 / 6 with rho_f = 1 (analytic volume)
    b.mass = float(mass) if mass is not None else float(rho_ratio) * np.pi * (2 * R) ** 3 / 6.0
    return b


def airfoil_body(le, chord, ca, sa, h_amp, h_omega, camber_m, camber_p, thick, t0=0.0) -> Body:
    """Airfoil extruded along z with its leading edge at le (x, y) at zero
    plunge; the pose at time t0 is set here."""
    import math
    b = Body()
    b.kind = BODY_AIRFOIL
    b.chord, b.ca, b.sa = float(chord), float(ca), float(sa)
    b.h_amp, b.h_omega = float(h_amp), float(h_omega)
    b.camber_m, b.camber_p = float(camber_m), float(camber_p)
    for k in range(5):
        b.thick[k] = float(thick[k])
    b.y_base = float(le[1])
    b.t = float(t0)
    b.X[0] = float(le[0])
    b.X[1] = b.y_base + b.h_amp * math.sin(b.h_omega * b.t)
    b.U[1] = b.h_amp * b.h_omega * math.cos(b.h_omega * b.t)
    return b


def planes_body(y_lo, y_hi, U_lo=(0.0, 0.0, 0.0), U_hi=(0.0, 0.0, 0.0)) -> Body:
    b = Body()
    b.kind = BODY_PLANES
    b.y_lo, b.y_hi = float(y_lo), float(y_hi)
    for a in range(3):
        b.U_lo[a], b.U_hi[a] = float(U_lo[a]), float(U_hi[a])
    return b


def mesh_body(X, rest, tris, length, wave_amp, wave_length, wave_period, ramp=False,
              U=(0.0, 0.0, 0.0), free=False, mass=1.0, t0=0.0, psi=0.0, omega=0.0) -> Body:
    """Triangulated swimmer (Sec. 4.3): rest[v] = (s, dy, dz) per vertex, tris
    (n, 3) vertex indices, centre line along +x.  free: False (held), True (x
    only) or a bit mask (1 x, 2 y, 4 yaw).  Held or free in x only, X is the
    head; free in y or yaw, X is the centre of mass and psi, omega the yaw
    angle and rate.  The arrays are kept alive by the returned Body."""
    b = Body()
    b.kind = BODY_MESH
    b.free_motion = (1 if free else 0) if isinstance(free, bool) else int(free)
    b.psi, b.omega = float(psi), float(omega)
    rest = np.ascontiguousarray(rest, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    b._arrays = (rest, tris)
    b.mesh_rest = rest.ctypes.data_as(C.POINTER(C.c_double))
    b.mesh_tris = tris.ctypes.data_as(C.POINTER(C.c_int))
    b.n_vertices, b.n_triangles = len(rest), len(tris)
    for a in range(3):
        b.X[a], b.U[a] = float(X[a]), float(U[a])
    b.length, b.wave_amp = float(length), float(wave_amp)
    b.wave_length, b.wave_period = float(wave_length), float(wave_period)
    b.wave_ramp = 1 if ramp else 0
    b.mass = float(mass)
    b.t = float(t0)
    return b


def fine_beta(beta: float) -> float:
    """b of the fine level of a ratio-2 block under acoustic scaling: the
    viscosity in fine lattice units is twice the coarse one."""
    return beta / (2.0 - beta)


class RefinedOracle:
    """Two-level block refinement over a coarse ``Oracle`` (Sec. 4.2's
    two-level grid; the readings are stated in kbc_oracle.c).  ``lo``, ``hi``:
    the block's corner coarse nodes, both included.  ``fine`` is an
    ``Oracle``-like view of the fine level, (2m + 2) nodes per axis with m =
    hi - lo: fine node j sits at coarse coordinate lo + j/2.  With lo = 0,
    hi = n on a periodic axis the block spans that axis (2n fine nodes,
    periodic, no surface along it).

    ``fine_body``: a body of the fine level in fine lattice units (sphere,
    airfoil or mesh; its solid nodes must stay four nodes inside the block's
    surface, which ``step`` checks).

    Use: initialise ``coarse`` and ``fine`` (``init_state`` / ``set_f``), call
    ``init()``, then ``step(n)`` (n coarse steps, 2n fine steps)."""

    def __init__(self, coarse: Oracle, lo, hi, fine_body: Body | None = None):
        self.coarse = coarse
        self.lo = tuple(int(v) for v in lo)
        self.hi = tuple(int(v) for v in hi)
        lo_a = (C.c_int * 3)(*self.lo)
        hi_a = (C.c_int * 3)(*self.hi)
        self._keep = getattr(fine_body, "_arrays", None)
        bp = C.byref(fine_body) if fine_body is not None else None
        self._r = lib().orc_refine_create(coarse._ctx, lo_a, hi_a, bp)
        if not self._r:
            raise ValueError("bad refinement block (needs 1 <= lo, hi <= n - 2, hi - lo >= 3, "
                             "fluid coarse nodes from lo - 1 to hi + 1, no planes body on the fine level)")
        n = coarse.shape
        # a block with lo = 0, hi = n on a periodic axis spans that axis
        self.full = tuple(l == 0 and h == nn and coarse.params.face[2 * a] == FACE_PERIODIC
                          for a, (l, h, nn) in enumerate(zip(self.lo, self.hi, n)))
        fine = Oracle.__new__(Oracle)
        fine._ctx = lib().orc_refine_fine(self._r)
        fine._borrowed = True
        fine.shape = tuple(2 * nn if f else 2 * (h - l) + 2
                           for l, h, nn, f in zip(self.lo, self.hi, n, self.full))
        fine.N = fine.shape[0] * fine.shape[1] * fine.shape[2]
        self.fine = fine

    def __del__(self):
        if getattr(self, "_r", None):
            self.fine._ctx = None
            lib().orc_refine_destroy(self._r)
            self._r = None

    def init(self):
        lib().orc_refine_init(self._r)

    def step(self, n: int = 1):
        if lib().orc_refine_step(self._r, int(n)) != 0:
            raise MemoryError("oracle step allocation failed")
        if self.fine.counters()["error"] == 2:
            raise ValueError("the fine body came within four nodes of the block's surface")

    def coarse_valid(self) -> np.ndarray:
        """(nz, ny, nx) bool: coarse nodes the refined step defines (all but
        those more than one layer inside the block's surface)."""
        nx, ny, nz = self.coarse.shape
        v = np.ones((nz, ny, nx), dtype=bool)
        sl = [slice(None) if f else slice(l + 2, h - 1) for l, h, f in zip(self.lo, self.hi, self.full)]
        v[sl[2], sl[1], sl[0]] = False
        return v

    def fine_valid(self) -> np.ndarray:
        """(nz, ny, nx) bool of the fine level: every node but the pad."""
        nx, ny, nz = self.fine.shape
        v = np.zeros((nz, ny, nx), dtype=bool)
        sl = [slice(None) if f else slice(0, nn - 1) for nn, f in zip(self.fine.shape, self.full)]
        v[sl[2], sl[1], sl[0]] = True
        return v
