"""ctypes binding of liblbm.so (C ABI in include/lbm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides the device buffers and the stream.  The
library is loaded from ``paper_1608_04658_gb300/_build/liblbm.so``; if it is
missing the import of this module fails with an error that says how to build
it.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import builder as _build

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_UNSTABLE = 0, 1, 2, 3, 4
LBM_ERR_TIMEOUT, LBM_ERR_STATE, LBM_ERR_UNSUPPORTED = 5, 6, 7
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_CUDA", 3: "LBM_ERR_OOM",
                4: "LBM_ERR_UNSTABLE", 5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_STATE",
                7: "LBM_ERR_UNSUPPORTED"}
STORAGES = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
FACE_PERIODIC, FACE_WALL, FACE_EQ, FACE_OUTFLOW = 0, 1, 2, 3
BODY_NONE, BODY_SPHERE, BODY_PLANES, BODY_AIRFOIL, BODY_MESH = 0, 1, 2, 3, 4
GAMMA_ANALYTIC, GAMMA_EXACT, GAMMA_LBGK = 0, 1, 2
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbm.h")


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("storage", C.c_int32),
                ("face", C.c_int32 * 6), ("gamma_mode", C.c_int32), ("options", C.c_int32),
                ("nu", C.c_double), ("rho0", C.c_double), ("u_face", C.c_double * 3)]


class Geometry(C.Structure):
    _fields_ = [("kind", C.c_int32), ("free_motion", C.c_int32),
                ("X", C.c_double * 3), ("U", C.c_double * 3), ("R", C.c_double),
                ("y_lo", C.c_double), ("y_hi", C.c_double),
                ("U_lo", C.c_double * 3), ("U_hi", C.c_double * 3),
                ("mass", C.c_double), ("rho_ratio", C.c_double), ("g", C.c_double * 3),
                ("chord", C.c_double), ("ca", C.c_double), ("sa", C.c_double), ("h_amp", C.c_double),
                ("h_omega", C.c_double), ("camber_m", C.c_double), ("camber_p", C.c_double),
                ("thick", C.c_double * 5), ("t0", C.c_double),
                ("mesh_rest", C.POINTER(C.c_double)), ("mesh_tris", C.POINTER(C.c_int32)),
                ("n_vertices", C.c_int32), ("n_triangles", C.c_int32),
                ("length", C.c_double), ("wave_amp", C.c_double), ("wave_length", C.c_double),
                ("wave_period", C.c_double), ("wave_ramp", C.c_int32), ("reserved_mesh", C.c_int32),
                ("psi", C.c_double), ("omega", C.c_double)]


class AdjointSpec(C.Structure):
    _fields_ = [("horizon", C.c_int32), ("checkpoint_every", C.c_int32), ("w_force", C.c_double * 3),
                ("lambda_T", C.c_void_p), ("lambda_0", C.c_void_p), ("reserved", C.c_int32 * 4)]


class BodyState(C.Structure):
    _fields_ = [("X", C.c_double * 3), ("U", C.c_double * 3), ("F", C.c_double * 3),
                ("M", C.c_double * 3), ("F_sum", C.c_double * 3), ("M_sum", C.c_double * 3),
                ("n_sum", C.c_int64), ("n_boundary", C.c_int32), ("n_uncovered", C.c_int32),
                ("n_links", C.c_int32), ("status", C.c_int32), ("n_band", C.c_int32),
                ("t", C.c_double), ("psi", C.c_double), ("omega", C.c_double), ("Izz", C.c_double)]


# lbm_force_record: F[3], M[3], t (doubles), status, reserved (int32)
RECORD_DOUBLES = 8
RECORD_DEPTH = 8

_lib = None
_D = C.POINTER(C.c_double)


# caller-supplied device allocator of lbm_set_allocator
_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


def declared_symbols() -> list[str]:
    """Entry points declared in include/lbm.h."""
    text = open(HEADER).read()
    return re.findall(r"LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", text)


def lib():
    """Load liblbm.so (built by paper_1608_04658_gb300.builder)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.SO):
            raise ImportError(f"liblbm.so not built ({_build.SO}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(_build.SO)
        vp = C.c_void_p
        L.lbm_create.argtypes = [C.POINTER(Params), vp, vp, vp, vp, C.POINTER(vp)]
        L.lbm_create.restype = C.c_int
        L.lbm_destroy.argtypes = [vp]
        L.lbm_destroy.restype = None
        L.lbm_last_error.argtypes = [vp]
        L.lbm_last_error.restype = C.c_char_p
        L.lbm_init_state.argtypes = [vp, vp, vp, vp, C.c_double]
        L.lbm_init_state.restype = C.c_int
        L.lbm_init_state_f32.argtypes = [vp, vp, vp, vp, C.c_double]
        L.lbm_init_state_f32.restype = C.c_int
        L.lbm_set_geometry.argtypes = [vp, C.POINTER(Geometry)]
        L.lbm_set_geometry.restype = C.c_int
        L.lbm_step.argtypes = [vp, C.c_int]
        L.lbm_step.restype = C.c_int
        L.lbm_current_buffer.argtypes = [vp]
        L.lbm_current_buffer.restype = C.c_int
        L.lbm_get_populations.argtypes = [vp, _D]
        L.lbm_get_populations.restype = C.c_int
        L.lbm_set_populations.argtypes = [vp, _D]
        L.lbm_set_populations.restype = C.c_int
        L.lbm_body_forces.argtypes = [vp, _D, _D, C.c_int]
        L.lbm_body_forces.restype = C.c_int
        L.lbm_body_forces_async.argtypes = [vp, vp, C.POINTER(C.c_int64)]
        L.lbm_body_forces_async.restype = C.c_int
        L.lbm_body_forces_wait.argtypes = [vp, C.c_int64]
        L.lbm_body_forces_wait.restype = C.c_int
        L.lbm_set_launch_order.argtypes = [vp, C.c_int]
        L.lbm_set_launch_order.restype = C.c_int
        L.lbm_launch_order.argtypes = [vp]
        L.lbm_launch_order.restype = C.c_int
        L.lbm_get_body.argtypes = [vp, C.POINTER(BodyState)]
        L.lbm_get_body.restype = C.c_int
        L.lbm_reset_average.argtypes = [vp]
        L.lbm_reset_average.restype = C.c_int
        L.lbm_totals.argtypes = [vp, _D]
        L.lbm_totals.restype = C.c_int
        L.lbm_kernel_launches.argtypes = [vp]
        L.lbm_kernel_launches.restype = C.c_int64
        L.lbm_save.argtypes = [vp, C.c_char_p]
        L.lbm_save.restype = C.c_int
        L.lbm_load.argtypes = [vp, C.c_char_p]
        L.lbm_load.restype = C.c_int
        L.lbm_profile_begin.argtypes = [vp, C.c_int]
        L.lbm_profile_begin.restype = C.c_int
        L.lbm_profile_end.argtypes = [vp, _D, C.POINTER(C.c_int64)]
        L.lbm_profile_end.restype = C.c_int
        L.lbm_adjoint_step.argtypes = [vp, C.POINTER(AdjointSpec), _D, _D]
        L.lbm_adjoint_step.restype = C.c_int
        L.lbm_set_slab.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int]
        L.lbm_set_slab.restype = C.c_int
        L.lbm_pack_layers.argtypes = [vp, C.c_int, C.c_int, vp]
        L.lbm_pack_layers.restype = C.c_int
        L.lbm_unpack_layers.argtypes = [vp, C.c_int, C.c_int, vp]
        L.lbm_unpack_layers.restype = C.c_int
        L.lbm_set_body_force.argtypes = [vp, _D, _D]
        L.lbm_set_body_force.restype = C.c_int
        L.lbm_step_interior.argtypes = [vp]
        L.lbm_step_interior.restype = C.c_int
        L.lbm_step_edges.argtypes = [vp]
        L.lbm_step_edges.restype = C.c_int
        L.lbm_body_force_to_device.argtypes = [vp, vp]
        L.lbm_body_force_to_device.restype = C.c_int
        L.lbm_sum_body_force.argtypes = [vp, vp, C.c_int]
        L.lbm_set_allocator.argtypes = [vp, _ALLOC_FN, _RELEASE_FN, vp]
        L.lbm_set_allocator.restype = C.c_int
        L.lbm_init_equilibrium.argtypes = [vp, vp, vp]
        L.lbm_init_equilibrium.restype = C.c_int
        L.lbm_refine_create.argtypes = [vp, vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(vp)]
        L.lbm_refine_create.restype = C.c_int
        L.lbm_refine_init.argtypes = [vp]
        L.lbm_refine_init.restype = C.c_int
        L.lbm_refine_step.argtypes = [vp, C.c_int]
        L.lbm_refine_step.restype = C.c_int
        L.lbm_refine_save.argtypes = [vp, C.c_char_p]
        L.lbm_refine_save.restype = C.c_int
        L.lbm_refine_load.argtypes = [vp, C.c_char_p]
        L.lbm_refine_load.restype = C.c_int
        L.lbm_refine_destroy.argtypes = [vp]
        L.lbm_refine_destroy.restype = None
        L.lbm_sum_body_force.restype = C.c_int
        _lib = L
    return _lib


def _torch():
    import torch
    return torch


_TORCH_DTYPES = {"fp64": "float64", "fp32": "float32", "fp16": "float16", "bf16": "bfloat16"}


def make_params(shape, nu, storage="fp32", faces=(0,) * 6, rho0=1.0, u_face=(0.0, 0.0, 0.0),
                gamma_mode=GAMMA_ANALYTIC, options=0) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = (int(v) for v in shape)
    p.storage = STORAGES[storage]
    for k in range(6):
        p.face[k] = int(faces[k])
    p.gamma_mode = int(gamma_mode)
    p.options = int(options)
    p.nu = float(nu)
    p.rho0 = float(rho0)
    for a in range(3):
        p.u_face[a] = float(u_face[a])
    return p


def sphere(X, R, U=(0.0, 0.0, 0.0), free=False, rho_ratio=1.5, g=(0.0, 0.0, 0.0), mass=None) -> Geometry:
    """Sphere of radius R at X; without a mass lbm_set_geometry takes
    rho_s pi D^3 / 6 with rho_s = rho_ratio rho0."""
    G = Geometry()
    G.kind = BODY_SPHERE
    G.free_motion = 1 if free else 0
    for a in range(3):
        G.X[a], G.U[a], G.g[a] = float(X[a]), float(U[a]), float(g[a])
    G.R = float(R)
    G.rho_ratio = float(rho_ratio)
    G.mass = float(mass) if mass is not None else 0.0
    return G


def airfoil(le, chord, ca, sa, h_amp, h_omega, camber_m, camber_p, thick, t0=0.0) -> Geometry:
    """Airfoil extruded along z, leading edge at le = (x, y) at zero plunge."""
    G = Geometry()
    G.kind = BODY_AIRFOIL
    G.X[0], G.X[1] = float(le[0]), float(le[1])
    G.chord, G.ca, G.sa = float(chord), float(ca), float(sa)
    G.h_amp, G.h_omega = float(h_amp), float(h_omega)
    G.camber_m, G.camber_p = float(camber_m), float(camber_p)
    for k in range(5):
        G.thick[k] = float(thick[k])
    G.t0 = float(t0)
    return G


def swimmer(X, rest, tris, length, wave_amp, wave_length, wave_period, ramp=False,
            U=(0.0, 0.0, 0.0), free=False, mass=1.0, t0=0.0, psi=0.0, omega=0.0) -> Geometry:
    """Triangulated swimmer (Sec. 4.3): rest (n, 3) = (s, dy, dz) per vertex,
    tris (m, 3) vertex indices, centre line along +x.  free: False (held),
    True (x only) or a bit mask (1 x, 2 y, 4 yaw); held or free in x only, X
    is the head, otherwise the centre of mass, psi/omega the initial yaw angle
    and rate.  The arrays are kept alive by the returned Geometry (the
    library copies them)."""
    import numpy as np
    G = Geometry()
    G.kind = BODY_MESH
    G.free_motion = (1 if free else 0) if isinstance(free, bool) else int(free)
    G.psi, G.omega = float(psi), float(omega)
    rest = np.ascontiguousarray(rest, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    G._arrays = (rest, tris)
    G.mesh_rest = rest.ctypes.data_as(C.POINTER(C.c_double))
    G.mesh_tris = tris.ctypes.data_as(C.POINTER(C.c_int32))
    G.n_vertices, G.n_triangles = len(rest), len(tris)
    for a in range(3):
        G.X[a], G.U[a] = float(X[a]), float(U[a])
    G.length, G.wave_amp = float(length), float(wave_amp)
    G.wave_length, G.wave_period = float(wave_length), float(wave_period)
    G.wave_ramp = 1 if ramp else 0
    G.mass = float(mass)
    G.t0 = float(t0)
    return G


def planes(y_lo, y_hi, U_lo=(0.0, 0.0, 0.0), U_hi=(0.0, 0.0, 0.0)) -> Geometry:
    G = Geometry()
    G.kind = BODY_PLANES
    G.y_lo, G.y_hi = float(y_lo), float(y_hi)
    for a in range(3):
        G.U_lo[a], G.U_hi[a] = float(U_lo[a]), float(U_hi[a])
    return G


class Lattice:
    """A D3Q27 lattice on the current CUDA device.

    shape = (nx, ny, nz); populations are torch tensors of shape (27, nz, ny, nx)
    in the storage dtype, holding g_i = f_i - W_i rho0.  Calls enqueue on the
    torch stream current at construction.
    """

    def __init__(self, shape, nu, storage="fp32", faces=(0,) * 6, rho0=1.0,
                 u_face=(0.0, 0.0, 0.0), gamma_mode=GAMMA_ANALYTIC, device=None, options=0):
        torch = _torch()
        self.shape = tuple(int(v) for v in shape)
        nx, ny, nz = self.shape
        self.N = nx * ny * nz
        self.storage = storage
        self.rho0 = float(rho0)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self.device.index is None:
            self.device = torch.device(self.device.type, torch.cuda.current_device())
        dt = getattr(torch, _TORCH_DTYPES[storage])
        self.f_a = torch.empty((27, nz, ny, nx), dtype=dt, device=self.device)
        self.f_b = torch.empty((27, nz, ny, nx), dtype=dt, device=self.device)
        self.flags = torch.zeros((nz, ny, nx), dtype=torch.uint8, device=self.device)
        self.stream = torch.cuda.current_stream(self.device)
        self.params = make_params(shape, nu, storage, faces, rho0, u_face, gamma_mode, options)
        ctx = C.c_void_p()
        st = lib().lbm_create(C.byref(self.params), self.f_a.data_ptr(), self.f_b.data_ptr(),
                              self.flags.data_ptr(), C.c_void_p(self.stream.cuda_stream), C.byref(ctx))
        if st != LBM_OK:
            raise LbmError(st, "lbm_create failed")
        self._ctx = ctx
        self._keep = []
        self._dependents = []  # weak references to the refinements that use this lattice

    # -------------------------------------------------------------- helpers
    def _check(self, st: int):
        if st != LBM_OK:
            raise LbmError(st, lib().lbm_last_error(self._ctx).decode())

    def close(self):
        # a refinement keeps pointers to its levels: it goes first
        for ref in getattr(self, "_dependents", ()):
            dep = ref()
            if dep is not None:
                dep.close()
        if getattr(self, "_ctx", None):
            lib().lbm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def f(self):
        """Tensor holding the current state."""
        return self.f_b if lib().lbm_current_buffer(self._ctx) else self.f_a

    # -------------------------------------------------------------- state
    def init_state(self, rho, u, xi=None, amp: float = 0.0):
        """f = f^eq(rho, u) + amp W xi on the device.  rho (nz,ny,nx), u (nz,ny,nx,3),
        xi (27,nz,ny,nx) or None; numpy arrays or torch tensors.  Contiguous
        tensors on the lattice's device or in pinned host memory, all float64
        or all float32, go to the kernel as they are (pinned pages read across
        the host link; lbm_init_state / lbm_init_state_f32); other data is
        copied to the device first (as float64)."""
        torch = _torch()
        dev = self.device

        def direct(a, dt):
            return (torch.is_tensor(a) and a.dtype == dt and a.is_contiguous()
                    and ((a.device.type == "cpu" and a.is_pinned()) or a.device == dev))

        for dt, fn in ((torch.float64, lib().lbm_init_state), (torch.float32, lib().lbm_init_state_f32)):
            if not (direct(rho, dt) and direct(u, dt) and (xi is None or direct(xi, dt))):
                continue
            st = fn(self._ctx, rho.data_ptr(), u.data_ptr(), xi.data_ptr() if xi is not None else None, float(amp))
            if st != LBM_ERR_ARG:  # (not addressable by the device: copied below)
                self._check(st)
                self.stream.synchronize()
                return

        def to_dev(a):
            if torch.is_tensor(a):
                return a.to(device=dev, dtype=torch.float64, non_blocking=True).contiguous()
            return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(dev).contiguous()

        with torch.cuda.stream(self.stream):
            t_rho, t_u = to_dev(rho), to_dev(u)
            t_xi = to_dev(xi) if xi is not None else None
        self.stream.synchronize()
        self._check(lib().lbm_init_state(self._ctx, t_rho.data_ptr(), t_u.data_ptr(),
                                         t_xi.data_ptr() if t_xi is not None else None, float(amp)))
        self.stream.synchronize()

    def init_equilibrium(self, rho, u):
        """f = f^eq(rho, u) (lbm_init_equilibrium); rho (nz,ny,nx), u (nz,ny,nx,3)."""
        torch = _torch()
        with torch.cuda.stream(self.stream):
            t_rho = torch.as_tensor(np.ascontiguousarray(rho, dtype=np.float64)).to(self.device)
            t_u = torch.as_tensor(np.ascontiguousarray(u, dtype=np.float64)).to(self.device)
        self.stream.synchronize()
        self._check(lib().lbm_init_equilibrium(self._ctx, t_rho.data_ptr(), t_u.data_ptr()))
        self.stream.synchronize()

    def use_allocator(self, alloc, release):
        """Route the library's device scratch of this lattice through Python
        callables (lbm_set_allocator): alloc(nbytes, stream) -> device address
        (int) or None, release(address, stream).  Call before set_geometry."""
        def a(nbytes, stream, user):
            try:
                p = alloc(int(nbytes), stream)
            except Exception:
                return None
            return int(p) if p else None

        def r(ptr, stream, user):
            try:
                release(int(ptr), stream)
            except Exception:
                pass
        cbs = (_ALLOC_FN(a), _RELEASE_FN(r))
        self._check(lib().lbm_set_allocator(self._ctx, cbs[0], cbs[1], None))
        self._alloc_cbs = cbs  # kept alive as long as the context

    def use_torch_allocator(self):
        """The library's scratch of this lattice from PyTorch's caching
        allocator (on the lattice's device and stream)."""
        torch = _torch()
        dev = self.device.index
        self.use_allocator(lambda n, stream: torch.cuda.caching_allocator_alloc(n, dev, stream),
                           lambda p, stream: torch.cuda.caching_allocator_delete(p))

    def set_geometry(self, g: Geometry):
        self._check(lib().lbm_set_geometry(self._ctx, C.byref(g)))

    def step(self, n: int = 1):
        self._check(lib().lbm_step(self._ctx, int(n)))

    def launches(self) -> int:
        """Kernels enqueued by the last step() call."""
        return int(lib().lbm_kernel_launches(self._ctx))

    def profile_begin(self, max_launches: int):
        """Bracket the next bulk stream-collide launches with CUDA events."""
        self._check(lib().lbm_profile_begin(self._ctx, int(max_launches)))

    def profile_end(self):
        """(summed bulk-kernel milliseconds, number of bracketed launches)."""
        ms = C.c_double()
        n = C.c_int64()
        self._check(lib().lbm_profile_end(self._ctx, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def populations(self, out: np.ndarray | None = None) -> np.ndarray:
        """Current state as full FP64 populations (27, nz, ny, nx); ``out`` may be
        a preallocated (e.g. pinned) C-contiguous float64 array."""
        nx, ny, nz = self.shape
        if out is None:
            out = np.empty((27, nz, ny, nx), dtype=np.float64)
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == 27 * self.N
        self._check(lib().lbm_get_populations(self._ctx, out.ctypes.data_as(_D)))
        return out

    def set_populations(self, f: np.ndarray):
        nx, ny, nz = self.shape
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(27, nz, ny, nx)
        self._check(lib().lbm_set_populations(self._ctx, f.ctypes.data_as(_D)))

    def body(self) -> dict:
        b = BodyState()
        self._check(lib().lbm_get_body(self._ctx, C.byref(b)))
        return dict(X=np.array(b.X), U=np.array(b.U), F=np.array(b.F), M=np.array(b.M),
                    F_sum=np.array(b.F_sum), M_sum=np.array(b.M_sum), n_sum=b.n_sum,
                    n_boundary=b.n_boundary, n_uncovered=b.n_uncovered, n_links=b.n_links,
                    status=b.status, n_band=b.n_band, t=b.t, psi=b.psi, omega=b.omega, Izz=b.Izz)

    def forces(self, averaged: bool = False):
        F = np.zeros(3)
        M = np.zeros(3)
        self._check(lib().lbm_body_forces(self._ctx, F.ctypes.data_as(_D), M.ctypes.data_as(_D),
                                          1 if averaged else 0))
        return F, M

    def set_launch_order(self, order: str):
        """'auto' (time both in the first steps), 'split' or 'sequential'
        (lbm_set_launch_order); the results do not depend on it."""
        self._check(lib().lbm_set_launch_order(self._ctx, {"auto": 0, "split": 1, "sequential": 2}[order]))

    def launch_order(self) -> str:
        return {0: "auto", 1: "split", 2: "sequential"}[lib().lbm_launch_order(self._ctx)]

    def forces_async(self) -> int:
        """Enqueue a copy of the last step's force and torque into a pinned
        host record (lbm_body_forces_async) and return its ticket at once; up
        to RECORD_DEPTH records may be outstanding."""
        torch = _torch()
        if getattr(self, "_rec", None) is None:
            self._rec = torch.zeros((RECORD_DEPTH, RECORD_DOUBLES), dtype=torch.float64, pin_memory=True)
            self._rec_next = 0
        k = self._rec_next % RECORD_DEPTH
        t = C.c_int64()
        self._check(lib().lbm_body_forces_async(self._ctx, C.c_void_p(self._rec.data_ptr() + 8 * RECORD_DOUBLES * k),
                                                C.byref(t)))
        assert t.value == self._rec_next
        self._rec_next += 1
        return t.value

    def forces_wait(self, ticket: int):
        """Wait for the record of ticket (lbm_body_forces_wait; raises like
        forces() on a failed step) and return its (F, M)."""
        self._check(lib().lbm_body_forces_wait(self._ctx, int(ticket)))
        r = self._rec[ticket % RECORD_DEPTH].numpy()
        return r[0:3].copy(), r[3:6].copy()

    def save(self, path: str):
        """Checkpoint the current state (populations, node marks, body) to path."""
        self._check(lib().lbm_save(self._ctx, os.fsencode(path)))

    def load(self, path: str):
        """Restore a checkpoint written by save() for the same lattice and body."""
        self._check(lib().lbm_load(self._ctx, os.fsencode(path)))

    def reset_average(self):
        self._check(lib().lbm_reset_average(self._ctx))

    def adjoint(self, horizon: int, w_force=(0.0, 0.0, 0.0), lambda_T=None, want_lambda0: bool = False,
                checkpoint_every: int = 0):
        """Runs horizon steps and the adjoint sweep (lbm_adjoint_step).  J is
        the mean of w_force . F over the steps plus lambda_T . f at the end
        (lambda_T: device tensor (27, nz, ny, nx) of float64 for FP64 storage,
        float32 otherwise).  Returns dict(J, dJ_dtheta, lambda_0)."""
        torch = _torch()
        spec = AdjointSpec()
        spec.horizon = int(horizon)
        spec.checkpoint_every = int(checkpoint_every)
        for a in range(3):
            spec.w_force[a] = float(w_force[a])
        rdt = torch.float64 if self.storage == "fp64" else torch.float32
        nx, ny, nz = self.shape
        if lambda_T is not None:
            lambda_T = lambda_T.to(device=self.device, dtype=rdt).contiguous()
            spec.lambda_T = lambda_T.data_ptr()
        lam0 = None
        if want_lambda0:
            lam0 = torch.zeros((27, nz, ny, nx), dtype=rdt, device=self.device)
            spec.lambda_0 = lam0.data_ptr()
        J = np.zeros(1)
        dJ = np.zeros(3)
        self._check(lib().lbm_adjoint_step(self._ctx, C.byref(spec), J.ctypes.data_as(_D), dJ.ctypes.data_as(_D)))
        return dict(J=float(J[0]), dJ_dtheta=dJ, lambda_0=lam0)

    # -------------------------------------------------------------- slabs
    def set_slab(self, zoff: int, zper: int, own_lo: int, own_hi: int):
        """This lattice is a slab of a box periodic in z with zper layers, its
        layer k the box's layer zoff + k, its own layers [own_lo, own_hi)
        (lbm_set_slab; before set_geometry)."""
        self._check(lib().lbm_set_slab(self._ctx, int(zoff), int(zper), int(own_lo), int(own_hi)))

    def pack_layers(self, z0: int, n: int, out=None):
        """The current state's layers [z0, z0 + n), all 27 planes, as a device
        tensor (27, n, ny, nx) of the storage type (lbm_pack_layers)."""
        torch = _torch()
        nx, ny, _ = self.shape
        if out is None:
            out = torch.empty((27, n, ny, nx), dtype=self.f_a.dtype, device=self.device)
        self._check(lib().lbm_pack_layers(self._ctx, int(z0), int(n), C.c_void_p(out.data_ptr())))
        return out

    def unpack_layers(self, z0: int, src):
        """Writes a (27, n, ny, nx) device tensor of the storage type into the
        current state's layers [z0, z0 + n) (lbm_unpack_layers)."""
        src = src.contiguous()
        self._check(lib().lbm_unpack_layers(self._ctx, int(z0), int(src.shape[1]), C.c_void_p(src.data_ptr())))

    def set_body_force(self, F, M):
        """Replaces the body's current force and torque (lbm_set_body_force)."""
        Fa = np.ascontiguousarray(F, dtype=np.float64)
        Ma = np.ascontiguousarray(M, dtype=np.float64)
        self._check(lib().lbm_set_body_force(self._ctx, Fa.ctypes.data_as(_D), Ma.ctypes.data_as(_D)))

    def step_interior(self):
        """A slab step's own layers that pull from no halo layer
        (lbm_step_interior); step_edges completes the step."""
        self._check(lib().lbm_step_interior(self._ctx))

    def step_edges(self):
        """The rest of a slab step, after the halo layers were refilled
        (lbm_step_edges)."""
        self._check(lib().lbm_step_edges(self._ctx))

    def body_force_to(self, out=None):
        """The body's current force and torque (6 doubles) copied into a device
        tensor, without a host synchronisation (lbm_body_force_to_device)."""
        torch = _torch()
        if out is None:
            out = torch.empty(6, dtype=torch.float64, device=self.device)
        if out.dtype != torch.float64 or out.numel() < 6 or not out.is_contiguous() or out.device != self.device:
            raise ValueError("body_force_to: a contiguous float64 tensor of 6 values on the lattice's device")
        self._check(lib().lbm_body_force_to_device(self._ctx, C.c_void_p(out.data_ptr())))
        return out

    def sum_body_force(self, parts):
        """Replaces the body's force and torque by the sum, in row order, of the
        rows of a device tensor (nparts, 6) of float64 (lbm_sum_body_force)."""
        torch = _torch()
        if parts.dtype != torch.float64 or parts.dim() != 2 or parts.shape[1] != 6 or not parts.is_contiguous() \
                or parts.device != self.device:
            raise ValueError("sum_body_force: a contiguous float64 tensor (nparts, 6) on the lattice's device")
        self._check(lib().lbm_sum_body_force(self._ctx, C.c_void_p(parts.data_ptr()), int(parts.shape[0])))

    def totals(self) -> np.ndarray:
        out = np.zeros(5)
        self._check(lib().lbm_totals(self._ctx, out.ctypes.data_as(_D)))
        return out


def fine_shape(coarse_shape, faces, lo, hi):
    """(spanned axes, fine lattice shape) of a ratio-2 block over the coarse
    nodes [lo, hi]: an axis with lo = 0, hi = n and periodic faces is spanned
    (2n fine nodes), any other holds 2 (hi - lo) + 2 (the block's 2m + 1
    nodes and a pad)."""
    full = tuple(int(l) == 0 and int(h) == int(n) and int(faces[2 * a]) == FACE_PERIODIC
                 for a, (l, h, n) in enumerate(zip(lo, hi, coarse_shape)))
    shape = tuple(2 * int(n) if f else 2 * (int(h) - int(l)) + 2
                  for l, h, n, f in zip(lo, hi, coarse_shape, full))
    return full, shape


def fine_nu(nu: float) -> float:
    """Viscosity of the fine level of a ratio-2 block in its own lattice units
    (acoustic scaling: twice the coarse value)."""
    return 2.0 * float(nu)


class Refinement:
    """Two-level block refinement (lbm_refine_*; Sec. 4.2's two-level grid).

    ``coarse`` is a bodiless Lattice; the block covers its nodes [lo, hi] per
    axis (both ends included; lo = 0, hi = n on a periodic axis spans it).  The fine Lattice (2 (hi - lo) + 2 nodes per
    axis, periodic faces, twice the coarse viscosity, same storage, stabilizer
    and stream) is created here as ``self.fine``: fine node j sits at coarse
    coordinate lo + j/2.  Initialise both levels, call ``init()``, then
    ``step(n)`` (n coarse steps, 2n fine steps).  Closing either Lattice
    closes this object first (it holds pointers to both levels)."""

    def __init__(self, coarse: Lattice, lo, hi):
        self.coarse = coarse
        self.lo = tuple(int(v) for v in lo)
        self.hi = tuple(int(v) for v in hi)
        p = coarse.params
        self.full, shape = fine_shape(coarse.shape, list(p.face), self.lo, self.hi)
        self.fine = Lattice(shape, fine_nu(p.nu), coarse.storage, rho0=coarse.rho0, gamma_mode=p.gamma_mode,
                            device=coarse.device)
        r = C.c_void_p()
        lo_a = (C.c_int32 * 3)(*self.lo)
        hi_a = (C.c_int32 * 3)(*self.hi)
        st = lib().lbm_refine_create(coarse._ctx, self.fine._ctx, lo_a, hi_a, C.byref(r))
        if st != LBM_OK:
            err = LbmError(st, lib().lbm_last_error(coarse._ctx).decode())
            self.fine.close()  # nothing refers to it yet: give its memory back now
            raise err
        self._r = r
        import weakref
        coarse._dependents.append(weakref.ref(self))
        self.fine._dependents.append(weakref.ref(self))

    def close(self):
        if getattr(self, "_r", None):
            lib().lbm_refine_destroy(self._r)
            self._r = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self):
        self.coarse._check(lib().lbm_refine_init(self._r))

    def step(self, n: int = 1):
        self.coarse._check(lib().lbm_refine_step(self._r, int(n)))

    def save(self, path: str):
        """The coupling's state (lbm_refine_save); save both levels beside it."""
        self.coarse._check(lib().lbm_refine_save(self._r, str(path).encode()))

    def load(self, path: str):
        """Resume from lbm_refine_save's file (in place of init()), after both
        levels have loaded theirs."""
        self.coarse._check(lib().lbm_refine_load(self._r, str(path).encode()))
