"""Seeded synthetic inputs shared by the tests, the smoke check and the
benchmark.

This module holds no arithmetic of the lattice Boltzmann method: it draws
counter-based random numbers and writes the analytic initial fields and the
workload parameters of the configurations.  The oracle and the CUDA path each
turn these fields into populations with their own code.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014) of
``seed * 2^32 + counter``: one 64-bit output per counter, mapped to [0, 1)
by its top 53 bits.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """splitmix64 output for each uint64 counter value (state = counter * golden)."""
    with np.errstate(over="ignore"):
        z = (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n uniforms in [0,1) for (seed, stream); counters seed<<40 | stream<<32 | k."""
    k = np.arange(n, dtype=np.uint64)
    base = (np.uint64(seed & 0xFFFFFF) << np.uint64(40)) | (np.uint64(stream & 0xFF) << np.uint64(32))
    z = splitmix64(base + k)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def parity_fields(shape, seed: int, drho: float = 0.01, umax: float = 0.05):
    """Random macroscopic fields and a non-equilibrium noise for parity tests.

    Returns rho (nz,ny,nx) = 1 + drho*U(-1,1), u (nz,ny,nx,3) with components
    umax*U(-1,1), and xi (27,nz,ny,nx) = U(-1,1).  A side builds
    f_i = f_i^eq(rho, u) + amp * W_i * xi_i with its own equilibrium.
    """
    nx, ny, nz = shape
    N = nx * ny * nz
    rho = 1.0 + drho * (2.0 * uniform(seed, 0, N) - 1.0)
    u = umax * (2.0 * uniform(seed, 1, 3 * N) - 1.0)
    xi = 2.0 * uniform(seed, 2, 27 * N) - 1.0
    return (rho.reshape(nz, ny, nx), u.reshape(nz, ny, nx, 3), xi.reshape(27, nz, ny, nx))


def taylor_green_fields(shape, u0: float = 0.05):
    """Taylor-Green vortex on a periodic box, x^ = 2 pi x / n per axis:
    u = u0 sin x^ cos y^ cos z^, v = -u0 cos x^ sin y^ cos z^, w = 0,
    rho = 1 + (3 u0^2 / 16)(cos 2x^ + cos 2y^)(cos 2z^ + 2)."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(2 * np.pi * np.arange(nz) / nz, 2 * np.pi * np.arange(ny) / ny,
                          2 * np.pi * np.arange(nx) / nx, indexing="ij")
    u = np.zeros((nz, ny, nx, 3))
    u[..., 0] = u0 * np.sin(x) * np.cos(y) * np.cos(z)
    u[..., 1] = -u0 * np.cos(x) * np.sin(y) * np.cos(z)
    rho = 1.0 + 3.0 * u0 ** 2 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    return rho, u


def shear_wave_fields(shape, u0: float, axis_u: int = 0, axis_k: int = 1):
    """u_{axis_u} = u0 sin(2 pi x_{axis_k} / n_{axis_k}), rho = 1."""
    nx, ny, nz = shape
    coords = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xk = coords[2 - axis_k]
    n = shape[axis_k]
    u = np.zeros((nz, ny, nx, 3))
    u[..., axis_u] = u0 * np.sin(2 * np.pi * xk / n)
    return np.ones((nz, ny, nx)), u


def uniform_fields(shape, u=(0.0, 0.0, 0.0), rho: float = 1.0):
    nx, ny, nz = shape
    uu = np.zeros((nz, ny, nx, 3))
    uu[...] = np.asarray(u, dtype=np.float64)
    return np.full((nz, ny, nx), rho), uu


# ------------------------------------------------------------------ workloads
def tgv_periodic(n: int = 32, u0: float = 0.05, re: float = 1600.0):
    """Plain method on a periodic n^3 Taylor-Green box; nu from Re = u0 (n/2pi)/nu."""
    nu = u0 * (n / (2 * math.pi)) / re
    return dict(name=f"tgv_periodic_{n}^3", shape=(n, n, n), nu=nu, u0=u0, faces=(0,) * 6)


def sedimenting_sphere(shape=(128, 128, 256), D: float = 16.0, rho_ratio: float = 1.5,
                       u_t: float = 0.04, re: float = 100.0, cd: float = 1.1):
    """Two-way coupled sedimenting sphere: no-slip x and y walls (halfway
    bounce-back), periodic z, gravity along -z.  nu from Re = u_t D / nu = 100
    and gravity from the terminal-velocity force balance
    rho_s/rho_f = 1 + 3 u_t^2 C_d / (4 D g) with C_d = 1.1."""
    nx, ny, nz = shape
    nu = u_t * D / re
    g = 3.0 * u_t ** 2 * cd / (4.0 * D * (rho_ratio - 1.0))
    # centre off the lattice planes so no node sits on the surface
    X = (nx / 2 - 0.5 + 0.123, ny / 2 - 0.5 + 0.0567, 0.75 * nz + 0.311)
    return dict(name=f"sedimenting_sphere_{nx}x{ny}x{nz}_D{D:g}", shape=shape, nu=nu, D=D,
                X=X, rho_ratio=rho_ratio, g=(0.0, 0.0, -g), faces=(1, 1, 1, 1, 0, 0))


def airfoil_thickness(t_max: float = 0.0425, x_max: float = 0.25, a0: float = 0.126,
                      te_slope: float = -0.10):
    """Coefficients (a0..a4) of the half thickness t(x) = a0 sqrt(x) + a1 x +
    a2 x^2 + a3 x^3 + a4 x^4 with t(x_max) = t_max, t'(x_max) = 0, t(1) = 0,
    t'(1) = te_slope and a fixed leading-edge term a0 (8.5% thick at 25% chord
    by default)."""
    A = np.array([[x_max, x_max ** 2, x_max ** 3, x_max ** 4],
                  [1.0, 2 * x_max, 3 * x_max ** 2, 4 * x_max ** 3],
                  [1.0, 1.0, 1.0, 1.0],
                  [1.0, 2.0, 3.0, 4.0]])
    rhs = np.array([t_max - a0 * math.sqrt(x_max), -0.5 * a0 / math.sqrt(x_max), -a0, te_slope - 0.5 * a0])
    a = np.linalg.solve(A, rhs)
    return (a0, *[float(v) for v in a])


def plunging_airfoil(shape=(1024, 512, 64), chord: float = 128.0, u_inf: float = 0.05,
                     re: float = 40000.0, k: float = 3.93, h0: float = 0.05, alpha_deg: float = 4.0,
                     le=(256.37, 256.29)):
    """Plunging cambered airfoil: chord 128, extruded over a periodic span,
    equilibrium inflow at x-, zero-gradient outflow at x+, equilibrium
    far field on the y faces; plunge h(t) = h0 c sin(2 pi f t) along y with
    reduced frequency k = pi f c / u_inf; nu = u_inf c / Re."""
    nx, ny, nz = shape
    f = k * u_inf / (math.pi * chord)
    a = math.radians(alpha_deg)
    return dict(name=f"plunging_airfoil_{nx}x{ny}x{nz}_c{chord:g}", shape=shape, nu=u_inf * chord / re,
                chord=chord, ca=math.cos(a), sa=math.sin(a), h_amp=h0 * chord, h_omega=2 * math.pi * f,
                camber_m=0.015, camber_p=0.35, thick=airfoil_thickness(), le=le,
                faces=(2, 3, 2, 2, 0, 0), u_face=(u_inf, 0.0, 0.0))


def refined_block(shape=(512, 256, 64), lo=(128, 64, 8), hi=(383, 191, 55), u_inf: float = 0.05,
                  nu: float = 1e-3, amp: float = 0.01):
    """Two-level grid (Sec. 4.2 runs the airfoil on one): a bodiless coarse box
    with the airfoil box's faces (equilibrium inflow x-, outflow x+,
    equilibrium far field y, periodic z) and a ratio-2 block over the coarse
    nodes [lo, hi]; the fine lattice holds 2 (hi - lo) + 2 nodes per axis.
    The flow is the free stream plus a Taylor-Green perturbation of
    amplitude amp (refined_fields)."""
    nx, ny, nz = shape
    fine = tuple(2 * (h - l) + 2 for l, h in zip(lo, hi))
    return dict(name=f"refined_block_{nx}x{ny}x{nz}_fine_{fine[0]}x{fine[1]}x{fine[2]}", shape=shape,
                lo=lo, hi=hi, fine_shape=fine, nu=nu, faces=(2, 3, 2, 2, 0, 0), u_face=(u_inf, 0.0, 0.0),
                u_inf=u_inf, amp=amp)


def refined_airfoil(shape=(512, 256, 32), lo=(96, 64, 0), hi=(351, 191, 32), chord: float = 128.0,
                    u_inf: float = 0.05, re: float = 40000.0, k: float = 3.93, h0: float = 0.05,
                    alpha_deg: float = 4.0, le=(128.37, 128.29)):
    """The plunging airfoil (Sec. 4.2) on a two-level grid: a coarse box with
    the airfoil box's faces and a ratio-2 block over [lo, hi] in x and y that
    spans the periodic span (z), the airfoil on the fine level in fine
    lattice units (chord 128, leading edge at le of the fine lattice), so the
    airfoil sees the resolution of the single-level 1024 x 512 x 64 box near
    it.  Viscosity and plunge in fine units: nu_f = u_inf c / Re, the reduced
    frequency k = pi f c / u_inf per fine step; the coarse level takes nu_f /
    2 (acoustic scaling)."""
    nx, ny, nz = shape
    fine = tuple(2 * n if (l == 0 and h == n and a == 2) else 2 * (h - l) + 2
                 for a, (l, h, n) in enumerate(zip(lo, hi, shape)))
    f = k * u_inf / (math.pi * chord)
    a = math.radians(alpha_deg)
    nu_f = u_inf * chord / re
    return dict(name=f"refined_airfoil_{nx}x{ny}x{nz}_fine_{fine[0]}x{fine[1]}x{fine[2]}_c{chord:g}",
                shape=shape, lo=lo, hi=hi, fine_shape=fine, nu=nu_f / 2, faces=(2, 3, 2, 2, 0, 0),
                u_face=(u_inf, 0.0, 0.0), u_inf=u_inf, chord=chord, ca=math.cos(a), sa=math.sin(a),
                h_amp=h0 * chord, h_omega=2 * math.pi * f, camber_m=0.015, camber_p=0.35,
                thick=airfoil_thickness(), le=le)


def refined_fields(wl, level: str):
    """(rho, u) of the refined block workload on the coarse or the fine level:
    u = (u_inf, 0, 0) + amp * (sin x^ cos y^ cos z^, -cos x^ sin y^ cos z^, 0)
    with x^ = 2 pi x / n over the coarse box, evaluated at the level's node
    positions (fine node j at coarse coordinate lo + j/2); rho = 1."""
    nx, ny, nz = wl["shape"]
    if level == "coarse":
        dims, org, h = wl["shape"], (0, 0, 0), 1.0
    else:
        dims, org, h = wl["fine_shape"], wl["lo"], 0.5
    ax = [2 * np.pi * (org[a] + h * np.arange(dims[a])) / wl["shape"][a] for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    u = np.zeros((dims[2], dims[1], dims[0], 3))
    u[..., 0] = wl["u_inf"] + wl["amp"] * np.sin(x) * np.cos(y) * np.cos(z)
    u[..., 1] = -wl["amp"] * np.cos(x) * np.sin(y) * np.cos(z)
    return np.ones((dims[2], dims[1], dims[0])), u


# ------------------------------------------------------------------ swimmer
def swimmer_half_width(s, L: float):
    """Half width w(s) of the anguilliform body (Sec. 4.3): sqrt(2 w_h s - s^2)
    up to s_b, a quadratic decrease to w_t at s_t, then linear to zero at the
    tail; w_h = s_b = 0.04 L, s_t = 0.95 L, w_t = 0.01 L."""
    s = np.asarray(s, dtype=np.float64)
    wh = sb = 0.04 * L
    st, wt = 0.95 * L, 0.01 * L
    a = np.sqrt(np.clip(2.0 * wh * s - s * s, 0.0, None))
    b = wh - (wh - wt) * ((s - sb) / (st - sb)) ** 2
    c = wt * (L - s) / (L - st)
    return np.where(s < sb, a, np.where(s < st, b, np.clip(c, 0.0, None)))


def swimmer_half_height(s, L: float):
    """Half height h(s) = b sqrt(1 - ((s - a)/a)^2), a = 0.51 L, b = 0.08 L (Sec. 4.3)."""
    s = np.asarray(s, dtype=np.float64)
    a, b = 0.51 * L, 0.08 * L
    return b * np.sqrt(np.clip(1.0 - ((s - a) / a) ** 2, 0.0, None))


def swimmer_mesh(L: float, segments: int = 150, ring: int = 64):
    """Closed triangulated surface of elliptic cross sections along the centre
    line (Sec. 4.3: 150 segments).  Returns (rest, tris): rest[v] = (s, dy, dz),
    the arc position and the offsets of vertex v from the centre line, and
    tris[k] = three vertex indices, counter-clockwise seen from outside.
    Vertex 0 is the head (s = 0), then `segments` rings of `ring` vertices at
    s = k L / segments, k = 1..segments, then the tail-cap centre (s = L).  The
    tail ring has zero width, so the cap triangles have zero area."""
    rest = [(0.0, 0.0, 0.0)]
    phi = 2.0 * np.pi * (np.arange(ring) + 0.5) / ring
    for k in range(1, segments + 1):
        s = L * k / segments
        w = float(swimmer_half_width(s, L))
        h = float(swimmer_half_height(s, L))
        for j in range(ring):
            rest.append((s, w * math.cos(phi[j]), h * math.sin(phi[j])))
    tail = len(rest)
    rest.append((float(L), 0.0, 0.0))

    def rv(k, j):  # vertex of ring k (1-based), position j
        return 1 + (k - 1) * ring + (j % ring)

    tris = []
    # (ds, dy, dz) axes: outward normal of the head fan points to -s
    for j in range(ring):
        tris.append((0, rv(1, j + 1), rv(1, j)))
    for k in range(1, segments):
        for j in range(ring):
            a, b = rv(k, j), rv(k, j + 1)
            c, d = rv(k + 1, j), rv(k + 1, j + 1)
            tris.append((a, b, d))
            tris.append((a, d, c))
    for j in range(ring):
        tris.append((tail, rv(segments, j), rv(segments, j + 1)))
    return np.asarray(rest, dtype=np.float64), np.asarray(tris, dtype=np.int32)


def swimmer_volume(L: float, n: int = 200001) -> float:
    """Volume of the analytic body, integral of pi w(s) h(s) ds (trapezoidal rule)."""
    s = np.linspace(0.0, L, n)
    return float(np.trapezoid(np.pi * swimmer_half_width(s, L) * swimmer_half_height(s, L), s))


def anguilliform_swimmer(shape=(768, 256, 256), L: float = 128.0, period: float = 4000.0,
                         amp: float = 0.125, wavelength=None, re: float = 7142.0,
                         segments: int = 150, ring: int = 64, ramp: bool = False,
                         head=None):
    """Self-propelled anguilliform swimmer (Sec. 4.3): body of length L, midline
    y(s,t) = amp L (s/L + 0.03125)/1.03125 sin(2 pi (s/lambda - t/T)), free in x,
    neutrally buoyant (m = rho0 V), all faces periodic; nu from Re = (L^2/T)/nu.
    The head starts at 2/3 of the box length, heading -x; the centre line sits
    off the lattice planes."""
    nx, ny, nz = shape
    if head is None:
        head = (round(2 * nx / 3) + 0.137, ny / 2 + 0.371, nz / 2 + 0.293)
    rest, tris = swimmer_mesh(L, segments, ring)
    return dict(name=f"anguilliform_swimmer_{nx}x{ny}x{nz}_L{L:g}", shape=shape,
                nu=(L * L / period) / re, L=L, period=period, amp=amp,
                wavelength=L if wavelength is None else wavelength, ramp=int(ramp),
                X=tuple(head), mass=swimmer_volume(L), rest=rest, tris=tris, faces=(0,) * 6)


def differentiated_swimmer(shape=(256, 128, 128), L: float = 64.0, period: float = 4000.0,
                           amp: float = 0.125, re: float = 7142.0, segments: int = 150, ring: int = 64):
    """The swimmer of Sec. 4.3 held in place (no free motion) in a 4L x 2L x 2L
    periodic box, for gradients of its mean thrust with respect to the
    kinematic parameters; same midline law, nu = (L^2/T)/Re."""
    nx, ny, nz = shape
    rest, tris = swimmer_mesh(L, segments, ring)
    head = (nx / 2 - L / 2 + 0.137, ny / 2 + 0.371, nz / 2 + 0.293)
    return dict(name=f"differentiated_swimmer_{nx}x{ny}x{nz}_L{L:g}", shape=shape, nu=(L * L / period) / re,
                L=L, period=period, amp=amp, wavelength=L, ramp=0, X=head, mass=swimmer_volume(L),
                rest=rest, tris=tris, faces=(0,) * 6)
