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
