"""Differentiable restatement of the plain KBC step in PyTorch FP64.

TEST INFRASTRUCTURE ONLY.  Only the test suite may import this module.  It
restates, with whole-lattice tensor operations, the step of arXiv 1608.04658
for a box without an immersed body, so that PyTorch's autograd tape gives a
reference gradient of any function of the state after a few steps.  It shares
no code with the CUDA library or with the C oracle.

  Sec. 2, Eq. (kineticEq)  pull streaming F_i(x) = f'_i(x - c_i), box faces
                           periodic / halfway bounce-back wall / equilibrium /
                           zero-gradient outflow, precedence wall > equilibrium
                           > clamped or wrapped source;
  Sec. 2, Eq. (feq_min)    exact D3Q27 product-form equilibrium;
  Sec. 2, Eq. (kbc_relax)  KBC split (s = deviatoric natural second moments,
                           h = the rest of the deviation) and the analytic
                           stabilizer g = 1/b - (2 - 1/b) <ds|dh>/<dh|dh>
                           (g = 2 when <dh|dh> <= 1e-300, or always in LBGK
                           mode).
Arrays are (27, nz, ny, nx) with direction i = 9(cx+1) + 3(cy+1) + (cz+1).
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64
PERIODIC, WALL, EQ, OUTFLOW = 0, 1, 2, 3


def lattice():
    c = np.array([[a, b, d] for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)], dtype=np.int64)
    w1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
    W = np.array([w1[a] * w1[b] * w1[d] for a, b, d in c])
    return c, W


C_NP, W_NP = lattice()
C = torch.tensor(C_NP, dtype=DT)
W = torch.tensor(W_NP, dtype=DT)


def equilibrium(rho: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """f^eq_i = rho prod_a w(c_ia) (2 - S_a) B_a^{c_ia}, S = sqrt(1 + 3u^2),
    B = (2u + S)/(1 - u); rho (...), u (3, ...) -> (27, ...)."""
    S = torch.sqrt(1.0 + 3.0 * u * u)
    B = (2.0 * u + S) / (1.0 - u)
    shape = (27,) + (1,) * rho.dim()
    out = rho.unsqueeze(0).expand((27,) + tuple(rho.shape)).clone()
    for a in range(3):
        ca = C[:, a].reshape(shape)
        w = torch.where(ca == 0, torch.tensor(2.0 / 3.0, dtype=DT), torch.tensor(1.0 / 6.0, dtype=DT))
        out = out * w * (2.0 - S[a]).unsqueeze(0) * torch.pow(B[a].unsqueeze(0), ca)
    return out


def collide(f: torch.Tensor, beta: float, lbgk: bool = False) -> torch.Tensor:
    """KBC collision f' = f - b (2 ds + g dh) of populations f (27, ...)."""
    shape = (27,) + (1,) * (f.dim() - 1)
    cc = [C[:, a].reshape(shape) for a in range(3)]
    rho = f.sum(0)
    u = torch.stack([(cc[a] * f).sum(0) for a in range(3)]) / rho
    fe = equilibrium(rho, u)
    df = f - fe
    # natural second moments of the deviation and their deviatoric part; s is
    # rebuilt from them: one unit of M_ab (a != b) is c_a c_b / 4 on the four
    # edge directions of the ab plane; one unit of M_aa is 1/2 on the two
    # +-a faces and -1 on the rest population, and the rest terms cancel for
    # the traceless deviatoric part
    P = [[(cc[a] * cc[b] * df).sum(0) for b in range(3)] for a in range(3)]
    tr = P[0][0] + P[1][1] + P[2][2]
    zero = torch.zeros((), dtype=DT)
    ds = torch.zeros_like(f)
    for a in range(3):
        for b in range(a + 1, 3):
            k = 3 - a - b
            edge = (cc[a] != 0) & (cc[b] != 0) & (cc[k] == 0)
            ds = ds + torch.where(edge, cc[a] * cc[b] / 4.0, zero) * P[a][b]
        face = (cc[a] != 0) & (cc[(a + 1) % 3] == 0) & (cc[(a + 2) % 3] == 0)
        ds = ds + torch.where(face, torch.full((), 0.5, dtype=DT), zero) * (P[a][a] - tr / 3.0)
    dh = df - ds
    sh = (ds * dh / fe).sum(0)
    hh = (dh * dh / fe).sum(0)
    if lbgk:
        g = torch.full_like(hh, 2.0)
    else:
        safe = torch.where(hh > 1e-300, hh, torch.ones_like(hh))
        g = torch.where(hh > 1e-300, 1.0 / beta - (2.0 - 1.0 / beta) * sh / safe, torch.full_like(hh, 2.0))
    return f - beta * (2.0 * ds + g.unsqueeze(0) * dh)


class Box:
    """Pull streaming on an nx x ny x nz box with faces (x-, x+, y-, y+, z-, z+)."""

    def __init__(self, shape, faces=(PERIODIC,) * 6, rho0=1.0, u_face=(0.0, 0.0, 0.0)):
        nx, ny, nz = shape
        self.shape = shape
        n = np.array([nx, ny, nz])
        N = nx * ny * nz
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        pos = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
        src = np.zeros((27, N), dtype=np.int64)
        kind = np.zeros((27, N), dtype=np.int64)  # 0 node, 1 wall, 2 equilibrium
        for i in range(27):
            p = pos - C_NP[i]
            wall = np.zeros(N, bool)
            eq = np.zeros(N, bool)
            for a in range(3):
                lo, hi = p[:, a] < 0, p[:, a] >= n[a]
                for side, m in ((0, lo), (1, hi)):
                    f = faces[2 * a + side]
                    if f == PERIODIC:
                        p[m, a] = (p[m, a] + n[a]) % n[a]
                    elif f == OUTFLOW:
                        p[m, a] = 0 if side == 0 else n[a] - 1
                    elif f == WALL:
                        wall |= m
                    else:
                        eq |= m
            p = np.clip(p, 0, n - 1)
            src[i] = p[:, 0] + nx * (p[:, 1] + ny * p[:, 2])
            kind[i] = np.where(wall, 1, np.where(eq, 2, 0))
        self.src = torch.tensor(src)
        self.kind = torch.tensor(kind)
        u = torch.tensor(u_face, dtype=DT).reshape(3)
        self.feq_face = equilibrium(torch.tensor(rho0, dtype=DT), u)

    def stream(self, f: torch.Tensor) -> torch.Tensor:
        nz, ny, nx = f.shape[1:]
        flat = f.reshape(27, -1)
        out = []
        for i in range(27):
            node = flat[i][self.src[i]]
            bb = flat[26 - i]
            v = torch.where(self.kind[i] == 1, bb, node)
            v = torch.where(self.kind[i] == 2, self.feq_face[i].expand_as(v), v)
            out.append(v)
        return torch.stack(out).reshape(27, nz, ny, nx)

    def step(self, f: torch.Tensor, beta: float, lbgk: bool = False) -> torch.Tensor:
        return collide(self.stream(f), beta, lbgk)
