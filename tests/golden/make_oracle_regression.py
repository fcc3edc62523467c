"""Writes tests/golden/oracle_regression.txt: outputs of short oracle runs of
each body kind and of the two-level grid (force, torque, body state, and
three sums of the populations' deviations from rest: plain, squared, and
weighted by cos(0.37 n) over the flat index n, which a permutation would
change), so a
change to the oracle's arithmetic shows up as a failing comparison that its
commit must then justify from the paper.  Calls only the oracle and the seeded
input generators.

    python tests/golden/make_oracle_regression.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "oracle_regression.txt")


def cases():
    """name -> (shape, Oracle keyword arguments, body factory, steps)."""
    wl = synth.plunging_airfoil()
    rest, tris = synth.swimmer_mesh(24.0, 24, 12)
    return {
        "periodic_kbc": ((12, 10, 8), dict(nu=0.01), lambda: None, 5),
        "periodic_exact_gamma": ((8, 8, 8), dict(nu=0.01, gamma_mode=oracle.MODE_EXACT), lambda: None, 3),
        "sphere_free_walls": ((16, 14, 18), dict(nu=0.02, faces=(1, 1, 1, 1, 0, 0)),
                              lambda: oracle.sphere_body((7.3, 6.6, 9.1), 3.1, U=(0.05, -0.02, -0.1), free=True,
                                                         g=(0.0, 0.0, -1e-3)), 5),
        "airfoil_plunging": ((40, 24, 3), dict(nu=0.02, faces=(2, 3, 2, 2, 0, 0), u_face=(0.05, 0.0, 0.0)),
                             lambda: oracle.airfoil_body((10.3, 12.2), 20.0, wl["ca"], wl["sa"], 3.0, 0.1,
                                                         wl["camber_m"], wl["camber_p"], wl["thick"], 3.0), 4),
        "swimmer_free_xyyaw": ((48, 24, 20), dict(nu=0.02),
                               lambda: oracle.mesh_body((22.137, 12.371, 10.293), rest, tris, 24.0, 0.125, 24.0, 32.0,
                                                        free=7, mass=synth.swimmer_volume(24.0), psi=0.1,
                                                        omega=0.002), 3),
    }


def run(name, shape, kw, make_body, steps):
    body = make_body()
    o = oracle.Oracle(shape, body=body, **kw) if body is not None else oracle.Oracle(shape, **kw)
    rho, u, xi = synth.parity_fields(shape, 21)
    o.init_state(rho, u * 0.5, xi, 1e-3)
    o.step(steps)
    _, W = oracle.lattice()
    g = (o.get_f() - W[:, None, None, None]).reshape(-1)  # deviations from rest, rho0 = 1
    b = o.body
    vals = {"g_sum": float(g.sum()), "g_sq_sum": float((g * g).sum()),
            "g_cos": float((g * np.cos(0.37 * np.arange(g.size))).sum())}
    if body is not None:
        for k in ("F", "M", "X", "U"):
            for a in range(3):
                vals[f"{k}{a}"] = float(getattr(b, k)[a])
        vals["psi"], vals["omega"] = float(b.psi), float(b.omega)
    return vals


def refined_cases():
    """name -> (coarse shape, lo, hi, Oracle keyword arguments, fine body factory, coarse steps)."""
    return {
        "refined_block": ((20, 16, 14), (4, 3, 3), (13, 11, 9), dict(nu=0.02), lambda: None, 3),
        "refined_span_free_sphere": ((24, 20, 8), (6, 5, 0), (17, 14, 8), dict(nu=0.02),
                                     lambda: oracle.sphere_body((11.3, 9.4, 7.6), 2.6, U=(0.02, 0.005, 0.01),
                                                                free=True, rho_ratio=2.0), 3),
    }


def run_refined(name, shape, lo, hi, kw, make_body, steps):
    body = make_body()
    o = oracle.Oracle(shape, **kw)
    rho, u, xi = synth.parity_fields(shape, 22)
    o.init_state(rho, u * 0.5, xi, 1e-3)
    r = oracle.RefinedOracle(o, lo, hi, fine_body=body)
    frho, fu, fxi = synth.parity_fields(r.fine.shape, 23)
    r.fine.init_state(frho, fu * 0.5, fxi, 1e-3)
    r.init()
    r.step(steps)
    _, W = oracle.lattice()
    vals = {}
    for lev, f, valid in (("c", o.get_f(), r.coarse_valid()), ("f", r.fine.get_f(), r.fine_valid())):
        g = (f - W[:, None, None, None])[:, valid].reshape(-1)
        vals[f"{lev}_g_sum"] = float(g.sum())
        vals[f"{lev}_g_sq_sum"] = float((g * g).sum())
        vals[f"{lev}_g_cos"] = float((g * np.cos(0.37 * np.arange(g.size))).sum())
    if body is not None:
        b = r.fine.body
        for k in ("F", "M", "X", "U"):
            for a in range(3):
                vals[f"{k}{a}"] = float(getattr(b, k)[a])
    return vals


def compute():
    res = {name: run(name, *c) for name, c in cases().items()}
    res.update({name: run_refined(name, *c) for name, c in refined_cases().items()})
    return res


def main():
    res = compute()
    with open(OUT, "w") as fh:
        fh.write("# Outputs of short FP64 oracle runs (tests/golden/make_oracle_regression.py):\n")
        fh.write("# case key value (repr of the double)\n")
        for name, vals in res.items():
            for k, v in vals.items():
                fh.write(f"{name} {k} {v!r}\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
