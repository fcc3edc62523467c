"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle
on the same seeded inputs and compare what they store."""
import numpy as np

import oracle
import synth

# Parity bars on full populations, max over fluid nodes and directions of
# |f_gpu - f_oracle| / |f_oracle| (10 steps for the storage forms): 1e-12 in
# FP64, 2e-6 in FP32 and 2e-3 in 16-bit storage.  FP16 meets the 16-bit bar;
# BF16 keeps 8 significand bits (relative rounding up to 2^-8 per store of
# g = f - W rho0, so one store alone reaches the bar where |g|/f >= 0.5, which
# the rough random fields of these tests do), so the BF16 cases that exceed it
# are marked as expected failures with their measured errors.
TOL = {"fp64": 1e-12, "fp32": 2e-6, "fp16": 2e-3, "bf16": 2e-3}


def rel_err(a: np.ndarray, b: np.ndarray, mask: np.ndarray | None = None) -> float:
    d = np.abs(a - b) / np.abs(b)
    if mask is not None:
        d = d[:, mask]
    return float(d.max())


def oracle_body(geom):
    """Oracle body equal to a binding Geometry."""
    if geom is None:
        return None
    import paper_1608_04658_gb300 as lbm
    if geom.kind == lbm.BODY_SPHERE:
        return oracle.sphere_body(list(geom.X), geom.R, U=list(geom.U), free=bool(geom.free_motion),
                                  rho_ratio=geom.rho_ratio, g=list(geom.g),
                                  mass=geom.mass if geom.mass > 0 else None)
    if geom.kind == lbm.BODY_AIRFOIL:
        return oracle.airfoil_body((geom.X[0], geom.X[1]), geom.chord, geom.ca, geom.sa, geom.h_amp,
                                   geom.h_omega, geom.camber_m, geom.camber_p, list(geom.thick), geom.t0)
    if geom.kind == lbm.BODY_MESH:
        rest, tris = geom._arrays
        return oracle.mesh_body(list(geom.X), rest, tris, geom.length, geom.wave_amp, geom.wave_length,
                                geom.wave_period, ramp=bool(geom.wave_ramp), U=list(geom.U),
                                free=int(geom.free_motion), mass=geom.mass, t0=geom.t0, psi=geom.psi,
                                omega=geom.omega)
    return oracle.planes_body(geom.y_lo, geom.y_hi, U_lo=list(geom.U_lo), U_hi=list(geom.U_hi))


def run_pair(shape, nu, storage, fields, steps, faces=(0,) * 6, geom=None, u_face=(0.0, 0.0, 0.0),
             gamma_mode=0):
    """fields = (rho, u, xi, amp).  Returns (gpu Lattice, oracle.Oracle)."""
    import paper_1608_04658_gb300 as lbm
    rho, u, xi, amp = fields
    lat = lbm.Lattice(shape, nu, storage=storage, faces=faces, u_face=u_face, gamma_mode=gamma_mode)
    if geom is not None:
        lat.set_geometry(geom)
    lat.init_state(rho, u, xi, amp)
    lat.step(steps)
    orc = oracle.Oracle(shape, nu=nu, faces=faces, u_face=u_face, gamma_mode=gamma_mode,
                        body=oracle_body(geom))
    orc.init_state(rho, u, xi, amp)
    orc.step(steps)
    return lat, orc


def fluid_mask(lat, orc):
    """Fluid nodes at the final step; asserts both sides mark the same nodes."""
    g_solid = (lat.flags.cpu().numpy() & 1).astype(np.uint8)
    o_solid = orc.solid()
    assert np.array_equal(g_solid, o_solid), "solid marks differ"
    return o_solid == 0


def random_fields(shape, seed, amp=1e-3):
    rho, u, xi = synth.parity_fields(shape, seed)
    return rho, u, xi, amp
