// Body geometry on the device: solid test, nearest image on periodic axes,
// pull sources under the box rules, link fraction and wall velocity
// (arXiv 1608.04658, Secs. 3 and 4.1).
//
// Floating-point decisions that set node marks are taken in IEEE double with
// explicitly rounded operations (no FMA contraction), so they reproduce the
// same decisions as a plain double evaluation of the same expressions.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

__device__ __forceinline__ int wrap_or_clip(int u, int n, int periodic)
{
    if (periodic) {
        int r = u % n;
        return r < 0 ? r + n : r;
    }
    return u;
}

// Displacement of lattice coordinate p from the centre coordinate X on one
// axis; on a periodic axis the nearest image (X in [0, n), one add or
// subtract of n when |d| > n/2).
__device__ __forceinline__ double axis_offset(int p, double X, int n, int periodic)
{
    double d = __dsub_rn((double)p, X);
    if (periodic) {
        const double h = 0.5 * (double)n;
        if (d > h) d = __dsub_rn(d, (double)n);
        else if (d < -h) d = __dadd_rn(d, (double)n);
    }
    return d;
}

// Airfoil in its chord frame (see lbm_geometry): camber line and half thickness
__device__ __forceinline__ double airfoil_camber(const GeomParams &G, double xi)
{
    const double m = G.camber_m, p = G.camber_p;
    if (xi < p) return __dmul_rn(__ddiv_rn(m, __dmul_rn(p, p)), __dsub_rn(__dmul_rn(__dmul_rn(2.0, p), xi), __dmul_rn(xi, xi)));
    const double q = __dsub_rn(1.0, p);
    return __dmul_rn(__ddiv_rn(m, __dmul_rn(q, q)),
                     __dsub_rn(__dadd_rn(__dsub_rn(1.0, __dmul_rn(2.0, p)), __dmul_rn(__dmul_rn(2.0, p), xi)), __dmul_rn(xi, xi)));
}

__device__ __forceinline__ double airfoil_half_thickness(const GeomParams &G, double xi)
{
    const double *a = G.thick;
    const double poly = __dmul_rn(xi, __dadd_rn(a[1], __dmul_rn(xi, __dadd_rn(a[2], __dmul_rn(xi, __dadd_rn(a[3], __dmul_rn(xi, a[4])))))));
    return __dadd_rn(__dmul_rn(a[0], __dsqrt_rn(xi)), poly);
}

__device__ __forceinline__ bool inside_airfoil(const GeomParams &G, const double X[3], double x, double y)
{
    const double dx = __dsub_rn(x, X[0]), dy = __dsub_rn(y, X[1]);
    const double xi = __ddiv_rn(__dsub_rn(__dmul_rn(dx, G.ca), __dmul_rn(dy, G.sa)), G.chord);
    const double eta = __ddiv_rn(__dadd_rn(__dmul_rn(dx, G.sa), __dmul_rn(dy, G.ca)), G.chord);
    if (xi < 0.0 || xi > 1.0) return false;
    return fabs(__dsub_rn(eta, airfoil_camber(G, xi))) < airfoil_half_thickness(G, xi);
}

__device__ __forceinline__ bool inside_body(const GeomParams &G, const Lattice &L, const double X[3],
                                            int x, int y, int z)
{
    if (G.kind == LBM_BODY_AIRFOIL) return inside_airfoil(G, X, (double)x, (double)y);
    if (G.kind == LBM_BODY_SPHERE) {
        const double dx = axis_offset(x, X[0], L.nx, G.periodic[0]);
        const double dy = axis_offset(y, X[1], L.ny, G.periodic[1]);
        const double dz = axis_offset(z, X[2], L.nz, G.periodic[2]);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        return d2 < __dmul_rn(G.R, G.R);
    }
    if (G.kind == LBM_BODY_PLANES) return (double)y < G.y_lo || (double)y > G.y_hi;
    return false;
}

// Pull source x - c under the box rules; node index, or -1 when a wall or
// equilibrium face serves the pull (such a source is never solid).
__device__ __forceinline__ int pull_source(const Lattice &L, int x, int y, int z, int cx, int cy, int cz)
{
    int p[3] = {x - cx, y - cy, z - cz};
    const int n[3] = {L.nx, L.ny, L.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int face = -1;
        if (p[a] < 0) face = L.face[2 * a];
        else if (p[a] >= n[a]) face = L.face[2 * a + 1];
        if (face < 0) continue;
        if (face == LBM_FACE_PERIODIC) p[a] = (p[a] + n[a]) % n[a];
        else if (face == LBM_FACE_OUTFLOW) p[a] = p[a] < 0 ? 0 : n[a] - 1;
        else return -1;
    }
    return p[0] + L.nx * (p[1] + L.ny * p[2]);
}

// x + d with periodic wrap; -1 when it leaves the box through a non-periodic face
__device__ __forceinline__ int neighbour(const Lattice &L, int x, int y, int z, int dx, int dy, int dz)
{
    int p[3] = {x + dx, y + dy, z + dz};
    const int n[3] = {L.nx, L.ny, L.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (p[a] >= 0 && p[a] < n[a]) continue;
        const int face = p[a] < 0 ? L.face[2 * a] : L.face[2 * a + 1];
        if (face != LBM_FACE_PERIODIC) return -1;
        p[a] = (p[a] + n[a]) % n[a];
    }
    return p[0] + L.nx * (p[1] + L.ny * p[2]);
}

// Link of boundary node (x, y, z) towards the solid node x - c: fraction q of
// the link at which the wall is crossed (wall point x_w = x - q c, q in (0,1])
// and the wall velocity there.
__device__ __forceinline__ void link_data(const Lattice &L, const GeomParams &G, const DevBody *b,
                                          int x, int y, int z, int cx, int cy, int cz, double &q,
                                          double uw[3])
{
    if (G.kind == LBM_BODY_SPHERE) {
        const double d0 = axis_offset(x, b->X[0], L.nx, G.periodic[0]);
        const double d1 = axis_offset(y, b->X[1], L.ny, G.periodic[1]);
        const double d2 = axis_offset(z, b->X[2], L.nz, G.periodic[2]);
        const double cc = (double)(cx * cx + cy * cy + cz * cz);
        const double cd = cx * d0 + cy * d1 + cz * d2;
        const double dd = d0 * d0 + d1 * d1 + d2 * d2;
        const double disc = cd * cd - cc * (dd - G.R * G.R);
        q = (cd - sqrt(fmax(disc, 0.0))) / cc;
        uw[0] = b->U[0];
        uw[1] = b->U[1];
        uw[2] = b->U[2];
    } else if (G.kind == LBM_BODY_AIRFOIL) {
        // crossing of the link x - s c, s in [0, 1], by 50 bisections
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 50; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (inside_airfoil(G, b->X, __dsub_rn((double)x, __dmul_rn(mid, (double)cx)),
                               __dsub_rn((double)y, __dmul_rn(mid, (double)cy))))
                hi = mid;
            else
                lo = mid;
        }
        q = 0.5 * (lo + hi);
        uw[0] = b->U[0];
        uw[1] = b->U[1];
        uw[2] = b->U[2];
    } else {  // planes
        const double yb = (double)y;
        const bool low = (double)(y - cy) < G.y_lo;
        q = low ? (yb - G.y_lo) / (double)cy : (G.y_hi - yb) / (double)(-cy);
        const double *v = low ? G.U_lo : G.U_hi;
        uw[0] = v[0];
        uw[1] = v[1];
        uw[2] = v[2];
    }
}

// torque arm origin: displacement of (x, y, z) from the body reference point
// (sphere centre; airfoil leading edge at z = 0; the lattice origin otherwise)
__device__ __forceinline__ double body_offset(const Lattice &L, const GeomParams &G, const DevBody *b,
                                              int a, int p)
{
    if (G.kind == LBM_BODY_AIRFOIL) return a < 2 ? __dsub_rn((double)p, b->X[a]) : (double)p;
    if (G.kind != LBM_BODY_SPHERE) return (double)p;
    const int n = a == 0 ? L.nx : (a == 1 ? L.ny : L.nz);
    return axis_offset(p, b->X[a], n, G.periodic[a]);
}

}  // namespace lbm
