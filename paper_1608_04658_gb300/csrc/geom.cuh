// Body geometry on the device: solid test, nearest image on periodic axes,
// pull sources under the box rules, link fraction and wall velocity
// (arXiv 1608.04658, Secs. 3 and 4.1).
//
// Floating-point decisions that set node marks are taken in IEEE double with
// explicitly rounded operations (no FMA contraction), so they reproduce the
// same decisions as a plain double evaluation of the same expressions.
#pragma once

#include "body.cuh"

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

// Displacement of lattice coordinate p on axis a from the body coordinate X
// in the whole box's frame: a slab's z layers sit at zoff of a box periodic
// in z with zper layers (nearest image there), other axes as axis_offset.
__device__ __forceinline__ double frame_offset(int a, int p, double X, int n, int periodic, int zoff, int zper)
{
    if (a == 2 && zper > 0) return axis_offset(p + zoff, X, zper, 1);
    return axis_offset(p, X, n, periodic);
}

// A z coordinate of the whole box in a slab's own frame, at the image
// nearest the slab's middle layer (no slab: unchanged).
__device__ __forceinline__ double slab_z(const GeomParams &G, double Zg, int nz)
{
    if (G.zper <= 0) return Zg;
    double z = __dsub_rn(Zg, (double)G.zoff);
    const double mid = 0.5 * (double)nz, per = (double)G.zper;
    if (z - mid > 0.5 * per) z = __dsub_rn(z, per);
    else if (z - mid < -0.5 * per) z = __dadd_rn(z, per);
    return z;
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
        const double dz = frame_offset(2, z, X[2], L.nz, G.periodic[2], G.zoff, G.zper);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        return d2 < __dmul_rn(G.R, G.R);
    }
    if (G.kind == LBM_BODY_PLANES) return (double)y < G.y_lo || (double)y > G.y_hi;
    return false;
}

// ---------------------------------------------------------------- swimmer mesh
// Anguilliform swimmer (Sec. 4.3): midline, material velocity, ray-parity
// solid test on per-column crossing lists and the link search on triangle
// cells.  The solid decision (edge values, crossing abscissa) uses the same
// explicitly rounded double expressions as a plain evaluation.
constexpr double MESH_PI = 3.14159265358979323846;

// y(s,t) = r(t) a L (s/L + 0.03125)/1.03125 sin(2 pi (s/lambda - t/T))
__device__ __forceinline__ double swimmer_midline(const GeomParams &G, double s, double t)
{
    double r = 1.0;
    if (G.wave_ramp) {
        if (t < 0.0) r = 0.0;
        else if (t < G.wave_period)
            r = __dmul_rn(0.5, __dsub_rn(1.0, cos(__ddiv_rn(__dmul_rn(MESH_PI, t), G.wave_period))));
    }
    const double A = __ddiv_rn(__dmul_rn(__dmul_rn(G.wave_amp, G.length), __dadd_rn(__ddiv_rn(s, G.length), 0.03125)),
                               1.03125);
    const double arg = __dmul_rn(2.0 * MESH_PI, __dsub_rn(__ddiv_rn(s, G.wave_length), __ddiv_rn(t, G.wave_period)));
    return __dmul_rn(r, __dmul_rn(A, sin(arg)));
}

// material velocity at arc position s (already clamped to [0, L]) at the pose
// of body time t: U plus the central difference of the midline along y
__device__ __forceinline__ void swimmer_velocity(const GeomParams &G, const double U[3], double t, double s,
                                                 double v[3])
{
    const double m1 = swimmer_midline(G, s, __dadd_rn(t, 1.0));
    const double m0 = swimmer_midline(G, s, __dsub_rn(t, 1.0));
    v[0] = U[0];
    v[1] = __dadd_rn(U[1], __ddiv_rn(__dsub_rn(m1, m0), 2.0));
    v[2] = U[2];
}

__device__ __forceinline__ double clamp_arc(const GeomParams &G, double s)
{
    return s < 0.0 ? 0.0 : (s > G.length ? G.length : s);
}

// material velocity of the swimmer at world point (px, py) of the current
// pose.  Head frame: that of the arc position px - X0.  Centre-of-mass frame:
// U + omega e_z x (p - X) + R(psi) ((0, y_rate(s), 0) - c_dot) at the
// body-frame abscissa s of p (Sec. 4.3, rigid motion plus deformation)
__device__ __forceinline__ void mesh_material_velocity(const GeomParams &G, const DevBody *b, double px, double py,
                                                       double v[3])
{
    if (!G.com_frame) {
        swimmer_velocity(G, b->U, b->t, clamp_arc(G, px - b->X[0]), v);
        return;
    }
    const double cs = cos(b->psi), sn = sin(b->psi);
    const double rx = px - b->X[0], ry = py - b->X[1];
    const double s = clamp_arc(G, cs * rx + sn * ry + b->com[0]);
    const double rate = (swimmer_midline(G, s, b->t + 1.0) - swimmer_midline(G, s, b->t - 1.0)) / 2.0;
    const double wx = -b->com_dot[0], wy = rate - b->com_dot[1];
    v[0] = b->U[0] - b->omega * ry + (cs * wx - sn * wy);
    v[1] = b->U[1] + b->omega * rx + (sn * wx + cs * wy);
    v[2] = b->U[2];
}

// edge value of the (y, z) projection of directed edge u -> v at (y, z),
// evaluated from the lower-index vertex; sign with zero counted positive in
// that direction
__device__ __forceinline__ double mesh_edge(const double *__restrict__ P, int u, int v, double y, double z, int &sg)
{
    const int a = u < v ? u : v, b = u < v ? v : u;
    const double Ay = P[3 * a + 1], Az = P[3 * a + 2], By = P[3 * b + 1], Bz = P[3 * b + 2];
    double val = __dsub_rn(__dmul_rn(__dsub_rn(By, Ay), __dsub_rn(z, Az)), __dmul_rn(__dsub_rn(Bz, Az), __dsub_rn(y, Ay)));
    sg = val >= 0.0 ? 1 : -1;
    if (u > v) { val = -val; sg = -sg; }
    return val;
}

// does the line {(., y, z)} cross triangle t?  xc = crossing abscissa
__device__ __forceinline__ bool mesh_column_crossing(const double *__restrict__ P, int t0, int t1, int t2,
                                                     double y, double z, double &xc)
{
    int s0, s1, s2;
    const double e0 = mesh_edge(P, t1, t2, y, z, s0);
    const double e1 = mesh_edge(P, t2, t0, y, z, s1);
    const double e2 = mesh_edge(P, t0, t1, y, z, s2);
    if (s0 != s1 || s1 != s2) return false;
    const double den = __dadd_rn(__dadd_rn(e0, e1), e2);
    if (den == 0.0) return false;
    const double num = __dadd_rn(__dadd_rn(__dmul_rn(e0, P[3 * t0]), __dmul_rn(e1, P[3 * t1])), __dmul_rn(e2, P[3 * t2]));
    xc = __ddiv_rn(num, den);
    return true;
}

// parity of the crossings of band column col beyond x
__device__ __forceinline__ bool mesh_inside_column(const GeomParams &G, int col, double x)
{
    const int n = min(G.col_count[col], MESH_COL_CAP);
    const double *xs = G.col_x + (size_t)col * MESH_COL_CAP;
    int k = 0;
    for (int j = 0; j < n; ++j) k += xs[j] > x;
    return k & 1;
}

// triangle hit by a link and the barycentric coordinates of the wall point
// (tri = -1 for the no-hit fallback)
struct MeshHit {
    int tri;
    double u, v;
};

__device__ __forceinline__ double det3(const double a[3], const double b[3], const double d[3])
{
    return a[0] * (b[1] * d[2] - b[2] * d[1]) - a[1] * (b[0] * d[2] - b[2] * d[0]) + a[2] * (b[0] * d[1] - b[1] * d[0]);
}

// Single-precision forms of the link search, used when the populations are
// stored in FP32 or 16 bits (their collision runs in FP32): coordinates are
// taken relative to the node in double and then rounded, so the link
// fraction keeps about 1e-7 absolute accuracy.  The solid marks themselves
// stay the double decisions above.
__device__ __forceinline__ float det3f(const float a[3], const float b[3], const float d[3])
{
    return a[0] * (b[1] * d[2] - b[2] * d[1]) - a[1] * (b[0] * d[2] - b[2] * d[0]) + a[2] * (b[0] * d[1] - b[1] * d[0]);
}

// Warp-cooperative form of the mesh link search for a boundary node: the
// missing links (bits of mask) are taken one at a time by the whole warp;
// each lane tests a strided share of the candidate triangles (same tests as
// mesh_link for double, mesh_link_f for float), and a warp arg-min over
// (s, triangle index) picks the first crossing.  Lane i receives q, u_w and
// the hit of link i.  Every lane of the warp must call it.
template <typename R>
__device__ void mesh_links_warp(const GeomParams &G, const DevBody *b, int x, int y, int z, uint32_t mask, int lane,
                                double &q, double uw[3], MeshHit &hitout)
{
    constexpr bool single = sizeof(R) == 4;
    const int p[3] = {x, y, z};
    const double *P = G.mesh_pos;
    uint32_t m = mask;
    while (m) {
        const int i = __ffs(m) - 1;
        m &= m - 1;
        const int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
        int c0[3], c1[3];
        float lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            const int e0 = min(p[a], p[a] - c[a]), e1 = max(p[a], p[a] - c[a]);
            lo[a] = (float)e0;
            hi[a] = (float)e1;
            c0[a] = max(0, (e0 - b->band_lo[a]) / MESH_CELL);
            c1[a] = min(G.cells[a] - 1, (e1 - b->band_lo[a]) / MESH_CELL);
        }
        // candidate values in the search precision (float coordinates relative
        // to the node from the split vertex positions; double as in the oracle)
        R best = R(2), bu = R(0), bv = R(0);
        int bt = -1;
        for (int kz = c0[2]; kz <= c1[2]; ++kz)
            for (int ky = c0[1]; ky <= c1[1]; ++ky)
                for (int kx = c0[0]; kx <= c1[0]; ++kx) {
                    const int cell = kx + G.cells[0] * (ky + G.cells[1] * kz);
                    const int n = min(G.cell_count[cell], MESH_CELL_CAP);
                    const int *list = G.cell_tri + (size_t)cell * MESH_CELL_CAP;
                    for (int j = lane; j < n; j += 32) {
                        const int k = list[j];
                        const float *bx = G.tri_box + 6 * (size_t)k;
                        if (bx[3] < lo[0] || bx[0] > hi[0] || bx[4] < lo[1] || bx[1] > hi[1] || bx[5] < lo[2] ||
                            bx[2] > hi[2])
                            continue;
                        const int t0 = G.mesh_tris[3 * k], t1 = G.mesh_tris[3 * k + 1], t2 = G.mesh_tris[3 * k + 2];
                        R sv, u, v;
                        if (single) {
                            constexpr float EPS = 1e-6f;
                            float A[3], e1[3], e2[3], r[3];
                            for (int a = 0; a < 3; ++a) {
                                const float pa = (float)(G.mesh_ipos[3 * t0 + a] - p[a]) + G.mesh_frac[3 * t0 + a];
                                const float pb = (float)(G.mesh_ipos[3 * t1 + a] - p[a]) + G.mesh_frac[3 * t1 + a];
                                const float pc = (float)(G.mesh_ipos[3 * t2 + a] - p[a]) + G.mesh_frac[3 * t2 + a];
                                A[a] = pa;
                                e1[a] = pb - pa;
                                e2[a] = pc - pa;
                                r[a] = -pa;
                            }
                            const float dc[3] = {(float)c[0], (float)c[1], (float)c[2]};
                            const float D = det3f(e1, e2, dc);
                            if (D == 0.0f) continue;
                            const float iD = 1.0f / D;
                            const float uf = det3f(r, e2, dc) * iD, vf = det3f(e1, r, dc) * iD;
                            const float sf = det3f(e1, e2, r) * iD;
                            if (uf < -EPS || vf < -EPS || uf + vf > 1.0f + EPS || sf < -EPS || sf > 1.0f + EPS) continue;
                            sv = (R)fminf(fmaxf(sf, 0.0f), 1.0f);
                            u = (R)uf;
                            v = (R)vf;
                        } else {
                            double e1[3], e2[3], r[3];
                            for (int a = 0; a < 3; ++a) {
                                e1[a] = P[3 * t1 + a] - P[3 * t0 + a];
                                e2[a] = P[3 * t2 + a] - P[3 * t0 + a];
                                r[a] = (double)p[a] - P[3 * t0 + a];
                            }
                            const double dc[3] = {(double)c[0], (double)c[1], (double)c[2]};
                            const double D = det3(e1, e2, dc);
                            if (D == 0.0) continue;
                            const double ud = det3(r, e2, dc) / D;
                            const double vd = det3(e1, r, dc) / D;
                            const double sd = det3(e1, e2, r) / D;
                            if (ud < 0.0 || vd < 0.0 || ud + vd > 1.0 || sd < 0.0 || sd > 1.0) continue;
                            sv = (R)sd;
                            u = (R)ud;
                            v = (R)vd;
                        }
                        if (sv < best || (sv == best && k < bt)) {
                            best = sv;
                            bt = k;
                            bu = u;
                            bv = v;
                        }
                    }
                }
        // arg-min over the warp, ties to the lower triangle index
        for (int o = 16; o > 0; o >>= 1) {
            const R ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
            const R ou = __shfl_xor_sync(0xffffffffu, bu, o);
            const R ov = __shfl_xor_sync(0xffffffffu, bv, o);
            if (ot >= 0 && (bt < 0 || ob < best || (ob == best && ot < bt))) {
                best = ob;
                bt = ot;
                bu = ou;
                bv = ov;
            }
        }
        if (lane == i) {
            hitout.tri = bt;
            hitout.u = bu;
            hitout.v = bv;
            if (bt < 0) {
                q = 0.5;
                mesh_material_velocity(G, b, (double)x - 0.5 * c[0], (double)y - 0.5 * c[1], uw);
            } else {
                q = best;
                const int t0 = G.mesh_tris[3 * bt], t1 = G.mesh_tris[3 * bt + 1], t2 = G.mesh_tris[3 * bt + 2];
                for (int a = 0; a < 3; ++a)
                    uw[a] = (1.0 - bu - bv) * G.mesh_vel[3 * t0 + a] + bu * G.mesh_vel[3 * t1 + a] +
                            bv * G.mesh_vel[3 * t2 + a];
            }
        }
    }
}

// airfoil link in the chord frame: node position and link direction in
// double, the 24 halvings in float with reciprocal constants
__device__ __forceinline__ bool inside_airfoil_f(const GeomParams &G, float xi, float eta)
{
    if (xi < 0.0f || xi > 1.0f) return false;
    const float p = (float)G.camber_p;
    const float yc = xi < p ? (float)G.camber_k1 * (2.0f * p * xi - xi * xi)
                            : (float)G.camber_k2 * ((1.0f - 2.0f * p) + 2.0f * p * xi - xi * xi);
    const float t = (float)G.thick[0] * sqrtf(xi) +
                    xi * ((float)G.thick[1] + xi * ((float)G.thick[2] + xi * ((float)G.thick[3] + xi * (float)G.thick[4])));
    return fabsf(eta - yc) < t;
}

__device__ __forceinline__ double link_airfoil_f(const GeomParams &G, const DevBody *b, int x, int y, int cx, int cy)
{
    const double dx = (double)x - b->X[0], dy = (double)y - b->X[1];
    const float xi0 = (float)((dx * G.ca - dy * G.sa) * G.inv_chord);
    const float eta0 = (float)((dx * G.sa + dy * G.ca) * G.inv_chord);
    const float dxi = (float)(-(cx * G.ca - cy * G.sa) * G.inv_chord);
    const float deta = (float)(-(cx * G.sa + cy * G.ca) * G.inv_chord);
    float lo = 0.0f, hi = 1.0f;
    for (int it = 0; it < 24; ++it) {
        const float mid = 0.5f * (lo + hi);
        if (inside_airfoil_f(G, xi0 + mid * dxi, eta0 + mid * deta)) hi = mid;
        else lo = mid;
    }
    return 0.5 * ((double)lo + (double)hi);
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
// and the wall velocity there.  R is the collision arithmetic: double keeps
// the plain double evaluation; float uses the single-precision bisection for
// the airfoil.  Mesh links are found for a whole node at once by
// mesh_links_warp.
template <typename R>
__device__ __forceinline__ void link_data(const Lattice &L, const GeomParams &G, const DevBody *b,
                                          int x, int y, int z, int cx, int cy, int cz, double &q,
                                          double uw[3])
{
    constexpr bool single = sizeof(R) == 4;
    if (G.kind == LBM_BODY_AIRFOIL && single) {
        q = link_airfoil_f(G, b, x, y, cx, cy);
        uw[0] = b->U[0];
        uw[1] = b->U[1];
        uw[2] = b->U[2];
    } else if (G.kind == LBM_BODY_SPHERE) {
        const double d0 = axis_offset(x, b->X[0], L.nx, G.periodic[0]);
        const double d1 = axis_offset(y, b->X[1], L.ny, G.periodic[1]);
        const double d2 = frame_offset(2, z, b->X[2], L.nz, G.periodic[2], G.zoff, G.zper);
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

// ---------------------------------------------------------------- swimmer tangents
// Derivatives with respect to theta = (wave_amp, wave_length, wave_period) of
// the midline y(s,t) = r(t) a env(s) sin(phi), env = L (s/L + 0.03125)/1.03125,
// phi = 2 pi (s/lambda - t/T), r the optional ramp (1 - cos(pi t/T))/2 on
// [0, T):
//   dy/da = r env sin(phi),  dy/dlambda = -r a env cos(phi) 2 pi s/lambda^2,
//   dy/dT = r a env cos(phi) 2 pi t/T^2 + (dr/dT) a env sin(phi),
//   dr/dT = -(1/2) sin(pi t/T) pi t/T^2.
__device__ __forceinline__ void swimmer_midline_tangent(const GeomParams &G, double s, double t, double d[3])
{
    const double T = G.wave_period, lam = G.wave_length, a = G.wave_amp;
    double r = 1.0, drT = 0.0;
    if (G.wave_ramp) {
        if (t < 0.0) r = 0.0;
        else if (t < T) {
            r = 0.5 * (1.0 - cos(MESH_PI * t / T));
            drT = -0.5 * sin(MESH_PI * t / T) * MESH_PI * t / (T * T);
        }
    }
    const double env = G.length * (s / G.length + 0.03125) / 1.03125;
    const double ph = 2.0 * MESH_PI * (s / lam - t / T);
    const double sn = sin(ph), cs = cos(ph);
    d[0] = r * env * sn;
    d[1] = -r * a * env * cs * 2.0 * MESH_PI * s / (lam * lam);
    d[2] = r * a * env * cs * 2.0 * MESH_PI * t / (T * T) + drT * a * env * sn;
}

// theta-tangent of the material velocity (only its y component moves):
// the central difference (dy(s,t+1) - dy(s,t-1))/2
__device__ __forceinline__ void swimmer_velocity_tangent(const GeomParams &G, double t, double s, double dv[3])
{
    double d1[3], d0[3];
    swimmer_midline_tangent(G, s, t + 1.0, d1);
    swimmer_midline_tangent(G, s, t - 1.0, d0);
    for (int k = 0; k < 3; ++k) dv[k] = 0.5 * (d1[k] - d0[k]);
}

// theta-tangents of a mesh link's fraction q and wall velocity u_w.  The wall
// point H = x_b - q c lies on the plane n.(H - A) = 0 of the hit triangle
// (A, B, C), n = (B - A) x (C - A), so dq = (dn.(H - A) - n.dA)/(n.c); the
// barycentric coordinates follow from dH - dA = du e1 + dv e2 + u de1 + v de2
// (normal equations with e1, e2); u_w = (1-u-v) V_A + u V_B + v V_C.  Vertex
// positions move only in y, by the midline tangent at the pose's time
// (per-vertex tangents in G.mesh_dy / G.mesh_dvy).  R is the collision
// arithmetic: the vertices are taken relative to the node in double, the
// rest runs in R (the link search's own precision).
template <typename R>
__device__ __noinline__ static void mesh_link_tangent(const GeomParams &G, const DevBody *b, int x, int y, int z, int cx, int cy, int cz,
                                  double q, const MeshHit &h, double dq[3], double duw[3][3])
{
    if (h.tri < 0) {
        double dv[3];
        swimmer_velocity_tangent(G, b->t, clamp_arc(G, (double)x - 0.5 * cx - b->X[0]), dv);
        for (int k = 0; k < 3; ++k) {
            dq[k] = 0.0;
            duw[k][0] = 0.0;
            duw[k][1] = dv[k];
            duw[k][2] = 0.0;
        }
        return;
    }
    const int tv[3] = {G.mesh_tris[3 * h.tri], G.mesh_tris[3 * h.tri + 1], G.mesh_tris[3 * h.tri + 2]};
    const double xb[3] = {(double)x, (double)y, (double)z};
    R P[3][3], V[3][3], dy[3], dvy[3][3];
    for (int m = 0; m < 3; ++m)
        for (int a = 0; a < 3; ++a) {
            P[m][a] = (R)(G.mesh_pos[3 * tv[m] + a] - xb[a]);
            V[m][a] = (R)G.mesh_vel[3 * tv[m] + a];
        }
    const R c[3] = {R(cx), R(cy), R(cz)};
    R e1[3], e2[3], H[3], n[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = P[1][a] - P[0][a];
        e2[a] = P[2][a] - P[0][a];
        H[a] = -(R)q * c[a] - P[0][a];
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const R nc = n[0] * c[0] + n[1] * c[1] + n[2] * c[2];
    const R g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    const R g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    const R g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    const R gdet = g11 * g22 - g12 * g12;
    const R hu = (R)h.u, hv = (R)h.v, hw = R(1) - hu - hv;
    for (int k = 0; k < 3; ++k) {
        for (int m = 0; m < 3; ++m) {
            dy[m] = (R)G.mesh_dy[3 * tv[m] + k];
            dvy[m][k] = (R)G.mesh_dvy[3 * tv[m] + k];
        }
        // vertex displacements along y only: de1 = (0, dB - dA, 0), de2 = (0, dC - dA, 0)
        const R dA = dy[0], d1 = dy[1] - dA, d2 = dy[2] - dA;
        // dn = de1 x e2 + e1 x de2 (its y component vanishes)
        R dn[3];
        dn[0] = d1 * e2[2] - e1[2] * d2;
        dn[1] = R(0);
        dn[2] = e1[0] * d2 - d1 * e2[0];
        const R ds = nc != R(0) ? ((dn[0] * H[0] + dn[1] * H[1] + dn[2] * H[2]) - n[1] * dA) / nc : R(0);
        R rhs[3];
        rhs[0] = -ds * c[0];
        rhs[1] = -ds * c[1] - hu * d1 - hv * d2 - dA;
        rhs[2] = -ds * c[2];
        const R b1 = e1[0] * rhs[0] + e1[1] * rhs[1] + e1[2] * rhs[2];
        const R b2 = e2[0] * rhs[0] + e2[1] * rhs[1] + e2[2] * rhs[2];
        const R du = gdet != R(0) ? (b1 * g22 - b2 * g12) / gdet : R(0);
        const R dv = gdet != R(0) ? (g11 * b2 - g12 * b1) / gdet : R(0);
        dq[k] = (double)ds;
        for (int a = 0; a < 3; ++a) duw[k][a] = (double)(du * (V[1][a] - V[0][a]) + dv * (V[2][a] - V[0][a]));
        duw[k][1] += (double)(hw * dvy[0][k] + hu * dvy[1][k] + hv * dvy[2][k]);
    }
}

// d y(s,t) / ds of the midline (Sec. 4.3): r(t) [a/1.03125 sin(ph) + A(s) cos(ph) 2 pi/lambda],
// A(s) = a L (s/L + 0.03125)/1.03125, ph = 2 pi (s/lambda - t/T)
__device__ __forceinline__ double swimmer_midline_ds(const GeomParams &G, double s, double t)
{
    double r = 1.0;
    if (G.wave_ramp) {
        if (t < 0.0) r = 0.0;
        else if (t < G.wave_period) r = 0.5 * (1.0 - cos(MESH_PI * t / G.wave_period));
    }
    const double A = G.wave_amp * G.length * (s / G.length + 0.03125) / 1.03125;
    const double ph = 2.0 * MESH_PI * (s / G.wave_length - t / G.wave_period);
    return r * (G.wave_amp / 1.03125 * sin(ph) + A * cos(ph) * 2.0 * MESH_PI / G.wave_length);
}

// d/dX0 of the material velocity's y component at the node's arc position
// s = x - X0 (the central difference of the midline): -d rate / ds, zero where
// s is clamped to the ends
__device__ __forceinline__ double swimmer_rate_dX(const GeomParams &G, double t, double s_raw)
{
    if (s_raw < 0.0 || s_raw > G.length) return 0.0;
    return -0.5 * (swimmer_midline_ds(G, s_raw, t + 1.0) - swimmer_midline_ds(G, s_raw, t - 1.0));
}

// Derivatives of a mesh link's fraction q and wall velocity u_w with respect
// to the head's position X0 along x (the swimmer free along x, head frame):
// every vertex moves by e_x, so with the plane and barycentric relations of
// mesh_link_tangent dq = -n_x/(n.c) and du e1 + dv e2 = -dq c - e_x; the
// vertex velocities (U plus the midline's rate at the material position) do
// not change.  d/dU0 is q: 0, u_w: e_x.
__device__ __noinline__ static void mesh_link_body_tangent(const GeomParams &G, const DevBody *b, int x, int y, int z,
                                                           int cx, int cy, int cz, double q, const MeshHit &h,
                                                           double &dq, double duw[3])
{
    if (h.tri < 0) {
        dq = 0.0;
        duw[0] = 0.0;
        duw[1] = swimmer_rate_dX(G, b->t, (double)x - 0.5 * cx - b->X[0]);
        duw[2] = 0.0;
        return;
    }
    const int tv[3] = {G.mesh_tris[3 * h.tri], G.mesh_tris[3 * h.tri + 1], G.mesh_tris[3 * h.tri + 2]};
    double P[3][3], V[3][3];
    for (int m = 0; m < 3; ++m)
        for (int a = 0; a < 3; ++a) {
            P[m][a] = G.mesh_pos[3 * tv[m] + a];
            V[m][a] = G.mesh_vel[3 * tv[m] + a];
        }
    const double c[3] = {(double)cx, (double)cy, (double)cz};
    double e1[3], e2[3], n[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = P[1][a] - P[0][a];
        e2[a] = P[2][a] - P[0][a];
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double nc = n[0] * c[0] + n[1] * c[1] + n[2] * c[2];
    const double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    const double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    const double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    const double gdet = g11 * g22 - g12 * g12;
    dq = nc != 0.0 ? -n[0] / nc : 0.0;
    double rhs[3];
    for (int a = 0; a < 3; ++a) rhs[a] = -dq * c[a];
    rhs[0] -= 1.0;
    const double b1 = e1[0] * rhs[0] + e1[1] * rhs[1] + e1[2] * rhs[2];
    const double b2 = e2[0] * rhs[0] + e2[1] * rhs[1] + e2[2] * rhs[2];
    const double du = gdet != 0.0 ? (b1 * g22 - b2 * g12) / gdet : 0.0;
    const double dv = gdet != 0.0 ? (g11 * b2 - g12 * b1) / gdet : 0.0;
    for (int a = 0; a < 3; ++a) duw[a] = du * (V[1][a] - V[0][a]) + dv * (V[2][a] - V[0][a]);
}

// ---------------------------------------------------------------- centre-of-mass frame tangents
// The swimmer free in y or yaw (centre-of-mass frame): derivatives of the
// pose at body time tau with respect to nine directions, the kinematic
// parameters theta_0..2 and the body state X_x, X_y, psi, U_x, U_y, omega:
//   vertex  p = X + R(psi) (b(tau) - c(tau)),
//   velocity  v = U + omega e_z x (p - X) + R(psi) (b_dot - c_dot).
// dc, dcdot and dI are the theta-derivatives of the centre of mass c(tau), of
// its central-difference rate and of the moment of inertia I(tau).
constexpr int COM_DIRS = 9;

struct ComTangents {
    double dc[3][2];
    double dcdot[3][2];
    double dI[3];
};

// per-vertex derivatives of position and velocity for the nine directions
__device__ __forceinline__ void com_vertex_tangents(const GeomParams &G, const DevBody *b, const ComTangents &ct,
                                                    int v, double dP[COM_DIRS][3], double dV[COM_DIRS][3])
{
    const double cs = cos(b->psi), sn = sin(b->psi), w = b->omega;
    const double P[3] = {G.mesh_pos[3 * v], G.mesh_pos[3 * v + 1], G.mesh_pos[3 * v + 2]};
    const double Vv[3] = {G.mesh_vel[3 * v], G.mesh_vel[3 * v + 1], G.mesh_vel[3 * v + 2]};
    const double rx = P[0] - b->X[0], ry = P[1] - b->X[1];
    for (int d = 0; d < COM_DIRS; ++d)
        for (int a = 0; a < 3; ++a) dP[d][a] = dV[d][a] = 0.0;
    for (int k = 0; k < 3; ++k) {
        // body-frame displacement (-dc_x, dy_theta - dc_y), rotated
        const double bx = -ct.dc[k][0], by = G.mesh_dy[3 * v + k] - ct.dc[k][1];
        dP[k][0] = cs * bx - sn * by;
        dP[k][1] = sn * bx + cs * by;
        const double wx = -ct.dcdot[k][0], wy = G.mesh_dvy[3 * v + k] - ct.dcdot[k][1];
        dV[k][0] = -w * dP[k][1] + (cs * wx - sn * wy);
        dV[k][1] = w * dP[k][0] + (sn * wx + cs * wy);
    }
    dP[3][0] = 1.0;
    dP[4][1] = 1.0;
    // rotation about X: dp = e_z x r, dv = omega e_z x dp + e_z x (R w)
    dP[5][0] = -ry;
    dP[5][1] = rx;
    const double Rw[2] = {Vv[0] - b->U[0] + w * ry, Vv[1] - b->U[1] - w * rx};
    dV[5][0] = -w * dP[5][1] - Rw[1];
    dV[5][1] = w * dP[5][0] + Rw[0];
    dV[6][0] = 1.0;
    dV[7][1] = 1.0;
    dV[8][0] = -ry;
    dV[8][1] = rx;
}

// derivatives of the material velocity at the fixed world point (px, py)
// (mesh_material_velocity in the centre-of-mass frame): its arc position
// s = [R^T (p - X)]_x + c_x moves with X, psi and c_x
__device__ __forceinline__ void com_material_velocity_tangents(const GeomParams &G, const DevBody *b,
                                                               const ComTangents &ct, double px, double py,
                                                               double du[COM_DIRS][3])
{
    const double cs = cos(b->psi), sn = sin(b->psi), w = b->omega;
    const double rx = px - b->X[0], ry = py - b->X[1];
    const double s_raw = cs * rx + sn * ry + b->com[0];
    const double s = clamp_arc(G, s_raw);
    // d rate / ds (0 where the arc position is clamped)
    const double rs = -swimmer_rate_dX(G, b->t, s_raw);
    const double rate = (swimmer_midline(G, s, b->t + 1.0) - swimmer_midline(G, s, b->t - 1.0)) / 2.0;
    const double Rw[2] = {cs * (-b->com_dot[0]) - sn * (rate - b->com_dot[1]),
                          sn * (-b->com_dot[0]) + cs * (rate - b->com_dot[1])};
    double dvt[3];
    swimmer_velocity_tangent(G, b->t, s, dvt);
    for (int d = 0; d < COM_DIRS; ++d) du[d][0] = du[d][1] = du[d][2] = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double wx = -ct.dcdot[k][0], wy = dvt[k] + rs * ct.dc[k][0] - ct.dcdot[k][1];
        du[k][0] = cs * wx - sn * wy;
        du[k][1] = sn * wx + cs * wy;
    }
    // X: r moves by -e_a, s by -(cs, sn)_a
    du[3][0] = -sn * (-cs * rs);
    du[3][1] = -w + cs * (-cs * rs);
    du[4][0] = w - sn * (-sn * rs);
    du[4][1] = cs * (-sn * rs);
    // psi: e_z x (R w) + R (0, rate' ds/dpsi)
    const double dsp = -sn * rx + cs * ry;
    du[5][0] = -Rw[1] - sn * rs * dsp;
    du[5][1] = Rw[0] + cs * rs * dsp;
    du[6][0] = 1.0;
    du[7][1] = 1.0;
    du[8][0] = -ry;
    du[8][1] = rx;
}

// derivatives of a link's fraction q and wall velocity u_w for the nine
// directions (plane and barycentric relations of mesh_link_tangent with
// general vertex displacements and velocity changes)
__device__ __noinline__ static void com_link_tangents(const GeomParams &G, const DevBody *b, const ComTangents &ct,
                                                      int x, int y, int z, int cx, int cy, int cz, double q,
                                                      const MeshHit &h, double dq[COM_DIRS],
                                                      double duw[COM_DIRS][3])
{
    if (h.tri < 0) {
        com_material_velocity_tangents(G, b, ct, (double)x - 0.5 * cx, (double)y - 0.5 * cy, duw);
        for (int d = 0; d < COM_DIRS; ++d) dq[d] = 0.0;
        return;
    }
    const int tv[3] = {G.mesh_tris[3 * h.tri], G.mesh_tris[3 * h.tri + 1], G.mesh_tris[3 * h.tri + 2]};
    double P[3][3], V[3][3];
    for (int m = 0; m < 3; ++m)
        for (int a = 0; a < 3; ++a) {
            P[m][a] = G.mesh_pos[3 * tv[m] + a];
            V[m][a] = G.mesh_vel[3 * tv[m] + a];
        }
    const double c[3] = {(double)cx, (double)cy, (double)cz};
    double e1[3], e2[3], H[3], n[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = P[1][a] - P[0][a];
        e2[a] = P[2][a] - P[0][a];
    }
    H[0] = (double)x - q * c[0] - P[0][0];
    H[1] = (double)y - q * c[1] - P[0][1];
    H[2] = (double)z - q * c[2] - P[0][2];
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double nc = n[0] * c[0] + n[1] * c[1] + n[2] * c[2];
    const double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    const double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    const double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    const double gdet = g11 * g22 - g12 * g12;
    double dP[3][COM_DIRS][3], dV[3][COM_DIRS][3];
    for (int m = 0; m < 3; ++m) com_vertex_tangents(G, b, ct, tv[m], dP[m], dV[m]);
    for (int d = 0; d < COM_DIRS; ++d) {
        double de1[3], de2[3], dn[3];
        for (int a = 0; a < 3; ++a) {
            de1[a] = dP[1][d][a] - dP[0][d][a];
            de2[a] = dP[2][d][a] - dP[0][d][a];
        }
        dn[0] = de1[1] * e2[2] - de1[2] * e2[1] + e1[1] * de2[2] - e1[2] * de2[1];
        dn[1] = de1[2] * e2[0] - de1[0] * e2[2] + e1[2] * de2[0] - e1[0] * de2[2];
        dn[2] = de1[0] * e2[1] - de1[1] * e2[0] + e1[0] * de2[1] - e1[1] * de2[0];
        const double ds = nc != 0.0 ? ((dn[0] * H[0] + dn[1] * H[1] + dn[2] * H[2]) -
                                       (n[0] * dP[0][d][0] + n[1] * dP[0][d][1] + n[2] * dP[0][d][2])) / nc
                                    : 0.0;
        double rhs[3];
        for (int a = 0; a < 3; ++a) rhs[a] = -ds * c[a] - dP[0][d][a] - h.u * de1[a] - h.v * de2[a];
        const double b1 = e1[0] * rhs[0] + e1[1] * rhs[1] + e1[2] * rhs[2];
        const double b2 = e2[0] * rhs[0] + e2[1] * rhs[1] + e2[2] * rhs[2];
        const double du = gdet != 0.0 ? (b1 * g22 - b2 * g12) / gdet : 0.0;
        const double dv = gdet != 0.0 ? (g11 * b2 - g12 * b1) / gdet : 0.0;
        dq[d] = ds;
        for (int a = 0; a < 3; ++a)
            duw[d][a] = du * (V[1][a] - V[0][a]) + dv * (V[2][a] - V[0][a]) + (1.0 - h.u - h.v) * dV[0][d][a] +
                        h.u * dV[1][d][a] + h.v * dV[2][d][a];
    }
}

// ---------------------------------------------------------------- airfoil tangents
// Derivatives with respect to theta = (h_amp, h_omega) of the plunge at body
// time t (Sec. 4.2): X1 = y_base + A sin(w t), U1 = A w cos(w t).
__device__ __forceinline__ void airfoil_plunge_tangent(const GeomParams &G, double t, double dX1[2], double dU1[2])
{
    const double A = G.h_amp, w = G.h_omega, sn = sin(w * t), cs = cos(w * t);
    dX1[0] = sn;
    dX1[1] = A * t * cs;
    dU1[0] = w * cs;
    dU1[1] = A * cs - A * w * t * sn;
}

// dq/dtheta of an airfoil link.  The wall point H = x_b - q c stays on the
// plunging surface phi(H - X) = 0, phi = |eta - y_c(xi)| - t(xi) in the chord
// frame, so dq = -(grad phi . dX)/(grad phi . c) with dX = (0, dX1, 0).
__device__ __forceinline__ void airfoil_link_tangent(const GeomParams &G, const DevBody *b, int x, int y, int cx,
                                                     int cy, double q, double dq[2])
{
    const double dx = (double)x - q * cx - b->X[0], dy = (double)y - q * cy - b->X[1];
    const double xi = (dx * G.ca - dy * G.sa) * G.inv_chord, eta = (dx * G.sa + dy * G.ca) * G.inv_chord;
    const double p = G.camber_p, xc = fmin(fmax(xi, 1e-12), 1.0);
    const double yc = xc < p ? G.camber_k1 * (2.0 * p * xc - xc * xc)
                             : G.camber_k2 * ((1.0 - 2.0 * p) + 2.0 * p * xc - xc * xc);
    const double ycp = (xc < p ? G.camber_k1 : G.camber_k2) * (2.0 * p - 2.0 * xc);
    const double *a = G.thick;
    const double tp = 0.5 * a[0] / sqrt(xc) + a[1] + xc * (2.0 * a[2] + xc * (3.0 * a[3] + xc * 4.0 * a[4]));
    const double sg = eta - yc >= 0.0 ? 1.0 : -1.0;
    const double dxi = -sg * ycp - tp, deta = sg;
    const double gx = (dxi * G.ca + deta * G.sa) * G.inv_chord, gy = (-dxi * G.sa + deta * G.ca) * G.inv_chord;
    const double gc = gx * cx + gy * cy;
    double dX1[2], dU1[2];
    airfoil_plunge_tangent(G, b->t, dX1, dU1);
    for (int k = 0; k < 2; ++k) dq[k] = gc != 0.0 ? -gy * dX1[k] / gc : 0.0;
}

// torque arm origin: displacement of (x, y, z) from the body reference point
// (sphere centre; airfoil leading edge at z = 0; swimmer head on the centre
// line; the lattice origin otherwise)
__device__ __forceinline__ double body_offset(const Lattice &L, const GeomParams &G, const DevBody *b,
                                              int a, int p)
{
    // (the mesh: a slab's z in the slab's frame, where its pose is placed;
    // the other bodies: a slab's z is that of the whole box)
    if (G.kind == LBM_BODY_MESH) return __dsub_rn((double)p, a == 2 ? slab_z(G, b->X[2], L.nz) : b->X[a]);
    const int pz = a == 2 && G.zper > 0 ? p + G.zoff : p;
    if (G.kind == LBM_BODY_AIRFOIL) return a < 2 ? __dsub_rn((double)p, b->X[a]) : (double)pz;
    if (G.kind != LBM_BODY_SPHERE) return (double)pz;
    const int n = a == 0 ? L.nx : (a == 1 ? L.ny : L.nz);
    return frame_offset(a, p, b->X[a], n, G.periodic[a], G.zoff, G.zper);
}

}  // namespace lbm
