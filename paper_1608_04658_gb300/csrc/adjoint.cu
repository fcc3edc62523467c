// Reverse-mode adjoint of the time step and the checkpointed driver behind
// lbm_adjoint_step (arXiv 1608.04658: Sec. 2 collision and pull streaming,
// Sec. 3 Grad boundary and refill, Sec. 4.1 momentum exchange, Sec. 4.3
// swimmer kinematics).
//
// Forward step t -> t+1: S^t is the stored post-collision state, the refill
// R_t overwrites the nodes uncovered at t+1 (St^t = R_t(S^t)), every node x
// fluid at t+1 pulls F_i(x) from St^t (boundary nodes complete the missing
// F_i with Grad's distribution) and stores S^{t+1}(x) = C(F(x)); the
// momentum exchange gives the force F^t of the step.
//
// The adjoint of S^{t+1} is never stored as a full array.  Each node x fluid
// at t+1 stores
//     Lam^t(x)_i = dJ/dF_i(x)      (0 for missing directions, 0 at solid nodes)
// and the adjoint of St^t at node y is the transpose of the pull plus what the
// boundary and refill adjoints add at nearby nodes (band buffer ext^t):
//     lambda(St^t)(y)_i = sum over the nodes x that pulled St^t(y)_i of
//                         Lam^t(x)_i  +  ext^t(y)_i,
// the pull transpose covering the periodic wrap, wall bounce-back and the
// outflow clamp.  lambda(S^t)(y) = 0 where y is refilled in step t, else
// lambda(St^t)(y).  The marks, boundary links and refilled nodes of each step
// are those of the forward run (held fixed).
#include <vector>
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstring>

#include "ctx.cuh"
#include "lanes.cuh"
#include "pull.cuh"

namespace lbm {

// ----------------------------------------------------------------- collision VJP
// 1-D equilibrium factors of one axis for the adjoint: phi(c) = 1 + e(c), its
// reciprocal r(c), e(c) (shifted form, see axis_eq) and the logarithmic
// derivatives dl(c) = d ln phi(c) / du = D0 + c dlnB with
//   D0 = -(3u/S)/(2 - S),   dlnB = (2 + 3u/S)/(2u + S) + 1/(1 - u).
// (reciprocals and square roots by rcp_fast / sqrt_fast: the hardware
// approximations in FP32, exact in FP64)
template <typename R>
__device__ __forceinline__ void axis_eq_adj(R u, R e[3], R phi[3], R r[3], R dl[3])
{
    const R u2 = u * u;
    const R S = sqrt_fast(R(1) + R(3) * u2);
    const R iS = rcp_fast(S);
    const R sig = R(3) * u2 * rcp_fast(S + R(1));
    const R oms = R(1) - sig;
    const R i1u = rcp_fast(R(1) - u);
    const R bp = (R(3) * u + sig) * i1u;
    const R i1bp = rcp_fast(R(1) + bp);
    const R bm = -bp * i1bp;
    e[0] = bm * oms - sig;
    e[1] = -sig;
    e[2] = bp * oms - sig;
    phi[0] = oms * (R(1) + bm);
    phi[1] = oms;
    phi[2] = oms * (R(1) + bp);
    const R ioms = rcp_fast(oms);
    r[0] = ioms * (R(1) + bp);
    r[1] = ioms;
    r[2] = ioms * i1bp;
    const R sp = R(3) * u * iS;
    const R D0 = -sp * ioms;
    const R dlnB = (R(2) + sp) * i1u * i1bp + i1u;
    dl[0] = D0 - dlnB;
    dl[1] = D0;
    dl[2] = D0 + dlnB;
}

// Transpose of the KBC collision f' = f - b (2 ds + g dh) (Eq. kbc_relax with
// the analytic stabilizer), per node: lam holds dJ/df' on entry and dJ/df on
// exit; g are the shifted pre-collision populations.  Backward sweep:
//   ds_bar = -2b lam + a_bar dh/feq,  dh_bar = -b g lam + a_bar ds/feq + 2 b_bar dh/feq,
//   g_bar = -b <lam, dh>,  a = <ds|dh>, b = <dh|dh>, g = 1/b - (2 - 1/b) a/b,
//   df_bar = dh_bar + S^T (ds_bar - dh_bar),   feq_bar = -df_bar - (a_bar ds dh + b_bar dh^2)/feq^2,
//   then f^eq(rho, u) and u = j/rho back to f.
// Operation count as in the forward collision: moments from the x-lines of
// the velocity cube, f^eq and 1/f^eq as products of per-axis factors with the
// x-y pairs formed once, the shear values formed once.
template <typename R>
__device__ void kbc_vjp(const R g[Q], R lam[Q], R beta, R inv_beta, R rho0, int gamma_mode)
{
    R Ls[9], Ld[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        Ld[l] = g[18 + l] - g[l];
        Ls[l] = (g[18 + l] + g[l]) + g[9 + l];
    }
    const R drho = ((Ls[0] + Ls[1]) + (Ls[2] + Ls[3])) + ((Ls[4] + Ls[5]) + ((Ls[6] + Ls[7]) + Ls[8]));
    const R jx = ((Ld[0] + Ld[1]) + (Ld[2] + Ld[3])) + ((Ld[4] + Ld[5]) + ((Ld[6] + Ld[7]) + Ld[8]));
    const R jy = ((Ls[6] + Ls[7]) + Ls[8]) - ((Ls[0] + Ls[1]) + Ls[2]);
    const R jz = ((Ls[2] + Ls[5]) + Ls[8]) - ((Ls[0] + Ls[3]) + Ls[6]);
    const R rho = rho0 + drho, irho = rcp_fast(rho);
    const R u[3] = {jx * irho, jy * irho, jz * irho};
    R ex[3], ey[3], ez[3], px[3], py[3], pz[3], rx[3], ry[3], rz[3], dl[3][3];
    axis_eq_adj(u[0], ex, px, rx, dl[0]);
    axis_eq_adj(u[1], ey, py, ry, dl[1]);
    axis_eq_adj(u[2], ez, pz, rz, dl[2]);
    // f^eq_i = Fxy[cx][cy] Fz[cz], 1/f^eq_i = Rxy[cx][cy] Rz[cz] (1-D weights
    // w(0) = 2/3, w(+-1) = 1/6 and rho folded in)
    R Fxy[3][3], Rxy[3][3], Fz[3], Rz[3], exy[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const R w = a == 1 ? R(2.0 / 3.0) : R(1.0 / 6.0), iw = a == 1 ? R(1.5) : R(6);
        Fz[a] = w * pz[a];
        Rz[a] = iw * rz[a];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const R wb = b == 1 ? R(2.0 / 3.0) : R(1.0 / 6.0), iwb = b == 1 ? R(1.5) : R(6);
            Fxy[a][b] = rho * (w * px[a]) * (wb * py[b]);
            Rxy[a][b] = irho * (iw * rx[a]) * (iwb * ry[b]);
            exy[a][b] = ey[b] * px[a] + ex[a];
        }
    }
    R rw[4], dw[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const R w = k == 0 ? R(8) / R(27) : k == 1 ? R(2) / R(27) : k == 2 ? R(1) / R(54) : R(1) / R(216);
        rw[k] = rho * w;
        dw[k] = drho * w;
    }
    R d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const R E = exy[cx + 1][cy + 1] * pz[cz + 1] + ez[cz + 1];
        d[i] = g[i] - (rw[nz] * E + dw[nz]);
    }
    R A[9], B[9], T[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        A[l] = d[18 + l] + d[l];
        B[l] = d[18 + l] - d[l];
        T[l] = A[l] + d[9 + l];
    }
    const R pxx = ((A[0] + A[1]) + (A[2] + A[3])) + ((A[4] + A[5]) + ((A[6] + A[7]) + A[8]));
    const R pxy = ((B[6] + B[7]) + B[8]) - ((B[0] + B[1]) + B[2]);
    const R pxz = ((B[2] + B[5]) + B[8]) - ((B[0] + B[3]) + B[6]);
    const R pyy = ((T[0] + T[1]) + T[2]) + ((T[6] + T[7]) + T[8]);
    const R pzz = ((T[0] + T[3]) + T[6]) + ((T[2] + T[5]) + T[8]);
    const R pyz = (T[0] + T[8]) - (T[2] + T[6]);
    const R nxz = pxx - pzz, nyz = pyy - pzz;
    const R sx = (R(2) * nxz - nyz) * R(1.0 / 6.0);
    const R sy = (R(2) * nyz - nxz) * R(1.0 / 6.0);
    const R sz = -(nxz + nyz) * R(1.0 / 6.0);
    const R qxy = R(0.25) * pxy, qxz = R(0.25) * pxz, qyz = R(0.25) * pyz;
    R sh = 0, hh = 0, lh = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const R ifeq = Rxy[cx + 1][cy + 1] * Rz[cz + 1];
        if (nz == 1 || nz == 2) {
            const R ds = shear_part<R>(i, sx, sy, sz, qxy, qxz, qyz);
            const R dh = d[i] - ds;
            const R t = dh * ifeq;
            sh += ds * t;
            hh += dh * t;
            lh += lam[i] * dh;
        } else {
            hh += d[i] * (d[i] * ifeq);
            lh += lam[i] * d[i];
        }
    }
    const bool analytic = gamma_mode == LBM_GAMMA_ANALYTIC && hh > gamma_floor<R>();
    const R ihh = analytic ? rcp_fast(hh) : R(0);
    const R gam = analytic ? inv_beta - (R(2) - inv_beta) * sh * ihh : R(2);
    const R gb = -beta * lh;
    const R kk = R(2) - inv_beta;
    const R ab = -kk * gb * ihh;
    // (kk gb)(sh/hh)/hh: the square hh^2 would underflow in FP32 near rest
    const R bb = kk * gb * (sh * ihh) * ihh;
    const R cl_s = -R(2) * beta, cl_h = -beta * gam, bb2 = R(2) * bb;
    // shear sums of ds_bar - dh_bar (faces and edges carry ds)
    R Sx = 0, Sy = 0, Sz = 0, Qxy = 0, Qxz = 0, Qyz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        if (nz != 1 && nz != 2) continue;
        const R ifeq = Rxy[cx + 1][cy + 1] * Rz[cz + 1];
        const R ds = shear_part<R>(i, sx, sy, sz, qxy, qxz, qyz);
        const R dh = d[i] - ds;
        // (ds_bar - dh_bar) = (cl_s - cl_h) lam + (ab (dh - ds) - 2 bb dh) / feq
        const R t = (cl_s - cl_h) * lam[i] + (ab * (dh - ds) - bb2 * dh) * ifeq;
        if (nz == 1) {
            if (cx) Sx += t;
            else if (cy) Sy += t;
            else Sz += t;
        } else {
            if (cz == 0) Qxy += R(cx * cy) * t;
            else if (cy == 0) Qxz += R(cx * cz) * t;
            else Qyz += R(cy * cz) * t;
        }
    }
    const R nxzb = (R(2) * Sx - Sy - Sz) * R(1.0 / 6.0);
    const R nyzb = (R(2) * Sy - Sx - Sz) * R(1.0 / 6.0);
    const R pzzb = -(nxzb + nyzb);
    const R pxyb = R(0.25) * Qxy, pxzb = R(0.25) * Qxz, pyzb = R(0.25) * Qyz;
    R rhob = 0, ub0 = 0, ub1 = 0, ub2 = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const R ifeq = Rxy[cx + 1][cy + 1] * Rz[cz + 1];
        const R feq = Fxy[cx + 1][cy + 1] * Fz[cz + 1];
        // rest and corners carry no shear part (ds = 0, dh = d)
        const bool sh_i = nz == 1 || nz == 2;
        const R ds = sh_i ? shear_part<R>(i, sx, sy, sz, qxy, qxz, qyz) : R(0);
        const R dh = sh_i ? d[i] - ds : d[i];
        const R dhb = cl_h * lam[i] + (sh_i ? ab * ds + bb2 * dh : bb2 * dh) * ifeq;
        // S^T of the shear sums: only the terms with nonzero c_a c_b (known
        // per direction at compile time; a product with 0 would still cost an
        // instruction)
        R dfb = dhb;
        if (cx) dfb += nxzb;
        if (cy) dfb += nyzb;
        if (cz) dfb += pzzb;
        if (cx && cy) dfb = cx * cy > 0 ? dfb + pxyb : dfb - pxyb;
        if (cx && cz) dfb = cx * cz > 0 ? dfb + pxzb : dfb - pxzb;
        if (cy && cz) dfb = cy * cz > 0 ? dfb + pyzb : dfb - pyzb;
        // feq_bar * feq
        const R t = -(sh_i ? ab * ds + bb * dh : bb * dh) * dh * ifeq - dfb * feq;
        rhob += t;
        ub0 += t * dl[0][cx + 1];
        ub1 += t * dl[1][cy + 1];
        ub2 += t * dl[2][cz + 1];
        lam[i] += dfb;
    }
    rhob *= irho;
    const R jb[3] = {ub0 * irho, ub1 * irho, ub2 * irho};
    rhob -= (ub0 * u[0] + ub1 * u[1] + ub2 * u[2]) * irho;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        R v = rhob;
        if (cx_of(i)) v = cx_of(i) > 0 ? v + jb[0] : v - jb[0];
        if (cy_of(i)) v = cy_of(i) > 0 ? v + jb[1] : v - jb[1];
        if (cz_of(i)) v = cz_of(i) > 0 ? v + jb[2] : v - jb[2];
        lam[i] += v;
    }
}

// The same transpose with lane i < 27 holding g_i and lam_i (boundary nodes);
// returns dJ/dg_i.
template <typename R>
__device__ R kbc_vjp_lanes(R g, R lam, int i, R beta, R inv_beta, R rho0, int gamma_mode)
{
    const bool act = i < Q;
    const int cx = act ? cx_of(i) : 0, cy = act ? cy_of(i) : 0, cz = act ? cz_of(i) : 0;
    const int nz = act ? nonzero_of(i) : 0;
    const R gv = act ? g : R(0), lv = act ? lam : R(0);
    const R drho = wsum(gv);
    const R jx = wsum(R(cx) * gv), jy = wsum(R(cy) * gv), jz = wsum(R(cz) * gv);
    const R rho = rho0 + drho, irho = R(1) / rho;
    const R u[3] = {jx * irho, jy * irho, jz * irho};
    R e[3][3], phi[3][3], rr[3][3], dl[3][3];
    for (int a = 0; a < 3; ++a) axis_eq_adj(u[a], e[a], phi[a], rr[a], dl[a]);
    const R exy = pick(e[0], cx) + pick(e[1], cy) + pick(e[0], cx) * pick(e[1], cy);
    const R E = exy + pick(e[2], cz) + exy * pick(e[2], cz);
    const R d = act ? gv - weight<R>(i) * (drho + rho * E) : R(0);
    const R pxx = wsum(R(cx * cx) * d), pyy = wsum(R(cy * cy) * d), pzz = wsum(R(cz * cz) * d);
    const R pxy = wsum(R(cx * cy) * d), pxz = wsum(R(cx * cz) * d), pyz = wsum(R(cy * cz) * d);
    const R nxz = pxx - pzz, nyz = pyy - pzz;
    const R ds = act ? shear_part_raw<R>(i, nxz, nyz, pxy, pxz, pyz) : R(0);
    const R dh = d - ds;
    const R ifeq = act ? irho * inv_weight<R>(i) * pick(rr[0], cx) * pick(rr[1], cy) * pick(rr[2], cz) : R(0);
    const R feq = act ? rho * weight<R>(i) * pick(phi[0], cx) * pick(phi[1], cy) * pick(phi[2], cz) : R(0);
    const R sh = wsum(ds * dh * ifeq), hh = wsum(dh * dh * ifeq), lh = wsum(lv * dh);
    const bool analytic = gamma_mode == LBM_GAMMA_ANALYTIC && hh > gamma_floor<R>();
    const R gam = analytic ? inv_beta - (R(2) - inv_beta) * sh / hh : R(2);
    const R gb = -beta * lh;
    const R kk = R(2) - inv_beta;
    const R ab = analytic ? -kk * gb / hh : R(0);
    // (kk gb)(sh/hh)/hh: the square hh^2 would underflow in FP32 near rest
    const R bb = analytic ? kk * gb * (sh / hh) / hh : R(0);
    const R dsb = -R(2) * beta * lv + ab * dh * ifeq;
    const R dhb = -beta * gam * lv + ab * ds * ifeq + R(2) * bb * dh * ifeq;
    const R t = (nz == 1 || nz == 2) ? dsb - dhb : R(0);
    const R Sx = wsum((nz == 1 && cx) ? t : R(0));
    const R Sy = wsum((nz == 1 && cy) ? t : R(0));
    const R Sz = wsum((nz == 1 && cz) ? t : R(0));
    const R Qxy = wsum((nz == 2 && cz == 0) ? R(cx * cy) * t : R(0));
    const R Qxz = wsum((nz == 2 && cy == 0) ? R(cx * cz) * t : R(0));
    const R Qyz = wsum((nz == 2 && cx == 0) ? R(cy * cz) * t : R(0));
    const R nxzb = (R(2) * Sx - Sy - Sz) * R(1.0 / 6.0);
    const R nyzb = (R(2) * Sy - Sx - Sz) * R(1.0 / 6.0);
    const R dfb = dhb + nxzb * R(cx * cx) + nyzb * R(cy * cy) - (nxzb + nyzb) * R(cz * cz) +
                  R(0.25) * (Qxy * R(cx * cy) + Qxz * R(cx * cz) + Qyz * R(cy * cz));
    const R tf = act ? -(ab * ds * dh + bb * dh * dh) * ifeq - dfb * feq : R(0);
    R rhob = wsum(tf) * irho;
    const R ub[3] = {wsum(tf * pick(dl[0], cx)), wsum(tf * pick(dl[1], cy)), wsum(tf * pick(dl[2], cz))};
    rhob -= (ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2]) * irho;
    if (!act) return R(0);
    return lv + dfb + rhob + (R(cx) * ub[0] + R(cy) * ub[1] + R(cz) * ub[2]) * irho;
}

// ----------------------------------------------------------------- pull transpose
// Sum of Lam(x)_i over the nodes x whose pull of direction i read node y:
// per axis the reader coordinate y_a + c_a (wrapped on a periodic face, none
// through another face) and, on an outflow face layer, y_a itself (its source
// was clamped onto y); a wall face adds the bounce-back reader y itself for
// direction 26 - i.
template <typename R>
__device__ __forceinline__ R pull_transpose(const Lattice &L, const R *__restrict__ lam, int x, int y, int z, int i)
{
    const int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
    const int p[3] = {x, y, z}, n[3] = {L.nx, L.ny, L.nz};
    int r0[3], r1[3];
    bool h0[3], h1[3], wall = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int t = p[a] + c[a];
        h0[a] = true;
        r0[a] = t;
        if (t < 0 || t >= n[a]) {
            const int face = t < 0 ? L.face[2 * a] : L.face[2 * a + 1];
            if (face == LBM_FACE_PERIODIC) r0[a] = (t + n[a]) % n[a];
            else {
                h0[a] = false;
                if (face == LBM_FACE_WALL) wall = true;
            }
        }
        h1[a] = (c[a] == 1 && p[a] == 0 && L.face[2 * a] == LBM_FACE_OUTFLOW) ||
                (c[a] == -1 && p[a] == n[a] - 1 && L.face[2 * a + 1] == LBM_FACE_OUTFLOW);
        r1[a] = p[a];
    }
    const size_t N = (size_t)L.N;
    R s = 0;
    for (int m = 0; m < 8; ++m) {
        int q[3];
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            const bool alt = (m >> a) & 1;
            if (alt ? !h1[a] : !h0[a]) { ok = false; break; }
            q[a] = alt ? r1[a] : r0[a];
        }
        if (ok) s += lam[(size_t)i * N + q[0] + (size_t)L.nx * (q[1] + (size_t)L.ny * q[2])];
    }
    if (wall) s += lam[(size_t)(26 - i) * N + x + (size_t)L.nx * (y + (size_t)L.ny * z)];
    return s;
}

// Reader offsets for one axis: o[c+1] is the offset of the node at a + c (the
// node that pulled direction component c from a), wrapped on periodic faces.
// Returns true when the plain offsets do not describe every reader: a + c
// leaves the box through a non-periodic face, or a lies on an outflow face
// layer (clamped readers).
__device__ __forceinline__ bool axis_readers(int a, int n, int stride, int face_lo, int face_hi, int o[3])
{
    o[0] = -stride;
    o[1] = 0;
    o[2] = stride;
    bool special = false;
    if (a == 0) {
        if (face_lo == LBM_FACE_PERIODIC) o[0] = (n - 1) * stride;
        else special = true;
    }
    if (a == n - 1) {
        if (face_hi == LBM_FACE_PERIODIC) o[2] = -(n - 1) * stride;
        else special = true;
    }
    return special;
}

// band position of node (x, y, z) in the band of body state b, or -1
__device__ __forceinline__ int band_index(const Lattice &L, const GeomParams &G, const DevBody *b, int x, int y,
                                          int z)
{
    const int p[3] = {x, y, z}, n[3] = {L.nx, L.ny, L.nz};
    int l[3];
    for (int a = 0; a < 3; ++a) {
        int d = p[a] - b->band_lo[a];
        if (G.periodic[a]) d = ((d % n[a]) + n[a]) % n[a];
        if (d < 0 || d >= b->band_n[a]) return -1;
        l[a] = d;
    }
    return l[0] + G.cap[0] * (l[1] + G.cap[1] * l[2]);
}

// Where the adjoint of S^{t+1} comes from when step t is reversed.
template <typename R>
struct NextAdj {
    const R *lam;          // Lam^{t+1}, or lambda_T (direct), or NULL (zero)
    const double *ext;     // ext^{t+1} (band of step t+1)
    const DevBody *band;   // body state of step t+1 (band)
    const uint8_t *flags;  // marks after step t+1 (UNCOVERED: refilled in step t+1)
    int direct;            // 1: lam is the full adjoint of S^{t+1}
};

// lambda(S^{t+1})(x)_i
template <typename R>
__device__ __forceinline__ R next_adjoint(const Lattice &L, const GeomParams &G, const NextAdj<R> &A, int x, int y,
                                          int z, int n, int i)
{
    if (A.direct) return A.lam ? A.lam[(size_t)i * (size_t)L.N + n] : R(0);
    if (A.flags && (A.flags[n] & FL_UNCOVERED)) return R(0);
    R v = pull_transpose<R>(L, A.lam, x, y, z, i);
    if (A.ext) {
        const int k = band_index(L, G, A.band, x, y, z);
        if (k >= 0) v += (R)A.ext[(size_t)k * Q + i];
    }
    return v;
}

// lambda(S^{t+1})(x)_i on the rare path, out of line to keep the bulk
// kernel's code small
template <typename R>
__device__ __noinline__ R next_adjoint_rare(const Lattice &L, const GeomParams &G, const NextAdj<R> &A, int x, int y,
                                            int z, int n, int i)
{
    return next_adjoint<R>(L, G, A, x, y, z, n, i);
}

// ----------------------------------------------------------------- kernels
// Nodes fluid at t+1 without missing links: Lam^t(x) = C'(F(x))^T lambda(S^{t+1})(x);
// solid nodes get Lam^t = 0; boundary nodes are left to the boundary adjoint.
// Minimum resident blocks per SM requested for the bulk adjoint (a register
// cap; LBM_ADJ_MIN_BLOCKS overrides it at build time).
#ifndef LBM_ADJ_MIN_BLOCKS
#define LBM_ADJ_MIN_BLOCKS 4
#endif

// Launch modes as those of the bulk kernel (BulkMode): ALL every node;
// OUTSIDE the nodes outside box0 (the band of step t) and box1 (the band of
// step t+1, whose ext and refill marks the gather reads), which are fluid and
// no boundary node at t+1 and read neither; BAND the nodes of box0 that are
// not in box1 (capacity-box grid).
template <typename S>
__global__ void __launch_bounds__(128, LBM_ADJ_MIN_BLOCKS) adjoint_bulk_kernel(const Lattice L, const GeomParams G,
                                                           const S *__restrict__ st,
                                                           const NextAdj<typename Codec<S>::R> A,
                                                           const uint8_t *__restrict__ flags1,
                                                           typename Codec<S>::R *__restrict__ lam_out,
                                                           int mode, const int *__restrict__ box0,
                                                           const int *__restrict__ box1)
{
    using R = typename Codec<S>::R;
    int x, y, z;
    if (mode == BULK_BAND) {
        const int k = blockIdx.x * blockDim.x + threadIdx.x;
        const int lx = k % G.cap[0], ly = (k / G.cap[0]) % G.cap[1], lz = k / (G.cap[0] * G.cap[1]);
        if (lz >= G.cap[2] || lx >= box0[3] || ly >= box0[4] || lz >= box0[5]) return;
        x = sweep_coord(box0[0] + lx, L.nx);
        y = sweep_coord(box0[1] + ly, L.ny);
        z = sweep_coord(box0[2] + lz, L.nz);
        if (box1 && in_sweep_box(L, box1, x, y, z)) return;
    } else {
        x = blockIdx.x * blockDim.x + threadIdx.x;
        y = blockIdx.y;
        z = blockIdx.z;
        if (x >= L.nx) return;
        if (mode == BULK_OUTSIDE && ((box0 && in_sweep_box(L, box0, x, y, z)) || (box1 && in_sweep_box(L, box1, x, y, z))))
            return;
    }
    const int n = x + L.nx * (y + L.ny * z);
    const size_t N = (size_t)L.N;
    const uint8_t f1 = flags1 ? flags1[n] : 0;
    if (f1 & FL_SOLID) {
#pragma unroll
        for (int i = 0; i < Q; ++i) lam_out[(size_t)i * N + n] = R(0);
        return;
    }
    if (f1 & FL_BOUNDARY) return;
    R lam[Q];
    int ox[3], oy[3], oz[3];
    bool special = axis_readers(x, L.nx, 1, L.face[0], L.face[1], ox);
    special |= axis_readers(y, L.ny, L.nx, L.face[2], L.face[3], oy);
    special |= axis_readers(z, L.nz, L.nx * L.ny, L.face[4], L.face[5], oz);
    if (A.direct || special || (A.flags && (A.flags[n] & FL_UNCOVERED))) {
#pragma unroll
        for (int i = 0; i < Q; ++i) lam[i] = next_adjoint_rare<R>(L, G, A, x, y, z, n, i);
    } else {
        const R *p = A.lam + n;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            lam[i] = p[(long long)i * (long long)N + (ox[cx_of(i) + 1] + oy[cy_of(i) + 1] + oz[cz_of(i) + 1])];
        if (A.ext) {
            const int k = band_index(L, G, A.band, x, y, z);
            if (k >= 0) {
#pragma unroll
                for (int i = 0; i < Q; ++i) lam[i] += (R)A.ext[(size_t)k * Q + i];
            }
        }
    }
    R g[Q];
    gather_global<S>(L, st, x, y, z, n, g);
    kbc_vjp<R>(g, lam, (R)L.beta, (R)L.inv_beta, (R)L.rho0, L.gamma_mode);
#pragma unroll
    for (int i = 0; i < Q; ++i) lam_out[(size_t)i * N + n] = lam[i];
}

// ----------------------------------------------------------------- centre-of-mass frame
// theta-derivatives of the mesh's volume sums (divergence theorem, as the
// forward mass kernel): per triangle d = e1 x e2, V += d_x h1(x)/6,
// S_x += d_x h2(x)/24, S_xx += d_x h3(x)/60, S_y += d_y h2(y)/24,
// S_yy += d_y h3(y)/60; only the vertices' y moves with theta (by the
// midline tangent), so d_x and the y polynomials carry the derivative.
// Sums: at tau (V, Sx, Sy, Sxx, Syy and their 3 theta-derivatives, 20) and at
// tau -+ 1 (V, Sx, Sy and derivatives, 12 each): 44 per triangle.
constexpr int COM_SUMS = 44;

__device__ __forceinline__ void com_triangle_sums(const GeomParams &G, int k, double t, bool second, double *acc)
{
    double P[3][3], ty[3][3];
    for (int m = 0; m < 3; ++m) {
        const int iv = G.mesh_tris[3 * k + m];
        const double s = G.mesh_rest[3 * iv];
        P[m][0] = s;
        P[m][1] = swimmer_midline(G, s, t) + G.mesh_rest[3 * iv + 1];
        P[m][2] = G.mesh_rest[3 * iv + 2];
        swimmer_midline_tangent(G, s, t, ty[m]);
    }
    const double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
    const double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
    const double dx = e1[1] * e2[2] - e1[2] * e2[1], dy = e1[2] * e2[0] - e1[0] * e2[2];
    const double x0 = P[0][0], x1 = P[1][0], x2 = P[2][0];
    const double y0 = P[0][1], y1 = P[1][1], y2 = P[2][1];
    const double hx1 = x0 + x1 + x2;
    const double hx2 = x0 * x0 + x1 * x1 + x2 * x2 + x0 * x1 + x0 * x2 + x1 * x2;
    const double hx3 = x0 * x0 * x0 + x1 * x1 * x1 + x2 * x2 * x2 + x0 * x0 * (x1 + x2) + x1 * x1 * (x0 + x2) +
                       x2 * x2 * (x0 + x1) + x0 * x1 * x2;
    const double hy2 = y0 * y0 + y1 * y1 + y2 * y2 + y0 * y1 + y0 * y2 + y1 * y2;
    const double hy3 = y0 * y0 * y0 + y1 * y1 * y1 + y2 * y2 * y2 + y0 * y0 * (y1 + y2) + y1 * y1 * (y0 + y2) +
                       y2 * y2 * (y0 + y1) + y0 * y1 * y2;
    // d h2 / d y_m and d h3 / d y_m
    const double g2[3] = {2 * y0 + y1 + y2, 2 * y1 + y0 + y2, 2 * y2 + y0 + y1};
    const double g3[3] = {3 * y0 * y0 + 2 * y0 * (y1 + y2) + y1 * y1 + y2 * y2 + y1 * y2,
                          3 * y1 * y1 + 2 * y1 * (y0 + y2) + y0 * y0 + y2 * y2 + y0 * y2,
                          3 * y2 * y2 + 2 * y2 * (y0 + y1) + y0 * y0 + y1 * y1 + y0 * y1};
    acc[0] += dx * hx1 / 6.0;
    acc[1] += dx * hx2 / 24.0;
    acc[2] += dy * hy2 / 24.0;
    int o = 3;
    if (second) {
        acc[3] += dx * hx3 / 60.0;
        acc[4] += dy * hy3 / 60.0;
        o = 5;
    }
    for (int j = 0; j < 3; ++j) {
        const double ddx = (ty[1][j] - ty[0][j]) * e2[2] - e1[2] * (ty[2][j] - ty[0][j]);
        const double dh2 = g2[0] * ty[0][j] + g2[1] * ty[1][j] + g2[2] * ty[2][j];
        acc[o + 0] += ddx * hx1 / 6.0;
        acc[o + 1] += ddx * hx2 / 24.0;
        acc[o + 2] += dy * dh2 / 24.0;
        if (second) {
            const double dh3 = g3[0] * ty[0][j] + g3[1] * ty[1][j] + g3[2] * ty[2][j];
            acc[o + 3] += ddx * hx3 / 60.0;
            acc[o + 4] += dy * dh3 / 60.0;
            o += 5;
        } else {
            o += 3;
        }
    }
}

// ComTangents of the pose of body state b (time tau = b->t): block partials,
// a fixed-order last-block sum, then dc = d(S/V), dc_dot, dI with
// I = (m/V)(Sxx + Syy) - m (cx^2 + cy^2)
__global__ void __launch_bounds__(256) com_tangent_kernel(const GeomParams G, const DevBody *__restrict__ b,
                                                          double *__restrict__ partials, unsigned *__restrict__ ticket,
                                                          ComTangents *__restrict__ out)
{
    double acc[COM_SUMS];
    for (int c = 0; c < COM_SUMS; ++c) acc[c] = 0.0;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < G.n_triangles) {
        com_triangle_sums(G, k, b->t, true, acc);
        com_triangle_sums(G, k, b->t + 1.0, false, acc + 20);
        com_triangle_sums(G, k, b->t - 1.0, false, acc + 32);
    }
    __shared__ double sm[8][COM_SUMS];
    __shared__ bool last;
    for (int c = 0; c < COM_SUMS; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < COM_SUMS) {
        double v = 0;
        for (int w = 0; w < 8; ++w) v += sm[w][threadIdx.x];
        partials[blockIdx.x * COM_SUMS + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double S[COM_SUMS];
    if (threadIdx.x < COM_SUMS) {
        double v = 0;
        for (int p = 0; p < (int)gridDim.x; ++p) v += ((volatile double *)partials)[p * COM_SUMS + threadIdx.x];
        S[threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double m = G.mass;
    const double V = S[0], cx = S[1] / V, cy = S[2] / V;
    const double Vp = S[20], Vm = S[32];
    for (int j = 0; j < 3; ++j) {
        const double dV = S[5 + 5 * j], dSx = S[6 + 5 * j], dSy = S[7 + 5 * j];
        const double dSxx = S[8 + 5 * j], dSyy = S[9 + 5 * j];
        const double dcx = (dSx - cx * dV) / V, dcy = (dSy - cy * dV) / V;
        out->dc[j][0] = dcx;
        out->dc[j][1] = dcy;
        out->dI[j] = -m * dV / (V * V) * (S[3] + S[4]) + m / V * (dSxx + dSyy) - 2.0 * m * (cx * dcx + cy * dcy);
        const double dVp = S[23 + 3 * j], dVm = S[35 + 3 * j];
        const double dcxp = (S[24 + 3 * j] - S[21] / Vp * dVp) / Vp, dcyp = (S[25 + 3 * j] - S[22] / Vp * dVp) / Vp;
        const double dcxm = (S[36 + 3 * j] - S[33] / Vm * dVm) / Vm, dcym = (S[37 + 3 * j] - S[34] / Vm * dVm) / Vm;
        out->dcdot[j][0] = (dcxp - dcxm) / 2.0;
        out->dcdot[j][1] = (dcyp - dcym) / 2.0;
    }
    *ticket = 0u;
}

// adds (ub . (c_m - u_k)) / rho_k + rb to ext[node k][m] for every lane k with a
// non-zero velocity or density adjoint; all lanes m < 27 write one entry each
template <typename R>
__device__ __forceinline__ void scatter_moment_adjoints(const Lattice &L, const GeomParams &G, const DevBody *b,
                                                        int lane, int nk, bool has, const R ubk[3], R rbk,
                                                        const R (*su)[4], double *__restrict__ ext)
{
    unsigned m = __ballot_sync(FULL, has);
    while (m) {
        const int k = __ffs(m) - 1;
        m &= m - 1;
        const int node = __shfl_sync(FULL, nk, k);
        const R u0 = __shfl_sync(FULL, ubk[0], k), u1 = __shfl_sync(FULL, ubk[1], k);
        const R u2 = __shfl_sync(FULL, ubk[2], k), r = __shfl_sync(FULL, rbk, k);
        int x, y, z;
        node_xyz(L, node, x, y, z);
        const int kb = band_index(L, G, b, x, y, z);
        if (kb >= 0 && lane < Q) {
            const R rho = su[k][0];
            const R v = (u0 * (R(cx_of(lane)) - su[k][1]) + u1 * (R(cy_of(lane)) - su[k][2]) +
                         u2 * (R(cz_of(lane)) - su[k][3])) / rho + r;
            atomicAdd(ext + (size_t)kb * Q + lane, (double)v);
        }
    }
}

// fd_gradient transposed: velocity adjoints of the staged neighbourhood (lane
// k) and of the centre velocity from du_bar
template <typename R>
__device__ __forceinline__ void fd_gradient_adj(const int *sok, const R dub[3][3], int lane, R unb[3], R ucb[3])
{
    const int step[3] = {9, 3, 1};
    for (int b = 0; b < 3; ++b) {
        const int kp = 13 + step[b], km = 13 - step[b];
        const bool op = sok[kp], om = sok[km];
        for (int a = 0; a < 3; ++a) {
            const R v = dub[a][b];
            if (op && om) {
                if (lane == kp) unb[a] += R(0.5) * v;
                if (lane == km) unb[a] -= R(0.5) * v;
            } else if (op) {
                if (lane == kp) unb[a] += v;
                ucb[a] -= v;
            } else if (om) {
                ucb[a] += v;
                if (lane == km) unb[a] -= v;
            }
        }
    }
}

// transposes of grad_shifted and pressure_excess for lane-held gb = dJ/dg*_i:
// accumulates rho_bar, u_bar (3) and du_bar (3x3)
template <typename R>
__device__ __forceinline__ void grad_pressure_adj(R gb, int i, bool act, R rho, const R u[3], const R du[3][3],
                                                  R beta, R &rhob, R ub[3], R dub[3][3])
{
    const R cx = act ? R(cx_of(i)) : R(0), cy = act ? R(cy_of(i)) : R(0), cz = act ? R(cz_of(i)) : R(0);
    const R w = act ? weight<R>(i) * gb : R(0);
    const R cu = cx * u[0] + cy * u[1] + cz * u[2];
    rhob += wsum(w * (R(1) + R(3) * cu));
    ub[0] += wsum(w * R(3) * rho * cx);
    ub[1] += wsum(w * R(3) * rho * cy);
    ub[2] += wsum(w * R(3) * rho * cz);
    const R third = R(1.0 / 3.0);
    R Qb[6];
    Qb[0] = wsum(w * R(4.5) * (cx * cx - third));
    Qb[1] = wsum(w * R(4.5) * (cy * cy - third));
    Qb[2] = wsum(w * R(4.5) * (cz * cz - third));
    Qb[3] = wsum(w * R(9) * cx * cy);
    Qb[4] = wsum(w * R(9) * cx * cz);
    Qb[5] = wsum(w * R(9) * cy * cz);
    // Qt_ab = rho u_a u_b - (rho / (6 beta)) (du_ab + du_ba)
    const R k6 = R(1) / (R(6) * beta);
    const int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
    for (int m = 0; m < 6; ++m) {
        const int a = A[m], b = B[m];
        rhob += Qb[m] * (u[a] * u[b] - k6 * (du[a][b] + du[b][a]));
        ub[a] += Qb[m] * rho * u[b];
        ub[b] += Qb[m] * rho * u[a];
        dub[a][b] -= Qb[m] * rho * k6;
        dub[b][a] -= Qb[m] * rho * k6;
    }
}

// Adjoint state of a swimmer free along x (head frame), in device memory:
// a_X, a_U = dJ/dX0, dJ/dU0 of the body state of the step last reversed, and
// the weights of the force of the step reversed next in J: w/T plus, along x,
// a_U/m (the force enters U0 of the state after it, U' = U + F/m).  For a held
// or prescribed body only the weights are used (w/T, constant).
struct BodyAdjoint {
    double aX[3], aU[3];  // dJ/dX, dJ/dU of the free axes
    double aPsi, aL;      // dJ/dpsi, dJ/d(I omega) (yaw free)
    double fw[3];         // weights of the force of the step reversed next
    double mw;            // weight of the torque M_z of the step reversed next (yaw free)
    double dth[3];        // dJ/dtheta through omega = I omega / I(theta)
};

// one writer per band position and reversed step: derivatives with respect to
// (X_x, X_y, psi, U_x, U_y, omega) for the swimmer, (X_x, X_y, X_z, U_x, U_y,
// U_z) for the sphere, from the boundary node there (0..5) and from the
// refilled node there (6..11)
constexpr int BODY_SLOTS = 12;

// Boundary nodes of step t: forward recomputation of the Grad completion
// (same operations as the boundary kernel), then its transpose.
template <typename S>
__global__ void __launch_bounds__(BWARPS * 32) adjoint_boundary_kernel(
    const Lattice L, const GeomParams G, const DevBody *__restrict__ b, const int *__restrict__ blist,
    const int *__restrict__ bpos, const S *__restrict__ st, const NextAdj<typename Codec<S>::R> A,
    const uint8_t *__restrict__ flags1, typename Codec<S>::R *__restrict__ lam_out, double *__restrict__ ext,
    double *__restrict__ tslots, const BodyAdjoint *__restrict__ badj, double *__restrict__ bslot,
    const ComTangents *__restrict__ ct)
{
    using R = typename Codec<S>::R;
    __shared__ R s_f[BWARPS][Q][28];
    __shared__ R s_u[BWARPS][Q][4];
    __shared__ int s_ok[BWARPS][Q];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    R (*sf)[28] = s_f[w];
    R (*su)[4] = s_u[w];
    int *sok = s_ok[w];
    const int count = min(b->n_boundary, G.cap_boundary);
    const size_t N = (size_t)L.N;
    const R rho0 = (R)L.rho0, beta = (R)L.beta;
    const double fw[3] = {badj->fw[0], badj->fw[1], badj->fw[2]};
    const double mw = badj->mw;

    for (int slot = blockIdx.x * BWARPS + w; slot < count; slot += gridDim.x * BWARPS) {
        const int n = blist[slot];
        int x, y, z;
        node_xyz(L, n, x, y, z);
        const int i = lane;
        const bool act = i < Q;
        const int cx = act ? cx_of(i) : 0, cy = act ? cy_of(i) : 0, cz = act ? cz_of(i) : 0;
        bool solid_src = false;
        if (act && i != 13) {
            const int src = pull_source(L, x, y, z, cx, cy, cz);
            solid_src = src >= 0 && (flags1[src] & FL_SOLID);
        }
        const uint32_t mask = __ballot_sync(FULL, solid_src);
        int nk = -1;
        if (act) nk = neighbour(L, x, y, z, cx, cy, cz);
        if (act) sok[lane] = nk >= 0 && !(flags1[nk] & FL_SOLID);
        __syncwarp();
        const uint32_t need = (1u << 13) | (1u << 22) | (1u << 4) | (1u << 16) | (1u << 10) |
                              (1u << 14) | (1u << 12) | mask;
        stage<S, R>(L, st, lane, nk, need, sf, su, sok);
        const bool miss = act && ((mask >> i) & 1u);
        // known pulls (face rules as in the bulk kernel)
        R Fi = R(0);
        if (act && !miss) {
            int p[3] = {x - cx, y - cy, z - cz};
            const int nn[3] = {L.nx, L.ny, L.nz};
            int kind = 0;
            for (int a = 0; a < 3; ++a) {
                int face = -1;
                if (p[a] < 0) face = L.face[2 * a];
                else if (p[a] >= nn[a]) face = L.face[2 * a + 1];
                if (face < 0) continue;
                if (face == LBM_FACE_PERIODIC) p[a] = (p[a] + nn[a]) % nn[a];
                else if (face == LBM_FACE_OUTFLOW) p[a] = p[a] < 0 ? 0 : nn[a] - 1;
                else if (face == LBM_FACE_WALL) kind = 2;
                else kind = kind > 1 ? kind : 1;
            }
            if (kind == 2) Fi = sf[13][26 - i];
            else if (kind == 1) Fi = (R)L.g_face[i];
            else Fi = Codec<S>::load(st + (size_t)i * N + (p[0] + L.nx * (p[1] + L.ny * p[2])));
        }
        const R fbb = act ? sf[13][26 - (act ? i : 0)] : R(0);
        double q = 0, uw[3] = {0, 0, 0};
        MeshHit hit{-1, 0.0, 0.0};
        if (G.kind == LBM_BODY_MESH) mesh_links_warp<R>(G, b, x, y, z, mask, lane, q, uw, hit);
        else if (miss) link_data<R>(L, G, b, x, y, z, cx, cy, cz, q, uw);
        const R gstat = miss ? fbb : Fi;
        const R dyn = miss ? R(6) * weight<R>(i) * rho0 * (R(cx) * (R)uw[0] + R(cy) * (R)uw[1] + R(cz) * (R)uw[2])
                           : R(0);
        const R qq = (R)q;
        R ut[3] = {0, 0, 0};
        if (miss) {
            if (sok[i]) {
                for (int a = 0; a < 3; ++a) ut[a] = (qq * su[i][1 + a] + (R)uw[a]) / (R(1) + qq);
            } else {
                for (int a = 0; a < 3; ++a) ut[a] = (R)uw[a];
            }
        }
        const R nmiss = R(__popc(mask));
        const R rho_t = rho0 + wsum(act ? gstat : R(0)) + wsum(dyn);
        R u_t[3];
        for (int a = 0; a < 3; ++a) u_t[a] = wsum(ut[a]) / nmiss;
        R du[3][3];
        const R uc[3] = {su[13][1], su[13][2], su[13][3]};
        fd_gradient<R>(su, sok, uc, du);
        R Qt[6];
        pressure_excess<R>(rho_t, u_t, du, beta, Qt);
        R gi = Fi;
        if (miss) gi = grad_shifted<R>(i, rho_t, rho0, u_t, Qt);

        // ---- adjoint
        const R lam = act ? next_adjoint<R>(L, G, A, x, y, z, n, i) : R(0);
        R Fb = kbc_vjp_lanes<R>(gi, lam, i, beta, (R)L.inv_beta, rho0, L.gamma_mode);
        // momentum exchange in J: dF_a = (-c_a - uw_a) fout - (c_a - uw_a) fin
        // (the link arithmetic in R, the collision's precision; fin - fout as
        // the difference of the shifted values, where W rho0 cancels)
        R uwb[3] = {0, 0, 0};
        R fbbb = 0;
        // the torque M_z about X of the free yaw enters J with weight mw:
        // M_z = r_x dF_y - r_y dF_x, r = x_b - q c - X
        double qb_m = 0.0, gXm[2] = {0.0, 0.0};
        if (miss) {
            const R Wr = weight<R>(i) * rho0;
            const R fout = fbb + Wr, fin = gi + Wr, dio = gi - fbb;
            const R c[3] = {R(cx), R(cy), R(cz)};
            R sin_ = 0, sout = 0;
            for (int a = 0; a < 3; ++a) {
                const R u = (R)uw[a], f = (R)fw[a];
                sin_ -= (c[a] - u) * f;
                sout += (-c[a] - u) * f;
                uwb[a] += f * dio;
            }
            if (mw != 0.0) {
                const double cd[3] = {(double)cx, (double)cy, (double)cz};
                const double fo = (double)fout, fi = (double)fin, dd = (double)dio;
                const double r0 = body_offset(L, G, b, 0, x) - q * cd[0], r1 = body_offset(L, G, b, 1, y) - q * cd[1];
                const double dFx = (-cd[0] - uw[0]) * fo - (cd[0] - uw[0]) * fi;
                const double dFy = (-cd[1] - uw[1]) * fo - (cd[1] - uw[1]) * fi;
                sin_ += (R)(mw * (-r0 * (cd[1] - uw[1]) + r1 * (cd[0] - uw[0])));
                sout += (R)(mw * (r0 * (-cd[1] - uw[1]) - r1 * (-cd[0] - uw[0])));
                uwb[0] -= (R)(mw * r1 * dd);
                uwb[1] += (R)(mw * r0 * dd);
                qb_m = mw * (-cd[0] * dFy + cd[1] * dFx);
                gXm[0] = -mw * dFy;
                gXm[1] = mw * dFx;
            }
            Fb += sin_;
            fbbb += sout;
        }
        // Grad completion (missing lanes) and pressure excess
        R rhob = 0, utb[3] = {0, 0, 0}, dub[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        grad_pressure_adj<R>(miss ? Fb : R(0), i, act, rho_t, u_t, du, beta, rhob, utb, dub);
        // u_t = mean over missing links of (q u_f + u_w)/(1 + q), or u_w
        R unb[3] = {0, 0, 0}, ucb[3] = {0, 0, 0};
        R qb = 0;
        if (miss) {
            const R inv1q = R(1) / (R(1) + qq);
            for (int a = 0; a < 3; ++a) {
                const R v = utb[a] / nmiss;
                if (sok[i]) {
                    unb[a] += v * qq * inv1q;
                    uwb[a] += v * inv1q;
                    qb += v * (su[i][1 + a] - (R)uw[a]) * inv1q * inv1q;
                } else {
                    uwb[a] += v;
                }
            }
        }
        qb += (R)qb_m;
        // rho_t = rho0 + sum gstat + sum dyn
        R lam_row = 0;
        if (act && !miss) lam_row = Fb + rhob;
        if (miss) {
            fbbb += rhob;
            for (int a = 0; a < 3; ++a)
                uwb[a] += rhob * R(6) * weight<R>(i) * rho0 * R(a == 0 ? cx : a == 1 ? cy : cz);
        }
        fd_gradient_adj<R>(sok, dub, lane, unb, ucb);
        if (lane == 13)
            for (int a = 0; a < 3; ++a) unb[a] += ucb[a];
        // outputs: Lam row of this node, ext at this node and at the neighbours
        if (act) lam_out[(size_t)i * N + n] = lam_row;
        const int kb = band_index(L, G, b, x, y, z);
        if (miss && kb >= 0) atomicAdd(ext + (size_t)kb * Q + (26 - i), (double)fbbb);
        const bool has = act && nk >= 0 && (unb[0] != R(0) || unb[1] != R(0) || unb[2] != R(0));
        scatter_moment_adjoints<R>(L, G, b, lane, nk, has, unb, R(0), su, ext);
        // parameters: dJ/dtheta through q and u_w of each missing link
        double tb[3] = {0, 0, 0};
        double gb[6] = {0, 0, 0, 0, 0, 0};  // (X_x, X_y, psi, U_x, U_y, omega)
        if (miss && G.kind == LBM_BODY_MESH && G.com_frame) {
            double dq[COM_DIRS], duw[COM_DIRS][3];
            com_link_tangents(G, b, *ct, x, y, z, cx, cy, cz, q, hit, dq, duw);
            for (int d = 0; d < COM_DIRS; ++d) {
                const double v = qb * dq[d] + uwb[0] * duw[d][0] + uwb[1] * duw[d][1] + uwb[2] * duw[d][2];
                if (d < 3) tb[d] = v;
                else gb[d - 3] = v;
            }
            gb[0] += gXm[0];
            gb[1] += gXm[1];
        } else if (miss && G.kind == LBM_BODY_MESH) {
            double dq[3], duw[3][3];
            mesh_link_tangent<R>(G, b, x, y, z, cx, cy, cz, q, hit, dq, duw);
            for (int k = 0; k < 3; ++k)
                tb[k] = (double)(qb * (R)dq[k] + uwb[0] * (R)duw[k][0] + uwb[1] * (R)duw[k][1] + uwb[2] * (R)duw[k][2]);
            if (bslot) {
                // the head frame: every vertex moves with X0, u_w with U0
                double dqX, duwX[3];
                mesh_link_body_tangent(G, b, x, y, z, cx, cy, cz, q, hit, dqX, duwX);
                gb[0] = qb * dqX + uwb[0] * duwX[0] + uwb[1] * duwX[1] + uwb[2] * duwX[2];
                gb[3] = uwb[0];
            }
        } else if (miss && G.kind == LBM_BODY_SPHERE && bslot) {
            // the free sphere: q = (c.d - sqrt(disc))/|c|^2 with d = x_b - X,
            // disc = (c.d)^2 - |c|^2 (|d|^2 - R^2); u_w = U
            const double d[3] = {body_offset(L, G, b, 0, x), body_offset(L, G, b, 1, y), body_offset(L, G, b, 2, z)};
            const double c[3] = {(double)cx, (double)cy, (double)cz};
            const double cc = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
            const double cd = c[0] * d[0] + c[1] * d[1] + c[2] * d[2];
            const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            const double sq = sqrt(fmax(cd * cd - cc * (dd - G.R * G.R), 0.0));
            for (int a = 0; a < 3; ++a) {
                const double dqdd = sq > 0.0 ? (c[a] - (cd * c[a] - cc * d[a]) / sq) / cc : 0.0;
                gb[a] = -qb * dqdd;
                gb[3 + a] = uwb[a];
            }
        } else if (miss && G.kind == LBM_BODY_AIRFOIL) {
            double dq[2], dX1[2], dU1[2];
            airfoil_link_tangent(G, b, x, y, cx, cy, q, dq);
            airfoil_plunge_tangent(G, b->t, dX1, dU1);
            for (int k = 0; k < 2; ++k) tb[k] = qb * dq[k] + uwb[1] * dU1[k];
        }
        // per-node sums over the links in R; the slots sum the nodes in double
        for (int k = 0; k < 3; ++k) {
            R v = (R)tb[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
            if (lane == 0) tslots[(size_t)bpos[slot] * 6 + k] += (double)v;
        }
        // the free body's state through q and u_w of each missing link
        if (bslot) {
            for (int d = 0; d < 6; ++d) {
                double v = gb[d];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
                if (lane == 0) bslot[(size_t)bpos[slot] * BODY_SLOTS + d] = v;
            }
        }
        __syncwarp();
    }
}

// Refilled nodes of step t: transpose of the refill (Grad distribution of the
// neighbour-mean density, the body velocity and the finite-difference
// gradient), fed by lambda(St^t) at the node.
template <typename S>
__global__ void __launch_bounds__(BWARPS * 32) adjoint_refill_kernel(
    const Lattice L, const GeomParams G, const DevBody *__restrict__ b, const int *__restrict__ ulist,
    const int *__restrict__ upos, const S *__restrict__ st, const typename Codec<S>::R *__restrict__ lam_t,
    const uint8_t *__restrict__ flags1, double *__restrict__ ext, double *__restrict__ tslots,
    double *__restrict__ bslot, const ComTangents *__restrict__ ct)
{
    using R = typename Codec<S>::R;
    __shared__ R s_f[BWARPS][Q][28];
    __shared__ R s_u[BWARPS][Q][4];
    __shared__ int s_ok[BWARPS][Q];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    R (*sf)[28] = s_f[w];
    R (*su)[4] = s_u[w];
    int *sok = s_ok[w];
    const int count = min(b->n_uncovered, G.cap_uncovered);
    const R rho0 = (R)L.rho0, beta = (R)L.beta;
    for (int slot = blockIdx.x * BWARPS + w; slot < count; slot += gridDim.x * BWARPS) {
        const int n = ulist[slot];
        int x, y, z;
        node_xyz(L, n, x, y, z);
        const bool act = lane < Q;
        int nk = -1;
        if (act && lane != 13) nk = neighbour(L, x, y, z, cx_of(lane), cy_of(lane), cz_of(lane));
        if (act) sok[lane] = nk >= 0 && !(flags1[nk] & FL_SOLID_PREV);
        __syncwarp();
        const uint32_t need = __ballot_sync(FULL, act && sok[lane]);
        stage<S, R>(L, st, lane, nk, need, sf, su, sok);
        const R cnt = R(__popc(need));
        const R rsum = wsum((act && sok[lane]) ? su[lane][0] : R(0));
        const R rho = cnt > R(0) ? rsum / cnt : rho0;
        double ud[3] = {b->U[0], b->U[1], b->U[2]};
        if (G.kind == LBM_BODY_PLANES) {
            const double *v = (double)y < 0.5 * (G.y_lo + G.y_hi) ? G.U_lo : G.U_hi;
            ud[0] = v[0]; ud[1] = v[1]; ud[2] = v[2];
        } else if (G.kind == LBM_BODY_MESH) {
            mesh_material_velocity(G, b, (double)x, (double)y, ud);
        }
        const R u[3] = {(R)ud[0], (R)ud[1], (R)ud[2]};
        R du[3][3];
        fd_gradient<R>(su, sok, u, du);
        // adjoint of the refilled populations: lambda(St^t) at the node
        R lam = 0;
        if (act) {
            lam = pull_transpose<R>(L, lam_t, x, y, z, lane);
            const int kb = band_index(L, G, b, x, y, z);
            if (kb >= 0) lam += (R)ext[(size_t)kb * Q + lane];
        }
        R rhob = 0, ub[3] = {0, 0, 0}, dub[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        grad_pressure_adj<R>(lam, lane, act, rho, u, du, beta, rhob, ub, dub);
        R unb[3] = {0, 0, 0}, ucb[3] = {0, 0, 0};
        fd_gradient_adj<R>(sok, dub, lane, unb, ucb);
        for (int a = 0; a < 3; ++a) ub[a] += ucb[a];
        // rho = mean of the neighbours' densities
        const R rkb = (act && sok[lane] && cnt > R(0)) ? rhob / cnt : R(0);
        const bool has = act && sok[lane] && (rkb != R(0) || unb[0] != R(0) || unb[1] != R(0) || unb[2] != R(0));
        scatter_moment_adjoints<R>(L, G, b, lane, nk, has, unb, rkb, su, ext);
        // parameters through the body velocity
        double tb[3] = {0, 0, 0};
        double gb[6] = {0, 0, 0, 0, 0, 0};
        if (lane == 0 && G.kind == LBM_BODY_MESH && G.com_frame) {
            double du[COM_DIRS][3];
            com_material_velocity_tangents(G, b, *ct, (double)x, (double)y, du);
            for (int d = 0; d < COM_DIRS; ++d) {
                const double v = (double)ub[0] * du[d][0] + (double)ub[1] * du[d][1] + (double)ub[2] * du[d][2];
                if (d < 3) tb[d] = v;
                else gb[d - 3] = v;
            }
        } else if (lane == 0 && G.kind == LBM_BODY_MESH) {
            double dv[3];
            swimmer_velocity_tangent(G, b->t, clamp_arc(G, (double)x - b->X[0]), dv);
            for (int k = 0; k < 3; ++k) tb[k] = (double)ub[1] * dv[k];
            // the head frame: U0 e_x + rate(x - X0) e_y
            gb[0] = (double)ub[1] * swimmer_rate_dX(G, b->t, (double)x - b->X[0]);
            gb[3] = (double)ub[0];
        } else if (lane == 0 && G.kind == LBM_BODY_SPHERE) {
            for (int a = 0; a < 3; ++a) gb[3 + a] = (double)ub[a];  // the refill velocity is U
        } else if (lane == 0 && G.kind == LBM_BODY_AIRFOIL) {
            double dX1[2], dU1[2];
            airfoil_plunge_tangent(G, b->t, dX1, dU1);
            for (int k = 0; k < 2; ++k) tb[k] = (double)ub[1] * dU1[k];
        }
        if (lane == 0)
            for (int k = 0; k < 3; ++k) tslots[(size_t)upos[slot] * 6 + 3 + k] += tb[k];
        // the free body's state through the refill velocity
        if (lane == 0 && bslot)
            for (int d = 0; d < 6; ++d) bslot[(size_t)upos[slot] * BODY_SLOTS + 6 + d] = gb[d];
        __syncwarp();
    }
}

// theta-tangents of every mesh vertex at the pose of body state b[j]: dy/dtheta
// (position) and the central difference of it (velocity), 3 + 3 per vertex,
// into dy[j] / dvy[j], for the steps j = blockIdx.y of a recomputed segment
// at once.  One warp per block: the FP64 arithmetic spread over as many SMs
// as there are warps, not over the few schedulers of a handful of large
// blocks.
constexpr int TANGENT_THREADS = 32;
__global__ void __launch_bounds__(TANGENT_THREADS) vertex_tangent_kernel(const GeomParams G, const DevBody *__restrict__ b,
                                                                         double *const *__restrict__ dy,
                                                                         double *const *__restrict__ dvy)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (v >= G.n_vertices) return;
    const double s = G.mesh_rest[3 * v], t = b[j].t;
    swimmer_midline_tangent(G, s, t, dy[j] + 3 * (size_t)v);
    swimmer_velocity_tangent(G, t, s, dvy[j] + 3 * (size_t)v);
}

// One reversed step of the free body's state (explicit Euler, Sec. 4.3, on
// the free degrees: X' = X + U, U' = U + F/m; yaw: psi' = psi + omega,
// L' = L + M_z, omega = L / I(tau)).  The step's geometry gives g over
// (X_x, X_y, psi, U_x, U_y, omega) (sum of the band slots, fixed order; the
// slots are cleared for the next step), then per free axis
// a_X = g_X + a_X', a_U = g_U + a_X' + a_U' and the force of the step
// reversed next weighs w/T + a_U/m; with yaw free a_omega = g_omega + a_psi',
// a_psi = g_psi + a_psi', a_L = a_omega / I + a_L', the torque of the step
// reversed next weighs a_L, and theta reaches omega through I(theta):
// dJ/dtheta += a_omega (-omega / I) dI/dtheta.
__global__ void __launch_bounds__(256) body_reduce_kernel(double *__restrict__ slots, int nslots,
                                                          BodyAdjoint *__restrict__ badj, const GeomParams G,
                                                          const DevBody *__restrict__ b,
                                                          const ComTangents *__restrict__ ct, double wx, double wy,
                                                          double wz)
{
    __shared__ double sm[256][6];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int s = threadIdx.x; s < nslots; s += 256) {
        double *p = slots + (size_t)s * BODY_SLOTS;
        for (int d = 0; d < 6; ++d) {
            v[d] += p[d] + p[6 + d];
            p[d] = p[6 + d] = 0.0;
        }
    }
    for (int d = 0; d < 6; ++d) sm[threadIdx.x][d] = v[d];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int d = 0; d < 6; ++d) sm[threadIdx.x][d] += sm[threadIdx.x + h][d];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double *g = sm[0];
    const double w[3] = {wx, wy, wz};
    if (G.kind == LBM_BODY_SPHERE) {
        // the free sphere (Sec. 4.1): X' = X + U, U' = U + F/m + (1 - rho_f/rho_s) g on all axes
        for (int a = 0; a < 3; ++a) {
            const double aX = g[a] + badj->aX[a];
            const double aU = g[3 + a] + badj->aX[a] + badj->aU[a];
            badj->aX[a] = aX;
            badj->aU[a] = aU;
            badj->fw[a] = w[a] + aU * G.inv_mass;
        }
        return;
    }
    for (int a = 0; a < 2; ++a) {
        if (!(G.free_motion & (1 << a))) continue;
        const double aX = g[a] + badj->aX[a];
        const double aU = g[3 + a] + badj->aX[a] + badj->aU[a];
        badj->aX[a] = aX;
        badj->aU[a] = aU;
        badj->fw[a] = w[a] + aU * G.inv_mass;
    }
    if (G.com_frame && (G.free_motion & 4)) {
        const double aw = g[5] + badj->aPsi;
        badj->aPsi = g[2] + badj->aPsi;
        badj->aL = aw / b->Izz + badj->aL;
        badj->mw = badj->aL;
        for (int k = 0; k < 3; ++k) badj->dth[k] += aw * (-b->omega / b->Izz) * ct->dI[k];
    }
}

// The free yaw's initial angular momentum L^0 = I(t0; theta) omega_0 (set when
// the geometry is given) also moves with theta: dJ/dtheta += a_L omega_0 dI/dtheta
// with a_L the adjoint of L after the first step, dI at the initial pose.
__global__ void initial_spin_kernel(BodyAdjoint *__restrict__ badj, const DevBody *__restrict__ b0,
                                    const ComTangents *__restrict__ ct)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int k = 0; k < 3; ++k) badj->dth[k] += badj->aL * b0->omega * ct->dI[k];
}

// acc[k] = sum over band slots of slot[6 s + k] + slot[6 s + 3 + k], fixed
// order (the slots hold each band position's sums over all reversed steps:
// one writer per slot and step, so the totals do not depend on timing)
__global__ void __launch_bounds__(256) theta_reduce_kernel(const double *__restrict__ slots, int nslots,
                                                            double *__restrict__ acc)
{
    __shared__ double sm[256][3];
    double v[3] = {0, 0, 0};
    for (int s = threadIdx.x; s < nslots; s += 256)
        for (int k = 0; k < 3; ++k) v[k] += slots[(size_t)s * 6 + k] + slots[(size_t)s * 6 + 3 + k];
    for (int k = 0; k < 3; ++k) sm[threadIdx.x][k] = v[k];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int k = 0; k < 3; ++k) sm[threadIdx.x][k] += sm[threadIdx.x + h][k];
        __syncthreads();
    }
    if (threadIdx.x < 3) acc[threadIdx.x] = sm[0][threadIdx.x];
}

// lambda(S^0): the transpose of step 0's pull and band contributions, zero at
// nodes refilled in step 0
template <typename R>
__global__ void lambda0_kernel(const Lattice L, const GeomParams G, const NextAdj<R> A, R *__restrict__ out)
{
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    const int x = (int)(n % L.nx), y = (int)((n / L.nx) % L.ny), z = (int)(n / ((long long)L.nx * L.ny));
    for (int i = 0; i < Q; ++i) out[(size_t)i * (size_t)L.N + n] = next_adjoint<R>(L, G, A, x, y, z, (int)n, i);
}

// per-block partial sums of lambda_T . f over nodes fluid at the end
template <typename S>
__global__ void __launch_bounds__(256) terminal_kernel(const Lattice L, const S *__restrict__ f,
                                                        const typename Codec<S>::R *__restrict__ lamT,
                                                        const uint8_t *__restrict__ flags, double *__restrict__ part)
{
    __shared__ double sm[256];
    double acc = 0;
    for (long long n = blockIdx.x * 256LL + threadIdx.x; n < L.N; n += (long long)gridDim.x * 256) {
        if (flags && (flags[n] & FL_SOLID)) continue;
        for (int i = 0; i < Q; ++i) {
            const size_t k = (size_t)i * (size_t)L.N + n;
            acc += (double)lamT[k] * ((double)Codec<S>::load(f + k) + weight<double>(i) * L.rho0);
        }
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

}  // namespace lbm

// ----------------------------------------------------------------- driver
using namespace lbm;

namespace {

lbm_status afail(lbm_ctx *c, lbm_status st, const std::string &msg)
{
    if (c) c->err = msg;
    return st;
}

#define ADJ_CUDA(call, where)                                                                           \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            st = afail(ctx, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e_));          \
            goto done;                                                                                  \
        }                                                                                               \
    } while (0)

// device buffers of one adjoint call (through the context's allocator),
// released together once the context's streams are idle
struct AdjBuffers {
    lbm_ctx *ctx;
    std::vector<void *> ptrs;
    explicit AdjBuffers(lbm_ctx *c) : ctx(c) {}
    template <typename T>
    bool get(T **p, size_t count)
    {
        void *v = nullptr;
        if (ctx_malloc(ctx, &v, count * sizeof(T)) != cudaSuccess) {
            *p = nullptr;
            return false;
        }
        ptrs.push_back(v);
        *p = static_cast<T *>(v);
        return true;
    }
    ~AdjBuffers()
    {
        if (!ptrs.empty()) {
            cudaStreamSynchronize(ctx->stream);
            cudaStreamSynchronize(ctx->side);
        }
        for (void *p : ptrs) ctx_release(ctx, p);
    }
};

// one forward step from fa into fb with the context's body scratch and the
// given marks (the launch sequences of lbm_step; the force reduction only for
// a free body, whose next pose needs it)
cudaError_t forward_step(lbm_ctx *ctx, void *fa, void *fb, uint8_t *flags)
{
    int nl = 0;
    cudaError_t e;
    const uint8_t *fl = ctx->has_body ? flags : nullptr;
    int cur = ctx->bcur;
    int *status = &ctx->S.body[cur].status;
    if (ctx->has_body && sweep_ahead(ctx->G) && ctx->order != ORDER_SEQUENTIAL) {
        // split order, as in lbm_step: the nodes outside the sweep box beside
        // the body's geometry, refill, boundary nodes and the box's nodes
        const int prev = ctx->bcur;
        cur = prev ^ 1;
        status = &ctx->S.body[cur].status;
        const int *sweep = ctx->S.body[prev].sweep;
        if ((e = cudaEventRecord(ctx->ev_fork, ctx->stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0)) != cudaSuccess ||
            (e = launch_geometry(ctx->L, ctx->G, ctx->S, prev, flags, ctx->side, &nl)) != cudaSuccess ||
            (e = launch_refill(ctx->storage, ctx->L, ctx->G, ctx->S, cur, fa, flags, ctx->side)) != cudaSuccess ||
            (e = launch_boundary(ctx->storage, ctx->L, ctx->G, ctx->S, cur, fa, fb, flags, ctx->side)) !=
                cudaSuccess ||
            (ctx->G.free_motion && (e = launch_forces(ctx->G, ctx->S, cur, ctx->side, &nl)) != cudaSuccess) ||
            (e = launch_bulk(ctx->storage, ctx->L, fa, fb, flags, status, ctx->side, BULK_BAND, sweep, ctx->G.cap)) !=
                cudaSuccess ||
            (e = cudaEventRecord(ctx->ev_join, ctx->side)) != cudaSuccess ||
            (e = launch_bulk(ctx->storage, ctx->L, fa, fb, nullptr, status, ctx->stream, BULK_OUTSIDE, sweep)) !=
                cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0)) != cudaSuccess)
            return e;
        ctx->bcur = cur;
        return cudaSuccess;
    }
    if (ctx->has_body) {
        const int prev = ctx->bcur;
        cur = prev ^ 1;
        status = &ctx->S.body[cur].status;
        if ((e = launch_geometry(ctx->L, ctx->G, ctx->S, prev, flags, ctx->stream, &nl)) != cudaSuccess) return e;
        if ((e = launch_refill(ctx->storage, ctx->L, ctx->G, ctx->S, cur, fa, flags, ctx->stream)) != cudaSuccess)
            return e;
        // boundary nodes beside the bulk kernel, as in lbm_step
        if ((e = cudaEventRecord(ctx->ev_fork, ctx->stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0)) != cudaSuccess) return e;
        if ((e = launch_boundary(ctx->storage, ctx->L, ctx->G, ctx->S, cur, fa, fb, flags, ctx->side)) != cudaSuccess)
            return e;
        if (ctx->G.free_motion && (e = launch_forces(ctx->G, ctx->S, cur, ctx->side, &nl)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(ctx->ev_join, ctx->side)) != cudaSuccess) return e;
    }
    if ((e = launch_bulk(ctx->storage, ctx->L, fa, fb, fl, status, ctx->stream)) != cudaSuccess) return e;
    if (ctx->has_body && (e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0)) != cudaSuccess) return e;
    ctx->bcur = cur;
    return cudaSuccess;
}

// Grid of the boundary and refill adjoints: one warp per listed node, at most
// LBM_ADJ_LIST_BLOCKS blocks (a build-time override, as the forward list
// kernels' LBM_LIST_BLOCKS)
#ifndef LBM_ADJ_LIST_BLOCKS
#define LBM_ADJ_LIST_BLOCKS 1216
#endif

int list_blocks(int cap)
{
    int nb = (cap + BWARPS - 1) / BWARPS;
    return nb < 1 ? 1 : (nb > LBM_ADJ_LIST_BLOCKS ? LBM_ADJ_LIST_BLOCKS : nb);
}

// the reverse of step t for storage type S.  The caller has put step t's
// geometry in place: the body state of step t in S.body[0], the one its
// geometry gave in S.body[1], its marks in flags1 and its lists and mesh
// arrays in the context's scratch.  Sequential order: the caller has also
// cleared ext.  Split order (split, a band known ahead): the boundary and
// refill adjoints and the bulk adjoint over the two steps' bands run on the
// side stream, beside the bulk adjoint of the nodes outside them.
template <typename S>
cudaError_t reverse_step(lbm_ctx *ctx, const S *st, const NextAdj<typename Codec<S>::R> &A, uint8_t *flags1,
                         typename Codec<S>::R *lam_out, double *ext, double *tslots, BodyAdjoint *badj,
                         double *bslot, double wx, double wy, double wz, ComTangents *ct, double *cpart,
                         unsigned *cticket, bool split)
{
    using R = typename Codec<S>::R;
    const Lattice &L = ctx->L;
    const GeomParams &G = ctx->G;
    Scratch &Sc = ctx->S;
    cudaStream_t s = ctx->stream;
    cudaStream_t side = ctx->side;
    cudaError_t e;
    const int bx = L.nx >= 128 ? 128 : ((L.nx + 31) / 32) * 32;
    dim3 grid((L.nx + bx - 1) / bx, L.ny, L.nz);
    if (split) {
        // band of step t (stored with state t) and of step t+1 (A.band)
        const int *box0 = (const int *)((const char *)(Sc.body + 0) + offsetof(DevBody, sweep));
        const int *box1 = A.band ? (const int *)((const char *)A.band + offsetof(DevBody, band_lo)) : nullptr;
        const DevBody *b = Sc.body + 1;
        const int capv = G.cap[0] * G.cap[1] * G.cap[2];
        const unsigned nbb = (unsigned)((capv + 127) / 128);
        if ((e = cudaEventRecord(ctx->ev_fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, ctx->ev_fork, 0)) != cudaSuccess) return e;
        ctx->bcur = 1;
        if ((e = cudaMemsetAsync(ext, 0, (size_t)capv * Q * sizeof(double), side)) != cudaSuccess) return e;
        adjoint_boundary_kernel<S><<<list_blocks(G.cap_boundary), BWARPS * 32, 0, side>>>(
            L, G, b, Sc.blist, Sc.bpos, st, A, flags1, lam_out, ext, tslots, badj, bslot, ct);
        adjoint_bulk_kernel<S><<<nbb, 128, 0, side>>>(L, G, st, A, flags1, lam_out, BULK_BAND, box0, nullptr);
        if (box1)
            adjoint_bulk_kernel<S><<<nbb, 128, 0, side>>>(L, G, st, A, flags1, lam_out, BULK_BAND, box1, box0);
        adjoint_refill_kernel<S><<<list_blocks(G.cap_uncovered), BWARPS * 32, 0, side>>>(
            L, G, b, Sc.ulist, Sc.upos, st, lam_out, flags1, ext, tslots, bslot, ct);
        if (bslot) body_reduce_kernel<<<1, 256, 0, side>>>(bslot, capv, badj, G, b, ct, wx, wy, wz);
        if ((e = cudaEventRecord(ctx->ev_join, side)) != cudaSuccess) return e;
        adjoint_bulk_kernel<S><<<grid, bx, 0, s>>>(L, G, st, A, nullptr, lam_out, BULK_OUTSIDE, box0, box1);
        if ((e = cudaStreamWaitEvent(s, ctx->ev_join, 0)) != cudaSuccess) return e;
        return cudaGetLastError();
    }
    const DevBody *b = Sc.body + ctx->bcur;
    // the boundary adjoint runs beside the bulk adjoint (disjoint rows of Lam^t)
    if (ctx->has_body) {
        if (G.kind == LBM_BODY_MESH && G.com_frame)
            com_tangent_kernel<<<(G.n_triangles + 255) / 256, 256, 0, s>>>(G, b, cpart, cticket, ct);
        if ((e = cudaEventRecord(ctx->ev_fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, ctx->ev_fork, 0)) != cudaSuccess) return e;
        adjoint_boundary_kernel<S><<<list_blocks(G.cap_boundary), BWARPS * 32, 0, side>>>(
            L, G, b, Sc.blist, Sc.bpos, st, A, flags1, lam_out, ext, tslots, badj, bslot, ct);
        if ((e = cudaEventRecord(ctx->ev_join, side)) != cudaSuccess) return e;
    }
    adjoint_bulk_kernel<S><<<grid, bx, 0, s>>>(L, G, st, A, ctx->has_body ? flags1 : nullptr, lam_out, BULK_ALL,
                                               nullptr, nullptr);
    if (ctx->has_body) {
        if ((e = cudaStreamWaitEvent(s, ctx->ev_join, 0)) != cudaSuccess) return e;
        adjoint_refill_kernel<S><<<list_blocks(G.cap_uncovered), BWARPS * 32, 0, s>>>(
            L, G, b, Sc.ulist, Sc.upos, st, lam_out, flags1, ext, tslots, bslot, ct);
        if (bslot)
            body_reduce_kernel<<<1, 256, 0, s>>>(bslot, G.cap[0] * G.cap[1] * G.cap[2], badj, G, b, ct, wx, wy, wz);
    }
    return cudaGetLastError();
}

// The arrays a step's geometry writes and the later kernels of that step (and
// of its reverse) read: the boundary and uncovered lists and, for the mesh,
// the pose and the column and cell lists.  The recompute pass gives every
// step of a segment a slot of its own, so the reversed step finds its
// geometry there instead of running it again.
struct GeoSlot {
    int *blist = nullptr, *bpos = nullptr, *ulist = nullptr, *upos = nullptr;
    double *mesh_pos = nullptr, *mesh_vel = nullptr, *col_x = nullptr;
    int *mesh_ipos = nullptr, *col_count = nullptr, *cell_count = nullptr, *cell_tri = nullptr;
    float *mesh_frac = nullptr, *tri_box = nullptr;
    double *tan_dy = nullptr, *tan_dvy = nullptr;  // the vertices' theta-tangents at the step's pose
};

static GeoSlot live_slot(const lbm_ctx *ctx)
{
    GeoSlot g;
    g.blist = ctx->S.blist;
    g.bpos = ctx->S.bpos;
    g.ulist = ctx->S.ulist;
    g.upos = ctx->S.upos;
    g.mesh_pos = ctx->S.mesh_pos;
    g.mesh_vel = ctx->S.mesh_vel;
    g.col_x = ctx->S.col_x;
    g.mesh_ipos = ctx->S.mesh_ipos;
    g.col_count = ctx->S.col_count;
    g.cell_count = ctx->S.cell_count;
    g.cell_tri = ctx->S.cell_tri;
    g.mesh_frac = ctx->S.mesh_frac;
    g.tri_box = ctx->S.tri_box;
    return g;
}

// points the context's scratch (and the geometry parameters' copies of the
// mesh arrays) at a slot
static void use_slot(lbm_ctx *ctx, const GeoSlot &g)
{
    Scratch &S = ctx->S;
    GeomParams &G = ctx->G;
    S.blist = g.blist;
    S.bpos = g.bpos;
    S.ulist = g.ulist;
    S.upos = g.upos;
    if (G.kind != LBM_BODY_MESH) return;
    S.mesh_pos = G.mesh_pos = g.mesh_pos;
    S.mesh_vel = G.mesh_vel = g.mesh_vel;
    S.col_x = G.col_x = g.col_x;
    S.mesh_ipos = G.mesh_ipos = g.mesh_ipos;
    S.col_count = G.col_count = g.col_count;
    S.cell_count = G.cell_count = g.cell_count;
    S.cell_tri = G.cell_tri = g.cell_tri;
    S.mesh_frac = G.mesh_frac = g.mesh_frac;
    S.tri_box = G.tri_box = g.tri_box;
    G.mesh_dy = g.tan_dy;
    G.mesh_dvy = g.tan_dvy;
}

template <typename S>
lbm_status adjoint_run(lbm_ctx *ctx, const lbm_adjoint *spec, double *J, double dJ[3])
{
    using R = typename Codec<S>::R;
    const Lattice &L = ctx->L;
    const size_t N = (size_t)L.N;
    const size_t state = 27 * N;
    const int T = spec->horizon;
    int K = spec->checkpoint_every > 0 ? spec->checkpoint_every : (int)std::ceil(std::sqrt((double)T));
    if (K > T) K = T;
    const int nseg = (T + K - 1) / K;
    const bool body = ctx->has_body;
    const int cap = body ? ctx->G.cap[0] * ctx->G.cap[1] * ctx->G.cap[2] : 1;
    cudaStream_t s = ctx->stream;
    lbm_status st = LBM_OK;
    AdjBuffers B(ctx);
    S *ck = nullptr, *seg = nullptr;
    uint8_t *ckflags = nullptr, *segflags = nullptr, *wf[2] = {nullptr, nullptr}, *wrec = nullptr;
    DevBody *ckbody = nullptr, *segbody = nullptr, *adjbody = nullptr, *savebody = nullptr;
    R *lam[2] = {nullptr, nullptr};
    double *ext[2] = {nullptr, nullptr}, *tslots = nullptr, *acc = nullptr, *part = nullptr;
    double *tan_dy = nullptr, *tan_dvy = nullptr;
    double F0[3] = {0, 0, 0}, F1[3] = {0, 0, 0}, accv[3] = {0, 0, 0};
    // the swimmer free along x carries (X0, U0) as adjoint state
    const bool free_body = ctx->has_body && ctx->G.free_motion != 0;
    const BodyAdjoint badj0{{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, 0.0, 0.0,
                            {spec->w_force[0] / T, spec->w_force[1] / T, spec->w_force[2] / T}, 0.0, {0.0, 0.0, 0.0}};
    BodyAdjoint *badj = nullptr;
    double *bslot = nullptr;
    const bool com = free_body && ctx->G.kind == LBM_BODY_MESH && ctx->G.com_frame;
    // reverse steps in the split order when the band is known ahead
    const bool split = body && sweep_ahead(ctx->G) && ctx->order != ORDER_SEQUENTIAL;
    ComTangents *ct = nullptr;
    double *cpart = nullptr;
    unsigned *cticket = nullptr;
    BodyAdjoint hbadj{};
    DevBody hb{};
    int p = 0;
    const int save_bcur = ctx->bcur;
    const int nparts = 1024;
    double Jt = 0.0;

    if (!B.get(&ck, (size_t)nseg * state) || !B.get(&seg, (size_t)(K + 1) * state) ||
        !B.get(&ckflags, (size_t)nseg * N) || !B.get(&segflags, (size_t)(K + 1) * N) || !B.get(&wf[0], N) ||
        !B.get(&wf[1], N) || !B.get(&wrec, N) || !B.get(&ckbody, nseg) || !B.get(&segbody, K + 1) ||
        !B.get(&adjbody, 2) ||
        !B.get(&savebody, 2) || !B.get(&lam[0], state) || !B.get(&lam[1], state) ||
        !B.get(&ext[0], (size_t)cap * Q) || !B.get(&ext[1], (size_t)cap * Q) || !B.get(&tslots, (size_t)cap * 6) ||
        !B.get(&acc, 3) || !B.get(&part, nparts) || !B.get(&badj, 1) ||
        (free_body && !B.get(&bslot, (size_t)cap * BODY_SLOTS)) ||
        (com && (!B.get(&ct, 1) || !B.get(&cpart, (size_t)((ctx->G.n_triangles + 255) / 256) * COM_SUMS) ||
                 !B.get(&cticket, 1))) ||
        (body && ctx->G.kind == LBM_BODY_MESH &&
         (!B.get(&tan_dy, 3 * (size_t)ctx->G.n_vertices) || !B.get(&tan_dvy, 3 * (size_t)ctx->G.n_vertices))))
        return afail(ctx, LBM_ERR_OOM, "lbm_adjoint_step: device allocation of the checkpoints failed");
    // a geometry slot per step of a segment (see GeoSlot)
    const GeoSlot live = live_slot(ctx);
    std::vector<GeoSlot> slots(body ? K : 0);
    if (body) {
        const GeomParams &G = ctx->G;
        const size_t nv = (size_t)G.n_vertices, nt = (size_t)G.n_triangles;
        const size_t ncols = (size_t)G.cap[1] * G.cap[2], ncells = (size_t)G.cells[0] * G.cells[1] * G.cells[2];
        for (GeoSlot &g : slots) {
            bool ok = B.get(&g.blist, (size_t)G.cap_boundary) && B.get(&g.bpos, (size_t)G.cap_boundary) &&
                      B.get(&g.ulist, (size_t)G.cap_uncovered) && B.get(&g.upos, (size_t)G.cap_uncovered);
            if (ok && G.kind == LBM_BODY_MESH)
                ok = B.get(&g.mesh_pos, 3 * nv) && B.get(&g.mesh_vel, 3 * nv) && B.get(&g.mesh_ipos, 3 * nv) &&
                     B.get(&g.mesh_frac, 3 * nv) && B.get(&g.tri_box, 6 * nt) && B.get(&g.col_count, ncols) &&
                     B.get(&g.col_x, ncols * MESH_COL_CAP) && B.get(&g.cell_count, ncells) &&
                     B.get(&g.cell_tri, ncells * MESH_CELL_CAP) && B.get(&g.tan_dy, 3 * nv) &&
                     B.get(&g.tan_dvy, 3 * nv);
            if (!ok)
                return afail(ctx, LBM_ERR_OOM, "lbm_adjoint_step: device allocation of the geometry slots failed");
        }
    }
    // the slots' tangent arrays for the batched vertex tangents of a segment
    double **tanp = nullptr;
    if (body && ctx->G.kind == LBM_BODY_MESH) {
        if (!B.get(&tanp, 2 * (size_t)K))
            return afail(ctx, LBM_ERR_OOM, "lbm_adjoint_step: device allocation of the geometry slots failed");
        std::vector<double *> hp(2 * (size_t)K);
        for (int j = 0; j < K; ++j) {
            hp[j] = slots[j].tan_dy;
            hp[K + j] = slots[j].tan_dvy;
        }
        if (cudaMemcpy(tanp, hp.data(), hp.size() * sizeof(double *), cudaMemcpyHostToDevice) != cudaSuccess)
            return afail(ctx, LBM_ERR_CUDA, "lbm_adjoint_step: slot table upload failed");
    }
    ctx->G.mesh_dy = tan_dy;
    ctx->G.mesh_dvy = tan_dvy;

    // ---- forward over the horizon with checkpoints
    ADJ_CUDA(cudaMemcpyAsync(&hb, ctx->S.body + ctx->bcur, sizeof(DevBody), cudaMemcpyDeviceToHost, s), "body read");
    ADJ_CUDA(cudaStreamSynchronize(s), "sync");
    for (int a = 0; a < 3; ++a) F0[a] = hb.F_sum[a];
    for (int t = 0; t < T; ++t) {
        if (t % K == 0) {
            const int k = t / K;
            ADJ_CUDA(cudaMemcpyAsync(ck + (size_t)k * state, ctx->f[ctx->cur], state * sizeof(S),
                                     cudaMemcpyDeviceToDevice, s), "checkpoint");
            ADJ_CUDA(cudaMemcpyAsync(ckflags + (size_t)k * N, ctx->flags, N, cudaMemcpyDeviceToDevice, s), "checkpoint");
            ADJ_CUDA(cudaMemcpyAsync(ckbody + k, ctx->S.body + ctx->bcur, sizeof(DevBody), cudaMemcpyDeviceToDevice, s),
                     "checkpoint");
        }
        st = lbm_step(ctx, 1);
        if (st != LBM_OK) goto done;
    }
    ADJ_CUDA(cudaMemcpyAsync(&hb, ctx->S.body + ctx->bcur, sizeof(DevBody), cudaMemcpyDeviceToHost, s), "body read");
    ADJ_CUDA(cudaMemcpyAsync(savebody, ctx->S.body, 2 * sizeof(DevBody), cudaMemcpyDeviceToDevice, s), "body save");
    if (spec->lambda_T) {
        terminal_kernel<S><<<nparts, 256, 0, s>>>(L, (const S *)ctx->f[ctx->cur], (const R *)spec->lambda_T,
                                                  body ? ctx->flags : nullptr, part);
        std::vector<double> hp(nparts);
        ADJ_CUDA(cudaMemcpyAsync(hp.data(), part, nparts * sizeof(double), cudaMemcpyDeviceToHost, s), "terminal");
        ADJ_CUDA(cudaStreamSynchronize(s), "sync");
        for (int k = 0; k < nparts; ++k) Jt += hp[k];
    }
    ADJ_CUDA(cudaStreamSynchronize(s), "sync");
    if (hb.status & ST_UNSTABLE) {
        st = afail(ctx, LBM_ERR_UNSTABLE, "lbm_adjoint_step: a node went unstable in the forward run");
        goto done;
    }
    for (int a = 0; a < 3; ++a) F1[a] = hb.F_sum[a];
    *J = Jt;
    for (int a = 0; a < 3; ++a) *J += spec->w_force[a] * (F1[a] - F0[a]) / T;

    // ---- reverse sweep, one recomputed segment at a time
    ADJ_CUDA(cudaMemsetAsync(acc, 0, 3 * sizeof(double), s), "clear");
    ADJ_CUDA(cudaMemsetAsync(tslots, 0, (size_t)cap * 6 * sizeof(double), s), "clear");
    ADJ_CUDA(cudaMemcpyAsync(badj, &badj0, sizeof(BodyAdjoint), cudaMemcpyHostToDevice, s), "body adjoint");
    if (bslot) ADJ_CUDA(cudaMemsetAsync(bslot, 0, (size_t)cap * BODY_SLOTS * sizeof(double), s), "clear");
    if (cticket) ADJ_CUDA(cudaMemsetAsync(cticket, 0, sizeof(unsigned), s), "clear");
    {
        bool first = true;
        for (int sg = nseg - 1; sg >= 0; --sg) {
            NvtxRange nvtx_seg("adjoint segment");  // its recompute and its reversed steps
            const int t0 = sg * K, t1 = std::min(T, t0 + K);
            // recompute the segment: seg[j] holds St^{t0+j} once step t0+j has run
            ADJ_CUDA(cudaMemcpyAsync(seg, ck + (size_t)sg * state, state * sizeof(S), cudaMemcpyDeviceToDevice, s),
                     "restore");
            ADJ_CUDA(cudaMemcpyAsync(wrec, ckflags + (size_t)sg * N, N, cudaMemcpyDeviceToDevice, s), "restore");
            ctx->bcur = 0;
            ADJ_CUDA(cudaMemcpyAsync(ctx->S.body, ckbody + sg, sizeof(DevBody), cudaMemcpyDeviceToDevice, s), "restore");
            // segflags[j] / segbody[j]: marks and body state before step t0 + j,
            // which are also those that step t0 + j - 1's geometry left
            for (int t = t0; t <= t1; ++t) {
                const int j = t - t0;
                ADJ_CUDA(cudaMemcpyAsync(segflags + (size_t)j * N, wrec, N, cudaMemcpyDeviceToDevice, s), "seg flags");
                ADJ_CUDA(cudaMemcpyAsync(segbody + j, ctx->S.body + ctx->bcur, sizeof(DevBody), cudaMemcpyDeviceToDevice,
                                         s), "seg body");
                if (t == t1) break;
                if (body) use_slot(ctx, slots[j]);
                ADJ_CUDA(forward_step(ctx, seg + (size_t)j * state, seg + (size_t)(j + 1) * state, wrec), "recompute");
            }
            // the vertex tangents of every step of the segment at once, at the
            // pose each step's geometry left (segbody[j + 1])
            if (tanp) {
                const dim3 tg((ctx->G.n_vertices + TANGENT_THREADS - 1) / TANGENT_THREADS, t1 - t0);
                vertex_tangent_kernel<<<tg, TANGENT_THREADS, 0, s>>>(ctx->G, segbody + 1, tanp, tanp + K);
                ADJ_CUDA(cudaGetLastError(), "vertex tangents");
            }
            // reverse the segment's steps
            for (int t = t1 - 1; t >= t0; --t) {
                const int j = t - t0;
                // step t's geometry as the recompute left it: its marks, the
                // body state after it (the adjoint reads none of the force
                // fields the rest of the step wrote there) and its slot
                ADJ_CUDA(cudaMemcpyAsync(wf[p], segflags + (size_t)(j + 1) * N, N, cudaMemcpyDeviceToDevice, s),
                         "flags");
                ctx->bcur = 0;
                ADJ_CUDA(cudaMemcpyAsync(ctx->S.body, segbody + j, 2 * sizeof(DevBody), cudaMemcpyDeviceToDevice, s),
                         "body");
                if (body) use_slot(ctx, slots[j]);
                if (body && !split) {
                    ctx->bcur = 1;
                    ADJ_CUDA(cudaMemsetAsync(ext[p], 0, (size_t)cap * Q * sizeof(double), s), "clear");
                }
                NextAdj<R> A;
                if (first) {
                    A = NextAdj<R>{(const R *)spec->lambda_T, nullptr, nullptr, nullptr, 1};
                } else {
                    A = NextAdj<R>{lam[p ^ 1], body ? ext[p ^ 1] : nullptr, adjbody + (p ^ 1),
                                   body ? wf[p ^ 1] : nullptr, 0};
                }
                ADJ_CUDA(reverse_step<S>(ctx, seg + (size_t)j * state, A, wf[p], lam[p], ext[p], tslots, badj, bslot,
                                         badj0.fw[0], badj0.fw[1], badj0.fw[2], ct, cpart, cticket, split),
                         "reverse step");
                if (body)
                    ADJ_CUDA(cudaMemcpyAsync(adjbody + p, ctx->S.body + ctx->bcur, sizeof(DevBody),
                                             cudaMemcpyDeviceToDevice, s), "band");
                first = false;
                p ^= 1;
            }
        }
        // lambda(S^0) from the last reversed step (step 0)
        if (spec->lambda_0) {
            NextAdj<R> A{lam[p ^ 1], body ? ext[p ^ 1] : nullptr, adjbody + (p ^ 1), body ? wf[p ^ 1] : nullptr, 0};
            lambda0_kernel<R><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(L, ctx->G, A, (R *)spec->lambda_0);
            ADJ_CUDA(cudaGetLastError(), "lambda0");
        }
    }
    if (com && (ctx->G.free_motion & 4)) {
        com_tangent_kernel<<<(ctx->G.n_triangles + 255) / 256, 256, 0, s>>>(ctx->G, ckbody, cpart, cticket, ct);
        initial_spin_kernel<<<1, 32, 0, s>>>(badj, ckbody, ct);
    }
    if (body) theta_reduce_kernel<<<1, 256, 0, s>>>(tslots, cap, acc);
    ADJ_CUDA(cudaMemcpyAsync(accv, acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s), "theta");
    ADJ_CUDA(cudaMemcpyAsync(&hbadj, badj, sizeof(BodyAdjoint), cudaMemcpyDeviceToHost, s), "body adjoint");
    ADJ_CUDA(cudaStreamSynchronize(s), "sync");
    // plus what theta does through the free yaw's omega = L / I(theta)
    for (int k = 0; k < 3; ++k) dJ[k] = accv[k] + hbadj.dth[k];

done:
    use_slot(ctx, live);
    ctx->G.mesh_dy = nullptr;
    ctx->G.mesh_dvy = nullptr;
    // the context keeps the state after the horizon; restore its body copies
    cudaMemcpyAsync(ctx->S.body, savebody, 2 * sizeof(DevBody), cudaMemcpyDeviceToDevice, s);
    ctx->bcur = save_bcur;
    cudaStreamSynchronize(s);
    return st;
}

}  // namespace

extern "C" lbm_status lbm_adjoint_step(lbm_ctx *ctx, const lbm_adjoint *spec, double *J, double dJ_dtheta[3])
{
    NvtxRange nvtx_("lbm_adjoint_step");
    if (!ctx) return LBM_ERR_ARG;
    if (!spec || !J || !dJ_dtheta) return afail(ctx, LBM_ERR_ARG, "lbm_adjoint_step: null argument");
    if (spec->horizon < 1 || spec->checkpoint_every < 0)
        return afail(ctx, LBM_ERR_ARG, "lbm_adjoint_step: horizon >= 1 and checkpoint_every >= 0 required");
    for (int k = 0; k < 4; ++k)
        if (spec->reserved[k] != 0) return afail(ctx, LBM_ERR_ARG, "lbm_adjoint_step: reserved fields must be 0");
    if (!ctx->initialised) return afail(ctx, LBM_ERR_STATE, "lbm_adjoint_step: state not initialised");
    if (ctx->L.gamma_mode == LBM_GAMMA_EXACT)
        return afail(ctx, LBM_ERR_UNSUPPORTED, "lbm_adjoint_step: the exact stabilizer has no adjoint here");
    if (ctx->slab_zper > 0)
        return afail(ctx, LBM_ERR_UNSUPPORTED, "lbm_adjoint_step: a slab context has no adjoint here");
    for (int k = 0; k < 3; ++k) dJ_dtheta[k] = 0.0;
    *J = 0.0;
    if (drain_records(ctx) != cudaSuccess) return afail(ctx, LBM_ERR_CUDA, "lbm_adjoint_step: record copies");
    if (ctx->storage == LBM_FP64) return adjoint_run<double>(ctx, spec, J, dJ_dtheta);
    if (ctx->storage == LBM_FP32) return adjoint_run<float>(ctx, spec, J, dJ_dtheta);
    // 16-bit storage: states and checkpoints in the storage type, the adjoint
    // in FP32 (the rounding of each store passes the adjoint unchanged)
    if (ctx->storage == LBM_FP16) return adjoint_run<__half>(ctx, spec, J, dJ_dtheta);
    if (ctx->storage == LBM_BF16) return adjoint_run<__nv_bfloat16>(ctx, spec, J, dJ_dtheta);
    return afail(ctx, LBM_ERR_UNSUPPORTED, "lbm_adjoint_step: unknown storage");
}
