// KBC entropic collision of one node in shifted (deviation) form.
//
// Paper (arXiv 1608.04658) Sec. 2:
//   Eq. (kineticEq)  f' = (1 - b) f + b f^mirr
//   Eq. (kbc_relax)  f^mirr = k + (2 s^eq - s) + ((1 - g) h + g h^eq)
//                    => f' = f - b (2 ds + g dh)
//   Eq. (feq_min)    f^eq = exact D3Q27 minimiser of H (product form of
//                    Ansumali, Karlin, Oettinger 2003):
//                    f_i^eq = rho prod_a w(c_ia) (2 - S_a) B_a^{c_ia},
//                    S = sqrt(1 + 3 u^2), B = (2u + S)/(1 - u)
//   analytic stabilizer g = 1/b - (2 - 1/b) <ds|dh>/<dh|dh>, <X|Y> = sum X Y / f^eq
//
// Arithmetic is arranged so that FP32 keeps the precision of the small
// deviations: populations are carried as g_i = f_i - W_i rho0, and each 1-D
// equilibrium factor is written as w(c) (1 + e(c)) with e small:
//   sigma = S - 1 = 3u^2 / (S + 1),  2 - S = 1 - sigma,
//   B - 1 = (3u + sigma)/(1 - u),    1/B - 1 = -(3u + sigma)/(2u + S),
//   e(0) = -sigma,  e(+1) = (B-1)(1-sigma) - sigma,  e(-1) = (1/B-1)(1-sigma) - sigma,
// so g_i^eq = W_i (rho - rho0 + rho E_i) with E_i = prod_a (1 + e_a) - 1 formed
// without cancellation.  The KBC shear part ds (deviatoric natural second
// moments, trace left in h) expands on the D3Q27 directions to
//   +-x faces (2 N_xz - N_yz)/6, +-y faces (2 N_yz - N_xz)/6,
//   +-z faces -(N_xz + N_yz)/6, edges c_a c_b P_ab / 4, rest and corners 0,
// with N_xz = P_xx - P_zz, N_yz = P_yy - P_zz, P the second moments of df.
// The update is written g'_i = g_i^eq + (1 - b g) df_i + b (g - 2) ds_i.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

template <typename R> __device__ __forceinline__ R gamma_floor();
template <> __device__ __forceinline__ float gamma_floor<float>() { return 1e-30f; }
template <> __device__ __forceinline__ double gamma_floor<double>() { return 1e-300; }

// e(-1), e(0), e(+1) and 1/(1 + e) for one axis.
template <typename R>
__device__ __forceinline__ void axis_eq(R u, R e[3], R r[3])
{
    const R u2 = u * u;
    const R S = sqrt(R(1) + R(3) * u2);
    const R sig = R(3) * u2 / (S + R(1));
    const R a = R(3) * u + sig;
    const R oms = R(1) - sig;
    const R bp = a / (R(1) - u);
    const R bm = -a / (R(2) * u + S);
    e[0] = bm * oms - sig;
    e[1] = -sig;
    e[2] = bp * oms - sig;
    r[0] = R(1) / (R(1) + e[0]);
    r[1] = R(1) / oms;
    r[2] = R(1) / (R(1) + e[2]);
}

// Shear part ds_i for direction i from N_xz, N_yz and the off-diagonal P.
template <typename R>
__device__ __forceinline__ R shear_part(int i, R nxz, R nyz, R pxy, R pxz, R pyz)
{
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    const int nz = nonzero_of(i);
    if (nz == 1) {
        if (cx) return (R(2) * nxz - nyz) * R(1.0 / 6.0);
        if (cy) return (R(2) * nyz - nxz) * R(1.0 / 6.0);
        return -(nxz + nyz) * R(1.0 / 6.0);
    }
    if (nz == 2) {
        if (cz == 0) return R(cx * cy) * pxy * R(0.25);
        if (cy == 0) return R(cx * cz) * pxz * R(0.25);
        return R(cy * cz) * pyz * R(0.25);
    }
    return R(0);
}

// In-place collision of the 27 shifted populations g[] of one node.
// Returns false when the density is not finite and positive.
template <typename R>
__device__ __forceinline__ bool kbc_collide(R g[Q], R beta, R rho0, int gamma_mode)
{
    R drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += g[i];
        if (cx_of(i) > 0) jx += g[i]; else if (cx_of(i) < 0) jx -= g[i];
        if (cy_of(i) > 0) jy += g[i]; else if (cy_of(i) < 0) jy -= g[i];
        if (cz_of(i) > 0) jz += g[i]; else if (cz_of(i) < 0) jz -= g[i];
    }
    const R rho = rho0 + drho;
    const bool ok = rho > R(0) && rho < R(1e30);
    const R inv_rho = R(1) / rho;
    R ex[3], ey[3], ez[3], rx[3], ry[3], rz[3];
    axis_eq(jx * inv_rho, ex, rx);
    axis_eq(jy * inv_rho, ey, ry);
    axis_eq(jz * inv_rho, ez, rz);

    // df_i = g_i - g_i^eq (stored in g), and the second moments of df
    R pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        const R exy = ex[cx + 1] + ey[cy + 1] + ex[cx + 1] * ey[cy + 1];
        const R E = exy + ez[cz + 1] + exy * ez[cz + 1];
        const R geq = weight<R>(i) * (drho + rho * E);
        const R d = g[i] - geq;
        g[i] = d;
        if (cx) pxx += d;
        if (cy) pyy += d;
        if (cz) pzz += d;
        if (cx && cy) pxy += R(cx * cy) * d;
        if (cx && cz) pxz += R(cx * cz) * d;
        if (cy && cz) pyz += R(cy * cz) * d;
    }
    const R nxz = pxx - pzz, nyz = pyy - pzz;

    // entropic scalar products <ds|dh>, <dh|dh> with 1/f^eq = 1/(rho W) prod r
    R sh = 0, hh = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        const R ifeq = inv_rho * inv_weight<R>(i) * rx[cx + 1] * ry[cy + 1] * rz[cz + 1];
        const R ds = shear_part<R>(i, nxz, nyz, pxy, pxz, pyz);
        const R dh = g[i] - ds;
        sh += ds * dh * ifeq;
        hh += dh * dh * ifeq;
    }
    R gam = R(2);
    if (gamma_mode == LBM_GAMMA_ANALYTIC && hh > gamma_floor<R>()) {
        const R ib = R(1) / beta;
        gam = ib - (R(2) - ib) * sh / hh;
    }
    const R c1 = R(1) - beta * gam;
    const R c2 = beta * (gam - R(2));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        const R exy = ex[cx + 1] + ey[cy + 1] + ex[cx + 1] * ey[cy + 1];
        const R E = exy + ez[cz + 1] + exy * ez[cz + 1];
        const R geq = weight<R>(i) * (drho + rho * E);
        const R ds = shear_part<R>(i, nxz, nyz, pxy, pxz, pyz);
        g[i] = geq + c1 * g[i] + c2 * ds;
    }
    return ok;
}

// Equilibrium in shifted form, g_i^eq = f_i^eq(rho, u) - W_i rho0.
template <typename R>
__device__ __forceinline__ R shifted_feq(int i, R drho, R rho, const R ex[3], const R ey[3],
                                         const R ez[3])
{
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    const R exy = ex[cx + 1] + ey[cy + 1] + ex[cx + 1] * ey[cy + 1];
    const R E = exy + ez[cz + 1] + exy * ez[cz + 1];
    return weight<R>(i) * (drho + rho * E);
}

}  // namespace lbm
