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
//   B - 1 = (3u + sigma)/(1 - u),    1/B - 1 = -(B - 1)/B,
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

// correctly rounded reciprocal and square root of the arithmetic type
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_rn(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ double sqrt_rn(double x) { return sqrt(x); }

// e(-1), e(0), e(+1) and r(c) = 1/(1 + e(c)) for one axis.  With
// bp = B - 1 = (3u + sigma)/(1 - u) the other factors follow without a
// division each: 1/B - 1 = -bp/(1 + bp), 1 + e(+-1) = (1 - sigma) B^{+-1}.
template <typename R>
__device__ __forceinline__ void axis_eq(R u, R e[3], R r[3])
{
    const R u2 = u * u;
    const R S = sqrt_rn(R(1) + R(3) * u2);
    const R sig = R(3) * u2 * rcp(S + R(1));
    const R a = R(3) * u + sig;
    const R oms = R(1) - sig;
    const R bp = a * rcp(R(1) - u);
    const R bm = -bp * rcp(R(1) + bp);
    e[0] = bm * oms - sig;
    e[1] = -sig;
    e[2] = bp * oms - sig;
    const R r1 = rcp(oms);
    r[0] = r1 * (R(1) + bp);
    r[1] = r1;
    r[2] = r1 * (R(1) + bm);
}

// Shear part ds_i for direction i from the face values (sx, sy, sz) and the
// quarter off-diagonal moments (qxy, qxz, qyz).
template <typename R>
__device__ __forceinline__ R shear_part(int i, R sx, R sy, R sz, R qxy, R qxz, R qyz)
{
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    const int nz = nonzero_of(i);
    if (nz == 1) return cx ? sx : (cy ? sy : sz);
    if (nz == 2) {
        if (cz == 0) return cx * cy > 0 ? qxy : -qxy;
        if (cy == 0) return cx * cz > 0 ? qxz : -qxz;
        return cy * cz > 0 ? qyz : -qyz;
    }
    return R(0);
}

// Shear part from N_xz, N_yz and the off-diagonal second moments (used by the
// lane-parallel boundary collision).
template <typename R>
__device__ __forceinline__ R shear_part_raw(int i, R nxz, R nyz, R pxy, R pxz, R pyz)
{
    return shear_part<R>(i, (R(2) * nxz - nyz) * R(1.0 / 6.0), (R(2) * nyz - nxz) * R(1.0 / 6.0),
                         -(nxz + nyz) * R(1.0 / 6.0), R(0.25) * pxy, R(0.25) * pxz, R(0.25) * pyz);
}

// reciprocal / square root for the bulk collision: the hardware approximations
// (relative error about 1 ulp) in FP32, correctly rounded in FP64
__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_fast(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_fast(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double sqrt_fast(double x) { return sqrt(x); }

// e(c), Phi(c) = 1 + e(c) and r(c) = 1/Phi(c) for one axis (see axis_eq)
template <typename R>
__device__ __forceinline__ void axis_eq_phi(R u, R e[3], R phi[3], R r[3])
{
    const R u2 = u * u;
    const R S = sqrt_fast(R(1) + R(3) * u2);
    const R sig = R(3) * u2 * rcp_fast(S + R(1));
    const R a = R(3) * u + sig;
    const R oms = R(1) - sig;
    const R bp = a * rcp_fast(R(1) - u);
    const R bm = -bp * rcp_fast(R(1) + bp);
    e[0] = bm * oms - sig;
    e[1] = -sig;
    e[2] = bp * oms - sig;
    phi[0] = bm * oms + oms;
    phi[1] = oms;
    phi[2] = bp * oms + oms;
    const R r1 = rcp_fast(oms);
    r[0] = r1 * bp + r1;
    r[1] = r1;
    r[2] = r1 * bm + r1;
}

// log(1 + x) in the arithmetic type
__device__ __forceinline__ float log1p_r(float x) { return log1pf(x); }
__device__ __forceinline__ double log1p_r(double x) { return log1p(x); }

// Exact stabilizer (Eq. gamma_min): the root of
//   r(g) = sum_i dh_i log(f'_i(g)/f^eq_i) = sum_i dh_i log(1 + e_i - g B_i),
//   e_i = (dh_i - (2b - 1) ds_i)/f^eq_i,  B_i = b dh_i/f^eq_i,
// on the interval where every f'_i(g) is positive; r falls monotonically
// there (r' = -sum dh_i B_i/(1 + e_i - g B_i) <= 0).  Safeguarded Newton from
// the analytic value g0: the iterates bracket the root (each sets lo or hi by
// the sign of r), a step that leaves the bracket bisects it, and an iterate
// outside the positivity interval moves into it; until the step is below tol,
// at most 40 iterations.  e and B come from the caller through
// the per-direction values (dh, ds, 1/f^eq) the function below recomputes.
template <typename R, typename Terms>
__device__ R exact_gamma(const Terms &terms, R beta, R g0, R tol)
{
    // the positivity interval (lo, hi) is formed only once an iterate leaves
    // it (27 divisions; Newton from the analytic value, the root of the
    // linearised condition, seldom needs it)
    R lo = -R(1e30), hi = R(1e30);
    bool bracket = false;
    R g = g0;
    for (int it = 0; it < 40; ++it) {
        R r = 0, dr = 0;
        bool inside = true;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            R dh, ds, ifeq;
            terms(i, dh, ds, ifeq);
            const R e = (dh - (R(2) * beta - R(1)) * ds) * ifeq, B = beta * dh * ifeq;
            const R x = e - g * B;
            inside = inside && R(1) + x > R(0);
            r += dh * log1p_r(x);
            dr -= dh * B * rcp_fast(R(1) + x);  // (the slope only steers the step)
        }
        if (!inside) {
            if (!bracket) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    R dh, ds, ifeq;
                    terms(i, dh, ds, ifeq);
                    const R e = (dh - (R(2) * beta - R(1)) * ds) * ifeq, B = beta * dh * ifeq;
                    if (B > R(0)) hi = fmin(hi, (R(1) + e) / B);
                    else if (B < R(0)) lo = fmax(lo, (R(1) + e) / B);
                }
                bracket = true;
            }
            g = (lo > -R(1e29) && hi < R(1e29)) ? R(0.5) * (lo + hi) : (g <= lo ? lo + R(1) : hi - R(1));
            continue;
        }
        if (r > R(0)) lo = g;
        else hi = g;
        const R step = dr < R(0) ? r / dr : R(0);
        // converged: the Newton step is below the tolerance (tested before the
        // bracket, which the last iterate itself now bounds)
        if (fabs(step) <= tol * fmax(R(1), fabs(g))) {
            g -= step;
            break;
        }
        R gn = g - step;
        if (!(gn > lo && gn < hi)) gn = R(0.5) * (lo + hi);
        g = gn;
    }
    return g;
}

// In-place collision of the 27 shifted populations g[] of one node.
// Returns false when the density is not finite and positive.
//
// Operation count is kept low by regrouping (same mathematics):
//   - moments from the nine x-lines l = 3(cy+1) + (cz+1) of the velocity cube
//     (directions l, 9 + l, 18 + l have c_x = -1, 0, +1);
//   - E_i = Phi_x Phi_y Phi_z - 1 as exy = e_y Phi_x + e_x, E = exy Phi_z + e_z,
//     and g^eq_i = (rho W_i) E_i + W_i (rho - rho0);
//   - 1/f^eq_i = Rx Ry Rz with R_a(c) = r_a(c)/w(c) (1/rho folded into Rx).
template <typename R, bool EXACT = false>
__device__ __forceinline__ bool kbc_collide(R g[Q], R beta, R inv_beta, R rho0, int gamma_mode)
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
    const R rho = rho0 + drho;
    const bool ok = rho > R(0) && rho < R(1e30);
    const R inv_rho = rcp_fast(rho);
    R ex[3], ey[3], ez[3], px[3], py[3], pz[3], rx[3], ry[3], rz[3];
    axis_eq_phi(jx * inv_rho, ex, px, rx);
    axis_eq_phi(jy * inv_rho, ey, py, ry);
    axis_eq_phi(jz * inv_rho, ez, pz, rz);
    R rw[4], dw[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const R w = k == 0 ? R(8) / R(27) : k == 1 ? R(2) / R(27) : k == 2 ? R(1) / R(54) : R(1) / R(216);
        rw[k] = rho * w;
        dw[k] = drho * w;
    }
    R exy[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) exy[a][b] = ey[b] * px[a] + ex[a];

    // d = g - g^eq in place
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const R E = exy[cx + 1][cy + 1] * pz[cz + 1] + ez[cz + 1];
        g[i] = g[i] - (rw[nz] * E + dw[nz]);
    }
    // second moments of d from line sums
    R A[9], B[9], T[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        A[l] = g[18 + l] + g[l];
        B[l] = g[18 + l] - g[l];
        T[l] = A[l] + g[9 + l];
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

    // entropic scalar products <ds|dh>, <dh|dh>
    R Rx[3], Ry[3], Rz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R iw = c == 1 ? R(1.5) : R(6);
        Rx[c] = rx[c] * inv_rho * iw;
        Ry[c] = ry[c] * iw;
        Rz[c] = rz[c] * iw;
    }
    R sh = 0, hh = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const R ifeq = (Rx[cx + 1] * Ry[cy + 1]) * Rz[cz + 1];
        if (nz == 1 || nz == 2) {
            const R ds = shear_part<R>(i, sx, sy, sz, qxy, qxz, qyz);
            const R dh = g[i] - ds;
            const R t = dh * ifeq;
            sh += ds * t;
            hh += dh * t;
        } else {
            hh += g[i] * (g[i] * ifeq);
        }
    }
    R gam = R(2);
    if (gamma_mode != LBM_GAMMA_LBGK && hh > gamma_floor<R>())
        gam = inv_beta - (R(2) - inv_beta) * sh * rcp_fast(hh);
    if (EXACT && gamma_mode == LBM_GAMMA_EXACT && hh > gamma_floor<R>()) {
        const auto terms = [&](int i, R &dh, R &ds, R &ifeq) {
            const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
            ifeq = (Rx[cx + 1] * Ry[cy + 1]) * Rz[cz + 1];
            ds = (nz == 1 || nz == 2) ? shear_part<R>(i, sx, sy, sz, qxy, qxz, qyz) : R(0);
            dh = g[i] - ds;
        };
        gam = exact_gamma<R>(terms, beta, gam, sizeof(R) == 8 ? R(1e-14) : R(1e-6));
    }
    const R c1 = R(1) - beta * gam;
    const R c2 = beta * (gam - R(2));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const R E = exy[cx + 1][cy + 1] * pz[cz + 1] + ez[cz + 1];
        R v = c1 * g[i] + (rw[nz] * E + dw[nz]);
        if (nz == 1 || nz == 2) v += c2 * shear_part<R>(i, sx, sy, sz, qxy, qxz, qyz);
        g[i] = v;
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
