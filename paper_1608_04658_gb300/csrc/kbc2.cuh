// KBC entropic collision of two nodes at once in packed FP32x2 arithmetic
// (sm_100+ FADD2 / FMUL2 / FFMA2), for FP32 and 16-bit storage.
//
// Same mathematics as kbc_collide in kbc.cuh (arXiv 1608.04658, Sec. 2: Eqs.
// kineticEq, kbc_relax, feq_min and the analytic stabilizer); component .x is
// one node, .y the other.  The operation count is reduced by regrouping, not
// by changing what is computed:
//   - moments from the nine x-lines of the 3x3x3 velocity cube: per line
//     (cy, cz) the sum and difference of the c_x = +-1 populations;
//   - with Phi_a(c) = 1 + e_a(c), E_i = Phi_x Phi_y Phi_z - 1 is formed as
//     exy = e_y Phi_x + e_x, E = exy Phi_z + e_z (no cancellation), and
//     g^eq_i = (rho W_i) E_i + W_i (rho - rho0);
//   - 1/f^eq_i = prod_a R_a(c_ia) with the weight and 1/rho folded into the
//     per-axis factors R_a(c) = r_a(c) / w(c) (1/rho on the x axis);
//   - reciprocals and square roots with the hardware approximations
//     (rcp.approx / sqrt.approx, relative error about 1 ulp), which perturb
//     the equilibrium factors at the 1e-7 level.
#pragma once

#include <type_traits>

#include "kbc.cuh"

namespace lbm {

__device__ __forceinline__ float2 f2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp_fast(a.x), rcp_fast(a.y)); }
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(sqrt_fast(a.x), sqrt_fast(a.y)); }

// e(c), Phi(c) = 1 + e(c) and r(c) = 1/Phi(c), c = -1, 0, +1, for one axis
// (the factorisation of axis_eq in kbc.cuh)
__device__ __forceinline__ void axis_eq2(float2 u, float2 e[3], float2 phi[3], float2 r[3])
{
    const float2 one = f2(1.f), three = f2(3.f);
    const float2 u2 = mul2(u, u);
    const float2 S = sqrt2(fma2(three, u2, one));
    const float2 sig = mul2(mul2(three, u2), rcp2(add2(S, one)));
    const float2 a = fma2(three, u, sig);
    const float2 oms = sub2(one, sig);
    const float2 bp = mul2(a, rcp2(sub2(one, u)));
    const float2 bm = mul2(neg2(bp), rcp2(add2(one, bp)));
    e[0] = fma2(bm, oms, neg2(sig));
    e[1] = neg2(sig);
    e[2] = fma2(bp, oms, neg2(sig));
    phi[0] = fma2(bm, oms, oms);
    phi[1] = oms;
    phi[2] = fma2(bp, oms, oms);
    const float2 r1 = rcp2(oms);
    r[0] = fma2(r1, bp, r1);
    r[1] = r1;
    r[2] = fma2(r1, bm, r1);
}

template <int I, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (I < Q) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1>(f);
    }
}

template <int I>
__device__ __forceinline__ float2 shear2(float2 sx, float2 sy, float2 sz, float2 qxy, float2 qxz, float2 qyz)
{
    constexpr int cx = cx_of(I), cy = cy_of(I), cz = cz_of(I), nz = nonzero_of(I);
    if constexpr (nz == 1) return cx ? sx : (cy ? sy : sz);
    else if constexpr (nz == 2) {
        if constexpr (cz == 0) return cx * cy > 0 ? qxy : neg2(qxy);
        else if constexpr (cy == 0) return cx * cz > 0 ? qxz : neg2(qxz);
        else return cy * cz > 0 ? qyz : neg2(qyz);
    } else return f2(0.f);
}

// In-place collision of g[i] = (node a, node b) shifted populations; ok_a /
// ok_b report a finite, positive density per node.  Line l = 3(cy+1) + (cz+1)
// holds directions l (c_x = -1), 9 + l (c_x = 0) and 18 + l (c_x = +1).
__device__ __forceinline__ void kbc_collide2(float2 g[Q], float beta, float inv_beta, float rho0,
                                             int gamma_mode, bool &ok_a, bool &ok_b)
{
    // ---- conserved moments from line sums
    float2 Lsum[9], Ldif[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        Ldif[l] = sub2(g[18 + l], g[l]);
        Lsum[l] = add2(add2(g[18 + l], g[l]), g[9 + l]);
    }
    const float2 drho = add2(add2(add2(Lsum[0], Lsum[1]), add2(Lsum[2], Lsum[3])),
                             add2(add2(Lsum[4], Lsum[5]), add2(add2(Lsum[6], Lsum[7]), Lsum[8])));
    const float2 jx = add2(add2(add2(Ldif[0], Ldif[1]), add2(Ldif[2], Ldif[3])),
                           add2(add2(Ldif[4], Ldif[5]), add2(add2(Ldif[6], Ldif[7]), Ldif[8])));
    const float2 jy = sub2(add2(add2(Lsum[6], Lsum[7]), Lsum[8]), add2(add2(Lsum[0], Lsum[1]), Lsum[2]));
    const float2 jz = sub2(add2(add2(Lsum[2], Lsum[5]), Lsum[8]), add2(add2(Lsum[0], Lsum[3]), Lsum[6]));
    const float2 rho = add2(f2(rho0), drho);
    ok_a = rho.x > 0.f && rho.x < 1e30f;
    ok_b = rho.y > 0.f && rho.y < 1e30f;
    const float2 inv_rho = rcp2(rho);
    float2 ex[3], ey[3], ez[3], px[3], py[3], pz[3], rx[3], ry[3], rz[3];
    axis_eq2(mul2(jx, inv_rho), ex, px, rx);
    axis_eq2(mul2(jy, inv_rho), ey, py, ry);
    axis_eq2(mul2(jz, inv_rho), ez, pz, rz);
    // rho W and (rho - rho0) W per weight class (rest, face, edge, corner)
    float2 rw[4], dw[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float w = k == 0 ? 8.f / 27.f : k == 1 ? 2.f / 27.f : k == 2 ? 1.f / 54.f : 1.f / 216.f;
        rw[k] = mul2(rho, f2(w));
        dw[k] = mul2(drho, f2(w));
    }
    // exy[cx][cy] = (1+ex)(1+ey) - 1
    float2 exy[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) exy[a][b] = fma2(ey[b], px[a], ex[a]);

    // ---- non-equilibrium part d = g - g^eq (in place)
    static_for<0>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const float2 E = fma2(exy[cx + 1][cy + 1], pz[cz + 1], ez[cz + 1]);
        g[i] = sub2(g[i], fma2(rw[nz], E, dw[nz]));
    });
    // ---- second moments of d from line sums
    float2 A[9], B[9], T[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        A[l] = add2(g[18 + l], g[l]);
        B[l] = sub2(g[18 + l], g[l]);
        T[l] = add2(A[l], g[9 + l]);
    }
    const float2 pxx = add2(add2(add2(A[0], A[1]), add2(A[2], A[3])),
                            add2(add2(A[4], A[5]), add2(add2(A[6], A[7]), A[8])));
    const float2 pxy = sub2(add2(add2(B[6], B[7]), B[8]), add2(add2(B[0], B[1]), B[2]));
    const float2 pxz = sub2(add2(add2(B[2], B[5]), B[8]), add2(add2(B[0], B[3]), B[6]));
    const float2 pyy = add2(add2(add2(T[0], T[1]), T[2]), add2(add2(T[6], T[7]), T[8]));
    const float2 pzz = add2(add2(add2(T[0], T[3]), T[6]), add2(add2(T[2], T[5]), T[8]));
    const float2 pyz = sub2(add2(T[0], T[8]), add2(T[2], T[6]));
    const float2 nxz = sub2(pxx, pzz), nyz = sub2(pyy, pzz);
    const float2 sixth = f2(1.0f / 6.0f), quarter = f2(0.25f), two = f2(2.f);
    const float2 sx = mul2(sub2(mul2(two, nxz), nyz), sixth);
    const float2 sy = mul2(sub2(mul2(two, nyz), nxz), sixth);
    const float2 sz = mul2(neg2(add2(nxz, nyz)), sixth);
    const float2 qxy = mul2(quarter, pxy), qxz = mul2(quarter, pxz), qyz = mul2(quarter, pyz);

    // ---- entropic scalar products; 1/f^eq_i = Rx Ry Rz with R_a(c) = r_a(c)/w(c)
    float2 Rx[3], Ry[3], Rz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float iw = c == 1 ? 1.5f : 6.f;
        Rx[c] = mul2(mul2(rx[c], inv_rho), f2(iw));
        Ry[c] = mul2(ry[c], f2(iw));
        Rz[c] = mul2(rz[c], f2(iw));
    }
    float2 sh = f2(0.f), hh = f2(0.f);
    static_for<0>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const float2 ifeq = mul2(mul2(Rx[cx + 1], Ry[cy + 1]), Rz[cz + 1]);
        if constexpr (nz == 1 || nz == 2) {
            const float2 ds = shear2<i>(sx, sy, sz, qxy, qxz, qyz);
            const float2 dh = sub2(g[i], ds);
            const float2 t = mul2(dh, ifeq);
            sh = fma2(ds, t, sh);
            hh = fma2(dh, t, hh);
        } else {
            hh = fma2(g[i], mul2(g[i], ifeq), hh);
        }
    });
    float2 gam = f2(2.f);
    if (gamma_mode == LBM_GAMMA_ANALYTIC) {
        if (hh.x > 1e-30f) gam.x = inv_beta - (2.f - inv_beta) * sh.x * rcp_fast(hh.x);
        if (hh.y > 1e-30f) gam.y = inv_beta - (2.f - inv_beta) * sh.y * rcp_fast(hh.y);
    }
    // ---- g' = g^eq + (1 - b g) d + b (g - 2) ds
    const float2 c1 = sub2(f2(1.f), mul2(f2(beta), gam));
    const float2 c2 = mul2(f2(beta), sub2(gam, two));
    static_for<0>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const float2 E = fma2(exy[cx + 1][cy + 1], pz[cz + 1], ez[cz + 1]);
        float2 v = fma2(c1, g[i], fma2(rw[nz], E, dw[nz]));
        if constexpr (nz == 1 || nz == 2) v = fma2(c2, shear2<i>(sx, sy, sz, qxy, qxz, qyz), v);
        g[i] = v;
    });
}

}  // namespace lbm
