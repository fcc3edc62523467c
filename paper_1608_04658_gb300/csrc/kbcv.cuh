// KBC entropic collision of one node (float) or of two nodes at once
// (float2, packed FP32x2 arithmetic) in shifted form, for FP32 and 16-bit
// storage.  Same mathematics as kbc_collide (arXiv 1608.04658, Sec. 2,
// Eqs. kineticEq, kbc_relax, feq_min and the analytic stabilizer), written
// with explicit correctly rounded operations so that the one-node and the
// two-node forms give the same bits for a node: the two-node form does each
// operation of the one-node form on both lanes of a float2.
#pragma once

#include "kbc.cuh"

#ifndef LBM_RECOMPUTE_EQ
#define LBM_RECOMPUTE_EQ 1
#endif

namespace lbm {

// one node: V = float
struct F1 {
    using V = float;
    static __device__ __forceinline__ V c(float s) { return s; }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __fadd_rn(a, -b); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V d) { return __fmaf_rn(a, b, d); }
    static __device__ __forceinline__ V neg(V a) { return -a; }
    static __device__ __forceinline__ V rcp(V a) { return rcp_fast(a); }
    static __device__ __forceinline__ V sqrt(V a) { return sqrt_fast(a); }
    static __device__ __forceinline__ float lane(V a, int k) { return a; }
    static __device__ __forceinline__ V make(float a, float b) { return a; }
};

// two nodes: V = float2, lane x the first node, lane y the second
struct F2 {
    using V = float2;
    static __device__ __forceinline__ V c(float s) { return make_float2(s, s); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V d) { return __ffma2_rn(a, b, d); }
    static __device__ __forceinline__ V neg(V a) { return make_float2(-a.x, -a.y); }
    static __device__ __forceinline__ V rcp(V a) { return make_float2(rcp_fast(a.x), rcp_fast(a.y)); }
    static __device__ __forceinline__ V sqrt(V a) { return make_float2(sqrt_fast(a.x), sqrt_fast(a.y)); }
    static __device__ __forceinline__ float lane(V a, int k) { return k ? a.y : a.x; }
    static __device__ __forceinline__ V make(float a, float b) { return make_float2(a, b); }
};

// e(c), Phi(c) = 1 + e(c) and r(c) = 1/Phi(c) for one axis (see axis_eq)
template <typename O>
__device__ __forceinline__ void axis_eq_v(typename O::V u, typename O::V e[3], typename O::V phi[3],
                                          typename O::V r[3])
{
    using V = typename O::V;
    const V u2 = O::mul(u, u);
    const V S = O::sqrt(O::fma(O::c(3.f), u2, O::c(1.f)));
    const V sig = O::mul(O::mul(O::c(3.f), u2), O::rcp(O::add(S, O::c(1.f))));
    const V a = O::fma(O::c(3.f), u, sig);
    const V oms = O::sub(O::c(1.f), sig);
    const V bp = O::mul(a, O::rcp(O::sub(O::c(1.f), u)));
    const V bm = O::mul(O::neg(bp), O::rcp(O::add(O::c(1.f), bp)));
    const V nsig = O::neg(sig);
    e[0] = O::fma(bm, oms, nsig);
    e[1] = nsig;
    e[2] = O::fma(bp, oms, nsig);
    phi[0] = O::fma(bm, oms, oms);
    phi[1] = oms;
    phi[2] = O::fma(bp, oms, oms);
    const V r1 = O::rcp(oms);
    r[0] = O::fma(r1, bp, r1);
    r[1] = r1;
    r[2] = O::fma(r1, bm, r1);
}

// v, with a dependence on dep the compiler cannot see through: a value
// computed from it again after dep is formed is recomputed there, not kept
// live from its first evaluation
template <typename O>
__device__ __forceinline__ typename O::V after(typename O::V v, typename O::V dep)
{
    float out[2] = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < (int)(sizeof(v) / sizeof(float)); ++k)
        asm volatile("mov.b32 %0, %1;" : "=f"(out[k]) : "f"(O::lane(v, k)), "f"(O::lane(dep, k)));
    return O::make(out[0], out[1]);
}

// Shear part ds_i for direction i (faces sx, sy, sz; edges the signed
// quarter off-diagonal moments; rest and corners 0 are never asked for).
template <typename V>
__device__ __forceinline__ V shear_v(int i, V sx, V sy, V sz, V qxy, V qxz, V qyz)
{
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    if (nonzero_of(i) == 1) return cx ? sx : (cy ? sy : sz);
    if (cz == 0) return qxy;
    if (cy == 0) return qxz;
    return qyz;
}
// sign of the edge term of direction i (+1 for faces)
__host__ __device__ constexpr int shear_sign(int i)
{
    return nonzero_of(i) != 2 ? 1
         : cz_of(i) == 0 ? cx_of(i) * cy_of(i)
         : cy_of(i) == 0 ? cx_of(i) * cz_of(i)
                         : cy_of(i) * cz_of(i);
}

// In-place collision of the 27 shifted populations of one or two nodes
// (kbc_collide's regrouping: x-line moment sums, E_i = Phi_x Phi_y Phi_z - 1
// from the 1-D factors, 1/f^eq_i = Rx Ry Rz).  Returns a bit per node (bit 0
// the first, bit 1 the second) set when its density is finite and positive.
// gamma_mode: analytic stabilizer or LBGK (gamma = 2); the exact stabilizer
// has its own kernel instance.
template <typename O>
__device__ __forceinline__ int kbc_collide_v(typename O::V g[Q], float beta, float inv_beta, float rho0,
                                             int gamma_mode)
{
    using V = typename O::V;
    constexpr int NL = sizeof(V) / sizeof(float);
    V Ls[9], Ld[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        Ld[l] = O::sub(g[18 + l], g[l]);
        Ls[l] = O::add(O::add(g[18 + l], g[l]), g[9 + l]);
    }
#define LBM_SUM9(A) O::add(O::add(O::add(A[0], A[1]), O::add(A[2], A[3])), \
                           O::add(O::add(A[4], A[5]), O::add(O::add(A[6], A[7]), A[8])))
    const V drho = LBM_SUM9(Ls);
    const V jx = LBM_SUM9(Ld);
    const V jy = O::sub(O::add(O::add(Ls[6], Ls[7]), Ls[8]), O::add(O::add(Ls[0], Ls[1]), Ls[2]));
    const V jz = O::sub(O::add(O::add(Ls[2], Ls[5]), Ls[8]), O::add(O::add(Ls[0], Ls[3]), Ls[6]));
    const V rho = O::add(O::c(rho0), drho);
    int ok = 0;
#pragma unroll
    for (int k = 0; k < NL; ++k) {
        const float r = O::lane(rho, k);
        ok |= (r > 0.f && r < 1e30f) << k;
    }
    const V inv_rho = O::rcp(rho);
    V ex[3], ey[3], ez[3], px[3], py[3], pz[3], rx[3], ry[3], rz[3];
    axis_eq_v<O>(O::mul(jx, inv_rho), ex, px, rx);
    axis_eq_v<O>(O::mul(jy, inv_rho), ey, py, ry);
    axis_eq_v<O>(O::mul(jz, inv_rho), ez, pz, rz);
    V rw[4], dw[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float w = k == 0 ? 8.f / 27.f : k == 1 ? 2.f / 27.f : k == 2 ? 1.f / 54.f : 1.f / 216.f;
        rw[k] = O::mul(rho, O::c(w));
        dw[k] = O::mul(drho, O::c(w));
    }
    V exy[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) exy[a][b] = O::fma(ey[b], px[a], ex[a]);

    // d = g - g^eq in place
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const V E = O::fma(exy[cx + 1][cy + 1], pz[cz + 1], ez[cz + 1]);
        g[i] = O::sub(g[i], O::fma(rw[nz], E, dw[nz]));
    }
    // second moments of d from line sums
    V A[9], B[9], T[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        A[l] = O::add(g[18 + l], g[l]);
        B[l] = O::sub(g[18 + l], g[l]);
        T[l] = O::add(A[l], g[9 + l]);
    }
    const V pxx = LBM_SUM9(A);
#undef LBM_SUM9
    const V pxy = O::sub(O::add(O::add(B[6], B[7]), B[8]), O::add(O::add(B[0], B[1]), B[2]));
    const V pxz = O::sub(O::add(O::add(B[2], B[5]), B[8]), O::add(O::add(B[0], B[3]), B[6]));
    const V pyy = O::add(O::add(O::add(T[0], T[1]), T[2]), O::add(O::add(T[6], T[7]), T[8]));
    const V pzz = O::add(O::add(O::add(T[0], T[3]), T[6]), O::add(O::add(T[2], T[5]), T[8]));
    const V pyz = O::sub(O::add(T[0], T[8]), O::add(T[2], T[6]));
    const V nxz = O::sub(pxx, pzz), nyz = O::sub(pyy, pzz);
    const V sixth = O::c(1.f / 6.f);
    const V sx = O::mul(O::sub(O::add(nxz, nxz), nyz), sixth);
    const V sy = O::mul(O::sub(O::add(nyz, nyz), nxz), sixth);
    const V sz = O::mul(O::neg(O::add(nxz, nyz)), sixth);
    const V qxy = O::mul(O::c(0.25f), pxy), qxz = O::mul(O::c(0.25f), pxz), qyz = O::mul(O::c(0.25f), pyz);

    // entropic scalar products <ds|dh>, <dh|dh>
    V Rx[3], Ry[3], Rz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const V iw = O::c(c == 1 ? 1.5f : 6.f);
        Rx[c] = O::mul(O::mul(rx[c], inv_rho), iw);
        Ry[c] = O::mul(ry[c], iw);
        Rz[c] = O::mul(rz[c], iw);
    }
    V sh = O::c(0.f), hh = O::c(0.f);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const V ifeq = O::mul(O::mul(Rx[cx + 1], Ry[cy + 1]), Rz[cz + 1]);
        if (nz == 1 || nz == 2) {
            // ds = sign * shear value; dh = d - ds
            const V sv = shear_v<V>(i, sx, sy, sz, qxy, qxz, qyz);
            const V ds = shear_sign(i) > 0 ? sv : O::neg(sv);
            const V dh = O::sub(g[i], ds);
            const V t = O::mul(dh, ifeq);
            sh = O::fma(ds, t, sh);
            hh = O::fma(dh, t, hh);
        } else {
            hh = O::fma(g[i], O::mul(g[i], ifeq), hh);
        }
    }
    // stabilizer per node
    float c1v[NL], c2v[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
        const float shk = O::lane(sh, k), hhk = O::lane(hh, k);
        float gam = 2.f;
        if (gamma_mode != LBM_GAMMA_LBGK && hhk > 1e-30f)
            gam = __fsub_rn(inv_beta, __fmul_rn(__fmul_rn(__fsub_rn(2.f, inv_beta), shk), rcp_fast(hhk)));
        c1v[k] = __fsub_rn(1.f, __fmul_rn(beta, gam));
        c2v[k] = __fmul_rn(beta, __fsub_rn(gam, 2.f));
    }
    const V c1 = O::make(c1v[0], c1v[NL - 1]);
    const V c2 = O::make(c2v[0], c2v[NL - 1]);
#if LBM_RECOMPUTE_EQ
    // the equilibrium again from the same velocity, bit for bit the same
    // factors: keeping them across the scalar products needs some 46 more
    // registers, which the 16-bit two-node kernel would spill
    {
        const V ir = after<O>(inv_rho, hh);
        axis_eq_v<O>(O::mul(after<O>(jx, hh), ir), ex, px, rx);
        axis_eq_v<O>(O::mul(after<O>(jy, hh), ir), ey, py, ry);
        axis_eq_v<O>(O::mul(after<O>(jz, hh), ir), ez, pz, rz);
        const V rho2 = after<O>(rho, hh), drho2 = after<O>(drho, hh);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float w = k == 0 ? 8.f / 27.f : k == 1 ? 2.f / 27.f : k == 2 ? 1.f / 54.f : 1.f / 216.f;
            rw[k] = O::mul(rho2, O::c(w));
            dw[k] = O::mul(drho2, O::c(w));
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) exy[a][b] = O::fma(ey[b], px[a], ex[a]);
    }
#endif
    // g' = g^eq + c1 d + c2 ds
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i), nz = nonzero_of(i);
        const V E = O::fma(exy[cx + 1][cy + 1], pz[cz + 1], ez[cz + 1]);
        V v = O::fma(c1, g[i], O::fma(rw[nz], E, dw[nz]));
        if (nz == 1 || nz == 2) {
            const V sv = shear_v<V>(i, sx, sy, sz, qxy, qxz, qyz);
            v = O::fma(shear_sign(i) > 0 ? c2 : O::neg(c2), sv, v);
        }
        g[i] = v;
    }
    return ok;
}

}  // namespace lbm
