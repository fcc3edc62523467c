// Warp-per-node building blocks of the boundary and refill kernels and of
// their adjoints (arXiv 1608.04658, Secs. 2 and 3): lane i < 27 owns
// direction i; sums over directions are shuffle trees whose lane-0 result is
// broadcast, so every lane sees the same density, velocity and stabilizer.
#pragma once

#include "geom.cuh"
#include "kbc.cuh"

namespace lbm {

constexpr int BWARPS = 4;
constexpr unsigned FULL = 0xffffffffu;

template <typename R>
__device__ __forceinline__ R wsum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    return __shfl_sync(FULL, v, 0);
}

template <typename R>
__device__ __forceinline__ R pick(const R e[3], int c)
{
    return c < 0 ? e[0] : (c > 0 ? e[2] : e[1]);
}

// Lane-parallel KBC collision: lane i < 27 holds the shifted population g_i.
template <typename R>
__device__ R kbc_collide_lanes(R g, int i, R beta, R inv_beta, R rho0, int gamma_mode, bool &ok)
{
    const bool act = i < Q;
    const int cx = act ? cx_of(i) : 0, cy = act ? cy_of(i) : 0, cz = act ? cz_of(i) : 0;
    const R gv = act ? g : R(0);
    const R drho = wsum(gv);
    const R jx = wsum(R(cx) * gv), jy = wsum(R(cy) * gv), jz = wsum(R(cz) * gv);
    const R rho = rho0 + drho;
    ok = rho > R(0) && rho < R(1e30);
    const R inv_rho = rcp(rho);
    R ex[3], ey[3], ez[3], rx[3], ry[3], rz[3];
    axis_eq(jx * inv_rho, ex, rx);
    axis_eq(jy * inv_rho, ey, ry);
    axis_eq(jz * inv_rho, ez, rz);
    const R exy = pick(ex, cx) + pick(ey, cy) + pick(ex, cx) * pick(ey, cy);
    const R E = exy + pick(ez, cz) + exy * pick(ez, cz);
    const R geq = act ? weight<R>(i) * (drho + rho * E) : R(0);
    const R d = gv - geq;
    const R pxx = wsum(R(cx * cx) * d), pyy = wsum(R(cy * cy) * d), pzz = wsum(R(cz * cz) * d);
    const R pxy = wsum(R(cx * cy) * d), pxz = wsum(R(cx * cz) * d), pyz = wsum(R(cy * cz) * d);
    const R nxz = pxx - pzz, nyz = pyy - pzz;
    const R ds = act ? shear_part_raw<R>(i, nxz, nyz, pxy, pxz, pyz) : R(0);
    const R dh = d - ds;
    const R ifeq = act ? inv_rho * inv_weight<R>(i) * pick(rx, cx) * pick(ry, cy) * pick(rz, cz) : R(0);
    const R sh = wsum(ds * dh * ifeq), hh = wsum(dh * dh * ifeq);
    R gam = R(2);
    if (gamma_mode != LBM_GAMMA_LBGK && hh > gamma_floor<R>())
        gam = inv_beta - (R(2) - inv_beta) * sh * rcp(hh);
    if (gamma_mode == LBM_GAMMA_EXACT && hh > gamma_floor<R>()) {
        // exact stabilizer (see exact_gamma) with the directions on the lanes
        const R e = act ? (dh - (R(2) * beta - R(1)) * ds) * ifeq : R(0);
        const R B = act ? beta * dh * ifeq : R(0);
        R lo = B < R(0) ? (R(1) + e) / B : -R(1e30), hi = B > R(0) ? (R(1) + e) / B : R(1e30);
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmax(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmin(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        R g = gam;
        if (!(g > lo && g < hi))
            g = (lo > -R(1e29) && hi < R(1e29)) ? R(0.5) * (lo + hi) : (g <= lo ? lo + R(1) : hi - R(1));
        const R tol = sizeof(R) == 8 ? R(1e-14) : R(1e-6);
        for (int it = 0; it < 40; ++it) {
            const R x = e - g * B;
            const R r = wsum(act ? dh * log1p_r(x) : R(0));
            const R dr = wsum(act ? -dh * B / (R(1) + x) : R(0));
            if (r > R(0)) lo = g;
            else hi = g;
            const R step = dr < R(0) ? r / dr : R(0);
            if (fabs(step) <= tol * fmax(R(1), fabs(g))) {
                g -= step;
                break;
            }
            R gn = g - step;
            if (!(gn > lo && gn < hi)) gn = R(0.5) * (lo + hi);
            g = gn;
        }
        gam = g;
    }
    return geq + (R(1) - beta * gam) * d + beta * (gam - R(2)) * ds;
}

// Shifted Grad distribution g*_i = f*_i - W_i rho0 (Eq. grad, c_s^2 = 1/3):
//   f*_i = W_i [rho + 3 rho c.u + (9/2) Qt : (c c - I/3)],  Qt = Pi - rho/3 I.
template <typename R>
__device__ __forceinline__ R grad_shifted(int i, R rho, R rho0, const R u[3], const R Qt[6])
{
    const R cx = R(cx_of(i)), cy = R(cy_of(i)), cz = R(cz_of(i));
    const R cu = cx * u[0] + cy * u[1] + cz * u[2];
    // Qt = (xx, yy, zz, xy, xz, yz)
    const R qcc = Qt[0] * cx * cx + Qt[1] * cy * cy + Qt[2] * cz * cz
                + R(2) * (Qt[3] * cx * cy + Qt[4] * cx * cz + Qt[5] * cy * cz);
    const R tr = (Qt[0] + Qt[1] + Qt[2]) * R(1.0 / 3.0);
    return weight<R>(i) * ((rho - rho0) + R(3) * rho * cu + R(4.5) * (qcc - tr));
}

// Qt = rho u u - (rho c_s^2 / (2 beta)) (grad u + grad u^T)  (Eqs. pressure, pressure2)
template <typename R>
__device__ __forceinline__ void pressure_excess(R rho, const R u[3], const R du[3][3], R beta, R Qt[6])
{
    const R k = rho / (R(6) * beta);
    Qt[0] = rho * u[0] * u[0] - k * R(2) * du[0][0];
    Qt[1] = rho * u[1] * u[1] - k * R(2) * du[1][1];
    Qt[2] = rho * u[2] * u[2] - k * R(2) * du[2][2];
    Qt[3] = rho * u[0] * u[1] - k * (du[0][1] + du[1][0]);
    Qt[4] = rho * u[0] * u[2] - k * (du[0][2] + du[2][0]);
    Qt[5] = rho * u[1] * u[2] - k * (du[1][2] + du[2][1]);
}

// velocity gradient du[a][b] = d u_a / d x_b from the staged neighbourhood
template <typename R>
__device__ __forceinline__ void fd_gradient(const R (*su)[4], const int *sok, const R uc[3], R du[3][3])
{
    const int step[3] = {9, 3, 1};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const int kp = 13 + step[b], km = 13 - step[b];
        const bool op = sok[kp], om = sok[km];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R v = R(0);
            if (op && om) v = R(0.5) * (su[kp][1 + a] - su[km][1 + a]);
            else if (op) v = su[kp][1 + a] - uc[a];
            else if (om) v = uc[a] - su[km][1 + a];
            du[a][b] = v;
        }
    }
}

// Stage populations of neighbourhood nodes selected by 'need' into sf[k][i]
// and their density/velocity into su[k] (lane k).  sok[k] must be set.
template <typename S, typename R>
__device__ __forceinline__ void stage(const Lattice &L, const S *__restrict__ fa, int lane, int nk,
                                      uint32_t need, R (*sf)[28], R (*su)[4], const int *sok)
{
    const size_t N = (size_t)L.N;
    // all loads first, into registers, so they are in flight together (a
    // store to shared memory right behind each load would wait out one
    // memory latency per node)
    R v[Q];
    uint32_t got = 0;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int nodek = __shfl_sync(FULL, nk, k);
        const bool use = ((need >> k) & 1u) && nodek >= 0 && lane < Q;
        v[k] = use ? Codec<S>::load(fa + (size_t)lane * N + nodek) : R(0);
        got |= (use ? 1u : 0u) << k;
    }
#pragma unroll
    for (int k = 0; k < Q; ++k)
        if ((got >> k) & 1u) sf[k][lane] = v[k];
    __syncwarp();
    if (lane < Q && ((need >> lane) & 1u) && nk >= 0) {
        R r = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            const R v = sf[lane][i];
            r += v;
            j[0] += R(cx_of(i)) * v;
            j[1] += R(cy_of(i)) * v;
            j[2] += R(cz_of(i)) * v;
        }
        const R rho = R(L.rho0) + r;
        su[lane][0] = rho;
        su[lane][1] = j[0] / rho;
        su[lane][2] = j[1] / rho;
        su[lane][3] = j[2] / rho;
    }
    __syncwarp();
}

__device__ __forceinline__ void node_xyz(const Lattice &L, int n, int &x, int &y, int &z)
{
    x = n % L.nx;
    y = (n / L.nx) % L.ny;
    z = n / (L.nx * L.ny);
}

}  // namespace lbm
