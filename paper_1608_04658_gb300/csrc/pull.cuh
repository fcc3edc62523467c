// Pull streaming of one node under the box rules (arXiv 1608.04658, Sec. 2,
// Eq. kineticEq: F_i(x) = f'_i(x - c_i, t)), shared by the bulk kernel and
// its adjoint.
#pragma once

#include "kbc.cuh"

namespace lbm {

// Relative source offsets for velocity component c = -1, 0, +1 of a pull from
// a - c along one axis (stride = element distance of one step on that axis),
// and the kind of the source: 0 node in the box (wrapped on periodic faces,
// clamped on outflow faces), 1 equilibrium face, 2 wall face.
__device__ __forceinline__ void axis_off(int a, int n, int stride, int face_lo, int face_hi,
                                         int o[3], int k[3])
{
    o[1] = 0;
    k[1] = 0;
    // c = +1 pulls from a - 1
    o[2] = -stride;
    k[2] = 0;
    if (a == 0) {
        o[2] = 0;
        if (face_lo == LBM_FACE_PERIODIC) o[2] = (n - 1) * stride;
        else if (face_lo == LBM_FACE_WALL) k[2] = 2;
        else if (face_lo == LBM_FACE_EQ) k[2] = 1;
    }
    // c = -1 pulls from a + 1
    o[0] = stride;
    k[0] = 0;
    if (a == n - 1) {
        o[0] = 0;
        if (face_hi == LBM_FACE_PERIODIC) o[0] = -(n - 1) * stride;
        else if (face_hi == LBM_FACE_WALL) k[0] = 2;
        else if (face_hi == LBM_FACE_EQ) k[0] = 1;
    }
}

// coordinate c on axis a (n nodes) inside the sweep box sw = {lo[3], n[3]}
// (wrapping on a periodic axis, where lo lies in (-n, n))
__device__ __forceinline__ bool in_sweep(const int *__restrict__ sw, int a, int c, int n, bool periodic)
{
    int d = c - sw[a];
    if (periodic) {
        if (d < 0) d += n;
        else if (d >= n) d -= n;
    }
    return (unsigned)d < (unsigned)sw[3 + a];
}

__device__ __forceinline__ bool in_sweep_box(const Lattice &L, const int *__restrict__ sw, int x, int y, int z)
{
    return in_sweep(sw, 1, y, L.ny, L.face[2] == LBM_FACE_PERIODIC) &&
           in_sweep(sw, 2, z, L.nz, L.face[4] == LBM_FACE_PERIODIC) &&
           in_sweep(sw, 0, x, L.nx, L.face[0] == LBM_FACE_PERIODIC);
}

__device__ __forceinline__ int sweep_coord(int v, int n)
{
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// pulls of node (x, y, z) from global memory under the box rules
template <typename S>
__device__ __forceinline__ void gather_global(const Lattice &L, const S *__restrict__ fa, int x, int y, int z,
                                              int n, typename Codec<S>::R g[Q])
{
    using R = typename Codec<S>::R;
    int ox[3], oy[3], oz[3], kx[3], ky[3], kz[3];
    axis_off(x, L.nx, 1, L.face[0], L.face[1], ox, kx);
    axis_off(y, L.ny, L.nx, L.face[2], L.face[3], oy, ky);
    axis_off(z, L.nz, L.nx * L.ny, L.face[4], L.face[5], oz, kz);
    const S *p = fa + n;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        g[i] = Codec<S>::load(p + (L.plane[i] + ox[cx_of(i) + 1] + oy[cy_of(i) + 1] + oz[cz_of(i) + 1]));
    if (!(kx[0] | kx[2] | ky[0] | ky[2] | kz[0] | kz[2])) return;
    if (sizeof(S) > 2) {
        // precedence per direction: the largest kind over its three axes
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int k = max(kx[cx_of(i) + 1], max(ky[cy_of(i) + 1], kz[cz_of(i) + 1]));
            if (k == 2) g[i] = Codec<S>::load(p + L.plane[26 - i]);
            else if (k == 1) g[i] = (R)L.g_face[i];
        }
    } else {
        // (the shorter form for 16-bit storage, measured faster there) a face
        // touches the nine directions whose component along its axis points
        // away from it: equilibrium faces first, then walls, so a wall wins
        // where a pull leaves through both
        const int k[3][3] = {{kx[0], kx[1], kx[2]}, {ky[0], ky[1], ky[2]}, {kz[0], kz[1], kz[2]}};
#pragma unroll
        for (int pass = 1; pass <= 2; ++pass)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int side = 0; side < 3; side += 2) {
                    if (k[a][side] != pass) continue;
                    const int c = side - 1;  // component of the directions concerned
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const int ci = a == 0 ? cx_of(i) : a == 1 ? cy_of(i) : cz_of(i);
                        if (ci != c) continue;
                        if (pass == 2) g[i] = Codec<S>::load(p + L.plane[26 - i]);
                        else g[i] = (R)L.g_face[i];
                    }
                }
    }
}

}  // namespace lbm
