// Pull streaming of one node under the box rules (arXiv 1608.04658, Sec. 2,
// Eq. kineticEq: F_i(x) = f'_i(x - c_i, t)), shared by the bulk kernel and
// its adjoint.
#pragma once

#include "kbcv.cuh"

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

// The pulls of one node, as gather_global, written into lane H (0: x, 1: y)
// of the float2 populations of a node pair (the pair's node at an x face).
template <typename S, int H>
__device__ __forceinline__ void gather_node_lane(const Lattice &L, const S *__restrict__ fa, int x, int y, int z,
                                                 int n, float2 g[Q])
{
    int ox[3], oy[3], oz[3], kx[3], ky[3], kz[3];
    axis_off(x, L.nx, 1, L.face[0], L.face[1], ox, kx);
    axis_off(y, L.ny, L.nx, L.face[2], L.face[3], oy, ky);
    axis_off(z, L.nz, L.nx * L.ny, L.face[4], L.face[5], oz, kz);
    const S *p = fa + n;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int k = max(kx[cx_of(i) + 1], max(ky[cy_of(i) + 1], kz[cz_of(i) + 1]));
        const float v = k == 2 ? (float)Codec<S>::load(p + L.plane[26 - i])
                      : k == 1 ? L.g_face_f[i]
                               : (float)Codec<S>::load(p + (L.plane[i] + ox[cx_of(i) + 1] + oy[cy_of(i) + 1] +
                                                            oz[cz_of(i) + 1]));
        if (H) g[i].y = v;
        else g[i].x = v;
    }
}

// Storage word of two consecutive nodes along x: FP32 as float2 (8 bytes),
// 16-bit as a 4-byte pair; cross(a, b) is the pair (second node of a, first
// node of b).  The word address is even in nodes (n even, every plane and
// row offset even when nx is even), so these are aligned vector accesses.
template <typename S> struct Pair;
template <> struct Pair<float> {
    using W = float2;
    __device__ static W load(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    __device__ static W cross(W a, W b) { return make_float2(a.y, b.x); }
    __device__ static float2 unpack(W w) { return w; }
    __device__ static void store(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
};
template <> struct Pair<__half> {
    using W = __half2;
    __device__ static W load(const __half *p) { return *reinterpret_cast<const __half2 *>(p); }
    __device__ static W cross(W a, W b) { return __halves2half2(__high2half(a), __low2half(b)); }
    __device__ static float2 unpack(W w) { return __half22float2(w); }
    __device__ static void store(__half *p, float2 v) { *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x, v.y); }
};
template <> struct Pair<__nv_bfloat16> {
    using W = __nv_bfloat162;
    __device__ static W load(const __nv_bfloat16 *p) { return *reinterpret_cast<const __nv_bfloat162 *>(p); }
    __device__ static W cross(W a, W b) { return __halves2bfloat162(__high2bfloat16(a), __low2bfloat16(b)); }
    __device__ static float2 unpack(W w) { return __bfloat1622float2(w); }
    __device__ static void store(__nv_bfloat16 *p, float2 v)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v.x, v.y);
    }
};

// Pulls of the node pair (x0, x0 + 1), x0 even, nx even.  Every load of the
// pair is issued in one pass with addresses chosen by selects (a branch there
// would hold back the later loads until the earlier ones return).
//   XPER and YZPER (periodic box): per direction the source word of the pair
//   for c_x = 0, and for c_x = +-1 the pair assembled from two aligned words
//   of the source row (x0 - 2 | x0 and x0 | x0 + 2, wrapped around the row).
//   Otherwise: the source word at x0 and, for c_x = +-1, the outer node as a
//   single element: x0 - 1 or x0 + 2 inside the row, and at an x face the
//   wrapped node (periodic), the node's own opposite population (wall) or the
//   clamped source (outflow).  y and z faces, uniform over the pair's row,
//   are applied after the loads: a wall takes the pair's own opposite word
//   (loaded then), an equilibrium face its value.  A node on an equilibrium x
//   face, or on an x wall of a row with an equilibrium y or z face, is
//   gathered again on its own.
template <typename S, bool XPER, bool YZPER>
__device__ __forceinline__ void gather_pair(const Lattice &L, const S *__restrict__ fa, int x0, int y, int z,
                                            int n0, float2 g[Q])
{
    using P = Pair<S>;
    int oy[3], oz[3], ky[3], kz[3];
    axis_off(y, L.ny, L.nx, L.face[2], L.face[3], oy, ky);
    axis_off(z, L.nz, L.nx * L.ny, L.face[4], L.face[5], oz, kz);
    const S *p = fa + n0;
    if constexpr (XPER && YZPER) {
        const int xl = x0 == 0 ? L.nx - 2 : -2, xr = x0 + 2 >= L.nx ? 2 - L.nx : 2;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = cx_of(i);
            const S *q = p + (L.plane[i] + oy[cy_of(i) + 1] + oz[cz_of(i) + 1]);
            const typename P::W w = P::load(q);
            if (cx == 0) g[i] = P::unpack(w);
            else if (cx > 0) g[i] = P::unpack(P::cross(P::load(q + xl), w));   // sources x0 - 1, x0
            else g[i] = P::unpack(P::cross(w, P::load(q + xr)));               // sources x0 + 1, x0 + 2
        }
    } else {
        // element offsets (from the pair's first node) of the outer node of the
        // c_x = +1 directions (left) and c_x = -1 directions (right): dl / dr
        // relative to the source word, or the own opposite population when
        // own_l / own_r (a wall)
        int dl = -1, dr = 2;
        bool own_l = false, own_r = false, again_l = false, again_r = false;
        const bool eq_yz = !YZPER && ((ky[0] | ky[2] | kz[0] | kz[2]) & 1);
        if (x0 == 0) {
            const int f = L.face[0];
            dl = f == LBM_FACE_PERIODIC ? L.nx - 1 : 0;  // outflow: the clamped source x0
            own_l = f == LBM_FACE_WALL;
            again_l = f == LBM_FACE_EQ || (own_l && eq_yz);
        }
        if (x0 + 2 >= L.nx) {
            const int f = L.face[1];
            dr = f == LBM_FACE_PERIODIC ? 2 - L.nx : 1;  // outflow: the clamped source x0 + 1
            own_r = f == LBM_FACE_WALL;
            again_r = f == LBM_FACE_EQ || (own_r && eq_yz);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = cx_of(i);
            const int src = L.plane[i] + oy[cy_of(i) + 1] + oz[cz_of(i) + 1];
            const float2 m = P::unpack(P::load(p + src));
            if (cx == 0) {
                g[i] = m;
            } else if (cx > 0) {
                const int o = own_l ? L.plane[26 - i] : src + dl;            // source of node x0
                g[i] = make_float2((float)Codec<S>::load(p + o), m.x);
            } else {
                const int o = own_r ? L.plane[26 - i] + 1 : src + dr;        // source of node x0 + 1
                g[i] = make_float2(m.y, (float)Codec<S>::load(p + o));
            }
        }
        if (!YZPER) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int k = max(ky[cy_of(i) + 1], kz[cz_of(i) + 1]);
                if (k == 2) g[i] = P::unpack(P::load(p + L.plane[26 - i]));  // the pair's own bounce-back word
                else if (k == 1) g[i] = make_float2(L.g_face_f[i], L.g_face_f[i]);
            }
        }
        if (again_l) gather_node_lane<S, 0>(L, fa, 0, y, z, n0, g);
        if (again_r) gather_node_lane<S, 1>(L, fa, L.nx - 1, y, z, n0 + 1, g);
    }
}

}  // namespace lbm
