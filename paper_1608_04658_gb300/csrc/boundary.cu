// Moving-wall Grad boundary with KBC collision and momentum exchange, and the
// refill of uncovered nodes (arXiv 1608.04658, Sec. 3, Eqs. grad, pressure,
// pressure2, target velocity/density; Sec. 4.1 Galilean-invariant momentum
// exchange).
//
// One warp per listed node; lane i < 27 owns direction i.  The populations of
// the 3x3x3 neighbourhood that a node needs (itself, its six face neighbours
// for the finite-difference velocity gradient, and x_b + c_i for each missing
// i) are staged in shared memory as [node k][direction i]; lane k then forms
// the density and velocity of neighbourhood node k.  Sums over directions are
// shuffle trees whose lane-0 result is broadcast, so every lane sees the same
// density, velocity and stabilizer.
//
// Readings of points the paper leaves open (the oracle takes the same ones):
//   missing set D = {i : x_b - c_i solid at t+1}; wall point x_w = x_b - q_i c_i;
//   u_f,i from the previous-step state at x_b + c_i, or the wall velocity alone
//   when that node is not fluid; rho_dyn with rho0; f^bb_i = f'_{opp i}(x_b, t);
//   grad u: central difference where both face neighbours are fluid,
//   one-sided where one is, zero otherwise; Pi with rho_tgt and u_tgt; only
//   the missing populations are replaced; the node then collides with KBC.
//   Refill: mean density of the neighbours fluid at t (rho0 if none), the body
//   velocity (the swimmer's material velocity at the node's arc position),
//   gradient with the wall velocity at the centre.
#include "lanes.cuh"

namespace lbm {

// Minimum resident blocks per SM for the boundary and refill kernels: 7
// blocks of 128 threads cap them at 72 registers, so each of their blocks
// takes the registers of one bulk block on the SM it shares with the bulk
// launch beside it.
#ifndef LBM_LIST_MIN_BLOCKS
#define LBM_LIST_MIN_BLOCKS 7
#endif

template <typename S>
__global__ void __launch_bounds__(BWARPS * 32, LBM_LIST_MIN_BLOCKS) boundary_kernel(
    const Lattice L, const GeomParams G, DevBody *__restrict__ b, const int *__restrict__ blist,
    const int *__restrict__ bpos, double *__restrict__ bforce, const S *__restrict__ fa,
    S *__restrict__ fb, const uint8_t *__restrict__ flags)
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
    const R rho0 = (R)L.rho0;

    for (int slot = blockIdx.x * BWARPS + w; slot < count; slot += gridDim.x * BWARPS) {
        const int n = blist[slot];
        int x, y, z;
        node_xyz(L, n, x, y, z);
        const int i = lane;
        const bool act = i < Q;
        const int cx = act ? cx_of(i) : 0, cy = act ? cy_of(i) : 0, cz = act ? cz_of(i) : 0;
        // missing set: directions whose pull source is solid at t+1
        bool solid_src = false;
        if (act && i != 13) {
            const int src = pull_source(L, x, y, z, cx, cy, cz);
            solid_src = src >= 0 && (flags[src] & FL_SOLID);
        }
        const uint32_t mask = __ballot_sync(FULL, solid_src);

        // neighbourhood node k = lane: x_b + c_k
        int nk = -1;
        if (act) nk = neighbour(L, x, y, z, cx, cy, cz);
        if (act) sok[lane] = nk >= 0 && !(flags[nk] & FL_SOLID);
        __syncwarp();
        const uint32_t need = (1u << 13) | (1u << 22) | (1u << 4) | (1u << 16) | (1u << 10) |
                              (1u << 14) | (1u << 12) | mask;
        stage<S, R>(L, fa, lane, nk, need, sf, su, sok);

        const bool miss = act && ((mask >> i) & 1u);
        // known pulled populations (face rules as in the bulk kernel)
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
            else Fi = Codec<S>::load(fa + (size_t)i * N + (p[0] + L.nx * (p[1] + L.ny * p[2])));
        }
        // target density and velocity over the missing set
        const R fbb = act ? sf[13][26 - (act ? i : 0)] : R(0);  // shifted f'_{opp i}(x_b, t)
        double q = 0, uw[3] = {0, 0, 0};
        if (G.kind == LBM_BODY_MESH) {
            MeshHit hit{-1, 0.0, 0.0};
            mesh_links_warp<R>(G, b, x, y, z, mask, lane, q, uw, hit);
        } else if (miss) {
            link_data<R>(L, G, b, x, y, z, cx, cy, cz, q, uw);
        }
        const R gstat = miss ? fbb : Fi;
        const R dyn = miss ? R(6) * weight<R>(i) * rho0 * (R(cx) * (R)uw[0] + R(cy) * (R)uw[1] + R(cz) * (R)uw[2])
                           : R(0);
        R ut[3] = {0, 0, 0};
        if (miss) {
            const R qq = (R)q;
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
        pressure_excess<R>(rho_t, u_t, du, (R)L.beta, Qt);
        R gi = Fi;
        if (miss) gi = grad_shifted<R>(i, rho_t, rho0, u_t, Qt);

        // momentum exchange on missing links (FP64): the fluid hands the body
        // (c_opp - u_w) f'_opp(x_b, t) and gets back (c_i - u_w) F_i(x_b, t+1)
        double dF[6] = {0, 0, 0, 0, 0, 0};
        if (miss) {
            const double W = weight<double>(i) * L.rho0;
            const double fout = (double)fbb + W, fin = (double)gi + W;
            const double c[3] = {(double)cx, (double)cy, (double)cz};
            for (int a = 0; a < 3; ++a) dF[a] = (-c[a] - uw[a]) * fout - (c[a] - uw[a]) * fin;
            double r[3];
            r[0] = body_offset(L, G, b, 0, x) - q * c[0];
            r[1] = body_offset(L, G, b, 1, y) - q * c[1];
            r[2] = body_offset(L, G, b, 2, z) - q * c[2];
            dF[3] = r[1] * dF[2] - r[2] * dF[1];
            dF[4] = r[2] * dF[0] - r[0] * dF[2];
            dF[5] = r[0] * dF[1] - r[1] * dF[0];
        }
        const int pos = bpos[slot];
        // a slab's links count where it owns the fluid node
        const bool own = z >= G.own_lo && z < G.own_hi;
        for (int k = 0; k < 6; ++k) {
            double v = dF[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
            if (lane == 0) bforce[(size_t)pos * 6 + k] = own ? v : 0.0;
        }

        bool ok;
        const R out = kbc_collide_lanes<R>(gi, i, (R)L.beta, (R)L.inv_beta, rho0, L.gamma_mode, ok);
        if (lane == 0 && !ok) atomicOr(&b->status, ST_UNSTABLE);
        if (act) Codec<S>::store(fb + (size_t)i * N + n, out);
        __syncwarp();
    }
}

template <typename S>
__global__ void __launch_bounds__(BWARPS * 32, LBM_LIST_MIN_BLOCKS) refill_kernel(
    const Lattice L, const GeomParams G, const DevBody *__restrict__ b, const int *__restrict__ ulist,
    S *__restrict__ fa, const uint8_t *__restrict__ flags)
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
    const size_t N = (size_t)L.N;
    const R rho0 = (R)L.rho0;
    for (int slot = blockIdx.x * BWARPS + w; slot < count; slot += gridDim.x * BWARPS) {
        const int n = ulist[slot];
        int x, y, z;
        node_xyz(L, n, x, y, z);
        const bool act = lane < Q;
        int nk = -1;
        if (act && lane != 13) nk = neighbour(L, x, y, z, cx_of(lane), cy_of(lane), cz_of(lane));
        // neighbours that were fluid at t carry valid populations
        if (act) sok[lane] = nk >= 0 && !(flags[nk] & FL_SOLID_PREV);
        __syncwarp();
        uint32_t need = __ballot_sync(FULL, act && sok[lane]);
        stage<S, R>(L, fa, lane, nk, need, sf, su, sok);
        const R cnt = R(__popc(need));
        const R rsum = wsum((act && sok[lane]) ? su[lane][0] : R(0));
        const R rho = cnt > R(0) ? rsum / cnt : rho0;
        R u[3] = {(R)b->U[0], (R)b->U[1], (R)b->U[2]};
        if (G.kind == LBM_BODY_PLANES) {
            const double *v = (double)y < 0.5 * (G.y_lo + G.y_hi) ? G.U_lo : G.U_hi;
            u[0] = (R)v[0]; u[1] = (R)v[1]; u[2] = (R)v[2];
        } else if (G.kind == LBM_BODY_MESH) {
            // material velocity of the swimmer at the node's arc position
            double v[3];
            mesh_material_velocity(G, b, (double)x, (double)y, v);
            u[0] = (R)v[0]; u[1] = (R)v[1]; u[2] = (R)v[2];
        }
        R du[3][3], Qt[6];
        fd_gradient<R>(su, sok, u, du);
        pressure_excess<R>(rho, u, du, (R)L.beta, Qt);
        if (act) Codec<S>::store(fa + (size_t)lane * N + n, grad_shifted<R>(lane, rho, rho0, u, Qt));
        __syncwarp();
    }
}

// ----------------------------------------------------------------- launchers

// Grid of the list kernels (grid-stride over the list).  The boundary kernel
// runs beside the bulk kernel, and every resident block of it holds shared
// memory and registers the bulk kernel could use; LBM_LIST_BLOCKS caps the
// grid (build-time knob; two blocks per SM measured best for the sphere and
// the airfoil with the 72-register cap, FP16 sphere step 0.178 -> 0.167 ms
// against one block per SM).
#ifndef LBM_LIST_BLOCKS
#define LBM_LIST_BLOCKS 304
#endif
// The swimmer's boundary nodes each carry a triangle search, so its
// boundary kernel is the long part of the body's launch chain:
// LBM_MESH_LIST_BLOCKS gives it more blocks (608 took the 256x128x128
// swimmer's step from 0.359 to 0.256 ms).
#ifndef LBM_MESH_LIST_BLOCKS
#define LBM_MESH_LIST_BLOCKS 608
#endif
static int list_blocks(int cap, int max_blocks = LBM_LIST_BLOCKS)
{
    int nb = (cap + BWARPS - 1) / BWARPS;
    return nb < 1 ? 1 : (nb > max_blocks ? max_blocks : nb);
}

cudaError_t launch_boundary(int storage, const Lattice &L, const GeomParams &G, Scratch &S, int cur,
                            const void *fa, void *fb, const uint8_t *flags, cudaStream_t s)
{
    return dispatch_storage(storage, [&](auto tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        const int nb = list_blocks(G.cap_boundary, G.kind == LBM_BODY_MESH ? LBM_MESH_LIST_BLOCKS : LBM_LIST_BLOCKS);
        boundary_kernel<T><<<nb, BWARPS * 32, 0, s>>>(L, G, S.body + cur, S.blist, S.bpos, S.bforce, (const T *)fa,
                                                      (T *)fb, flags);
        return cudaGetLastError();
    });
}

cudaError_t launch_refill(int storage, const Lattice &L, const GeomParams &G, Scratch &S, int cur, void *fa,
                          const uint8_t *flags, cudaStream_t s)
{
    return dispatch_storage(storage, [&](auto tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        refill_kernel<T><<<list_blocks(G.cap_uncovered), BWARPS * 32, 0, s>>>(L, G, S.body + cur, S.ulist,
                                                                               (T *)fa, flags);
        return cudaGetLastError();
    });
}

}  // namespace lbm
