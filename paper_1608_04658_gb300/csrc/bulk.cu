// Bulk fused pull-stream + KBC collide (arXiv 1608.04658, Sec. 2, Eq. kineticEq
// with Eq. kbc_relax).
//
// One thread per node, threads along x (the fastest axis of every population
// plane) so each of the 27 plane loads and stores of a warp is one contiguous
// run; the +-1 x-shift of a pull touches one extra 32-byte sector per warp,
// which the neighbouring warp reads anyway, so DRAM traffic stays at one read
// and one write per population.  Nodes marked SOLID or BOUNDARY are left to
// the boundary kernel.  With a body, one launch takes the nodes outside the
// body's sweep box (no flag read) while the body's geometry runs beside it,
// and a second the nodes of the box once their marks are known.
#include <algorithm>
#include <type_traits>

#include "pull.cuh"

namespace lbm {

// Minimum resident blocks per SM requested from the register allocator: 7
// blocks of 128 threads cap the kernel at 72 registers (no spill) and give
// 28 warps per SM, which measured faster on GB300 than 80 registers with 6
// blocks or 64 registers with 8.
#ifndef LBM_BULK_MIN_BLOCKS
#define LBM_BULK_MIN_BLOCKS 7
#endif
// The exact stabilizer's Newton iteration and FP64 storage's double
// arithmetic spill heavily at 72 registers (280 and 1080 bytes of stack,
// traffic that reaches DRAM); they get fewer, wider blocks.
#ifndef LBM_BULK_MIN_BLOCKS_WIDE
#define LBM_BULK_MIN_BLOCKS_WIDE 4
#endif
template <typename S, bool EXACT>
struct BulkBlocks {
    static constexpr int value =
        (EXACT || std::is_same<S, double>::value) ? LBM_BULK_MIN_BLOCKS_WIDE : LBM_BULK_MIN_BLOCKS;
};

// Resident blocks per SM asked of the register allocator for the two-node
// kernel (64 threads, 128 nodes per block): 8 for FP32 storage, 7 for 16-bit
// storage; both then fit in 128 registers without spilling (the collision
// forms the equilibrium factors again after its scalar products instead of
// keeping them live), 16 warps per SM.  Measured on GB300 (swimmer box,
// fraction of the copy bandwidth): FP32 0.944 at 8 blocks against 0.896 at
// 6 (166 registers, 12 warps); FP16 0.576 at 7 against 0.452 at 9.
#ifndef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_MIN_BLOCKS 8
#endif
#ifndef LBM_PAIR_MIN_BLOCKS_16
#define LBM_PAIR_MIN_BLOCKS_16 7
#endif
template <typename S>
struct PairBlocks {
    static constexpr int value = sizeof(S) == 2 ? LBM_PAIR_MIN_BLOCKS_16 : LBM_PAIR_MIN_BLOCKS;
};
// FP32 storage takes the two-node kernel too (0: the one-node kernel with the
// same arithmetic)
#ifndef LBM_PAIR_FP32
#define LBM_PAIR_FP32 1
#endif

// VMATH: the collision with explicit FP32 operations (kbc_collide_v), which
// the two-node kernel shares bit for bit; otherwise kbc_collide (FP64
// storage, exact stabilizer).
template <typename S, bool EXACT, bool VMATH>
__global__ void __launch_bounds__(128, (BulkBlocks<S, EXACT>::value)) bulk_kernel(const Lattice L, const S *__restrict__ fa,
                                                   S *__restrict__ fb,
                                                   const uint8_t *__restrict__ flags,
                                                   int *__restrict__ status,
                                                   const int *__restrict__ sweep, int mode, int capx,
                                                   int capy, int z0)
{
    using R = typename Codec<S>::R;
    int x, y, z;
    if (mode == BULK_BAND) {
        // one thread per position of the capacity box, x fastest
        const int k = blockIdx.x * blockDim.x + threadIdx.x;
        const int lx = k % capx, ly = (k / capx) % capy, lz = k / (capx * capy);
        if (lx >= sweep[3] || ly >= sweep[4] || lz >= sweep[5]) return;
        x = sweep_coord(sweep[0] + lx, L.nx);
        y = sweep_coord(sweep[1] + ly, L.ny);
        z = sweep_coord(sweep[2] + lz, L.nz);
    } else {
        x = blockIdx.x * blockDim.x + threadIdx.x;
        y = blockIdx.y;
        z = z0 + (int)blockIdx.z;
        if (x >= L.nx) return;
        // y and z are uniform over the block, so only rows crossing the box
        // test x
        if (mode == BULK_OUTSIDE && in_sweep(sweep, 1, y, L.ny, L.face[2] == LBM_FACE_PERIODIC) &&
            in_sweep(sweep, 2, z, L.nz, L.face[4] == LBM_FACE_PERIODIC) &&
            in_sweep(sweep, 0, x, L.nx, L.face[0] == LBM_FACE_PERIODIC))
            return;
    }
    const int nx = L.nx, ny = L.ny;
    const int n = x + nx * (y + ny * z);
    if (flags != nullptr && (flags[n] & (FL_SOLID | FL_BOUNDARY))) return;

    // all 27 pulls are issued unconditionally (wall/equilibrium sources read
    // the node itself and are replaced afterwards)
    R g[Q];
    gather_global<S>(L, fa, x, y, z, n, g);
    bool ok;
    if constexpr (VMATH) ok = kbc_collide_v<F1>(g, L.beta_f, L.inv_beta_f, L.rho0_f, L.gamma_mode) & 1;
    else ok = kbc_collide<R, EXACT>(g, (R)L.beta, (R)L.inv_beta, (R)L.rho0, L.gamma_mode);
    if (!ok) atomicOr(status, ST_UNSTABLE);
    S *q = fb + n;
#pragma unroll
    for (int i = 0; i < Q; ++i) Codec<S>::store(q + L.plane[i], g[i]);
}

// Two nodes per thread, (x0, x0 + 1) with x0 even, for even nx: each pull
// is an aligned word of the pair (two for c_x = +-1), the collision runs on
// both nodes in packed FP32x2 arithmetic, each store writes the pair's word.
// Node selection as in bulk_kernel (ALL or OUTSIDE; the sweep box takes the
// one-node kernel), per node of the pair.  XPER: the x axis is periodic;
// YZPER: the y and z axes are.
template <typename S, bool XPER, bool YZPER>
__device__ __forceinline__ void pair_update(const Lattice &L, const S *__restrict__ fa, S *__restrict__ fb,
                                            const uint8_t *__restrict__ flags, int *__restrict__ status,
                                            const int *__restrict__ sweep, int mode, int x0, int y, int z)
{
    int act = 3;  // bit 0: node x0 is updated here, bit 1: node x0 + 1
    if (mode == BULK_OUTSIDE && in_sweep(sweep, 1, y, L.ny, L.face[2] == LBM_FACE_PERIODIC) &&
        in_sweep(sweep, 2, z, L.nz, L.face[4] == LBM_FACE_PERIODIC)) {
        act = (in_sweep(sweep, 0, x0, L.nx, XPER) ? 0 : 1) | (in_sweep(sweep, 0, x0 + 1, L.nx, XPER) ? 0 : 2);
        if (!act) return;
    }
    const int n0 = x0 + L.nx * (y + L.ny * z);
    if (flags != nullptr) {
        const unsigned fw = *reinterpret_cast<const unsigned short *>(flags + n0);
        if (fw & (FL_SOLID | FL_BOUNDARY)) act &= ~1;
        if ((fw >> 8) & (FL_SOLID | FL_BOUNDARY)) act &= ~2;
        if (!act) return;
    }
    float2 g[Q];
    gather_pair<S, XPER, YZPER>(L, fa, x0, y, z, n0, g);
    const int ok = kbc_collide_v<F2>(g, L.beta_f, L.inv_beta_f, L.rho0_f, L.gamma_mode);
    if (act & ~ok) atomicOr(status, ST_UNSTABLE);
    S *q = fb + n0;
    if (act == 3) {
#pragma unroll
        for (int i = 0; i < Q; ++i) Pair<S>::store(q + L.plane[i], g[i]);
    } else if (act == 1) {
#pragma unroll
        for (int i = 0; i < Q; ++i) Codec<S>::store(q + L.plane[i], g[i].x);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) Codec<S>::store(q + 1 + L.plane[i], g[i].y);
    }
}

// One block per 128 nodes of a row.  A row that touches no y or z face
// other than a periodic one pulls only from inside the box along y and z, so
// it takes the y/z-periodic form of the gather whatever the box's y and z
// faces are (the choice is uniform over the block).
template <typename S, bool XPER, bool YZPER>
__global__ void __launch_bounds__(64, PairBlocks<S>::value) bulk_pair_kernel(const Lattice L,
                                                                           const S *__restrict__ fa,
                                                                           S *__restrict__ fb,
                                                                           const uint8_t *__restrict__ flags,
                                                                           int *__restrict__ status,
                                                                           const int *__restrict__ sweep, int mode,
                                                                           int z0)
{
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= L.nx) return;
    const int y = blockIdx.y, z = z0 + (int)blockIdx.z;
    if constexpr (!YZPER) {
        const bool face_row = (L.face[2] != LBM_FACE_PERIODIC && (y == 0 || y == L.ny - 1)) ||
                              (L.face[4] != LBM_FACE_PERIODIC && (z == 0 || z == L.nz - 1));
        if (!face_row) {
            pair_update<S, XPER, true>(L, fa, fb, flags, status, sweep, mode, x0, y, z);
            return;
        }
    }
    pair_update<S, XPER, YZPER>(L, fa, fb, flags, status, sweep, mode, x0, y, z);
}

// ----------------------------------------------------------------- launchers
cudaError_t launch_bulk(int storage, const Lattice &L, const void *fa, void *fb,
                        const uint8_t *flags, int *status, cudaStream_t s, int mode, const int *sweep,
                        const int *cap, int z_lo, int z_n)
{
    if (mode != BULK_ALL && (!sweep || (mode == BULK_BAND && !cap))) return cudaErrorInvalidValue;
    if (z_n < 0) z_n = L.nz - z_lo;
    if (z_lo < 0 || z_lo + z_n > L.nz) return cudaErrorInvalidValue;
    if (z_n == 0 && mode != BULK_BAND) return cudaSuccess;
    return dispatch_storage(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        int bx = L.nx >= 128 ? 128 : ((L.nx + 31) / 32) * 32;
        dim3 grid((L.nx + bx - 1) / bx, L.ny, z_n);
        int capx = 1, capy = 1;
        if (mode == BULK_BAND) {
            bx = 128;
            capx = cap[0];
            capy = cap[1];
            const long long vol = (long long)cap[0] * cap[1] * cap[2];
            grid = dim3((unsigned)((vol + bx - 1) / bx), 1, 1);
        }
        // the exact stabilizer and FP64 storage keep kbc_collide; FP32 and
        // 16-bit storage with the analytic (or LBGK) stabilizer take the
        // explicit-operation collision, in the two-node kernel where the row
        // length allows (every node gets the same bits either way)
        constexpr bool VM = !std::is_same<S, double>::value;
        constexpr bool PAIR = VM && (LBM_PAIR_FP32 || !std::is_same<S, float>::value);
        if (L.gamma_mode == LBM_GAMMA_EXACT) {
            bulk_kernel<S, true, false><<<grid, bx, 0, s>>>(L, (const S *)fa, (S *)fb, flags, status, sweep, mode,
                                                            capx, capy, z_lo);
            return cudaGetLastError();
        }
        if constexpr (PAIR) {
            if (mode != BULK_BAND && (L.nx & 1) == 0) {
                const int kind = (L.face[0] == LBM_FACE_PERIODIC ? 1 : 0) +
                                 (L.face[2] == LBM_FACE_PERIODIC && L.face[4] == LBM_FACE_PERIODIC ? 2 : 0);
                auto kernel = kind == 3 ? bulk_pair_kernel<S, true, true>
                            : kind == 2 ? bulk_pair_kernel<S, false, true>
                            : kind == 1 ? bulk_pair_kernel<S, true, false>
                                        : bulk_pair_kernel<S, false, false>;
                const dim3 g2((L.nx + 127) / 128, L.ny, z_n);
                kernel<<<g2, 64, 0, s>>>(L, (const S *)fa, (S *)fb, flags, status, sweep, mode, z_lo);
                return cudaGetLastError();
            }
        }
        bulk_kernel<S, false, VM><<<grid, bx, 0, s>>>(L, (const S *)fa, (S *)fb, flags, status, sweep, mode,
                                                      capx, capy, z_lo);
        return cudaGetLastError();
    });
}

}  // namespace lbm
