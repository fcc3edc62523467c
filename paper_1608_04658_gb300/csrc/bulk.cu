// Bulk fused pull-stream + KBC collide (arXiv 1608.04658, Sec. 2, Eq. kineticEq
// with Eq. kbc_relax), plus state initialisation, plane codec and totals.
//
// One thread per node, threads along x (the fastest axis of every population
// plane) so each of the 27 plane loads and stores of a warp is one contiguous
// run; the +-1 x-shift of a pull touches one extra 32-byte sector per warp,
// which the neighbouring warp reads anyway, so DRAM traffic stays at one read
// and one write per population.  Nodes marked SOLID or BOUNDARY are left to
// the boundary kernel.
#include <type_traits>

#include "kbc2.cuh"

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
    if (kx[0] | kx[2] | ky[0] | ky[2] | kz[0] | kz[2]) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int k = max(kx[cx_of(i) + 1], max(ky[cy_of(i) + 1], kz[cz_of(i) + 1]));
            if (k == 2) g[i] = Codec<S>::load(p + L.plane[26 - i]);
            else if (k == 1) g[i] = (R)L.g_face[i];
        }
    }
}

template <typename S>
__global__ void __launch_bounds__(128) bulk_kernel(const Lattice L, const S *__restrict__ fa,
                                                   S *__restrict__ fb,
                                                   const uint8_t *__restrict__ flags,
                                                   int *__restrict__ status)
{
    using R = typename Codec<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    const int nx = L.nx, ny = L.ny;
    const int n = x + nx * (y + ny * z);
    if (flags != nullptr && (flags[n] & (FL_SOLID | FL_BOUNDARY))) return;

    // all 27 pulls are issued unconditionally (wall/equilibrium sources read
    // the node itself and are replaced afterwards)
    R g[Q];
    gather_global<S>(L, fa, x, y, z, n, g);
    const bool ok = kbc_collide<R>(g, (R)L.beta, (R)L.inv_beta, (R)L.rho0, L.gamma_mode);
    if (!ok) atomicOr(status, ST_UNSTABLE);
    S *q = fb + n;
#pragma unroll
    for (int i = 0; i < Q; ++i) Codec<S>::store(q + L.plane[i], g[i]);
}

// ------------------------------------------------------------- pipelined bulk
// Warp-specialised, persistent version of the same step.  A work item is a
// segment of ITEM = 32 * NCW nodes of one x-row.  Warp 0 is the producer: for
// an item it arms the stage's "full" mbarrier with the byte count, lanes 0..26
// each issue one bulk asynchronous copy (cp.async.bulk, completion counted on
// that mbarrier) of the source row segment of direction i, x-range
// [x0 - H, x0 + ITEM + H) clipped to the row (H = 16 bytes of halo so every
// copy starts and ends on a 16-byte boundary), and lanes resolve the x-face
// values (wall, equilibrium, periodic, outflow) of the segment's first and
// last node into a small edge area.  Warps 1..NCW are consumers, one node per
// thread: they wait on "full", read their 27 pulls from shared memory, release
// the stage on its "empty" mbarrier and collide.  With D stages the copies run
// D - 1 items ahead of the collision, so memory latency no longer depends on
// how many warps fit on an SM.  Items whose row lies on a non-periodic y/z
// face carry no copies; their consumers gather from global memory with the
// general face rules.  Every wait is bounded: on timeout the status word gets
// ST_TIMEOUT and the CTA returns after a bounded wait for its copies in flight.
constexpr long long WAIT_BUDGET = 4000000000LL;  // cycles

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > WAIT_BUDGET) return false;
    return true;
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_mbarrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// consumers handle NPT nodes each: 2 (packed FP32x2 collision) for FP32 and
// 16-bit storage, 1 for FP64
template <typename S> struct PipeShape {
    static constexpr int NPT = std::is_same_v<S, double> ? 1 : 2;
    static constexpr int NCW = std::is_same_v<S, double> ? 4 : 2;
};

template <typename S>
struct PipeCfg {
    using R = typename Codec<S>::R;
    static constexpr int NPT = PipeShape<S>::NPT, NCW = PipeShape<S>::NCW;
    static constexpr int H = 16 / (int)sizeof(S);
    static constexpr int ITEM = 32 * NCW * NPT;
    static constexpr int SEG = ITEM + 2 * H;
    static constexpr int D = sizeof(S) >= 4 ? 3 : 4;
    static constexpr size_t ROWS_BYTES = (size_t)Q * SEG * sizeof(S);  // multiple of 16
    static constexpr size_t EDGE_BYTES = (size_t)Q * 2 * sizeof(R);
    static constexpr size_t SMEM = D * (ROWS_BYTES + EDGE_BYTES);
    static constexpr int THREADS = 32 * (NCW + 1);
};

__device__ __forceinline__ bool row_on_yz_face(const Lattice &L, int y, int z)
{
    const bool fy = L.face[2] != LBM_FACE_PERIODIC && (y == 0 || y == L.ny - 1);
    const bool fz = L.face[4] != LBM_FACE_PERIODIC && (z == 0 || z == L.nz - 1);
    return fy || fz;
}

template <typename S>
__device__ __forceinline__ float2 smem_pair(const S *p);
template <> __device__ __forceinline__ float2 smem_pair<float>(const float *p)
{
    return *reinterpret_cast<const float2 *>(p);
}
template <> __device__ __forceinline__ float2 smem_pair<__half>(const __half *p)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
template <> __device__ __forceinline__ float2 smem_pair<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
}
template <typename S>
__device__ __forceinline__ void store_pair(S *p, float2 v);
template <> __device__ __forceinline__ void store_pair<float>(float *p, float2 v)
{
    *reinterpret_cast<float2 *>(p) = v;
}
template <> __device__ __forceinline__ void store_pair<__half>(__half *p, float2 v)
{
    *reinterpret_cast<__half2 *>(p) = __float22half2_rn(v);
}
template <> __device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16 *p, float2 v)
{
    *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(v);
}

template <typename S>
__global__ void __launch_bounds__(PipeCfg<S>::THREADS, 4) bulk_pipelined_kernel(
    const Lattice L, const S *__restrict__ fa, S *__restrict__ fb, const uint8_t *__restrict__ flags,
    int *__restrict__ status)
{
    using Cfg = PipeCfg<S>;
    using R = typename Cfg::R;
    constexpr int H = Cfg::H, ITEM = Cfg::ITEM, SEG = Cfg::SEG, D = Cfg::D, NCW = Cfg::NCW, NPT = Cfg::NPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S *rows = reinterpret_cast<S *>(smem_raw);                               // [D][Q][SEG]
    R *edges = reinterpret_cast<R *>(smem_raw + D * Cfg::ROWS_BYTES);        // [D][Q][2]
    __shared__ __align__(8) uint64_t full[D], empty[D];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = L.nx, ny = L.ny;
    const int nseg = (nx + ITEM - 1) / ITEM;
    const int items = ny * L.nz * nseg;
    if (threadIdx.x == 0) {
        for (int s = 0; s < D; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        fence_mbarrier_init();
    }
    __syncthreads();

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        int k = 0;
        for (int j = blockIdx.x; j < items; j += gridDim.x, ++k) {
            const int s = k % D;
            const uint32_t ph = (uint32_t)(k / D) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u)) {
                if (lane == 0) atomicOr(status, ST_TIMEOUT);
                // copies of earlier items may still be in flight
                for (int m = (k >= D ? k - D + 1 : 0); m < k; ++m) mbar_wait(&full[m % D], (uint32_t)(m / D) & 1u);
                return;
            }
            const int r = j / nseg, x0 = (j % nseg) * ITEM;
            const int y = r % ny, z = r / ny;
            const bool staged = !row_on_yz_face(L, y, z);
            const int lo = max(x0 - H, 0), hi = min(x0 + ITEM + H, nx);
            const uint32_t bytes = (uint32_t)(hi - lo) * (uint32_t)sizeof(S);
            if (staged && lane == 0) mbar_expect_tx(&full[s], bytes * Q);
            __syncwarp();
            if (staged) {
                if (lane < Q) {
                    const int i = lane;
                    int ys = y - cy_of(i), zs = z - cz_of(i);
                    if (ys < 0) ys += ny; else if (ys >= ny) ys -= ny;
                    if (zs < 0) zs += L.nz; else if (zs >= L.nz) zs -= L.nz;
                    const S *src = fa + L.plane[i] + (zs * ny + ys) * nx + lo;
                    bulk_copy_g2s(rows + (size_t)s * Q * SEG + i * SEG + (lo - (x0 - H)), src, bytes, &full[s]);
                }
                // x-face values: lanes 0..8 the last node of the row (c_x = -1,
                // i = lane), lanes 9..17 the first node (c_x = +1, i = lane + 9)
                const bool left = x0 == 0, right = x0 + ITEM >= nx;
                if ((lane < 9 && right) || (lane >= 9 && lane < 18 && left)) {
                    const int i = lane < 9 ? lane : lane + 9;
                    const int xn = lane < 9 ? nx - 1 : 0;  // node on the face
                    const int face = lane < 9 ? L.face[1] : L.face[0];
                    int ys = y - cy_of(i), zs = z - cz_of(i);
                    if (ys < 0) ys += ny; else if (ys >= ny) ys -= ny;
                    if (zs < 0) zs += L.nz; else if (zs >= L.nz) zs -= L.nz;
                    const S *srow = fa + L.plane[i] + (zs * ny + ys) * nx;
                    R v;
                    if (face == LBM_FACE_PERIODIC) v = Codec<S>::load(srow + (lane < 9 ? 0 : nx - 1));
                    else if (face == LBM_FACE_OUTFLOW) v = Codec<S>::load(srow + xn);
                    else if (face == LBM_FACE_WALL) v = Codec<S>::load(fa + L.plane[26 - i] + (z * ny + y) * nx + xn);
                    else v = (R)L.g_face[i];
                    edges[((size_t)s * Q + i) * 2 + (lane < 9 ? 1 : 0)] = v;
                }
            }
            __syncwarp();
            __threadfence_block();
            if (lane == 0) mbar_arrive(&full[s]);
        }
        return;
    }

    // -------------------------------------------------------------- consumers
    const int c = warp - 1;
    int k = 0;
    for (int j = blockIdx.x; j < items; j += gridDim.x, ++k) {
        const int s = k % D;
        const uint32_t ph = (uint32_t)(k / D) & 1u;
        if (!mbar_wait(&full[s], ph)) {
            if (lane == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
        const int r = j / nseg, x0 = (j % nseg) * ITEM;
        const int y = r % ny, z = r / ny;
        const int t = c * 32 + lane;
        const int x = x0 + NPT * t;
        const bool staged = !row_on_yz_face(L, y, z);
        const S *sb = rows + (size_t)s * Q * SEG + H + NPT * t;
        const R *eb = edges + (size_t)s * Q * 2;
        if constexpr (NPT == 1) {
            bool active = x < nx;
            int n = 0;
            if (active) {
                n = x + nx * (y + ny * z);
                if (flags != nullptr && (flags[n] & (FL_SOLID | FL_BOUNDARY))) active = false;
            }
            R g[Q];
            if (active && staged) {
#pragma unroll
                for (int i = 0; i < Q; ++i) g[i] = Codec<S>::load(sb + i * SEG - cx_of(i));
                if (x == 0) {
#pragma unroll
                    for (int i = 18; i < Q; ++i) g[i] = eb[i * 2 + 0];
                }
                if (x == nx - 1) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = eb[i * 2 + 1];
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (!active) continue;
            if (!staged) gather_global<S>(L, fa, x, y, z, n, g);
            const bool ok = kbc_collide<R>(g, (R)L.beta, (R)L.inv_beta, (R)L.rho0, L.gamma_mode);
            if (!ok) atomicOr(status, ST_UNSTABLE);
            S *q = fb + n;
#pragma unroll
            for (int i = 0; i < Q; ++i) Codec<S>::store(q + L.plane[i], g[i]);
        } else {
            // nodes x and x + 1 (nx is even on this path)
            const bool inrange = x < nx;
            int n = 0;
            bool act0 = inrange, act1 = inrange;
            if (inrange) {
                n = x + nx * (y + ny * z);
                if (flags != nullptr) {
                    const uint16_t fl = *reinterpret_cast<const uint16_t *>(flags + n);
                    act0 = !((fl & 0xff) & (FL_SOLID | FL_BOUNDARY));
                    act1 = !((fl >> 8) & (FL_SOLID | FL_BOUNDARY));
                }
            }
            float2 g[Q];
            if ((act0 || act1) && staged) {
                static_for<0>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    constexpr int cx = cx_of(i);
                    if constexpr (cx == 0) g[i] = smem_pair<S>(sb + i * SEG);
                    else g[i] = make_float2((float)Codec<S>::load(sb + i * SEG - cx),
                                            (float)Codec<S>::load(sb + i * SEG + 1 - cx));
                });
                if (x == 0) {
#pragma unroll
                    for (int i = 18; i < Q; ++i) g[i].x = eb[i * 2 + 0];
                }
                if (x + 1 == nx - 1) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i].y = eb[i * 2 + 1];
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (!(act0 || act1)) continue;
            if (!staged) {
                float ga[Q], gb[Q];
                gather_global<S>(L, fa, x, y, z, n, ga);
                gather_global<S>(L, fa, x + 1, y, z, n + 1, gb);
#pragma unroll
                for (int i = 0; i < Q; ++i) g[i] = make_float2(ga[i], gb[i]);
            }
            bool ok0, ok1;
            kbc_collide2(g, (float)L.beta, (float)L.inv_beta, (float)L.rho0, L.gamma_mode, ok0, ok1);
            if ((act0 && !ok0) || (act1 && !ok1)) atomicOr(status, ST_UNSTABLE);
            S *q = fb + n;
            if (act0 && act1) {
#pragma unroll
                for (int i = 0; i < Q; ++i) store_pair<S>(q + L.plane[i], g[i]);
            } else if (act0) {
#pragma unroll
                for (int i = 0; i < Q; ++i) Codec<S>::store(q + L.plane[i], g[i].x);
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) Codec<S>::store(q + 1 + L.plane[i], g[i].y);
            }
        }
    }
}

template <typename S>
static cudaError_t launch_pipelined(const Lattice &L, const S *fa, S *fb, const uint8_t *flags, int *status,
                                    cudaStream_t s)
{
    using Cfg = PipeCfg<S>;
    static int grid_cap = -1;
    if (grid_cap < 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(bulk_pipelined_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bulk_pipelined_kernel<S>, Cfg::THREADS,
                                                          Cfg::SMEM) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        grid_cap = sms * per_sm;
    }
    const int items = L.ny * L.nz * ((L.nx + Cfg::ITEM - 1) / Cfg::ITEM);
    const int grid = items < grid_cap ? items : grid_cap;
    bulk_pipelined_kernel<S><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(L, fa, fb, flags, status);
    return cudaGetLastError();
}

bool pipelined_eligible(int storage, const Lattice &L)
{
    const int es = storage == LBM_FP64 ? 8 : (storage == LBM_FP32 ? 4 : 2);
    return L.nx >= 2 && (L.nx * es) % 16 == 0;
}

template <typename S>
__global__ void init_kernel(const Lattice L, S *__restrict__ f, const double *__restrict__ rho,
                            const double *__restrict__ u, const double *__restrict__ xi, double amp)
{
    using R = typename Codec<S>::R;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    // equilibrium evaluated in double, then rounded once to storage
    double ex[3], ey[3], ez[3], rx[3], ry[3], rz[3];
    axis_eq<double>(u[3 * n + 0], ex, rx);
    axis_eq<double>(u[3 * n + 1], ey, ry);
    axis_eq<double>(u[3 * n + 2], ez, rz);
    const double r = rho[n], drho = r - L.rho0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        double g = shifted_feq<double>(i, drho, r, ex, ey, ez);
        if (xi) g += amp * weight<double>(i) * xi[(size_t)i * L.N + n];
        Codec<S>::store(f + (size_t)i * L.N + n, (R)g);
    }
}

template <typename S>
__global__ void decode_kernel(const Lattice L, const S *__restrict__ f, int i, double *__restrict__ out)
{
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    out[n] = (double)Codec<S>::load(f + (size_t)i * L.N + n) + weight<double>(i) * L.rho0;
}

template <typename S>
__global__ void encode_kernel(const Lattice L, S *__restrict__ f, int i, const double *__restrict__ in)
{
    using R = typename Codec<S>::R;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    Codec<S>::store(f + (size_t)i * L.N + n, (R)(in[n] - weight<double>(i) * L.rho0));
}

// Per-block FP64 partial sums of mass, momentum and kinetic energy over
// non-solid nodes; the host adds the block partials in block order.
template <typename S>
__global__ void __launch_bounds__(256) totals_kernel(const Lattice L, const S *__restrict__ f,
                                                     const uint8_t *__restrict__ flags,
                                                     double *__restrict__ partials)
{
    double acc[5] = {0, 0, 0, 0, 0};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < L.N;
         n += (long long)gridDim.x * blockDim.x) {
        if (flags && (flags[n] & FL_SOLID)) continue;
        double r = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            const double v = (double)Codec<S>::load(f + (size_t)i * L.N + n) + weight<double>(i) * L.rho0;
            r += v;
            j[0] += cx_of(i) * v;
            j[1] += cy_of(i) * v;
            j[2] += cz_of(i) * v;
        }
        acc[0] += r;
        acc[1] += j[0];
        acc[2] += j[1];
        acc[3] += j[2];
        acc[4] += 0.5 * (j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / r;
    }
    __shared__ double sm[8][5];
    for (int k = 0; k < 5; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sm[w][threadIdx.x];
        partials[blockIdx.x * 5 + threadIdx.x] = v;
    }
}

// ----------------------------------------------------------------- launchers
template <typename F>
static cudaError_t dispatch(int storage, F &&fn)
{
    switch (storage) {
    case LBM_FP64: return fn((double *)nullptr);
    case LBM_FP32: return fn((float *)nullptr);
    case LBM_FP16: return fn((__half *)nullptr);
    case LBM_BF16: return fn((__nv_bfloat16 *)nullptr);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bulk(int storage, const Lattice &L, const void *fa, void *fb,
                        const uint8_t *flags, int *status, cudaStream_t s)
{
    return dispatch(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (L.pipelined) return launch_pipelined<S>(L, (const S *)fa, (S *)fb, flags, status, s);
        const int bx = L.nx >= 128 ? 128 : ((L.nx + 31) / 32) * 32;
        dim3 grid((L.nx + bx - 1) / bx, L.ny, L.nz);
        bulk_kernel<S><<<grid, bx, 0, s>>>(L, (const S *)fa, (S *)fb, flags, status);
        return cudaGetLastError();
    });
}

cudaError_t launch_init(int storage, const Lattice &L, void *fa, const double *rho,
                        const double *u, const double *xi, double amp, cudaStream_t s)
{
    return dispatch(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        const int nb = (int)((L.N + 255) / 256);
        init_kernel<S><<<nb, 256, 0, s>>>(L, (S *)fa, rho, u, xi, amp);
        return cudaGetLastError();
    });
}

cudaError_t launch_decode_plane(int storage, const Lattice &L, const void *f, int i,
                                double *out, cudaStream_t s)
{
    return dispatch(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        const int nb = (int)((L.N + 255) / 256);
        decode_kernel<S><<<nb, 256, 0, s>>>(L, (const S *)f, i, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_encode_plane(int storage, const Lattice &L, void *f, int i,
                                const double *in, cudaStream_t s)
{
    return dispatch(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        const int nb = (int)((L.N + 255) / 256);
        encode_kernel<S><<<nb, 256, 0, s>>>(L, (S *)f, i, in);
        return cudaGetLastError();
    });
}

cudaError_t launch_totals(int storage, const Lattice &L, const void *f, const uint8_t *flags,
                          double *partials, int nblocks, double *out, cudaStream_t s)
{
    (void)out;
    return dispatch(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        totals_kernel<S><<<nblocks, 256, 0, s>>>(L, (const S *)f, flags, partials);
        return cudaGetLastError();
    });
}

}  // namespace lbm
