// Body motion, node marks, boundary-node compaction with link data, and the
// force/torque reduction (arXiv 1608.04658, Secs. 3 and 4.1).
//
// Per step (all on the device, no host round trip):
//   body_update   Newton's equations of the sphere by explicit Euler and the
//                 band (box around the body at t and t+1, +-2 nodes) that
//                 holds every node whose marks can change;
//   mark          SOLID / SOLID_PREV / UNCOVERED marks over the band;
//   count         BOUNDARY mark (fluid node with a solid pull source) and
//                 per-block counts of boundary and uncovered nodes;
//   scan          block offsets (one block, fixed order);
//   compact       boundary list in band order with missing mask, link
//                 fraction q_i and wall velocity u_w,i; uncovered list;
//   forces        FP64 warp-shuffle block partials of the per-node momentum
//                 exchange, then one block adds them in block order.
// Floating-point decisions that set marks (inside tests) are taken in
// IEEE double with explicitly rounded operations, so they do not depend on
// FMA contraction.
#include "kbc.cuh"

namespace lbm {

constexpr int BAND_MARGIN = 2;
constexpr int COUNT_THREADS = 256;

__device__ __forceinline__ int wrap_or_clip(int u, int n, int periodic)
{
    if (periodic) { int r = u % n; return r < 0 ? r + n : r; }
    return u;
}

// Displacement from the sphere centre, nearest image on periodic axes:
// d - n floor(d/n + 1/2).
__device__ __forceinline__ double sphere_axis_offset(int p, double X, int n, int periodic)
{
    double d = __dsub_rn((double)p, X);
    if (periodic) d = __dsub_rn(d, __dmul_rn((double)n, floor(__dadd_rn(__ddiv_rn(d, (double)n), 0.5))));
    return d;
}

__device__ __forceinline__ bool inside_body(const GeomParams &G, const Lattice &L,
                                            const double X[3], int x, int y, int z)
{
    if (G.kind == LBM_BODY_SPHERE) {
        const double dx = sphere_axis_offset(x, X[0], L.nx, G.periodic[0]);
        const double dy = sphere_axis_offset(y, X[1], L.ny, G.periodic[1]);
        const double dz = sphere_axis_offset(z, X[2], L.nz, G.periodic[2]);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        return d2 < __dmul_rn(G.R, G.R);
    }
    if (G.kind == LBM_BODY_PLANES) return (double)y < G.y_lo || (double)y > G.y_hi;
    return false;
}

// ----------------------------------------------------------------- body update
__global__ void body_update_kernel(const Lattice L, const GeomParams G, DevBody *__restrict__ b)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double Xo[3] = {b->X[0], b->X[1], b->X[2]};
    if (G.free_motion && G.kind == LBM_BODY_SPHERE) {
        for (int a = 0; a < 3; ++a) {
            const double acc = b->F[a] / G.mass + (1.0 - 1.0 / G.rho_ratio) * G.g[a];
            b->X[a] = b->X[a] + b->U[a];
            b->U[a] = b->U[a] + acc;
        }
    }
    const int n[3] = {L.nx, L.ny, L.nz};
    for (int a = 0; a < 3; ++a) {
        int lo, cnt;
        if (G.kind == LBM_BODY_SPHERE) {
            const double mn = fmin(Xo[a], b->X[a]) - G.R, mx = fmax(Xo[a], b->X[a]) + G.R;
            lo = (int)floor(mn) - BAND_MARGIN;
            const int hi = (int)floor(mx) + BAND_MARGIN + 1;
            cnt = hi - lo + 1;
        } else {
            lo = 0;
            cnt = n[a];
        }
        if (G.periodic[a]) {
            if (cnt >= n[a]) { lo = 0; cnt = n[a]; }
        } else {
            int hi = lo + cnt - 1;
            if (lo < 0) lo = 0;
            if (hi > n[a] - 1) hi = n[a] - 1;
            cnt = hi >= lo ? hi - lo + 1 : 0;
        }
        if (cnt > G.cap[a]) { cnt = G.cap[a]; b->status |= ST_BAND_OVERFLOW; }
        b->band_lo[a] = lo;
        b->band_n[a] = cnt;
    }
    b->n_links = 0;
}

// Band node k of the capacity box -> box coordinates; false if outside the band.
__device__ __forceinline__ bool band_node(const Lattice &L, const GeomParams &G, const DevBody *b,
                                          long long k, int &x, int &y, int &z)
{
    const int lx = (int)(k % G.cap[0]);
    const int ly = (int)((k / G.cap[0]) % G.cap[1]);
    const int lz = (int)(k / ((long long)G.cap[0] * G.cap[1]));
    if (lx >= b->band_n[0] || ly >= b->band_n[1] || lz >= b->band_n[2]) return false;
    x = wrap_or_clip(b->band_lo[0] + lx, L.nx, G.periodic[0]);
    y = wrap_or_clip(b->band_lo[1] + ly, L.ny, G.periodic[1]);
    z = wrap_or_clip(b->band_lo[2] + lz, L.nz, G.periodic[2]);
    return true;
}

__global__ void mark_kernel(const Lattice L, const GeomParams G, const DevBody *__restrict__ b,
                            uint8_t *__restrict__ flags)
{
    const long long cap = (long long)G.cap[0] * G.cap[1] * G.cap[2];
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= cap) return;
    int x, y, z;
    if (!band_node(L, G, b, k, x, y, z)) return;
    const long long n = x + (long long)L.nx * (y + (long long)L.ny * z);
    const uint8_t old = flags[n];
    const bool s0 = old & FL_SOLID;
    const bool s1 = inside_body(G, L, b->X, x, y, z);
    uint8_t f = 0;
    if (s1) f |= FL_SOLID;
    if (s0) f |= FL_SOLID_PREV;
    if (s0 && !s1) f |= FL_UNCOVERED;
    flags[n] = f;
}

// Pull source x - c under the box rules; returns the node index or -1 when
// the pull is served by a face (wall or equilibrium), never solid.
__device__ __forceinline__ long long pull_source(const Lattice &L, int x, int y, int z, int cx,
                                                 int cy, int cz)
{
    int p[3] = {x - cx, y - cy, z - cz};
    const int n[3] = {L.nx, L.ny, L.nz};
    for (int a = 0; a < 3; ++a) {
        int face = -1;
        if (p[a] < 0) face = L.face[2 * a];
        else if (p[a] >= n[a]) face = L.face[2 * a + 1];
        if (face < 0) continue;
        if (face == LBM_FACE_PERIODIC) p[a] = (p[a] + n[a]) % n[a];
        else if (face == LBM_FACE_OUTFLOW) p[a] = p[a] < 0 ? 0 : n[a] - 1;
        else return -1;
    }
    return p[0] + (long long)L.nx * (p[1] + (long long)L.ny * p[2]);
}

__device__ __forceinline__ uint32_t missing_mask(const Lattice &L, const uint8_t *flags, int x, int y, int z)
{
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (i == 13) continue;
        const long long s = pull_source(L, x, y, z, cx_of(i), cy_of(i), cz_of(i));
        if (s >= 0 && (flags[s] & FL_SOLID)) m |= 1u << i;
    }
    return m;
}

// block-exclusive rank of a predicate and the block total
__device__ __forceinline__ int block_rank(bool pred, int *warp_tot, int &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned ball = __ballot_sync(0xffffffffu, pred);
    const int in_warp = __popc(ball & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[w] = __popc(ball);
    __syncthreads();
    int before = 0;
    total = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        if (k < w) before += warp_tot[k];
        total += warp_tot[k];
    }
    __syncthreads();
    return before + in_warp;
}

__global__ void __launch_bounds__(COUNT_THREADS) count_kernel(const Lattice L, const GeomParams G,
                                                              DevBody *__restrict__ b,
                                                              uint8_t *__restrict__ flags,
                                                              int *__restrict__ blk_count,
                                                              int *__restrict__ blk_ucount)
{
    __shared__ int wt[COUNT_THREADS / 32];
    const long long cap = (long long)G.cap[0] * G.cap[1] * G.cap[2];
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    bool isb = false, isu = false;
    int links = 0;
    int x, y, z;
    if (k < cap && band_node(L, G, b, k, x, y, z)) {
        const long long n = x + (long long)L.nx * (y + (long long)L.ny * z);
        const uint8_t f = flags[n];
        if (!(f & FL_SOLID)) {
            const uint32_t m = missing_mask(L, flags, x, y, z);
            isb = m != 0;
            links = __popc(m);
            isu = f & FL_UNCOVERED;
        }
    }
    // the BOUNDARY mark is written after every thread has read its neighbours'
    // SOLID bits (other bits are untouched, so the order does not matter)
    int tb, tu;
    block_rank(isb, wt, tb);
    block_rank(isu, wt, tu);
    if (isb) {
        const long long n = x + (long long)L.nx * (y + (long long)L.ny * z);
        flags[n] |= FL_BOUNDARY;
    }
    for (int o = 16; o > 0; o >>= 1) links += __shfl_down_sync(0xffffffffu, links, o);
    if ((threadIdx.x & 31) == 0 && links) atomicAdd(&b->n_links, links);
    if (threadIdx.x == 0) {
        blk_count[blockIdx.x] = tb;
        blk_ucount[blockIdx.x] = tu;
    }
}

__global__ void scan_kernel(const GeomParams G, DevBody *__restrict__ b, const int *__restrict__ cnt,
                            const int *__restrict__ ucnt, int *__restrict__ off,
                            int *__restrict__ uoff, int nblocks)
{
    if (threadIdx.x != 0) return;
    int s = 0, u = 0;
    for (int k = 0; k < nblocks; ++k) {
        off[k] = s;
        uoff[k] = u;
        s += cnt[k];
        u += ucnt[k];
    }
    if (s > G.cap_boundary) { b->status |= ST_BAND_OVERFLOW; s = G.cap_boundary; }
    if (u > G.cap_uncovered) { b->status |= ST_BAND_OVERFLOW; u = G.cap_uncovered; }
    b->n_boundary = s;
    b->n_uncovered = u;
}

// link fraction q (wall point x_w = x_b - q c) and wall velocity for the
// missing direction c of boundary node (x, y, z)
__device__ __forceinline__ void link_data(const Lattice &L, const GeomParams &G, const DevBody *b,
                                          int x, int y, int z, int cx, int cy, int cz,
                                          double &q, double uw[3])
{
    if (G.kind == LBM_BODY_SPHERE) {
        const double d0 = sphere_axis_offset(x, b->X[0], L.nx, G.periodic[0]);
        const double d1 = sphere_axis_offset(y, b->X[1], L.ny, G.periodic[1]);
        const double d2 = sphere_axis_offset(z, b->X[2], L.nz, G.periodic[2]);
        const double cc = (double)(cx * cx + cy * cy + cz * cz);
        const double cd = cx * d0 + cy * d1 + cz * d2;
        const double dd = d0 * d0 + d1 * d1 + d2 * d2;
        const double disc = cd * cd - cc * (dd - G.R * G.R);
        q = (cd - sqrt(fmax(disc, 0.0))) / cc;
        uw[0] = b->U[0]; uw[1] = b->U[1]; uw[2] = b->U[2];
    } else {  // planes
        const double yb = (double)y;
        const bool low = (double)(y - cy) < G.y_lo;
        q = low ? (yb - G.y_lo) / (double)cy : (G.y_hi - yb) / (double)(-cy);
        const double *v = low ? G.U_lo : G.U_hi;
        uw[0] = v[0]; uw[1] = v[1]; uw[2] = v[2];
    }
}

__global__ void __launch_bounds__(COUNT_THREADS) compact_kernel(
    const Lattice L, const GeomParams G, const DevBody *__restrict__ b,
    const uint8_t *__restrict__ flags, const int *__restrict__ off, const int *__restrict__ uoff,
    int *__restrict__ bnode, uint32_t *__restrict__ bmask, double *__restrict__ bq,
    double *__restrict__ buw, int *__restrict__ unode)
{
    __shared__ int wt[COUNT_THREADS / 32];
    const long long cap = (long long)G.cap[0] * G.cap[1] * G.cap[2];
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    bool isb = false, isu = false;
    int x = 0, y = 0, z = 0;
    long long n = 0;
    if (k < cap && band_node(L, G, b, k, x, y, z)) {
        n = x + (long long)L.nx * (y + (long long)L.ny * z);
        const uint8_t f = flags[n];
        isb = (f & FL_BOUNDARY) != 0;
        isu = (f & FL_UNCOVERED) != 0;
    }
    int tb, tu;
    const int rb = block_rank(isb, wt, tb);
    const int ru = block_rank(isu, wt, tu);
    if (isb) {
        const int slot = off[blockIdx.x] + rb;
        if (slot < G.cap_boundary) {
            const uint32_t m = missing_mask(L, flags, x, y, z);
            bnode[slot] = (int)n;
            bmask[slot] = m;
            for (int i = 0; i < Q; ++i) {
                double q = 0, uw[3] = {0, 0, 0};
                if (m & (1u << i)) link_data(L, G, b, x, y, z, cx_of(i), cy_of(i), cz_of(i), q, uw);
                bq[(size_t)slot * Q + i] = q;
                buw[((size_t)slot * Q + i) * 3 + 0] = uw[0];
                buw[((size_t)slot * Q + i) * 3 + 1] = uw[1];
                buw[((size_t)slot * Q + i) * 3 + 2] = uw[2];
            }
        }
    }
    if (isu) {
        const int slot = uoff[blockIdx.x] + ru;
        if (slot < G.cap_uncovered) unode[slot] = (int)n;
    }
}

// initial marks: SOLID inside the body at X over the whole box
__global__ void mark_initial_kernel(const Lattice L, const GeomParams G, const double X0,
                                    const double X1, const double X2, uint8_t *__restrict__ flags)
{
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    const int x = (int)(n % L.nx), y = (int)((n / L.nx) % L.ny), z = (int)(n / ((long long)L.nx * L.ny));
    const double X[3] = {X0, X1, X2};
    flags[n] = inside_body(G, L, X, x, y, z) ? FL_SOLID : 0;
}

// ----------------------------------------------------------------- forces
// Momentum exchange per boundary node (6 doubles) -> per-block partials.
// Block p sums the contiguous slots [p*chunk, (p+1)*chunk) with a fixed
// assignment and a fixed shuffle tree, so the result is reproducible.
__global__ void __launch_bounds__(256) force_partials_kernel(const DevBody *__restrict__ b,
                                                             const double *__restrict__ bforce,
                                                             double *__restrict__ partials)
{
    const int count = b->n_boundary;
    const int chunk = (count + gridDim.x - 1) / gridDim.x;
    const int beg = blockIdx.x * chunk;
    const int end = min(count, beg + chunk);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int s = beg + threadIdx.x; s < end; s += blockDim.x)
        for (int k = 0; k < 6; ++k) acc[k] += bforce[(size_t)s * 6 + k];
    __shared__ double sm[8][6];
    for (int k = 0; k < 6; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sm[w][threadIdx.x];
        partials[blockIdx.x * 6 + threadIdx.x] = v;
    }
}

__global__ void force_final_kernel(DevBody *__restrict__ b, const double *__restrict__ partials, int np)
{
    if (threadIdx.x >= 6) return;
    double v = 0;
    for (int p = 0; p < np; ++p) v += partials[p * 6 + threadIdx.x];
    const int k = threadIdx.x;
    if (k < 3) { b->F[k] = v; b->F_sum[k] += v; }
    else { b->M[k - 3] = v; b->M_sum[k - 3] += v; }
    __syncwarp(0x3fu);
    if (k == 0) b->n_sum += 1;
}

// ----------------------------------------------------------------- launchers
static long long band_cap(const GeomParams &G) { return (long long)G.cap[0] * G.cap[1] * G.cap[2]; }

cudaError_t launch_body_update(const Lattice &L, const GeomParams &G, Scratch &S, cudaStream_t s)
{
    body_update_kernel<<<1, 32, 0, s>>>(L, G, S.body);
    return cudaGetLastError();
}

cudaError_t launch_geometry(const Lattice &L, const GeomParams &G, Scratch &S, uint8_t *flags,
                            cudaStream_t s, int *nlaunch)
{
    const long long cap = band_cap(G);
    const int nb = (int)((cap + COUNT_THREADS - 1) / COUNT_THREADS);
    mark_kernel<<<nb, COUNT_THREADS, 0, s>>>(L, G, S.body, flags);
    count_kernel<<<nb, COUNT_THREADS, 0, s>>>(L, G, S.body, flags, S.blk_count, S.blk_ucount);
    scan_kernel<<<1, 32, 0, s>>>(G, S.body, S.blk_count, S.blk_ucount, S.blk_off, S.blk_uoff, nb);
    compact_kernel<<<nb, COUNT_THREADS, 0, s>>>(L, G, S.body, flags, S.blk_off, S.blk_uoff, S.bnode,
                                                S.bmask, S.bq, S.buw, S.unode);
    *nlaunch += 4;
    return cudaGetLastError();
}

cudaError_t launch_mark_initial(const Lattice &L, const GeomParams &G, const double *X,
                                uint8_t *flags, cudaStream_t s)
{
    const int nb = (int)((L.N + 255) / 256);
    mark_initial_kernel<<<nb, 256, 0, s>>>(L, G, X[0], X[1], X[2], flags);
    return cudaGetLastError();
}

cudaError_t launch_forces(const Lattice &L, Scratch &S, cudaStream_t s, int *nlaunch)
{
    (void)L;
    force_partials_kernel<<<S.n_partials, 256, 0, s>>>(S.body, S.bforce, S.partials);
    force_final_kernel<<<1, 32, 0, s>>>(S.body, S.partials, S.n_partials);
    *nlaunch += 2;
    return cudaGetLastError();
}

}  // namespace lbm
