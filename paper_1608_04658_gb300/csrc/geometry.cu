// Body motion, node marks, boundary and uncovered lists, and the force/torque
// reduction (arXiv 1608.04658, Secs. 3 and 4.1).
//
// Per step, all on the device (no host round trip):
//   mark      every block advances the body from the previous state by
//             explicit Euler (block 0 stores it) and derives the band (box
//             around the body at t and t+1, +-2 nodes, holding every node
//             whose marks can change); band nodes get SOLID / SOLID_PREV /
//             UNCOVERED; the band-indexed force slots are cleared;
//   classify  BOUNDARY mark (fluid node with a solid pull source), append to
//             the boundary and uncovered lists, count missing links;
//   forces    after the boundary kernel has written each boundary node's
//             momentum exchange into its band slot: FP64 block partials over
//             the band in a fixed assignment, then the last block to finish
//             adds the partials with a fixed shuffle tree.  The result does not
//             depend on list order or block timing.
#include "geom.cuh"

namespace lbm {

constexpr int BAND_MARGIN = 2;
constexpr int GEOM_THREADS = 256;
constexpr int FORCE_THREADS = 256;

// Swimmer (Sec. 4.3): Euler step along x when free; band = the pose extent
// at t and t+1 plus the margin, which must stay inside the box.
__device__ void advance_mesh(const Lattice &L, const GeomParams &G, const DevBody *prev, bool advance,
                             double X[3], double U[3], int lo[3], int cnt[3], int &overflow)
{
    const int n[3] = {L.nx, L.ny, L.nz};
    overflow = 0;
    for (int a = 0; a < 3; ++a) {
        X[a] = prev->X[a];
        U[a] = prev->U[a];
    }
    if (advance && G.free_motion) {
        X[0] = __dadd_rn(prev->X[0], prev->U[0]);
        U[0] = __dadd_rn(prev->U[0], __dmul_rn(prev->F[0], G.inv_mass));
    }
    for (int a = 0; a < 3; ++a) {
        const double mn = fmin(prev->X[a], X[a]) + G.mesh_ext[2 * a];
        const double mx = fmax(prev->X[a], X[a]) + G.mesh_ext[2 * a + 1];
        int l = (int)floor(mn) - BAND_MARGIN;
        int hi = (int)floor(mx) + BAND_MARGIN + 1;
        if (l < 0) { l = 0; overflow = 1; }
        if (hi > n[a] - 1) { hi = n[a] - 1; overflow = 1; }
        int c = hi >= l ? hi - l + 1 : 0;
        if (c > G.cap[a]) { c = G.cap[a]; overflow = 1; }
        lo[a] = l;
        cnt[a] = c;
    }
}

// Explicit Euler update of the body (Sec. 4.1) and the band it sweeps.
__device__ void advance_body(const Lattice &L, const GeomParams &G, const DevBody *prev, double X[3],
                             double U[3], int lo[3], int cnt[3], int &overflow)
{
    if (G.kind == LBM_BODY_MESH) {
        advance_mesh(L, G, prev, true, X, U, lo, cnt, overflow);
        return;
    }
    const int n[3] = {L.nx, L.ny, L.nz};
    overflow = 0;
    if (G.kind == LBM_BODY_AIRFOIL) {
        // prescribed plunge (Sec. 4.2): y_le = y_base + A sin(w t)
        const double t1 = prev->t + 1.0;
        const double ph = __dmul_rn(G.h_omega, t1);
        X[0] = prev->X[0];
        X[1] = __dadd_rn(G.y_base, __dmul_rn(G.h_amp, sin(ph)));
        X[2] = prev->X[2];
        U[0] = 0.0;
        U[1] = __dmul_rn(__dmul_rn(G.h_amp, G.h_omega), cos(ph));
        U[2] = 0.0;
    }
    for (int a = 0; a < 3; ++a) {
        if (G.kind != LBM_BODY_AIRFOIL) {
            X[a] = prev->X[a];
            U[a] = prev->U[a];
        }
        if (G.free_motion && G.kind == LBM_BODY_SPHERE) {
            const double acc = __dadd_rn(__dmul_rn(prev->F[a], G.inv_mass), __dmul_rn(G.buoy, G.g[a]));
            X[a] = __dadd_rn(X[a], U[a]);
            U[a] = __dadd_rn(U[a], acc);
            if (G.periodic[a]) {
                if (X[a] >= (double)n[a]) X[a] = __dsub_rn(X[a], (double)n[a]);
                else if (X[a] < 0.0) X[a] = __dadd_rn(X[a], (double)n[a]);
            }
        }
        int l, c;
        if (G.kind == LBM_BODY_AIRFOIL && a < 2) {
            // profile box relative to the leading edge, at both poses
            const double bmin = G.box[2 * a], bmax = G.box[2 * a + 1];
            const double mn = fmin(prev->X[a], X[a]) + bmin, mx = fmax(prev->X[a], X[a]) + bmax;
            l = (int)floor(mn) - BAND_MARGIN;
            c = (int)floor(mx) + BAND_MARGIN + 1 - l + 1;
        } else if (G.kind == LBM_BODY_SPHERE) {
            // box of the sphere at both positions; on a periodic axis the old
            // centre is taken at the image nearest the new one
            double Xo = prev->X[a];
            if (G.periodic[a]) {
                const double h = 0.5 * (double)n[a];
                if (Xo - X[a] > h) Xo -= (double)n[a];
                else if (Xo - X[a] < -h) Xo += (double)n[a];
            }
            const double mn = fmin(Xo, X[a]) - G.R, mx = fmax(Xo, X[a]) + G.R;
            l = (int)floor(mn) - BAND_MARGIN;
            c = (int)floor(mx) + BAND_MARGIN + 1 - l + 1;
        } else {
            l = 0;
            c = n[a];
        }
        if (G.periodic[a]) {
            if (c >= n[a]) { l = 0; c = n[a]; }
        } else {
            int hi = l + c - 1;
            if (l < 0) l = 0;
            if (hi > n[a] - 1) hi = n[a] - 1;
            c = hi >= l ? hi - l + 1 : 0;
        }
        if (c > G.cap[a]) { c = G.cap[a]; overflow = 1; }
        lo[a] = l;
        cnt[a] = c;
    }
}

// capacity-box index k -> box coordinates; false outside the band
__device__ __forceinline__ bool band_node(const Lattice &L, const GeomParams &G, const int lo[3],
                                          const int cnt[3], int k, int &x, int &y, int &z)
{
    const int lx = k % G.cap[0];
    const int ly = (k / G.cap[0]) % G.cap[1];
    const int lz = k / (G.cap[0] * G.cap[1]);
    if (lx >= cnt[0] || ly >= cnt[1] || lz >= cnt[2]) return false;
    x = wrap_or_clip(lo[0] + lx, L.nx, G.periodic[0]);
    y = wrap_or_clip(lo[1] + ly, L.ny, G.periodic[1]);
    z = wrap_or_clip(lo[2] + lz, L.nz, G.periodic[2]);
    return true;
}

__global__ void __launch_bounds__(GEOM_THREADS) mark_kernel(const Lattice L, const GeomParams G,
                                                            const DevBody *__restrict__ prev,
                                                            DevBody *__restrict__ cur,
                                                            uint8_t *__restrict__ flags,
                                                            double *__restrict__ bforce)
{
    __shared__ double sX[3];
    __shared__ int slo[3], scnt[3];
    if (threadIdx.x == 0) {
        double X[3], U[3];
        int lo[3], cnt[3], ovf;
        advance_body(L, G, prev, X, U, lo, cnt, ovf);
        for (int a = 0; a < 3; ++a) { sX[a] = X[a]; slo[a] = lo[a]; scnt[a] = cnt[a]; }
        if (blockIdx.x == 0) {
            for (int a = 0; a < 3; ++a) {
                cur->X[a] = X[a];
                cur->U[a] = U[a];
                cur->F[a] = 0.0;
                cur->M[a] = 0.0;
                cur->F_sum[a] = prev->F_sum[a];
                cur->M_sum[a] = prev->M_sum[a];
                cur->band_lo[a] = lo[a];
                cur->band_n[a] = cnt[a];
            }
            cur->n_sum = prev->n_sum;
            cur->t = prev->t + 1.0;
            cur->n_boundary = 0;
            cur->n_uncovered = 0;
            cur->n_links = 0;
            const bool mesh_ovf = G.kind == LBM_BODY_MESH && *G.mesh_status;
            cur->status = prev->status | ((ovf || mesh_ovf) ? ST_BAND_OVERFLOW : 0);
        }
    }
    __syncthreads();
    const int cap = G.cap[0] * G.cap[1] * G.cap[2];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cap) return;
    for (int c = 0; c < 6; ++c) bforce[(size_t)k * 6 + c] = 0.0;
    int x, y, z;
    if (!band_node(L, G, slo, scnt, k, x, y, z)) return;
    const int n = x + L.nx * (y + L.ny * z);
    const double X[3] = {sX[0], sX[1], sX[2]};
    const bool s0 = flags[n] & FL_SOLID;
    bool s1;
    if (G.kind == LBM_BODY_MESH) {
        // ray parity on the column (y, z); the band lies inside the box, so x is unwrapped
        const int ly = (k / G.cap[0]) % G.cap[1], lz = k / (G.cap[0] * G.cap[1]);
        s1 = mesh_inside_column(G, ly + G.cap[1] * lz, (double)x);
    } else {
        s1 = inside_body(G, L, X, x, y, z);
    }
    uint8_t f = 0;
    if (s1) f |= FL_SOLID;
    if (s0) f |= FL_SOLID_PREV;
    if (s0 && !s1) f |= FL_UNCOVERED;
    flags[n] = f;
}

__global__ void __launch_bounds__(GEOM_THREADS) classify_kernel(const Lattice L, const GeomParams G,
                                                                DevBody *__restrict__ cur,
                                                                uint8_t *__restrict__ flags,
                                                                int *__restrict__ blist,
                                                                int *__restrict__ bpos,
                                                                int *__restrict__ ulist,
                                                                int *__restrict__ upos)
{
    const int cap = G.cap[0] * G.cap[1] * G.cap[2];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int links = 0;
    int x, y, z;
    const int lo[3] = {cur->band_lo[0], cur->band_lo[1], cur->band_lo[2]};
    const int cnt[3] = {cur->band_n[0], cur->band_n[1], cur->band_n[2]};
    if (k < cap && band_node(L, G, lo, cnt, k, x, y, z)) {
        const int n = x + L.nx * (y + L.ny * z);
        const uint8_t f = flags[n];
        if (!(f & FL_SOLID)) {
            // all 26 neighbour marks are read before any write of this kernel
            // can matter: writes only add BOUNDARY, readers test only SOLID
            uint32_t m = 0;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (i == 13) continue;
                const int s = pull_source(L, x, y, z, cx_of(i), cy_of(i), cz_of(i));
                if (s >= 0 && (flags[s] & FL_SOLID)) m |= 1u << i;
            }
            if (m) {
                flags[n] = f | FL_BOUNDARY;
                links = __popc(m);
                const int slot = atomicAdd(&cur->n_boundary, 1);
                if (slot < G.cap_boundary) { blist[slot] = n; bpos[slot] = k; }
                else atomicOr(&cur->status, ST_BAND_OVERFLOW);
            }
            if (f & FL_UNCOVERED) {
                const int slot = atomicAdd(&cur->n_uncovered, 1);
                if (slot < G.cap_uncovered) { ulist[slot] = n; upos[slot] = k; }
                else atomicOr(&cur->status, ST_BAND_OVERFLOW);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) links += __shfl_down_sync(0xffffffffu, links, o);
    if ((threadIdx.x & 31) == 0 && links) atomicAdd(&cur->n_links, links);
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
__global__ void __launch_bounds__(FORCE_THREADS) force_kernel(const GeomParams G, DevBody *__restrict__ cur,
                                                              const double *__restrict__ bforce,
                                                              double *__restrict__ partials,
                                                              unsigned *__restrict__ ticket)
{
    const int cap = G.cap[0] * G.cap[1] * G.cap[2];
    const int chunk = (cap + gridDim.x - 1) / gridDim.x;
    const int beg = blockIdx.x * chunk;
    const int end = min(cap, beg + chunk);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int s = beg + threadIdx.x; s < end; s += blockDim.x)
        for (int c = 0; c < 6; ++c) acc[c] += bforce[(size_t)s * 6 + c];
    __shared__ double sm[FORCE_THREADS / 32][6];
    __shared__ bool last;
    for (int c = 0; c < 6; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0;
        for (int w = 0; w < FORCE_THREADS / 32; ++w) v += sm[w][threadIdx.x];
        partials[blockIdx.x * 6 + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // last block: component c = warp c, lanes take partials lane, lane + 32, ...
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < 6) {
        double v = 0;
        for (int p = lane; p < (int)gridDim.x; p += 32) v += ((volatile double *)partials)[p * 6 + w];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) {
            if (w < 3) { cur->F[w] = v; cur->F_sum[w] += v; }
            else { cur->M[w - 3] = v; cur->M_sum[w - 3] += v; }
        }
    }
    if (threadIdx.x == 0) {
        cur->n_sum += 1;
        *ticket = 0u;
    }
}

// ----------------------------------------------------------------- swimmer mesh
constexpr int MESH_THREADS = 256;

// Pose of the mesh at the new step (or at the current one when !advance):
// vertex positions x = X0 + s, y = (X1 + y(s,t)) + dy, z = X2 + dz and
// velocities; clears the column and cell lists of the step.
__global__ void __launch_bounds__(MESH_THREADS) mesh_pose_kernel(const Lattice L, const GeomParams G,
                                                                 const DevBody *__restrict__ prev, int advance,
                                                                 int ncols, int ncells)
{
    __shared__ double sX[3], sU[3];
    if (threadIdx.x == 0) {
        double X[3], U[3];
        int lo[3], cnt[3], ovf;
        advance_mesh(L, G, prev, advance != 0, X, U, lo, cnt, ovf);
        for (int a = 0; a < 3; ++a) { sX[a] = X[a]; sU[a] = U[a]; }
    }
    __syncthreads();
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int c = gid; c < ncols; c += stride) G.col_count[c] = 0;
    for (int c = gid; c < ncells; c += stride) G.cell_count[c] = 0;
    if (gid == 0) *G.mesh_status = 0;
    if (gid >= G.n_vertices) return;
    const double t = advance ? __dadd_rn(prev->t, 1.0) : prev->t;
    const double s = G.mesh_rest[3 * gid], dy = G.mesh_rest[3 * gid + 1], dz = G.mesh_rest[3 * gid + 2];
    double *p = G.mesh_pos + 3 * (size_t)gid;
    p[0] = __dadd_rn(sX[0], s);
    p[1] = __dadd_rn(__dadd_rn(sX[1], swimmer_midline(G, s, t)), dy);
    p[2] = __dadd_rn(sX[2], dz);
    for (int a = 0; a < 3; ++a) {
        const double r = rint(p[a]);
        G.mesh_ipos[3 * (size_t)gid + a] = (int)r;
        G.mesh_frac[3 * (size_t)gid + a] = (float)(p[a] - r);
    }
    const double U[3] = {sU[0], sU[1], sU[2]};
    double v[3];
    swimmer_velocity(G, U, t, s, v);
    double *q = G.mesh_vel + 3 * (size_t)gid;
    q[0] = v[0];
    q[1] = v[1];
    q[2] = v[2];
}

// Per triangle: its box, the band columns whose line crosses it (with the
// crossing abscissa) and the band cells its box overlaps.
__global__ void __launch_bounds__(MESH_THREADS) mesh_bin_kernel(const Lattice L, const GeomParams G,
                                                                const DevBody *__restrict__ prev, int advance)
{
    __shared__ int slo[3], scnt[3];
    if (threadIdx.x == 0) {
        double X[3], U[3];
        int lo[3], cnt[3], ovf;
        advance_mesh(L, G, prev, advance != 0, X, U, lo, cnt, ovf);
        for (int a = 0; a < 3; ++a) { slo[a] = lo[a]; scnt[a] = cnt[a]; }
    }
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.n_triangles) return;
    const int t0 = G.mesh_tris[3 * k], t1 = G.mesh_tris[3 * k + 1], t2 = G.mesh_tris[3 * k + 2];
    const double *P = G.mesh_pos;
    double mn[3], mx[3];
    bool finite = true;
    for (int a = 0; a < 3; ++a) {
        mn[a] = fmin(fmin(P[3 * t0 + a], P[3 * t1 + a]), P[3 * t2 + a]);
        mx[a] = fmax(fmax(P[3 * t0 + a], P[3 * t1 + a]), P[3 * t2 + a]);
        finite = finite && isfinite(mn[a]) && isfinite(mx[a]);
        G.tri_box[6 * (size_t)k + a] = __double2float_rd(mn[a]);
        G.tri_box[6 * (size_t)k + 3 + a] = __double2float_ru(mx[a]);
    }
    if (!finite) {
        atomicOr(G.mesh_status, 1);
        return;
    }
    // columns (y, z) inside the triangle's box and the band
    const int y0 = max((int)ceil(mn[1]), slo[1]), y1 = min((int)floor(mx[1]), slo[1] + scnt[1] - 1);
    const int z0 = max((int)ceil(mn[2]), slo[2]), z1 = min((int)floor(mx[2]), slo[2] + scnt[2] - 1);
    for (int z = z0; z <= z1; ++z)
        for (int y = y0; y <= y1; ++y) {
            double xc;
            if (!mesh_column_crossing(P, t0, t1, t2, (double)y, (double)z, xc)) continue;
            const int col = (y - slo[1]) + G.cap[1] * (z - slo[2]);
            const int slot = atomicAdd(&G.col_count[col], 1);
            if (slot < MESH_COL_CAP) G.col_x[(size_t)col * MESH_COL_CAP + slot] = xc;
            else atomicOr(G.mesh_status, 1);
        }
    // cells of edge MESH_CELL from the band origin
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
        c0[a] = max(0, (int)floor((mn[a] - slo[a]) / MESH_CELL));
        c1[a] = min(G.cells[a] - 1, (int)floor((mx[a] - slo[a]) / MESH_CELL));
    }
    for (int kz = c0[2]; kz <= c1[2]; ++kz)
        for (int ky = c0[1]; ky <= c1[1]; ++ky)
            for (int kx = c0[0]; kx <= c1[0]; ++kx) {
                const int cell = kx + G.cells[0] * (ky + G.cells[1] * kz);
                const int slot = atomicAdd(&G.cell_count[cell], 1);
                if (slot < MESH_CELL_CAP) G.cell_tri[(size_t)cell * MESH_CELL_CAP + slot] = k;
                else atomicOr(G.mesh_status, 1);
            }
}

// initial marks of the mesh at the current pose: SOLID by column parity over
// the band (the flags were cleared); a pose outside the box or a list
// overflow is reported in mesh_status
__global__ void __launch_bounds__(GEOM_THREADS) mesh_mark_initial_kernel(const Lattice L, const GeomParams G,
                                                                         const DevBody *__restrict__ b,
                                                                         uint8_t *__restrict__ flags)
{
    __shared__ int slo[3], scnt[3];
    if (threadIdx.x == 0) {
        double X[3], U[3];
        int lo[3], cnt[3], ovf;
        advance_mesh(L, G, b, false, X, U, lo, cnt, ovf);
        for (int a = 0; a < 3; ++a) { slo[a] = lo[a]; scnt[a] = cnt[a]; }
        if (ovf && blockIdx.x == 0) atomicOr(G.mesh_status, 2);
    }
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int x, y, z;
    if (k >= G.cap[0] * G.cap[1] * G.cap[2] || !band_node(L, G, slo, scnt, k, x, y, z)) return;
    const int ly = (k / G.cap[0]) % G.cap[1], lz = k / (G.cap[0] * G.cap[1]);
    if (mesh_inside_column(G, ly + G.cap[1] * lz, (double)x)) flags[x + L.nx * (y + L.ny * z)] = FL_SOLID;
}

// ----------------------------------------------------------------- launchers
static int band_blocks(const GeomParams &G)
{
    const int cap = G.cap[0] * G.cap[1] * G.cap[2];
    return (cap + GEOM_THREADS - 1) / GEOM_THREADS;
}

cudaError_t launch_geometry(const Lattice &L, const GeomParams &G, Scratch &S, int prev, uint8_t *flags,
                            cudaStream_t s, int *nlaunch)
{
    const int nb = band_blocks(G);
    DevBody *bp = S.body + prev, *bc = S.body + (prev ^ 1);
    if (G.kind == LBM_BODY_MESH) {
        cudaError_t e = launch_mesh_prepare(L, G, S, prev, true, s, nlaunch);
        if (e != cudaSuccess) return e;
    }
    mark_kernel<<<nb, GEOM_THREADS, 0, s>>>(L, G, bp, bc, flags, S.bforce);
    classify_kernel<<<nb, GEOM_THREADS, 0, s>>>(L, G, bc, flags, S.blist, S.bpos, S.ulist, S.upos);
    *nlaunch += 2;
    return cudaGetLastError();
}

cudaError_t launch_mark_initial(const Lattice &L, const GeomParams &G, const double *X,
                                uint8_t *flags, cudaStream_t s)
{
    const int nb = (int)((L.N + 255) / 256);
    mark_initial_kernel<<<nb, 256, 0, s>>>(L, G, X[0], X[1], X[2], flags);
    return cudaGetLastError();
}

cudaError_t launch_forces(const GeomParams &G, Scratch &S, int cur, cudaStream_t s, int *nlaunch)
{
    force_kernel<<<S.n_partials, FORCE_THREADS, 0, s>>>(G, S.body + cur, S.bforce, S.partials, S.ticket);
    *nlaunch += 1;
    return cudaGetLastError();
}

}  // namespace lbm

namespace lbm {

cudaError_t launch_mesh_prepare(const Lattice &L, const GeomParams &G, Scratch &S, int prev, bool advance,
                                cudaStream_t s, int *nlaunch)
{
    const int ncols = G.cap[1] * G.cap[2];
    const int ncells = G.cells[0] * G.cells[1] * G.cells[2];
    const int nb_v = (G.n_vertices + MESH_THREADS - 1) / MESH_THREADS;
    const int nb_t = (G.n_triangles + MESH_THREADS - 1) / MESH_THREADS;
    mesh_pose_kernel<<<nb_v > 0 ? nb_v : 1, MESH_THREADS, 0, s>>>(L, G, S.body + prev, advance ? 1 : 0, ncols, ncells);
    mesh_bin_kernel<<<nb_t > 0 ? nb_t : 1, MESH_THREADS, 0, s>>>(L, G, S.body + prev, advance ? 1 : 0);
    *nlaunch += 2;
    return cudaGetLastError();
}

cudaError_t launch_mesh_mark_initial(const Lattice &L, const GeomParams &G, Scratch &S, int cur,
                                     uint8_t *flags, cudaStream_t s)
{
    int n = 0;
    cudaError_t e = launch_mesh_prepare(L, G, S, cur, false, s, &n);
    if (e != cudaSuccess) return e;
    mesh_mark_initial_kernel<<<band_blocks(G), GEOM_THREADS, 0, s>>>(L, G, S.body + cur, flags);
    return cudaGetLastError();
}

}  // namespace lbm
