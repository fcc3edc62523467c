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
__device__ void advance_mesh(const Lattice &L, const GeomParams &G, const DevBody *prev, const DevBody *next,
                             bool advance, double X[3], double U[3], int lo[3], int cnt[3], int &overflow)
{
    const int n[3] = {L.nx, L.ny, L.nz};
    overflow = 0;
    if (G.com_frame) {
        // centre-of-mass frame: the pose was advanced by mesh_mass_kernel into
        // next; band = lattice boxes of both poses (x, y), the z extent, margin
        for (int a = 0; a < 3; ++a) {
            X[a] = next->X[a];
            U[a] = next->U[a];
        }
        int l[3], h[3];
        l[0] = min(prev->ibox[0], next->ibox[0]) - BAND_MARGIN;
        h[0] = max(prev->ibox[1], next->ibox[1]) + BAND_MARGIN;
        l[1] = min(prev->ibox[2], next->ibox[2]) - BAND_MARGIN;
        h[1] = max(prev->ibox[3], next->ibox[3]) + BAND_MARGIN;
        const double Xz = slab_z(G, X[2], n[2]);
        l[2] = (int)floor(Xz + G.mesh_ext[4]) - BAND_MARGIN;
        h[2] = (int)floor(Xz + G.mesh_ext[5]) + BAND_MARGIN + 1;
        for (int a = 0; a < 3; ++a) {
            // a slab's z: cut at its layers (not an overflow)
            const bool cut = a == 2 && G.zper > 0;
            if (l[a] < 0) { l[a] = 0; overflow |= !cut; }
            if (h[a] > n[a] - 1) { h[a] = n[a] - 1; overflow |= !cut; }
            int c = h[a] >= l[a] ? h[a] - l[a] + 1 : 0;
            if (c > G.cap[a]) { c = G.cap[a]; overflow = 1; }
            lo[a] = l[a];
            cnt[a] = c;
        }
        return;
    }
    for (int a = 0; a < 3; ++a) {
        X[a] = prev->X[a];
        U[a] = prev->U[a];
    }
    if (advance && G.free_motion) {
        X[0] = __dadd_rn(prev->X[0], prev->U[0]);
        U[0] = __dadd_rn(prev->U[0], __dmul_rn(prev->F[0], G.inv_mass));
    }
    for (int a = 0; a < 3; ++a) {
        // a slab's z: the pose in its own frame, cut at its layers (not an overflow)
        const bool cut = a == 2 && G.zper > 0;
        const double Xp = cut ? slab_z(G, prev->X[2], n[2]) : prev->X[a];
        const double Xn = cut ? slab_z(G, X[2], n[2]) : X[a];
        const double mn = fmin(Xp, Xn) + G.mesh_ext[2 * a];
        const double mx = fmax(Xp, Xn) + G.mesh_ext[2 * a + 1];
        int l = (int)floor(mn) - BAND_MARGIN;
        int hi = (int)floor(mx) + BAND_MARGIN + 1;
        if (l < 0) { l = 0; overflow |= !cut; }
        if (hi > n[a] - 1) { hi = n[a] - 1; overflow |= !cut; }
        int c = hi >= l ? hi - l + 1 : 0;
        if (c > G.cap[a]) { c = G.cap[a]; overflow = 1; }
        lo[a] = l;
        cnt[a] = c;
    }
}

// Explicit Euler update of the body (Sec. 4.1) and the band it sweeps.
__device__ void advance_body(const Lattice &L, const GeomParams &G, const DevBody *prev, const DevBody *next,
                             double X[3], double U[3], int lo[3], int cnt[3], int &overflow)
{
    if (G.kind == LBM_BODY_MESH) {
        advance_mesh(L, G, prev, next, true, X, U, lo, cnt, overflow);
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
            // the centre wraps on a periodic axis (a slab's z: the whole box's)
            const int per = a == 2 && G.zper > 0 ? G.zper : (G.periodic[a] ? n[a] : 0);
            if (per) {
                if (X[a] >= (double)per) X[a] = __dsub_rn(X[a], (double)per);
                else if (X[a] < 0.0) X[a] = __dadd_rn(X[a], (double)per);
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
            double Xo = prev->X[a], Xn = X[a];
            if (G.periodic[a]) {
                const double h = 0.5 * (double)n[a];
                if (Xo - Xn > h) Xo -= (double)n[a];
                else if (Xo - Xn < -h) Xo += (double)n[a];
            }
            if (a == 2 && G.zper > 0) {
                // a slab: both centres in its own z frame, at the image of the
                // whole box nearest its layers (the box is not periodic)
                const double per = (double)G.zper, mid = 0.5 * (double)n[2];
                Xn -= (double)G.zoff;
                if (Xn - mid > 0.5 * per) Xn -= per;
                else if (Xn - mid < -0.5 * per) Xn += per;
                Xo -= (double)G.zoff;
                if (Xo - Xn > 0.5 * per) Xo -= per;
                else if (Xo - Xn < -0.5 * per) Xo += per;
            }
            const double mn = fmin(Xo, Xn) - G.R, mx = fmax(Xo, Xn) + G.R;
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

// band of the step that starts from body state b: the same function of b as
// the mark kernel of that step evaluates.  The band depends on b's pose,
// velocity and time only, not on its force, so it is final once the mark
// kernel has written b.
__device__ void store_sweep(const Lattice &L, const GeomParams &G, DevBody *b)
{
    double X[3], U[3];
    int lo[3], cnt[3], ovf;
    advance_body(L, G, b, b, X, U, lo, cnt, ovf);
    for (int a = 0; a < 3; ++a) {
        b->sweep[a] = lo[a];
        b->sweep[3 + a] = cnt[a];
    }
}

__global__ void sweep_init_kernel(const Lattice L, const GeomParams G, DevBody *__restrict__ b)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) store_sweep(L, G, b);
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
        advance_body(L, G, prev, cur, X, U, lo, cnt, ovf);
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
            // the band must be the sweep box the outside bulk launch skipped
            bool sweep_ok = true;
            if (sweep_ahead(G))
                for (int a = 0; a < 3; ++a)
                    sweep_ok = sweep_ok && prev->sweep[a] == lo[a] && prev->sweep[3 + a] == cnt[a];
            // atomic: a bulk launch of this step may already have raised a
            // bit; the slot's older bits are a subset of prev's (they only
            // accumulate)
            atomicOr(&cur->status, prev->status | ((ovf || mesh_ovf || !sweep_ok) ? ST_BAND_OVERFLOW : 0));
            if (sweep_ahead(G)) store_sweep(L, G, cur);
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

// Pose of the mesh at the new step (or at the current one when !advance):
// vertex positions x = X0 + s, y = (X1 + y(s,t)) + dy, z = X2 + dz (head
// frame) or X + R(psi) (b - c(t)) (centre-of-mass frame, with the lattice box
// of the pose) and velocities; clears the column and cell lists of the step.
__global__ void __launch_bounds__(MESH_THREADS) mesh_pose_kernel(const Lattice L, const GeomParams G,
                                                                 const DevBody *__restrict__ prev,
                                                                 DevBody *__restrict__ next, int advance,
                                                                 int ncols, int ncells)
{
    __shared__ double sX[3], sU[3];
    if (threadIdx.x == 0) {
        double X[3], U[3];
        int lo[3], cnt[3], ovf;
        if (G.com_frame) {
            for (int a = 0; a < 3; ++a) { X[a] = next->X[a]; U[a] = next->U[a]; }
        } else {
            advance_mesh(L, G, prev, next, advance != 0, X, U, lo, cnt, ovf);
        }
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
    if (G.com_frame) {
        // X + R(psi) (b - c(t)), b = (s, y(s,t) + dy, dz); velocity
        // U + omega e_z x (p - X) + R(psi) (b_dot - c_dot)
        const double cs = cos(next->psi), sn = sin(next->psi);
        const double qx = s - next->com[0], qy = (swimmer_midline(G, s, t) + dy) - next->com[1];
        p[0] = sX[0] + (cs * qx - sn * qy);
        p[1] = sX[1] + (sn * qx + cs * qy);
        p[2] = slab_z(G, sX[2], L.nz) + dz;
        const double rate = 0.5 * (swimmer_midline(G, s, t + 1.0) - swimmer_midline(G, s, t - 1.0));
        const double wx = -next->com_dot[0], wy = rate - next->com_dot[1];
        double *q = G.mesh_vel + 3 * (size_t)gid;
        q[0] = sU[0] - next->omega * (p[1] - sX[1]) + (cs * wx - sn * wy);
        q[1] = sU[1] + next->omega * (p[0] - sX[0]) + (sn * wx + cs * wy);
        q[2] = sU[2];
        for (int a = 0; a < 3; ++a) {
            const double r = rint(p[a]);
            G.mesh_ipos[3 * (size_t)gid + a] = (int)r;
            G.mesh_frac[3 * (size_t)gid + a] = (float)(p[a] - r);
        }
        atomicMin(&next->ibox[0], (int)floor(p[0]));
        atomicMax(&next->ibox[1], (int)ceil(p[0]));
        atomicMin(&next->ibox[2], (int)floor(p[1]));
        atomicMax(&next->ibox[3], (int)ceil(p[1]));
        return;
    }
    p[0] = __dadd_rn(sX[0], s);
    p[1] = __dadd_rn(__dadd_rn(sX[1], swimmer_midline(G, s, t)), dy);
    p[2] = __dadd_rn(slab_z(G, sX[2], L.nz), dz);  // a slab's pose in its own z frame
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
                                                                const DevBody *__restrict__ prev,
                                                                const DevBody *__restrict__ next, int advance)
{
    __shared__ int slo[3], scnt[3];
    if (threadIdx.x == 0) {
        double X[3], U[3];
        int lo[3], cnt[3], ovf;
        advance_mesh(L, G, prev, next, advance != 0, X, U, lo, cnt, ovf);
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
        advance_mesh(L, G, b, b, false, X, U, lo, cnt, ovf);
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

// Centre-of-mass frame: volume sums of the mesh in the body frame at t (V,
// int x, int y, int x^2, int y^2) and t -+ 1 (V, int x, int y) by the divergence
// theorem (per triangle d = (v1 - v0) x (v2 - v0), h_k the complete
// homogeneous symmetric polynomials of its vertex coordinates:
// V += d_x h1(x)/6, int x += d_x h2(x)/24, int x^2 += d_x h3(x)/60, likewise
// for y), block partials and a last-block fixed-order sum; that block then
// advances the body (Sec. 4.3, explicit Euler on the free degrees: X += U,
// U += F/m, psi += omega, I omega += M_z with I of the new pose) and resets
// the lattice box the pose kernel fills.
constexpr int MASS_SUMS = 11;

__device__ __forceinline__ void mesh_triangle_sums(const GeomParams &G, int k, double t, bool second,
                                                   double &v, double &sx, double &sy, double &sxx, double &syy)
{
    double P[3][2];
    double Z[3];
    for (int m = 0; m < 3; ++m) {
        const int iv = G.mesh_tris[3 * k + m];
        const double s = G.mesh_rest[3 * iv];
        P[m][0] = s;
        P[m][1] = swimmer_midline(G, s, t) + G.mesh_rest[3 * iv + 1];
        Z[m] = G.mesh_rest[3 * iv + 2];
    }
    const double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], Z[1] - Z[0]};
    const double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], Z[2] - Z[0]};
    const double dx = e1[1] * e2[2] - e1[2] * e2[1], dy = e1[2] * e2[0] - e1[0] * e2[2];
    double h1[2], h2[2], h3[2];
    for (int a = 0; a < 2; ++a) {
        const double x0 = P[0][a], x1 = P[1][a], x2 = P[2][a];
        h1[a] = x0 + x1 + x2;
        h2[a] = x0 * x0 + x1 * x1 + x2 * x2 + x0 * x1 + x0 * x2 + x1 * x2;
        h3[a] = second ? x0 * x0 * x0 + x1 * x1 * x1 + x2 * x2 * x2 + x0 * x0 * (x1 + x2) + x1 * x1 * (x0 + x2) +
                             x2 * x2 * (x0 + x1) + x0 * x1 * x2
                       : 0.0;
    }
    v = dx * h1[0] / 6.0;
    sx = dx * h2[0] / 24.0;
    sy = dy * h2[1] / 24.0;
    sxx = dx * h3[0] / 60.0;
    syy = dy * h3[1] / 60.0;
}

__global__ void __launch_bounds__(MESH_THREADS) mesh_mass_kernel(const Lattice L, const GeomParams G,
                                                                 const DevBody *__restrict__ prev,
                                                                 DevBody *__restrict__ next, int advance)
{
    const double t = advance ? prev->t + 1.0 : prev->t;
    double acc[MASS_SUMS] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < G.n_triangles) {
        double v, sx, sy, sxx, syy;
        mesh_triangle_sums(G, k, t, true, v, sx, sy, sxx, syy);
        acc[0] = v; acc[1] = sx; acc[2] = sy; acc[3] = sxx; acc[4] = syy;
        mesh_triangle_sums(G, k, t + 1.0, false, v, sx, sy, sxx, syy);
        acc[5] = v; acc[6] = sx; acc[7] = sy;
        mesh_triangle_sums(G, k, t - 1.0, false, v, sx, sy, sxx, syy);
        acc[8] = v; acc[9] = sx; acc[10] = sy;
    }
    __shared__ double sm[MESH_THREADS / 32][MASS_SUMS];
    __shared__ bool last;
    for (int c = 0; c < MASS_SUMS; ++c) {
        double x = acc[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5][c] = x;
    }
    __syncthreads();
    if (threadIdx.x < MASS_SUMS) {
        double x = 0;
        for (int w = 0; w < MESH_THREADS / 32; ++w) x += sm[w][threadIdx.x];
        G.mesh_partials[blockIdx.x * MASS_SUMS + threadIdx.x] = x;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(G.mesh_ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double S[MASS_SUMS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = w; c < MASS_SUMS; c += MESH_THREADS / 32) {
        double x = 0;
        for (int b = lane; b < (int)gridDim.x; b += 32) x += ((volatile double *)G.mesh_partials)[b * MASS_SUMS + c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) S[c] = x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double V = S[0], rho = G.mass / V;
    const double cx = S[1] / V, cy = S[2] / V;
    const double Izz = rho * ((S[3] + S[4]) - V * (cx * cx + cy * cy));
    double X[3], U[3];
    for (int a = 0; a < 3; ++a) { X[a] = prev->X[a]; U[a] = prev->U[a]; }
    double psi = prev->psi, omega = prev->omega, Iw;
    if (advance) {
        for (int a = 0; a < 2; ++a)
            if (G.free_motion & (1 << a)) {
                X[a] = X[a] + U[a];
                U[a] = U[a] + prev->F[a] * G.inv_mass;
            }
        if (G.free_motion & 4) {
            psi = psi + omega;
            Iw = prev->Iw + prev->M[2];
            omega = Iw / Izz;
        } else {
            Iw = Izz * omega;
        }
    } else {
        Iw = Izz * omega;
    }
    for (int a = 0; a < 3; ++a) { next->X[a] = X[a]; next->U[a] = U[a]; }
    next->t = t;
    next->psi = psi;
    next->omega = omega;
    next->Iw = Iw;
    next->Izz = Izz;
    next->com[0] = cx;
    next->com[1] = cy;
    next->com_dot[0] = (S[6] / S[5] - S[9] / S[8]) / 2.0;
    next->com_dot[1] = (S[7] / S[5] - S[10] / S[8]) / 2.0;
    next->ibox[0] = 0x7fffffff;
    next->ibox[1] = -0x7fffffff;
    next->ibox[2] = 0x7fffffff;
    next->ibox[3] = -0x7fffffff;
    *G.mesh_ticket = 0u;
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
        cudaError_t e;
        if (G.com_frame && (e = launch_mesh_body(L, G, S, prev, true, s, nlaunch)) != cudaSuccess) return e;
        if ((e = launch_mesh_prepare(L, G, S, prev, true, s, nlaunch)) != cudaSuccess) return e;
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

cudaError_t launch_sweep_init(const Lattice &L, const GeomParams &G, Scratch &S, int cur, cudaStream_t s)
{
    if (!sweep_ahead(G)) return cudaSuccess;
    sweep_init_kernel<<<1, 32, 0, s>>>(L, G, S.body + cur);
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
    DevBody *next = S.body + (advance ? prev ^ 1 : prev);
    mesh_pose_kernel<<<nb_v > 0 ? nb_v : 1, MESH_THREADS, 0, s>>>(L, G, S.body + prev, next, advance ? 1 : 0, ncols,
                                                                    ncells);
    mesh_bin_kernel<<<nb_t > 0 ? nb_t : 1, MESH_THREADS, 0, s>>>(L, G, S.body + prev, next, advance ? 1 : 0);
    *nlaunch += 2;
    return cudaGetLastError();
}

cudaError_t launch_mesh_mark_initial(const Lattice &L, const GeomParams &G, Scratch &S, int cur,
                                     uint8_t *flags, cudaStream_t s)
{
    int n = 0;
    cudaError_t e;
    if (G.com_frame && (e = launch_mesh_body(L, G, S, cur, false, s, &n)) != cudaSuccess) return e;
    e = launch_mesh_prepare(L, G, S, cur, false, s, &n);
    if (e != cudaSuccess) return e;
    mesh_mark_initial_kernel<<<band_blocks(G), GEOM_THREADS, 0, s>>>(L, G, S.body + cur, flags);
    return cudaGetLastError();
}

cudaError_t launch_mesh_body(const Lattice &L, const GeomParams &G, Scratch &S, int prev, bool advance,
                             cudaStream_t s, int *nlaunch)
{
    const int nb_t = (G.n_triangles + MESH_THREADS - 1) / MESH_THREADS;
    mesh_mass_kernel<<<nb_t > 0 ? nb_t : 1, MESH_THREADS, 0, s>>>(L, G, S.body + prev,
                                                                   S.body + (advance ? prev ^ 1 : prev),
                                                                   advance ? 1 : 0);
    *nlaunch += 1;
    return cudaGetLastError();
}

// replaces the force and torque of a body state, the running sums following
__global__ void set_force_kernel(DevBody *__restrict__ b, Force6 fm)
{
    if (threadIdx.x != 0) return;
    for (int a = 0; a < 3; ++a) {
        b->F_sum[a] = __dadd_rn(__dsub_rn(b->F_sum[a], b->F[a]), fm.v[a]);
        b->M_sum[a] = __dadd_rn(__dsub_rn(b->M_sum[a], b->M[a]), fm.v[3 + a]);
        b->F[a] = fm.v[a];
        b->M[a] = fm.v[3 + a];
    }
}

// the force and torque of a body state from n partial sums (6 doubles each,
// device), added in part order starting from part 0; running sums follow
__global__ void sum_force_kernel(DevBody *__restrict__ b, const double *__restrict__ parts, int n)
{
    if (threadIdx.x != 0) return;
    double fm[6];
    for (int k = 0; k < 6; ++k) fm[k] = parts[k];
    for (int p = 1; p < n; ++p)
        for (int k = 0; k < 6; ++k) fm[k] = __dadd_rn(fm[k], parts[6 * (size_t)p + k]);
    for (int a = 0; a < 3; ++a) {
        b->F_sum[a] = __dadd_rn(__dsub_rn(b->F_sum[a], b->F[a]), fm[a]);
        b->M_sum[a] = __dadd_rn(__dsub_rn(b->M_sum[a], b->M[a]), fm[3 + a]);
        b->F[a] = fm[a];
        b->M[a] = fm[3 + a];
    }
}

cudaError_t launch_sum_force(Scratch &S, int cur, const double *parts, int n, cudaStream_t s)
{
    sum_force_kernel<<<1, 32, 0, s>>>(S.body + cur, parts, n);
    return cudaGetLastError();
}

cudaError_t launch_set_force(Scratch &S, int cur, const double fm[6], cudaStream_t s)
{
    Force6 v;
    for (int k = 0; k < 6; ++k) v.v[k] = fm[k];
    set_force_kernel<<<1, 32, 0, s>>>(S.body + cur, v);
    return cudaGetLastError();
}

}  // namespace lbm
