// Two-level block refinement (arXiv 1608.04658, Sec. 4.2: the airfoil runs on
// a grid with two levels of resolution; the refinement algorithm is cited,
// not stated).  One fine block of ratio 2 inside a bodiless coarse lattice:
//
//   - fine node j (per axis) sits at coarse coordinate lo + j/2, j = 0 .. 2m
//     (m = hi - lo); the fine lattice has 2m + 2 nodes per axis, periodic
//     faces that no interior pull reaches, and a last pad layer nothing reads;
//   - acoustic scaling: two fine steps per coarse step, the same rho and u on
//     both levels, twice the viscosity in fine lattice units;
//   - the fine nodes on the block's surface are not updated by the fine
//     level (flagged solid for its bulk launch): their post-collision state
//     at fine time t' is the fine collision of a state rebuilt from the coarse
//     pre-collision moments (rho, u, Pi^neq) at t', trilinear in space from
//     the coarse nodes of the block's surface and linear in time;
//   - the coarse nodes strictly inside the block are skipped by the coarse
//     bulk launch; those one layer inside its surface (the only ones a
//     coarse update pulls from) take the coarse collision of a state rebuilt
//     from the pre-collision moments of the coincident fine node;
//   - a rebuilt state is the entropic equilibrium (Eq. feq_min) at (rho, u)
//     plus the second-order Hermite term of Grad's distribution (Eq. grad)
//     carrying the donor's Pi^neq = Pi - Pi(f^eq(rho, u)), rescaled by the
//     ratio of relaxation time x time step of the levels: b_c / (2 b_f)
//     coarse to fine, 2 b_f / b_c fine to coarse.
//
// Per coarse step: coarse surface moments at t+1 (pulled from the coarse
// state at t), the coarse bulk launch off the block's inside, two fine bulk
// launches, the surface fills (at t + 1/2 from the mean of the moments at t
// and t+1, at t+1 from those at t+1) and the coarse layer inside the surface
// from the fine state at t + 1/2's pulls; the fine launches on the shared
// stream, the rest beside them on a second stream.
// Moments are kept in the collision's arithmetic (double for FP64 storage,
// float otherwise) as rho - rho0, u, Pi^neq, one array per quantity.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>

#include "ctx.cuh"
#include "kbc.cuh"

using namespace lbm;

namespace lbm {

constexpr int NMOM = 10;  // rho - rho0, u (3), Pi^neq xx yy zz xy xz yz
constexpr int REFINE_THREADS = 128;

// A box of E[0] x E[1] x E[2] nodes whose surface lies along the closed
// axes only (along an open axis the box wraps around and has no ends).
struct SurfBox {
    int E[3];
    int closed[3];
};

// nodes of the box with some closed coordinate at 0 or E - 1
__host__ __device__ inline long long surface_count(const SurfBox &S)
{
    long long all = 1, in = 1;
    for (int a = 0; a < 3; ++a) {
        all *= S.E[a];
        in *= S.closed[a] ? S.E[a] - 2 : S.E[a];
    }
    return all - in;
}

// k-th of those nodes: the two end slabs of the closed axes in the order z,
// y, x, each slab without the nodes of the slabs before it (x fastest
// within a slab); *axis = the closed axis whose end slab holds the node.
// Surface counts stay far below 2^31, so the index arithmetic is 32-bit.
__device__ inline void surface_node(int k, const SurfBox &S, int c[3], int *axis = nullptr)
{
    int done[3] = {0, 0, 0};
    for (int t = 0; t < 3; ++t) {
        const int a = 2 - t;
        if (!S.closed[a]) continue;
        int r[3];
        for (int b = 0; b < 3; ++b) r[b] = b == a ? 1 : (done[b] ? S.E[b] - 2 : S.E[b]);
        const int slab = r[0] * r[1] * r[2];
        if (k < 2 * slab) {
            const bool far = k >= slab;
            if (far) k -= slab;
            c[a] = far ? S.E[a] - 1 : 0;
            for (int b = 0; b < 3; ++b) {
                if (b == a) continue;
                c[b] = k % r[b] + (done[b] ? 1 : 0);
                k /= r[b];
            }
            if (axis) *axis = a;
            return;
        }
        k -= 2 * slab;
        done[a] = 1;
    }
    c[0] = c[1] = c[2] = 0;  // k beyond the count (not reached)
    if (axis) *axis = 0;
}

// v wrapped into [0, n) when it is at most one period off
__device__ inline int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// (rho - rho0, u, Pi^neq) of the shifted pre-collision populations g
template <typename R>
__device__ inline void node_moments(const R g[Q], R rho0, R M[NMOM])
{
    R drho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += g[i];
        j[0] += R(cx_of(i)) * g[i];
        j[1] += R(cy_of(i)) * g[i];
        j[2] += R(cz_of(i)) * g[i];
    }
    const R rho = rho0 + drho;
    const R u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    R ex[3], ey[3], ez[3], rx[3], ry[3], rz[3];
    axis_eq(u[0], ex, rx);
    axis_eq(u[1], ey, ry);
    axis_eq(u[2], ez, rz);
    R P[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R d = g[i] - shifted_feq<R>(i, drho, rho, ex, ey, ez);
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        P[0] += R(cx * cx) * d;
        P[1] += R(cy * cy) * d;
        P[2] += R(cz * cz) * d;
        P[3] += R(cx * cy) * d;
        P[4] += R(cx * cz) * d;
        P[5] += R(cy * cz) * d;
    }
    M[0] = drho;
    M[1] = u[0];
    M[2] = u[1];
    M[3] = u[2];
#pragma unroll
    for (int k = 0; k < 6; ++k) M[4 + k] = P[k];
}

// shifted state f^eq(rho, u) + W_i (9/2) s Pi^neq : (c_i c_i - I/3) - W_i rho0
template <typename R>
__device__ inline void rebuild(const R M[NMOM], R s, R rho0, R g[Q])
{
    const R drho = M[0], rho = rho0 + drho;
    R ex[3], ey[3], ez[3], rx[3], ry[3], rz[3];
    axis_eq(M[1], ex, rx);
    axis_eq(M[2], ey, ry);
    axis_eq(M[3], ez, rz);
    const R third = R(1) / R(3);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        const R h = (R(cx * cx) - third) * M[4] + (R(cy * cy) - third) * M[5] + (R(cz * cz) - third) * M[6] +
                    R(2 * cx * cy) * M[7] + R(2 * cx * cz) * M[8] + R(2 * cy * cz) * M[9];
        g[i] = shifted_feq<R>(i, drho, rho, ex, ey, ez) + weight<R>(i) * (R(4.5) * s * h);
    }
}

struct Box3 {
    int lo[3];    // block corner in coarse nodes (0 on a spanned axis)
    int m[3];     // hi - lo per axis (n on a spanned axis)
    int full[3];  // 1: the block spans this periodic axis of the coarse box
    int n[3];     // coarse lattice size
    // coarse box (moments), fine surface box and the coarse layer inside the
    // surface, each with the spanned axes open
    __host__ __device__ SurfBox coarse_box() const
    {
        SurfBox S;
        for (int a = 0; a < 3; ++a) {
            S.E[a] = full[a] ? n[a] : m[a] + 1;
            S.closed[a] = !full[a];
        }
        return S;
    }
    __host__ __device__ SurfBox fine_box() const
    {
        SurfBox S;
        for (int a = 0; a < 3; ++a) {
            S.E[a] = full[a] ? 2 * n[a] : 2 * m[a] + 1;
            S.closed[a] = !full[a];
        }
        return S;
    }
    __host__ __device__ SurfBox shell_box() const
    {
        SurfBox S;
        for (int a = 0; a < 3; ++a) {
            S.E[a] = full[a] ? n[a] : m[a] - 1;
            S.closed[a] = !full[a];
        }
        return S;
    }
};

// Coarse pre-collision moments on the block's surface: PULL, the pulls of the
// next step from state f (the coarse state at t) into M, and the mean of the
// moments at t (Mt) and those into Mh (the half step's); otherwise f's own
// populations (the initial state) into M.  M[q * nbox + b], b the node's
// position in the block's coarse box.
template <typename S, bool PULL>
__global__ void __launch_bounds__(REFINE_THREADS) refine_moments_kernel(const Lattice L, const S *__restrict__ f,
                                                                        const Box3 B,
                                                                        typename Codec<S>::R *__restrict__ M,
                                                                        const typename Codec<S>::R *__restrict__ Mt,
                                                                        typename Codec<S>::R *__restrict__ Mh)
{
    using R = typename Codec<S>::R;
    const SurfBox SB = B.coarse_box();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= surface_count(SB)) return;
    int bc[3];
    surface_node(k, SB, bc);
    const int x = B.lo[0] + bc[0], y = B.lo[1] + bc[1], z = B.lo[2] + bc[2];
    R g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // a closed axis keeps its sources inside the box; a spanned one wraps
        const int sx = PULL ? wrap1(x - cx_of(i), L.nx) : x, sy = PULL ? wrap1(y - cy_of(i), L.ny) : y,
                  sz = PULL ? wrap1(z - cz_of(i), L.nz) : z;
        g[i] = Codec<S>::load(f + L.plane[i] + (sx + L.nx * (sy + L.ny * sz)));
    }
    R Mn[NMOM];
    node_moments<R>(g, (R)L.rho0, Mn);
    const long long nbox = (long long)SB.E[0] * SB.E[1] * SB.E[2];
    const long long b = bc[0] + (long long)SB.E[0] * (bc[1] + (long long)SB.E[1] * bc[2]);
#pragma unroll
    for (int q = 0; q < NMOM; ++q) {
        M[q * nbox + b] = Mn[q];
        if (PULL) Mh[q * nbox + b] = R(0.5) * (Mt[q * nbox + b] + Mn[q]);
    }
}

// Fine surface nodes of fine state ff from the coarse moments Ms of that
// time (the moments at t+1, or the half step's mean): trilinear from the
// coarse surface (each odd fine coordinate takes the mean of the two coarse
// nodes around it; a surface node's coordinate normal to its face is even,
// so at most the two in-plane ones are odd: four corners, some repeated),
// rebuilt with the coarse-to-fine factor and collided with the fine b.
template <typename S, bool EXACT>
__global__ void __launch_bounds__(REFINE_THREADS) refine_fill_kernel(const Lattice Lf, S *__restrict__ ff,
                                                                     const Box3 B,
                                                                     const typename Codec<S>::R *__restrict__ Ms,
                                                                     typename Codec<S>::R s_cf,
                                                                     const uint8_t *__restrict__ flags,
                                                                     int *__restrict__ st0, int *__restrict__ st1)
{
    using R = typename Codec<S>::R;
    const SurfBox SF = B.fine_box(), SC = B.coarse_box();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= surface_count(SF)) return;
    int j[3], a0;
    surface_node(k, SF, j, &a0);
    const int p = a0 == 0 ? 1 : 0, q = a0 == 2 ? 1 : 2;  // the in-plane axes
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = j[a] >> 1;
        hi[a] = lo[a] + (j[a] & 1);
        if (B.full[a] && hi[a] == B.n[a]) hi[a] = 0;  // the node after the last of a spanned axis
    }
    const int A0 = SC.E[0], A1 = SC.E[1];
    const int nbox = A0 * A1 * SC.E[2];
    int cidx[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int b[3] = {lo[0], lo[1], lo[2]};
        if (c & 1) b[p] = hi[p];
        if (c & 2) b[q] = hi[q];
        cidx[c] = b[0] + A0 * (b[1] + A1 * b[2]);
    }
    R M[NMOM];
#pragma unroll
    for (int m = 0; m < NMOM; ++m)
        M[m] = R(0.25) * ((Ms[m * nbox + cidx[0]] + Ms[m * nbox + cidx[1]]) +
                          (Ms[m * nbox + cidx[2]] + Ms[m * nbox + cidx[3]]));
    R g[Q];
    rebuild<R>(M, s_cf, (R)Lf.rho0, g);
    const int n = j[0] + Lf.nx * (j[1] + Lf.ny * j[2]);
    // a fine body whose band reached the surface has cleared its mark there
    const int bad = (kbc_collide<R, EXACT>(g, (R)Lf.beta, (R)Lf.inv_beta, (R)Lf.rho0, Lf.gamma_mode) ? 0 : ST_UNSTABLE) |
                    ((flags[n] & FL_SOLID) ? 0 : ST_BAND_OVERFLOW);
    if (bad) {
        atomicOr(st0, bad);
        atomicOr(st1, bad);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) Codec<S>::store(ff + Lf.plane[i] + n, g[i]);
}

// Coarse nodes one layer inside the block's surface at t+1: the pulls of the
// coincident fine node 2(X - lo) from the fine state at t + 1/2, their
// moments rebuilt with the fine-to-coarse factor and collided with the
// coarse b, written to the coarse state at t+1.
template <typename S, bool EXACT>
__global__ void __launch_bounds__(REFINE_THREADS) refine_restrict_kernel(const Lattice Lc, S *__restrict__ fc,
                                                                         const Lattice Lf,
                                                                         const S *__restrict__ ff, const Box3 B,
                                                                         typename Codec<S>::R s_fc,
                                                                         int *__restrict__ status)
{
    using R = typename Codec<S>::R;
    const SurfBox SS = B.shell_box();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= surface_count(SS)) return;
    int bs[3], X[3], j[3];
    surface_node(k, SS, bs);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        X[a] = B.full[a] ? bs[a] : B.lo[a] + 1 + bs[a];
        j[a] = 2 * (X[a] - B.lo[a]);
    }
    R g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i)
        g[i] = Codec<S>::load(ff + Lf.plane[i] + (wrap1(j[0] - cx_of(i), Lf.nx) +
                                                  Lf.nx * (wrap1(j[1] - cy_of(i), Lf.ny) +
                                                           Lf.ny * wrap1(j[2] - cz_of(i), Lf.nz))));
    R M[NMOM];
    node_moments<R>(g, (R)Lf.rho0, M);
    rebuild<R>(M, s_fc, (R)Lc.rho0, g);
    if (!kbc_collide<R, EXACT>(g, (R)Lc.beta, (R)Lc.inv_beta, (R)Lc.rho0, Lc.gamma_mode)) atomicOr(status, ST_UNSTABLE);
    const int n = X[0] + Lc.nx * (X[1] + Lc.ny * X[2]);
#pragma unroll
    for (int i = 0; i < Q; ++i) Codec<S>::store(fc + Lc.plane[i] + n, g[i]);
}

// fine-level marks: the block's surface and the pad are marked solid, so
// the fine bulk launch does not update them (the marks of a fine body,
// inside the block, are left as they are)
__global__ void refine_flags_kernel(uint8_t *flags, int nx, int ny, int nz, const Box3 B)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)nx * ny * nz) return;
    const int c[3] = {(int)(n % nx), (int)((n / nx) % ny), (int)(n / ((long long)nx * ny))};
    bool inner = true;
    for (int a = 0; a < 3; ++a)
        if (!B.full[a] && (c[a] < 1 || c[a] >= 2 * B.m[a])) inner = false;
    if (!inner) flags[n] |= FL_SOLID;
}

static unsigned blocks_for(long long n) { return (unsigned)((n + REFINE_THREADS - 1) / REFINE_THREADS); }

template <typename F>
static cudaError_t dispatch_exact(int storage, bool exact, F &&fn)
{
    return dispatch_storage(storage, [&](auto tag) {
        return exact ? fn(tag, std::true_type{}) : fn(tag, std::false_type{});
    });
}

}  // namespace lbm

// ---------------------------------------------------------------- host side
struct lbm_refine {
    lbm_ctx *c = nullptr, *f = nullptr;
    cudaStream_t stream = nullptr;    // the levels' shared stream (the caller's)
    Box3 B{};
    void *M[2] = {nullptr, nullptr};  // moments at t (slot mcur) and t+1
    void *Mh = nullptr;               // their mean, the half step's moments
    int mcur = 0;
    int *sweep = nullptr;             // device {lo + 1 (3), m - 1 (3)}: the coarse launch skips it
    // fork of the side stream (the coarse context's, unused without a body),
    // fine launch 1 done, first fill done, side work of the step done
    cudaEvent_t ev_fork = nullptr, ev_fine1 = nullptr, ev_fill = nullptr, ev_side = nullptr;
    bool ready = false;
    double s_cf = 0, s_fc = 0;
    int64_t launches = 0;
    int body_launches = 0;  // launches of a fine body's chain in the current lbm_refine_step
};

namespace {

lbm_status rfail(lbm_ctx *c, lbm_status st, const std::string &msg)
{
    if (c) c->err = msg;
    return st;
}

#define RF_CUDA(call, where)                                                                            \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return rfail(r->c, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void release(lbm_refine *r)
{
    for (cudaEvent_t e : {r->ev_fork, r->ev_fine1, r->ev_fill, r->ev_side})
        if (e) cudaEventDestroy(e);
    // the scratch came from the coarse context's allocator
    for (void *p : {r->M[0], r->M[1], r->Mh, (void *)r->sweep}) ctx_release(r->c, p);
    delete r;
}

cudaError_t launch_marks(const lbm_refine *r)
{
    const Lattice &Lf = r->f->L;
    refine_flags_kernel<<<blocks_for(Lf.N), REFINE_THREADS, 0, r->f->stream>>>(r->f->flags, Lf.nx, Lf.ny, Lf.nz, r->B);
    return cudaGetLastError();
}

cudaError_t launch_moments(const lbm_refine *r, const void *f, void *M, const void *Mt, void *Mh, bool pull,
                           cudaStream_t st)
{
    const long long n = surface_count(r->B.coarse_box());
    const lbm_ctx *c = r->c;
    return dispatch_storage(c->storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using R = typename Codec<S>::R;
        if (pull)
            refine_moments_kernel<S, true><<<blocks_for(n), REFINE_THREADS, 0, st>>>(c->L, (const S *)f, r->B, (R *)M,
                                                                                    (const R *)Mt, (R *)Mh);
        else
            refine_moments_kernel<S, false><<<blocks_for(n), REFINE_THREADS, 0, st>>>(c->L, (const S *)f, r->B, (R *)M,
                                                                                     nullptr, nullptr);
        return cudaGetLastError();
    });
}

cudaError_t launch_fill(const lbm_refine *r, void *ff, const void *Ms, cudaStream_t st)
{
    const long long n = surface_count(r->B.fine_box());
    const lbm_ctx *f = r->f;
    // both body slots: the step that reads the flag may be either
    int *st0 = &f->S.body[0].status, *st1 = &f->S.body[1].status;
    return dispatch_exact(f->storage, f->L.gamma_mode == LBM_GAMMA_EXACT, [&](auto tag, auto ex) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using R = typename Codec<S>::R;
        refine_fill_kernel<S, decltype(ex)::value><<<blocks_for(n), REFINE_THREADS, 0, st>>>(
            f->L, (S *)ff, r->B, (const R *)Ms, (R)r->s_cf, f->flags, st0, st1);
        return cudaGetLastError();
    });
}

cudaError_t launch_restrict(const lbm_refine *r, void *fc, const void *ff, cudaStream_t st)
{
    const long long n = surface_count(r->B.shell_box());
    const lbm_ctx *c = r->c;
    int *status = &c->S.body[c->bcur].status;
    return dispatch_exact(c->storage, c->L.gamma_mode == LBM_GAMMA_EXACT, [&](auto tag, auto ex) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using R = typename Codec<S>::R;
        refine_restrict_kernel<S, decltype(ex)::value><<<blocks_for(n), REFINE_THREADS, 0, st>>>(
            c->L, (S *)fc, r->f->L, (const S *)ff, r->B, (R)r->s_fc, status);
        return cudaGetLastError();
    });
}

// One fine step from fa to fb over the block's interior on the shared
// stream: one flag-aware bulk launch, or with a fine body the fine
// context's own step in the sequential order (geometry, refill, boundary
// and force beside the flag-aware bulk launch), whose buffers then advance.
cudaError_t fine_step(lbm_refine *r, void *fa, void *fb, int *status, cudaStream_t main)
{
    lbm_ctx *f = r->f;
    if (f->has_body) {
        int n = 0;
        const cudaError_t e = ctx_step_flagged(f, &n);
        r->body_launches += n - 1;  // the bulk launch is one of the seven counted per step
        return e;
    }
    cudaError_t e = ctx_prof_mark(f, 0);
    if (e == cudaSuccess) e = launch_bulk(f->storage, f->L, fa, fb, f->flags, status, main);
    if (e == cudaSuccess) e = ctx_prof_mark(f, 1);
    return e;
}

}  // namespace

extern "C" {

lbm_status lbm_refine_create(lbm_ctx *coarse, lbm_ctx *fine, const int32_t lo[3], const int32_t hi[3],
                             lbm_refine **out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!coarse || !fine || !lo || !hi || coarse == fine) return LBM_ERR_ARG;
    const Lattice &Lc = coarse->L, &Lf = fine->L;
    const int n[3] = {Lc.nx, Lc.ny, Lc.nz}, nf[3] = {Lf.nx, Lf.ny, Lf.nz};
    int full[3], closed = 0;
    for (int a = 0; a < 3; ++a) {
        // lo = 0, hi = n on a periodic axis: the block spans it
        full[a] = lo[a] == 0 && hi[a] == n[a] && Lc.face[2 * a] == LBM_FACE_PERIODIC;
        if (full[a]) {
            if (nf[a] != 2 * n[a])
                return rfail(coarse, LBM_ERR_ARG, "lbm_refine_create: the fine lattice needs 2n nodes along a spanned axis");
            continue;
        }
        closed++;
        if (lo[a] < 1 || hi[a] > n[a] - 2 || hi[a] - lo[a] < 3)
            return rfail(coarse, LBM_ERR_ARG, "lbm_refine_create: the block needs 1 <= lo, hi <= n - 2, hi - lo >= 3");
        if (nf[a] != 2 * (hi[a] - lo[a]) + 2)
            return rfail(coarse, LBM_ERR_ARG, "lbm_refine_create: the fine lattice needs 2 (hi - lo) + 2 nodes per axis");
    }
    if (!closed) return rfail(coarse, LBM_ERR_ARG, "lbm_refine_create: a block spanning every axis has no surface");
    for (int k = 0; k < 6; ++k)
        if (Lf.face[k] != LBM_FACE_PERIODIC)
            return rfail(coarse, LBM_ERR_ARG, "lbm_refine_create: the fine lattice's faces must be periodic");
    if (coarse->storage != fine->storage || Lc.gamma_mode != Lf.gamma_mode || Lc.rho0 != Lf.rho0)
        return rfail(coarse, LBM_ERR_ARG, "lbm_refine_create: storage, stabilizer and rho0 must match");
    if (coarse->stream != fine->stream)
        return rfail(coarse, LBM_ERR_ARG, "lbm_refine_create: both levels must enqueue on the same stream");
    // twice the coarse viscosity in fine lattice units: b_f = b_c / (2 - b_c)
    const double bf = Lc.beta / (2.0 - Lc.beta);
    if (!(std::fabs(Lf.beta - bf) <= 1e-12 * bf))
        return rfail(coarse, LBM_ERR_ARG, "lbm_refine_create: the fine viscosity must be twice the coarse one");
    if (coarse->has_body || coarse->slab_zper || fine->slab_zper || !fine->flags)
        return rfail(coarse, LBM_ERR_ARG, "lbm_refine_create: a bodiless coarse level and unsplit contexts");

    lbm_refine *r = new (std::nothrow) lbm_refine;
    if (!r) return LBM_ERR_OOM;
    r->c = coarse;
    r->f = fine;
    r->stream = coarse->stream;
    for (int a = 0; a < 3; ++a) {
        r->B.lo[a] = lo[a];
        r->B.m[a] = hi[a] - lo[a];
        r->B.full[a] = full[a];
        r->B.n[a] = n[a];
    }
    r->s_cf = Lc.beta / (2.0 * Lf.beta);
    r->s_fc = 2.0 * Lf.beta / Lc.beta;
    const size_t rsz = coarse->storage == LBM_FP64 ? sizeof(double) : sizeof(float);
    const SurfBox SC = r->B.coarse_box();
    const size_t nbox = (size_t)SC.E[0] * SC.E[1] * SC.E[2];
    if (ctx_malloc(coarse, &r->M[0], NMOM * nbox * rsz) != cudaSuccess ||
        ctx_malloc(coarse, &r->M[1], NMOM * nbox * rsz) != cudaSuccess ||
        ctx_malloc(coarse, &r->Mh, NMOM * nbox * rsz) != cudaSuccess ||
        ctx_alloc(coarse, &r->sweep, 6) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev_fine1, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev_fill, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev_side, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        release(r);
        return rfail(coarse, LBM_ERR_OOM, "lbm_refine_create: device allocation failed");
    }
    // the coarse launch skips the block's inside: along a spanned axis all of it
    int sw[6];
    for (int a = 0; a < 3; ++a) {
        sw[a] = full[a] ? 0 : lo[a] + 1;
        sw[3 + a] = full[a] ? n[a] : r->B.m[a] - 1;
    }
    cudaError_t e = cudaMemcpyAsync(r->sweep, sw, sizeof(sw), cudaMemcpyHostToDevice, coarse->stream);
    if (e == cudaSuccess) e = launch_marks(r);
    if (e == cudaSuccess) e = cudaStreamSynchronize(coarse->stream);
    if (e != cudaSuccess) {
        release(r);
        return rfail(coarse, LBM_ERR_CUDA, std::string("lbm_refine_create: ") + cudaGetErrorString(e));
    }
    *out = r;
    return LBM_OK;
}

}  // extern "C"

namespace {

// file of the coupling's state: the coarse surface moments of the last step
struct RefineFileHeader {
    char magic[8];
    int32_t version, storage;
    int32_t lo[3], m[3], n[3], full[3];
    int64_t bytes;
};

RefineFileHeader refine_header(const lbm_refine *r, int64_t bytes)
{
    RefineFileHeader h{};
    memcpy(h.magic, "LBMREF01", 8);
    h.version = 1;
    h.storage = r->c->storage;
    for (int a = 0; a < 3; ++a) {
        h.lo[a] = r->B.lo[a];
        h.m[a] = r->B.m[a];
        h.n[a] = r->B.n[a];
        h.full[a] = r->B.full[a];
    }
    h.bytes = bytes;
    return h;
}

int64_t moment_bytes(const lbm_refine *r)
{
    const SurfBox SC = r->B.coarse_box();
    const int64_t rsz = r->c->storage == LBM_FP64 ? 8 : 4;
    return (int64_t)NMOM * SC.E[0] * SC.E[1] * SC.E[2] * rsz;
}

}  // namespace

extern "C" {

lbm_status lbm_refine_save(lbm_refine *r, const char *path)
{
    if (!r) return LBM_ERR_ARG;
    if (!path) return rfail(r->c, LBM_ERR_ARG, "lbm_refine_save: null path");
    if (!r->ready) return rfail(r->c, LBM_ERR_STATE, "lbm_refine_save: lbm_refine_init has not run");
    const int64_t bytes = moment_bytes(r);
    std::string buf((size_t)bytes, '\0');
    RF_CUDA(cudaStreamSynchronize(r->stream), "sync");
    RF_CUDA(cudaMemcpy(&buf[0], r->M[r->mcur], (size_t)bytes, cudaMemcpyDeviceToHost), "moments");
    const RefineFileHeader h = refine_header(r, bytes);
    FILE *fp = fopen(path, "wb");
    if (!fp) return rfail(r->c, LBM_ERR_ARG, std::string("lbm_refine_save: cannot open ") + path);
    bool ok = fwrite(&h, sizeof(h), 1, fp) == 1 && fwrite(buf.data(), 1, (size_t)bytes, fp) == (size_t)bytes;
    ok = (fclose(fp) == 0) && ok;
    return ok ? LBM_OK : rfail(r->c, LBM_ERR_ARG, std::string("lbm_refine_save: write failed for ") + path);
}

lbm_status lbm_refine_load(lbm_refine *r, const char *path)
{
    if (!r) return LBM_ERR_ARG;
    if (!path) return rfail(r->c, LBM_ERR_ARG, "lbm_refine_load: null path");
    FILE *fp = fopen(path, "rb");
    if (!fp) return rfail(r->c, LBM_ERR_ARG, std::string("lbm_refine_load: cannot open ") + path);
    const int64_t bytes = moment_bytes(r);
    const RefineFileHeader want = refine_header(r, bytes);
    RefineFileHeader h{};
    std::string buf((size_t)bytes, '\0');
    const bool ok = fread(&h, sizeof(h), 1, fp) == 1 && memcmp(&h, &want, sizeof(h)) == 0 &&
                    fread(&buf[0], 1, (size_t)bytes, fp) == (size_t)bytes;
    fclose(fp);
    if (!ok) return rfail(r->c, LBM_ERR_ARG, std::string("lbm_refine_load: ") + path + " does not match this coupling");
    RF_CUDA(cudaStreamSynchronize(r->stream), "sync");
    RF_CUDA(cudaMemcpy(r->M[r->mcur], buf.data(), (size_t)bytes, cudaMemcpyHostToDevice), "moments");
    RF_CUDA(launch_marks(r), "refine marks");
    RF_CUDA(cudaStreamSynchronize(r->stream), "sync");
    r->ready = true;
    return LBM_OK;
}

void lbm_refine_destroy(lbm_refine *r)
{
    if (!r) return;
    // the side stream's work is ordered before each step's end on this stream
    cudaStreamSynchronize(r->stream);
    release(r);
}

lbm_status lbm_refine_init(lbm_refine *r)
{
    NvtxRange nvtx_("lbm_refine_init");
    if (!r) return LBM_ERR_ARG;
    if (!r->c->initialised || !r->f->initialised)
        return rfail(r->c, LBM_ERR_STATE, "lbm_refine_init: both levels must hold their initial state");
    if (r->c->has_body) return rfail(r->c, LBM_ERR_ARG, "lbm_refine_init: the coarse level carries a body");
    // walls mark the whole box; the airfoil spans the fine lattice's z extent,
    // which only a block spanning z leaves without a surface
    if (r->f->has_body && (r->f->G.kind == LBM_BODY_PLANES || (r->f->G.kind == LBM_BODY_AIRFOIL && !r->B.full[2])))
        return rfail(r->c, LBM_ERR_UNSUPPORTED,
                     "lbm_refine_init: a fine body must be a sphere, a mesh, or an airfoil in a block spanning z");
    // lbm_set_geometry on the fine level clears the surface marks
    RF_CUDA(launch_marks(r), "refine marks");
    RF_CUDA(launch_moments(r, r->c->f[r->c->cur], r->M[r->mcur], nullptr, nullptr, false, r->c->stream),
            "refine moments");
    RF_CUDA(launch_fill(r, r->f->f[r->f->cur], r->M[r->mcur], r->c->stream), "refine fill");
    r->ready = true;
    return LBM_OK;
}

lbm_status lbm_refine_step(lbm_refine *r, int nsteps)
{
    NvtxRange nvtx_("lbm_refine_step");
    if (!r) return LBM_ERR_ARG;
    if (nsteps < 0) return rfail(r->c, LBM_ERR_ARG, "lbm_refine_step: nsteps < 0");
    if (!r->ready) return rfail(r->c, LBM_ERR_STATE, "lbm_refine_step: lbm_refine_init has not run");
    // a body set on the coarse level after the coupling was made
    if (r->c->has_body) return rfail(r->c, LBM_ERR_STATE, "lbm_refine_step: the coarse level carries a body");
    lbm_ctx *c = r->c, *f = r->f;
    // The fine launches run on the shared stream; the coupling kernels and
    // the coarse launch on the side stream beside them.  They write disjoint
    // nodes: the fine launches the block's interior, the fills its surface
    // (flagged solid to the fine launch), the coarse launch the nodes off the
    // block's inside, the restriction the layer inside the surface.  Orders
    // kept by events: the first fill (fine state at t + 1/2) before the second
    // fine launch reads it; the restriction (which pulls from the fine state
    // at t + 1/2) and the second fill (fine state at t + 1, read by the first
    // fine launch) after the first fine launch; the next step after all.
    cudaStream_t main = c->stream, side = c->side;
    for (int s = 0; s < nsteps; ++s) {
        void *ca = c->f[c->cur], *cb = c->f[c->cur ^ 1];
        void *fa = f->f[f->cur], *fb = f->f[f->cur ^ 1];
        void *Mt = r->M[r->mcur], *Mn = r->M[r->mcur ^ 1];
        int *cstat = &c->S.body[c->bcur].status, *fstat = &f->S.body[0].status;
        RF_CUDA(cudaEventRecord(r->ev_fork, main), "fork");
        RF_CUDA(cudaStreamWaitEvent(side, r->ev_fork, 0), "fork wait");
        RF_CUDA(launch_moments(r, ca, Mn, Mt, r->Mh, true, side), "refine moments");
        RF_CUDA(launch_fill(r, fb, r->Mh, side), "refine fill");
        RF_CUDA(cudaEventRecord(r->ev_fill, side), "fill event");
        RF_CUDA(launch_bulk(c->storage, c->L, ca, cb, nullptr, cstat, side, BULK_OUTSIDE, r->sweep), "coarse bulk");
        RF_CUDA(fine_step(r, fa, fb, fstat, main), "fine step");
        RF_CUDA(cudaEventRecord(r->ev_fine1, main), "fine event");
        RF_CUDA(cudaStreamWaitEvent(side, r->ev_fine1, 0), "fine wait");
        RF_CUDA(launch_restrict(r, cb, fb, side), "refine restrict");
        RF_CUDA(launch_fill(r, fa, Mn, side), "refine fill");
        RF_CUDA(cudaEventRecord(r->ev_side, side), "side event");
        RF_CUDA(cudaStreamWaitEvent(main, r->ev_fill, 0), "fill wait");
        RF_CUDA(fine_step(r, fb, fa, fstat, main), "fine step");
        RF_CUDA(cudaStreamWaitEvent(main, r->ev_side, 0), "side wait");
        c->cur ^= 1;
        r->mcur ^= 1;
    }
    r->launches = 7LL * nsteps + r->body_launches;
    c->launches = r->launches;
    r->body_launches = 0;
    return LBM_OK;
}

}  // extern "C"
