// C ABI of liblbm.so (declared in include/lbm.h): argument checks, scratch
// management and the per-step launch sequence.  Host code only enqueues
// kernels; the state, the body and its force never leave the device during
// lbm_step.
#include <cstddef>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.cuh"

using namespace lbm;

namespace {

lbm_status fail(lbm_ctx *c, lbm_status st, const std::string &msg)
{
    if (c) c->err = msg;
    return st;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(call, where)                                        \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);     \
    } while (0)

size_t elem_size(int storage)
{
    switch (storage) {
    case LBM_FP64: return 8;
    case LBM_FP32: return 4;
    case LBM_FP16: return 2;
    case LBM_BF16: return 2;
    default: return 0;
    }
}

double host_weight(int i)
{
    const int nz = (i / 9 != 1) + ((i / 3) % 3 != 1) + (i % 3 != 1);
    return nz == 0 ? 8.0 / 27.0 : nz == 1 ? 2.0 / 27.0 : nz == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
}

// shifted equilibrium for the EQ faces, exact product form (host, double)
void face_equilibrium(double rho0, const double u[3], double out[27])
{
    double fac[3][3];
    for (int a = 0; a < 3; ++a) {
        const double S = std::sqrt(1.0 + 3.0 * u[a] * u[a]);
        const double B = (2.0 * u[a] + S) / (1.0 - u[a]);
        fac[a][0] = (2.0 - S) / B;
        fac[a][1] = 2.0 - S;
        fac[a][2] = (2.0 - S) * B;
    }
    for (int i = 0; i < 27; ++i) {
        const int cx = i / 9, cy = (i / 3) % 3, cz = i % 3;
        out[i] = host_weight(i) * (rho0 * fac[0][cx] * fac[1][cy] * fac[2][cz] - rho0);
    }
}

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

// the body's scratch of lbm_set_geometry (through the context's allocator);
// the body slots of lbm_create too unless keep_body
void free_scratch(lbm_ctx *ctx, bool keep_body)
{
    Scratch &S = ctx->S;
    // a caller's allocator may hand the blocks out again at once
    if (ctx->dev_release && ctx->live_blocks) {
        cudaStreamSynchronize(ctx->stream);
        if (ctx->side) cudaStreamSynchronize(ctx->side);
    }
    for (void *p : {(void *)S.blist, (void *)S.bpos, (void *)S.ulist, (void *)S.upos, (void *)S.bforce,
                    (void *)S.partials, (void *)S.ticket, (void *)S.mesh_rest, (void *)S.mesh_pos,
                    (void *)S.mesh_vel, (void *)S.col_x, (void *)S.mesh_tris, (void *)S.col_count,
                    (void *)S.cell_count, (void *)S.cell_tri, (void *)S.mesh_status, (void *)S.tri_box,
                    (void *)S.mesh_ipos, (void *)S.mesh_frac, (void *)S.mesh_partials, (void *)S.mesh_ticket})
        ctx_release(ctx, p);
    DevBody *b = S.body;
    S = Scratch{};
    if (keep_body) S.body = b;
    else cudaFree(b);
}

}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_params *p, void *f_a, void *f_b, uint8_t *flags, void *stream,
                      lbm_ctx **out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!p || !f_a || !f_b || !flags) return LBM_ERR_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LBM_ERR_ARG;
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (27 * N >= (1LL << 31)) return LBM_ERR_ARG;  // 32-bit element offsets
    const size_t es = elem_size(p->storage);
    if (es == 0) return LBM_ERR_ARG;
    if (((uintptr_t)f_a % 16) || ((uintptr_t)f_b % 16)) return LBM_ERR_ARG;
    for (int k = 0; k < 6; ++k)
        if (p->face[k] < LBM_FACE_PERIODIC || p->face[k] > LBM_FACE_OUTFLOW) return LBM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if ((p->face[2 * a] == LBM_FACE_PERIODIC) != (p->face[2 * a + 1] == LBM_FACE_PERIODIC))
            return LBM_ERR_ARG;
    if (!(p->nu >= 0.0) || !std::isfinite(p->nu) || !(p->rho0 > 0.0)) return LBM_ERR_ARG;
    if (p->gamma_mode != LBM_GAMMA_ANALYTIC && p->gamma_mode != LBM_GAMMA_EXACT && p->gamma_mode != LBM_GAMMA_LBGK)
        return LBM_ERR_ARG;
    if (p->options != 0) return LBM_ERR_ARG;

    lbm_ctx *ctx = new (std::nothrow) lbm_ctx();
    if (!ctx) return LBM_ERR_OOM;
    Lattice &L = ctx->L;
    L.nx = p->nx; L.ny = p->ny; L.nz = p->nz; L.N = N;
    for (int i = 0; i < Q; ++i) L.plane[i] = (int)(i * N);
    for (int k = 0; k < 6; ++k) L.face[k] = p->face[k];
    L.gamma_mode = p->gamma_mode;
    L.beta = 1.0 / (6.0 * p->nu + 1.0);
    L.inv_beta = 6.0 * p->nu + 1.0;
    L.rho0 = p->rho0;
    for (int a = 0; a < 3; ++a) L.u_face[a] = p->u_face[a];
    face_equilibrium(p->rho0, p->u_face, L.g_face);
    L.beta_f = (float)L.beta;
    L.inv_beta_f = (float)L.inv_beta;
    L.rho0_f = (float)L.rho0;
    for (int i = 0; i < Q; ++i) L.g_face_f[i] = (float)L.g_face[i];
    ctx->storage = p->storage;
    ctx->elem = es;
    ctx->f[0] = f_a;
    ctx->f[1] = f_b;
    ctx->flags = flags;
    ctx->stream = (cudaStream_t)stream;
    if (dalloc(&ctx->S.body, 2) != cudaSuccess || dalloc(&ctx->tot_partials, (size_t)ctx->tot_blocks * 5) != cudaSuccess) {
        free_scratch(ctx, false);
        cudaFree(ctx->tot_partials);
        delete ctx;
        return LBM_ERR_OOM;
    }
    // the side stream carries the body's geometry and boundary work beside the
    // bulk launch on the caller's stream: the greatest priority, so its
    // blocks take the SM slots that bulk blocks free first
    int prio_least = 0, prio_greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) prio_greatest = 0;
    bool trial_ok = true;
    for (cudaEvent_t &e : ctx->ev_trial) trial_ok = trial_ok && cudaEventCreate(&e) == cudaSuccess;
    if (!trial_ok || cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        free_scratch(ctx, false);
        cudaFree(ctx->tot_partials);
        if (ctx->side) cudaStreamDestroy(ctx->side);
        if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
        if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
        for (cudaEvent_t e : ctx->ev_trial)
            if (e) cudaEventDestroy(e);
        delete ctx;
        return LBM_ERR_CUDA;
    }
    DevBody zero[2] = {};
    if (cudaMemcpyAsync(ctx->S.body, zero, sizeof(zero), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(flags, 0, (size_t)N, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        free_scratch(ctx, false);
        cudaFree(ctx->tot_partials);
        delete ctx;
        return LBM_ERR_CUDA;
    }
    *out = ctx;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    cudaStreamSynchronize(ctx->side);
    if (ctx->copy) cudaStreamSynchronize(ctx->copy);
    // the scratch goes back while the streams still exist (a caller's
    // allocator is given the context's stream with each block)
    free_scratch(ctx, false);
    ctx_release(ctx, ctx->plane);
    ctx->plane = nullptr;
    for (cudaEvent_t e : ctx->prof) cudaEventDestroy(e);
    cudaEventDestroy(ctx->ev_fork);
    cudaEventDestroy(ctx->ev_join);
    for (cudaEvent_t e : ctx->ev_trial) cudaEventDestroy(e);
    cudaStreamDestroy(ctx->side);
    if (ctx->copy) {
        cudaStreamSynchronize(ctx->copy);
        cudaEventDestroy(ctx->ev_step);
        for (cudaEvent_t e : ctx->ev_copy) cudaEventDestroy(e);
        for (cudaEvent_t e : ctx->ev_slot) cudaEventDestroy(e);
        cudaStreamDestroy(ctx->copy);
    }
    cudaFree(ctx->tot_partials);
    delete ctx;
}

lbm_status lbm_set_allocator(lbm_ctx *ctx, lbm_alloc_fn alloc, lbm_release_fn release, void *user)
{
    if (!ctx) return LBM_ERR_ARG;
    if ((alloc == nullptr) != (release == nullptr))
        return fail(ctx, LBM_ERR_ARG, "lbm_set_allocator: give both functions or neither");
    if (ctx->live_blocks != 0)
        return fail(ctx, LBM_ERR_STATE, "lbm_set_allocator: the context already holds scratch from another allocator");
    ctx->dev_alloc = alloc;
    ctx->dev_release = release;
    ctx->alloc_user = user;
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

}  // extern "C"

// The device address of a buffer the kernels may read: device or managed
// memory as it is, pinned host memory by its mapped device address; nullptr
// for memory the device cannot address (pageable host memory).
template <typename T>
static const T *device_view(const T *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return (const T *)a.devicePointer;
    return nullptr;
}

template <typename T>
static lbm_status init_state(lbm_ctx *ctx, const T *rho, const T *u, const T *xi, double amp, const char *name)
{
    NvtxRange nvtx_(name);
    if (!ctx) return LBM_ERR_ARG;
    if (!rho || !u) return fail(ctx, LBM_ERR_ARG, std::string(name) + ": rho and u are required");
    const T *drho = device_view(rho), *du = device_view(u), *dxi = xi ? device_view(xi) : nullptr;
    if (!drho || !du || (xi && !dxi))
        return fail(ctx, LBM_ERR_ARG, std::string(name) + ": a field is neither device memory nor pinned host memory");
    LBM_CUDA(launch_init<T>(ctx->storage, ctx->L, ctx->f[ctx->cur], drho, du, dxi, amp, ctx->stream), name);
    ctx->initialised = true;
    ctx->interior_pending = false;
    return LBM_OK;
}

extern "C" {

lbm_status lbm_init_state(lbm_ctx *ctx, const double *rho, const double *u, const double *xi, double amp)
{
    return init_state<double>(ctx, rho, u, xi, amp, "lbm_init_state");
}

lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const double *rho, const double *u)
{
    return init_state<double>(ctx, rho, u, nullptr, 0.0, "lbm_init_equilibrium");
}

lbm_status lbm_init_state_f32(lbm_ctx *ctx, const float *rho, const float *u, const float *xi, double amp)
{
    return init_state<float>(ctx, rho, u, xi, amp, "lbm_init_state_f32");
}

lbm_status lbm_set_geometry(lbm_ctx *ctx, const lbm_geometry *g)
{
    NvtxRange nvtx_("lbm_set_geometry");
    if (!ctx) return LBM_ERR_ARG;
    if (!g) return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: null geometry");
    if (g->kind < LBM_BODY_NONE || g->kind > LBM_BODY_MESH)
        return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: unknown body kind");
    const Lattice &L = ctx->L;
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "sync");
    LBM_CUDA(drain_records(ctx), "record copies");
    free_scratch(ctx, true);
    // until the new body is in place the context has none and no node is
    // marked, so a call that fails below leaves a consistent bodiless context
    ctx->has_body = false;
    LBM_CUDA(cudaMemsetAsync(ctx->flags, 0, (size_t)L.N, ctx->stream), "flags clear");
    const bool body = g->kind != LBM_BODY_NONE;
    GeomParams &G = ctx->G;
    G = GeomParams{};
    ctx->order = ctx->order_request;
    ctx->trial = 0;
    G.kind = g->kind;
    G.free_motion = g->free_motion;
    G.zoff = ctx->slab_zoff;
    G.zper = ctx->slab_zper;
    G.own_lo = ctx->slab_zper > 0 ? ctx->slab_own_lo : 0;
    G.own_hi = ctx->slab_zper > 0 ? ctx->slab_own_hi : L.nz;
    if (ctx->slab_zper > 0 && g->kind == LBM_BODY_SPHERE && !(g->X[2] >= 0.0 && g->X[2] < (double)ctx->slab_zper))
        return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: sphere centre outside [0, zper) of the slab's whole box");
    G.R = g->R;
    G.y_lo = g->y_lo;
    G.y_hi = g->y_hi;
    for (int a = 0; a < 3; ++a) {
        G.U_lo[a] = g->U_lo[a];
        G.U_hi[a] = g->U_hi[a];
        G.g[a] = g->g[a];
        // (a slab's z is cut at its layers whatever its faces)
        G.periodic[a] = L.face[2 * a] == LBM_FACE_PERIODIC && !(a == 2 && ctx->slab_zper > 0);
    }
    // Sec. 4.1: a sphere given no mass takes m_s = rho_s pi D^3 / 6 with
    // rho_s = rho_ratio rho0 (the analytic volume, not the voxel count)
    double mass = g->mass;
    if (g->kind == LBM_BODY_SPHERE && !(mass > 0.0) && g->R > 0.0 && g->rho_ratio > 0.0) {
        const double D = 2.0 * g->R;
        mass = g->rho_ratio * L.rho0 * M_PI * D * D * D / 6.0;
    }
    G.inv_mass = mass > 0.0 ? 1.0 / mass : 0.0;
    G.buoy = g->rho_ratio > 0.0 ? 1.0 - 1.0 / g->rho_ratio : 0.0;
    const int n[3] = {L.nx, L.ny, L.nz};
    if (g->kind == LBM_BODY_SPHERE) {
        if (!(g->R > 0.0) || (g->free_motion && (!(mass > 0.0) || !(g->rho_ratio > 0.0))))
            return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: sphere needs R > 0 (and mass, rho_ratio > 0 when free)");
        for (int a = 0; a < 3; ++a) {
            const int c = (int)std::ceil(2.0 * g->R) + 9;
            G.cap[a] = c < n[a] ? c : n[a];
            if (G.periodic[a] && !(g->X[a] >= 0.0 && g->X[a] < (double)n[a]))
                return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: centre outside [0, n) on a periodic axis");
        }
    } else if (g->kind == LBM_BODY_AIRFOIL) {
        if (!(g->chord > 0.0) || !(fabs(g->ca * g->ca + g->sa * g->sa - 1.0) < 1e-12))
            return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: airfoil needs chord > 0 and ca^2 + sa^2 = 1");
        G.chord = g->chord; G.ca = g->ca; G.sa = g->sa;
        G.h_amp = g->h_amp; G.h_omega = g->h_omega;
        G.camber_m = g->camber_m; G.camber_p = g->camber_p;
        G.inv_chord = 1.0 / g->chord;
        G.camber_k1 = g->camber_p > 0.0 ? g->camber_m / (g->camber_p * g->camber_p) : 0.0;
        G.camber_k2 = g->camber_p < 1.0 ? g->camber_m / ((1.0 - g->camber_p) * (1.0 - g->camber_p)) : 0.0;
        for (int k = 0; k < 5; ++k) G.thick[k] = g->thick[k];
        G.y_base = g->X[1];
        // profile box in the lattice frame (relative to the leading edge) from a
        // dense sample of the outline, widened by one node
        double bx0 = 0, bx1 = 0, by0 = 0, by1 = 0;
        for (int k = 0; k <= 4096; ++k) {
            const double xi = k / 4096.0;
            const double yc = xi < g->camber_p
                                  ? g->camber_m / (g->camber_p * g->camber_p) * (2 * g->camber_p * xi - xi * xi)
                                  : g->camber_m / ((1 - g->camber_p) * (1 - g->camber_p)) *
                                        ((1 - 2 * g->camber_p) + 2 * g->camber_p * xi - xi * xi);
            const double t = g->thick[0] * std::sqrt(xi) +
                             xi * (g->thick[1] + xi * (g->thick[2] + xi * (g->thick[3] + xi * g->thick[4])));
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                const double eta = yc + sgn * t;
                const double dx = g->chord * (xi * g->ca + eta * g->sa);
                const double dy = g->chord * (-xi * g->sa + eta * g->ca);
                bx0 = std::min(bx0, dx); bx1 = std::max(bx1, dx);
                by0 = std::min(by0, dy); by1 = std::max(by1, dy);
            }
        }
        G.box[0] = bx0 - 1; G.box[1] = bx1 + 1; G.box[2] = by0 - 1; G.box[3] = by1 + 1;
        // band extent per axis: the profile box plus one step of plunge
        const double span[2] = {G.box[1] - G.box[0], G.box[3] - G.box[2] + 1.0};
        for (int a = 0; a < 2; ++a) {
            const int c = (int)std::ceil(span[a]) + 9;
            G.cap[a] = c < n[a] ? c : n[a];
        }
        G.cap[2] = n[2];
    } else if (g->kind == LBM_BODY_MESH) {
        const int nv = g->n_vertices, nt = g->n_triangles;
        if (!g->mesh_rest || !g->mesh_tris || nv < 4 || nt < 4 || nv > (1 << 24) || nt > (1 << 24) ||
            !(g->length > 0.0) || g->wave_length == 0.0 || g->wave_period == 0.0 || g->reserved_mesh != 0 ||
            (g->free_motion && !(g->mass > 0.0)) || g->free_motion < 0 || g->free_motion > 7 ||
            !std::isfinite(g->psi) || !std::isfinite(g->omega))
            return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: mesh needs vertices, triangles, length > 0, "
                                          "non-zero wavelength and period, free_motion in 0..7 (and mass > 0 "
                                          "when free), finite psi and omega");
        for (long long k = 0; k < 3LL * nt; ++k)
            if (g->mesh_tris[k] < 0 || g->mesh_tris[k] >= nv)
                return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: mesh triangle index out of range");
        double ext[6] = {INFINITY, -INFINITY, INFINITY, -INFINITY, INFINITY, -INFINITY};
        for (int v = 0; v < nv; ++v)
            for (int a = 0; a < 3; ++a) {
                const double r = g->mesh_rest[3 * v + a];
                if (!std::isfinite(r) || (a == 0 && r < 0.0))
                    return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: mesh rest data not finite (or s < 0)");
                ext[2 * a] = std::min(ext[2 * a], r);
                ext[2 * a + 1] = std::max(ext[2 * a + 1], r);
            }
        // lateral reach of the midline: its envelope at the largest arc position
        const double env = std::fabs(g->wave_amp) * g->length * (ext[1] / g->length + 0.03125) / 1.03125;
        ext[2] -= env;
        ext[3] += env;
        G.n_vertices = nv;
        G.n_triangles = nt;
        G.length = g->length;
        G.wave_amp = g->wave_amp;
        G.wave_length = g->wave_length;
        G.wave_period = g->wave_period;
        G.wave_ramp = g->wave_ramp ? 1 : 0;
        G.com_frame = (g->free_motion & 6) != 0;
        G.mass = g->mass;
        double span[3];
        for (int a = 0; a < 3; ++a) span[a] = ext[2 * a + 1] - ext[2 * a];
        if (G.com_frame) {
            // the body turns about its centre of mass: x and y reach at most
            // r_max from it.  The midline only shears along y, so the body
            // frame x of the centre of mass is that of the rest mesh; its y
            // lies within the envelope.
            double V = 0.0, Sx = 0.0;
            for (int k = 0; k < nt; ++k) {
                const int *tr = g->mesh_tris + 3 * k;
                const double *p0 = g->mesh_rest + 3 * tr[0], *p1 = g->mesh_rest + 3 * tr[1],
                             *p2 = g->mesh_rest + 3 * tr[2];
                const double d = (p1[1] - p0[1]) * (p2[2] - p0[2]) - (p1[2] - p0[2]) * (p2[1] - p0[1]);
                V += d * (p0[0] + p1[0] + p2[0]) / 6.0;
                Sx += d * (p0[0] * p0[0] + p1[0] * p1[0] + p2[0] * p2[0] + p0[0] * p1[0] + p0[0] * p2[0] +
                           p1[0] * p2[0]) / 24.0;
            }
            if (!(V > 0.0))
                return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: mesh volume not positive (triangles must be "
                                              "oriented outwards)");
            const double sc = Sx / V;
            double rmax = 0.0;
            for (int v = 0; v < nv; ++v) {
                const double *r = g->mesh_rest + 3 * v;
                rmax = std::max(rmax, std::hypot(r[0] - sc, std::fabs(r[1]) + 2.0 * env));
            }
            span[0] = span[1] = 2.0 * rmax + 3.0;
        }
        for (int a = 0; a < 3; ++a) {
            G.mesh_ext[2 * a] = ext[2 * a];
            G.mesh_ext[2 * a + 1] = ext[2 * a + 1];
            const int c = (int)std::ceil(span[a]) + 9;
            G.cap[a] = c < n[a] ? c : n[a];
            G.cells[a] = (G.cap[a] + MESH_CELL - 1) / MESH_CELL + 1;
        }
    } else {
        for (int a = 0; a < 3; ++a) G.cap[a] = n[a];
    }
    if (ctx->slab_zper > 0 && (g->kind == LBM_BODY_SPHERE || g->kind == LBM_BODY_MESH)) {
        // a slab marks and sweeps the image of the body nearest its middle
        // layer; any other image (zper away) must miss the layers whose marks
        // own nodes read, [own_lo - 1, own_hi], wherever the body is: half
        // the period less half the body's z extent beyond the farthest of
        // them from the middle
        const double ext = g->kind == LBM_BODY_SPHERE ? 2.0 * G.R : G.mesh_ext[5] - G.mesh_ext[4];
        const double mid = 0.5 * (double)L.nz;
        const double m = std::max(mid - (double)(ctx->slab_own_lo - 1), (double)ctx->slab_own_hi - mid);
        if (!(0.5 * ((double)ctx->slab_zper - ext) > m))
            return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: body too long in z for the slab (its z extent "
                                          "and the slab's layers reach the next image along z)");
    }
    const long long vol = (long long)G.cap[0] * G.cap[1] * G.cap[2];
    if (vol >= (1LL << 31) / 6) return fail(ctx, LBM_ERR_ARG, "lbm_set_geometry: body band too large");
    G.cap_boundary = (int)vol;
    G.cap_uncovered = (int)vol;
    Scratch &S = ctx->S;
    S.n_partials = 64;
    bool ok = true;
    if (body) {
        ok = ctx_alloc(ctx, &S.blist, vol) == cudaSuccess && ctx_alloc(ctx, &S.bpos, vol) == cudaSuccess &&
             ctx_alloc(ctx, &S.ulist, vol) == cudaSuccess && ctx_alloc(ctx, &S.upos, vol) == cudaSuccess &&
             ctx_alloc(ctx, &S.bforce, vol * 6) == cudaSuccess &&
             ctx_alloc(ctx, &S.partials, (size_t)S.n_partials * 6) == cudaSuccess && ctx_alloc(ctx, &S.ticket, 1) == cudaSuccess;
        if (ok) ok = cudaMemsetAsync(S.ticket, 0, sizeof(unsigned), ctx->stream) == cudaSuccess;
    }
    if (ok && g->kind == LBM_BODY_MESH) {
        const size_t nv = (size_t)G.n_vertices, nt = (size_t)G.n_triangles;
        const size_t ncols = (size_t)G.cap[1] * G.cap[2];
        const size_t ncells = (size_t)G.cells[0] * G.cells[1] * G.cells[2];
        ok = ctx_alloc(ctx, &S.mesh_rest, 3 * nv) == cudaSuccess && ctx_alloc(ctx, &S.mesh_pos, 3 * nv) == cudaSuccess &&
             ctx_alloc(ctx, &S.mesh_vel, 3 * nv) == cudaSuccess && ctx_alloc(ctx, &S.mesh_tris, 3 * nt) == cudaSuccess &&
             ctx_alloc(ctx, &S.tri_box, 6 * nt) == cudaSuccess && ctx_alloc(ctx, &S.col_count, ncols) == cudaSuccess &&
             ctx_alloc(ctx, &S.col_x, ncols * MESH_COL_CAP) == cudaSuccess && ctx_alloc(ctx, &S.cell_count, ncells) == cudaSuccess &&
             ctx_alloc(ctx, &S.cell_tri, ncells * MESH_CELL_CAP) == cudaSuccess && ctx_alloc(ctx, &S.mesh_status, 1) == cudaSuccess &&
             ctx_alloc(ctx, &S.mesh_ipos, 3 * nv) == cudaSuccess && ctx_alloc(ctx, &S.mesh_frac, 3 * nv) == cudaSuccess &&
             ctx_alloc(ctx, &S.mesh_partials, (nt + MESH_THREADS - 1) / MESH_THREADS * 11) == cudaSuccess &&
             ctx_alloc(ctx, &S.mesh_ticket, 1) == cudaSuccess;
        if (ok) ok = cudaMemsetAsync(S.mesh_ticket, 0, sizeof(unsigned), ctx->stream) == cudaSuccess;
        if (ok)
            ok = cudaMemcpy(S.mesh_rest, g->mesh_rest, 3 * nv * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
                 cudaMemcpy(S.mesh_tris, g->mesh_tris, 3 * nt * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
        G.mesh_rest = S.mesh_rest;
        G.mesh_tris = S.mesh_tris;
        G.mesh_pos = S.mesh_pos;
        G.mesh_vel = S.mesh_vel;
        G.tri_box = S.tri_box;
        G.col_count = S.col_count;
        G.col_x = S.col_x;
        G.cell_count = S.cell_count;
        G.cell_tri = S.cell_tri;
        G.mesh_status = S.mesh_status;
        G.mesh_ipos = S.mesh_ipos;
        G.mesh_frac = S.mesh_frac;
        G.mesh_partials = S.mesh_partials;
        G.mesh_ticket = S.mesh_ticket;
    }
    if (!ok) {
        free_scratch(ctx, true);
        return fail(ctx, LBM_ERR_OOM, "lbm_set_geometry: device allocation failed");
    }
    DevBody hb[2] = {};
    for (int a = 0; a < 3; ++a) { hb[0].X[a] = g->X[a]; hb[0].U[a] = g->U[a]; }
    if (g->kind == LBM_BODY_AIRFOIL) {
        hb[0].t = g->t0;
        hb[0].X[1] = g->X[1] + g->h_amp * std::sin(g->h_omega * g->t0);
        hb[0].U[0] = 0.0;
        hb[0].U[1] = g->h_amp * g->h_omega * std::cos(g->h_omega * g->t0);
        hb[0].U[2] = 0.0;
    }
    if (g->kind == LBM_BODY_MESH) {
        hb[0].t = g->t0;
        hb[0].psi = g->psi;
        hb[0].omega = g->omega;
    }
    ctx->bcur = 0;
    LBM_CUDA(cudaMemcpyAsync(S.body, hb, sizeof(hb), cudaMemcpyHostToDevice, ctx->stream), "body upload");
    if (g->kind == LBM_BODY_MESH) {
        LBM_CUDA(launch_mesh_mark_initial(L, G, S, 0, ctx->flags, ctx->stream), "initial marks");
        LBM_CUDA(launch_sweep_init(L, G, S, 0, ctx->stream), "sweep box");
        int mst = 0;
        LBM_CUDA(cudaMemcpyAsync(&mst, S.mesh_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "mesh status");
        LBM_CUDA(cudaStreamSynchronize(ctx->stream), "set_geometry");
        if (mst) {
            free_scratch(ctx, true);
            // no body: no node stays marked
            LBM_CUDA(cudaMemsetAsync(ctx->flags, 0, (size_t)L.N, ctx->stream), "flags clear");
            LBM_CUDA(cudaStreamSynchronize(ctx->stream), "set_geometry");
            return fail(ctx, LBM_ERR_ARG, (mst & 2) ? "lbm_set_geometry: mesh closer than two nodes to a box face"
                                                    : "lbm_set_geometry: mesh column or cell list overflow");
        }
        ctx->has_body = true;
        return LBM_OK;
    }
    if (body) {
        LBM_CUDA(launch_mark_initial(L, G, hb[0].X, ctx->flags, ctx->stream), "initial marks");
        LBM_CUDA(launch_sweep_init(L, G, S, 0, ctx->stream), "sweep box");
    }
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "set_geometry");
    ctx->has_body = body;
    return LBM_OK;
}

static cudaError_t prof_mark(lbm_ctx *ctx, int which) { return ctx_prof_mark(ctx, which); }

}  // extern "C"

cudaError_t ctx_prof_mark(lbm_ctx *ctx, int which)
{
    if (!ctx->prof_open) return cudaSuccess;
    const int k = 2 * ctx->prof_used + which;
    if (k >= (int)ctx->prof.size()) return cudaSuccess;
    cudaError_t e = cudaEventRecord(ctx->prof[k], ctx->stream);
    if (which == 1) ctx->prof_used++;
    return e;
}

extern "C" {

// Geometry and refill first, then the boundary nodes and the force on the
// side stream beside one bulk launch over all nodes (flags read when there is
// a body).
static cudaError_t sequential_step(lbm_ctx *ctx, void *fa, void *fb, int &cur, int *&status, int *launches_out)
{
    int &launches = *launches_out;
    const uint8_t *fl = ctx->has_body ? ctx->flags : nullptr;
    cudaError_t e;
    if (ctx->has_body) {
        const int prev = ctx->bcur;
        cur = prev ^ 1;
        status = &ctx->S.body[cur].status;
        if ((e = launch_geometry(ctx->L, ctx->G, ctx->S, prev, ctx->flags, ctx->stream, &launches)) != cudaSuccess ||
            (e = launch_refill(ctx->storage, ctx->L, ctx->G, ctx->S, cur, fa, ctx->flags, ctx->stream)) != cudaSuccess)
            return e;
        launches += 1;
        // the boundary nodes and the force reduction run on a side stream
        // beside the bulk kernel (they write disjoint nodes)
        if ((e = cudaEventRecord(ctx->ev_fork, ctx->stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0)) != cudaSuccess ||
            (e = launch_boundary(ctx->storage, ctx->L, ctx->G, ctx->S, cur, fa, fb, ctx->flags, ctx->side)) !=
                cudaSuccess ||
            (e = launch_forces(ctx->G, ctx->S, cur, ctx->side, &launches)) != cudaSuccess ||
            (e = cudaEventRecord(ctx->ev_join, ctx->side)) != cudaSuccess)
            return e;
        launches += 1;
    }
    if ((e = prof_mark(ctx, 0)) != cudaSuccess ||
        (e = launch_bulk(ctx->storage, ctx->L, fa, fb, fl, status, ctx->stream)) != cudaSuccess ||
        (e = prof_mark(ctx, 1)) != cudaSuccess)
        return e;
    if (ctx->has_body && (e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0)) != cudaSuccess) return e;
    launches += 1;
    return cudaSuccess;
}

}  // extern "C"

cudaError_t ctx_step_flagged(lbm_ctx *ctx, int *launches)
{
    void *fa = ctx->f[ctx->cur], *fb = ctx->f[ctx->cur ^ 1];
    int *status = &ctx->S.body[ctx->bcur].status;
    int cur = ctx->bcur;
    cudaError_t e;
    if (ctx->has_body && ctx->slot_pending[ctx->bcur ^ 1]) {
        if ((e = cudaStreamWaitEvent(ctx->stream, ctx->ev_slot[ctx->bcur ^ 1], 0)) != cudaSuccess) return e;
        ctx->slot_pending[ctx->bcur ^ 1] = false;
    }
    ctx->last_split = false;
    if ((e = sequential_step(ctx, fa, fb, cur, status, launches)) != cudaSuccess) return e;
    ctx->bcur = cur;
    ctx->cur ^= 1;
    return cudaSuccess;
}

extern "C" {

// Chooses the launch order once the trial steps have run: the order whose
// two timed steps took less (the first pair of trial steps only warms up).
static void choose_order(lbm_ctx *ctx)
{
    if (ctx->order != ORDER_UNDECIDED || ctx->trial < TRIAL_STEPS) return;
    if (cudaEventQuery(ctx->ev_trial[4]) != cudaSuccess) {
        cudaGetLastError();  // not reached yet: keep the split order meanwhile
        return;
    }
    float t[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; ++k)
        if (cudaEventElapsedTime(&t[k], ctx->ev_trial[k], ctx->ev_trial[k + 1]) != cudaSuccess) {
            cudaGetLastError();
            ctx->order = ORDER_SPLIT;
            return;
        }
    ctx->order = (t[0] + t[2] <= t[1] + t[3]) ? ORDER_SPLIT : ORDER_SEQUENTIAL;
}

lbm_status lbm_step(lbm_ctx *ctx, int nsteps)
{
    NvtxRange nvtx_("lbm_step");
    if (!ctx) return LBM_ERR_ARG;
    if (nsteps < 0) return fail(ctx, LBM_ERR_ARG, "lbm_step: nsteps < 0");
    if (!ctx->initialised) return fail(ctx, LBM_ERR_STATE, "lbm_step: state not initialised");
    if (ctx->interior_pending) return fail(ctx, LBM_ERR_STATE, "lbm_step: a step begun by lbm_step_interior is open");
    int launches = 0;
    choose_order(ctx);
    for (int s = 0; s < nsteps; ++s) {
        void *fa = ctx->f[ctx->cur], *fb = ctx->f[ctx->cur ^ 1];
        int *status = &ctx->S.body[ctx->bcur].status;
        int cur = ctx->bcur;
        // a step writes the body slot other than the current one: it waits
        // for a pending record copy out of that slot
        if (ctx->has_body && ctx->slot_pending[ctx->bcur ^ 1]) {
            LBM_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_slot[ctx->bcur ^ 1], 0), "record wait");
            ctx->slot_pending[ctx->bcur ^ 1] = false;
        }
        // the band of this step is known from the previous state: split, the
        // nodes outside it run on the caller's stream at once and the body's
        // geometry, refill, boundary nodes, force and the band's bulk nodes on
        // the side stream beside them; sequential, the geometry and refill run
        // first and the boundary nodes beside one flag-aware bulk launch.  The
        // results are the same; the trial steps time both.
        const bool ahead = ctx->has_body && sweep_ahead(ctx->G);
        bool split = ahead && ctx->order != ORDER_SEQUENTIAL;
        const bool trial = ahead && ctx->order == ORDER_UNDECIDED && ctx->trial < TRIAL_STEPS;
        if (trial) {
            split = ctx->trial % 2 == 0;
            if (ctx->trial >= 2) LBM_CUDA(cudaEventRecord(ctx->ev_trial[ctx->trial - 2], ctx->stream), "trial");
        }
        ctx->last_split = split;
        if (split) {
            const int prev = ctx->bcur;
            cur = prev ^ 1;
            status = &ctx->S.body[cur].status;
            const int *sweep = ctx->S.body[prev].sweep;
            LBM_CUDA(cudaEventRecord(ctx->ev_fork, ctx->stream), "fork");
            LBM_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0), "fork wait");
            LBM_CUDA(launch_geometry(ctx->L, ctx->G, ctx->S, prev, ctx->flags, ctx->side, &launches), "geometry");
            LBM_CUDA(launch_refill(ctx->storage, ctx->L, ctx->G, ctx->S, cur, fa, ctx->flags, ctx->side), "refill");
            LBM_CUDA(launch_boundary(ctx->storage, ctx->L, ctx->G, ctx->S, cur, fa, fb, ctx->flags, ctx->side), "boundary");
            LBM_CUDA(launch_forces(ctx->G, ctx->S, cur, ctx->side, &launches), "forces");
            LBM_CUDA(launch_bulk(ctx->storage, ctx->L, fa, fb, ctx->flags, status, ctx->side, BULK_BAND, sweep,
                                 ctx->G.cap), "bulk band");
            LBM_CUDA(cudaEventRecord(ctx->ev_join, ctx->side), "join");
            LBM_CUDA(prof_mark(ctx, 0), "profile event");
            LBM_CUDA(launch_bulk(ctx->storage, ctx->L, fa, fb, nullptr, status, ctx->stream, BULK_OUTSIDE, sweep),
                     "bulk outside");
            LBM_CUDA(prof_mark(ctx, 1), "profile event");
            LBM_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0), "join wait");
            launches += 4;
        } else {
            LBM_CUDA(sequential_step(ctx, fa, fb, cur, status, &launches), "step");
        }
        if (trial && ++ctx->trial == TRIAL_STEPS) LBM_CUDA(cudaEventRecord(ctx->ev_trial[4], ctx->stream), "trial");
        ctx->bcur = cur;
        ctx->cur ^= 1;
    }
    ctx->launches = launches;
    return LBM_OK;
}


// Two-phase step of a slab: the own layers that pull from no halo layer
// first, the rest once the caller has refilled the halo layers.
static void interior_range(const lbm_ctx *ctx, int &lo, int &hi)
{
    lo = ctx->slab_own_lo + 1;
    hi = ctx->slab_own_hi - 1;
    if (hi <= lo) lo = hi = ctx->slab_own_lo;  // too thin: all own layers are edges
}

lbm_status lbm_step_interior(lbm_ctx *ctx)
{
    NvtxRange nvtx_("lbm_step_interior");
    if (!ctx) return LBM_ERR_ARG;
    if (!ctx->initialised) return fail(ctx, LBM_ERR_STATE, "lbm_step_interior: state not initialised");
    if (ctx->slab_zper <= 0) return fail(ctx, LBM_ERR_STATE, "lbm_step_interior: not a slab (lbm_set_slab)");
    if (ctx->interior_pending)
        return fail(ctx, LBM_ERR_STATE, "lbm_step_interior: the previous step's edges are still to run");
    ctx->launches = 0;
    // only where the band is known ahead and the split order is asked for;
    // otherwise lbm_step_edges runs the whole step
    if (ctx->has_body && (!sweep_ahead(ctx->G) || ctx->order != ORDER_SPLIT)) return LBM_OK;
    void *fa = ctx->f[ctx->cur], *fb = ctx->f[ctx->cur ^ 1];
    const int next = ctx->bcur ^ 1;
    if (ctx->has_body && ctx->slot_pending[next]) {
        LBM_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_slot[next], 0), "record wait");
        ctx->slot_pending[next] = false;
    }
    int *status = ctx->has_body ? &ctx->S.body[next].status : &ctx->S.body[ctx->bcur].status;
    const int *sweep = ctx->has_body ? ctx->S.body[ctx->bcur].sweep : nullptr;
    int lo, hi;
    interior_range(ctx, lo, hi);
    LBM_CUDA(prof_mark(ctx, 0), "profile event");
    LBM_CUDA(launch_bulk(ctx->storage, ctx->L, fa, fb, nullptr, status, ctx->stream,
                         ctx->has_body ? BULK_OUTSIDE : BULK_ALL, sweep, nullptr, lo, hi - lo),
             "bulk interior");
    LBM_CUDA(prof_mark(ctx, 1), "profile event");
    ctx->launches = hi > lo ? 1 : 0;
    ctx->interior_pending = true;
    return LBM_OK;
}

lbm_status lbm_step_edges(lbm_ctx *ctx)
{
    NvtxRange nvtx_("lbm_step_edges");
    if (!ctx) return LBM_ERR_ARG;
    if (!ctx->interior_pending) {
        if (ctx->slab_zper <= 0) return fail(ctx, LBM_ERR_STATE, "lbm_step_edges: not a slab (lbm_set_slab)");
        return lbm_step(ctx, 1);
    }
    ctx->interior_pending = false;
    int launches = ctx->launches;
    void *fa = ctx->f[ctx->cur], *fb = ctx->f[ctx->cur ^ 1];
    int cur = ctx->bcur;
    int *status = &ctx->S.body[cur].status;
    const int *sweep = nullptr;
    if (ctx->has_body) {
        // the body's chain as in the split order of lbm_step
        const int prev = ctx->bcur;
        cur = prev ^ 1;
        status = &ctx->S.body[cur].status;
        sweep = ctx->S.body[prev].sweep;
        LBM_CUDA(cudaEventRecord(ctx->ev_fork, ctx->stream), "fork");
        LBM_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0), "fork wait");
        LBM_CUDA(launch_geometry(ctx->L, ctx->G, ctx->S, prev, ctx->flags, ctx->side, &launches), "geometry");
        LBM_CUDA(launch_refill(ctx->storage, ctx->L, ctx->G, ctx->S, cur, fa, ctx->flags, ctx->side), "refill");
        LBM_CUDA(launch_boundary(ctx->storage, ctx->L, ctx->G, ctx->S, cur, fa, fb, ctx->flags, ctx->side), "boundary");
        LBM_CUDA(launch_forces(ctx->G, ctx->S, cur, ctx->side, &launches), "forces");
        LBM_CUDA(launch_bulk(ctx->storage, ctx->L, fa, fb, ctx->flags, status, ctx->side, BULK_BAND, sweep,
                             ctx->G.cap), "bulk band");
        LBM_CUDA(cudaEventRecord(ctx->ev_join, ctx->side), "join");
        launches += 3;
    }
    int lo, hi;
    interior_range(ctx, lo, hi);
    const int mode = ctx->has_body ? BULK_OUTSIDE : BULK_ALL;
    LBM_CUDA(launch_bulk(ctx->storage, ctx->L, fa, fb, nullptr, status, ctx->stream, mode, sweep, nullptr,
                         ctx->slab_own_lo, lo - ctx->slab_own_lo), "bulk edge");
    LBM_CUDA(launch_bulk(ctx->storage, ctx->L, fa, fb, nullptr, status, ctx->stream, mode, sweep, nullptr,
                         hi, ctx->slab_own_hi - hi), "bulk edge");
    launches += (lo > ctx->slab_own_lo) + (ctx->slab_own_hi > hi);
    if (ctx->has_body) LBM_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0), "join wait");
    ctx->last_split = ctx->has_body;
    ctx->bcur = cur;
    ctx->cur ^= 1;
    ctx->launches = launches;
    return LBM_OK;
}

int lbm_current_buffer(const lbm_ctx *ctx) { return ctx ? ctx->cur : -1; }

lbm_status lbm_set_launch_order(lbm_ctx *ctx, int order)
{
    if (!ctx) return LBM_ERR_ARG;
    if (order != LBM_ORDER_AUTO && order != LBM_ORDER_SPLIT && order != LBM_ORDER_SEQUENTIAL)
        return fail(ctx, LBM_ERR_ARG, "lbm_set_launch_order: unknown order");
    ctx->order_request = order;
    ctx->order = order;
    ctx->trial = 0;
    return LBM_OK;
}

int lbm_launch_order(const lbm_ctx *ctx) { return ctx ? ctx->order : -1; }

int64_t lbm_kernel_launches(const lbm_ctx *ctx) { return ctx ? ctx->launches : -1; }

static lbm_status ensure_plane(lbm_ctx *ctx)
{
    if (ctx->plane) return LBM_OK;
    if (ctx_alloc(ctx, &ctx->plane, (size_t)ctx->L.N) != cudaSuccess)
        return fail(ctx, LBM_ERR_OOM, "plane buffer allocation failed");
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx *ctx, double *host_f)
{
    NvtxRange nvtx_("lbm_get_populations");
    if (!ctx) return LBM_ERR_ARG;
    if (!host_f) return fail(ctx, LBM_ERR_ARG, "lbm_get_populations: null output");
    lbm_status st = ensure_plane(ctx);
    if (st != LBM_OK) return st;
    const size_t N = (size_t)ctx->L.N;
    for (int i = 0; i < Q; ++i) {
        LBM_CUDA(launch_decode_plane(ctx->storage, ctx->L, ctx->f[ctx->cur], i, ctx->plane, ctx->stream), "decode");
        LBM_CUDA(cudaMemcpyAsync(host_f + (size_t)i * N, ctx->plane, N * sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->stream), "copy out");
        LBM_CUDA(cudaStreamSynchronize(ctx->stream), "sync");
    }
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx *ctx, const double *host_f)
{
    if (!ctx) return LBM_ERR_ARG;
    if (!host_f) return fail(ctx, LBM_ERR_ARG, "lbm_set_populations: null input");
    lbm_status st = ensure_plane(ctx);
    if (st != LBM_OK) return st;
    const size_t N = (size_t)ctx->L.N;
    for (int i = 0; i < Q; ++i) {
        LBM_CUDA(cudaMemcpyAsync(ctx->plane, host_f + (size_t)i * N, N * sizeof(double),
                                 cudaMemcpyHostToDevice, ctx->stream), "copy in");
        LBM_CUDA(launch_encode_plane(ctx->storage, ctx->L, ctx->f[ctx->cur], i, ctx->plane, ctx->stream), "encode");
        LBM_CUDA(cudaStreamSynchronize(ctx->stream), "sync");
    }
    ctx->initialised = true;
    ctx->interior_pending = false;
    return LBM_OK;
}

lbm_status lbm_get_body(lbm_ctx *ctx, lbm_body_state *out)
{
    if (!ctx) return LBM_ERR_ARG;
    if (!out) return fail(ctx, LBM_ERR_ARG, "lbm_get_body: null output");
    DevBody hb;
    LBM_CUDA(cudaMemcpyAsync(&hb, ctx->S.body + ctx->bcur, sizeof(hb), cudaMemcpyDeviceToHost, ctx->stream),
             "body read");
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "sync");
    for (int a = 0; a < 3; ++a) {
        out->X[a] = hb.X[a]; out->U[a] = hb.U[a];
        out->F[a] = hb.F[a]; out->M[a] = hb.M[a];
        out->F_sum[a] = hb.F_sum[a]; out->M_sum[a] = hb.M_sum[a];
    }
    out->n_sum = hb.n_sum;
    out->n_boundary = hb.n_boundary;
    out->n_uncovered = hb.n_uncovered;
    out->n_links = hb.n_links;
    out->status = hb.status;
    out->n_band = ctx->has_body && ctx->last_split ? hb.band_n[0] * hb.band_n[1] * hb.band_n[2] : 0;
    out->t = hb.t;
    out->psi = hb.psi;
    out->omega = hb.omega;
    out->Izz = hb.Izz;
    return LBM_OK;
}

lbm_status lbm_body_forces(lbm_ctx *ctx, double F[3], double M[3], int averaged)
{
    if (!ctx) return LBM_ERR_ARG;
    if (!F || !M) return fail(ctx, LBM_ERR_ARG, "lbm_body_forces: null output");
    lbm_body_state b;
    lbm_status st = lbm_get_body(ctx, &b);
    if (st != LBM_OK) return st;
    for (int a = 0; a < 3; ++a) {
        if (averaged) {
            const double n = b.n_sum > 0 ? (double)b.n_sum : 1.0;
            F[a] = b.F_sum[a] / n;
            M[a] = b.M_sum[a] / n;
        } else {
            F[a] = b.F[a];
            M[a] = b.M[a];
        }
    }
    if (b.status & ST_UNSTABLE) return fail(ctx, LBM_ERR_UNSTABLE, "a node had non-finite or non-positive density");
    if (b.status & ST_BAND_OVERFLOW) return fail(ctx, LBM_ERR_STATE, "body band or boundary list overflowed its capacity");
    return LBM_OK;
}

lbm_status lbm_body_forces_async(lbm_ctx *ctx, lbm_force_record *out, int64_t *ticket)
{
    if (!ctx) return LBM_ERR_ARG;
    if (!out || !ticket) return fail(ctx, LBM_ERR_ARG, "lbm_body_forces_async: null argument");
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, out) != cudaSuccess || attr.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return fail(ctx, LBM_ERR_ARG, "lbm_body_forces_async: the record must be page-locked host memory");
    }
    if (!ctx->copy) {
        bool ok = cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&ctx->ev_step, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < LBM_RECORD_DEPTH; ++k)
            ok = cudaEventCreateWithFlags(&ctx->ev_copy[k], cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < 2; ++k)
            ok = cudaEventCreateWithFlags(&ctx->ev_slot[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) return fail(ctx, LBM_ERR_CUDA, "lbm_body_forces_async: stream or event creation failed");
    }
    const int slot = ctx->bcur;
    const DevBody *src = ctx->S.body + slot;
    const int k = (int)(ctx->next_ticket % LBM_RECORD_DEPTH);
    LBM_CUDA(cudaEventRecord(ctx->ev_step, ctx->stream), "record step");
    LBM_CUDA(cudaStreamWaitEvent(ctx->copy, ctx->ev_step, 0), "record wait");
    // F and M are adjacent in both structures
    LBM_CUDA(cudaMemcpyAsync(out->F, src->F, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->copy), "record F, M");
    LBM_CUDA(cudaMemcpyAsync(&out->t, &src->t, sizeof(double), cudaMemcpyDeviceToHost, ctx->copy), "record t");
    LBM_CUDA(cudaMemcpyAsync(&out->status, &src->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->copy),
             "record status");
    LBM_CUDA(cudaEventRecord(ctx->ev_copy[k], ctx->copy), "record done");
    LBM_CUDA(cudaEventRecord(ctx->ev_slot[slot], ctx->copy), "slot done");
    ctx->slot_pending[slot] = true;
    ctx->rec[k] = out;
    *ticket = ctx->next_ticket++;
    return LBM_OK;
}

lbm_status lbm_body_forces_wait(lbm_ctx *ctx, int64_t ticket)
{
    if (!ctx) return LBM_ERR_ARG;
    if (ticket < 0 || ticket >= ctx->next_ticket)
        return fail(ctx, LBM_ERR_ARG, "lbm_body_forces_wait: ticket not issued");
    // an older ticket's ring entry was recorded again by a later copy, which
    // lands after it
    const int k = (int)(ticket % LBM_RECORD_DEPTH);
    LBM_CUDA(cudaEventSynchronize(ctx->ev_copy[k]), "record wait");
    if (ticket < ctx->next_ticket - LBM_RECORD_DEPTH) return LBM_OK;
    const int st = ctx->rec[k]->status;
    if (st & ST_UNSTABLE) return fail(ctx, LBM_ERR_UNSTABLE, "a node had non-finite or non-positive density");
    if (st & ST_BAND_OVERFLOW) return fail(ctx, LBM_ERR_STATE, "body band or boundary list overflowed its capacity");
    return LBM_OK;
}

lbm_status lbm_reset_average(lbm_ctx *ctx)
{
    if (!ctx) return LBM_ERR_ARG;
    DevBody *b = ctx->S.body + ctx->bcur;
    LBM_CUDA(cudaMemsetAsync(&b->F_sum, 0, sizeof(b->F_sum) + sizeof(b->M_sum) + sizeof(b->n_sum), ctx->stream), "reset");
    return LBM_OK;
}

lbm_status lbm_totals(lbm_ctx *ctx, double out[5])
{
    NvtxRange nvtx_("lbm_totals");
    if (!ctx) return LBM_ERR_ARG;
    if (!out) return fail(ctx, LBM_ERR_ARG, "lbm_totals: null output");
    const uint8_t *fl = ctx->has_body ? ctx->flags : nullptr;
    LBM_CUDA(launch_totals(ctx->storage, ctx->L, ctx->f[ctx->cur], fl, ctx->tot_partials, ctx->tot_blocks,
                           nullptr, ctx->stream), "totals");
    std::vector<double> h((size_t)ctx->tot_blocks * 5);
    LBM_CUDA(cudaMemcpyAsync(h.data(), ctx->tot_partials, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             ctx->stream), "totals read");
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "sync");
    for (int k = 0; k < 5; ++k) out[k] = 0;
    for (int b = 0; b < ctx->tot_blocks; ++b)
        for (int k = 0; k < 5; ++k) out[k] += h[(size_t)b * 5 + k];
    return LBM_OK;
}

namespace {
struct CheckpointHeader {
    char magic[8];
    int32_t version, nx, ny, nz, storage, body_kind, reserved;
    int64_t pop_bytes, flag_bytes, body_bytes;
};

// device <-> file in chunks through a host buffer
bool copy_to_file(FILE *fp, const void *dev, size_t bytes, cudaStream_t s)
{
    std::vector<char> buf(std::min<size_t>(bytes, (size_t)64 << 20));
    for (size_t off = 0; off < bytes; off += buf.size()) {
        const size_t n = std::min(buf.size(), bytes - off);
        if (cudaMemcpyAsync(buf.data(), (const char *)dev + off, n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess || fwrite(buf.data(), 1, n, fp) != n)
            return false;
    }
    return true;
}

bool copy_from_file(FILE *fp, void *dev, size_t bytes, cudaStream_t s)
{
    std::vector<char> buf(std::min<size_t>(bytes, (size_t)64 << 20));
    for (size_t off = 0; off < bytes; off += buf.size()) {
        const size_t n = std::min(buf.size(), bytes - off);
        if (fread(buf.data(), 1, n, fp) != n ||
            cudaMemcpyAsync((char *)dev + off, buf.data(), n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return false;
    }
    return true;
}
}  // namespace

lbm_status lbm_save(lbm_ctx *ctx, const char *path)
{
    if (!ctx) return LBM_ERR_ARG;
    if (!path) return fail(ctx, LBM_ERR_ARG, "lbm_save: null path");
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "sync");
    CheckpointHeader h{};
    memcpy(h.magic, "LBMKBC01", 8);
    h.version = 1;
    h.nx = ctx->L.nx; h.ny = ctx->L.ny; h.nz = ctx->L.nz;
    h.storage = ctx->storage;
    h.body_kind = ctx->has_body ? ctx->G.kind : LBM_BODY_NONE;
    h.pop_bytes = (int64_t)Q * ctx->L.N * (int64_t)ctx->elem;
    h.flag_bytes = ctx->L.N;
    h.body_bytes = sizeof(DevBody);
    FILE *fp = fopen(path, "wb");
    if (!fp) return fail(ctx, LBM_ERR_ARG, std::string("lbm_save: cannot open ") + path);
    bool ok = fwrite(&h, sizeof(h), 1, fp) == 1 &&
              copy_to_file(fp, ctx->f[ctx->cur], (size_t)h.pop_bytes, ctx->stream) &&
              copy_to_file(fp, ctx->flags, (size_t)h.flag_bytes, ctx->stream) &&
              copy_to_file(fp, ctx->S.body + ctx->bcur, sizeof(DevBody), ctx->stream);
    ok = (fclose(fp) == 0) && ok;
    return ok ? LBM_OK : fail(ctx, LBM_ERR_ARG, std::string("lbm_save: write failed for ") + path);
}

lbm_status lbm_load(lbm_ctx *ctx, const char *path)
{
    if (!ctx) return LBM_ERR_ARG;
    if (!path) return fail(ctx, LBM_ERR_ARG, "lbm_load: null path");
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(ctx, LBM_ERR_ARG, std::string("lbm_load: cannot open ") + path);
    CheckpointHeader h{};
    const bool hdr = fread(&h, sizeof(h), 1, fp) == 1;
    const int kind = ctx->has_body ? ctx->G.kind : LBM_BODY_NONE;
    if (!hdr || memcmp(h.magic, "LBMKBC01", 8) != 0 || h.version != 1 || h.nx != ctx->L.nx ||
        h.ny != ctx->L.ny || h.nz != ctx->L.nz || h.storage != ctx->storage || h.body_kind != kind ||
        h.pop_bytes != (int64_t)Q * ctx->L.N * (int64_t)ctx->elem || h.flag_bytes != ctx->L.N ||
        h.body_bytes != (int64_t)sizeof(DevBody)) {
        fclose(fp);
        return fail(ctx, LBM_ERR_ARG, std::string("lbm_load: ") + path + " does not match this context");
    }
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "sync");
    LBM_CUDA(drain_records(ctx), "record copies");
    bool ok = copy_from_file(fp, ctx->f[ctx->cur], (size_t)h.pop_bytes, ctx->stream) &&
              copy_from_file(fp, ctx->flags, (size_t)h.flag_bytes, ctx->stream) &&
              copy_from_file(fp, ctx->S.body + ctx->bcur, sizeof(DevBody), ctx->stream);
    fclose(fp);
    if (!ok) return fail(ctx, LBM_ERR_ARG, std::string("lbm_load: read failed for ") + path);
    ctx->initialised = true;
    ctx->interior_pending = false;
    return LBM_OK;
}

lbm_status lbm_profile_begin(lbm_ctx *ctx, int max_launches)
{
    if (!ctx) return LBM_ERR_ARG;
    if (max_launches < 1) return fail(ctx, LBM_ERR_ARG, "lbm_profile_begin: max_launches < 1");
    if (ctx->prof_open) return fail(ctx, LBM_ERR_STATE, "lbm_profile_begin: a profile is already open");
    ctx->prof.assign((size_t)2 * max_launches, nullptr);
    for (auto &e : ctx->prof) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto &f : ctx->prof) if (f) cudaEventDestroy(f);
            ctx->prof.clear();
            return fail(ctx, LBM_ERR_CUDA, "lbm_profile_begin: event creation failed");
        }
    }
    ctx->prof_used = 0;
    ctx->prof_open = true;
    return LBM_OK;
}

lbm_status lbm_profile_end(lbm_ctx *ctx, double *total_ms, int64_t *launches)
{
    if (!ctx) return LBM_ERR_ARG;
    if (!ctx->prof_open) return fail(ctx, LBM_ERR_STATE, "lbm_profile_end: no profile open");
    if (!total_ms || !launches) return fail(ctx, LBM_ERR_ARG, "lbm_profile_end: null output");
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "sync");
    double sum = 0;
    for (int k = 0; k < ctx->prof_used; ++k) {
        float ms = 0;
        LBM_CUDA(cudaEventElapsedTime(&ms, ctx->prof[2 * k], ctx->prof[2 * k + 1]), "elapsed");
        sum += ms;
    }
    *total_ms = sum;
    *launches = ctx->prof_used;
    for (cudaEvent_t e : ctx->prof) cudaEventDestroy(e);
    ctx->prof.clear();
    ctx->prof_open = false;
    ctx->prof_used = 0;
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- slabs
lbm_status lbm_set_slab(lbm_ctx *ctx, int zoff, int zper, int own_lo, int own_hi)
{
    if (!ctx) return LBM_ERR_ARG;
    const Lattice &L = ctx->L;
    if (ctx->has_body) return fail(ctx, LBM_ERR_STATE, "lbm_set_slab: call it before lbm_set_geometry");
    if (zper < L.nz - 2 || zper < 1 || own_lo < 0 || own_hi > L.nz || own_lo >= own_hi)
        return fail(ctx, LBM_ERR_ARG, "lbm_set_slab: need zper >= nz - 2 and 0 <= own_lo < own_hi <= nz");
    if (L.face[4] != L.face[5] || (L.face[4] != LBM_FACE_WALL && L.face[4] != LBM_FACE_PERIODIC))
        return fail(ctx, LBM_ERR_ARG, "lbm_set_slab: the slab's own z faces must be both walls or both periodic");
    ctx->slab_zoff = zoff;
    ctx->slab_zper = zper;
    ctx->slab_own_lo = own_lo;
    ctx->slab_own_hi = own_hi;
    return LBM_OK;
}

// layers [z0, z0 + nlayers) of all 27 planes of the current state <-> a
// plane-major contiguous buffer: one strided copy (27 rows, pitch N)
static lbm_status copy_layers(lbm_ctx *ctx, int z0, int nlayers, void *buf, bool pack)
{
    if (!ctx) return LBM_ERR_ARG;
    const Lattice &L = ctx->L;
    if (!buf || nlayers < 1 || z0 < 0 || z0 + nlayers > L.nz)
        return fail(ctx, LBM_ERR_ARG, "lbm_pack_layers / lbm_unpack_layers: layers outside the box or null buffer");
    const size_t e = ctx->elem, layer = (size_t)L.nx * L.ny * e;
    char *state = (char *)ctx->f[ctx->cur] + (size_t)z0 * layer;
    const size_t width = (size_t)nlayers * layer, pitch = (size_t)L.N * e;
    cudaError_t err = pack ? cudaMemcpy2DAsync(buf, width, state, pitch, width, Q, cudaMemcpyDeviceToDevice, ctx->stream)
                           : cudaMemcpy2DAsync(state, pitch, buf, width, width, Q, cudaMemcpyDeviceToDevice, ctx->stream);
    if (err != cudaSuccess) return cuda_fail(ctx, err, pack ? "lbm_pack_layers" : "lbm_unpack_layers");
    return LBM_OK;
}

lbm_status lbm_pack_layers(lbm_ctx *ctx, int z0, int nlayers, void *dst) { return copy_layers(ctx, z0, nlayers, dst, true); }

lbm_status lbm_unpack_layers(lbm_ctx *ctx, int z0, int nlayers, const void *src)
{
    return copy_layers(ctx, z0, nlayers, const_cast<void *>(src), false);
}

lbm_status lbm_set_body_force(lbm_ctx *ctx, const double F[3], const double M[3])
{
    if (!ctx) return LBM_ERR_ARG;
    if (!F || !M) return fail(ctx, LBM_ERR_ARG, "lbm_set_body_force: null force or torque");
    if (!ctx->has_body) return fail(ctx, LBM_ERR_STATE, "lbm_set_body_force: no body");
    double fm[6];
    for (int a = 0; a < 3; ++a) {
        fm[a] = F[a];
        fm[3 + a] = M[a];
    }
    LBM_CUDA(launch_set_force(ctx->S, ctx->bcur, fm, ctx->stream), "lbm_set_body_force");
    return LBM_OK;
}

lbm_status lbm_body_force_to_device(lbm_ctx *ctx, double *dst)
{
    if (!ctx) return LBM_ERR_ARG;
    if (!dst) return fail(ctx, LBM_ERR_ARG, "lbm_body_force_to_device: null buffer");
    if (!ctx->has_body) return fail(ctx, LBM_ERR_STATE, "lbm_body_force_to_device: no body");
    const DevBody *b = ctx->S.body + ctx->bcur;
    static_assert(offsetof(DevBody, M) == offsetof(DevBody, F) + 3 * sizeof(double), "F and M adjacent");
    LBM_CUDA(cudaMemcpyAsync(dst, b->F, 6 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream),
             "lbm_body_force_to_device");
    return LBM_OK;
}

lbm_status lbm_sum_body_force(lbm_ctx *ctx, const double *parts, int nparts)
{
    if (!ctx) return LBM_ERR_ARG;
    if (!parts || nparts < 1) return fail(ctx, LBM_ERR_ARG, "lbm_sum_body_force: null buffer or no parts");
    if (!ctx->has_body) return fail(ctx, LBM_ERR_STATE, "lbm_sum_body_force: no body");
    LBM_CUDA(launch_sum_force(ctx->S, ctx->bcur, parts, nparts, ctx->stream), "lbm_sum_body_force");
    return LBM_OK;
}
