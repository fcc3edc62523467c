/*
 * C ABI of the GB300 entropic lattice Boltzmann library (liblbm.so).
 *
 * Method: Dorschner, Chikatamarla, Karlin, "Entropic lattice Boltzmann method
 * for moving and deforming geometries in three dimensions", arXiv 1608.04658.
 *   - Sec. 2, Eqs. (kineticEq), (kbc_relax), (feq_min) and the analytic
 *     stabilizer: the D3Q27 KBC stream + collide step (lbm_step).
 *   - Sec. 3, Eqs. (grad), (pressure), (pressure2), target density and
 *     velocity, refill: the moving-wall boundary (lbm_step, geometry set by
 *     lbm_set_geometry).
 *   - Sec. 4.1: Galilean-invariant momentum exchange and Newton's equations
 *     of the sphere with Euler integration (lbm_step, lbm_body_forces).
 *   - Sec. 4.2: plunging airfoil (prescribed plunge); Sec. 4.3: triangulated
 *     anguilliform swimmer with a prescribed midline deformation, held or
 *     free in any of x, y and yaw (lbm_set_geometry).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an lbm_status; LBM_OK is 0.  On failure the message
 *     is kept in the context and returned by lbm_last_error.  No C++
 *     exception crosses the ABI.
 *   - Lattice layout: populations are structure-of-arrays, element
 *     f[i * N + x + nx * (y + ny * z)] with N = nx * ny * nz and direction
 *     index i = 9 (cx + 1) + 3 (cy + 1) + (cz + 1) (opposite direction 26 - i).
 *   - Stored value: the shifted population g_i = f_i - W_i * rho0 in the
 *     storage type (FP64, FP32, FP16 or BF16, round-to-nearest-even); the
 *     collision computes in FP64 for FP64 storage and in FP32 otherwise.
 *   - The stored state is the post-collision population f'_i(x, t), the
 *     right side of Eq. (kineticEq).
 *   - Calls are asynchronous on the context's CUDA stream unless documented
 *     as synchronising.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,         /* invalid argument: sizes, null pointers, mixed faces */
    LBM_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    LBM_ERR_OOM = 3,         /* device allocation failed */
    LBM_ERR_UNSTABLE = 4,    /* a node had non-finite or non-positive density */
    LBM_ERR_TIMEOUT = 5,     /* reserved: no kernel of this library waits on a device
                                flag or barrier, so no call returns it */
    LBM_ERR_STATE = 6,       /* call out of order (e.g. step before init) */
    LBM_ERR_UNSUPPORTED = 7  /* option not built */
} lbm_status;

typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16 = 2, LBM_BF16 = 3 } lbm_storage;

/* Box faces.  The paper specifies none; these are the conditions the
 * workloads need.  For a pull F_i(x) = f'_i(x - c_i) whose source leaves the
 * box through a face:
 *   PERIODIC  the source wraps around (both faces of an axis must be periodic),
 *   WALL      halfway bounce-back at rest: F_i(x) = f'_{26-i}(x),
 *   EQ        F_i(x) = f_i^eq(rho0, u_face),
 *   OUTFLOW   the source is clamped onto the face (zero-gradient).
 * When a source leaves through several faces, WALL wins over EQ, and EQ over
 * the clamped or wrapped source. */
typedef enum { LBM_FACE_PERIODIC = 0, LBM_FACE_WALL = 1, LBM_FACE_EQ = 2, LBM_FACE_OUTFLOW = 3 } lbm_face;

/* Stabilizer: ANALYTIC is gamma = 1/beta - (2 - 1/beta) <ds|dh>/<dh|dh>
 * (Sec. 2; gamma = 2 when <dh|dh> underflows).  EXACT is the root of Eq.
 * (gamma_min), sum_i dh_i log(f'_i(gamma)/f^eq_i) = 0, on the interval where
 * every post-collision population stays positive (safeguarded Newton from the
 * analytic value, at most 40 iterations; not supported by lbm_adjoint_step).
 * LBGK forces gamma = 2, which is BGK with relaxation 2 beta. */
typedef enum { LBM_GAMMA_ANALYTIC = 0, LBM_GAMMA_EXACT = 1, LBM_GAMMA_LBGK = 2 } lbm_gamma_mode;


typedef struct {
    int32_t nx, ny, nz;   /* lattice size, each >= 1, 27 * nx * ny * nz < 2^31 */
    int32_t storage;      /* lbm_storage */
    int32_t face[6];      /* lbm_face for x-, x+, y-, y+, z-, z+ */
    int32_t gamma_mode;   /* lbm_gamma_mode */
    int32_t options;      /* reserved, must be 0 */
    double nu;            /* kinematic viscosity: beta = 1/(6 nu + 1) (Sec. 2, c_s^2 = 1/3) */
    double rho0;          /* reference density of the shifted storage and of rho_dyn */
    double u_face[3];     /* velocity of EQ faces */
} lbm_params;

typedef enum {
    LBM_BODY_NONE = 0, LBM_BODY_SPHERE = 1, LBM_BODY_PLANES = 2, LBM_BODY_AIRFOIL = 3, LBM_BODY_MESH = 4
} lbm_body_kind;

/* Immersed body.  A node is solid when its centre lies inside the body
 * (strictly).  On periodic axes the sphere is taken at its nearest image.
 *   SPHERE: centre X, radius R, translational velocity U.  With free_motion
 *     the centre follows Newton's equations (Sec. 4.1) by explicit Euler:
 *     X += U, then U += F/mass + (1 - 1/rho_ratio) g, with F the momentum-
 *     exchange force of the previous step.
 *   PLANES: solid where y < y_lo or y > y_hi; walls move with U_lo / U_hi.
 *   AIRFOIL: extruded along z, leading edge at (X[0], X[1]) at zero plunge.
 *     In the chord frame xi = (dx ca - dy sa)/chord, eta = (dx sa + dy ca)/chord
 *     (dx, dy from the leading edge, (ca, sa) the cosine and sine of the nose-up
 *     angle of attack) a node is solid when 0 <= xi <= 1 and
 *     |eta - y_c(xi)| < t(xi): y_c the four-digit camber line of maximum
 *     camber_m at chord position camber_p, t(xi) = thick[0] sqrt(xi) + thick[1] xi
 *     + ... + thick[4] xi^4.  Prescribed plunge (Sec. 4.2): the leading edge is at
 *     y = X[1] + h_amp sin(h_omega t) at step t (t0 at lbm_set_geometry); the
 *     wall moves with the plunge velocity.  Link fractions are found by 50
 *     bisections of the link.
 *   MESH: closed triangulated swimmer (Sec. 4.3).  mesh_rest holds, per
 *     vertex, its arc position s >= 0 along the centre line and its offsets
 *     (dy, dz) from it; mesh_tris three vertex indices per triangle (a closed,
 *     consistently oriented surface).  Both are host arrays, copied.  At step t
 *     vertex v sits at (X[0] + s, (X[1] + y(s,t)) + dy, X[2] + dz) with the
 *     midline y(s,t) = r(t) wave_amp length (s/length + 0.03125)/1.03125
 *     sin(2 pi (s/wave_length - t/wave_period)); r(t) = (1 - cos(pi t/T))/2 for
 *     0 <= t < T with wave_ramp, 1 otherwise.  Its velocity is U plus the
 *     central difference (y(s,t+1) - y(s,t-1))/2 along y.  A node is solid when
 *     the ray from it along +x crosses the surface an odd number of times
 *     (edge functions of the (y, z) projection, each edge evaluated from its
 *     lower-index vertex, zero counted positive).  A link's wall point is its
 *     first crossing with a triangle; the wall velocity there is the
 *     barycentric interpolation of the vertex velocities.  free_motion is a
 *     bit mask of the free degrees of freedom: 1 x, 2 y, 4 yaw.  Held (0) or
 *     free in x only (1), X is the head and Newton's equation along x is
 *     advanced by explicit Euler: X[0] += U[0], then U[0] += F[0]/mass.  With
 *     y or yaw free, X is the centre of mass and the body frame turns by psi
 *     about z: vertex v sits at X + R(psi) (b_v - c(t)), b_v = (s, y(s,t) + dy,
 *     dz), c(t) the centre of mass of the mesh (divergence theorem, density
 *     mass / volume); its velocity is U + omega e_z x (p - X) +
 *     R(psi) (b_v_dot - c_dot) (central differences); Euler on the free
 *     degrees: X += U, U += F/mass, psi += omega, I omega += M_z with I the
 *     moment of inertia about the vertical axis through the centre of mass of
 *     the new pose (d(I omega)/dt = M of Sec. 4.3).  t0 is the time of the
 *     initial pose.  The body must stay two nodes clear of every box face; a pose
 *     outside that sets status bit 2 (band overflow), as does a column crossed
 *     more than 32 times or a 2x2x2 cell overlapped by more than 384
 *     triangles. */
typedef struct {
    int32_t kind;         /* lbm_body_kind */
    int32_t free_motion;  /* 1: integrate the sphere's translation */
    double X[3];
    double U[3];
    double R;
    double y_lo, y_hi;
    double U_lo[3], U_hi[3];
    double mass;          /* body mass; a SPHERE given 0 takes m_s = rho_s pi D^3 / 6
                             (rho_s = rho_ratio rho0, analytic volume, Sec. 4.1) */
    double rho_ratio;     /* rho_s / rho_f */
    double g[3];          /* gravity */
    double chord, ca, sa, h_amp, h_omega, camber_m, camber_p, thick[5], t0;  /* AIRFOIL; t0 also MESH */
    const double *mesh_rest;   /* MESH: host, 3 doubles (s, dy, dz) per vertex */
    const int32_t *mesh_tris;  /* MESH: host, 3 vertex indices per triangle */
    int32_t n_vertices, n_triangles;
    double length;             /* MESH: body length L */
    double wave_amp;           /* MESH: midline amplitude factor (0.125 in Sec. 4.3) */
    double wave_length;        /* MESH: lambda */
    double wave_period;        /* MESH: T, steps */
    int32_t wave_ramp;         /* MESH: 1 to ramp the amplitude up over the first period */
    int32_t reserved_mesh;     /* must be 0 */
    double psi, omega;         /* MESH free in y or yaw: initial yaw angle and rate (rad, rad/step) */
} lbm_geometry;

/* Body state on the device, read back by lbm_get_body. */
typedef struct {
    double X[3], U[3];    /* pose at the current step */
    double F[3], M[3];    /* force and torque of the fluid on the body, last step */
    double F_sum[3], M_sum[3]; /* sums since the last lbm_reset_average */
    int64_t n_sum;        /* number of steps in the sums */
    int32_t n_boundary;   /* boundary nodes of the last step */
    int32_t n_uncovered;  /* nodes refilled in the last step */
    int32_t n_links;      /* missing populations of the last step */
    int32_t status;       /* device status bits (1: unstable node, 2: band overflow) */
    int32_t n_band;       /* nodes of the last step's sweep box, updated by a launch of their own after the
                             body's marks (0 when the step used one flag-aware bulk launch) */
    double t;             /* time of the current pose (prescribed motion), steps */
    double psi, omega;    /* MESH in the centre-of-mass frame: yaw angle and rate */
    double Izz;           /* MESH in the centre-of-mass frame: moment of inertia of the pose */
} lbm_body_state;

typedef struct lbm_ctx lbm_ctx;

/* Creates a context over caller-owned device buffers.
 *   f_a, f_b  device buffers of 27 * N elements of the storage type
 *             (8, 4, 2 or 2 bytes each), 16-byte aligned; f_a holds the state.
 *   flags     device buffer of N bytes (node marks, written by the library).
 *   stream    cudaStream_t to enqueue on (NULL: the legacy default stream).
 * The library never frees the caller's buffers.  Returns LBM_ERR_ARG for
 * bad sizes or null pointers.  *out is NULL on failure. */
LBM_API lbm_status lbm_create(const lbm_params *p, void *f_a, void *f_b, uint8_t *flags,
                              void *stream, lbm_ctx **out);

/* Device allocator for the library's own scratch (boundary lists and body
 * arrays of lbm_set_geometry, the checkpoints and work arrays of
 * lbm_adjoint_step, the plane buffer of lbm_get/set_populations, the
 * moments of lbm_refine_create on a coarse context).  The paper has no such
 * interface; it lets a caller that pools its device memory (PyTorch's caching
 * allocator, an application arena) hand the library that memory instead of
 * plain cudaMalloc / cudaFree.
 *   alloc(bytes, stream, user)  returns device memory of the context's device,
 *                               at least 256-byte aligned, or NULL (the
 *                               calling entry point then fails with
 *                               LBM_ERR_OOM; a block that is not 256-byte
 *                               aligned is given back at once and counts as
 *                               NULL); stream is the context's stream;
 *   release(ptr, stream, user)  gives a block back; the library calls it only
 *                               when no work of its own that uses the block
 *                               is still in flight on any stream.
 * Both NULL restores cudaMalloc / cudaFree.  The few small buffers of
 * lbm_create itself stay cudaMalloc'd.  Call it before the first call that
 * allocates scratch: LBM_ERR_STATE once the context holds scratch from the
 * other allocator; LBM_ERR_ARG for a null context or only one of the two
 * functions. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*lbm_release_fn)(void *ptr, void *stream, void *user);
LBM_API lbm_status lbm_set_allocator(lbm_ctx *ctx, lbm_alloc_fn alloc, lbm_release_fn release, void *user);

/* Sets the state to the entropic equilibrium f_i = f_i^eq(rho, u) (Eq.
 * feq_min): lbm_init_state without the noise term; rho and u as there. */
LBM_API lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const double *rho, const double *u);

/* Releases the context and the library's own device scratch. */
LBM_API void lbm_destroy(lbm_ctx *ctx);

/* Message of the last failed call on this context ("" if none). */
LBM_API const char *lbm_last_error(const lbm_ctx *ctx);

/* Sets the state to f_i = f_i^eq(rho, u) + amp * W_i * xi_i (Eq. feq_min, exact
 * D3Q27 equilibrium), computed on the device in the collision's arithmetic
 * (double for FP64 storage, FP32 for the others) and rounded once to storage.
 *   rho  N doubles; u 3N doubles node-major (u[3n + a]);
 *   xi   27N doubles direction-major, or NULL for none;
 * each in device memory or in pinned host memory (cudaHostAlloc: the kernel
 * reads it across the host link at its mapped device address); anything else
 * (pageable host memory) is LBM_ERR_ARG. */
LBM_API lbm_status lbm_init_state(lbm_ctx *ctx, const double *rho, const double *u,
                                  const double *xi, double amp);
/* The same from single-precision fields (half the bytes to move; each value
 * is taken exactly as the double it converts to). */
LBM_API lbm_status lbm_init_state_f32(lbm_ctx *ctx, const float *rho, const float *u,
                                      const float *xi, double amp);

/* Sets the immersed body (copied; may be called again to replace it) and
 * marks the nodes inside it as solid at the current step.  Allocates the
 * library's boundary scratch (sized from the body) with cudaMalloc. */
LBM_API lbm_status lbm_set_geometry(lbm_ctx *ctx, const lbm_geometry *g);

/* Advances nsteps time steps (Eq. kineticEq with the KBC collision, Grad
 * boundaries, refill, momentum exchange and body update), asynchronously.
 * After an odd number of total steps the state lives in f_b: see
 * lbm_current_buffer. */
LBM_API lbm_status lbm_step(lbm_ctx *ctx, int nsteps);

/* 0 if the current state is in f_a, 1 if in f_b. */
LBM_API int lbm_current_buffer(const lbm_ctx *ctx);

/* Copies the current state to host memory as full populations
 * f_i = g_i + W_i rho0 in double, layout as above (27 * N doubles).
 * Synchronises the context stream. */
LBM_API lbm_status lbm_get_populations(lbm_ctx *ctx, double *host_f);

/* Sets the current state from full host populations (27 * N doubles),
 * rounding to the storage type.  Synchronises. */
LBM_API lbm_status lbm_set_populations(lbm_ctx *ctx, const double *host_f);

/* Force and torque of the fluid on the body (Sec. 4.1, Galilean-invariant
 * momentum exchange); averaged != 0 returns the mean since the last
 * lbm_reset_average.  Synchronises.  Returns LBM_ERR_UNSTABLE if a node went
 * unstable since creation. */
LBM_API lbm_status lbm_body_forces(lbm_ctx *ctx, double F[3], double M[3], int averaged);

/* Force record of one step, written by lbm_body_forces_async. */
typedef struct {
    double F[3], M[3];  /* force and torque of the fluid on the body, as lbm_body_forces (averaged = 0) */
    double t;           /* time of the body pose after that step */
    int32_t status;     /* device status bits after that step (as lbm_body_state.status) */
    int32_t reserved;
} lbm_force_record;

/* Depth of the ring of outstanding asynchronous force records per context. */
#define LBM_RECORD_DEPTH 8

/* Asynchronous form of lbm_body_forces (Sec. 4.1, the same momentum exchange
 * force): enqueues, behind the work already on the context's stream, a copy
 * of the last step's force, torque, time and status into *out and returns at
 * once, so the host can enqueue the next steps while the copy is in flight.
 * out must be page-locked host memory (cudaHostAlloc / cudaHostRegister, a
 * pinned torch tensor) owned by the caller and left untouched until
 * lbm_body_forces_wait on the returned *ticket has returned; LBM_ERR_ARG
 * otherwise.  The copy runs on a library stream of its own; the step that
 * would overwrite the copied body state waits for it on the device.  At most
 * LBM_RECORD_DEPTH records should be outstanding: a ticket older than that is
 * waited for through a later copy. */
LBM_API lbm_status lbm_body_forces_async(lbm_ctx *ctx, lbm_force_record *out, int64_t *ticket);

/* Blocks until the record of ticket has landed in host memory, then returns
 * the error lbm_body_forces would return for that step's status bits
 * (LBM_ERR_UNSTABLE, LBM_ERR_STATE) or LBM_OK.  LBM_ERR_ARG
 * for a ticket not yet issued. */
LBM_API lbm_status lbm_body_forces_wait(lbm_ctx *ctx, int64_t ticket);

/* Full body state (pose, forces, counters, status).  Synchronises. */
LBM_API lbm_status lbm_get_body(lbm_ctx *ctx, lbm_body_state *out);

/* Clears the force/torque sums used for averages (asynchronous). */
LBM_API lbm_status lbm_reset_average(lbm_ctx *ctx);

/* Checkpoint of the current state: a header (lattice size, storage, body kind),
 * the stored populations in their storage type, the node marks and the body
 * state, written to the file at path.  lbm_load reads such a file into a
 * context created with the same lattice size and storage and given the same
 * body with lbm_set_geometry; stepping on from it continues bit for bit.
 * Both synchronise.  LBM_ERR_ARG for a mismatching or unreadable file. */
LBM_API lbm_status lbm_save(lbm_ctx *ctx, const char *path);
LBM_API lbm_status lbm_load(lbm_ctx *ctx, const char *path);

/* Mass, momentum (3) and kinetic energy summed over fluid nodes in double,
 * written to host out[5].  Synchronises. */
LBM_API lbm_status lbm_totals(lbm_ctx *ctx, double out[5]);

/* Launch order of the steps of a body whose band is known before its
 * geometry runs (sphere, airfoil, swimmer free at most along x).
 * LBM_ORDER_SPLIT: the nodes outside the body's band are updated on the
 * caller's stream while the body's geometry, boundary nodes, force and the
 * band's nodes run beside them on a library stream.  LBM_ORDER_SEQUENTIAL:
 * the geometry runs first, then one bulk launch over all nodes beside the
 * boundary nodes.  Both give the same results bit for bit; which is faster
 * depends on the size of the box against the body's work.  LBM_ORDER_AUTO
 * (the default): the first six steps after lbm_set_geometry alternate the two,
 * the last four of them timed with CUDA events, and the faster is kept. */
#define LBM_ORDER_AUTO 0
#define LBM_ORDER_SPLIT 1
#define LBM_ORDER_SEQUENTIAL 2

/* Requests a launch order (LBM_ORDER_*) for this and later geometries;
 * LBM_ERR_ARG for another value. */
LBM_API lbm_status lbm_set_launch_order(lbm_ctx *ctx, int order);

/* The order in use: LBM_ORDER_SPLIT or LBM_ORDER_SEQUENTIAL once chosen,
 * LBM_ORDER_AUTO while the trial is still open (split steps meanwhile), -1
 * for a null context. */
LBM_API int lbm_launch_order(const lbm_ctx *ctx);

/* Number of device kernels the last lbm_step call enqueued. */
LBM_API int64_t lbm_kernel_launches(const lbm_ctx *ctx);

/* Kernel timing with CUDA events on the context stream.  After
 * lbm_profile_begin(ctx, max_launches), each bulk stream-collide launch of the
 * following lbm_step calls (up to max_launches) is bracketed by two events.
 * lbm_profile_end synchronises, returns the summed device time of the
 * bracketed launches in *total_ms and their number in *launches, and releases
 * the events.  Returns LBM_ERR_STATE if no profile is open. */
LBM_API lbm_status lbm_profile_begin(lbm_ctx *ctx, int max_launches);
LBM_API lbm_status lbm_profile_end(lbm_ctx *ctx, double *total_ms, int64_t *launches);

/* Adjoint (reverse-mode) gradient of a time-averaged force objective over a
 * horizon of steps, by a hand-written adjoint of every part of lbm_step: the
 * KBC collision with its exact Jacobian (the stabilizer's dependence on f
 * included), the pull streaming with the box faces, the Grad boundary
 * (target density and velocity, finite-difference velocity gradient, link
 * fraction and wall velocity), the refill and the momentum exchange.  The
 * node marks, boundary links and refilled nodes of each step are taken as
 * fixed (piecewise-constant in the parameters).
 *
 * Objective: J = (1/horizon) sum_{t=0}^{horizon-1} w_force . F^t
 *              + sum over nodes fluid at the end of lambda_T . f(horizon),
 * F^t the force of the fluid on the body in step t (Sec. 4.1 momentum
 * exchange), f(horizon) the full populations after the last step.
 * Parameters theta (dJ_dtheta[3]):
 *   MESH: (wave_amp, wave_length, wave_period) of the midline (Sec. 4.3);
 *   AIRFOIL: (h_amp, h_omega) of the plunge (Sec. 4.2), third entry 0;
 *   other bodies: none (zeros).
 * The body is held, prescribed or free.  The free degrees of its state are
 * adjoint state too (the sphere's centre and velocity; the swimmer's head X0
 * and U0 in the head frame, or its centre of mass, velocity, yaw angle and
 * angular momentum in the centre-of-mass frame), carried back through the
 * explicit Euler update, the links' fraction and wall velocity, the refill
 * velocity and the momentum-exchange force and torque; theta also reaches the
 * swimmer's pose through the centre of mass c(t) and its rate, and the yaw
 * rate through the moment of inertia I(theta) (omega = L / I, the initial
 * L = I(t0) omega included).
 * Storage FP64 (arithmetic in double), FP32 or 16-bit (arithmetic in float;
 * 16-bit: the states and checkpoints in the storage type, each store's
 * rounding passing the adjoint unchanged).  The exact stabilizer returns
 * LBM_ERR_UNSUPPORTED.
 *
 * Memory: the forward states are kept by checkpoint-and-recompute: every
 * checkpoint_every steps (0: ceil(sqrt(horizon))) a state is kept, and each
 * segment is recomputed once during the reverse sweep; the call allocates
 * (ceil(horizon/K) + K + 3) state buffers of 27 N elements and frees them
 * before returning (LBM_ERR_OOM if they do not fit).
 *
 * On return the context has advanced by horizon steps, exactly as
 * lbm_step(horizon) would have (the forces of those steps are in the body
 * sums).  Synchronises. */
typedef struct {
    int32_t horizon;          /* steps, >= 1 */
    int32_t checkpoint_every; /* K, 0 for ceil(sqrt(horizon)) */
    double w_force[3];        /* weights of the mean force in J */
    const void *lambda_T;     /* device, 27 N values (double for FP64 storage, float for FP32) in
                                 the population layout, or NULL */
    void *lambda_0;           /* device out, same layout: dJ/df at the start (0 at solid and
                                 refilled nodes), or NULL */
    int32_t reserved[4];      /* must be 0 */
} lbm_adjoint;

LBM_API lbm_status lbm_adjoint_step(lbm_ctx *ctx, const lbm_adjoint *spec, double *J, double dJ_dtheta[3]);

/* ---- slab decomposition: one box split along z over several contexts ----
 * The paper gives no parallel scheme; this places its step on slabs of the
 * box, one exchange of edge layers per step (Sec. 2 streaming reads one layer
 * across a cut; the Sec. 3 refill of a node in that layer reads one more).
 *
 * lbm_set_slab: the context's lattice is a slab of a box periodic in z with
 * zper layers: its z layer k is the box's layer (zoff + k) mod zper.  Its
 * layers [own_lo, own_hi) are its own; the others are halo layers that the
 * caller refills before every step with the neighbouring slabs' own layers
 * (two halo layers per side are needed).  The body's pose stays in the box's
 * z (lbm_body_state reports it there): the sphere, airfoil and planes test
 * and wrap in the box's z; the mesh is placed in the slab's frame at the
 * image of its z nearest the slab's middle layer (its band cut at the slab's
 * layers).  The sphere's and the mesh's bands cover the image nearest the
 * slab's middle layer mid = nz / 2, so every other image must miss the
 * layers whose marks own nodes read, [own_lo - 1, own_hi]:
 * lbm_set_geometry fails with LBM_ERR_ARG unless (zper - e) / 2 > m, e the
 * body's z extent (sphere 2R, mesh that of its rest mesh) and m the largest
 * distance of those layers from mid.  The force and
 * torque of a step sum the links of own fluid nodes only; the caller adds the
 * slabs' sums (in a fixed slab order, so every slab holds the same bits) and
 * hands the total to every slab with lbm_set_body_force before the next step,
 * so the body copies move alike.  The context's own z faces must be both
 * walls or both periodic: no own node reads across them, and periodic faces
 * let the bulk kernel take its all-periodic form when x and y are periodic
 * too.  No adjoint on a slab.  Call before lbm_set_geometry.
 * Errors: LBM_ERR_ARG (sizes, faces), LBM_ERR_STATE (a body is already set). */
LBM_API lbm_status lbm_set_slab(lbm_ctx *ctx, int zoff, int zper, int own_lo, int own_hi);

/* A step of a slab in two calls, so that the halo exchange can run beside
 * the bulk of the step: lbm_step_interior enqueues the bulk update of the own
 * layers that pull from no halo layer, [own_lo + 1, own_hi - 1), for the
 * nodes outside the body's sweep box; the caller then refills the halo layers
 * (lbm_unpack_layers) and lbm_step_edges enqueues the rest of the step (the
 * body's chain, the first and last own layers) and ends it.  The own layers
 * get the bits of lbm_step; the halo layers of the new state are left as they
 * were (the next exchange refills them).  It applies without a body, and
 * with a body whose sweep box is known ahead once the split launch order is
 * asked for (lbm_set_launch_order); otherwise lbm_step_interior enqueues
 * nothing and lbm_step_edges runs the whole step.  lbm_step, and a second
 * lbm_step_interior, while a step is open: LBM_ERR_STATE; both calls on a
 * context that is not a slab: LBM_ERR_STATE. */
LBM_API lbm_status lbm_step_interior(lbm_ctx *ctx);
LBM_API lbm_status lbm_step_edges(lbm_ctx *ctx);

/* Copies the z layers [z0, z0 + nlayers) of the current state, all 27
 * planes, to dst / from src: device buffers of 27 * nlayers * nx * ny
 * elements of the storage type, plane-major (plane i first, then its
 * layers, x fastest), in the stored shifted form.  Asynchronous on the
 * context stream (one strided copy).  LBM_ERR_ARG for layers outside the box
 * or a null buffer. */
LBM_API lbm_status lbm_pack_layers(lbm_ctx *ctx, int z0, int nlayers, void *dst);
LBM_API lbm_status lbm_unpack_layers(lbm_ctx *ctx, int z0, int nlayers, const void *src);

/* Replaces the force F and torque M (host arrays of 3) of the body's current
 * state: the next step's Euler update reads them, and the running sums of
 * lbm_body_forces' average follow.  Asynchronous on the context stream.
 * LBM_ERR_STATE without a body. */
LBM_API lbm_status lbm_set_body_force(lbm_ctx *ctx, const double F[3], const double M[3]);

/* The same hand-over without the host: lbm_body_force_to_device copies the
 * body's current force and torque (F x, y, z, then M x, y, z: 6 doubles) to
 * the device buffer dst; lbm_sum_body_force replaces them by the sum of
 * nparts such records at parts (device, 6 * nparts doubles, record k at
 * 6k), added in record order from record 0 (the same bits as that order of
 * additions on the host).  Both asynchronous on the context stream; dst and
 * parts must stay valid until the stream reaches the call.  LBM_ERR_ARG for
 * a null buffer or nparts < 1, LBM_ERR_STATE without a body. */
LBM_API lbm_status lbm_body_force_to_device(lbm_ctx *ctx, double *dst);
LBM_API lbm_status lbm_sum_body_force(lbm_ctx *ctx, const double *parts, int nparts);

/* ---------------------------------------------------- two-level block refinement
 * Sec. 4.2 runs the airfoil on a grid with two levels of resolution and cites
 * the refinement algorithm without stating it.  This is one fine block of
 * ratio 2 inside a bodiless coarse lattice; the fine level may carry a body:
 *   - fine node j (per axis) sits at coarse coordinate lo + j/2, j = 0 .. 2m,
 *     m = hi - lo; the fine context's lattice has 2m + 2 nodes per axis and
 *     periodic faces (no interior pull reaches them; the last layer is a pad
 *     that nothing reads);
 *   - acoustic scaling: the fine level takes two steps per coarse step with
 *     the same rho and u and twice the coarse viscosity (its nu must be 2 nu
 *     of the coarse context, so b_f = b_c / (2 - b_c), Sec. 2's b);
 *   - the fine nodes on the block's surface are not updated by the fine
 *     level: each fine time they take the fine KBC collision of the entropic
 *     equilibrium (Eq. feq_min) at the coarse (rho, u) plus the second-order
 *     Hermite term of Grad's distribution (Eq. grad) carrying the coarse
 *     pre-collision Pi^neq times b_c / (2 b_f), the coarse moments taken
 *     trilinearly from the coarse nodes of the block's surface and linearly
 *     in time (the mean of t and t+1 at the half step);
 *   - the coarse nodes strictly inside the block are not updated by the
 *     coarse level; those one layer inside its surface take the coarse KBC
 *     collision of the same rebuild from the pre-collision moments of the
 *     coincident fine node, with the factor 2 b_f / b_c.
 *
 * A block may span a whole periodic axis of the coarse box (lo = 0 and hi =
 * n on that axis; the paper's airfoil is periodic along its span): it has no
 * surface along that axis, the fine lattice holds 2n nodes there (periodic,
 * no pad) and the surface interpolation wraps with the axis.  At least one
 * axis must stay closed.
 *
 * lbm_refine_create couples coarse and fine (both from lbm_create, the same
 * storage, stabilizer, rho0 and stream, no slab) over the block of
 * coarse nodes [lo, hi] (both ends included, per axis 1 <= lo, hi <= n - 2
 * and hi - lo >= 3, unless spanned).  It writes the fine context's flags
 * (the block's surface and the pad marked solid), takes its device scratch
 * (three sets of 10 moments per node of the block's coarse box: t, t+1 and
 * their mean) from the coarse context's allocator (cudaMalloc unless
 * lbm_set_allocator gave another) and synchronises the stream.  The coarse
 * context must carry no body; the fine one may (below).  Errors:
 * LBM_ERR_ARG for a mismatch, with the reason in lbm_last_error(coarse);
 * LBM_ERR_OOM.  *out is NULL on failure.
 *
 * A body on the fine level (lbm_set_geometry on the fine context, before
 * lbm_refine_init): a sphere, a swimmer mesh, or (in a block spanning z) the
 * airfoil, in fine lattice units (fine node j at fine coordinate j), stepped
 * by the fine level like a lattice of
 * its own, two steps per coarse step (its geometry, refill, Grad boundary,
 * force and Euler update each fine step; lbm_body_forces on the fine context
 * reads it in fine units).  Along closed axes its solid nodes must stay four
 * nodes inside the block's surface (fine coordinates in [4, 2m - 4]) so that
 * its band never reaches the surface; a band that does clears a surface
 * mark, which the surface fill reports as LBM_ERR_STATE from lbm_body_forces
 * on the fine context.  Walls, and the airfoil (extruded over the fine
 * lattice's z extent) in a block that does not span z, are
 * LBM_ERR_UNSUPPORTED at lbm_refine_init.
 *
 * lbm_refine_init, once both levels hold their initial state (lbm_init_state
 * or lbm_set_populations): re-marks the fine surface (lbm_set_geometry clears
 * the marks), takes the coarse moments at t = 0 from the coarse populations
 * themselves and sets the fine surface from them.  LBM_ERR_STATE if a level
 * has no state.
 *
 * lbm_refine_step advances nsteps coarse steps (2 nsteps fine steps),
 * asynchronously on the shared stream; afterwards read each level with
 * lbm_get_populations as usual.  Do not call lbm_step on either context of a
 * coupled pair.  Coarse nodes more than one layer inside the block's surface
 * and the fine pad hold no defined state.  LBM_ERR_STATE before
 * lbm_refine_init, or once the coarse context has been given a body.
 * lbm_kernel_launches(coarse) then counts the kernels the call enqueued
 * (seven per coarse step, plus a fine body's chain).  A fine profile
 * (lbm_profile_begin on the fine context) times the fine bulk launches.
 *
 * Checkpoints: lbm_save / lbm_load each level as usual, and lbm_refine_save /
 * lbm_refine_load the coupling's own state, the coarse surface moments of
 * the last step (a header naming the block and the storage, then the
 * moments; synchronises; LBM_ERR_ARG for a file of another coupling,
 * LBM_ERR_STATE for a save before lbm_refine_init).  Both levels loaded and
 * lbm_refine_load (in place of lbm_refine_init) continue the run bit for bit.
 * lbm_refine_init after a load instead takes the moments from the loaded
 * coarse populations (the t = 0 reading) and departs from the uninterrupted
 * run from its first step on.
 *
 * lbm_refine_destroy synchronises the stream and frees the scratch; the two
 * contexts stay valid.  Destroy the coupling before either context: it keeps
 * pointers to both. */
typedef struct lbm_refine lbm_refine;
LBM_API lbm_status lbm_refine_create(lbm_ctx *coarse, lbm_ctx *fine, const int32_t lo[3], const int32_t hi[3],
                                     lbm_refine **out);
LBM_API lbm_status lbm_refine_init(lbm_refine *r);
LBM_API lbm_status lbm_refine_step(lbm_refine *r, int nsteps);
LBM_API lbm_status lbm_refine_save(lbm_refine *r, const char *path);
LBM_API lbm_status lbm_refine_load(lbm_refine *r, const char *path);
LBM_API void lbm_refine_destroy(lbm_refine *r);

/* Global sums without a context and without device allocation.  The paper
 * has no counterpart to this entry point; it exists for callers that cannot
 * call cudaMalloc: applications that hand all device memory to their own
 * pool allocator, and monitoring code that must not enter the CUDA allocator
 * (which takes a process-wide lock and may synchronise the device) while a
 * time-stepping loop runs.
 *   p      lattice description (nx, ny, nz, storage, rho0; other fields unused)
 *   f      device populations, 27 * N elements of p->storage in the shifted
 *          layout of lbm_create
 *   flags  device node marks (N bytes) or NULL; nodes marked solid are skipped
 *   out    device output, 5 doubles: mass, momentum x/y/z, kinetic energy
 *   stream cudaStream_t to enqueue on (NULL: the legacy default stream)
 * Same sums as lbm_totals (same summands, another addition order), written
 * asynchronously to out.  The work space is a fixed array inside the library
 * (160 KB on every GPU that loads it, held until the process exits), so
 * lattices of more than 67,108,864 nodes are rejected with LBM_ERR_ARG.  The
 * kernels run on the current device: f, out and flags must be device memory
 * of that device (LBM_ERR_ARG otherwise).  The first call on a device looks
 * up that array's device address and keeps it for the life of the process
 * (a cudaDeviceReset of the device invalidates it); make that first call
 * before any stream capture.  All calls share the array: calls ordered on one
 * stream are safe, calls whose kernels overlap on the GPU race.  If a CUDA
 * error from earlier work is pending on the calling thread, nothing is
 * enqueued, LBM_ERR_CUDA is returned and the error is left in place for its
 * owner.  No error message is kept (there is no context); the status says
 * what failed. */
LBM_API lbm_status lbm_totals_noalloc(const lbm_params *p, const void *f, const uint8_t *flags,
                                      double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
