/*
 * FP64 CPU oracle for the entropic (KBC) lattice Boltzmann step with Grad
 * wall boundaries for moving bodies and momentum-exchange force coupling.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Paper: Dorschner, Chikatamarla, Karlin, "Entropic lattice Boltzmann method
 * for moving and deforming geometries in three dimensions" (arXiv 1608.04658).
 *   Sec. 2  Eq. (kineticEq)   stream + convex combination with the mirror state
 *           Eq. (kbc_relax)   KBC mirror state  k + (2 s^eq - s) + ((1-g) h + g h^eq)
 *           Eq. (feq_min)     entropic equilibrium (exact D3Q27 product solution)
 *           Eq. (gamma_min)   exact stabilizer (post-collision entropy minimum)
 *           analytic stabilizer  g = 1/b - (2 - 1/b) <ds|dh>/<dh|dh>
 *   Sec. 3  Eq. (grad)        Grad distribution f*(rho, u, Pi)
 *           Eqs. (pressure, pressure2)  Pi = Pi^eq + Pi^neq
 *           target velocity / target density (static + dynamic parts), refill
 *   Sec. 4.1  Newton's equations for the sphere, Euler integration,
 *             Galilean-invariant momentum exchange (Wen et al.)
 *   Sec. 4.2  plunging airfoil (analytic cambered stand-in, prescribed plunge)
 *   Sec. 4.3  anguilliform swimmer: triangulated body of elliptic cross
 *             sections, prescribed midline deformation, free translation
 *   Sec. 4.2  two-level grid (cited, not stated): one fine block of ratio 2
 *             coupled through rebuilt states (readings at the end of the file)
 *
 * Readings of points the paper leaves open are listed at the top of each
 * routine that takes them.  All arithmetic is IEEE double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 27
#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------- lattice */
/* D3Q27: c_i in {-1,0,1}^3 with index i = 9(cx+1) + 3(cy+1) + (cz+1), so the
 * opposite direction of i is 26 - i.  Weights are products of the 1-D weights
 * (2/3 for 0, 1/6 for +-1), c_s^2 = 1/3 (Sec. 2, standard D3Q27). */
static int C[Q][3];
static double W[Q];
static int tables_done = 0;

static double w1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

static void tables(void)
{
    if (tables_done) return;
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
            for (int c = -1; c <= 1; ++c) {
                int i = 9 * (a + 1) + 3 * (b + 1) + (c + 1);
                C[i][0] = a; C[i][1] = b; C[i][2] = c;
                W[i] = w1(a) * w1(b) * w1(c);
            }
    tables_done = 1;
}

static int opp(int i) { return 26 - i; }

void orc_lattice(int *c_out, double *w_out)
{
    tables();
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c_out[3 * i + a] = C[i][a];
        w_out[i] = W[i];
    }
}

/* ------------------------------------------------------------ equilibrium */
/* Eq. (feq_min): minimiser of H = sum f ln(f/W) under fixed rho, j.  The
 * exact D3Q27 solution (Ansumali, Karlin, Oettinger 2003, cited in Sec. 2) is
 * a product over the three axes:
 *   f_i^eq = rho * prod_a  w(c_ia) (2 - S_a) B_a^{c_ia},
 *   S_a = sqrt(1 + 3 u_a^2),  B_a = (2 u_a + S_a) / (1 - u_a). */
void orc_feq(double rho, const double *u, double *feq)
{
    tables();
    double fac[3][3]; /* fac[a][c+1] */
    for (int a = 0; a < 3; ++a) {
        double S = sqrt(1.0 + 3.0 * u[a] * u[a]);
        double B = (2.0 * u[a] + S) / (1.0 - u[a]);
        fac[a][0] = w1(-1) * (2.0 - S) / B;
        fac[a][1] = w1(0) * (2.0 - S);
        fac[a][2] = w1(1) * (2.0 - S) * B;
    }
    for (int i = 0; i < Q; ++i)
        feq[i] = rho * fac[0][C[i][0] + 1] * fac[1][C[i][1] + 1] * fac[2][C[i][2] + 1];
}

/* ---------------------------------------------------------------- moments */
static void moments(const double *f, double *rho, double *u)
{
    double r = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) j[a] += C[i][a] * f[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

/* 1-D dual basis of the monomials {1, c, c^2} on {-1,0,1}:
 * sum_c A_p(c) c^q = delta_pq.  A_0 = 1 - c^2, A_1 = c/2, A_2 = (3c^2 - 2)/2. */
static double A0(int c) { return 1.0 - (double)(c * c); }
static double A1(int c) { return 0.5 * c; }
static double A2(int c) { return 0.5 * (3.0 * c * c - 2.0); }

/* KBC split of the deviation df = f - f^eq (Sec. 2, Eq. kbc_relax).  The
 * kinematic part k carries the conserved moments, which f and f^eq share, so
 * dk = 0.  The shear part s carries the deviatoric (traceless) part of the
 * natural second moments P_ab = sum c_a c_b f; the trace is left in h because
 * the bulk viscosity relaxes with g*b (Sec. 2, xi = c_s^2 (1/(g b) - 1/2)).
 * s is rebuilt from its moments with the tensor-product dual basis, so that
 * its only non-zero natural moments are the deviatoric second moments.
 * dh = df - ds collects everything else. */
void orc_kbc_split(const double *f, double *feq, double *ds, double *dh)
{
    tables();
    double rho, u[3];
    moments(f, &rho, u);
    orc_feq(rho, u, feq);
    double df[Q], P[3][3] = {{0}};
    for (int i = 0; i < Q; ++i) {
        df[i] = f[i] - feq[i];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) P[a][b] += C[i][a] * C[i][b] * df[i];
    }
    double tr = P[0][0] + P[1][1] + P[2][2];
    double dev[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) dev[a][b] = P[a][b] - (a == b ? tr / 3.0 : 0.0);
    for (int i = 0; i < Q; ++i) {
        const int *c = C[i];
        double s = 0;
        /* diagonal moments M200, M020, M002 */
        s += dev[0][0] * A2(c[0]) * A0(c[1]) * A0(c[2]);
        s += dev[1][1] * A0(c[0]) * A2(c[1]) * A0(c[2]);
        s += dev[2][2] * A0(c[0]) * A0(c[1]) * A2(c[2]);
        /* off-diagonal moments M110, M101, M011 */
        s += dev[0][1] * A1(c[0]) * A1(c[1]) * A0(c[2]);
        s += dev[0][2] * A1(c[0]) * A0(c[1]) * A1(c[2]);
        s += dev[1][2] * A0(c[0]) * A1(c[1]) * A1(c[2]);
        ds[i] = s;
        dh[i] = df[i] - s;
    }
}

/* Entropic scalar product <X|Y> = sum X_i Y_i / f_i^eq (Sec. 2). */
static double esp(const double *X, const double *Y, const double *feq)
{
    double s = 0;
    for (int i = 0; i < Q; ++i) s += X[i] * Y[i] / feq[i];
    return s;
}

/* Discrete entropy H(f) = sum f ln(f/W) (Eq. feq_min). */
double orc_entropy(const double *f)
{
    tables();
    double H = 0;
    for (int i = 0; i < Q; ++i) H += f[i] * log(f[i] / W[i]);
    return H;
}

/* Left side of Eq. (gamma_min) as a function of the stabilizer g. */
double orc_gamma_residual(const double *ds, const double *dh, const double *feq,
                          double beta, double g)
{
    double s = 0;
    for (int i = 0; i < Q; ++i)
        s += dh[i] * log(1.0 + ((1.0 - beta * g) * dh[i] - (2.0 * beta - 1.0) * ds[i]) / feq[i]);
    return s;
}

/* Exact stabilizer: the root of Eq. (gamma_min).  Reading: the root is taken
 * on the interval of g where every post-collision population stays positive;
 * there the left side falls monotonically from +inf to -inf (its derivative is
 * -b sum dh_i^2 / f'_i), so plain bisection to machine precision finds the
 * unique root.  Returns 2 (the LBGK value) when dh vanishes. */
double orc_gamma_exact(const double *ds, const double *dh, const double *feq, double beta)
{
    double lo = -INFINITY, hi = INFINITY;
    int any = 0;
    for (int i = 0; i < Q; ++i) {
        /* positivity of f'_i:  a_i - g b_i > 0 */
        double a = feq[i] + dh[i] - (2.0 * beta - 1.0) * ds[i];
        double b = beta * dh[i];
        if (b > 0) { any = 1; if (a / b < hi) hi = a / b; }
        else if (b < 0) { any = 1; if (a / b > lo) lo = a / b; }
    }
    if (!any) return 2.0;
    for (int it = 0; it < 2000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double r = orc_gamma_residual(ds, dh, feq, beta, mid);
        if (r > 0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* KBC collision (Eqs. kineticEq, kbc_relax):
 *   f' = (1-b) f + b f^mirr = f - b (2 ds + g dh).
 * mode 0: analytic stabilizer  g = 1/b - (2 - 1/b) <ds|dh>/<dh|dh>;
 *         reading: when <dh|dh> underflows (<= 1e-300) g = 2 (dh is then
 *         zero, so the value does not matter); no clamping of g.
 * mode 1: exact stabilizer, the root of Eq. (gamma_min).
 * mode 2: g forced to 2, which is LBGK with relaxation 2b. */
double orc_collide(const double *f, double beta, int mode, double *out)
{
    double feq[Q], ds[Q], dh[Q], g;
    orc_kbc_split(f, feq, ds, dh);
    if (mode == 1) {
        g = orc_gamma_exact(ds, dh, feq, beta);
    } else if (mode == 2) {
        g = 2.0;
    } else {
        double hh = esp(dh, dh, feq);
        double sh = esp(ds, dh, feq);
        g = hh > 1e-300 ? 1.0 / beta - (2.0 - 1.0 / beta) * sh / hh : 2.0;
    }
    for (int i = 0; i < Q; ++i) out[i] = f[i] - beta * (2.0 * ds[i] + g * dh[i]);
    return g;
}

/* Grad distribution, Eq. (grad), with c_s^2 = 1/3:
 *   f*_i = W_i [ rho + 3 rho c_i.u + (9/2) (Pi - rho/3 I) : (c_i c_i - 1/3 I) ]. */
void orc_grad(double rho, const double *u, const double *Pi, double *out)
{
    tables();
    for (int i = 0; i < Q; ++i) {
        const int *c = C[i];
        double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        double contr = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double P = Pi[3 * a + b] - (a == b ? rho / 3.0 : 0.0);
                double H = c[a] * c[b] - (a == b ? 1.0 / 3.0 : 0.0);
                contr += P * H;
            }
        out[i] = W[i] * (rho + 3.0 * rho * cu + 4.5 * contr);
    }
}

/* Pressure tensor, Eqs. (pressure, pressure2):
 *   Pi = rho c_s^2 I + rho u u - (rho c_s^2 / (2 b)) (grad u + grad u^T),
 * with dudx[a][b] = d u_a / d x_b. */
static void pressure_tensor(double rho, const double *u, double dudx[3][3], double beta, double *Pi)
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            Pi[3 * a + b] = (a == b ? rho / 3.0 : 0.0) + rho * u[a] * u[b]
                            - rho / 3.0 / (2.0 * beta) * (dudx[a][b] + dudx[b][a]);
}

/* ----------------------------------------------------------------- lattice state */
enum { FACE_PERIODIC = 0, FACE_WALL = 1, FACE_EQ = 2, FACE_OUTFLOW = 3 };
enum { BODY_NONE = 0, BODY_SPHERE = 1, BODY_PLANES = 2, BODY_AIRFOIL = 3, BODY_MESH = 4 };

typedef struct {
    int nx, ny, nz;
    int face[6];       /* x-, x+, y-, y+, z-, z+ */
    int gamma_mode;    /* 0 analytic, 1 exact root, 2 LBGK */
    int pad_;
    double beta;       /* 1/(6 nu + 1) from nu = c_s^2 (1/(2b) - 1/2) */
    double rho0;
    double u_face[3];  /* velocity of the equilibrium faces */
} orc_params;

typedef struct {
    int kind;
    int free_motion;   /* 1: integrate translation (Newton + Euler) */
    double X[3];       /* sphere centre */
    double U[3];       /* translational velocity */
    double R;          /* sphere radius */
    double y_lo, y_hi; /* planes: solid where y < y_lo or y > y_hi */
    double U_lo[3], U_hi[3];
    double mass;       /* m_s */
    double rho_ratio;  /* rho_s / rho_f */
    double g[3];       /* gravity */
    double F[3], M[3]; /* hydrodynamic force and torque of the last step */
    /* airfoil extruded along z, leading edge at X (current, plunging in y) */
    double chord;      /* chord length c */
    double ca, sa;     /* cos and sin of the angle of attack (nose up) */
    double h_amp;      /* plunge amplitude (lattice units) */
    double h_omega;    /* plunge angular frequency (rad per step) */
    double camber_m, camber_p; /* camber line: maximum and its chord position */
    double thick[5];   /* half thickness a0 sqrt(x) + a1 x + a2 x^2 + a3 x^3 + a4 x^4 */
    double y_base;     /* leading-edge y at zero plunge */
    double t;          /* time of the current pose (steps) */
    /* triangulated swimmer: head at X (X[0] moves with U[0] when free), the
     * centre line along +x at (X[1], X[2]) displaced by the midline in y */
    const double *mesh_rest; /* (s, dy, dz) per vertex */
    const int *mesh_tris;    /* three vertex indices per triangle */
    int n_vertices, n_triangles;
    double length;     /* body length L */
    double wave_amp;   /* midline amplitude factor (0.125 in Sec. 4.3) */
    double wave_length;/* lambda */
    double wave_period;/* T (steps) */
    int wave_ramp;     /* 1: amplitude ramp over the first period */
    int pad2_;
    /* swimmer free in y or in yaw (free_motion bits 2, 4): X is the centre of
     * mass and the body frame turns by psi about z */
    double psi, omega; /* yaw angle and rate */
    double Iw;         /* angular momentum about the centre of mass, I_zz omega */
    double Izz;        /* moment of inertia of the current pose */
    double com[2];     /* centre of mass in the body frame (x, y) at the current pose */
    double com_dot[2]; /* its central-difference rate */
} orc_body;

typedef struct {
    orc_params p;
    orc_body b;
    long N;
    double *fa, *fb;      /* f[i*N + n], post-collision state */
    uint8_t *solid0;      /* solid at t */
    uint8_t *solid1;      /* solid at t+1 */
    double feq_face[Q];
    long step;
    long n_links, n_boundary, n_refill;
    double *vpos, *vvel;  /* mesh vertex positions and velocities at the current pose */
    double box_lo[3], box_hi[3]; /* bounding box of the mesh vertices */
    int error;            /* 1: the mesh left the box */
    int own_zlo, own_zhi; /* z layers whose boundary links enter F and M (the whole box by default) */
    int zf_origin, zf_period; /* slab frame: layer k sits at z = (k + origin) mod period (period 0: off) */
} orc_ctx;

static long nid(const orc_ctx *c, int x, int y, int z)
{
    return x + (long)c->p.nx * (y + (long)c->p.ny * z);
}

/* Displacement of a node from the sphere centre.  Reading (the paper's
 * sedimenting sphere falls through a periodic box): on a periodic axis the
 * centre is kept in [0, n) and the sphere is taken at its nearest image, by
 * adding or subtracting n once when |d| exceeds n/2. */
static void sphere_offset(const orc_ctx *c, double x, double y, double z, double *d)
{
    const orc_body *b = &c->b;
    double p[3] = {x, y, z};
    int n[3] = {c->p.nx, c->p.ny, c->p.nz};
    int zper = c->p.face[4] == FACE_PERIODIC;
    if (c->zf_period > 0) {
        /* a slab of a larger box periodic in z: the layer's position there */
        const long k = ((long)z + c->zf_origin) % c->zf_period;
        p[2] = (double)(k < 0 ? k + c->zf_period : k);
        n[2] = c->zf_period;
        zper = 1;
    }
    for (int a = 0; a < 3; ++a) {
        d[a] = p[a] - b->X[a];
        if (a == 2 ? zper : c->p.face[2 * a] == FACE_PERIODIC) {
            double h = 0.5 * n[a];
            if (d[a] > h) d[a] = d[a] - n[a];
            else if (d[a] < -h) d[a] = d[a] + n[a];
        }
    }
}

/* Airfoil (Sec. 4.2 plunging airfoil, analytic cambered stand-in): in the
 * chord frame (xi along the chord from the leading edge, eta normal to it, both
 * in chords) a point is inside when 0 <= xi <= 1 and |eta - y_c(xi)| < t(xi),
 * y_c the camber line of the four-digit form and t the half thickness. */
static double camber(const orc_body *b, double xi)
{
    double m = b->camber_m, p = b->camber_p;
    if (xi < p) return m / (p * p) * (2.0 * p * xi - xi * xi);
    return m / ((1.0 - p) * (1.0 - p)) * ((1.0 - 2.0 * p) + 2.0 * p * xi - xi * xi);
}

static double half_thickness(const orc_body *b, double xi)
{
    const double *a = b->thick;
    return a[0] * sqrt(xi) + xi * (a[1] + xi * (a[2] + xi * (a[3] + xi * a[4])));
}

static int inside_airfoil(const orc_body *b, double x, double y)
{
    double dx = x - b->X[0], dy = y - b->X[1];
    double xi = (dx * b->ca - dy * b->sa) / b->chord;
    double eta = (dx * b->sa + dy * b->ca) / b->chord;
    if (xi < 0.0 || xi > 1.0) return 0;
    return fabs(eta - camber(b, xi)) < half_thickness(b, xi);
}


/* Anguilliform swimmer (Sec. 4.3).  Lateral midline displacement at arc
 * position s and time t:
 *   y(s,t) = r(t) a L (s/L + 0.03125)/1.03125 sin(2 pi (s/lambda - t/T)),
 * with the ramp r(t) = (1 - cos(pi t/T))/2 for 0 <= t <= T, 1 after it, 0
 * before t = 0 (when enabled; 1 otherwise).  Readings: the cross sections stay
 * normal to x and s is measured along x from the head (no arc-length
 * correction); the body translates only along x. */
static double midline(const orc_body *b, double s, double t)
{
    double r = 1.0;
    if (b->wave_ramp) {
        if (t < 0.0) r = 0.0;
        else if (t < b->wave_period) r = 0.5 * (1.0 - cos(ORC_PI * t / b->wave_period));
    }
    double A = b->wave_amp * b->length * (s / b->length + 0.03125) / 1.03125;
    return r * (A * sin(2.0 * ORC_PI * (s / b->wave_length - t / b->wave_period)));
}

/* Velocity of the body material at arc position s at the current pose:
 * translation U plus the midline velocity by the central difference
 * (y(s, t+1) - y(s, t-1)) / 2 (Sec. 4.3: finite differences of the given
 * deformation). */
static void body_field_velocity(const orc_body *b, double s, double *v)
{
    v[0] = b->U[0];
    v[1] = b->U[1] + (midline(b, s, b->t + 1.0) - midline(b, s, b->t - 1.0)) / 2.0;
    v[2] = b->U[2];
}

/* Free in y or in yaw: the centre-of-mass frame. */
static int com_frame(const orc_body *b) { return (b->free_motion & 6) != 0; }

/* Body-frame position of vertex v at time t: (s, y(s,t) + dy, dz). */
static void body_point(const orc_body *b, int v, double t, double *q)
{
    const double *r = b->mesh_rest + 3 * v;
    q[0] = r[0];
    q[1] = midline(b, r[0], t) + r[1];
    q[2] = r[2];
}

/* Volume, centre of mass (x, y) and moment of inertia about the vertical axis
 * through it of the closed mesh at time t, in the body frame, for density
 * rho.  Divergence theorem: for a polynomial p with F . e_a = P, dP/da = p,
 * the volume integral of p is the sum over triangles of the integral of P n_a;
 * over a flat triangle the mean of x^k is h_k(x0, x1, x2) / C(k+2, 2) (h_k the
 * complete homogeneous symmetric polynomial of the vertex coordinates), and
 * n_a dA integrates to d_a / 2 with d = (v1 - v0) x (v2 - v0).  Hence
 *   V = sum d_x h1(x)/6,  int x = sum d_x h2(x)/24,  int x^2 = sum d_x h3(x)/60,
 * and likewise for y. */
static void mesh_mass(const orc_body *b, double t, double rho, double *V, double *cx, double *cy, double *Izz)
{
    double v0 = 0, sx = 0, sy = 0, sxx = 0, syy = 0;
    for (int k = 0; k < b->n_triangles; ++k) {
        const int *tr = b->mesh_tris + 3 * k;
        double P[3][3];
        for (int m = 0; m < 3; ++m) body_point(b, tr[m], t, P[m]);
        double e1[3], e2[3], d[3];
        for (int a = 0; a < 3; ++a) { e1[a] = P[1][a] - P[0][a]; e2[a] = P[2][a] - P[0][a]; }
        d[0] = e1[1] * e2[2] - e1[2] * e2[1];
        d[1] = e1[2] * e2[0] - e1[0] * e2[2];
        d[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double h[2][4];
        for (int a = 0; a < 2; ++a) {
            const double x0 = P[0][a], x1 = P[1][a], x2 = P[2][a];
            h[a][1] = x0 + x1 + x2;
            h[a][2] = x0 * x0 + x1 * x1 + x2 * x2 + x0 * x1 + x0 * x2 + x1 * x2;
            h[a][3] = x0 * x0 * x0 + x1 * x1 * x1 + x2 * x2 * x2 + x0 * x0 * (x1 + x2) + x1 * x1 * (x0 + x2) +
                      x2 * x2 * (x0 + x1) + x0 * x1 * x2;
        }
        v0 += d[0] * h[0][1] / 6.0;
        sx += d[0] * h[0][2] / 24.0;
        sy += d[1] * h[1][2] / 24.0;
        sxx += d[0] * h[0][3] / 60.0;
        syy += d[1] * h[1][3] / 60.0;
    }
    *V = v0;
    *cx = sx / v0;
    *cy = sy / v0;
    *Izz = rho * ((sxx + syy) - v0 * (*cx * *cx + *cy * *cy));
}

/* Body-frame velocity of a material point at arc position s: the midline's
 * central difference (Sec. 4.3, finite differences of the given deformation). */
static double midline_rate(const orc_body *b, double s)
{
    return (midline(b, s, b->t + 1.0) - midline(b, s, b->t - 1.0)) / 2.0;
}

/* Velocity of the body material at world point p (current pose).  Head frame:
 * U + (0, y_rate(s), 0) at s = p_x - X0 (clamped to [0, L]).  Centre-of-mass
 * frame: U + omega e_z x (p - X) + R(psi) ((0, y_rate(s), 0) - c_dot), with s
 * the body-frame abscissa of p. */
static void material_velocity(const orc_body *b, const double *p, double *v)
{
    if (!com_frame(b)) {
        double s = p[0] - b->X[0];
        body_field_velocity(b, s < 0.0 ? 0.0 : s > b->length ? b->length : s, v);
        return;
    }
    const double cs = cos(b->psi), sn = sin(b->psi);
    const double rx = p[0] - b->X[0], ry = p[1] - b->X[1];
    double s = cs * rx + sn * ry + b->com[0];
    s = s < 0.0 ? 0.0 : s > b->length ? b->length : s;
    const double wx = -b->com_dot[0], wy = midline_rate(b, s) - b->com_dot[1];
    v[0] = b->U[0] - b->omega * ry + (cs * wx - sn * wy);
    v[1] = b->U[1] + b->omega * rx + (sn * wx + cs * wy);
    v[2] = b->U[2];
}

/* Vertex positions and velocities of the mesh at the current pose.  Head
 * frame: x = X0 + s, y = (X1 + y(s,t)) + dy, z = X2 + dz.  Centre-of-mass
 * frame: X + R(psi) (b - c(t)) with b the body-frame point and c(t) the centre
 * of mass of the mesh at t, and the velocity of material_velocity. */
static void mesh_pose(orc_ctx *c)
{
    orc_body *b = &c->b;
    for (int a = 0; a < 3; ++a) { c->box_lo[a] = INFINITY; c->box_hi[a] = -INFINITY; }
    const int cf = com_frame(b);
    if (cf) {
        double V, cx, cy, I, Vp, cxp, cyp, Ip, Vm, cxm, cym, Im;
        double rho = 1.0;
        mesh_mass(b, b->t, 1.0, &V, &cx, &cy, &I);
        rho = b->mass / V;
        mesh_mass(b, b->t + 1.0, rho, &Vp, &cxp, &cyp, &Ip);
        mesh_mass(b, b->t - 1.0, rho, &Vm, &cxm, &cym, &Im);
        b->com[0] = cx;
        b->com[1] = cy;
        b->com_dot[0] = (cxp - cxm) / 2.0;
        b->com_dot[1] = (cyp - cym) / 2.0;
        b->Izz = rho * I;
    }
    const double cs = cos(b->psi), sn = sin(b->psi);
    for (int v = 0; v < b->n_vertices; ++v) {
        const double *r = b->mesh_rest + 3 * v;
        double *p = c->vpos + 3 * v;
        if (cf) {
            double q[3];
            body_point(b, v, b->t, q);
            const double qx = q[0] - b->com[0], qy = q[1] - b->com[1];
            p[0] = b->X[0] + (cs * qx - sn * qy);
            p[1] = b->X[1] + (sn * qx + cs * qy);
            p[2] = b->X[2] + q[2];
            material_velocity(b, p, c->vvel + 3 * v);
        } else {
            p[0] = b->X[0] + r[0];
            p[1] = (b->X[1] + midline(b, r[0], b->t)) + r[1];
            p[2] = b->X[2] + r[2];
            body_field_velocity(b, r[0], c->vvel + 3 * v);
        }
        for (int a = 0; a < 3; ++a) {
            if (p[a] < c->box_lo[a]) c->box_lo[a] = p[a];
            if (p[a] > c->box_hi[a]) c->box_hi[a] = p[a];
        }
    }
    const int n[3] = {c->p.nx, c->p.ny, c->p.nz};
    for (int a = 0; a < 3; ++a)
        if (c->box_lo[a] < 2.0 || c->box_hi[a] > n[a] - 3.0) c->error = 1;
}

/* Edge value of the (y, z) projection of the directed edge u -> v at (y, z):
 * the 2-D cross product (P_b - P_a) x (p - P_a), taken with the lower vertex
 * index as a, so the two triangles sharing an edge get exactly opposite
 * values; its sign, with zero counted as positive in that lower-index
 * direction, is returned. */
static int edge_value(const double *P, int u, int v, double y, double z, double *e)
{
    int a = u < v ? u : v, bb = u < v ? v : u;
    const double *A = P + 3 * a, *B = P + 3 * bb;
    double val = (B[1] - A[1]) * (z - A[2]) - (B[2] - A[2]) * (y - A[1]);
    int sg = val >= 0.0 ? 1 : -1;
    if (u > v) { val = -val; sg = -sg; }
    *e = val;
    return sg;
}

/* A node is inside the closed mesh when the ray from it along +x crosses the
 * surface an odd number of times.  The ray meets triangle (A, B, C) when the
 * three edge values of its (y, z) projection share one sign; the crossing is
 * at x = (e_BC x_A + e_CA x_B + e_AB x_C) / (e_BC + e_CA + e_AB) (barycentric
 * weights of the projection) and counts when it lies strictly beyond x. */
static int inside_mesh(const orc_ctx *c, double x, double y, double z)
{
    if (x < c->box_lo[0] || x > c->box_hi[0] || y < c->box_lo[1] || y > c->box_hi[1] ||
        z < c->box_lo[2] || z > c->box_hi[2])
        return 0;
    const orc_body *b = &c->b;
    const double *P = c->vpos;
    int crossings = 0;
    for (int k = 0; k < b->n_triangles; ++k) {
        const int *t = b->mesh_tris + 3 * k;
        double e0, e1, e2;
        int s0 = edge_value(P, t[1], t[2], y, z, &e0);
        int s1 = edge_value(P, t[2], t[0], y, z, &e1);
        int s2 = edge_value(P, t[0], t[1], y, z, &e2);
        if (s0 != s1 || s1 != s2) continue;
        double den = (e0 + e1) + e2;
        if (den == 0.0) continue;
        double xc = ((e0 * P[3 * t[0]] + e1 * P[3 * t[1]]) + e2 * P[3 * t[2]]) / den;
        if (xc > x) crossings++;
    }
    return crossings & 1;
}

static double det3(const double *a, const double *b, const double *d)
{
    return a[0] * (b[1] * d[2] - b[2] * d[1]) - a[1] * (b[0] * d[2] - b[2] * d[0])
         + a[2] * (b[0] * d[1] - b[1] * d[0]);
}

/* Link of boundary node x_b towards the solid node x_b - c: the first point
 * x_b - s c, s in [0, 1], on any triangle.  Each triangle A + u (B - A) +
 * v (C - A) is solved for (u, v, s) by Cramer's rule and hit when u, v >= 0,
 * u + v <= 1.  The wall velocity is the barycentric interpolation of the
 * vertex velocities at the hit (Sec. 4.3).  Reading: a link that meets no
 * triangle (only possible through round-off at an edge) takes q = 1/2 and the
 * body velocity at the link's midpoint. */
static double mesh_link(const orc_ctx *c, double x, double y, double z, const int *ci, double *uw)
{
    const orc_body *b = &c->b;
    const double *P = c->vpos;
    const double cv[3] = {ci[0], ci[1], ci[2]};
    double best = INFINITY;
    for (int k = 0; k < b->n_triangles; ++k) {
        const int *t = b->mesh_tris + 3 * k;
        const double *A = P + 3 * t[0], *B = P + 3 * t[1], *C3 = P + 3 * t[2];
        double e1[3], e2[3], r[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = B[a] - A[a];
            e2[a] = C3[a] - A[a];
        }
        r[0] = x - A[0]; r[1] = y - A[1]; r[2] = z - A[2];
        double D = det3(e1, e2, cv);
        if (D == 0.0) continue;
        double u = det3(r, e2, cv) / D;
        double v = det3(e1, r, cv) / D;
        double s = det3(e1, e2, r) / D;
        if (u < 0.0 || v < 0.0 || u + v > 1.0 || s < 0.0 || s > 1.0) continue;
        if (s < best) {
            best = s;
            for (int a = 0; a < 3; ++a)
                uw[a] = (1.0 - u - v) * c->vvel[3 * t[0] + a] + u * c->vvel[3 * t[1] + a]
                      + v * c->vvel[3 * t[2] + a];
        }
    }
    if (best == INFINITY) {
        best = 0.5;
        const double mid[3] = {x - 0.5 * ci[0], y - 0.5 * ci[1], z - 0.5 * ci[2]};
        material_velocity(b, mid, uw);
    }
    return best;
}

static int inside_body(const orc_ctx *c, double x, double y, double z)
{
    const orc_body *b = &c->b;
    if (b->kind == BODY_MESH) return inside_mesh(c, x, y, z);
    if (b->kind == BODY_AIRFOIL) return inside_airfoil(b, x, y);
    if (b->kind == BODY_SPHERE) {
        double d[3];
        sphere_offset(c, x, y, z, d);
        return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < b->R * b->R;
    }
    if (b->kind == BODY_PLANES) return y < b->y_lo || y > b->y_hi;
    return 0;
}

/* Fraction q of the link from fluid x_b towards the solid node x_b - c where the
 * wall is crossed: the wall point is x_w = x_b - q c, q in (0, 1]. */
static double link_q(const orc_ctx *c, double x, double y, double z, const int *ci)
{
    const orc_body *b = &c->b;
    if (b->kind == BODY_SPHERE) {
        double d[3];
        sphere_offset(c, x, y, z, d);
        double cc = ci[0] * ci[0] + ci[1] * ci[1] + ci[2] * ci[2];
        double cd = ci[0] * d[0] + ci[1] * d[1] + ci[2] * d[2];
        double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        /* |d - s c|^2 = R^2, smaller root */
        double disc = cd * cd - cc * (dd - b->R * b->R);
        return (cd - sqrt(disc)) / cc;
    }
    if (b->kind == BODY_PLANES) {
        if (y - ci[1] < b->y_lo) return (y - b->y_lo) / ci[1];
        return (b->y_hi - y) / (-ci[1]);
    }
    if (b->kind == BODY_AIRFOIL) {
        /* reading: the crossing of the link x_b - s c (s in [0,1]) by bisection
         * on the inside test, 50 halvings */
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 50; ++it) {
            double mid = 0.5 * (lo + hi);
            if (inside_airfoil(b, x - mid * ci[0], y - mid * ci[1])) hi = mid;
            else lo = mid;
        }
        return 0.5 * (lo + hi);
    }
    return 0.5;
}

/* Velocity of the body surface at the wall point (translation only: the
 * sphere and the channel walls do not rotate; the swimmer's material velocity
 * at the point's arc position). */
static void wall_velocity(const orc_body *b, double x_solid, double y_solid, double z_solid, double *uw)
{
    if (b->kind == BODY_MESH) {
        const double p[3] = {x_solid, y_solid, z_solid};
        material_velocity(b, p, uw);
        return;
    }
    if (b->kind == BODY_PLANES) {
        const double *v = y_solid < b->y_lo ? b->U_lo : b->U_hi;
        for (int a = 0; a < 3; ++a) uw[a] = v[a];
        return;
    }
    for (int a = 0; a < 3; ++a) uw[a] = b->U[a];
}

/* Source of the pull F_i(x) = f'_i(x - c_i).  Box faces (the paper gives none):
 * per axis, a source outside [0,n) wraps on a periodic face, is clamped to the
 * face (zero-gradient) on an outflow face, and is marked wall / equilibrium on
 * those faces.  Precedence when several axes leave the box: wall, then
 * equilibrium, then the clamped/wrapped interior source.
 * Returns 0 (interior source in s[]), 1 (wall), 2 (equilibrium). */
static int pull_source(const orc_ctx *c, int x, int y, int z, int i, int *s)
{
    int pos[3] = {x - C[i][0], y - C[i][1], z - C[i][2]};
    int n[3] = {c->p.nx, c->p.ny, c->p.nz};
    int wall = 0, eq = 0;
    for (int a = 0; a < 3; ++a) {
        int face = -1;
        if (pos[a] < 0) face = c->p.face[2 * a];
        else if (pos[a] >= n[a]) face = c->p.face[2 * a + 1];
        if (face < 0) continue;
        if (face == FACE_PERIODIC) pos[a] = (pos[a] + n[a]) % n[a];
        else if (face == FACE_OUTFLOW) pos[a] = pos[a] < 0 ? 0 : n[a] - 1;
        else if (face == FACE_WALL) wall = 1;
        else eq = 1;
    }
    if (wall) return 1;
    if (eq) return 2;
    for (int a = 0; a < 3; ++a) s[a] = pos[a];
    return 0;
}

/* Neighbour position x + d for finite differences and interpolation: wraps on
 * periodic faces, otherwise outside the box is unavailable (returns -1). */
static long neighbour(const orc_ctx *c, int x, int y, int z, int dx, int dy, int dz)
{
    int pos[3] = {x + dx, y + dy, z + dz};
    int n[3] = {c->p.nx, c->p.ny, c->p.nz};
    for (int a = 0; a < 3; ++a) {
        if (pos[a] >= 0 && pos[a] < n[a]) continue;
        int face = pos[a] < 0 ? c->p.face[2 * a] : c->p.face[2 * a + 1];
        if (face != FACE_PERIODIC) return -1;
        pos[a] = (pos[a] + n[a]) % n[a];
    }
    return nid(c, pos[0], pos[1], pos[2]);
}

static void node_moments(const orc_ctx *c, const double *f, long n, double *rho, double *u)
{
    double g[Q];
    for (int i = 0; i < Q; ++i) g[i] = f[i * c->N + n];
    moments(g, rho, u);
}

/* Velocity gradient by finite differences of the previous-step velocities
 * (Sec. 3: "computing grad u using a finite difference scheme and the velocity
 * values from the previous time step").  Reading: central difference where
 * both face neighbours are available, first-order one-sided where one is,
 * zero where neither is.  u_centre is the velocity used at the node itself. */
static void velocity_gradient(const orc_ctx *c, int x, int y, int z, const double *u_centre,
                              const uint8_t *solid, double dudx[3][3])
{
    for (int b = 0; b < 3; ++b) {
        int e[3] = {0, 0, 0};
        e[b] = 1;
        long np = neighbour(c, x, y, z, e[0], e[1], e[2]);
        long nm = neighbour(c, x, y, z, -e[0], -e[1], -e[2]);
        int okp = np >= 0 && !solid[np];
        int okm = nm >= 0 && !solid[nm];
        double up[3] = {0, 0, 0}, um[3] = {0, 0, 0}, r;
        if (okp) node_moments(c, c->fa, np, &r, up);
        if (okm) node_moments(c, c->fa, nm, &r, um);
        for (int a = 0; a < 3; ++a) {
            if (okp && okm) dudx[a][b] = 0.5 * (up[a] - um[a]);
            else if (okp) dudx[a][b] = up[a] - u_centre[a];
            else if (okm) dudx[a][b] = u_centre[a] - um[a];
            else dudx[a][b] = 0.0;
        }
    }
}

/* Refill of a node uncovered by the moving body (Sec. 3): the Grad
 * distribution with the wall velocity, a local density average and the pressure
 * tensor evaluated as for the wall boundary.  Readings: the density average is
 * the mean density of the neighbours among the 26 that were fluid at t (rho0 if
 * none); the velocity is the body velocity at the node; the gradient uses the
 * node's own wall velocity at its centre and the neighbours fluid at t. */
static void refill(orc_ctx *c, int x, int y, int z)
{
    long n = nid(c, x, y, z);
    double rsum = 0;
    int cnt = 0;
    for (int i = 0; i < Q; ++i) {
        if (i == 13) continue;
        long m = neighbour(c, x, y, z, C[i][0], C[i][1], C[i][2]);
        if (m < 0 || c->solid0[m]) continue;
        double r, u[3];
        node_moments(c, c->fa, m, &r, u);
        rsum += r;
        cnt++;
    }
    double rho = cnt ? rsum / cnt : c->p.rho0;
    double uw[3];
    wall_velocity(&c->b, (double)x, (double)y, (double)z, uw);
    double dudx[3][3], Pi[9], f[Q];
    velocity_gradient(c, x, y, z, uw, c->solid0, dudx);
    pressure_tensor(rho, uw, dudx, c->p.beta, Pi);
    orc_grad(rho, uw, Pi, f);
    for (int i = 0; i < Q; ++i) c->fa[i * c->N + n] = f[i];
    c->n_refill++;
}

/* Pull of fluid node (x,y,z) for the step to t+1 (Eq. kineticEq):
 * F_i = f'_i(x - c_i, t) from the box rules; missing[i] = 1 where the source
 * is solid at t+1 (then F_i = 0 until the wall boundary fills it).  Returns
 * the number of missing directions. */
static int gather_node(const orc_ctx *c, int x, int y, int z, double *Fi, int *missing)
{
    const long N = c->N;
    const long n = nid(c, x, y, z);
    int nmiss = 0;
    for (int i = 0; i < Q; ++i) {
        int s[3];
        int kind = pull_source(c, x, y, z, i, s);
        missing[i] = 0;
        if (kind == 1) Fi[i] = c->fa[opp(i) * N + n];         /* halfway bounce-back */
        else if (kind == 2) Fi[i] = c->feq_face[i];           /* equilibrium face */
        else {
            long m = nid(c, s[0], s[1], s[2]);
            if (c->solid1[m]) { missing[i] = 1; nmiss++; Fi[i] = 0.0; }
            else Fi[i] = c->fa[i * N + m];
        }
    }
    return nmiss;
}

/* Targets of the Grad boundary at x_b (Sec. 3), D = {i : x_b - c_i solid at
 * t+1}.  For each missing i: the link fraction q_i and the wall velocity
 * u_w,i; the static density sums the known pulls and the bounce-back
 * populations, the dynamic density the wall motion, and the target velocity
 * averages the interpolations between the wall point and the fluid node
 * x_b + c_i. */
static void wall_targets(const orc_ctx *c, int x, int y, int z, const double *Fi, const int *missing,
                         int nmiss, double *q, double uw[][3], double *rho_stat_out, double *rho_dyn_out,
                         double *utgt)
{
    const long N = c->N;
    const long n = nid(c, x, y, z);
    double rho_stat = 0, rho_dyn = 0;
    for (int a = 0; a < 3; ++a) utgt[a] = 0.0;
    for (int i = 0; i < Q; ++i) {
        if (!missing[i]) { rho_stat += Fi[i]; continue; }
        const int *ci = C[i];
        if (c->b.kind == BODY_MESH) {
            q[i] = mesh_link(c, x, y, z, ci, uw[i]);
        } else {
            q[i] = link_q(c, x, y, z, ci);
            wall_velocity(&c->b, (double)(x - ci[0]), (double)(y - ci[1]), (double)(z - ci[2]), uw[i]);
        }
        /* f^bb_i = f'_{opp i}(x_b, t): the population that left x_b towards
         * the wall and returns reflected (halfway bounce-back). */
        rho_stat += c->fa[opp(i) * N + n];
        /* Reading: rho_dyn uses the reference density rho0. */
        rho_dyn += 6.0 * W[i] * c->p.rho0 * (ci[0] * uw[i][0] + ci[1] * uw[i][1] + ci[2] * uw[i][2]);
        /* target velocity: linear interpolation between the wall point at
         * -q and the fluid node x_f = x_b + c_i at +1, read at x_b.
         * Reading: if x_f is not fluid the term is the wall velocity. */
        long mf = neighbour(c, x, y, z, ci[0], ci[1], ci[2]);
        if (mf >= 0 && !c->solid1[mf]) {
            double rf, uf[3];
            node_moments(c, c->fa, mf, &rf, uf);
            for (int a = 0; a < 3; ++a) utgt[a] += (q[i] * uf[a] + uw[i][a]) / (1.0 + q[i]);
        } else {
            for (int a = 0; a < 3; ++a) utgt[a] += uw[i][a];
        }
    }
    for (int a = 0; a < 3; ++a) utgt[a] /= nmiss;
    *rho_stat_out = rho_stat;
    *rho_dyn_out = rho_dyn;
}

/* Post-collision state of fluid node (x,y,z) at t+1, written to out[27].
 * Adds the node's momentum-exchange force and torque to F, M. */
static void node_update(orc_ctx *c, int x, int y, int z, double *out, double *F, double *M)
{
    const long N = c->N;
    const long n = nid(c, x, y, z);
    double Fi[Q];
    int missing[Q];
    const int nmiss = gather_node(c, x, y, z, Fi, missing);
    if (nmiss) {
        double q[Q], uw[Q][3];
        double rho_stat, rho_dyn, utgt[3];
        double rb, ub[3];
        node_moments(c, c->fa, n, &rb, ub);
        wall_targets(c, x, y, z, Fi, missing, nmiss, q, uw, &rho_stat, &rho_dyn, utgt);
        double rho = rho_stat + rho_dyn;
        double dudx[3][3], Pi[9], fs[Q];
        velocity_gradient(c, x, y, z, ub, c->solid1, dudx);
        pressure_tensor(rho, utgt, dudx, c->p.beta, Pi);
        orc_grad(rho, utgt, Pi, fs);
        for (int i = 0; i < Q; ++i)
            if (missing[i]) Fi[i] = fs[i];
        /* Galilean-invariant momentum exchange on each link (Sec. 4.1, Wen et
         * al.): the fluid hands the body (c_opp - u_w) f'_opp(x_b, t) and gets
         * back (c_i - u_w) F_i(x_b, t+1).  Torque arm: x_w - X_c. */
        for (int i = 0; i < Q; ++i) {
            if (!missing[i]) continue;
            const int *ci = C[i];
            double fout = c->fa[opp(i) * N + n];
            double dF[3];
            for (int a = 0; a < 3; ++a)
                dF[a] = (-ci[a] - uw[i][a]) * fout - (ci[a] - uw[i][a]) * Fi[i];
            /* torque arm from the body's reference point: sphere centre,
             * airfoil leading edge at z = 0, swimmer head on the centre line,
             * the lattice origin otherwise */
            double r[3];
            if (c->b.kind == BODY_SPHERE) sphere_offset(c, x, y, z, r);
            else if (c->b.kind == BODY_AIRFOIL) { r[0] = x - c->b.X[0]; r[1] = y - c->b.X[1]; r[2] = z; }
            else if (c->b.kind == BODY_MESH) { r[0] = x - c->b.X[0]; r[1] = y - c->b.X[1]; r[2] = z - c->b.X[2]; }
            else { r[0] = x; r[1] = y; r[2] = z; }
            for (int a = 0; a < 3; ++a) r[a] -= q[i] * ci[a];
            F[0] += dF[0]; F[1] += dF[1]; F[2] += dF[2];
            M[0] += r[1] * dF[2] - r[2] * dF[1];
            M[1] += r[2] * dF[0] - r[0] * dF[2];
            M[2] += r[0] * dF[1] - r[1] * dF[0];
            c->n_links++;
        }
        c->n_boundary++;
    }
    orc_collide(Fi, c->p.beta, c->p.gamma_mode, out);
}

/* ------------------------------------------------------------------ public */
orc_ctx *orc_create(const orc_params *p, const orc_body *b)
{
    tables();
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (!c) return NULL;
    c->p = *p;
    c->b = *b;
    c->N = (long)p->nx * p->ny * p->nz;
    c->own_zlo = 0;
    c->own_zhi = p->nz;
    c->fa = (double *)calloc((size_t)Q * c->N, sizeof(double));
    c->solid0 = (uint8_t *)calloc((size_t)c->N, 1);
    c->solid1 = (uint8_t *)calloc((size_t)c->N, 1);
    if (!c->fa || !c->solid0 || !c->solid1) return NULL;
    if (b->kind == BODY_MESH) {
        c->vpos = (double *)calloc((size_t)3 * b->n_vertices, sizeof(double));
        c->vvel = (double *)calloc((size_t)3 * b->n_vertices, sizeof(double));
        if (!c->vpos || !c->vvel) return NULL;
        mesh_pose(c);
        if (com_frame(&c->b)) c->b.Iw = c->b.Izz * c->b.omega;
    }
    orc_feq(p->rho0, p->u_face, c->feq_face);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x)
                c->solid0[nid(c, x, y, z)] = (uint8_t)inside_body(c, x, y, z);
    return c;
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free(c->fa); free(c->fb); free(c->solid0); free(c->solid1); free(c->vpos); free(c->vvel); free(c);
}

void orc_set_f(orc_ctx *c, const double *f) { memcpy(c->fa, f, sizeof(double) * Q * c->N); }
void orc_get_f(const orc_ctx *c, double *f) { memcpy(f, c->fa, sizeof(double) * Q * c->N); }
void orc_get_solid(const orc_ctx *c, uint8_t *s) { memcpy(s, c->solid0, (size_t)c->N); }
void orc_get_body(const orc_ctx *c, orc_body *b) { *b = c->b; }
void orc_set_body(orc_ctx *c, const orc_body *b)
{
    c->b = *b;
    if (b->kind == BODY_MESH && c->vpos) mesh_pose(c);
}
/* Vertex positions and velocities of the mesh at the current pose (3 n_vertices each). */
void orc_mesh_pose(const orc_ctx *c, double *pos, double *vel)
{
    memcpy(pos, c->vpos, sizeof(double) * 3 * c->b.n_vertices);
    memcpy(vel, c->vvel, sizeof(double) * 3 * c->b.n_vertices);
}

/* Mass properties of the mesh at time t in the body frame for unit density:
 * out = (V, cx, cy, Izz). */
void orc_mesh_mass(const orc_ctx *c, double t, double *out)
{
    mesh_mass(&c->b, t, 1.0, out, out + 1, out + 2, out + 3);
}

/* Link fraction q and wall velocity of the link from (x, y, z) along -c_i at
 * the current pose of the mesh. */
double orc_mesh_link(const orc_ctx *c, int x, int y, int z, int i, double *uw)
{
    return mesh_link(c, x, y, z, C[i], uw);
}

/* Link fraction q and wall velocity of the link from fluid node (x, y, z) to
 * the solid node (x, y, z) - c_i at the current pose, for any body: the values
 * the boundary step takes. */
double orc_link(const orc_ctx *c, int x, int y, int z, int i, double *uw)
{
    const int *ci = C[i];
    if (c->b.kind == BODY_MESH) return mesh_link(c, x, y, z, ci, uw);
    wall_velocity(&c->b, (double)(x - ci[0]), (double)(y - ci[1]), (double)(z - ci[2]), uw);
    return link_q(c, x, y, z, ci);
}

/* Restricts the force and torque sums of later steps to the boundary nodes of
 * the z layers [z_lo, z_hi) (one slab of a decomposed box); every node is
 * still updated. */
void orc_set_owned_z(orc_ctx *c, int z_lo, int z_hi)
{
    c->own_zlo = z_lo;
    c->own_zhi = z_hi;
}

/* Places the box as a slab of a box periodic in z with `period` layers: layer
 * k sits at z = (k + origin) mod period for the sphere's geometry, nearest
 * image and centre wrap, so a slab sees the sphere exactly as the whole box
 * does.  Recomputes the solid marks of the current pose. */
void orc_set_z_frame(orc_ctx *c, int origin, int period)
{
    c->zf_origin = origin;
    c->zf_period = period;
    const orc_params *p = &c->p;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x)
                c->solid0[nid(c, x, y, z)] = (uint8_t)inside_body(c, x, y, z);
}

long orc_counter(const orc_ctx *c, int which)
{
    return which == 0 ? c->step : which == 1 ? c->n_boundary : which == 2 ? c->n_links
         : which == 3 ? c->n_refill : c->error;
}

/* Initial state f = f^eq(rho(x), u(x)) + amp * W_i * xi_i(x) from host fields
 * rho[N], u[3N] (node-major), xi[27N] (direction-major; NULL for none). */
void orc_init_state(orc_ctx *c, const double *rho, const double *u, const double *xi, double amp)
{
    double feq[Q];
    for (long n = 0; n < c->N; ++n) {
        double un[3] = {u[3 * n], u[3 * n + 1], u[3 * n + 2]};
        orc_feq(rho[n], un, feq);
        for (int i = 0; i < Q; ++i)
            c->fa[i * c->N + n] = feq[i] + (xi ? amp * W[i] * xi[i * c->N + n] : 0.0);
    }
}

/* Newton's equations of the sphere (Sec. 4.1) by explicit Euler:
 * X^{t+1} = X^t + U^t,  U^{t+1} = U^t + F^t / m_s + (1 - rho_f/rho_s) g.
 * On periodic axes the centre is wrapped back into [0, n). */
static void body_update(orc_ctx *c)
{
    orc_body *b = &c->b;
    if (b->kind == BODY_AIRFOIL) {
        /* prescribed plunge (Sec. 4.2): y_le(t) = y_base + A sin(w t) */
        b->t = b->t + 1.0;
        b->X[1] = b->y_base + b->h_amp * sin(b->h_omega * b->t);
        b->U[1] = b->h_amp * b->h_omega * cos(b->h_omega * b->t);
        return;
    }
    if (b->kind == BODY_MESH) {
        /* Sec. 4.3: Newton's equations by explicit Euler on the free degrees
         * of freedom (bit 1 x, bit 2 y, bit 4 yaw): X += U, U += F / m;
         * psi += omega, (I omega) += M_z with I of the new pose (the yaw
         * equation d(I omega)/dt = M as printed); then the new pose */
        b->t = b->t + 1.0;
        for (int a = 0; a < 2; ++a)
            if (b->free_motion & (1 << a)) {
                b->X[a] = b->X[a] + b->U[a];
                b->U[a] = b->U[a] + b->F[a] / b->mass;
            }
        if (b->free_motion & 4) {
            double V, cx, cy, I;
            mesh_mass(b, b->t, 1.0, &V, &cx, &cy, &I);
            b->psi = b->psi + b->omega;
            b->Iw = b->Iw + b->M[2];
            b->omega = b->Iw / (b->mass / V * I);
        }
        mesh_pose(c);
        return;
    }
    if (!b->free_motion) return;
    int n[3] = {c->p.nx, c->p.ny, c->p.nz};
    int per[3] = {c->p.face[0] == FACE_PERIODIC, c->p.face[2] == FACE_PERIODIC, c->p.face[4] == FACE_PERIODIC};
    if (c->zf_period > 0) {
        n[2] = c->zf_period;
        per[2] = 1;
    }
    for (int a = 0; a < 3; ++a) {
        double acc = b->F[a] / b->mass + (1.0 - 1.0 / b->rho_ratio) * b->g[a];
        b->X[a] = b->X[a] + b->U[a];
        b->U[a] = b->U[a] + acc;
        if (per[a]) {
            if (b->X[a] >= n[a]) b->X[a] = b->X[a] - n[a];
            else if (b->X[a] < 0.0) b->X[a] = b->X[a] + n[a];
        }
    }
}

/* Geometry and refill for the step t -> t+1: moves the body, marks solid
 * nodes at t+1 and refills uncovered nodes in the current state. */
static void step_prepare(orc_ctx *c)
{
    body_update(c);
    const orc_params *p = &c->p;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x)
                c->solid1[nid(c, x, y, z)] = (uint8_t)inside_body(c, x, y, z);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = nid(c, x, y, z);
                if (c->solid0[n] && !c->solid1[n]) refill(c, x, y, z);
            }
}

/* One or more full steps t -> t+1 (stream + collide with Grad boundaries and
 * momentum exchange).  Solid nodes carry their state unchanged. */
int orc_step(orc_ctx *c, int nsteps)
{
    const orc_params *p = &c->p;
    if (!c->fb) {
        c->fb = (double *)calloc((size_t)Q * c->N, sizeof(double));
        if (!c->fb) return 1;
    }
    for (int s = 0; s < nsteps; ++s) {
        step_prepare(c);
        double F[3] = {0, 0, 0}, M[3] = {0, 0, 0}, out[Q];
        double Fx[3] = {0, 0, 0}, Mx[3] = {0, 0, 0}; /* sums outside the owned layers, dropped */
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long n = nid(c, x, y, z);
                    if (c->solid1[n]) {
                        for (int i = 0; i < Q; ++i) c->fb[i * c->N + n] = c->fa[i * c->N + n];
                        continue;
                    }
                    const int own = z >= c->own_zlo && z < c->own_zhi;
                    node_update(c, x, y, z, out, own ? F : Fx, own ? M : Mx);
                    for (int i = 0; i < Q; ++i) c->fb[i * c->N + n] = out[i];
                }
        double *t = c->fa; c->fa = c->fb; c->fb = t;
        uint8_t *u = c->solid0; c->solid0 = c->solid1; c->solid1 = u;
        for (int a = 0; a < 3; ++a) { c->b.F[a] = F[a]; c->b.M[a] = M[a]; }
        c->step++;
    }
    return 0;
}

/* One step evaluated only at the listed nodes: moves the body, updates the
 * solid marks, refills, and writes the new post-collision populations of the
 * listed nodes to out[k*27 + i] (NaN for nodes solid at t+1).  The state is
 * left as after the refill, not advanced. */
int orc_step_sampled(orc_ctx *c, long nsample, const long *nodes, double *out)
{
    step_prepare(c);
    const orc_params *p = &c->p;
    double F[3] = {0, 0, 0}, M[3] = {0, 0, 0};
    for (long k = 0; k < nsample; ++k) {
        long n = nodes[k];
        int x = (int)(n % p->nx), y = (int)((n / p->nx) % p->ny), z = (int)(n / ((long)p->nx * p->ny));
        if (c->solid1[n]) {
            for (int i = 0; i < Q; ++i) out[k * Q + i] = NAN;
            continue;
        }
        node_update(c, x, y, z, out + k * Q, F, M);
    }
    return 0;
}

/* The Grad boundary's targets for one step evaluated at the listed nodes:
 * moves the body, updates the solid marks and refills as orc_step does, then
 * writes per node out[k*7 + 0..6] = (number of missing directions, static
 * density, dynamic density, target density, target velocity), with the
 * densities and velocity NaN where the node is no boundary node at t+1.  The
 * state is left as after the refill, not advanced. */
int orc_wall_targets_sampled(orc_ctx *c, long nsample, const long *nodes, double *out)
{
    step_prepare(c);
    const orc_params *p = &c->p;
    for (long k = 0; k < nsample; ++k) {
        long n = nodes[k];
        int x = (int)(n % p->nx), y = (int)((n / p->nx) % p->ny), z = (int)(n / ((long)p->nx * p->ny));
        double *o = out + k * 7;
        for (int j = 0; j < 7; ++j) o[j] = NAN;
        o[0] = 0.0;
        if (c->solid1[n]) continue;
        double Fi[Q];
        int missing[Q];
        const int nmiss = gather_node(c, x, y, z, Fi, missing);
        if (!nmiss) continue;
        double q[Q], uw[Q][3], rho_stat, rho_dyn, utgt[3];
        wall_targets(c, x, y, z, Fi, missing, nmiss, q, uw, &rho_stat, &rho_dyn, utgt);
        o[0] = nmiss;
        o[1] = rho_stat;
        o[2] = rho_dyn;
        o[3] = rho_stat + rho_dyn;
        for (int a = 0; a < 3; ++a) o[4 + a] = utgt[a];
    }
    return 0;
}

/* Global sums over fluid nodes: mass, momentum (3), kinetic energy. */
void orc_totals(const orc_ctx *c, double *out)
{
    for (int k = 0; k < 5; ++k) out[k] = 0;
    for (long n = 0; n < c->N; ++n) {
        if (c->solid0[n]) continue;
        double r, u[3];
        node_moments(c, c->fa, n, &r, u);
        out[0] += r;
        for (int a = 0; a < 3; ++a) out[1 + a] += r * u[a];
        out[4] += 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    }
}

/* ------------------------------------------------ two-level block refinement */
/* Sec. 4.2 runs the airfoil on a grid with two levels of resolution and cites
 * its refinement algorithm without stating it.  Readings (the paper is silent
 * on every one of them):
 *  - one fine block of ratio 2 inside the coarse lattice, vertex-coincident:
 *    fine node j (per axis) sits at coarse coordinate lo + j/2, j = 0 .. 2m,
 *    m = hi - lo; the fine lattice holds 2m + 2 nodes per axis, the last one
 *    a pad that no update reads;
 *  - acoustic scaling: the fine level takes two steps of half the coarse time
 *    step; u and rho are the same numbers on both levels and the viscosity in
 *    fine lattice units is twice the coarse one, b_f = b_c / (2 - b_c);
 *  - the fine nodes on the block's surface (some j in {0, 2m}) are not
 *    updated by the fine level: their post-collision state at fine time t' is
 *    the fine collision of a state rebuilt from the coarse pre-collision
 *    moments (rho, u, Pi^neq) at t', taken trilinearly in space from the
 *    coarse nodes of the block's surface and linearly in time;
 *  - the coarse nodes strictly inside the block are not updated by the coarse
 *    level; those one layer inside its surface (the only ones a coarse update
 *    pulls from) take, after the fine level reaches t+1, the coarse collision
 *    of a state rebuilt from the pre-collision moments of the coincident fine
 *    node (fine node 2(X - lo));
 *  - a rebuilt state is the entropic equilibrium (Eq. feq_min) at (rho, u)
 *    plus the second-order Hermite term of Grad's distribution (Eq. grad)
 *    carrying the donor's non-equilibrium pressure tensor Pi^neq = Pi -
 *    Pi(f^eq(rho, u)), rescaled by the ratio of the two levels' relaxation
 *    times times time steps: b_c / (2 b_f) coarse to fine, 2 b_f / b_c fine
 *    to coarse (tau = 1/(2b) in each level's units; Pi^neq ~ tau dt grad u);
 *  - the coarse moments at t = 0 are those of the initial coarse state.
 * A block may also span a whole periodic axis of the coarse box (lo = 0,
 * hi = n on that axis; the paper's airfoil is periodic along its span): along
 * that axis it has no surface, the fine lattice holds 2n nodes with periodic
 * wrap and no pad, and every coarse node along it belongs to the block.  At
 * least one axis must be closed (1 <= lo, hi <= n - 2, hi - lo >= 3).
 * The coarse level may carry a body outside the block (its nodes from lo - 1
 * to hi + 1 must be fluid and no boundary node).  The fine level may carry a
 * body of its own (sphere, airfoil or mesh, in fine lattice units: the fine
 * level steps it like any lattice, two steps per coarse step); along closed
 * axes its solid nodes must stay at least four nodes inside the block's
 * surface (j in [4, 2m - 4]), else the step sets the fine level's error
 * counter. */
typedef struct {
    orc_ctx *c, *f;
    int lo[3], hi[3], m[3];
    int full[3];           /* 1: the block spans this periodic axis */
    int ext[3];            /* coarse box extent per axis: m + 1, or n if full */
    double *Mold, *Mnew;   /* 10 moments per coarse node of the box */
    double s_cf, s_fc;     /* Pi^neq factors coarse -> fine, fine -> coarse */
} orc_refine;

enum { NMOM = 10 };  /* rho, u (3), Pi^neq xx yy zz xy xz yz */

/* index of coarse node X in the block's box (X in the box) */
static long rbox(const orc_refine *r, const int *X)
{
    int b[3];
    for (int a = 0; a < 3; ++a) b[a] = X[a] - r->lo[a];
    return b[0] + (long)r->ext[0] * (b[1] + (long)r->ext[1] * b[2]);
}

/* coarse node X lies in the block's box (both ends of closed axes included) */
static int in_box(const orc_refine *r, const int *X)
{
    for (int a = 0; a < 3; ++a)
        if (!r->full[a] && (X[a] < r->lo[a] || X[a] > r->hi[a])) return 0;
    return 1;
}

/* coarse node X lies strictly inside the block (closed axes strictly
 * between lo and hi; any coordinate along a spanned axis) */
static int in_inside(const orc_refine *r, const int *X)
{
    for (int a = 0; a < 3; ++a)
        if (!r->full[a] && (X[a] <= r->lo[a] || X[a] >= r->hi[a])) return 0;
    return 1;
}

/* fine node j lies on the block's surface (some closed axis at 0 or 2m) */
static int fine_on_surface(const orc_refine *r, const int *j)
{
    for (int a = 0; a < 3; ++a)
        if (!r->full[a] && (j[a] == 0 || j[a] == 2 * r->m[a])) return 1;
    return 0;
}

/* fine node j is updated by the fine level (closed axes 1 <= j < 2m) */
static int fine_inner(const orc_refine *r, const int *j)
{
    for (int a = 0; a < 3; ++a)
        if (!r->full[a] && (j[a] < 1 || j[a] >= 2 * r->m[a])) return 0;
    return 1;
}

/* (rho, u, Pi^neq) of pre-collision populations F. */
static void refine_moments(const double *F, double *M)
{
    double rho, u[3], feq[Q], P[6] = {0, 0, 0, 0, 0, 0};
    moments(F, &rho, u);
    orc_feq(rho, u, feq);
    for (int i = 0; i < Q; ++i) {
        const int *c = C[i];
        double d = F[i] - feq[i];
        P[0] += c[0] * c[0] * d; P[1] += c[1] * c[1] * d; P[2] += c[2] * c[2] * d;
        P[3] += c[0] * c[1] * d; P[4] += c[0] * c[2] * d; P[5] += c[1] * c[2] * d;
    }
    M[0] = rho;
    for (int a = 0; a < 3; ++a) M[1 + a] = u[a];
    for (int k = 0; k < 6; ++k) M[4 + k] = P[k];
}

/* Post-collision state of a receiving node: f^eq(rho, u) + Hermite term of
 * s * Pi^neq, collided with the receiver's b. */
static void refine_rebuild(const double *M, double s, double beta, int mode, double *out)
{
    double u[3] = {M[1], M[2], M[3]}, z[3] = {0, 0, 0}, feq[Q], hn[Q], f[Q];
    double Pn[9] = {s * M[4], s * M[7], s * M[8],
                    s * M[7], s * M[5], s * M[9],
                    s * M[8], s * M[9], s * M[6]};
    orc_feq(M[0], u, feq);
    orc_grad(0.0, z, Pn, hn);  /* W_i (9/2) Pn : (c_i c_i - I/3) */
    for (int i = 0; i < Q; ++i) f[i] = feq[i] + hn[i];
    orc_collide(f, beta, mode, out);
}

/* Fills the fine surface nodes of fine state fs from the coarse moments at
 * (1 - w) Mold + w Mnew. */
static void refine_fill_ghosts(orc_refine *r, double *fs, double w)
{
    orc_ctx *f = r->f;
    int n[3] = {r->c->p.nx, r->c->p.ny, r->c->p.nz};
    for (int jz = 0; jz < f->p.nz; ++jz)
        for (int jy = 0; jy < f->p.ny; ++jy)
            for (int jx = 0; jx < f->p.nx; ++jx) {
                int j[3] = {jx, jy, jz};
                if (!fine_on_surface(r, j)) continue;
                int pad = 0;
                for (int a = 0; a < 3; ++a)
                    if (!r->full[a] && j[a] > 2 * r->m[a]) pad = 1;
                if (pad) continue;
                /* per axis: one coarse node (even j) or the two around it
                 * (the second wrapping on a spanned axis) */
                int X0[3], nk[3];
                for (int a = 0; a < 3; ++a) {
                    X0[a] = r->lo[a] + j[a] / 2;
                    nk[a] = (j[a] & 1) ? 2 : 1;
                }
                double M[NMOM] = {0};
                for (int dz = 0; dz < nk[2]; ++dz)
                    for (int dy = 0; dy < nk[1]; ++dy)
                        for (int dx = 0; dx < nk[0]; ++dx) {
                            double wt = 1.0 / (nk[0] * nk[1] * nk[2]);
                            int X[3] = {X0[0] + dx, X0[1] + dy, X0[2] + dz};
                            for (int a = 0; a < 3; ++a)
                                if (r->full[a] && X[a] >= n[a]) X[a] -= n[a];
                            long b = rbox(r, X);
                            for (int k = 0; k < NMOM; ++k)
                                M[k] += wt * ((1.0 - w) * r->Mold[b * NMOM + k] + w * r->Mnew[b * NMOM + k]);
                        }
                double out[Q];
                refine_rebuild(M, r->s_cf, f->p.beta, f->p.gamma_mode, out);
                long nn = nid(f, jx, jy, jz);
                for (int i = 0; i < Q; ++i) fs[i * f->N + nn] = out[i];
            }
}

/* Creates the fine level of the block [lo, hi] (coarse node coordinates,
 * both ends included; lo = 0, hi = n on a periodic axis the block spans)
 * over coarse level c.  Returns NULL on a bad block. */
orc_refine *orc_refine_create(orc_ctx *c, const int *lo, const int *hi, const orc_body *fine_body)
{
    int n[3] = {c->p.nx, c->p.ny, c->p.nz}, full[3], closed = 0;
    for (int a = 0; a < 3; ++a) {
        full[a] = lo[a] == 0 && hi[a] == n[a] && c->p.face[2 * a] == FACE_PERIODIC;
        if (full[a]) continue;
        closed++;
        if (lo[a] < 1 || hi[a] > n[a] - 2 || hi[a] - lo[a] < 3) return NULL;
    }
    if (!closed) return NULL;
    if (fine_body && fine_body->kind == BODY_PLANES) return NULL;
    orc_refine *r = (orc_refine *)calloc(1, sizeof(orc_refine));
    if (!r) return NULL;
    r->c = c;
    orc_params pf = c->p;
    int nf[3];
    for (int a = 0; a < 3; ++a) {
        r->lo[a] = lo[a];
        r->hi[a] = hi[a];
        r->m[a] = hi[a] - lo[a];
        r->full[a] = full[a];
        r->ext[a] = full[a] ? n[a] : r->m[a] + 1;
        nf[a] = full[a] ? 2 * n[a] : 2 * r->m[a] + 2;
    }
    /* coarse nodes one layer around the block are fluid */
    for (int z = 0; z < n[2]; ++z)
        for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x) {
                int X[3] = {x, y, z}, near = 1;
                for (int a = 0; a < 3; ++a)
                    if (!full[a] && (X[a] < lo[a] - 1 || X[a] > hi[a] + 1)) near = 0;
                if (near && c->solid0[nid(c, x, y, z)]) { free(r); return NULL; }
            }
    pf.nx = nf[0];
    pf.ny = nf[1];
    pf.nz = nf[2];
    for (int k = 0; k < 6; ++k) pf.face[k] = FACE_PERIODIC;
    pf.beta = c->p.beta / (2.0 - c->p.beta);
    orc_body none;
    memset(&none, 0, sizeof(none));
    r->f = orc_create(&pf, fine_body ? fine_body : &none);
    if (!r->f) return NULL;
    long nb = (long)r->ext[0] * r->ext[1] * r->ext[2];
    r->Mold = (double *)calloc((size_t)nb * NMOM, sizeof(double));
    r->Mnew = (double *)calloc((size_t)nb * NMOM, sizeof(double));
    r->f->fb = (double *)calloc((size_t)Q * r->f->N, sizeof(double));
    if (!r->Mold || !r->Mnew || !r->f->fb) return NULL;
    r->s_cf = c->p.beta / (2.0 * pf.beta);
    r->s_fc = 2.0 * pf.beta / c->p.beta;
    return r;
}

orc_ctx *orc_refine_fine(orc_refine *r) { return r->f; }

void orc_refine_destroy(orc_refine *r)
{
    if (!r) return;
    orc_destroy(r->f);
    free(r->Mold);
    free(r->Mnew);
    free(r);
}

/* After both levels hold their initial state: the coarse moments at t = 0
 * (from the coarse populations themselves) and the fine surface from them. */
void orc_refine_init(orc_refine *r)
{
    orc_ctx *c = r->c;
    for (int z = 0; z < c->p.nz; ++z)
        for (int y = 0; y < c->p.ny; ++y)
            for (int x = 0; x < c->p.nx; ++x) {
                int X[3] = {x, y, z};
                if (!in_box(r, X) || in_inside(r, X)) continue;
                double g[Q];
                long n = nid(c, x, y, z);
                for (int i = 0; i < Q; ++i) g[i] = c->fa[i * c->N + n];
                refine_moments(g, r->Mold + rbox(r, X) * NMOM);
            }
    refine_fill_ghosts(r, r->f->fa, 0.0);
}

/* One fine step over the nodes off the block's surface and pad (fa -> fb),
 * with the fine body's geometry, refill, Grad boundary and force as a step
 * of the fine lattice alone takes them. */
static void refine_fine_interior(orc_refine *r)
{
    orc_ctx *f = r->f;
    double out[Q], F[3] = {0, 0, 0}, M[3] = {0, 0, 0};
    step_prepare(f);
    for (int jz = 0; jz < f->p.nz; ++jz)
        for (int jy = 0; jy < f->p.ny; ++jy)
            for (int jx = 0; jx < f->p.nx; ++jx) {
                long n = nid(f, jx, jy, jz);
                int j[3] = {jx, jy, jz};
                int inner = fine_inner(r, j), clear = 1;
                for (int a = 0; a < 3; ++a)
                    if (!r->full[a] && (j[a] < 4 || j[a] > 2 * r->m[a] - 4)) clear = 0;
                if (f->solid1[n] && !clear) f->error = 2;
                if (!inner || f->solid1[n]) {
                    for (int i = 0; i < Q; ++i) f->fb[i * f->N + n] = f->fa[i * f->N + n];
                    continue;
                }
                node_update(f, jx, jy, jz, out, F, M);
                for (int i = 0; i < Q; ++i) f->fb[i * f->N + n] = out[i];
            }
    uint8_t *u = f->solid0; f->solid0 = f->solid1; f->solid1 = u;
    for (int a = 0; a < 3; ++a) { f->b.F[a] = F[a]; f->b.M[a] = M[a]; }
}

/* Coarse step t -> t+1 and two fine steps, as the readings above state. */
int orc_refine_step(orc_refine *r, int nsteps)
{
    orc_ctx *c = r->c, *f = r->f;
    if (!c->fb) {
        c->fb = (double *)calloc((size_t)Q * c->N, sizeof(double));
        if (!c->fb) return 1;
    }
    for (int s = 0; s < nsteps; ++s) {
        step_prepare(c);
        /* coarse pre-collision moments at t+1 on the block's surface */
        for (int z = 0; z < c->p.nz; ++z)
            for (int y = 0; y < c->p.ny; ++y)
                for (int x = 0; x < c->p.nx; ++x) {
                    int X[3] = {x, y, z};
                    if (!in_box(r, X) || in_inside(r, X)) continue;
                    double Fi[Q];
                    int missing[Q];
                    gather_node(c, x, y, z, Fi, missing);
                    refine_moments(Fi, r->Mnew + rbox(r, X) * NMOM);
                }
        /* coarse update off the block's inside */
        double F[3] = {0, 0, 0}, M[3] = {0, 0, 0}, out[Q];
        for (int z = 0; z < c->p.nz; ++z)
            for (int y = 0; y < c->p.ny; ++y)
                for (int x = 0; x < c->p.nx; ++x) {
                    long n = nid(c, x, y, z);
                    int X[3] = {x, y, z};
                    if (in_inside(r, X) || c->solid1[n]) {
                        for (int i = 0; i < Q; ++i) c->fb[i * c->N + n] = c->fa[i * c->N + n];
                        continue;
                    }
                    node_update(c, x, y, z, out, F, M);
                    for (int i = 0; i < Q; ++i) c->fb[i * c->N + n] = out[i];
                }
        /* fine step to t + 1/2, surface at t + 1/2 */
        refine_fine_interior(r);
        refine_fill_ghosts(r, f->fb, 0.5);
        double *t = f->fa; f->fa = f->fb; f->fb = t;
        /* fine step to t + 1, surface at t + 1 */
        refine_fine_interior(r);
        refine_fill_ghosts(r, f->fb, 1.0);
        /* coarse nodes one layer inside the surface from the fine level: the
         * pre-collision moments at t+1 of the coincident fine node are its
         * pulls from the fine state at t + 1/2 (still in f->fa) */
        for (int z = 0; z < c->p.nz; ++z)
            for (int y = 0; y < c->p.ny; ++y)
                for (int x = 0; x < c->p.nx; ++x) {
                    int X[3] = {x, y, z}, shell = 0;
                    if (!in_inside(r, X)) continue;
                    for (int a = 0; a < 3; ++a)
                        if (!r->full[a] && (X[a] == r->lo[a] + 1 || X[a] == r->hi[a] - 1)) shell = 1;
                    if (!shell) continue;
                    double Fi[Q], Mf[NMOM];
                    int missing[Q];
                    gather_node(f, 2 * (x - r->lo[0]), 2 * (y - r->lo[1]), 2 * (z - r->lo[2]), Fi, missing);
                    refine_moments(Fi, Mf);
                    refine_rebuild(Mf, r->s_fc, c->p.beta, c->p.gamma_mode, out);
                    long n = nid(c, x, y, z);
                    for (int i = 0; i < Q; ++i) c->fb[i * c->N + n] = out[i];
                }
        t = f->fa; f->fa = f->fb; f->fb = t;
        t = c->fa; c->fa = c->fb; c->fb = t;
        uint8_t *u = c->solid0; c->solid0 = c->solid1; c->solid1 = u;
        for (int a = 0; a < 3; ++a) { c->b.F[a] = F[a]; c->b.M[a] = M[a]; }
        t = r->Mold; r->Mold = r->Mnew; r->Mnew = t;
        c->step++;
        f->step += 2;
    }
    return 0;
}
