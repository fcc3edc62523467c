// Immersed-body state shared by the geometry, boundary and API translation
// units of liblbm.so (arXiv 1608.04658, Secs. 3 and 4): body parameters,
// the device body state, the library's boundary scratch and their launchers.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

// swimmer mesh lists (Sec. 4.3 body)
constexpr int MESH_COL_CAP = 32;    // crossings kept per band column
constexpr int MESH_CELL = 2;        // edge of a triangle cell (lattice units)
constexpr int MESH_CELL_CAP = 384;  // triangles kept per cell
constexpr int MESH_THREADS = 256;   // block size of the per-vertex and per-triangle mesh kernels

struct GeomParams {
    int kind;
    int free_motion;
    double R;
    double y_lo, y_hi;
    double U_lo[3], U_hi[3];
    double inv_mass;     // 1 / m_s
    double buoy;         // 1 - rho_f / rho_s
    double g[3];
    // airfoil
    double chord, ca, sa, h_amp, h_omega, camber_m, camber_p, thick[5], y_base;
    double inv_chord, camber_k1, camber_k2;  // 1/c, m/p^2, m/(1-p)^2 (single-precision link search)
    double box[4];       // profile box relative to the leading edge: dx min/max, dy min/max
    // swimmer mesh (device arrays owned by Scratch)
    const double *mesh_rest;  // (s, dy, dz) per vertex
    const int *mesh_tris;     // three vertex indices per triangle
    double *mesh_pos;         // vertex positions at the current pose
    double *mesh_vel;         // vertex velocities at the current pose
    int *mesh_ipos;           // vertex positions split as nearest lattice point ...
    float *mesh_frac;         // ... plus the remainder in [-1/2, 1/2] (FP32 link search)
    float *tri_box;           // per triangle: min x, y, z, max x, y, z (rounded outwards)
    int *col_count;           // crossings per band column (y, z)
    double *col_x;            // [column][MESH_COL_CAP] crossing abscissae
    int *cell_count;          // triangles per band cell
    int *cell_tri;            // [cell][MESH_CELL_CAP] triangle indices
    int *mesh_status;         // overflow of the column or cell lists in this step
    double *mesh_partials;    // centre-of-mass frame: per-block volume sums (9 per block)
    unsigned *mesh_ticket;    // last-block counter of their reduction
    double *mesh_dy, *mesh_dvy; // adjoint only: theta-tangents of vertex position / velocity (y)
    int n_vertices, n_triangles;
    int cells[3];             // cell grid of the band capacity box
    double length, wave_amp, wave_length, wave_period;
    int wave_ramp;
    int com_frame;            // free in y or yaw: X is the centre of mass, yaw psi
    double mass;              // body mass (density mass / mesh volume in the centre-of-mass frame)
    double mesh_ext[6];       // pose extent relative to the head: x, y, z min/max
    int periodic[3];
    // slab of a box split along z (lbm_set_slab): local z layer k is layer
    // zoff + k (mod zper) of the whole box; zper = 0: no slab.  The force and
    // torque sum the links of the own layers [own_lo, own_hi) only.
    int zoff, zper, own_lo, own_hi;
    int cap[3];          // band capacity per axis
    int cap_boundary;    // slots in the boundary list
    int cap_uncovered;   // slots in the uncovered list
};

// Body state; two copies alternate between steps (the mark kernel reads the
// previous one and writes the next).
struct DevBody {
    double X[3], U[3];
    double F[3], M[3];
    double F_sum[3], M_sum[3];
    long long n_sum;
    int band_lo[3], band_n[3];
    int n_boundary, n_uncovered, n_links;
    int status;
    double t;            // time of the current pose (prescribed motion)
    // swimmer in the centre-of-mass frame
    double psi, omega;   // yaw angle and rate
    double Iw, Izz;      // angular momentum and moment of inertia about the centre of mass
    double com[2];       // centre of mass in the body frame at the pose
    double com_dot[2];   // its central-difference rate
    int ibox[4];         // lattice x/y box of the pose: x min, x max, y min, y max
    // band of the step that starts from this state {lo x, y, z, n x, y, z}
    // (the box the mark kernel of that step sweeps)
    int sweep[6];
};

// scratch owned by the library for the boundary path
struct Scratch {
    DevBody *body;       // [2]
    int *blist;          // [cap_boundary] node index of each boundary node
    int *bpos;           // [cap_boundary] band position of each boundary node
    int *ulist;          // [cap_uncovered] node index of each uncovered node
    int *upos;           // [cap_uncovered] band position of each uncovered node
    double *bforce;      // [band capacity * 6] force and torque per band position
    double *partials;    // [n_partials * 6]
    unsigned *ticket;    // last-block counter of the force reduction
    int n_partials;
    // swimmer mesh
    double *mesh_rest, *mesh_pos, *mesh_vel, *col_x;
    int *mesh_tris, *col_count, *cell_count, *cell_tri, *mesh_status, *mesh_ipos;
    float *tri_box, *mesh_frac;
    double *mesh_partials;
    unsigned *mesh_ticket;
};

// launchers ------------------------------------------------------------------
cudaError_t launch_geometry(const Lattice &L, const GeomParams &G, Scratch &S, int prev, uint8_t *flags,
                            cudaStream_t s, int *nlaunch);
cudaError_t launch_mark_initial(const Lattice &L, const GeomParams &G, const double *X,
                                uint8_t *flags, cudaStream_t s);
cudaError_t launch_refill(int storage, const Lattice &L, const GeomParams &G, Scratch &S, int cur,
                          void *fa, const uint8_t *flags, cudaStream_t s);
cudaError_t launch_boundary(int storage, const Lattice &L, const GeomParams &G, Scratch &S, int cur,
                            const void *fa, void *fb, const uint8_t *flags, cudaStream_t s);
cudaError_t launch_forces(const GeomParams &G, Scratch &S, int cur, cudaStream_t s, int *nlaunch);
cudaError_t launch_sweep_init(const Lattice &L, const GeomParams &G, Scratch &S, int cur, cudaStream_t s);
struct Force6 {
    double v[6];
};
cudaError_t launch_set_force(Scratch &S, int cur, const double fm[6], cudaStream_t s);
cudaError_t launch_sum_force(Scratch &S, int cur, const double *parts, int n, cudaStream_t s);
// true when the band is known before the step's geometry runs (all bodies but
// the walls, whose band is the whole box, and the swimmer in the
// centre-of-mass frame, whose band follows from the pose of the step)
__host__ __device__ inline bool sweep_ahead(const GeomParams &G)
{
    return G.kind != LBM_BODY_NONE && G.kind != LBM_BODY_PLANES && !(G.kind == LBM_BODY_MESH && G.com_frame);
}
cudaError_t launch_mesh_prepare(const Lattice &L, const GeomParams &G, Scratch &S, int prev, bool advance,
                                cudaStream_t s, int *nlaunch);
cudaError_t launch_mesh_body(const Lattice &L, const GeomParams &G, Scratch &S, int prev, bool advance,
                             cudaStream_t s, int *nlaunch);
cudaError_t launch_mesh_mark_initial(const Lattice &L, const GeomParams &G, Scratch &S, int cur,
                                     uint8_t *flags, cudaStream_t s);

}  // namespace lbm
