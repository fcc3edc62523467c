// Internal declarations shared by the CUDA translation units of liblbm.so.
// Lattice: D3Q27, direction i = 9(cx+1) + 3(cy+1) + (cz+1), opposite 26 - i,
// weights W = w(cx) w(cy) w(cz) with w(0) = 2/3, w(+-1) = 1/6, c_s^2 = 1/3.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/lbm.h"

namespace lbm {

constexpr int Q = 27;

// node marks (flags byte)
constexpr uint8_t FL_SOLID = 1;      // inside the body at the current step
constexpr uint8_t FL_SOLID_PREV = 2; // inside the body at the previous step
constexpr uint8_t FL_BOUNDARY = 4;   // fluid node with at least one solid pull source
constexpr uint8_t FL_UNCOVERED = 8;  // solid at the previous step, fluid now

// swimmer mesh lists (Sec. 4.3 body)
constexpr int MESH_COL_CAP = 32;    // crossings kept per band column
constexpr int MESH_CELL = 2;        // edge of a triangle cell (lattice units)
constexpr int MESH_CELL_CAP = 384;  // triangles kept per cell

// device status bits
constexpr int ST_UNSTABLE = 1;
constexpr int ST_BAND_OVERFLOW = 2;
constexpr int ST_TIMEOUT = 4;        // a bounded wait on an mbarrier gave up

__host__ __device__ constexpr int cx_of(int i) { return i / 9 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int nonzero_of(int i)
{
    return (cx_of(i) != 0) + (cy_of(i) != 0) + (cz_of(i) != 0);
}
// weight by number of non-zero components: 8/27, 2/27, 1/54, 1/216
template <typename T>
__host__ __device__ constexpr T weight(int i)
{
    return nonzero_of(i) == 0 ? T(8) / T(27)
         : nonzero_of(i) == 1 ? T(2) / T(27)
         : nonzero_of(i) == 2 ? T(1) / T(54)
                              : T(1) / T(216);
}
template <typename T>
__host__ __device__ constexpr T inv_weight(int i)
{
    return nonzero_of(i) == 0 ? T(27) / T(8)
         : nonzero_of(i) == 1 ? T(27) / T(2)
         : nonzero_of(i) == 2 ? T(54)
                              : T(216);
}

// ---------------------------------------------------------------- storage codec
template <typename S> struct Codec;
template <> struct Codec<double> {
    using R = double;
    __device__ static double load(const double *p) { return *p; }
    __device__ static void store(double *p, double v) { *p = v; }
};
template <> struct Codec<float> {
    using R = float;
    __device__ static float load(const float *p) { return *p; }
    __device__ static void store(float *p, float v) { *p = v; }
};
template <> struct Codec<__half> {
    using R = float;
    __device__ static float load(const __half *p) { return __half2float(*p); }
    __device__ static void store(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Codec<__nv_bfloat16> {
    using R = float;
    __device__ static float load(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    __device__ static void store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------- parameters
struct Lattice {
    int nx, ny, nz;
    long long N;
    int plane[27];      // i * N: offset of population plane i (27 N < 2^31)
    int face[6];
    int gamma_mode;
    double beta;
    double inv_beta;
    double rho0;
    double u_face[3];
    double g_face[27];  // f^eq(rho0, u_face) - W rho0 for EQ faces
};

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
    float *tri_box;           // per triangle: min x, y, z, max x, y, z (rounded outwards)
    int *col_count;           // crossings per band column (y, z)
    double *col_x;            // [column][MESH_COL_CAP] crossing abscissae
    int *cell_count;          // triangles per band cell
    int *cell_tri;            // [cell][MESH_CELL_CAP] triangle indices
    int *mesh_status;         // overflow of the column or cell lists in this step
    int n_vertices, n_triangles;
    int cells[3];             // cell grid of the band capacity box
    double length, wave_amp, wave_length, wave_period;
    int wave_ramp;
    double mesh_ext[6];       // pose extent relative to the head: x, y, z min/max
    int periodic[3];
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
};

// scratch owned by the library for the boundary path
struct Scratch {
    DevBody *body;       // [2]
    int *blist;          // [cap_boundary] node index of each boundary node
    int *bpos;           // [cap_boundary] band position of each boundary node
    int *ulist;          // [cap_uncovered] node index of each uncovered node
    double *bforce;      // [band capacity * 6] force and torque per band position
    double *partials;    // [n_partials * 6]
    unsigned *ticket;    // last-block counter of the force reduction
    int n_partials;
    // swimmer mesh
    double *mesh_rest, *mesh_pos, *mesh_vel, *col_x;
    int *mesh_tris, *col_count, *cell_count, *cell_tri, *mesh_status;
    float *tri_box;
};

// launchers ------------------------------------------------------------------
cudaError_t launch_bulk(int storage, const Lattice &L, const void *fa, void *fb,
                        const uint8_t *flags, int *status, cudaStream_t s);
cudaError_t launch_init(int storage, const Lattice &L, void *fa, const double *rho,
                        const double *u, const double *xi, double amp, cudaStream_t s);
cudaError_t launch_decode_plane(int storage, const Lattice &L, const void *f, int i,
                                double *out, cudaStream_t s);
cudaError_t launch_encode_plane(int storage, const Lattice &L, void *f, int i,
                                const double *in, cudaStream_t s);
cudaError_t launch_totals(int storage, const Lattice &L, const void *f, const uint8_t *flags,
                          double *partials, int nblocks, double *out, cudaStream_t s);

cudaError_t launch_geometry(const Lattice &L, const GeomParams &G, Scratch &S, int prev, uint8_t *flags,
                            cudaStream_t s, int *nlaunch);
cudaError_t launch_mark_initial(const Lattice &L, const GeomParams &G, const double *X,
                                uint8_t *flags, cudaStream_t s);
cudaError_t launch_refill(int storage, const Lattice &L, const GeomParams &G, Scratch &S, int cur,
                          void *fa, const uint8_t *flags, cudaStream_t s);
cudaError_t launch_boundary(int storage, const Lattice &L, const GeomParams &G, Scratch &S, int cur,
                            const void *fa, void *fb, const uint8_t *flags, cudaStream_t s);
cudaError_t launch_forces(const GeomParams &G, Scratch &S, int cur, cudaStream_t s, int *nlaunch);
cudaError_t launch_mesh_prepare(const Lattice &L, const GeomParams &G, Scratch &S, int prev, bool advance,
                                cudaStream_t s, int *nlaunch);
cudaError_t launch_mesh_mark_initial(const Lattice &L, const GeomParams &G, Scratch &S, int cur,
                                     uint8_t *flags, cudaStream_t s);

}  // namespace lbm
