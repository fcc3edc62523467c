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

// device status bits
constexpr int ST_UNSTABLE = 1;
constexpr int ST_BAND_OVERFLOW = 2;

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
    // the same parameters rounded once to FP32 for the FP32 arithmetic of the
    // bulk kernels (no FP64 conversion on the device)
    float beta_f, inv_beta_f, rho0_f;
    float g_face_f[27];
};

// Which nodes one bulk launch updates.  ALL: every node (those flagged SOLID
// or BOUNDARY skipped when flags are given).  OUTSIDE: the nodes outside the
// body's sweep box, which are fluid and no boundary node at t and t+1, so no
// flag is read.  BAND: the nodes of the sweep box (flags read).  sweep =
// {lo x, lo y, lo z, n x, n y, n z} of the box, in device memory (wrapping on
// periodic axes); cap = capacity of the box per axis (the BAND grid).
enum BulkMode { BULK_ALL = 0, BULK_OUTSIDE = 1, BULK_BAND = 2 };

// Calls fn with a null pointer of the storage type (one instantiation per
// storage form).
template <typename F>
static cudaError_t dispatch_storage(int storage, F &&fn)
{
    switch (storage) {
    case LBM_FP64: return fn((double *)nullptr);
    case LBM_FP32: return fn((float *)nullptr);
    case LBM_FP16: return fn((__half *)nullptr);
    case LBM_BF16: return fn((__nv_bfloat16 *)nullptr);
    default: return cudaErrorInvalidValue;
    }
}

// launchers ------------------------------------------------------------------
// z_lo, z_n: the z layers [z_lo, z_lo + z_n) of ALL and OUTSIDE launches
// (z_n < 0: to the last layer); BAND launches take the box's layers.
cudaError_t launch_bulk(int storage, const Lattice &L, const void *fa, void *fb,
                        const uint8_t *flags, int *status, cudaStream_t s, int mode = BULK_ALL,
                        const int *sweep = nullptr, const int *cap = nullptr, int z_lo = 0, int z_n = -1);
// the initial state from density, velocity and noise fields in double (T =
// double) or single precision (T = float)
template <typename T>
cudaError_t launch_init(int storage, const Lattice &L, void *fa, const T *rho, const T *u, const T *xi, double amp,
                        cudaStream_t s);
cudaError_t launch_decode_plane(int storage, const Lattice &L, const void *f, int i,
                                double *out, cudaStream_t s);
cudaError_t launch_encode_plane(int storage, const Lattice &L, void *f, int i,
                                const double *in, cudaStream_t s);
cudaError_t launch_totals(int storage, const Lattice &L, const void *f, const uint8_t *flags,
                          double *partials, int nblocks, double *out, cudaStream_t s);

}  // namespace lbm
