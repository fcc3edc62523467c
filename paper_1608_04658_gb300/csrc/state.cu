// State set-up and read-out kernels: the initial equilibrium state (Sec. 2,
// Eq. feq_min, the exact product-form equilibrium), the decoding and encoding
// of one population plane, and the per-block FP64 partial sums of mass,
// momentum and kinetic energy.
#include <type_traits>

#include "kbc.cuh"

namespace lbm {

// f = f^eq(rho, u) + amp W xi (Eq. feq_min) with the fields in double (T =
// double) or single precision (T = float).
template <typename S, typename T>
__global__ void init_kernel(const Lattice L, S *__restrict__ f, const T *__restrict__ rho,
                            const T *__restrict__ u, const T *__restrict__ xi, double amp)
{
    using R = typename Codec<S>::R;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    // equilibrium evaluated in the collision's arithmetic R (double for FP64
    // storage, FP32 otherwise: GB300's FP64 rate made the double evaluation
    // the slowest part of setting up a large lattice), the density excess
    // taken in double; then rounded once to storage
    R ex[3], ey[3], ez[3], rx[3], ry[3], rz[3];
    axis_eq<R>((R)u[3 * n + 0], ex, rx);
    axis_eq<R>((R)u[3 * n + 1], ey, ry);
    axis_eq<R>((R)u[3 * n + 2], ez, rz);
    const double r = (double)rho[n];
    const R drho = (R)(r - L.rho0), rr = (R)r;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        R g = shifted_feq<R>(i, drho, rr, ex, ey, ez);
        if (xi) g += (R)(amp * weight<double>(i) * (double)xi[(size_t)i * L.N + n]);
        Codec<S>::store(f + (size_t)i * L.N + n, g);
    }
}

template <typename S>
__global__ void decode_kernel(const Lattice L, const S *__restrict__ f, int i, double *__restrict__ out)
{
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    out[n] = (double)Codec<S>::load(f + (size_t)i * L.N + n) + weight<double>(i) * L.rho0;
}

template <typename S>
__global__ void encode_kernel(const Lattice L, S *__restrict__ f, int i, const double *__restrict__ in)
{
    using R = typename Codec<S>::R;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    Codec<S>::store(f + (size_t)i * L.N + n, (R)(in[n] - weight<double>(i) * L.rho0));
}

// Per-block FP64 partial sums of mass, momentum and kinetic energy over
// non-solid nodes; the host adds the block partials in block order.
template <typename S>
__global__ void __launch_bounds__(256) totals_kernel(const Lattice L, const S *__restrict__ f,
                                                     const uint8_t *__restrict__ flags,
                                                     double *__restrict__ partials)
{
    double acc[5] = {0, 0, 0, 0, 0};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < L.N;
         n += (long long)gridDim.x * blockDim.x) {
        if (flags && (flags[n] & FL_SOLID)) continue;
        double r = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            const double v = (double)Codec<S>::load(f + (size_t)i * L.N + n) + weight<double>(i) * L.rho0;
            r += v;
            j[0] += cx_of(i) * v;
            j[1] += cy_of(i) * v;
            j[2] += cz_of(i) * v;
        }
        acc[0] += r;
        acc[1] += j[0];
        acc[2] += j[1];
        acc[3] += j[2];
        acc[4] += 0.5 * (j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / r;
    }
    __shared__ double sm[8][5];
    for (int k = 0; k < 5; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sm[w][threadIdx.x];
        partials[blockIdx.x * 5 + threadIdx.x] = v;
    }
}

// ----------------------------------------------------------------- launchers
template <typename T>
cudaError_t launch_init(int storage, const Lattice &L, void *fa, const T *rho, const T *u, const T *xi, double amp,
                        cudaStream_t s)
{
    return dispatch_storage(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        const int nb = (int)((L.N + 255) / 256);
        init_kernel<S, T><<<nb, 256, 0, s>>>(L, (S *)fa, rho, u, xi, amp);
        return cudaGetLastError();
    });
}
template cudaError_t launch_init<double>(int, const Lattice &, void *, const double *, const double *,
                                         const double *, double, cudaStream_t);
template cudaError_t launch_init<float>(int, const Lattice &, void *, const float *, const float *, const float *,
                                        double, cudaStream_t);

cudaError_t launch_decode_plane(int storage, const Lattice &L, const void *f, int i,
                                double *out, cudaStream_t s)
{
    return dispatch_storage(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        const int nb = (int)((L.N + 255) / 256);
        decode_kernel<S><<<nb, 256, 0, s>>>(L, (const S *)f, i, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_encode_plane(int storage, const Lattice &L, void *f, int i,
                                const double *in, cudaStream_t s)
{
    return dispatch_storage(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        const int nb = (int)((L.N + 255) / 256);
        encode_kernel<S><<<nb, 256, 0, s>>>(L, (S *)f, i, in);
        return cudaGetLastError();
    });
}

cudaError_t launch_totals(int storage, const Lattice &L, const void *f, const uint8_t *flags,
                          double *partials, int nblocks, double *out, cudaStream_t s)
{
    (void)out;
    return dispatch_storage(storage, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        totals_kernel<S><<<nblocks, 256, 0, s>>>(L, (const S *)f, flags, partials);
        return cudaGetLastError();
    });
}

}  // namespace lbm
