// lbm_totals_noalloc: the global mass / momentum / kinetic-energy reduction of
// lbm_totals without a context and without any device allocation.
//
// Scratch: the per-block partial sums live in a file-scope __device__ array
// of NOALLOC_MAX_PARTIALS x 5 doubles (160 KB).  Every GPU that loads the
// library holds it until the process exits, and every call shares it.  Each
// block sums a fixed chunk of NOALLOC_CHUNK consecutive nodes, so a lattice of
// more than NOALLOC_MAX_PARTIALS * NOALLOC_CHUNK nodes is rejected.  The
// partials are fully rewritten by every call (nothing has to start at zero);
// two calls whose kernels overlap on the GPU would race on them.  The array's
// device address is looked up on the first call on each device and kept for
// the life of the process (a cudaDeviceReset of that device invalidates it,
// as it does every other device pointer the caller holds).
#include <mutex>

#include "lbm_internal.cuh"

namespace lbm {

constexpr int NOALLOC_CHUNK = 16384;         // nodes per block partial
constexpr int NOALLOC_MAX_PARTIALS = 4096;   // -> at most 67,108,864 nodes
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double noalloc_partials[NOALLOC_MAX_PARTIALS * 5];

template <typename S>
__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_partial_kernel(const S *__restrict__ f,
                                                                          const uint8_t *__restrict__ flags,
                                                                          long long N, double rho0,
                                                                          double *__restrict__ partials)
{
    const long long beg = (long long)blockIdx.x * NOALLOC_CHUNK;
    const long long end = beg + NOALLOC_CHUNK < N ? beg + NOALLOC_CHUNK : N;
    double acc[5] = {0, 0, 0, 0, 0};
    for (long long n = beg + threadIdx.x; n < end; n += NOALLOC_THREADS) {
        if (flags && (flags[n] & FL_SOLID)) continue;
        double r = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            const double v = (double)Codec<S>::load(f + (size_t)i * N + n) + weight<double>(i) * rho0;
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
    __shared__ double sm[NOALLOC_THREADS / 32][5];
    for (int k = 0; k < 5; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0;
        for (int w = 0; w < NOALLOC_THREADS / 32; ++w) v += sm[w][threadIdx.x];
        partials[blockIdx.x * 5 + threadIdx.x] = v;
    }
}

// one warp per sum; lanes take partials lane, lane + 32, ... then a shuffle tree
__global__ void noalloc_final_kernel(const double *__restrict__ partials, int nparts, double *__restrict__ out)
{
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= 5) return;
    double v = 0;
    for (int p = lane; p < nparts; p += 32) v += partials[p * 5 + k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[k] = v;
}

// true when p is device (or managed) memory that device dev can address
static bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();  // the query's own error, raised just now
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// device address of the scratch array on device dev, looked up once per
// device (the first call on a device does it)
static double *scratch_on_device(int dev, lbm_status &st)
{
    static std::mutex mu;
    static double *addr[NOALLOC_MAX_DEVICES] = {};
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        st = LBM_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, noalloc_partials) != cudaSuccess || !p) {
            st = LBM_ERR_CUDA;
            return nullptr;
        }
        addr[dev] = static_cast<double *>(p);
    }
    st = LBM_OK;
    return addr[dev];
}

}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_totals_noalloc(const lbm_params *p, const void *f, const uint8_t *flags, double *out,
                                         void *stream)
{
    if (!p || !f || !out) return LBM_ERR_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || !(p->rho0 > 0.0)) return LBM_ERR_ARG;
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (27 * N >= (1LL << 31)) return LBM_ERR_ARG;
    if (N > (long long)NOALLOC_MAX_PARTIALS * NOALLOC_CHUNK) return LBM_ERR_ARG;
    if (p->storage < LBM_FP64 || p->storage > LBM_BF16) return LBM_ERR_ARG;
    // an error left pending by earlier, unrelated work stays with its owner:
    // enqueue nothing and leave it in place
    if (cudaPeekAtLastError() != cudaSuccess) return LBM_ERR_CUDA;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
    // the kernels run on the current device, so the buffers must live there
    if (!on_device(f, dev) || !on_device(out, dev) || (flags && !on_device(flags, dev))) return LBM_ERR_ARG;
    lbm_status st;
    double *scratch = scratch_on_device(dev, st);
    if (!scratch) return st;
    const int nparts = (int)((N + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK);
    cudaStream_t s = (cudaStream_t)stream;
    switch (p->storage) {
    case LBM_FP64:
        noalloc_partial_kernel<double><<<nparts, NOALLOC_THREADS, 0, s>>>((const double *)f, flags, N, p->rho0, scratch);
        break;
    case LBM_FP32:
        noalloc_partial_kernel<float><<<nparts, NOALLOC_THREADS, 0, s>>>((const float *)f, flags, N, p->rho0, scratch);
        break;
    case LBM_FP16:
        noalloc_partial_kernel<__half><<<nparts, NOALLOC_THREADS, 0, s>>>((const __half *)f, flags, N, p->rho0, scratch);
        break;
    case LBM_BF16:
        noalloc_partial_kernel<__nv_bfloat16><<<nparts, NOALLOC_THREADS, 0, s>>>((const __nv_bfloat16 *)f, flags, N,
                                                                                p->rho0, scratch);
        break;
    default: return LBM_ERR_ARG;
    }
    // nothing was pending before the launches, so an error now is their own
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    noalloc_final_kernel<<<1, 5 * 32, 0, s>>>(scratch, nparts, out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
