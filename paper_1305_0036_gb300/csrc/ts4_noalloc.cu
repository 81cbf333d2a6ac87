// ts_reduce_sz_static: the norm and <S^z_j> of a caller's device state without
// any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need these
// numbers: host applications whose device memory is owned by their own pool
// allocator and handed out only to them, plug-ins that must not grow the
// device footprint behind their host's back, and loops that must not allocate
// once they have started.  This entry point serves them: the caller passes the
// state and a device output buffer, and the only scratch memory used -- the
// per-block partial sums -- is a fixed array with static storage in this file.
//
// The array is TS_STATIC_MAX_BLOCKS * (TS_STATIC_MAX_N + 1) doubles (about
// 280 KB); every GPU that loads the library holds it until the process exits.
// Its device address is looked up once per device with cudaGetSymbolAddress,
// on the first call made while that device is current; make that first call
// before starting any stream capture.  Every call shares the array and leaves
// its partial sums in it; the reduction writes every partial it later reads,
// so nothing has to start at zero.  Calls whose kernels overlap on the GPU
// (for example on two streams) race on the array and must not be issued.
#include "../../include/ts4.h"
#include "ts4_kernels.cuh"

#include <mutex>

namespace {

constexpr int TS_STATIC_MAX_N = 34;
constexpr int TS_STATIC_MAX_BLOCKS = 1024;
constexpr int TS_STATIC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_sz_partials[TS_STATIC_MAX_BLOCKS * (TS_STATIC_MAX_N + 1)];

std::mutex g_setup_mutex;
double *g_partials_addr[TS_STATIC_MAX_DEVICES] = {};

// Sums the block partials (stride N + 1) and writes out[0] = norm, out[1 + j] = <S^z_j>.
__global__ void k_sz_finish_static(const double *__restrict__ part, int nblk, int N, double *__restrict__ out)
{
    __shared__ double sums[TS_STATIC_MAX_N + 1];
    for (int k = threadIdx.x; k <= N; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; b++)
            s += part[(size_t)b * (N + 1) + k];
        sums[k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= N; k += blockDim.x)
        out[k] = (k == 0) ? sums[0] : sums[k] - 0.5 * sums[0];
}

} // namespace

extern "C" ts_status ts_reduce_sz_static(const void *psi_dev, int N, ts_prec prec, double *out_dev,
                                         void *cuda_stream)
{
    if (!psi_dev || !out_dev || N < 1 || N > TS_STATIC_MAX_N || (prec != TS_C64 && prec != TS_C128))
        return TS_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TS_STATIC_MAX_DEVICES)
        return TS_ERR_CUDA;
    double *part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            // the symbol's device address for the current device (set-up, once per device)
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_sz_partials) != cudaSuccess || !p)
                return TS_ERR_CUDA;
            g_partials_addr[dev] = static_cast<double *>(p);
        }
        part = g_partials_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // a power of two of at most TS_STATIC_MAX_BLOCKS blocks (k_sum_sz's span layout)
    const unsigned nb = ts4::sum_sz_blocks(N, TS_STATIC_MAX_BLOCKS);
    if (nb > (unsigned)TS_STATIC_MAX_BLOCKS)
        return TS_ERR_ARG;
    if (prec == TS_C64)
        ts4::k_sum_sz<float2><<<(unsigned)nb, 256, 0, st>>>((const float2 *)psi_dev, N, part);
    else
        ts4::k_sum_sz<double2><<<(unsigned)nb, 256, 0, st>>>((const double2 *)psi_dev, N, part);
    k_sz_finish_static<<<1, 64, 0, st>>>(part, (int)nb, N, out_dev);
    return cudaGetLastError() == cudaSuccess ? TS_OK : TS_ERR_CUDA;
}
