// Conserved quantities without any device allocation.
//
// sph_conserved needs a context, and a context allocates its scratch with
// cudaMalloc.  Some callers cannot do that: code that reports the energy
// error from inside a region that must not synchronise the device (cudaMalloc
// may block until outstanding work finishes), or a host framework that owns
// all device memory and only lends this library its particle arrays.  For
// them, sph_conserved_noalloc keeps its per-block partial sums in the
// fixed-size device array below instead of context scratch.
//
// The array belongs to the library image: every GPU on which the library is
// loaded holds its 256 KB until the process exits.  All calls share it, so
// two calls whose kernels overlap on the GPU (different streams without
// ordering) race on it; calls on one stream are ordered and safe.  Each call
// overwrites every partial it later reads (blocks 0..nb-1), so nothing has to
// be cleared between calls.
#include <mutex>

#include "sph_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaChunk = 4096;      // particles summed by one block
constexpr int kNaMaxBlocks = 4096;  // partial-sum slots in the static array
static_assert((long long)kNaChunk * kNaMaxBlocks == SPH_CONSERVED_NOALLOC_MAX_N,
              "the static scratch must cover SPH_CONSERVED_NOALLOC_MAX_N particles");

// 8 partial sums per block, laid out [quantity][block]
static __device__ __align__(256) double g_na_partials[8 * kNaMaxBlocks];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
double *g_na_dev_ptr[kNaMaxDevices] = {};

// block b sums particles [b * kNaChunk, (b + 1) * kNaChunk) in FP64
__global__ void __launch_bounds__(kNaThreads) na_block_kernel(const float4 *__restrict__ pos,
                                                              const float4 *__restrict__ vel,
                                                              int64_t n, double *part, int nb)
{
    __shared__ double sm[8][kNaThreads];
    double e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t begin = (int64_t)blockIdx.x * kNaChunk;
    const int64_t end = begin + kNaChunk < n ? begin + kNaChunk : n;
    for (int64_t i = begin + threadIdx.x; i < end; i += kNaThreads) {
        float4 p = pos[i], v = vel[i];
        double m = p.w, x = p.x, y = p.y, z = p.z, vx = v.x, vy = v.y, vz = v.z;
        e[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        e[1] += m * (double)v.w;
        e[2] += m * vx;
        e[3] += m * vy;
        e[4] += m * vz;
        e[5] += m * (y * vz - z * vy);
        e[6] += m * (z * vx - x * vz);
        e[7] += m * (x * vy - y * vx);
    }
    for (int k = 0; k < 8; ++k) sm[k][threadIdx.x] = e[k];
    __syncthreads();
    for (int s = kNaThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 8; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 8) part[threadIdx.x * nb + blockIdx.x] = sm[threadIdx.x][0];
}

// adds the nb block sums in block order; nb == 0 writes zeros
__global__ void na_final_kernel(const double *part, int nb, double *out8)
{
    int k = threadIdx.x;
    if (k < 8) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[k * nb + b];
        out8[k] = s;
    }
}

// Device address of g_na_partials on the current device.  The first call on
// each device looks it up (cudaGetSymbolAddress, no allocation) and caches it.
sph_status na_scratch(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ERR_CUDA;
    if (dev < 0 || dev >= kNaMaxDevices) return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_dev_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_partials);
        if (e != cudaSuccess || !p) return SPH_ERR_CUDA;
        g_na_dev_ptr[dev] = (double *)p;
    }
    *out = g_na_dev_ptr[dev];
    return SPH_OK;
}

}  // namespace

extern "C" sph_status sph_conserved_noalloc(int64_t n, const float *d_pos, const float *d_vel,
                                            double *d_out8, void *stream)
{
    if (n < 0 || n > SPH_CONSERVED_NOALLOC_MAX_N) return SPH_ERR_INVALID_ARG;
    if (!d_out8 || (n > 0 && (!d_pos || !d_vel))) return SPH_ERR_INVALID_ARG;
    if (((uintptr_t)d_pos & 15u) || ((uintptr_t)d_vel & 15u) || ((uintptr_t)d_out8 & 7u))
        return SPH_ERR_INVALID_ARG;
    double *part = nullptr;
    sph_status st = na_scratch(&part);
    if (st != SPH_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((n + kNaChunk - 1) / kNaChunk);
    if (nb > 0)
        na_block_kernel<<<nb, kNaThreads, 0, s>>>((const float4 *)d_pos, (const float4 *)d_vel, n,
                                                  part, nb);
    na_final_kernel<<<1, 32, 0, s>>>(part, nb, d_out8);
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
