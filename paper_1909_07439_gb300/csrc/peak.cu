// FP32 throughput probe: the measured denominator of the pair passes'
// roofline.  Every thread runs 8 independent multiply-add chains (enough
// independent work to hide the FMA latency at full occupancy), either as
// scalar FP32 fused multiply-adds or as packed FP32x2 ones (two lanes of
// arithmetic per instruction).  The chains' values are consumed so that the
// compiler keeps every operation; the sink is written only for a value the
// chains cannot reach.
#include "sph_internal.cuh"

namespace sph {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) ffma_chain_kernel(float *sink, int iters, float a, float b)
{
    float acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = fmaf(acc[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    if (s == -1.2345e30f) *sink = s;
}

__global__ void __launch_bounds__(256) ffma2_chain_kernel(float *sink, int iters, float a, float b)
{
    float2 acc[kChains];
    const float2 aa = make_float2(a, a), bb = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        acc[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)(threadIdx.x - k) * 1e-3f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = __ffma2_rn(acc[k], aa, bb);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k].x + acc[k].y;
    if (s == -1.2345e30f) *sink = s;
}

}  // namespace sph

extern "C" sph_status sph_fp32_probe(float *d_sink, int blocks, int iters, int packed, void *stream)
{
    if (!d_sink || blocks < 1 || iters < 1 || (packed != 0 && packed != 1)) return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // a in (0, 1) keeps the chains bounded: x -> a x + b converges to b / (1 - a)
    if (packed)
        sph::ffma2_chain_kernel<<<blocks, 256, 0, st>>>(d_sink, iters, 0.999f, 1e-3f);
    else
        sph::ffma_chain_kernel<<<blocks, 256, 0, st>>>(d_sink, iters, 0.999f, 1e-3f);
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
