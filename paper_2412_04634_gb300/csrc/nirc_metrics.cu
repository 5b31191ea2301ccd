// nirc_metrics.cu -- frame metric: mean relative squared error (paper:
// MRSE, used for every equal-time comparison), mean over pixels and RGB of
// (I - R)^2 / (R^2 + eps).  Each term is formed in binary32 (IEEE divide;
// at most four roundings, ~2.4e-7 relative) and the frame-level sum is
// accumulated in FP64, the only FP64 arithmetic on the GPU (FP64 divides
// would make this HBM-light kernel bound by the FP64 unit).  Grid-stride
// float4 reads, per-thread FP64 sums, warp and block reductions, one FP64
// atomic add per block into the zeroed output.
#include "nirc_internal.h"

namespace nirc {

constexpr int kMrseThreads = 256;

__device__ __forceinline__ float rel_sq(float a, float b, float eps) {
    const float d = __fsub_rn(a, b);
    return __fdiv_rn(__fmul_rn(d, d), __fadd_rn(__fmul_rn(b, b), eps));
}

__global__ void __launch_bounds__(kMrseThreads) k_mrse(const float4* __restrict__ img, const float4* __restrict__ ref,
                                                      uint64_t n, float eps, double scale, double* __restrict__ out) {
    double acc = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * kMrseThreads + threadIdx.x; i < n; i += (uint64_t)gridDim.x * kMrseThreads) {
        const float4 a = __ldg(img + i), b = __ldg(ref + i);
        acc += (double)rel_sq(a.x, b.x, eps) + (double)rel_sq(a.y, b.y, eps) + (double)rel_sq(a.z, b.z, eps);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double part[kMrseThreads / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kMrseThreads / 32 ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(out, v * scale);
    }
}

cudaError_t launch_mrse(const float* img, const float* ref, uint64_t n, float eps, double* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
    if (e != cudaSuccess || n == 0) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (n + kMrseThreads - 1) / kMrseThreads;
    if (blocks > (uint64_t)sms * 4) blocks = (uint64_t)sms * 4;
    k_mrse<<<(uint32_t)blocks, kMrseThreads, 0, st>>>(reinterpret_cast<const float4*>(img),
                                                      reinterpret_cast<const float4*>(ref), n, eps,
                                                      1.0 / (3.0 * (double)n), out);
    return cudaGetLastError();
}

}  // namespace nirc
