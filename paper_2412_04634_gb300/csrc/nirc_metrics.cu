// nirc_metrics.cu -- frame metric: mean relative squared error (paper:
// MRSE, used for every equal-time comparison), mean over pixels and RGB of
// (I - R)^2 / (R^2 + eps), accumulated in FP64 (the only FP64 arithmetic on
// the GPU).  Grid-stride float4 reads, per-thread FP64 sums, warp and block
// reductions, one FP64 atomic add per block into the zeroed output.
#include "nirc_internal.h"

namespace nirc {

constexpr int kMrseThreads = 256;

__global__ void __launch_bounds__(kMrseThreads) k_mrse(const float4* __restrict__ img, const float4* __restrict__ ref,
                                                      uint64_t n, double eps, double scale, double* __restrict__ out) {
    double acc = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * kMrseThreads + threadIdx.x; i < n; i += (uint64_t)gridDim.x * kMrseThreads) {
        const float4 a = __ldg(img + i), b = __ldg(ref + i);
        const double d0 = (double)a.x - b.x, d1 = (double)a.y - b.y, d2 = (double)a.z - b.z;
        acc += d0 * d0 / ((double)b.x * b.x + eps) + d1 * d1 / ((double)b.y * b.y + eps) +
               d2 * d2 / ((double)b.z * b.z + eps);
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
                                                      reinterpret_cast<const float4*>(ref), n, (double)eps,
                                                      1.0 / (3.0 * (double)n), out);
    return cudaGetLastError();
}

}  // namespace nirc
