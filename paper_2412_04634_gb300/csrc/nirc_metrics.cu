// nirc_metrics.cu -- per-pixel frame reductions: the later-vertex sums of
// the multi-vertex estimator (k_mv_accumulate), and the frame metric: mean
// relative squared error (paper:
// MRSE, used for every equal-time comparison), mean over pixels and RGB of
// (I - R)^2 / (R^2 + eps).  Each term is formed in binary32 (IEEE divide;
// at most four roundings, ~2.4e-7 relative).  A thread adds its terms into a
// pair of binary32 values (hi + lo: TwoSum (Knuth) gives each add's exact
// rounding error, which lo collects), so its partial sum carries about 48
// significant bits; the pairs are then combined in FP64 (warp and block
// reductions, one FP64 atomic add per block into the zeroed output).  GB300's
// FP64 unit is slow: the former per-term FP64 adds (six FP64 operations per
// pixel) bound this HBM-light kernel, which now issues three per thread.
// Grid-stride float4 reads.
#include "nirc_internal.h"

namespace nirc {

constexpr int kMrseThreads = 256;

__device__ __forceinline__ float rel_sq(float a, float b, float eps) {
    const float d = __fsub_rn(a, b);
    return __fdiv_rn(__fmul_rn(d, d), __fadd_rn(__fmul_rn(b, b), eps));
}

__global__ void __launch_bounds__(kMrseThreads) k_mrse(const float4* __restrict__ img, const float4* __restrict__ ref,
                                                      uint64_t n, float eps, double scale, double* __restrict__ out) {
    float hi = 0.f, lo = 0.f;  // this thread's terms: hi + lo
    for (uint64_t i = (uint64_t)blockIdx.x * kMrseThreads + threadIdx.x; i < n; i += (uint64_t)gridDim.x * kMrseThreads) {
        const float4 a = __ldg(img + i), b = __ldg(ref + i);
        const float t[3] = {rel_sq(a.x, b.x, eps), rel_sq(a.y, b.y, eps), rel_sq(a.z, b.z, eps)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float sum = __fadd_rn(hi, t[k]);
            const float bv = __fsub_rn(sum, hi);  // TwoSum: hi + t = sum + err exactly
            const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bv)), __fsub_rn(t[k], bv));
            lo = __fadd_rn(lo, err);
            hi = sum;
        }
    }
    double acc = (double)hi + (double)lo;
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

// Multi-vertex estimator: pixel p gains the later-vertex terms of its M
// residual paths (units p M .. p M + M - 1), added in unit order.
__global__ void k_mv_accumulate(float4* __restrict__ out, float* __restrict__ lr, const float4* __restrict__ o2,
                                const float4* __restrict__ o3, uint64_t P, uint32_t M) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (uint64_t)gridDim.x * blockDim.x) {
        float3 a = make_float3(0.f, 0.f, 0.f);
        for (uint32_t j = 0; j < M; ++j) {
            const uint64_t u = p * M + j;
            if (o2) {
                const float4 v = o2[u];
                a.x += v.x;
                a.y += v.y;
                a.z += v.z;
            }
            if (o3) {
                const float4 v = o3[u];
                a.x += v.x;
                a.y += v.y;
                a.z += v.z;
            }
        }
        float4 o = out[p];
        out[p] = make_float4(o.x + a.x, o.y + a.y, o.z + a.z, o.w);
        if (lr) {
            lr[3 * p] += a.x;
            lr[3 * p + 1] += a.y;
            lr[3 * p + 2] += a.z;
        }
    }
}

cudaError_t launch_mv_accumulate(float* out_rgba, float* lr, const float4* o2, const float4* o3, uint64_t P,
                                 uint32_t M, cudaStream_t st) {
    if (P == 0 || (!o2 && !o3)) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (P + 255) / 256;
    if (blocks > (uint64_t)sms * 8) blocks = (uint64_t)sms * 8;
    k_mv_accumulate<<<(uint32_t)blocks, 256, 0, st>>>(reinterpret_cast<float4*>(out_rgba), lr, o2, o3, P, M);
    return cudaGetLastError();
}

cudaError_t launch_mrse(const float* img, const float* ref, uint64_t n, float eps, double* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
    if (e != cudaSuccess || n == 0) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (n + kMrseThreads - 1) / kMrseThreads;
    if (blocks > (uint64_t)sms * 8) blocks = (uint64_t)sms * 8;  // 8 blocks of 256 threads per SM
    k_mrse<<<(uint32_t)blocks, kMrseThreads, 0, st>>>(reinterpret_cast<const float4*>(img),
                                                      reinterpret_cast<const float4*>(ref), n, eps,
                                                      1.0 / (3.0 * (double)n), out);
    return cudaGetLastError();
}

}  // namespace nirc
