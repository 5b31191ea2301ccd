// nirc_gradw_tc.cu -- weight and bias gradients of the training step as
// tcgen05 MMAs.  For a layer with deltas delta [out][t] and inputs x [in][t]
// (both stored with the samples contiguous, i.e. K-major for K = samples):
//   D [o][i] = sum_t delta[o][t] x[i][t]   (i < in)   = dW
//   D [o][in] = sum_t delta[o][t]                       = db
// with A = the delta rows (M = 128: rows >= out are zero) and B = the input
// rows plus one row of ones (N = 80).  A CTA (two warpgroups) takes one
// layer and a slice of the samples, walks it in blocks of 64 samples (a
// 128-byte BF16 row), copying the stored BF16 values into a 128-byte
// swizzled operand stage while the MMA of the previous block runs, and adds
// its out x (in + 1) sums into the gradient with float atomics (warps 0-3,
// which own the accumulator's TMEM lanes).  Every mbarrier wait is bounded;
// a timeout sets *err.
#include "nirc_gradw_tc.h"
#include "nirc_tc.cuh"

namespace nirc {

namespace {

constexpr uint32_t kDwThreads = 256;  // two warpgroups share the loads; warps 0-3 own the TMEM lanes
constexpr uint32_t kDwBlock = 64;       // samples per operand block
constexpr uint32_t kDwN = 80;           // B rows: inputs, the ones row, zeros
constexpr uint32_t kDwA = 16384;        // 128 rows x 128 bytes
constexpr uint32_t kDwB = kDwN * 128;   // 80 rows x 128 bytes
constexpr uint32_t kDwStage = kDwA + kDwB;
constexpr uint32_t kDwSmem = 1024 + 2 * kDwStage + 64;

// Eight BF16 samples t .. t + 7 of a row (zeros past t1), packed in pairs.
template <bool kVec>
__device__ __forceinline__ uint4 load8(const uint16_t* __restrict__ src, uint64_t t, uint64_t t1) {
    if (kVec && t + 8 <= t1) return __ldg(reinterpret_cast<const uint4*>(src + t));
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t lo = t + 2 * k < t1 ? __ldg(src + t + 2 * k) : 0u;
        const uint32_t hi = t + 2 * k + 1 < t1 ? __ldg(src + t + 2 * k + 1) : 0u;
        w[k] = lo | (hi << 16);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

template <bool kVec>
__global__ void __launch_bounds__(kDwThreads) k_grad_w_tc(DwJobs jobs, uint64_t m, uint64_t slice, int* err) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const DwJob J = jobs.j[blockIdx.y];
    const uint64_t t0 = (uint64_t)blockIdx.x * slice;
    if (t0 >= m) return;  // uniform over the CTA, before any allocation
    const uint64_t t1 = t0 + slice < m ? t0 + slice : m;
    const uint32_t t = threadIdx.x, warp = t >> 5;
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (sbase - raw);
    const uint32_t misc = sbase + 2 * kDwStage;
    volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(gbase + 2 * kDwStage + 32);

    if (warp == 0) tc::tmem_alloc(misc + 32, 128);
    if (t == 0) {
        tc::mbar_init(misc, 1);
        tc::mbar_init(misc + 8, 1);
        tc::fence_mbar_init();
    }
    // both stages start as zeros; the ones row of B is written once
    {
        uint4* z = reinterpret_cast<uint4*>(gbase);
        for (uint32_t i = t; i < 2 * kDwStage / 16; i += kDwThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    {
        const uint32_t one2 = pack2<1>(1.f, 1.f);
        for (uint32_t i = t; i < 2 * 8; i += kDwThreads)
            sts_chunk(sbase + (i >> 3) * kDwStage + kDwA, J.in, i & 7u, one2, one2, one2, one2);
    }
    const uint32_t tmem = *tmem_holder;
    const uint32_t idesc = tc::idesc_f16(1, 128, kDwN);
    const uint32_t n_items = (J.out + J.in) * 8u;  // 16-byte chunks of one block
    const uint64_t n_blocks = (t1 - t0 + kDwBlock - 1) / kDwBlock;
    uint32_t phase[2] = {0u, 0u};
    bool abort = false;
    for (uint64_t c = 0; c < n_blocks; ++c) {
        const uint32_t s = (uint32_t)(c & 1u);
        const uint32_t tA = sbase + s * kDwStage, tB = tA + kDwA;
        if (c >= 2 && !abort) {  // the MMA that read this stage (block c - 2) has finished
            if (!tc::mbar_wait_bounded(misc + 8 * s, phase[s])) {
                abort = true;
                atomicExch(err, 1);
            }
            phase[s] ^= 1u;
            tc::fence_after_sync();
        }
        const uint64_t tb = t0 + c * kDwBlock;
        for (uint32_t it = t; it < n_items; it += kDwThreads) {
            const uint32_t row = it >> 3, ch = it & 7u;
            const bool is_a = row < J.out;
            const uint32_t r = is_a ? row : row - J.out;
            const uint16_t* src = is_a ? J.dl + (uint64_t)r * J.ld_dl : J.x + (uint64_t)r * J.ld_x;
            const uint4 v = load8<kVec>(src, tb + 8u * ch, t1);
            sts_chunk(is_a ? tA : tB, r, ch, v.x, v.y, v.z, v.w);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (t == 0 && !abort) {
            tc::fence_after_sync();
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k)
                tc::mma_f16(tmem, tc::sdesc(tA + 32u * k), tc::sdesc(tB + 32u * k), idesc, (c > 0 || k > 0) ? 1u : 0u);
            tc::mma_commit(misc + 8 * s);
        }
    }
    // the last commit covers every earlier MMA
    {
        const uint32_t s = (uint32_t)((n_blocks - 1) & 1u);
        abort = __syncthreads_or(abort ? 1 : 0) != 0;  // uniform from here on
        if (!abort && !tc::mbar_wait_bounded(misc + 8 * s, phase[s])) {
            abort = true;
            atomicExch(err, 1);
        }
        tc::fence_after_sync();
    }
    if (!abort && warp < 4) {
        // row t of D (TMEM lane t): 32 columns at a time; column `in` is the bias sum
        const uint32_t trow = tmem + ((32u * warp) << 16);
        float* gw = J.gw + (uint64_t)t * J.in;
#pragma unroll 1
        for (uint32_t c0 = 0; c0 < kDwN; c0 += 32) {
            uint32_t v[32];
            tc::tmem_ld32(trow + c0, v);
            tc::tmem_wait_ld();
            if (t < J.out) {
#pragma unroll
                for (uint32_t k = 0; k < 32; ++k) {
                    const uint32_t i = c0 + k;
                    if (i < J.in) atomicAdd(gw + i, __uint_as_float(v[k]));
                    else if (i == J.in) atomicAdd(J.gw + (uint64_t)J.out * J.in + t, __uint_as_float(v[k]));
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 128);
    }
}

}  // namespace

cudaError_t launch_grad_w_tc(const nirc_handle* h, const DwJobs& jobs, uint64_t m, cudaStream_t st) {
    if (m == 0 || jobs.n_jobs == 0) return cudaSuccess;
    bool vec = true;
    for (uint32_t l = 0; l < jobs.n_jobs; ++l) {
        const DwJob& J = jobs.j[l];
        if (J.out == 0 || J.out > 64 || J.in == 0 || J.in + 1 > kDwN) return cudaErrorInvalidValue;
        vec = vec && (J.ld_dl % 8 == 0) && (J.ld_x % 8 == 0) && (reinterpret_cast<uintptr_t>(J.dl) % 16 == 0) &&
              (reinterpret_cast<uintptr_t>(J.x) % 16 == 0);
    }
    // about four CTAs per SM over all jobs (54 KB of shared memory each: the loads of a block
    // are latency-bound), at least 512 samples each (a multiple of the block)
    const uint64_t want = (4ull * (uint64_t)h->num_sms + jobs.n_jobs - 1) / jobs.n_jobs;
    uint64_t slice = (m + want - 1) / want;
    if (slice < 512) slice = 512;
    slice = (slice + kDwBlock - 1) / kDwBlock * kDwBlock;
    const dim3 grid((uint32_t)((m + slice - 1) / slice), jobs.n_jobs);
    auto kern = vec ? k_grad_w_tc<true> : k_grad_w_tc<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwSmem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kDwThreads, kDwSmem, st>>>(jobs, m, slice, h->dev_err);
    count_kernels(h);
    return cudaGetLastError();
}

}  // namespace nirc
