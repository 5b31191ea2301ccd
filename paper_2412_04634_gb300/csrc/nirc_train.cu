// nirc_train.cu -- on-line training step of the cache (FP32 SIMT) and the
// backward pass of the bare query.
//
// Loss: relative L2 of eq. 12 with p_r = 1,
//   L = 1/(3n) sum_t sum_rgb valid_t (f - n)^2 / (sg(n)^2 + eps),
// so dL/dn = -2 (f - n) / ((n^2 + eps) 3n) with the denominator held
// constant (stop-gradient), and dL/dz = dL/dn * n below the output clamp.
// The query backward takes dL/dn from the caller instead (every row counts).
//
//  k_train_fwd   per sample: encoding, layers, loss, dL/dz; optionally the
//                network input and ReLU outputs as [feature][sample]
//                columns (coalesced) for the backward
//  k_train_bwd   per sample: deltas through the ReLU layers (transposed
//                weights in shared memory), then the hash-feature gradient
//                scattered into the table gradient with one float2 atomic
//                for both features of an entry; on the coarse dense levels
//                (few cells, many samples per cell) lanes of a warp that hit
//                the same entry are combined first (__match_any_sync) and
//                only the group leader issues the atomic
//  dW, db        per layer: dW = delta x^T and db = delta 1, a plain GEMM
//                and GEMV over the samples: k_grad_w (4x4 register tiles
//                over 32-sample chunks staged in shared memory, combined by
//                float atomics, or in deterministic mode by block partials
//                summed in a fixed order); passes of >= 2^18 samples in the
//                default mode use k_grad_w_big (a block per layer and slice
//                of the samples, double-buffered stages of 64 samples)
//  k_adam        dense bias-corrected Adam over every parameter (untouched
//                hash entries have g = 0), FP32 master weights and moments,
//                FP16 copy of the hash table refreshed in the same pass
//
// Deterministic mode (nirc_set_deterministic): identical inputs give
// bit-identical losses, gradients and weights whatever the scheduling.  Block
// partial sums of the loss and of dW are written out and added in a fixed
// order; the hash-table gradient goes through a separate pass: the backward
// stores dL/de per sample and level with the level's max |dL/de|, then
// k_hash_scatter_fixed adds w * dL/de into 64-bit fixed-point accumulators
// (integer atomics are order-independent) with a power-of-two scale per level
// chosen so that no entry can overflow, and k_hash_fixed_to_float converts
// them back.  Each contribution keeps FP32 relative precision; the sum is
// exact.
//
// Activations: stored (one forward writes every layer's output for the whole
// batch, n x (n_in + 2 x 64 x hidden) floats) or recomputed (the first
// forward keeps only dL/dz; the batch is then walked in chunks whose
// forward is run again with stores into a chunk-sized buffer, followed by
// that chunk's backward and weight gradients).  Recomputation trades one
// extra forward for O(chunk) instead of O(n) activation memory; a chunk of
// 2^15 samples keeps the activation buffer (~78 MB) inside the 129 MB L2.
#include <cmath>

#include "nirc_gradw_tc.h"
#include "nirc_internal.h"
#include "nirc_simt.cuh"

namespace nirc {

constexpr int kTrainThreads = 128;
constexpr int kGradChunk = 32;
constexpr int kGradThreads = 352;  // 16 x 22 tiles of 4 x 4

// Column-major per-sample buffers.  e / act / delta hold `ld` samples (the
// whole batch when stored, one chunk when recomputed); dz covers the whole
// batch with its own leading dimension, already offset to the launch's first
// sample.

enum LossKind : int {
    kLossRelL2 = 0,    // eq. 12 against targets, valid records only
    kLossUpstream = 1, // dL/dn given per row (query backward), every row
    kLossNone = 2      // recompute pass: dz already known
};

static uint64_t act_floats_per_sample(const NetShape& s) { return (uint64_t)s.n_in + 2ull * kWidth * s.hidden; }

static uint64_t chunk_of(const nirc_handle* h, uint64_t n) {
    return h->store_activations ? n : (n < h->recompute_chunk ? n : h->recompute_chunk);
}

static uint64_t round64(uint64_t floats) { return (floats + 63) & ~63ull; }

// Extra buffers of deterministic mode (all offsets 256-byte aligned).
struct DetPtrs {
    float* de;                 // [2 levels][n]: dL/de of the hash features
    unsigned* lvl_max;         // [16]: max |dL/de| per level (float bits)
    float* loss_part;          // [grid]: per-block loss sums
    float* gw_part;            // [gx][n_mlp]: per-block weight gradients
    unsigned long long* acc;   // [n_hash]: fixed-point hash gradient
};

static uint64_t max_grad_blocks(const nirc_handle* h) { return 2ull * (uint64_t)h->num_sms + 1; }
// Forward / backward grids: at most two 128-thread blocks per SM.
static uint64_t max_train_blocks(const nirc_handle* h) { return 2ull * (uint64_t)h->num_sms; }

static uint64_t det_floats(const nirc_handle* h, uint64_t n) {
    const NetShape& s = h->shape;
    return round64(2ull * s.levels * n) + 64 + round64(max_train_blocks(h)) + round64(max_grad_blocks(h) * s.n_mlp) +
           2 * round64(s.n_hash);
}

size_t train_scratch_bytes(const nirc_handle* h, uint64_t n) {
    const uint64_t c = chunk_of(h, n);
    uint64_t f = round64(3 * n + c * act_floats_per_sample(h->shape));
    if (h->deterministic) f += det_floats(h, n);
    return (size_t)f * sizeof(float) + 256;
}

// From this many samples per pass on, the sliced k_grad_w_big computes the
// weight gradients (k_grad_w's one 32-sample chunk per block iteration leaves
// it bound by its loads and barriers on long passes).
constexpr uint64_t kGradBigMinSamples = 1ull << 18;

static TrainPtrs carve(void* base, const NetShape& s, uint64_t n, uint64_t chunk) {
    float* f = reinterpret_cast<float*>(base);
    TrainPtrs t;
    t.dz = f;
    t.dz_ld = n;
    t.e = f + 3 * n;
    t.act = t.e + (size_t)s.n_in * chunk;
    t.delta = t.act + (size_t)s.hidden * kWidth * chunk;
    t.ld = chunk;
    return t;
}

static DetPtrs carve_det(const nirc_handle* h, void* base, uint64_t n, uint64_t chunk) {
    const NetShape& s = h->shape;
    float* f = reinterpret_cast<float*>(base) + round64(3 * n + chunk * act_floats_per_sample(s));
    DetPtrs d;
    d.de = f;
    f += round64(2ull * s.levels * n);
    d.lvl_max = reinterpret_cast<unsigned*>(f);
    f += 64;
    d.loss_part = f;
    f += round64(max_train_blocks(h));
    d.gw_part = f;
    f += round64(max_grad_blocks(h) * s.n_mlp);
    d.acc = reinterpret_cast<unsigned long long*>(f);
    return d;
}

// Power-of-two scale of level sums: every entry receives at most 8 n
// contributions of magnitude <= m, so |sum| * scale < 2^61.
__device__ __forceinline__ float fixed_scale(float m, uint64_t n) {
    if (!(m > 0.f)) return 1.f;
    int e = 0;
    frexpf(8.f * (float)n * m, &e);
    return ldexpf(1.f, min(61 - e, 100));
}

template <bool kSh>
__global__ void __launch_bounds__(kTrainThreads, 2)
    k_train_fwd(NetShape s, GridParams g, float z_clamp, float loss_eps, float scale, const float* __restrict__ packed,
                const float* __restrict__ table, const nirc_record* __restrict__ recs, const float* __restrict__ dirs,
                const float* __restrict__ targets, uint64_t n, TrainPtrs tp, int store, int kind,
                float* __restrict__ loss_accum, float* __restrict__ loss_part) {
    extern __shared__ __align__(16) float smem[];
    __shared__ float warp_loss[kTrainThreads / 32];
    float loss_run = 0.f;  // this lane's warp sums over the iterations (lane 0)
    float* sw = smem;
    float* act = smem + s.packed_floats + threadIdx.x;
    const int stride = kTrainThreads;
    stage_weights(sw, packed, s.packed_floats);
    __syncthreads();
    // Uniform trip count per block: the loss reduction below uses full-warp shuffles.
    for (uint64_t first = (uint64_t)blockIdx.x * kTrainThreads; first < n; first += (uint64_t)gridDim.x * kTrainThreads) {
        const bool in_range = first + threadIdx.x < n;
        const uint64_t t = in_range ? first + threadIdx.x : 0;
        const float4* rq = reinterpret_cast<const float4*>(recs + t);
        const float4 r0 = __ldg(rq), r1 = __ldg(rq + 1), r2 = __ldg(rq + 2), r3 = __ldg(rq + 3);
        const bool valid = in_range && (kind == kLossUpstream || (__float_as_uint(r3.z) & 1u));
        const bool keep = in_range && store;
        const V3 p{r0.x, r0.y, r0.z}, nn{r0.w, r1.x, r1.y};
        const V3 wi{__ldg(dirs + 3 * t), __ldg(dirs + 3 * t + 1), __ldg(dirs + 3 * t + 2)};
        encode_surface(s, g, table, p, nn, make_float3(r2.y, r2.z, r2.w), r3.x, act, stride);  // [pos][surf]
        constexpr int nd = dir_features<kSh>();
        float edir[nd];
        dir_encode<kSh>(wi, edir);
        // network input in parameter order [pos][dir][surf]
        if (keep) {
            const uint64_t ld = tp.ld;
            for (uint32_t k = 0; k < s.n_pos; ++k) tp.e[(uint64_t)k * ld + t] = act[k * stride];
#pragma unroll
            for (uint32_t k = 0; k < (uint32_t)nd; ++k) tp.e[(uint64_t)(s.n_pos + k) * ld + t] = edir[k];
            for (uint32_t k = 0; k < s.n_surf; ++k)
                tp.e[(uint64_t)(s.n_pos + nd + k) * ld + t] = act[(s.n_pos + k) * stride];
        }

        float2 acc[32];
        load_bias(acc, sw + s.off_b0);
        for (uint32_t i = 0; i < s.n_pix; ++i) fma_row(acc, sw + s.off_wpix + i * kWidth, act[i * stride]);
#pragma unroll
        for (int i = 0; i < nd; ++i) fma_row(acc, sw + s.off_wdir + i * kWidth, edir[i]);
        for (uint32_t l = 0; l < s.hidden; ++l) {
            float* ag = tp.act + ((uint64_t)l * kWidth) * tp.ld + t;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const float a0 = fmaxf(acc[q].x, 0.f), a1 = fmaxf(acc[q].y, 0.f);
                if (keep) {
                    ag[(uint64_t)(2 * q) * tp.ld] = a0;
                    ag[(uint64_t)(2 * q + 1) * tp.ld] = a1;
                }
                act[(2 * q) * stride] = a0;
                act[(2 * q + 1) * stride] = a1;
            }
            if (l + 1 == s.hidden) break;
            const float* Wl = sw + s.off_hidden + l * (kWidth * kWidth + kWidth);
            load_bias(acc, Wl + kWidth * kWidth);
#pragma unroll 2
            for (int i = 0; i < (int)kWidth; ++i) fma_row(acc, Wl + i * kWidth, act[i * stride]);
        }
        const float* Wo = sw + s.off_out;
        float z[3] = {Wo[256], Wo[257], Wo[258]};
        for (int i = 0; i < (int)kWidth; ++i) {
            const float a = act[i * stride];
            z[0] += Wo[4 * i] * a;
            z[1] += Wo[4 * i + 1] * a;
            z[2] += Wo[4 * i + 2] * a;
        }
        if (kind == kLossNone) continue;  // block-uniform
        float lt = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // radiance: n = exp(min(z, clamp)), dn/dz = n below the clamp; visibility: V = sigmoid(z), dV/dz = V (1 - V)
            const bool clamped = !s.vis && !(z[c] <= z_clamp);
            const float nv = out_act(s.vis, z[c], z_clamp);
            const float dact = s.vis ? nv * (1.f - nv) : (clamped ? 0.f : nv);
            const float f = in_range ? __ldg(targets + 3 * t + c) : 0.f;
            float dz = 0.f;
            if (kind == kLossUpstream) {
                // f holds dL/dn; the accumulated value is sum dL/dn * n
                if (valid) {
                    lt += f * nv;
                    dz = f * dact;
                }
            } else if (s.vis) {
                // visibility: plain L2, (f - V)^2
                const float diff = f - nv;
                if (valid) {
                    lt += diff * diff * scale;
                    dz = -2.f * diff * scale * dact;
                }
            } else {
                const float den = nv * nv + loss_eps;
                const float diff = f - nv;
                if (valid) {
                    lt += diff * diff / den * scale;
                    dz = -2.f * diff / den * scale * dact;
                }
            }
            if (in_range) tp.dz[(uint64_t)c * tp.dz_ld + t] = dz;
        }
        for (int o = 16; o > 0; o >>= 1) lt += __shfl_xor_sync(0xffffffffu, lt, o);
        loss_run += lt;
    }
    if (kind == kLossNone) return;
    // block sum in a fixed order: one atomic per block, or one partial per
    // block in deterministic mode
    if ((threadIdx.x & 31) == 0) warp_loss[threadIdx.x >> 5] = loss_run;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < kTrainThreads / 32; ++w) b += warp_loss[w];
        if (loss_part) loss_part[blockIdx.x] = b;
        else if (loss_accum) atomicAdd(loss_accum, b);
    }
}

__device__ __forceinline__ float dot64(const float* __restrict__ wrow, const float (&d)[64]) {
    const float4* w4 = reinterpret_cast<const float4*>(wrow);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float4 w = w4[q];
        s0 += w.x * d[4 * q];
        s1 += w.y * d[4 * q + 1];
        s2 += w.z * d[4 * q + 2];
        s3 += w.w * d[4 * q + 3];
    }
    return (s0 + s1) + (s2 + s3);
}

__global__ void __launch_bounds__(kTrainThreads, 2)
    k_train_bwd(NetShape s, GridParams g, const float* __restrict__ packed, const nirc_record* __restrict__ recs,
                uint64_t n, TrainPtrs tp, int all_records, float* __restrict__ grad_table, float* __restrict__ de_out,
                uint64_t de_ld, unsigned* __restrict__ lvl_max) {
    extern __shared__ __align__(16) float smem[];
    float* sw = smem;
    stage_weights(sw, packed, s.packed_floats);
    __syncthreads();
    const uint64_t ld = tp.ld;
    // Uniform trip count per block: the hash scatter uses full-warp collectives.
    for (uint64_t first = (uint64_t)blockIdx.x * kTrainThreads; first < n; first += (uint64_t)gridDim.x * kTrainThreads) {
        const bool in_range = first + threadIdx.x < n;
        const uint64_t t = in_range ? first + threadIdx.x : first;
        const float dz0 = tp.dz[t], dz1 = tp.dz[tp.dz_ld + t], dz2 = tp.dz[2 * tp.dz_ld + t];
        float d[64];
        const float* Wo = sw + s.off_out;
        const uint32_t H = s.hidden;
        {
            const float* ag = tp.act + ((uint64_t)(H - 1) * kWidth) * ld + t;
            float* dg = tp.delta + ((uint64_t)(H - 1) * kWidth) * ld + t;
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                const float4 w = *reinterpret_cast<const float4*>(Wo + 4 * i);
                const float v = w.x * dz0 + w.y * dz1 + w.z * dz2;
                d[i] = ag[(uint64_t)i * ld] > 0.f ? v : 0.f;
                if (in_range) dg[(uint64_t)i * ld] = d[i];
            }
        }
        for (int l = (int)H - 1; l >= 1; --l) {
            // delta_{l-1}[i] = (sum_o W_l[o][i] delta_l[o]) [act_{l-1}[i] > 0]; W_l^T row i = W_l[:, i]
            const float* Wl = sw + s.off_hidden + (l - 1) * (kWidth * kWidth + kWidth);
            const float* ag = tp.act + ((uint64_t)(l - 1) * kWidth) * ld + t;
            float* dg = tp.delta + ((uint64_t)(l - 1) * kWidth) * ld + t;
            float dn[64];
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                const float v = dot64(Wl + i * kWidth, d);
                dn[i] = ag[(uint64_t)i * ld] > 0.f ? v : 0.f;
            }
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                d[i] = dn[i];
                if (in_range) dg[(uint64_t)i * ld] = dn[i];
            }
        }
        if (s.hashgrid) {
            const float4* rq = reinterpret_cast<const float4*>(recs + t);
            const float4 r0 = __ldg(rq), r3 = __ldg(rq + 3);
            const bool valid = in_range && (all_records || (__float_as_uint(r3.z) & 1u));
            const V3 p{r0.x, r0.y, r0.z};
            const uint64_t T = (uint64_t)g.mask + 1;
            for (uint32_t l = 0; l < g.n_levels; ++l) {
                // dL/de for the two features of level l: W0[:, k] = Wpix^T row k
                const float de0 = dot64(sw + s.off_wpix + (2 * l) * kWidth, d);
                const float de1 = dot64(sw + s.off_wpix + (2 * l + 1) * kWidth, d);
                if (de_out) {
                    // deterministic mode: k_hash_scatter_fixed adds these later
                    const float a0 = valid ? de0 : 0.f, a1 = valid ? de1 : 0.f;
                    if (in_range) {
                        de_out[(uint64_t)(2 * l) * de_ld + t] = a0;
                        de_out[(uint64_t)(2 * l + 1) * de_ld + t] = a1;
                    }
                    const unsigned mx = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(fabsf(a0), fabsf(a1))));
                    if ((threadIdx.x & 31) == 0) atomicMax(lvl_max + l, mx);
                    continue;
                }
                uint32_t idx[8];
                float w[8];
                grid_corners(g.level[l], g.mask, p, idx, w);
                float* gt = grad_table + (uint64_t)l * T * 2;
                if (g.level[l].dense) {
                    // coarse levels: few cells, many samples per cell
#pragma unroll
                    for (int c = 0; c < 8; ++c) scatter_pair(gt, idx[c], valid, w[c] * de0, w[c] * de1);
                } else if (valid) {
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        atomicAdd(reinterpret_cast<float2*>(gt + 2 * (uint64_t)idx[c]),
                                  make_float2(w[c] * de0, w[c] * de1));
                }
            }
        }
    }
}

// Deterministic hash-table gradient: acc[l][idx][f] += w * dL/de[l][f] *
// scale_l as 64-bit integers.
__global__ void __launch_bounds__(256)
    k_hash_scatter_fixed(GridParams g, const nirc_record* __restrict__ recs, uint64_t n,
                         const float* __restrict__ de, const unsigned* __restrict__ lvl_max,
                         unsigned long long* __restrict__ acc) {
    const uint64_t T = (uint64_t)g.mask + 1;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        const float4 r0 = __ldg(reinterpret_cast<const float4*>(recs + t));
        const V3 p{r0.x, r0.y, r0.z};
        for (uint32_t l = 0; l < g.n_levels; ++l) {
            const float de0 = de[(uint64_t)(2 * l) * n + t], de1 = de[(uint64_t)(2 * l + 1) * n + t];
            if (de0 == 0.f && de1 == 0.f) continue;
            const float sc = fixed_scale(__uint_as_float(lvl_max[l]), n);
            uint32_t idx[8];
            float w[8];
            grid_corners(g.level[l], g.mask, p, idx, w);
            unsigned long long* a = acc + (uint64_t)l * T * 2;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const long long v0 = __float2ll_rn(w[c] * de0 * sc), v1 = __float2ll_rn(w[c] * de1 * sc);
                if (v0) atomicAdd(a + 2 * (uint64_t)idx[c], (unsigned long long)v0);
                if (v1) atomicAdd(a + 2 * (uint64_t)idx[c] + 1, (unsigned long long)v1);
            }
        }
    }
}

__global__ void k_hash_fixed_to_float(GridParams g, uint64_t n, const unsigned* __restrict__ lvl_max,
                                      const unsigned long long* __restrict__ acc, float* __restrict__ grad_table) {
    const uint64_t per_level = ((uint64_t)g.mask + 1) * 2;
    const uint64_t total = per_level * g.n_levels;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t l = (uint32_t)(i / per_level);
        const float inv = 1.f / fixed_scale(__uint_as_float(lvl_max[l]), n);  // power of two: exact
        grad_table[i] = __ll2float_rn((long long)acc[i]) * inv;
    }
}

// dst[j] (+)= sum_r src[r * cols + j] over r = 0..rows-1 in order.
__global__ void k_sum_rows(const float* __restrict__ src, uint64_t rows, uint64_t cols, float* __restrict__ dst,
                           int accumulate) {
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cols; j += (uint64_t)gridDim.x * blockDim.x) {
        float v = accumulate ? dst[j] : 0.f;
        for (uint64_t r = 0; r < rows; ++r) v += src[r * cols + j];
        dst[j] = v;
    }
}

struct GradJob {
    const float* dl;  // [out][ld_dl]
    const float* x;   // [in][ld_x]
    float* gw;        // W [out][in] followed by b [out]
    uint64_t ld_dl, ld_x;
    uint32_t out, in;
};
struct GradJobs {
    GradJob j[kMaxHidden + 1];
    float* part;     // deterministic mode: block b writes W/b of job l at
    uint64_t pstride;//   part + b * pstride + (gw - grad); else atomics into gw
    const float* grad_base;
};

template <bool kPartial>
__global__ void __launch_bounds__(kGradThreads) k_grad_w(GradJobs jobs, uint64_t n) {
    const GradJob J = jobs.j[blockIdx.y];
    __shared__ __align__(16) float ds[kGradChunk][64 + 4];
    __shared__ __align__(16) float xs[kGradChunk][88 + 4];
    const int tid = threadIdx.x;
    const int ot = tid / 22, it = tid % 22;
    float acc[4][4] = {};
    for (int k = tid; k < kGradChunk * (64 + 4); k += kGradThreads) (&ds[0][0])[k] = 0.f;
    for (int k = tid; k < kGradChunk * (88 + 4); k += kGradThreads) (&xs[0][0])[k] = 0.f;
    const uint64_t n_chunks = (n + kGradChunk - 1) / kGradChunk;
    for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const uint64_t t0 = c * kGradChunk;
        __syncthreads();
        for (int k = tid; k < (int)J.out * kGradChunk; k += kGradThreads) {
            const int o = k / kGradChunk, tt = k % kGradChunk;
            ds[tt][o] = t0 + tt < n ? J.dl[(uint64_t)o * J.ld_dl + t0 + tt] : 0.f;
        }
        for (int k = tid; k < (int)J.in * kGradChunk; k += kGradThreads) {
            const int i = k / kGradChunk, tt = k % kGradChunk;
            xs[tt][i] = t0 + tt < n ? J.x[(uint64_t)i * J.ld_x + t0 + tt] : 0.f;
        }
        for (int tt = tid; tt < kGradChunk; tt += kGradThreads) xs[tt][J.in] = 1.f;  // bias column
        __syncthreads();
        if (4 * ot < (int)J.out && 4 * it <= (int)J.in) {
#pragma unroll 8
            for (int tt = 0; tt < kGradChunk; ++tt) {
                const float4 dv = *reinterpret_cast<const float4*>(&ds[tt][4 * ot]);
                const float4 xv = *reinterpret_cast<const float4*>(&xs[tt][4 * it]);
                const float da[4] = {dv.x, dv.y, dv.z, dv.w}, xa[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] += da[a] * xa[b];
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int o = 4 * ot + a, i = 4 * it + b;
            if (o < (int)J.out && i <= (int)J.in) {
                float* dst = i < (int)J.in ? J.gw + (uint64_t)o * J.in + i : J.gw + (uint64_t)J.out * J.in + o;
                if constexpr (kPartial) jobs.part[blockIdx.x * jobs.pstride + (uint64_t)(dst - jobs.grad_base)] = acc[a][b];
                else atomicAdd(dst, acc[a][b]);
            }
        }
}

// Weight and bias gradients of passes of many samples (FP32): one block per
// (layer, slice of the samples) accumulates the whole dW | db tile of its
// layer over its slice and adds it into the gradient with float atomics at
// the end.  The samples stream through shared memory in stages of 64 in the
// [feature][sample] layout of the stored columns (coalesced loads, the next
// stage's loads in flight in registers while the current one is consumed);
// thread (ot, it) owns outputs 4 ot .. 4 ot + 3 and inputs it + 16 b
// (b < 6, the input after the last one being the bias row of ones), and
// reads 4 consecutive samples of each with one 16-byte shared load.
constexpr int kGwStage = 64;
constexpr int kGwThreads = 256;
constexpr int kGwRowPad = kGwStage + 4;  // 68 floats: 16-byte rows, rows of consecutive `it` on distinct banks
constexpr int kGwDsFloats = 64 * kGwRowPad;
constexpr int kGwDsLoads = 64 * kGwStage / kGwThreads;  // 16
// NB input groups of 16 rows: inputs + bias row <= 16 NB (5 for up to 79 inputs, 6 for up to 95)
template <int NB>
constexpr size_t gw_smem_bytes() { return 2 * (size_t)(kGwDsFloats + 16 * NB * kGwRowPad) * sizeof(float); }

template <int NB>
__global__ void __launch_bounds__(kGwThreads, 2) k_grad_w_big(GradJobs jobs, uint64_t n, uint64_t slice) {
    constexpr int kGwXsFloats = 16 * NB * kGwRowPad;
    constexpr int kGwXsLoads = kGwStage * 16 * NB / kGwThreads;  // 4 NB
    const GradJob J = jobs.j[blockIdx.y];
    extern __shared__ __align__(16) float gw_smem[];
    const int tid = threadIdx.x, ot = tid >> 4, it = tid & 15;
    const uint64_t t_begin = (uint64_t)blockIdx.x * slice;
    const uint64_t t_end = t_begin + slice < n ? t_begin + slice : n;
    if (t_begin >= t_end) return;
    const int xrows = (int)J.in + 1;  // inputs and the bias row
    // rows the layer does not use stay zero in both buffers
    for (int k = tid; k < 2 * (kGwDsFloats + kGwXsFloats); k += kGwThreads) gw_smem[k] = 0.f;
    float rd[kGwDsLoads], rx[kGwXsLoads];
    auto fetch = [&](uint64_t t0) {
#pragma unroll
        for (int q = 0; q < kGwDsLoads; ++q) {
            const int idx = tid + kGwThreads * q, o = idx / kGwStage;
            const uint64_t t = t0 + (uint64_t)(idx % kGwStage);
            rd[q] = (o < (int)J.out && t < t_end) ? __ldg(J.dl + (uint64_t)o * J.ld_dl + t) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < kGwXsLoads; ++q) {
            const int idx = tid + kGwThreads * q, i = idx / kGwStage;
            const uint64_t t = t0 + (uint64_t)(idx % kGwStage);
            float v = 0.f;
            if (t < t_end) v = i < (int)J.in ? __ldg(J.x + (uint64_t)i * J.ld_x + t) : (i == (int)J.in ? 1.f : 0.f);
            rx[q] = v;
        }
    };
    auto stash = [&](int buf) {
        float* ds = gw_smem + buf * (kGwDsFloats + kGwXsFloats);
        float* xs = ds + kGwDsFloats;
#pragma unroll
        for (int q = 0; q < kGwDsLoads; ++q) {
            const int idx = tid + kGwThreads * q;
            ds[(idx / kGwStage) * kGwRowPad + idx % kGwStage] = rd[q];
        }
#pragma unroll
        for (int q = 0; q < kGwXsLoads; ++q) {
            const int idx = tid + kGwThreads * q, i = idx / kGwStage;
            if (i < xrows) xs[i * kGwRowPad + idx % kGwStage] = rx[q];
        }
    };
    float acc[4][NB] = {};
    fetch(t_begin);
    __syncthreads();  // the zero fill before the first stash
    stash(0);
    __syncthreads();
    int buf = 0;
    for (uint64_t t0 = t_begin; t0 < t_end; t0 += kGwStage) {
        const bool more = t0 + kGwStage < t_end;
        if (more) fetch(t0 + kGwStage);
        const float* ds = gw_smem + buf * (kGwDsFloats + kGwXsFloats);
        const float* xs = ds + kGwDsFloats;
#pragma unroll 4
        for (int tt = 0; tt < kGwStage; tt += 4) {
            float4 d[4], x[NB];
#pragma unroll
            for (int a = 0; a < 4; ++a) d[a] = *reinterpret_cast<const float4*>(ds + (4 * ot + a) * kGwRowPad + tt);
#pragma unroll
            for (int b = 0; b < NB; ++b) x[b] = *reinterpret_cast<const float4*>(xs + (it + 16 * b) * kGwRowPad + tt);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    acc[a][b] += d[a].x * x[b].x + d[a].y * x[b].y + d[a].z * x[b].z + d[a].w * x[b].w;
        }
        if (more) {
            stash(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int o = 4 * ot + a, i = it + 16 * b;
            if (o < (int)J.out && i <= (int)J.in)
                atomicAdd(i < (int)J.in ? J.gw + (uint64_t)o * J.in + i : J.gw + (uint64_t)J.out * J.in + o, acc[a][b]);
        }
}

// Dense bias-corrected Adam over all parameters, four at a time (16-byte
// loads and stores of the 256-byte aligned arrays); the FP16 copy of the
// hash table follows its entries.
__device__ __forceinline__ float adam_one(float gi, float& mi, float& vi, float pi, float lr, float b1, float b2,
                                          float eps, float inv_bc1, float inv_bc2) {
    mi = b1 * mi + (1.f - b1) * gi;
    vi = b2 * vi + (1.f - b2) * gi * gi;
    return pi - lr * (mi * inv_bc1) / (sqrtf(vi * inv_bc2) + eps);
}

__global__ void k_adam(uint64_t n_params, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float inv_bc1,
                       float inv_bc2, __half* __restrict__ hash16, uint64_t hash_off) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n4 = n_params / 4;
    for (uint64_t q = tid; q < n4; q += stride) {
        const float4 g4 = reinterpret_cast<const float4*>(g)[q];
        float4 m4 = reinterpret_cast<const float4*>(m)[q];
        float4 v4 = reinterpret_cast<const float4*>(v)[q];
        float4 p4 = reinterpret_cast<const float4*>(p)[q];
        p4.x = adam_one(g4.x, m4.x, v4.x, p4.x, lr, b1, b2, eps, inv_bc1, inv_bc2);
        p4.y = adam_one(g4.y, m4.y, v4.y, p4.y, lr, b1, b2, eps, inv_bc1, inv_bc2);
        p4.z = adam_one(g4.z, m4.z, v4.z, p4.z, lr, b1, b2, eps, inv_bc1, inv_bc2);
        p4.w = adam_one(g4.w, m4.w, v4.w, p4.w, lr, b1, b2, eps, inv_bc1, inv_bc2);
        reinterpret_cast<float4*>(m)[q] = m4;
        reinterpret_cast<float4*>(v)[q] = v4;
        reinterpret_cast<float4*>(p)[q] = p4;
        if (hash16) {
            const uint64_t i = 4 * q;
            const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (i + k >= hash_off) hash16[i + k - hash_off] = __float2half_rn(pv[k]);
        }
    }
    for (uint64_t i = 4 * n4 + tid; i < n_params; i += stride) {
        float mi = m[i], vi = v[i];
        const float pi = adam_one(g[i], mi, vi, p[i], lr, b1, b2, eps, inv_bc1, inv_bc2);
        m[i] = mi;
        v[i] = vi;
        p[i] = pi;
        if (hash16 && i >= hash_off) hash16[i - hash_off] = __float2half_rn(pi);
    }
}

__global__ void k_hash_to_half(uint64_t n, const float* __restrict__ src, __half* __restrict__ dst) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = __float2half_rn(src[i]);
}

cudaError_t launch_hash_to_half(const nirc_handle* h, cudaStream_t st) {
    if (!h->shape.n_hash || !h->hash16) return cudaSuccess;
    k_hash_to_half<<<4 * h->num_sms, 256, 0, st>>>(h->shape.n_hash, h->params + h->shape.hash_off, h->hash16);
    count_kernels(h);
    return cudaGetLastError();
}

// Forward, backward and weight gradients of n samples into h->grad (zeroed
// first); the loss (or sum dL/dn * n) lands in h->loss_accum.
static cudaError_t train_pass(nirc_handle* h, const nirc_record* recs, const float* dirs, const float* targets,
                              uint64_t n, int kind, cudaStream_t st) {
    const NetShape& s = h->shape;
    const uint64_t chunk = chunk_of(h, n);
    const bool store = chunk == n;
    TrainPtrs tp = carve(h->train_scratch, s, n, chunk);
    const bool det = h->deterministic != 0;
    const bool det_hash = det && s.hashgrid;
    DetPtrs dp{};
    if (det) dp = carve_det(h, h->train_scratch, n, chunk);
    cudaError_t e;
    if ((e = cudaMemsetAsync(h->grad, 0, s.n_dev * sizeof(float), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(h->loss_accum, 0, sizeof(float), st)) != cudaSuccess) return e;
    if (det_hash) {
        if ((e = cudaMemsetAsync(dp.lvl_max, 0, 64 * sizeof(unsigned), st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(dp.acc, 0, s.n_hash * sizeof(unsigned long long), st)) != cudaSuccess) return e;
    }
    const size_t smem_f = (size_t)s.packed_floats * 4 + (size_t)kTrainThreads * kWidth * 4;
    const size_t smem_b = (size_t)s.packed_floats * 4;
    auto fwd = s.sh ? k_train_fwd<true> : k_train_fwd<false>;
    if ((e = cudaFuncSetAttribute(fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_train_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b)) != cudaSuccess)
        return e;
    const float scale = 1.0f / (3.0f * (float)n);
    const float* table = h->params + s.hash_off;
    auto blocks_for = [&](uint64_t m) {  // two 128-thread blocks per SM fit (shared memory and registers)
        uint64_t b = (m + kTrainThreads - 1) / kTrainThreads;
        return (uint32_t)(b > max_train_blocks(h) ? max_train_blocks(h) : b);
    };
    // tensor-core training (nirc_set_train_precision): forward, loss and
    // backward of each chunk in one kernel, weight gradients as below
    const bool tcmode = kind == kLossRelL2 && train_tc_supported(h);
    if (!tcmode) {
        // full-batch forward: loss and dL/dz, activations only when stored
        timer_begin(h, NIRC_K_TRAIN_FWD, st);
        const uint32_t fwd_blocks = blocks_for(n);
        fwd<<<fwd_blocks, kTrainThreads, smem_f, st>>>(s, h->grid, h->cfg.z_clamp, h->cfg.loss_eps, scale, h->packed,
                                                      table, recs, dirs, targets, n, tp, store ? 1 : 0, kind,
                                                      h->loss_accum, det ? dp.loss_part : nullptr);
        count_kernels(h);
        timer_end(h, NIRC_K_TRAIN_FWD, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (det) {
            k_sum_rows<<<1, 32, 0, st>>>(dp.loss_part, fwd_blocks, 1, h->loss_accum, 0);
            count_kernels(h);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    for (uint64_t c0 = 0; c0 < n; c0 += chunk) {
        const uint64_t m = n - c0 < chunk ? n - c0 : chunk;
        TrainPtrs tc = tp;
        tc.dz = tp.dz + c0;
        if (tcmode) {
            timer_begin(h, NIRC_K_TRAIN_FWD, st);
            e = launch_train_tc(h, recs + c0, dirs + 3 * c0, targets + 3 * c0, m, scale, tc, h->grad + s.hash_off,
                                h->loss_accum, st);
            timer_end(h, NIRC_K_TRAIN_FWD, st);
            if (e != cudaSuccess) return e;
        } else if (!store) {
            timer_begin(h, NIRC_K_TRAIN_FWD, st);
            fwd<<<blocks_for(m), kTrainThreads, smem_f, st>>>(s, h->grid, h->cfg.z_clamp, h->cfg.loss_eps, scale,
                                                             h->packed, table, recs + c0, dirs + 3 * c0,
                                                             targets + 3 * c0, m, tc, 1, kLossNone, nullptr, nullptr);
            count_kernels(h);
            timer_end(h, NIRC_K_TRAIN_FWD, st);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (!tcmode) {
            timer_begin(h, NIRC_K_TRAIN_BWD, st);
            k_train_bwd<<<blocks_for(m), kTrainThreads, smem_b, st>>>(
                s, h->grid, h->packed, recs + c0, m, tc, kind == kLossUpstream ? 1 : 0, h->grad + s.hash_off,
                det_hash ? dp.de + c0 : nullptr, n, dp.lvl_max);
            count_kernels(h);
            timer_end(h, NIRC_K_TRAIN_BWD, st);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }

        // weight gradients, layer 0 = input layer
        GradJobs jobs;
        uint64_t off = 0;
        for (uint32_t l = 0; l <= s.hidden; ++l) {
            GradJob& J = jobs.j[l];
            J.out = l == s.hidden ? 3 : kWidth;
            J.in = l == 0 ? s.n_in : kWidth;
            J.dl = l == s.hidden ? tc.dz : tc.delta + (uint64_t)l * kWidth * tc.ld;
            J.ld_dl = l == s.hidden ? tc.dz_ld : tc.ld;
            J.x = l == 0 ? tc.e : tc.act + (uint64_t)(l - 1) * kWidth * tc.ld;
            J.ld_x = tc.ld;
            J.gw = h->grad + off;
            off += (uint64_t)J.out * J.in + J.out;
        }
        jobs.part = det ? dp.gw_part : nullptr;
        jobs.pstride = s.n_mlp;
        jobs.grad_base = h->grad;
        const uint64_t n_chunks = (m + kGradChunk - 1) / kGradChunk;
        uint64_t gx = (2ull * h->num_sms + s.hidden) / (s.hidden + 1);
        if (gx > n_chunks) gx = n_chunks;
        if (gx < 1) gx = 1;
        timer_begin(h, NIRC_K_TRAIN_GRADW, st);
        if (tcmode) {
            // tensor-core training: every layer's dW and db as BF16 MMAs in one launch
            DwJobs dj;
            dj.n_jobs = s.hidden + 1;
            // the tensor-core training kernel stored these buffers as BF16: element (row, sample)
            // of a buffer at its base + row * ld + sample, so the layers' offsets count 2-byte elements
            const uint16_t* e16 = reinterpret_cast<const uint16_t*>(tc.e);
            const uint16_t* act16 = reinterpret_cast<const uint16_t*>(tc.act);
            const uint16_t* delta16 = reinterpret_cast<const uint16_t*>(tc.delta);
            const uint16_t* dz16 = reinterpret_cast<const uint16_t*>(tc.dz);
            for (uint32_t l = 0; l <= s.hidden; ++l) {
                const GradJob& J = jobs.j[l];
                const uint16_t* dl = l == s.hidden ? dz16 : delta16 + (uint64_t)l * kWidth * tc.ld;
                const uint16_t* x = l == 0 ? e16 : act16 + (uint64_t)(l - 1) * kWidth * tc.ld;
                dj.j[l] = DwJob{dl, x, J.gw, J.ld_dl, J.ld_x, J.out, J.in};
            }
            if ((e = launch_grad_w_tc(h, dj, m, st)) != cudaSuccess) {
                timer_end(h, NIRC_K_TRAIN_GRADW, st);
                return e;
            }
        } else if (!det && (m < kGradBigMinSamples || s.n_in + 1 > 96)) {  // k_grad_w_big holds <= 95 inputs
            k_grad_w<false><<<dim3((uint32_t)gx, s.hidden + 1), kGradThreads, 0, st>>>(jobs, m);
            count_kernels(h);
        } else if (det) {
            k_grad_w<true><<<dim3((uint32_t)gx, s.hidden + 1), kGradThreads, 0, st>>>(jobs, m);
            count_kernels(h);
            if ((e = cudaGetLastError()) == cudaSuccess) {
                // chunks add their block partials into grad in chunk order
                k_sum_rows<<<(uint32_t)((s.n_mlp + 255) / 256), 256, 0, st>>>(dp.gw_part, gx, s.n_mlp, h->grad, 1);
                count_kernels(h);
            }
        } else {
            // long passes: one block per (layer, slice of about 4 per SM's share of the samples)
            uint64_t slice = (m * (s.hidden + 1) + 4ull * h->num_sms - 1) / (4ull * h->num_sms);
            slice = (slice + kGwStage - 1) / kGwStage * kGwStage;
            if (slice < 1024) slice = 1024;
            const uint64_t n_slices = (m + slice - 1) / slice;
            const bool nb5 = s.n_in + 1 <= 80;
            const size_t smem = nb5 ? gw_smem_bytes<5>() : gw_smem_bytes<6>();
            e = cudaFuncSetAttribute(nb5 ? k_grad_w_big<5> : k_grad_w_big<6>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) {
                timer_end(h, NIRC_K_TRAIN_GRADW, st);
                return e;
            }
            const dim3 grid((uint32_t)n_slices, s.hidden + 1);
            if (nb5) k_grad_w_big<5><<<grid, kGwThreads, smem, st>>>(jobs, m, slice);
            else k_grad_w_big<6><<<grid, kGwThreads, smem, st>>>(jobs, m, slice);
            count_kernels(h);
        }
        timer_end(h, NIRC_K_TRAIN_GRADW, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (det_hash) {
        timer_begin(h, NIRC_K_TRAIN_BWD, st);
        k_hash_scatter_fixed<<<4 * h->num_sms, 256, 0, st>>>(h->grid, recs, n, dp.de, dp.lvl_max, dp.acc);
        count_kernels(h);
        if ((e = cudaGetLastError()) == cudaSuccess) {
            k_hash_fixed_to_float<<<4 * h->num_sms, 256, 0, st>>>(h->grid, n, dp.lvl_max, dp.acc,
                                                                  h->grad + s.hash_off);
            count_kernels(h);
        }
        timer_end(h, NIRC_K_TRAIN_BWD, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_train_step(nirc_handle* h, const nirc_record* recs, const float* dirs, const float* targets,
                              uint64_t n, float* d_loss, cudaStream_t st) {
    const NetShape& s = h->shape;
    cudaError_t e = train_pass(h, recs, dirs, targets, n, kLossRelL2, st);
    if (e != cudaSuccess) return e;
    h->step += 1;
    const double b1 = h->cfg.beta1, b2 = h->cfg.beta2;
    const float inv_bc1 = (float)(1.0 / (1.0 - std::pow(b1, (double)h->step)));
    const float inv_bc2 = (float)(1.0 / (1.0 - std::pow(b2, (double)h->step)));
    const uint64_t np = s.n_dev;
    timer_begin(h, NIRC_K_ADAM, st);
    k_adam<<<8 * h->num_sms, 256, 0, st>>>(np, h->params, h->adam_m, h->adam_v, h->grad, h->cfg.lr, h->cfg.beta1,
                                          h->cfg.beta2, h->cfg.adam_eps, inv_bc1, inv_bc2, h->hash16, s.hash_off);
    count_kernels(h);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_repack_simt(h, st);
    if (e == cudaSuccess) e = launch_repack_tc(h, st);
    timer_end(h, NIRC_K_ADAM, st);
    if (e != cudaSuccess) return e;
    if (d_loss) {
        if ((e = cudaMemcpyAsync(d_loss, h->loss_accum, sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_query_bwd(nirc_handle* h, const nirc_record* recs, const float* dirs, const float* grad_out,
                             uint64_t n, float* d_value, cudaStream_t st) {
    cudaError_t e = train_pass(h, recs, dirs, grad_out, n, kLossUpstream, st);
    if (e == cudaSuccess && d_value)
        e = cudaMemcpyAsync(d_value, h->loss_accum, sizeof(float), cudaMemcpyDeviceToDevice, st);
    return e;
}

}  // namespace nirc
