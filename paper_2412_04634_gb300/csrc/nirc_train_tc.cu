// nirc_train_tc.cu -- the training step's forward and backward on the
// tensor cores (tcgen05, TMEM accumulators): the same loss, gradients and
// buffers as the FP32 kernels of nirc_train.cu (relative L2 of eq. 12,
// hash-grid scatter, stored activations and deltas for the weight-gradient
// kernels), with the layer products as MMAs.
//
// The stored network inputs, activations, deltas and dL/dz are BF16 (the
// element (row, sample) of a buffer at its base + row * ld + sample, two bytes
// each): the weight gradients take them as BF16 MMA operands, so the
// rounding is the one those operands need anyway, at half the bytes.
//
// One warpgroup (128 threads; thread = training record = TMEM lane) takes a
// tile of 128 records at a time, four warpgroups per CTA:
//  encode    hash-grid features (FP16 copy of the table) and surface
//            features into the A tile, direction features into a second
//            A tile; the values go to the e buffer (BF16) for dW0
//  forward   layer 0 = W0_surf e_surf + W0_dir e_dir (4 + 1 or 2 MMAs), the
//            hidden and output layers with their biases added by an MMA
//            against the ones atom (the cache kernel's FP16 image); each
//            epilogue keeps the ReLU mask of its 64 units as two 32-bit
//            words, stores the activations (BF16) and writes the FP16 A tile
//  loss      n = exp(min(z, z_clamp)) (or the visibility sigmoid), the
//            sample's term of eq. 12 and dL/dz
//  backward  delta of the last hidden layer = mask (W_out^T dL/dz) in FP32;
//            then delta_{l-1} = mask (W_l^T delta_l) as FP16 MMAs against
//            the transposed weights; deltas stored (BF16) for dW; finally
//            dL/de_pos = W0_pos^T delta_0 (one MMA, N = 32) scattered into
//            the hash-table gradient like the FP32 backward.  The deltas
//            span many orders of magnitude (they carry the 1 / (3 n) of the
//            loss and the record's 1 / (n^2 + eps)), far below FP16's range,
//            so each record's delta row enters the MMA scaled by 2^-e, e the
//            exponent of its largest element, and the accumulator row is
//            multiplied back by 2^e: both exact, so every record keeps
//            FP16's 11 significant bits whatever its magnitude.
// Every mbarrier wait is bounded; a timeout sets *err and the tile's
// remaining MMAs are skipped.
#include "nirc_internal.h"
#include "nirc_simt.cuh"
#include "nirc_tc.cuh"

namespace nirc {

namespace trimg {
// Backward part of the training image, after the forward part (the cache
// network's FP16 image): FP16 transposed hidden weights (row = input unit,
// K = output unit), the transposed position columns of W0 (row = position
// feature, K = unit), FP32 W_out [3][64].
__host__ __device__ inline uint32_t off_fwd_end(uint32_t H) { return (tcimg::off_scales(H) + 64u + 1023u) & ~1023u; }
__host__ __device__ inline uint32_t off_wht(uint32_t H, uint32_t slot) { return off_fwd_end(H) + 8192u * slot; }
__host__ __device__ inline uint32_t off_w0pt(uint32_t H) { return off_fwd_end(H) + 8192u * (H - 1); }
__host__ __device__ inline uint32_t off_wout32(uint32_t H) { return off_w0pt(H) + 8192u; }
__host__ __device__ inline uint32_t bytes(uint32_t H) { return off_wout32(H) + 3u * 64u * 4u; }
}  // namespace trimg

size_t train_tc_image_bytes(uint32_t hidden) { return trimg::bytes(hidden); }

// The backward part of the image from the FP32 master weights.
__global__ void k_repack_train_bwd(NetShape s, const float* __restrict__ params, uint8_t* __restrict__ img) {
    const uint32_t H = s.hidden;
    const uint64_t n_in = s.n_in;
    const uint32_t n_t = 4096u * H;  // H - 1 hidden tiles + the W0 position tile
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n_t) {
        const uint32_t m = idx / 4096, n = (idx % 4096) / 64, k = idx % 64;
        float v = 0.f;
        uint32_t off;
        if (m + 1 < H) {  // hidden layer m + 1: element (input n, output k) = W[k][n]
            off = trimg::off_wht(H, m);
            v = params[64 * n_in + 64 + (uint64_t)m * (64 * 64 + 64) + k * 64 + n];
        } else {  // W0 position columns: element (feature n, unit k) = W0[k][n]
            off = trimg::off_w0pt(H);
            if (n < s.n_pos) v = params[(uint64_t)k * n_in + n];
        }
        *reinterpret_cast<uint16_t*>(img + off + tc::sw128_offset(n, k)) = __half_as_ushort(__float2half_rn(v));
        return;
    }
    const uint32_t j = idx - n_t;
    if (j >= 3 * 64) return;
    reinterpret_cast<float*>(img + trimg::off_wout32(H))[j] =
        params[64 * n_in + 64 + (uint64_t)(H - 1) * (64 * 64 + 64) + j];
}

struct TrTcArgs {
    NetShape s;
    GridParams g;
    uint64_t n;        // records of this chunk
    uint32_t n_tiles;  // ceil(n / 128)
    uint32_t img_bytes;
    float scale;  // 1 / (3 n_batch)
    float loss_eps, z_clamp;
};

constexpr uint32_t kTrWarpgroups = 4;

// Exponent e of m > 0 (m in [2^e, 2^(e+1))), clamped so that 2^e and 2^-e
// are normal floats; 0 for m = 0.
__device__ __forceinline__ int row_exp(float m) {
    const int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;
    return m > 0.f ? max(-126, min(126, e)) : 0;
}
__device__ __forceinline__ float pow2i(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }
constexpr uint32_t kTrWgStride = 32768;  // A tile 16 KB | direction / delta tile 16 KB
constexpr uint32_t kTrMiscBytes = 128;   // mbarriers, TMEM holder, abort flags

template <bool kSh>
__global__ void __launch_bounds__(kTrWarpgroups * 128, 1)
    k_train_tc(TrTcArgs a, const uint8_t* __restrict__ img_g, const __half2* __restrict__ hash16,
               const nirc_record* __restrict__ recs, const float* __restrict__ dirs,
               const float* __restrict__ targets, TrainPtrs tp, float* __restrict__ grad_table,
               float* __restrict__ loss_accum, int* __restrict__ err) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (sbase - raw);
    const uint32_t n_wg = blockDim.x >> 7;
    const uint32_t wg = threadIdx.x >> 7, t = threadIdx.x & 127u, quarter = t >> 5;
    const uint32_t img_al = (a.img_bytes + 1023u) & ~1023u;
    const uint32_t tA = sbase + img_al + wg * kTrWgStride, tD = tA + 16384u;
    const uint32_t misc = sbase + img_al + n_wg * kTrWgStride;
    uint8_t* miscg = gbase + img_al + n_wg * kTrWgStride;
    const uint32_t mbar = misc + 8u * wg;
    volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(miscg + 64);
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(miscg + 80 + 4 * wg);
    const uint32_t tmem_cols = n_wg <= 1 ? 64u : (n_wg <= 2 ? 128u : (n_wg <= 4 ? 256u : 512u));
    const uint32_t H = a.s.hidden;

    {
        const float4* src = reinterpret_cast<const float4*>(img_g);
        float4* dst = reinterpret_cast<float4*>(gbase);
        for (uint32_t i = threadIdx.x; i < a.img_bytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    if (threadIdx.x < 32) tc::tmem_alloc(misc + 64, tmem_cols);
    if (threadIdx.x == 0) {
        for (uint32_t w = 0; w < n_wg; ++w) {
            tc::mbar_init(misc + 8u * w, 1);
            *reinterpret_cast<volatile uint32_t*>(miscg + 80 + 4 * w) = 0u;
        }
        tc::fence_mbar_init();
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder + 64u * wg;
    const uint32_t tmem_row = tmem + ((32u * quarter) << 16);
    const uint32_t bar_id = 1 + wg;
    uint32_t phase = 0;

    const float* bias = reinterpret_cast<const float*>(gbase + tcimg::off_bias(H));
    const float* wout32 = reinterpret_cast<const float*>(gbase + trimg::off_wout32(H));
    const uint32_t id64 = tc::idesc_f16(0, 128, 64), id16 = tc::idesc_f16(0, 128, 16);
    const uint32_t id32 = tc::idesc_f16(0, 128, 32);
    const uint32_t ones = sbase + tcimg::off_ones(H), bmma = sbase + tcimg::off_bmma(H);

    auto sync_wg = [&]() {
        tc::fence_proxy_async();
        tc::fence_before_sync();
        tc::named_bar(bar_id, 128);
    };
    auto wait_mma = [&]() {
        if (!*abort_flag) {
            if (!tc::mbar_wait_bounded(mbar, phase)) {
                *abort_flag = 1u;
                atomicExch(err, 1);
            }
        }
        phase ^= 1u;
        tc::fence_after_sync();
    };
    // A (K = 64) x B, plus optionally bias slot j against the ones atom, plus
    // optionally a second A (K = 16 kd) x B2: one commit
    auto issue = [&](uint32_t a_tile, uint32_t b_tile, uint32_t idesc, int bias_slot, uint32_t a2, uint32_t b2,
                     uint32_t kd) {
        if (t == 0 && !*abort_flag) {
            tc::fence_after_sync();
#pragma unroll
            for (uint32_t s = 0; s < 4; ++s) tc::mma_f16(tmem, tc::sdesc(a_tile + 32 * s), tc::sdesc(b_tile + 32 * s), idesc, s);
            for (uint32_t s = 0; s < kd; ++s) tc::mma_f16(tmem, tc::sdesc(a2 + 32 * s), tc::sdesc(b2 + 32 * s), idesc, 1);
            if (bias_slot >= 0) {
                const uint32_t j = (uint32_t)bias_slot;
                tc::mma_f16(tmem, tc::sdesc_rep8(ones), tc::sdesc(bmma + 8192u * (j >> 2) + 32u * (j & 3u)), idesc, 1);
            }
            tc::mma_commit(mbar);
        }
    };
    // Forward epilogue: + bias (layer 0 only), ReLU mask, activations out (BF16), FP16 A tile.
    auto fwd_epilogue = [&](const float* b, uint16_t* gact, bool store, uint32_t (&mask)[2]) {
#pragma unroll
        for (uint32_t half = 0; half < 2; ++half) {
            uint32_t v[32];
            tc::tmem_ld32(tmem_row + 32u * half, v);
            tc::tmem_wait_ld();
            float x[32];
            uint32_t m = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                x[i] = __uint_as_float(v[i]) + (b ? b[32 * half + i] : 0.f);
                m |= (x[i] > 0.f ? 1u : 0u) << i;
                x[i] = fmaxf(x[i], 0.f);
            }
            mask[half] = m;
            if (store) {
#pragma unroll
                for (int i = 0; i < 32; ++i) gact[(uint64_t)(32 * half + i) * tp.ld] = to16<1>(x[i]);
            }
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q) sts_chunk8<0>(tA, t, 4 * half + q, x + 8 * q);
        }
    };
    // Backward epilogue: delta = mask * accumulator * 2^e_in, FP32 out, the
    // FP16 A tile scaled by 2^-e of its own row maximum (returned).
    auto bwd_epilogue = [&](uint16_t* gdelta, bool store, const uint32_t (&mask)[2], int e_in) -> int {
        const float un = pow2i(e_in);
        float m = 0.f;
#pragma unroll
        for (uint32_t half = 0; half < 2; ++half) {
            uint32_t v[32];
            tc::tmem_ld32(tmem_row + 32u * half, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if ((mask[half] >> i) & 1u) m = fmaxf(m, fabsf(__uint_as_float(v[i])));
        }
        const int e = row_exp(m * un);
        const float sc = pow2i(-e);
#pragma unroll
        for (uint32_t half = 0; half < 2; ++half) {
            uint32_t v[32];
            tc::tmem_ld32(tmem_row + 32u * half, v);
            tc::tmem_wait_ld();
            float x[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = (mask[half] >> i) & 1u ? __uint_as_float(v[i]) * un : 0.f;
            if (store) {
#pragma unroll
                for (int i = 0; i < 32; ++i) gdelta[(uint64_t)(32 * half + i) * tp.ld] = to16<1>(x[i]);
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] *= sc;
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q) sts_chunk8<0>(tA, t, 4 * half + q, x + 8 * q);
        }
        return e;
    };

    const uint32_t n_dir = kSh ? kShFeatures : kDirFeatures;
    float loss_run = 0.f;
    for (uint32_t tile = blockIdx.x * n_wg + wg; tile < a.n_tiles; tile += gridDim.x * n_wg) {
        const uint64_t sidx = (uint64_t)tile * 128u + t;
        const bool in = sidx < a.n;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
        V3 wi{0.f, 0.f, 1.f};
        if (in) {
            const float4* rq = reinterpret_cast<const float4*>(recs + sidx);
            r0 = __ldg(rq);
            r1 = __ldg(rq + 1);
            r2 = __ldg(rq + 2);
            r3 = __ldg(rq + 3);
            wi = V3{__ldg(dirs + 3 * sidx), __ldg(dirs + 3 * sidx + 1), __ldg(dirs + 3 * sidx + 2)};
        }
        const bool valid = in && (__float_as_uint(r3.z) & 1u);
        const V3 p{r0.x, r0.y, r0.z}, nrm{r0.w, r1.x, r1.y};
        uint16_t* ge = reinterpret_cast<uint16_t*>(tp.e) + sidx;
        // ------------------------------------------------ encoding
        {
            float f[8];
            uint32_t c = 0, k = 0;  // A chunk, feature index in parameter order
            if (a.s.hashgrid) {
                const uint64_t T = (uint64_t)a.g.mask + 1;
                for (uint32_t l0 = 0; l0 < a.g.n_levels; l0 += 4, ++c) {
#pragma unroll
                    for (uint32_t q = 0; q < 4; ++q) {
                        const uint32_t l = l0 + q;
                        uint32_t idx[8];
                        float w[8];
                        grid_corners(a.g.level[l], a.g.mask, p, idx, w);
                        const __half2* tab = hash16 + (uint64_t)l * T;
                        float f0 = 0.f, f1 = 0.f;
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const float2 v = __half22float2(__ldg(tab + idx[kk]));
                            f0 += w[kk] * v.x;
                            f1 += w[kk] * v.y;
                        }
                        f[2 * q] = f0;
                        f[2 * q + 1] = f1;
                    }
                    sts_chunk8<0>(tA, t, c, f);
                    if (in)
                        for (int q = 0; q < 8; ++q) ge[(uint64_t)(k + q) * tp.ld] = to16<1>(f[q]);
                    k += 8;
                }
            } else {
                const float pv[3] = {p.x, p.y, p.z};
                for (int d = 0; d < 3; ++d, ++c) {
                    freq4(pv[d], f);
                    sts_chunk8<0>(tA, t, c, f);
                    if (in)
                        for (int q = 0; q < 8; ++q) ge[(uint64_t)(k + q) * tp.ld] = to16<1>(f[q]);
                    k += 8;
                }
            }
            // surface features after the direction features in parameter order
            const uint32_t ks = a.s.n_pos + n_dir;
            if constexpr (kSh) {
                float ph[16];
                phi_features(nrm, make_float3(r2.y, r2.z, r2.w), r3.x, ph);
                ph[15] = 0.f;
                sts_chunk8<0>(tA, t, c++, ph);
                sts_chunk8<0>(tA, t, c++, ph + 8);
                if (in)
                    for (uint32_t q = 0; q < kPhiFeatures; ++q) ge[(uint64_t)(ks + q) * tp.ld] = to16<1>(ph[q]);
            } else {
                const float nv[3] = {nrm.x, nrm.y, nrm.z};
                for (int d = 0; d < 3; ++d, ++c) {
                    freq4(nv[d], f);
                    sts_chunk8<0>(tA, t, c, f);
                    if (in)
                        for (int q = 0; q < 8; ++q) ge[(uint64_t)(ks + 8 * d + q) * tp.ld] = to16<1>(f[q]);
                }
            }
            for (; c < 8; ++c) sts_chunk(tA, t, c, 0u, 0u, 0u, 0u);
            // direction features: second A tile, K = 16 (frequency) or 32 (spherical harmonics)
            float e[32];
            if constexpr (kSh) {
                sh_basis25(wi, e);
            } else {
                float th, ph;
                dir_angles(wi, th, ph);
                freq4(th, e);
                freq4(ph, e + 8);
            }
#pragma unroll
            for (uint32_t i = kSh ? 25u : 16u; i < 32; ++i) e[i] = 0.f;
#pragma unroll
            for (uint32_t q = 0; q < (kSh ? 4u : 2u); ++q) sts_chunk8<0>(tD, t, q, e + 8 * q);
            if (in)
                for (uint32_t q = 0; q < n_dir; ++q) ge[(uint64_t)(a.s.n_pos + q) * tp.ld] = to16<1>(e[q]);
        }
        // ------------------------------------------------ forward
        uint32_t mask[kMaxHidden][2];
        sync_wg();
        issue(tA, sbase + tcimg::off_w0pix(), id64, -1, tD, sbase + tcimg::off_w0dir(), kSh ? 2u : 1u);
        wait_mma();
        uint16_t* const act16 = reinterpret_cast<uint16_t*>(tp.act);
        uint16_t* const delta16 = reinterpret_cast<uint16_t*>(tp.delta);
        fwd_epilogue(bias, act16 + sidx, in, mask[0]);
        for (uint32_t l = 1; l < H; ++l) {
            sync_wg();
            issue(tA, sbase + tcimg::off_wh(l - 1), id64, (int)(l - 1), 0u, 0u, 0u);
            wait_mma();
            fwd_epilogue(nullptr, act16 + (uint64_t)l * 64 * tp.ld + sidx, in, mask[l]);
        }
        sync_wg();
        issue(tA, sbase + tcimg::off_wout(H), id16, (int)(H - 1), 0u, 0u, 0u);
        wait_mma();
        float dz[3];
        {
            uint32_t v[4];
            tc::tmem_ld4(tmem_row, v);
            tc::tmem_wait_ld();
            const bool vis = a.s.vis;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float z = __uint_as_float(v[c]);
                const bool clamped = !vis && !(z <= a.z_clamp);
                const float nv = out_act(vis, z, a.z_clamp);
                const float dact = vis ? nv * (1.f - nv) : (clamped ? 0.f : nv);
                const float f = in ? __ldg(targets + 3 * sidx + c) : 0.f;
                const float diff = f - nv;
                dz[c] = 0.f;
                if (valid) {
                    if (vis) {
                        loss_run += diff * diff * a.scale;
                        dz[c] = -2.f * diff * a.scale * dact;
                    } else {
                        const float den = nv * nv + a.loss_eps;
                        loss_run += diff * diff / den * a.scale;
                        dz[c] = -2.f * diff / den * a.scale * dact;
                    }
                }
                if (in) reinterpret_cast<uint16_t*>(tp.dz)[(uint64_t)c * tp.dz_ld + sidx] = to16<1>(dz[c]);
            }
        }
        // ------------------------------------------------ backward
        int ex;  // exponent of the delta row in the A tile
        {
            // delta of the last hidden layer: mask (W_out^T dz), FP32
            const uint32_t* mk = mask[H - 1];
            auto delta_out = [&](uint32_t u) {
                return (mk[u >> 5] >> (u & 31u)) & 1u
                           ? wout32[u] * dz[0] + wout32[64 + u] * dz[1] + wout32[128 + u] * dz[2]
                           : 0.f;
            };
            float m = 0.f;
#pragma unroll 8
            for (uint32_t u = 0; u < 64; ++u) m = fmaxf(m, fabsf(delta_out(u)));
            ex = row_exp(m);
            const float sc = pow2i(-ex);
            uint16_t* gd = delta16 + (uint64_t)(H - 1) * 64 * tp.ld + sidx;
#pragma unroll
            for (uint32_t half = 0; half < 2; ++half) {
                float x[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) x[i] = delta_out(32 * half + i);
                if (in) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) gd[(uint64_t)(32 * half + i) * tp.ld] = to16<1>(x[i]);
                }
#pragma unroll
                for (int i = 0; i < 32; ++i) x[i] *= sc;
#pragma unroll
                for (uint32_t q = 0; q < 4; ++q) sts_chunk8<0>(tA, t, 4 * half + q, x + 8 * q);
            }
        }
        for (uint32_t l = H - 1; l >= 1; --l) {
            // delta_{l-1} = mask_{l-1} (W_l^T delta_l): A = delta_l 2^-ex (FP16), B = W_l transposed
            sync_wg();
            issue(tA, sbase + trimg::off_wht(H, l - 1), id64, -1, 0u, 0u, 0u);
            wait_mma();
            ex = bwd_epilogue(delta16 + (uint64_t)(l - 1) * 64 * tp.ld + sidx, in, mask[l - 1], ex);
        }
        if (a.s.hashgrid) {
            // dL/de of the position features: W0_pos^T delta_0 (N = 32), scattered like the FP32 backward
            sync_wg();
            issue(tA, sbase + trimg::off_w0pt(H), id32, -1, 0u, 0u, 0u);
            wait_mma();
            uint32_t v[32];
            tc::tmem_ld32(tmem_row, v);
            tc::tmem_wait_ld();
            const float un = pow2i(ex);
            const uint64_t T = (uint64_t)a.g.mask + 1;
            for (uint32_t l = 0; l < a.g.n_levels; ++l) {
                const float de0 = __uint_as_float(v[2 * l]) * un, de1 = __uint_as_float(v[2 * l + 1]) * un;
                uint32_t idx[8];
                float w[8];
                grid_corners(a.g.level[l], a.g.mask, p, idx, w);
                float* gt = grad_table + (uint64_t)l * T * 2;
                if (a.g.level[l].dense) {
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
    for (int o = 16; o > 0; o >>= 1) loss_run += __shfl_xor_sync(0xffffffffu, loss_run, o);
    if ((threadIdx.x & 31) == 0 && loss_run != 0.f) atomicAdd(loss_accum, loss_run);

    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(*tmem_holder, tmem_cols);
    }
}

bool train_tc_shape_ok(const NetShape& s) {
    return s.hidden >= 1 && s.hidden <= kMaxHidden && (s.n_pos == 24 || s.n_pos == 32);
}

bool train_tc_supported(const nirc_handle* h) {
    return h->packed_train != nullptr && !h->deterministic && train_tc_shape_ok(h->shape);
}

cudaError_t launch_repack_train(const nirc_handle* h, cudaStream_t st) {
    if (!h->packed_train) return cudaSuccess;
    uint8_t* img = reinterpret_cast<uint8_t*>(h->packed_train);
    cudaError_t e = launch_repack_fwd16(h, img, st);
    if (e != cudaSuccess) return e;
    const uint32_t n = 4096u * h->shape.hidden + 3 * 64;
    k_repack_train_bwd<<<(n + 255) / 256, 256, 0, st>>>(h->shape, h->params, img);
    count_kernels(h);
    return cudaGetLastError();
}

cudaError_t launch_train_tc(const nirc_handle* h, const nirc_record* recs, const float* dirs, const float* targets,
                            uint64_t m, float scale, const TrainPtrs& tp, float* grad_table, float* loss_accum,
                            cudaStream_t st) {
    TrTcArgs a;
    a.s = h->shape;
    a.g = h->grid;
    a.n = m;
    a.n_tiles = (uint32_t)((m + 127) / 128);
    a.img_bytes = (uint32_t)trimg::bytes(h->shape.hidden);
    a.scale = scale;
    a.loss_eps = h->cfg.loss_eps;
    a.z_clamp = h->cfg.z_clamp;
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    uint32_t n_wg = kTrWarpgroups;
    auto smem_for = [&](uint32_t w) {
        return (size_t)1024 + ((a.img_bytes + 1023u) & ~1023u) + (size_t)w * kTrWgStride + kTrMiscBytes;
    };
    while (n_wg > 1 && smem_for(n_wg) > (size_t)max_smem) --n_wg;
    const size_t smem = smem_for(n_wg);
    if (smem > (size_t)max_smem) return cudaErrorInvalidConfiguration;
    uint32_t grid = (a.n_tiles + n_wg - 1) / n_wg;
    if (grid > (uint32_t)h->num_sms) grid = h->num_sms;
    if (grid < 1) grid = 1;
    auto kern = h->shape.sh ? k_train_tc<true> : k_train_tc<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, n_wg * 128, smem, st>>>(a, reinterpret_cast<const uint8_t*>(h->packed_train),
                                         reinterpret_cast<const __half2*>(h->hash16), recs, dirs, targets, tp,
                                         grad_table, loss_accum, h->dev_err);
    count_kernels(h);
    return cudaGetLastError();
}

}  // namespace nirc
