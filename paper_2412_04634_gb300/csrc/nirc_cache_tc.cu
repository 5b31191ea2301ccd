// nirc_cache_tc.cu -- tensor-core (tcgen05, TMEM accumulators) evaluation of
// the cache integral, FP16 or BF16 operands with FP32 accumulation.
//
// Work unit: a block of 128 pixels; with S = N + M rows per pixel it holds
// exactly S row tiles of 128 rows.  One warpgroup (128 threads, thread t =
// tile row t = TMEM lane t) owns a block at a time; a CTA runs up to five
// warpgroups so that one warpgroup's SIMT work (sampling, encodings,
// epilogues) overlaps another's MMAs.
//
//  pixel stage   thread t encodes pixel t's surface (hash grid or frequency
//                position features + normal features) into an A tile; one
//                128x64x64 MMA with the surface columns of layer 0 gives
//                h_pix = W0[:, pix] e_pix + b0 for the 128 pixels, stored as a
//                16-bit K-major operand H (K = pixel index).  This is the
//                paper's shared per-surface encoding: computed once per
//                shading point and reused by all its N + M rows.
//  row tile      thread t samples its row's direction (cache rows) or reads
//                it (residual rows), encodes it and writes the A row
//                [e_dir (16) | one-hot of its pixel within a 48-wide window];
//                layer 0 = W0_dir e_dir + H onehot (1 + up to 3 MMAs, K = 16
//                each), then the hidden layers (4 MMAs each) and the output
//                layer (N = 16, 3 used); each epilogue reads its row from
//                TMEM, adds the bias, applies ReLU, rounds to 16 bits and
//                writes the next A tile in shared memory.  The network input
//                and output never touch global memory.
//  reduction     per-row contributions w * n go to shared memory; one thread
//                per pixel sums its rows in sample order (compensated FP32),
//                carrying a pixel that straddles two tiles, and writes the
//                pixel (eq. L_mlmc = L_e + L_c + L_r).
//
// The paper's input (NIRC_INPUT_SH): the pixel stage encodes [position |
// albedo, one-blob normal and roughness]; H is stored pixel-major (row t =
// pixel t's h_pix in 16 bits, the A-tile swizzle); a row writes the 25
// spherical harmonics of its direction (K = 32, two MMAs against the SH
// columns of layer 0) and the layer-0 epilogue adds its pixel's H row.  Any
// S >= 1 works (no one-hot window).
//
// FP8 (E4M3) mode: the hidden 64x64 layers run as kind::f8f6f4 MMAs (K = 32,
// two per layer) on E4M3 weights and activations with per-layer scales:
// weights W / s_w with s_w = amax|W| / 448 (taken when the weights are
// packed), activations a / s_a with s_a = amax(a) / 448 from the previous
// launch (delayed scaling: every FP8 launch records the amax of each hidden
// layer's input, which the next launch uses); the accumulator is multiplied
// back by s_w s_a in the epilogue.  Layer 0 (with the per-pixel product) and
// the output layer stay FP16.  The first FP8 launch after new weights is
// preceded by one FP16 launch that only records the activation amax.
//
// Every mbarrier wait is bounded (about 2 s); a timeout sets *err, stops
// further MMAs of that warpgroup and the kernel still frees its TMEM.
#include "nirc_internal.h"
#include "nirc_tc.cuh"

namespace nirc {


size_t tc_image_bytes(uint32_t hidden) { return tcimg::off_scales(hidden) + 64; }

constexpr float kE4M3Max = 448.f;

__device__ __forceinline__ uint8_t to_e4m3(float v) { return (uint8_t)(tc::pack_e4m3x4(v, 0.f, 0.f, 0.f) & 0xFFu); }

// s_w of each hidden layer (one block per layer): amax |W| / 448, 1 for an all-zero layer.
__global__ void k_weight_scales(NetShape s, const float* __restrict__ params, uint8_t* __restrict__ img) {
    __shared__ float red[256];
    const uint32_t l = blockIdx.x;  // hidden slot: layer l + 1
    const uint64_t b = 64ull * s.n_in + 64 + (uint64_t)l * (64 * 64 + 64);
    float m = 0.f;
    for (uint32_t i = threadIdx.x; i < 64 * 64; i += blockDim.x) m = fmaxf(m, fabsf(params[b + i]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (uint32_t o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        reinterpret_cast<float*>(img + tcimg::off_scales(s.hidden))[l] = red[0] > 0.f ? red[0] / kE4M3Max : 1.f;
}

// Delayed activation scaling: the amax recorded by the last launch becomes
// the history the next launch scales with.  buf[0..8) history (float),
// buf[8..16) current (float bits, atomicMax).
__global__ void k_amax_roll(uint32_t* buf, uint32_t n) {
    const uint32_t j = threadIdx.x;
    if (j < n) {
        const uint32_t cur = buf[8 + j];
        if (cur) buf[j] = cur;
        buf[8 + j] = 0u;
    }
}

constexpr uint32_t kMiscBytes = 256;     // mbarriers, TMEM holder, abort flags, FP8 scales and amax
// Per warpgroup: the two swizzled operand tiles (A 16 KB | H 16 KB, 1024-byte
// aligned), and apart from them the small arrays (contributions 2 KB | carry
// slots and warp partials 512 B).
constexpr uint32_t kWgStride = 32768;
constexpr uint32_t kOffA = 0, kOffH = 16384;
constexpr uint32_t kSmallStride = 2560;
constexpr uint32_t kOffContrib = 0, kOffCarry = 2048;

template <uint32_t AB>
__global__ void k_repack_tc(NetShape s, const float* __restrict__ params, uint8_t* __restrict__ img) {
    const uint32_t H = s.hidden;
    const uint32_t n_mat = 64 * 64 * (2 + (H - 1)) + 16 * 64;
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t n_in = s.n_in;
    if (idx < n_mat) {
        uint32_t m = idx / 4096, r = idx % 4096;
        uint32_t n = r / 64, k = r % 64;
        float v = 0.f;
        uint32_t off;
        if (m == 0) {  // surface columns of layer 0: [pos][surf] -> master columns [pos][dir][surf]
            off = tcimg::off_w0pix();
            if (k < s.n_pos) v = params[n * n_in + k];
            else if (k < s.n_pix) v = params[n * n_in + k + s.n_dir];
        } else if (m == 1) {  // direction columns of layer 0
            off = tcimg::off_w0dir();
            if (k < s.n_dir) v = params[n * n_in + s.n_pos + k];
        } else if (m < 2 + (H - 1)) {
            const uint32_t l = m - 2;  // hidden layer l + 1
            off = tcimg::off_wh(l);
            const uint64_t b = 64 * n_in + 64 + (uint64_t)l * (64 * 64 + 64);
            v = params[b + n * 64 + k];
        } else {
            off = tcimg::off_wout(H);
            r = idx - 4096 * (2 + (H - 1));
            n = r / 64;
            k = r % 64;
            const uint64_t b = 64 * n_in + 64 + (uint64_t)(H - 1) * (64 * 64 + 64);
            if (n < 3) v = params[b + n * 64 + k];
        }
        if (AB == 2 && m >= 2 && m < 2 + (H - 1)) {  // FP8 hidden layer, scaled by s_w
            const float sw = reinterpret_cast<const float*>(img + tcimg::off_scales(H))[m - 2];
            img[off + tc::sw128_offset_b8(n, k)] = to_e4m3(v / sw);
            return;
        }
        const uint16_t bits = AB == 1 ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
        *reinterpret_cast<uint16_t*>(img + off + tc::sw128_offset(n, k)) = bits;
        return;
    }
    const uint32_t j = idx - n_mat;
    if (j >= tcimg::n_bias(H)) return;
    float v = 0.f;
    if (j < 64) {
        v = params[64 * n_in + j];
    } else if (j < 64 + (H - 1) * 64) {
        const uint32_t l = (j - 64) / 64, o = (j - 64) % 64;
        v = params[64 * n_in + 64 + (uint64_t)l * (64 * 64 + 64) + 4096 + o];
    } else {
        const uint32_t c = j - 64 - (H - 1) * 64;
        if (c < 3) v = params[64 * n_in + 64 + (uint64_t)(H - 1) * (64 * 64 + 64) + 3 * 64 + c];
    }
    reinterpret_cast<float*>(img + tcimg::off_bias(H))[j] = v;
}

// Bias tiles and the ones atom of the weight image (after k_repack_tc has
// written the FP32 biases): one thread per 16-bit element.
template <uint32_t AB>
__global__ void k_repack_bias_mma(uint32_t H, uint8_t* __restrict__ img) {
    const uint32_t n_tile = 64 * 64 * tcimg::n_btiles(H);
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    const float* fb = reinterpret_cast<const float*>(img + tcimg::off_bias(H));
    auto bits = [](float v) -> uint16_t {
        return AB == 1 ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
    };
    auto back = [](uint16_t b) -> float {
        return AB == 1 ? __bfloat162float(__ushort_as_bfloat16(b)) : __half2float(__ushort_as_half(b));
    };
    if (idx < n_tile) {
        const uint32_t tile = idx / 4096, n = (idx % 4096) / 64, k = idx % 64;
        const uint32_t j = 4 * tile + k / 16, kk = k % 16;
        uint16_t v = 0;
        if (j < H && kk < 2) {
            float b = 0.f;
            if (j + 1 < H) b = fb[64 + j * 64 + n];              // hidden layer j + 1
            else if (n < 3) b = fb[64 + (H - 1) * 64 + n];       // output layer
            const uint16_t hi = bits(b);
            v = kk == 0 ? hi : bits(b - back(hi));
        }
        *reinterpret_cast<uint16_t*>(img + tcimg::off_bmma(H) + tile * 8192 + tc::sw128_offset(n, k)) = v;
        return;
    }
    const uint32_t o = idx - n_tile;
    if (o >= 8 * 64) return;
    const uint32_t r = o / 64, k = o % 64;
    *reinterpret_cast<uint16_t*>(img + tcimg::off_ones(H) + tc::sw128_offset(r, k)) = k < 2 ? bits(1.f) : 0;
}

struct TcArgs {
    uint32_t W, H, N, M, k0, k1;
    uint32_t unit_div, purpose;  // Philox counters of the cache samples (CachePass)
    const SceneHeader* env_hd;   // light mode 2 with a visibility cache: cache values times L_env
    uint32_t env_nprims;
    uint32_t S, P, n_blocks;
    float z_clamp;
    uint32_t img_bytes;
    NetShape s;
    GridParams g;
};

// Epilogue of one layer for row r: 64 accumulators from TMEM (two halves of
// 32 columns), times `mul` (kMul: the FP8 scales s_w s_a of the layer),
// + bias (none for layer 0 of the frequency input, whose h_pix holds b0;
// kHrow: layer 0 of the paper's input adds row `pr` of the pixel-major
// 16-bit tile at `hrow`, h_pix of the row's pixel), ReLU, then either 16-bit
// rounding into the next A tile (chunks 0-7) or, kF8Out, scaling by 1/s_a of
// the next layer and E4M3 rounding (chunks 0-3).  kRec: the warp's amax of
// the ReLU outputs goes into the shared word at s_amax (atomicMax on bits).
template <uint32_t AB16, bool kF8Out, bool kMul, bool kRec, bool kHrow = false>
__device__ __forceinline__ void epilogue(uint32_t taddr, const float* __restrict__ bias, float mul, float inv_sa,
                                         uint32_t tile, uint32_t r, uint32_t* s_amax, uint32_t hrow = 0,
                                         uint32_t pr = 0) {
    float mx = 0.f;
#pragma unroll
    for (uint32_t half = 0; half < 2; ++half) {
        uint32_t v[32];
        tc::tmem_ld32(taddr + 32u * half, v);
        tc::tmem_wait_ld();
        float x[32];
        if constexpr (kHrow) {
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q) {
                const uint32_t c = 4u * half + q;
                const uint4 hv = tc::lds128(hrow + (pr >> 3) * 1024u + (pr & 7u) * 128u + (((c ^ pr) & 7u) << 4));
                const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 hh = tc::unpack2<AB16>(hw[j]);
                    const float2 a2 = make_float2(__uint_as_float(v[8 * q + 2 * j]), __uint_as_float(v[8 * q + 2 * j + 1]));
                    const float2 y = kMul ? __ffma2_rn(a2, make_float2(mul, mul), hh) : __fadd2_rn(a2, hh);
                    x[8 * q + 2 * j] = y.x;
                    x[8 * q + 2 * j + 1] = y.y;
                }
            }
        } else if (bias) {
            const float4* b4 = reinterpret_cast<const float4*>(bias + 32u * half);  // 128-bit broadcast loads
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 bb = b4[i];
                const float2 a0 = make_float2(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1]));
                const float2 a1 = make_float2(__uint_as_float(v[4 * i + 2]), __uint_as_float(v[4 * i + 3]));
                const float2 y0 = kMul ? __ffma2_rn(a0, make_float2(mul, mul), make_float2(bb.x, bb.y))
                                       : __fadd2_rn(a0, make_float2(bb.x, bb.y));
                const float2 y1 = kMul ? __ffma2_rn(a1, make_float2(mul, mul), make_float2(bb.z, bb.w))
                                       : __fadd2_rn(a1, make_float2(bb.z, bb.w));
                x[4 * i] = y0.x;
                x[4 * i + 1] = y0.y;
                x[4 * i + 2] = y1.x;
                x[4 * i + 3] = y1.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = kMul ? __uint_as_float(v[i]) * mul : __uint_as_float(v[i]);
        }
        if constexpr (kRec || kF8Out) {
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = fmaxf(x[i], 0.f);
        }
        if constexpr (kRec) {
#pragma unroll
            for (int i = 0; i < 32; ++i) mx = fmaxf(mx, x[i]);
        }
        if constexpr (kF8Out) {
#pragma unroll
            for (uint32_t q = 0; q < 2; ++q) {
                const float* y = x + 16 * q;
                uint32_t d[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    d[j] = tc::pack_e4m3x4(y[4 * j] * inv_sa, y[4 * j + 1] * inv_sa, y[4 * j + 2] * inv_sa,
                                           y[4 * j + 3] * inv_sa);
                sts_chunk(tile, r, 2u * half + q, d[0], d[1], d[2], d[3]);
            }
        } else {
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q) {
                const float* y = x + 8 * q;
                sts_chunk(tile, r, 4u * half + q, pack2_relu<AB16>(y[0], y[1]), pack2_relu<AB16>(y[2], y[3]),
                          pack2_relu<AB16>(y[4], y[5]), pack2_relu<AB16>(y[6], y[7]));
            }
        }
    }
    if constexpr (kRec) {
        const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
        if ((threadIdx.x & 31u) == 0) atomicMax(s_amax, m);
    }
}

// sin/cos of 2^k a for k = 0..3 from (sin a, cos a), by the double-angle identities.
__device__ __forceinline__ void octaves(float s, float c, float* e) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        e[2 * k] = s;
        e[2 * k + 1] = c;
        const float s2 = 2.0f * s * c;
        const float c2 = (c - s) * (c + s);
        s = s2;
        c = c2;
    }
}

// Direction features of w without transcendentals (hardware rsqrt and fast
// divide: the features are continuous network inputs): with theta = acos(w_z) and
// phi' = atan2(w_y, w_x) mapped to [0, 2 pi), pi theta_hat = theta and
// pi phi_hat = phi' / 2, so sin/cos follow from w_z and from the half-angle
// identities in forms free of cancellation.
__device__ __forceinline__ void dir_features_fast(V3 w, float* e) {
    const float c = fminf(fmaxf(w.z, -1.f), 1.f);
    const float s = fast_sqrt((1.f - c) * (1.f + c));
    octaves(s, c, e);
    const float r2 = w.x * w.x + w.y * w.y;
    float sp = 0.f, cp = 1.f;
    if (r2 > 0.f) {
        const float rr = rsqrtf(r2);
        const float r = r2 * rr;
        const float ir = 0.5f * rr;
        if (w.x >= 0.f) {
            const float a = r + w.x;
            cp = fast_sqrt(a * ir);
            sp = fast_sqrt(__fdividef(w.y * w.y * ir, a));
        } else {
            const float a = r - w.x;
            sp = fast_sqrt(a * ir);
            cp = fast_sqrt(__fdividef(w.y * w.y * ir, a));
        }
        const bool upper = (w.y > 0.f) || (w.y == 0.f && w.x >= 0.f);
        if (!upper) cp = -cp;
    }
    octaves(sp, cp, e + 8);
}

// AB: 0 FP16, 1 BF16, 2 FP8 hidden layers (FP16 elsewhere).  kAmax: record
// the amax of every hidden layer's input activations into amax[8 + l].
template <uint32_t AB, bool kAmax, bool kSh>
__global__ void __launch_bounds__(640, 1)
    k_cache_tc(TcArgs a, const uint8_t* __restrict__ img_g, const __half2* __restrict__ hash16,
               const nirc_record* __restrict__ recs, const PixelBase* __restrict__ base,
               const ResidRow* __restrict__ rows, const float4* __restrict__ beta, float4* __restrict__ out,
               float* __restrict__ lc_out,
               float* __restrict__ lr_out, uint64_t* __restrict__ sig_out, uint32_t* __restrict__ count,
               float* __restrict__ row_n, int* __restrict__ err, uint32_t* __restrict__ amax) {
    constexpr uint32_t AB16 = AB == 1 ? 1u : 0u;  // type of the 16-bit layers
    constexpr bool kF8 = AB == 2;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (sbase - raw);
    const uint32_t n_wg = blockDim.x >> 7;
    const uint32_t wg = threadIdx.x >> 7, t = threadIdx.x & 127u, quarter = t >> 5;
    const uint32_t img_al = (a.img_bytes + 1023u) & ~1023u;
    const uint32_t wgs = sbase + img_al + wg * kWgStride;  // this warpgroup's operand tiles (shared address)
    const uint32_t small_al = img_al + n_wg * kWgStride;
    uint8_t* wgg = gbase + small_al + wg * kSmallStride;   // this warpgroup's small arrays (generic pointer)
    const uint32_t misc = sbase + small_al + n_wg * kSmallStride;
    uint8_t* miscg = gbase + small_al + n_wg * kSmallStride;
    const uint32_t mbar = misc + 8u * wg;
    volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(miscg + 64);
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(miscg + 80 + 4 * wg);
    const uint32_t tmem_cols = n_wg <= 1 ? 64u : (n_wg <= 2 ? 128u : (n_wg <= 4 ? 256u : 512u));

    uint32_t* s_amax = reinterpret_cast<uint32_t*>(miscg + 128);  // [8]
    float* s_mul = reinterpret_cast<float*>(miscg + 160);         // [8] s_w s_a per hidden slot
    float* s_inv = reinterpret_cast<float*>(miscg + 192);         // [8] 1 / s_a per hidden slot

    // stage the weight image
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
        for (uint32_t j = 0; j < 8; ++j) {
            s_amax[j] = 0u;
            float sa = 1.f;
            if (kF8 && j + 1 < a.s.hidden) {
                const float h = __uint_as_float(amax[j]);
                sa = h > 0.f ? h / kE4M3Max : 1.f;
            }
            const float sw = kF8 && j + 1 < a.s.hidden
                                 ? reinterpret_cast<const float*>(img_g + tcimg::off_scales(a.s.hidden))[j]
                                 : 1.f;
            s_mul[j] = sw * sa;
            s_inv[j] = 1.f / sa;
        }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder + 64u * wg;
    const uint32_t tmem_row = tmem + ((32u * quarter) << 16);
    const uint32_t bar_id = 1 + wg;
    uint32_t phase = 0;

    const uint32_t w0pix = sbase + tcimg::off_w0pix(), w0dir = sbase + tcimg::off_w0dir();
    const uint32_t wout = sbase + tcimg::off_wout(a.s.hidden);
    const float* bias = reinterpret_cast<const float*>(gbase + tcimg::off_bias(a.s.hidden));
    const uint32_t tA = wgs + kOffA, tH = wgs + kOffH;
    float4* s_contrib = reinterpret_cast<float4*>(wgg + kOffContrib);
    float* s_carry = reinterpret_cast<float*>(wgg + kOffCarry);  // two slots of 16 floats
    const uint32_t id64 = tc::idesc_f16(AB16, 128, 64), id16 = tc::idesc_f16(AB16, 128, 16);
    const uint32_t id64_e4m3 = tc::idesc_f16(0, 128, 64);  // E4M3 x E4M3 has type code 0 too
    const uint16_t one16 = AB16 ? 0x3F80u : 0x3C00u;

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
    auto issue_k64 = [&](uint32_t a_tile, uint32_t b_tile, uint32_t idesc) {
        if (t == 0 && !*abort_flag) {
            tc::fence_after_sync();
#pragma unroll
            for (uint32_t s = 0; s < 4; ++s) tc::mma_f16(tmem, tc::sdesc(a_tile + 32 * s), tc::sdesc(b_tile + 32 * s), idesc, s);
            tc::mma_commit(mbar);
        }
    };
    // 4 K-steps, then the bias slot j as one more K = 16 step against the ones atom
    const uint32_t ones = sbase + tcimg::off_ones(a.s.hidden), bmma = sbase + tcimg::off_bmma(a.s.hidden);
    auto issue_k64_bias = [&](uint32_t a_tile, uint32_t b_tile, uint32_t idesc, uint32_t j) {
        if (t == 0 && !*abort_flag) {
            tc::fence_after_sync();
#pragma unroll
            for (uint32_t s = 0; s < 4; ++s) tc::mma_f16(tmem, tc::sdesc(a_tile + 32 * s), tc::sdesc(b_tile + 32 * s), idesc, s);
            tc::mma_f16(tmem, tc::sdesc_rep8(ones), tc::sdesc(bmma + 8192u * (j >> 2) + 32u * (j & 3u)), idesc, 1);
            tc::mma_commit(mbar);
        }
    };
    auto issue_k64_e4m3 = [&](uint32_t a_tile, uint32_t b_tile) {
        if (t == 0 && !*abort_flag) {
            tc::fence_after_sync();
#pragma unroll
            for (uint32_t s = 0; s < 2; ++s)
                tc::mma_e4m3(tmem, tc::sdesc(a_tile + 32 * s), tc::sdesc(b_tile + 32 * s), id64_e4m3, s);
            tc::mma_commit(mbar);
        }
    };

    const uint32_t S = a.S;
    for (uint32_t blk = blockIdx.x * n_wg + wg; blk < a.n_blocks; blk += gridDim.x * n_wg) {
        const uint32_t p0 = blk * 128u;
        const uint32_t npix = min(128u, a.P - p0);
        // ------------------------------------------------ pixel stage
        {
            float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
            if (t < npix) {
                const float4* rq = reinterpret_cast<const float4*>(recs + p0 + t);
                r0 = __ldg(rq);
                r1 = __ldg(rq + 1);
                if constexpr (kSh) {
                    r2 = __ldg(rq + 2);
                    r3 = __ldg(rq + 3);
                }
            }
            const V3 p{r0.x, r0.y, r0.z}, n{r0.w, r1.x, r1.y};
            float f[8];
            uint32_t c = 0;  // next chunk of the A row
            if (a.s.hashgrid) {
                const uint64_t T = (uint64_t)a.g.mask + 1;
                for (uint32_t l0 = 0; l0 < a.g.n_levels; l0 += 4, ++c) {  // 12 or 16 levels
#pragma unroll
                    for (uint32_t q = 0; q < 4; ++q) {
                        const uint32_t l = l0 + q;
                        uint32_t idx[8];
                        float w[8];
                        grid_corners(a.g.level[l], a.g.mask, p, idx, w);
                        const __half2* tab = hash16 + (uint64_t)l * T;
                        float f0 = 0.f, f1 = 0.f;
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const float2 v = __half22float2(__ldg(tab + idx[k]));
                            f0 += w[k] * v.x;
                            f1 += w[k] * v.y;
                        }
                        f[2 * q] = f0;
                        f[2 * q + 1] = f1;
                    }
                    sts_chunk8<AB16>(tA, t, c, f);
                }
            } else {
                freq4(p.x, f);
                sts_chunk8<AB16>(tA, t, c++, f);
                freq4(p.y, f);
                sts_chunk8<AB16>(tA, t, c++, f);
                freq4(p.z, f);
                sts_chunk8<AB16>(tA, t, c++, f);
            }
            if constexpr (kSh) {
                float ph[16];
                phi_features(n, make_float3(r2.y, r2.z, r2.w), r3.x, ph);
                ph[15] = 0.f;
                sts_chunk8<AB16>(tA, t, c++, ph);
                sts_chunk8<AB16>(tA, t, c++, ph + 8);
            } else {
                freq4(n.x, f);
                sts_chunk8<AB16>(tA, t, c++, f);
                freq4(n.y, f);
                sts_chunk8<AB16>(tA, t, c++, f);
                freq4(n.z, f);
                sts_chunk8<AB16>(tA, t, c++, f);
            }
            for (; c < 8; ++c) sts_chunk(tA, t, c, 0u, 0u, 0u, 0u);
        }
        sync_wg();
        issue_k64(tA, w0pix, id64);
        wait_mma();
        if constexpr (kSh) {
            // H pixel-major: row t = h_pix of pixel t = accumulator + b0, 16-bit
#pragma unroll
            for (uint32_t half = 0; half < 2; ++half) {
                uint32_t v[32];
                tc::tmem_ld32(tmem_row + 32u * half, v);
                tc::tmem_wait_ld();
#pragma unroll
                for (uint32_t q = 0; q < 4; ++q) {
                    float y[8];
#pragma unroll
                    for (uint32_t j = 0; j < 8; ++j) y[j] = __uint_as_float(v[8 * q + j]) + bias[32 * half + 8 * q + j];
                    sts_chunk8<AB16>(tH, t, 4 * half + q, y);
                }
            }
        } else {
            // H operand: element (n = output unit, k = pixel t), h = accumulator + b0
            const uint32_t hk = tH + (t >> 6) * 8192u;
#pragma unroll
            for (uint32_t half = 0; half < 2; ++half) {
                uint32_t v[32];
                tc::tmem_ld32(tmem_row + 32u * half, v);
                tc::tmem_wait_ld();
#pragma unroll
                for (uint32_t o = 0; o < 32; ++o) {
                    const uint32_t oo = 32u * half + o;
                    tc::sts16(hk + tc::sw128_offset(oo, t & 63u), to16<AB16>(__uint_as_float(v[o]) + bias[oo]));
                }
            }
        }
        sync_wg();

        // ------------------------------------------------ row tiles
        const uint32_t R = npix * S;
        uint32_t jt = 0;
        for (uint32_t j0 = 0; j0 < R; j0 += 128u, ++jt) {
            const uint32_t r = j0 + t;
            const bool rin = r < R;
            const uint32_t pl = rin ? r / S : 0u;
            const uint32_t s = rin ? r - pl * S : 0u;
            const uint32_t pf = j0 / S;
            const uint32_t plast = min((j0 + 127u) / S, npix - 1u);
            // one-hot window [kb, kb + 16 n_oh) covers pixels pf..plast and stays inside H's 128 columns
            const uint32_t n_oh = (plast - (pf & ~15u) + 16u) >> 4;  // <= 3 for S >= 4
            const uint32_t kb = min(pf & ~15u, 128u - 16u * n_oh);

            V3 wi{0.f, 0.f, 1.f};
            float3 w = make_float3(0.f, 0.f, 0.f);
            bool ok = false;
            uint32_t word = 0;
            {
                // all four words of the record at once (one L1 round trip)
                const float4* rq = reinterpret_cast<const float4*>(recs + p0 + pl);
                const float4 q0 = __ldg(rq), q1 = __ldg(rq + 1), q2 = __ldg(rq + 2), q3 = __ldg(rq + 3);
                const uint32_t flags = __float_as_uint(q3.z);
                if (rin && (flags & 1u)) {
                    if (s < a.N) {
                        // Philox counter of the sample: (unit / unit_div, (unit % unit_div) << 16 | s)
                        const uint32_t u = p0 + pl;
                        const uint32_t c0 = a.unit_div == 1u ? u : u / a.unit_div;
                        const uint32_t c1 = a.unit_div == 1u ? s : (((u - c0 * a.unit_div) << 16) | s);
                        const BsdfSample bs =
                            sample_bsdf(V3{q0.w, q1.x, q1.y}, V3{q1.z, q1.w, q2.x}, make_float3(q2.y, q2.z, q2.w),
                                        q3.x, (flags >> 1) & 3u, a.k0, a.k1, c0, c1, a.purpose);
                        wi = bs.wi;
                        w = bs.w;
                        ok = bs.valid;
                        word = bs.word;
                    } else {
                        const ResidRow* rr = rows + (uint64_t)(p0 + pl) * a.M + (s - a.N);
                        const float4 d = __ldg(&rr->wi), ww = __ldg(&rr->w);
                        wi = V3{d.x, d.y, d.z};
                        w = make_float3(ww.x, ww.y, ww.z);
                        ok = d.w != 0.f;
                    }
                }
            }
            if constexpr (kSh) {
                // columns 0..31: the 25 spherical harmonics, zero padded (layer 0 reads K = 32)
                float e[32];
                sh_basis25(wi, e);
#pragma unroll
                for (int i = 25; i < 32; ++i) e[i] = 0.f;
#pragma unroll
                for (uint32_t c = 0; c < 4; ++c) sts_chunk8<AB16>(tA, t, c, e + 8 * c);
            } else {
                float e[16];
                dir_features_fast(wi, e);
                sts_chunk8<AB16>(tA, t, 0u, e);
                sts_chunk8<AB16>(tA, t, 1u, e + 8);
                const uint32_t oh = rin ? pl - kb : 0xFFFFu;  // one-hot position among columns 16..63
#pragma unroll
                for (uint32_t c = 2; c < 8; ++c) {
                    uint32_t d[4] = {0u, 0u, 0u, 0u};
                    const uint32_t lo = (c - 2) * 8;
                    if (oh >= lo && oh < lo + 8) {
                        const uint32_t e2 = oh - lo;
                        d[e2 >> 1] = (uint32_t)one16 << ((e2 & 1u) * 16);
                    }
                    sts_chunk(tA, t, c, d[0], d[1], d[2], d[3]);
                }
            }
            sync_wg();
            if (t == 0 && !*abort_flag) {
                tc::fence_after_sync();
                tc::mma_f16(tmem, tc::sdesc(tA), tc::sdesc(w0dir), id64, 0);
                if constexpr (kSh) {
                    tc::mma_f16(tmem, tc::sdesc(tA + 32u), tc::sdesc(w0dir + 32u), id64, 1);
                } else {
                    for (uint32_t qq = 1; qq <= n_oh; ++qq) {
                        const uint32_t kk = kb + 16u * (qq - 1);
                        tc::mma_f16(tmem, tc::sdesc(tA + 32u * qq),
                                    tc::sdesc(tH + (kk >> 6) * 8192u + (kk & 63u) * 2u), id64, 1);
                    }
                }
                tc::mma_commit(mbar);
            }
            wait_mma();
            for (uint32_t l = 0; l < a.s.hidden; ++l) {
                // epilogue of layer l (l = 0: h_pix already holds b0; 16-bit hidden layers: the
                // bias came with the MMA), then the MMAs of layer l + 1
                const float* bl = (l == 0 || !kF8) ? nullptr : bias + 64 + (l - 1) * 64;
                const bool next_hidden = l + 1 < a.s.hidden;
                if (kSh && l == 0) {
                    // layer 0 of the paper's input: + h_pix of the row's pixel (H row pl)
                    if constexpr (kF8) {
                        if (next_hidden) epilogue<0, true, false, true, true>(tmem_row, nullptr, 1.f, s_inv[0], tA, t, s_amax, tH, pl);
                        else epilogue<0, false, false, false, true>(tmem_row, nullptr, 1.f, 1.f, tA, t, nullptr, tH, pl);
                    } else if constexpr (kAmax) {
                        if (next_hidden) epilogue<AB16, false, false, true, true>(tmem_row, nullptr, 1.f, 1.f, tA, t, s_amax, tH, pl);
                        else epilogue<AB16, false, false, false, true>(tmem_row, nullptr, 1.f, 1.f, tA, t, nullptr, tH, pl);
                    } else {
                        epilogue<AB16, false, false, false, true>(tmem_row, nullptr, 1.f, 1.f, tA, t, nullptr, tH, pl);
                    }
                } else if constexpr (kF8) {
                    const float mul = l == 0 ? 1.f : s_mul[l - 1];
                    if (next_hidden) epilogue<0, true, true, true>(tmem_row, bl, mul, s_inv[l], tA, t, s_amax + l);
                    else epilogue<0, false, true, false>(tmem_row, bl, mul, 1.f, tA, t, nullptr);
                } else if constexpr (kAmax) {
                    if (next_hidden) epilogue<AB16, false, false, true>(tmem_row, bl, 1.f, 1.f, tA, t, s_amax + l);
                    else epilogue<AB16, false, false, false>(tmem_row, bl, 1.f, 1.f, tA, t, nullptr);
                } else {
                    epilogue<AB16, false, false, false>(tmem_row, bl, 1.f, 1.f, tA, t, nullptr);
                }
                sync_wg();
                if (next_hidden) {
                    if constexpr (kF8) issue_k64_e4m3(tA, sbase + tcimg::off_wh(l));
                    else issue_k64_bias(tA, sbase + tcimg::off_wh(l), id64, l);
                } else {
                    issue_k64_bias(tA, wout, id16, a.s.hidden - 1u);
                }
                wait_mma();
            }
            float3 nv;
            {
                uint32_t v[4];
                tc::tmem_ld4(tmem_row, v);
                tc::tmem_wait_ld();
                const bool vis = a.s.vis;  // the output bias came with the MMA
                nv.x = out_act(vis, __uint_as_float(v[0]), a.z_clamp);
                nv.y = out_act(vis, __uint_as_float(v[1]), a.z_clamp);
                nv.z = out_act(vis, __uint_as_float(v[2]), a.z_clamp);
                if (a.env_hd && ok) {  // visibility cache: n = V L_env(w)
                    const float3 le = env_radiance(env_from(a.env_hd, a.env_nprims), wi);
                    nv.x *= le.x;
                    nv.y *= le.y;
                    nv.z *= le.z;
                }
            }
            if (row_n && rin) {
                float* rn = row_n + 3 * ((uint64_t)p0 * S + r);
                rn[0] = ok ? nv.x : 0.f;
                rn[1] = ok ? nv.y : 0.f;
                rn[2] = ok ? nv.z : 0.f;
            }
            // ---- per-pixel sums.  Rows are ordered by pixel, so each pixel is a
            // contiguous segment: a pairwise tree over the warp's lanes (shuffle
            // down by 1, 2, 4, 8, 16, adding only within the segment) leaves each
            // segment's warp-local sum in its first lane, in an order fixed by
            // the row positions.  That lane then adds the partials of later
            // warps whose first rows belong to the same pixel and the previous
            // tile's carry, and either writes the pixel or carries it on.
            const uint32_t lane = t & 31u, warp = t >> 5;
            const uint32_t s_row = rin ? r - pl * S : 0u;
            const bool is_cache = s_row < a.N;
            float v[7];
            {
                const float3 cw = ok ? make_float3(w.x * nv.x, w.y * nv.y, w.z * nv.z) : make_float3(0.f, 0.f, 0.f);
                v[0] = is_cache ? cw.x : 0.f;
                v[1] = is_cache ? cw.y : 0.f;
                v[2] = is_cache ? cw.z : 0.f;
                v[3] = is_cache ? 0.f : cw.x;
                v[4] = is_cache ? 0.f : cw.y;
                v[5] = is_cache ? 0.f : cw.z;
                v[6] = (is_cache && ok) ? 1.f : 0.f;
            }
            const uint32_t seg = rin ? pl : 0xFFFFFFFFu;
#pragma unroll
            for (uint32_t off = 1; off < 32; off <<= 1) {
                const uint32_t oseg = __shfl_down_sync(0xffffffffu, seg, off);
                float o[7];
#pragma unroll
                for (int k = 0; k < 7; ++k) o[k] = __shfl_down_sync(0xffffffffu, v[k], off);
                if (lane + off < 32u && oseg == seg) {
#pragma unroll
                    for (int k = 0; k < 7; ++k) v[k] += o[k];
                }
            }
            float* s_part = s_carry + 32;                                              // 4 warps x 8 floats
            uint64_t* s_sigc = reinterpret_cast<uint64_t*>(s_carry + 64);              // 2 signature carry slots
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < 7; ++k) s_part[8 * warp + k] = v[k];
                s_part[8 * warp + 7] = __uint_as_float(seg);
            }
            if (sig_out) s_contrib[t] = make_float4(0.f, 0.f, 0.f, __uint_as_float(word));
            tc::fence_before_sync();
            tc::named_bar(bar_id, 128);

            const uint32_t prev_seg = __shfl_up_sync(0xffffffffu, seg, 1);
            const bool head = rin && (lane > 0 ? prev_seg != seg
                                               : (warp == 0 || (j0 + 32u * warp - 1u) / S != pl));
            if (head) {
                const uint32_t q = pl;
                const uint32_t q_lo = q * S, q_hi = q_lo + S;
                const float* cin = s_carry + 16u * (jt & 1u);    // written by the previous tile
                float* cout = s_carry + 16u * ((jt + 1u) & 1u);  // read by the next tile
                float acc[7];
                const bool cont_in = q_lo < j0;
#pragma unroll
                for (int k = 0; k < 7; ++k) acc[k] = cont_in ? cin[k] : 0.f;
#pragma unroll
                for (int k = 0; k < 7; ++k) acc[k] += v[k];
                for (uint32_t ww = warp + 1; ww < 4; ++ww) {
                    if (__float_as_uint(s_part[8 * ww + 7]) != seg) break;
#pragma unroll
                    for (int k = 0; k < 7; ++k) acc[k] += s_part[8 * ww + k];
                }
                // decision signature of the cache samples (sequential, only when requested)
                uint64_t sig = 0;
                if (sig_out) {
                    sig = cont_in ? s_sigc[jt & 1u] : kSigInit;
                    const bool qvalid = __float_as_uint(__ldg(reinterpret_cast<const float4*>(recs + p0 + q) + 3).z) & 1u;
                    const uint32_t lo = max(q_lo, j0), hi = min(min(q_hi, j0 + 128u), q_lo + a.N);
                    if (qvalid)
                        for (uint32_t rr = lo; rr < hi; ++rr) sig = sig_mix(sig, __float_as_uint(s_contrib[rr - j0].w));
                }
                if (q_hi > j0 + 128u) {  // continues in the next tile
#pragma unroll
                    for (int k = 0; k < 7; ++k) cout[k] = acc[k];
                    if (sig_out) s_sigc[(jt + 1u) & 1u] = sig;
                } else {
                    const uint32_t gp = p0 + q;
                    PixelBase b;
                    if (base) {
                        b = base[gp];
                    } else {
                        b.le = b.wl = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    float Lc[3] = {0.f, 0.f, 0.f}, Lr[3] = {b.wl.x, b.wl.y, b.wl.z};
                    if (a.N) {
                        const float inv = 1.0f / (float)a.N;
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) Lc[cc] = acc[cc] * inv;
                    }
                    if (a.M && a.N) {  // without a cache level nothing is subtracted
                        const float inv = 1.0f / (float)a.M;
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) Lr[cc] -= acc[3 + cc] * inv;
                    }
                    if (beta) {  // the unit's throughput (biased stopping vertex, later vertex of a residual path)
                        const float4 bt = beta[gp];
                        const float bb[3] = {bt.x, bt.y, bt.z};
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) {
                            Lc[cc] *= bb[cc];
                            Lr[cc] *= bb[cc];
                        }
                    }
                    out[gp] = make_float4(b.le.x + Lc[0] + Lr[0], b.le.y + Lc[1] + Lr[1], b.le.z + Lc[2] + Lr[2], 1.f);
                    if (lc_out) {
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) lc_out[3 * (uint64_t)gp + cc] = Lc[cc];
                    }
                    if (lr_out) {
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) lr_out[3 * (uint64_t)gp + cc] = Lr[cc];
                    }
                    if (sig_out) sig_out[2 * (uint64_t)gp + 1] = sig;
                    if (count) count[gp] += (uint32_t)acc[6];
                }
            }
            // no barrier here: the next tile's barriers order s_contrib and the carry slots
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(*tmem_holder, tmem_cols);
    }
    if constexpr (kAmax) {
        if (threadIdx.x < a.s.hidden - 1) atomicMax(amax + 8 + threadIdx.x, s_amax[threadIdx.x]);
    }
}

static size_t tc_smem_bytes(uint32_t img_bytes, uint32_t n_wg) {
    return 1024 + ((img_bytes + 1023) & ~1023u) + (size_t)n_wg * (kWgStride + kSmallStride) + kMiscBytes;
}

cudaError_t launch_repack_tc(const nirc_handle* h, cudaStream_t st) {
    // the tensor-core training image follows the same weights
    cudaError_t et = launch_repack_train(h, st);
    if (et != cudaSuccess) return et;
    if (!h->packed_tc) return cudaSuccess;
    const uint32_t H = h->shape.hidden;
    const uint32_t n = 64 * 64 * (2 + (H - 1)) + 16 * 64 + tcimg::n_bias(H);
    uint8_t* img = reinterpret_cast<uint8_t*>(h->packed_tc);
    const uint32_t nb = 64 * 64 * tcimg::n_btiles(H) + 8 * 64;
    if (h->cfg.precision == NIRC_BF16_TC) {
        k_repack_tc<1><<<(n + 255) / 256, 256, 0, st>>>(h->shape, h->params, img);
        count_kernels(h);
        k_repack_bias_mma<1><<<(nb + 255) / 256, 256, 0, st>>>(H, img);
        count_kernels(h);
    } else if (h->cfg.precision == NIRC_FP8_E4M3_TC) {
        if (H > 1) {
            k_weight_scales<<<H - 1, 256, 0, st>>>(h->shape, h->params, img);
            count_kernels(h);
        }
        k_repack_tc<2><<<(n + 255) / 256, 256, 0, st>>>(h->shape, h->params, img);
        count_kernels(h);
        k_repack_bias_mma<0><<<(nb + 255) / 256, 256, 0, st>>>(H, img);
        count_kernels(h);
        // FP16 image for the launch that calibrates the activation scales
        uint8_t* img16 = reinterpret_cast<uint8_t*>(h->packed_tc16);
        k_repack_tc<0><<<(n + 255) / 256, 256, 0, st>>>(h->shape, h->params, img16);
        count_kernels(h);
        k_repack_bias_mma<0><<<(nb + 255) / 256, 256, 0, st>>>(H, img16);
        count_kernels(h);
    } else {
        k_repack_tc<0><<<(n + 255) / 256, 256, 0, st>>>(h->shape, h->params, img);
        count_kernels(h);
        k_repack_bias_mma<0><<<(nb + 255) / 256, 256, 0, st>>>(H, img);
        count_kernels(h);
    }
    return cudaGetLastError();
}

cudaError_t launch_repack_fwd16(const nirc_handle* h, uint8_t* img, cudaStream_t st) {
    const uint32_t H = h->shape.hidden;
    const uint32_t n = 64 * 64 * (2 + (H - 1)) + 16 * 64 + tcimg::n_bias(H);
    const uint32_t nb = 64 * 64 * tcimg::n_btiles(H) + 8 * 64;
    k_repack_tc<0><<<(n + 255) / 256, 256, 0, st>>>(h->shape, h->params, img);
    count_kernels(h);
    k_repack_bias_mma<0><<<(nb + 255) / 256, 256, 0, st>>>(H, img);
    count_kernels(h);
    return cudaGetLastError();
}

bool tc_supported(const nirc_handle* h, const nirc_frame_desc& fd) {
    return (h->cfg.precision == NIRC_FP16_TC || h->cfg.precision == NIRC_BF16_TC ||
            h->cfg.precision == NIRC_FP8_E4M3_TC) &&
           fd.cache_mode == 0 && fd.n_cache + fd.n_resid >= (h->shape.sh ? 1u : 4u) && h->packed_tc != nullptr &&
           (h->shape.n_pos == 24 || h->shape.n_pos == 32);
}

template <uint32_t AB, bool kAmax, bool kSh>
static cudaError_t launch_tc_kernel(uint32_t grid, uint32_t threads, size_t smem, cudaStream_t st, const TcArgs& a,
                                      const void* img, const __half2* hash, const nirc_record* recs,
                                      const PixelBase* base, const ResidRow* rows, const float4* beta, float* out,
                                      float* lc, float* lr, uint64_t* sig, uint32_t* count, float* row_n, int* err,
                                      uint32_t* amax) {
    cudaError_t e =
        cudaFuncSetAttribute(k_cache_tc<AB, kAmax, kSh>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_cache_tc<AB, kAmax, kSh><<<grid, threads, smem, st>>>(a, reinterpret_cast<const uint8_t*>(img), hash, recs, base,
                                                            rows, beta, reinterpret_cast<float4*>(out), lc, lr, sig,
                                                            count, row_n, err, amax);
    return cudaGetLastError();
}

// The instance for the network input of a.s (frequency or the paper's).
template <uint32_t AB, bool kAmax>
static cudaError_t launch_tc_instance(uint32_t grid, uint32_t threads, size_t smem, cudaStream_t st, const TcArgs& a,
                                      const void* img, const __half2* hash, const nirc_record* recs,
                                      const PixelBase* base, const ResidRow* rows, const float4* beta, float* out,
                                      float* lc, float* lr, uint64_t* sig, uint32_t* count, float* row_n, int* err,
                                      uint32_t* amax) {
    if (a.s.sh)
        return launch_tc_kernel<AB, kAmax, true>(grid, threads, smem, st, a, img, hash, recs, base, rows, beta, out, lc,
                                                 lr, sig, count, row_n, err, amax);
    return launch_tc_kernel<AB, kAmax, false>(grid, threads, smem, st, a, img, hash, recs, base, rows, beta, out, lc,
                                              lr, sig, count, row_n, err, amax);
}

cudaError_t launch_cache_tc(const nirc_handle* h, const nirc_frame_desc& fd, const nirc_record* recs,
                            const PixelBase* base, const ResidRow* rows, const float4* beta, float* out_rgba,
                            float* lc, float* lr, uint64_t* sig, uint32_t* count, float* row_n, int* err,
                            cudaStream_t st, CachePass pass, EnvSource env) {
    TcArgs a;
    a.unit_div = pass.unit_div;
    a.purpose = pass.purpose;
    a.env_hd = reinterpret_cast<const SceneHeader*>(env.scene);
    a.env_nprims = env.n_prims;
    a.W = fd.width;
    a.H = fd.height;
    a.N = fd.n_cache;
    a.M = fd.n_resid;
    a.k0 = (uint32_t)fd.seed;
    a.k1 = fd.frame;
    a.S = fd.n_cache + fd.n_resid;
    a.P = fd.width * fd.height;
    a.n_blocks = (a.P + 127) / 128;
    a.z_clamp = h->cfg.z_clamp;
    a.img_bytes = (uint32_t)tc_image_bytes(h->shape.hidden);
    a.s = h->shape;
    a.g = h->grid;
    int dev = h->device, max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    uint32_t n_wg = 5;
    while (n_wg > 1 && tc_smem_bytes(a.img_bytes, n_wg) > (size_t)max_smem) --n_wg;
    const size_t smem = tc_smem_bytes(a.img_bytes, n_wg);
    if (smem > (size_t)max_smem) return cudaErrorInvalidConfiguration;
    uint32_t grid = (a.n_blocks + n_wg - 1) / n_wg;
    if (grid > (uint32_t)h->num_sms) grid = h->num_sms;
    const __half2* hash = reinterpret_cast<const __half2*>(h->hash16);
    const uint32_t threads = n_wg * 128;
    count_kernels(h);  // the cache kernel; FP8 adds an amax roll (and a calibration pair) below
    if (h->cfg.precision == NIRC_BF16_TC)
        return launch_tc_instance<1, false>(grid, threads, smem, st, a, h->packed_tc, hash, recs, base, rows, beta, out_rgba,
                                            lc, lr, sig, count, row_n, err, nullptr);
    if (h->cfg.precision != NIRC_FP8_E4M3_TC)
        return launch_tc_instance<0, false>(grid, threads, smem, st, a, h->packed_tc, hash, recs, base, rows, beta, out_rgba,
                                            lc, lr, sig, count, row_n, err, nullptr);
    cudaError_t e = cudaSuccess;
    uint32_t* amax = h->fp8_amax;
    const uint32_t n_slots = h->shape.hidden - 1;
    if (!h->fp8_calibrated) {
        // one FP16 launch records the activation amax (its image is overwritten below)
        e = launch_tc_instance<0, true>(grid, threads, smem, st, a, h->packed_tc16, hash, recs, base, rows, beta, out_rgba,
                                        nullptr, nullptr, nullptr, nullptr, nullptr, err, amax);
        if (e == cudaSuccess) k_amax_roll<<<1, 32, 0, st>>>(amax, n_slots);
        count_kernels(h, 2);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const_cast<nirc_handle*>(h)->fp8_calibrated = true;
    }
    e = launch_tc_instance<2, true>(grid, threads, smem, st, a, h->packed_tc, hash, recs, base, rows, beta, out_rgba, lc, lr,
                                    sig, count, row_n, err, amax);
    if (e == cudaSuccess) k_amax_roll<<<1, 32, 0, st>>>(amax, n_slots);
    count_kernels(h);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace nirc
