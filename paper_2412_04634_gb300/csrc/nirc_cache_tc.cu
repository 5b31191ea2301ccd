// nirc_cache_tc.cu -- tensor-core (tcgen05, TMEM accumulators) evaluation of
// the cache integral: FP16 operands, split BF16 operands (hi + lo) or E4M3
// hidden layers, always with FP32 accumulation.
//
// Work unit: a block of up to 128 pixels; with S = N + M rows per pixel a
// full block holds exactly S row tiles of 128 rows.  One warpgroup (128
// threads, thread t = tile row t = TMEM lane t) owns a block at a time:
// whole blocks round robin over the launch's warpgroups, then the pixels
// left after the last whole round in equal smaller blocks, one per
// warpgroup (at 1080p a last round of whole blocks ran on 48 of the 152
// SMs); a CTA runs up to five
// warpgroups so that one warpgroup's SIMT work (sampling, encodings,
// epilogues) overlaps another's MMAs.  Each warpgroup owns a slice of tensor
// memory: the accumulator D (64 columns) and the A operand of the next MMA
// (32 columns of packed 16-bit pairs; split BF16: a second 32 for the
// remainders), so the activations go from TMEM to registers to TMEM and
// never through shared memory (E4M3 hidden-layer operands excepted, which
// stay in a swizzled shared tile).
//
//  pixel stage   thread t encodes pixel t's surface (hash grid or frequency
//                position features + normal features) into A; one
//                128x64x64 MMA with the surface columns of layer 0 gives
//                h_pix = W0[:, pix] e_pix + b0 for the 128 pixels, stored as a
//                16-bit K-major operand H in shared memory (K = pixel index;
//                no swizzling, so a K step starts at any multiple of 8 pixels).
//                This is the paper's shared per-surface encoding: computed
//                once per shading point and reused by all its N + M rows.
//  row tile      thread t samples its row's direction (cache rows) or reads
//                it (residual rows), encodes it and writes its A row
//                [e_dir (16) | one-hot of its pixel within a window of the
//                tile's pixels, 16 columns for S >= 16, up to 48 for S >= 4];
//                layer 0 = W0_dir e_dir + H onehot (1 + 1..3 MMAs, K = 16
//                each), then the hidden layers (4 MMAs and a bias MMA each)
//                and the output layer (N = 16, 3 used); each epilogue reads its
//                row from TMEM, applies ReLU, rounds to 16 bits and writes the
//                next A row back to TMEM.  The network input and output never
//                touch global memory.
//  reduction     per-row contributions w * n go to shared memory in row
//                order; per pixel and pair of channels one lane adds its rows
//                in sample order with Kahan compensation (eq. L_mlmc = L_e +
//                L_c + L_r; packed FP32 pairs), carrying the running sums and
//                compensations of a pixel that straddles two tiles; a pixel's
//                four lanes are lanes of one warp, which write the finished
//                pixel.  A tile's sums are formed while the next tile's
//                layer-0 MMA runs.
//
// Split BF16 (NIRC_BF16_TC): every 16-bit operand x is carried as hi =
// bf16(x) and lo = bf16(x - hi); each K step issues hi*hi + lo*hi + hi*lo,
// which keeps about 16 significant bits of every product (BF16's 8 bits
// alone miss the 2e-2 bound on n = exp(z) for trained logits of -6 .. -10).
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
#include <cstring>

#include "nirc_internal.h"
#include "nirc_tc.cuh"

namespace nirc {

size_t tc_image_bytes(uint32_t hidden) { return tcimg::bytes_split(hidden); }

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

constexpr uint32_t kMiscBytes = 256;  // mbarriers, TMEM holder, abort flags, FP8 scales and amax
// Per warpgroup, shared memory: the swizzled operand tiles (1024-byte
// aligned; H, and the E4M3 A tile of FP8 mode or the H remainder of split
// BF16), then apart from them the reduction arrays: row contributions of two
// tiles (2 x 128 x 8 floats: a tile's sums are formed while the next tile's
// first MMA runs) and two carry slots.
constexpr uint32_t kSmallStride = 8192 + 256;
constexpr uint32_t kOffRows = 0, kOffCarry = 8192;  // two row buffers (128 x 32 B each) | carry slots
// Per warpgroup, tensor memory columns: D (64) | A (32) | A remainder (32, split BF16).
constexpr uint32_t kTmD = 0, kTmA = 64, kTmLo = 96;

template <uint32_t AB>
constexpr uint32_t wg_tile_bytes() { return AB == 0 ? 16384u : 32768u; }
template <uint32_t AB>
constexpr uint32_t wg_tmem_cols() { return AB == 1 ? 128u : 96u; }

// What every CTA of a launch shares: the network's shape and encoding.
struct TcArgs {
    float z_clamp;
    uint32_t img_bytes;
    NetShape s;
    GridParams g;
};

// One frame (or cache pass) of a launch: a launch serves up to kTcMaxJobs of
// them at once (the frame-request server's batches), CTAs [cta0, cta0 +
// n_cta) working on job j, each staging that job's weight image once.
struct TcJob {
    const uint8_t* img;          // weight image (the job's cache)
    const __half2* hash16;       // FP16 hash table
    const nirc_record* recs;
    const PixelBase* base;
    const ResidRow* rows;
    const float4* beta;
    float4* out;
    float *lc, *lr, *row_n;
    uint64_t* sig;
    uint32_t* count;
    int* err;                    // the cache's bounded-wait flag
    const SceneHeader* env_hd;   // light mode 2 with a visibility cache: cache values times L_env
    uint64_t s_magic;            // floor(2^40 / S) + 1: x / S = (x * s_magic) >> 40 for x S < 2^40
    uint32_t N, M, k0, k1;
    uint32_t unit_div, purpose;  // Philox counters of the cache samples (CachePass)
    uint32_t env_nprims;
    uint32_t S, P, n_blocks;
    uint32_t cta0, n_cta;
};
constexpr uint32_t kTcMaxJobs = 16;
struct TcJobs {
    uint32_t n;
    TcJob j[kTcMaxJobs];
};

__device__ __forceinline__ uint32_t div_s(uint32_t x, uint64_t magic) {
    return (uint32_t)(((uint64_t)x * magic) >> 40);
}

// relu(lo), relu(hi) rounded to BF16 and the remainders, both packed.
__device__ __forceinline__ void split_relu_bf16(float lo, float hi, uint32_t& w_hi, uint32_t& w_lo) {
    const float a = fmaxf(lo, 0.f), b = fmaxf(hi, 0.f);
    w_hi = tc::pack_bf16(a, b);
    w_lo = tc::pack_bf16(a - __uint_as_float(w_hi << 16), b - __uint_as_float(w_hi & 0xFFFF0000u));
}
__device__ __forceinline__ void split_bf16(float lo, float hi, uint32_t& w_hi, uint32_t& w_lo) {
    w_hi = tc::pack_bf16(lo, hi);
    w_lo = tc::pack_bf16(lo - __uint_as_float(w_hi << 16), hi - __uint_as_float(w_hi & 0xFFFF0000u));
}

// Pack 16 consecutive K elements into 8 words of the operand type (and the
// remainders when kSplit).
template <uint32_t AB16, bool kSplit>
__device__ __forceinline__ void pack8w(const float* x, uint32_t* hi, uint32_t* lo) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if constexpr (kSplit) split_bf16(x[2 * j], x[2 * j + 1], hi[j], lo[j]);
        else hi[j] = pack2<AB16>(x[2 * j], x[2 * j + 1]);
    }
}

// Epilogue of one layer for row r: 64 accumulators from TMEM (two halves of
// 32 columns), times `mul` (kMul: the FP8 scales s_w s_a of the layer),
// + bias (none for layer 0 of the frequency input, whose h_pix holds b0, and
// none for 16-bit layers, whose bias came with the MMA; kHrow: layer 0 of
// the paper's input adds row `pr` of the pixel-major 16-bit tile at `hrow`,
// and with kSplit its remainder tile at `hrow_lo`), ReLU, then either
// 16-bit rounding into the TMEM A operand at `ta` (and the remainders at
// `ta + 32` with kSplit), or, kF8Out, scaling by 1/s_a of the next layer and
// E4M3 rounding into the shared A tile.  kRec: the warp's amax of the ReLU
// outputs goes into the shared word at s_amax (atomicMax on bits).
template <uint32_t AB16, bool kSplit, bool kF8Out, bool kMul, bool kRec, bool kHrow = false>
__device__ __forceinline__ void epilogue(uint32_t tD, uint32_t ta, const float* __restrict__ bias, float mul,
                                         float inv_sa, uint32_t stile, uint32_t r, uint32_t* s_amax,
                                         uint32_t hrow = 0, uint32_t hrow_lo = 0, uint32_t pr = 0) {
    float mx = 0.f;
#pragma unroll
    for (uint32_t half = 0; half < 2; ++half) {
        uint32_t v[32];
        tc::tmem_ld32(tD + 32u * half, v);
        tc::tmem_wait_ld();
        float x[32];
        if constexpr (kHrow) {
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q) {
                const uint32_t c = 4u * half + q;
                const uint32_t off = (pr >> 3) * 1024u + (pr & 7u) * 128u + (((c ^ pr) & 7u) << 4);
                const uint4 hv = tc::lds128(hrow + off);
                uint4 hl = make_uint4(0u, 0u, 0u, 0u);
                if constexpr (kSplit) hl = tc::lds128(hrow_lo + off);
                const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {hl.x, hl.y, hl.z, hl.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float2 hh = tc::unpack2<AB16>(hw[j]);
                    if constexpr (kSplit) {
                        const float2 ll = tc::unpack2<1>(lw[j]);
                        hh.x += ll.x;
                        hh.y += ll.y;
                    }
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
                sts_chunk(stile, r, 2u * half + q, d[0], d[1], d[2], d[3]);
            }
        } else {
            uint32_t w[16];
            if constexpr (kSplit) {
                uint32_t wl[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) split_relu_bf16(x[2 * j], x[2 * j + 1], w[j], wl[j]);
                tc::tmem_st16(ta + 32u + 16u * half, wl);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) w[j] = pack2_relu<AB16>(x[2 * j], x[2 * j + 1]);
            }
            tc::tmem_st16(ta + 16u * half, w);
        }
    }
    if constexpr (kRec) {
        const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
        if ((threadIdx.x & 31u) == 0) atomicMax(s_amax, m);
    }
}

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
        if (AB == 1) {  // split operands: the remainder v - bf16(v), rounded to BF16
            const float rest = v - __bfloat162float(__ushort_as_bfloat16(bits));
            *reinterpret_cast<uint16_t*>(img + tcimg::off_lo(H) + off + tc::sw128_offset(n, k)) =
                __bfloat16_as_ushort(__float2bfloat16_rn(rest));
        }
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

// AB: 0 FP16, 1 split BF16, 2 FP8 hidden layers (FP16 elsewhere).  kAmax:
// record the amax of every hidden layer's input activations into amax[8 + l].
template <uint32_t AB, bool kAmax, bool kSh>
__global__ void __launch_bounds__(640, 1)
    k_cache_tc(TcArgs a, const __grid_constant__ TcJobs jobs, uint32_t* __restrict__ amax) {
    uint32_t ji = 0;  // this CTA's job
    while (ji + 1 < jobs.n && blockIdx.x >= jobs.j[ji + 1].cta0) ++ji;
    const TcJob& J = jobs.j[ji];
    const uint8_t* __restrict__ img_g = J.img;
    const __half2* __restrict__ hash16 = J.hash16;
    const nirc_record* __restrict__ recs = J.recs;
    const PixelBase* __restrict__ base = J.base;
    const ResidRow* __restrict__ rows = J.rows;
    const float4* __restrict__ beta = J.beta;
    float4* __restrict__ out = J.out;
    float* __restrict__ lc_out = J.lc;
    float* __restrict__ lr_out = J.lr;
    uint64_t* __restrict__ sig_out = J.sig;
    uint32_t* __restrict__ count = J.count;
    float* __restrict__ row_n = J.row_n;
    int* __restrict__ err = J.err;
    constexpr uint32_t AB16 = AB == 1 ? 1u : 0u;  // type of the 16-bit layers
    constexpr bool kF8 = AB == 2;
    constexpr bool kSplit = AB == 1;
    constexpr uint32_t kTile = wg_tile_bytes<AB>();
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (sbase - raw);
    const uint32_t n_wg = blockDim.x >> 7;
    const uint32_t wg = threadIdx.x >> 7, t = threadIdx.x & 127u, quarter = t >> 5;
    const uint32_t img_al = (a.img_bytes + 1023u) & ~1023u;
    const uint32_t wgs = sbase + img_al + wg * kTile;      // this warpgroup's operand tiles (shared address)
    const uint32_t small_al = img_al + n_wg * kTile;
    uint8_t* wgg = gbase + small_al + wg * kSmallStride;   // this warpgroup's reduction arrays (generic pointer)
    const uint32_t misc = sbase + small_al + n_wg * kSmallStride;
    uint8_t* miscg = gbase + small_al + n_wg * kSmallStride;
    const uint32_t mbar = misc + 8u * wg;
    volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(miscg + 64);
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(miscg + 80 + 4 * wg);
    uint32_t* s_amax = reinterpret_cast<uint32_t*>(miscg + 128);  // [8]
    float* s_mul = reinterpret_cast<float*>(miscg + 160);         // [8] s_w s_a per hidden slot
    float* s_inv = reinterpret_cast<float*>(miscg + 192);         // [8] 1 / s_a per hidden slot

    // stage the weight image
    {
        const float4* src = reinterpret_cast<const float4*>(img_g);
        float4* dst = reinterpret_cast<float4*>(gbase);
        for (uint32_t i = threadIdx.x; i < a.img_bytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    uint32_t tmem_cols = 32;  // power of two >= the warpgroups' slices
    while (tmem_cols < n_wg * wg_tmem_cols<AB>()) tmem_cols <<= 1;
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
    // tensor memory of this warpgroup: D | A | A remainder; lane base 0 for the MMAs,
    // 32 * quarter for this warp's loads and stores
    const uint32_t tm = *tmem_holder + wg_tmem_cols<AB>() * wg;
    const uint32_t lane = (32u * quarter) << 16;
    const uint32_t tmD = tm + kTmD, tmA = tm + kTmA, tmLo = tm + kTmLo;
    const uint32_t tDr = tmD + lane, tAr = tmA + lane;
    const uint32_t bar_id = 1 + wg;
    uint32_t phase = 0;

    const uint32_t H = a.s.hidden;
    const uint32_t lo_off = tcimg::off_lo(H);  // split BF16: remainder tiles at the same relative offsets
    const uint32_t w0pix = sbase + tcimg::off_w0pix(), w0dir = sbase + tcimg::off_w0dir();
    const uint32_t wout = sbase + tcimg::off_wout(H);
    const float* bias = reinterpret_cast<const float*>(gbase + tcimg::off_bias(H));
    const uint32_t tA8 = wgs;                          // FP8: E4M3 A tile of the hidden layers
    const uint32_t tH = wgs + (kF8 ? 16384u : 0u);     // h_pix operand
    const uint32_t tHlo = wgs + 16384u;                // split BF16: its remainder
    const uint32_t id64 = tc::idesc_f16(AB16, 128, 64), id16 = tc::idesc_f16(AB16, 128, 16);
    const uint32_t id64_e4m3 = tc::idesc_f16(0, 128, 64);  // E4M3 x E4M3 has type code 0 too
    const uint16_t one16 = AB16 ? 0x3F80u : 0x3C00u;
    float* s_rows2 = reinterpret_cast<float*>(wgg + kOffRows);   // [2][128][8] contributions of a tile's rows
    float* s_carry = reinterpret_cast<float*>(wgg + kOffCarry);  // 2 slots x 4 lanes x (sum, comp) pairs
    uint64_t* s_sigc = reinterpret_cast<uint64_t*>(wgg + kOffCarry + 128);  // 2 signature carry slots

    auto sync_wg = [&]() {
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
    // D (+)= A x B^T over K = 16 * n_k with A in TMEM at column a_col (8 columns per
    // K step) and B the swizzled shared tile at b; split BF16 adds lo*hi and hi*lo.
    auto mma_ta = [&](uint32_t a_col, uint32_t b, uint32_t idesc, uint32_t n_k, bool acc0) {
#pragma unroll 1
        for (uint32_t s = 0; s < n_k; ++s) {
            tc::mma_f16_ta(tmD, tmA + a_col + 8u * s, tc::sdesc(b + 32u * s), idesc, (acc0 || s > 0) ? 1u : 0u);
            if constexpr (kSplit) {
                tc::mma_f16_ta(tmD, tmLo + a_col + 8u * s, tc::sdesc(b + 32u * s), idesc, 1u);
                tc::mma_f16_ta(tmD, tmA + a_col + 8u * s, tc::sdesc(b + lo_off + 32u * s), idesc, 1u);
            }
        }
    };
    // 4 K-steps from the TMEM operand, then the bias slot j as one more K = 16 step against the ones atom
    const uint32_t ones = sbase + tcimg::off_ones(H), bmma = sbase + tcimg::off_bmma(H);
    auto issue_layer = [&](uint32_t w_tile, uint32_t idesc, uint32_t j, uint32_t issuer) {
        if (t == issuer && !*abort_flag) {
            tc::fence_after_sync();
            mma_ta(0u, w_tile, idesc, 4u, false);
            tc::mma_f16(tmD, tc::sdesc_rep8(ones), tc::sdesc(bmma + 8192u * (j >> 2) + 32u * (j & 3u)), idesc, 1);
            tc::mma_commit(mbar);
        }
    };
    auto issue_e4m3 = [&](uint32_t b_tile, uint32_t issuer) {
        if (t == issuer && !*abort_flag) {
            tc::fence_after_sync();
#pragma unroll
            for (uint32_t s = 0; s < 2; ++s)
                tc::mma_e4m3(tmD, tc::sdesc(tA8 + 32 * s), tc::sdesc(b_tile + 32 * s), id64_e4m3, s);
            tc::mma_commit(mbar);
        }
    };
    // one 8-feature chunk c of this thread's A row (4 columns; the remainders 32 columns further)
    auto put_chunk = [&](uint32_t c, const float* f) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if constexpr (kSplit) split_bf16(f[2 * j], f[2 * j + 1], hi[j], lo[j]);
            else hi[j] = pack2<AB16>(f[2 * j], f[2 * j + 1]);
        }
        tc::tmem_st4(tAr + 4u * c, hi[0], hi[1], hi[2], hi[3]);
        if constexpr (kSplit) tc::tmem_st4(tAr + 32u + 4u * c, lo[0], lo[1], lo[2], lo[3]);
    };

    const uint32_t S = J.S;
    const uint32_t R_full = 128u * S;
    // blocks of 128 pixels dealt round robin over the job's warpgroups in whole rounds; the
    // pixels left after the last whole round are split evenly (one block of up to 128 pixels
    // each), so no warpgroup runs a whole extra block while the others have finished
    const uint32_t wg_job = (blockIdx.x - J.cta0) * n_wg + wg, n_wg_job = J.n_cta * n_wg;
    const uint32_t rounds = (J.P / 128u) / n_wg_job;
    const uint32_t tail0 = rounds * n_wg_job * 128u, tail = J.P - tail0;
    for (uint32_t k = 0; k <= rounds; ++k) {
        uint32_t p0 = (k * n_wg_job + wg_job) * 128u, npix = 128u;
        if (k == rounds) {
            p0 = tail0 + (uint32_t)((uint64_t)tail * wg_job / n_wg_job);
            npix = tail0 + (uint32_t)((uint64_t)tail * (wg_job + 1u) / n_wg_job) - p0;
            if (npix == 0u) break;
        }
        // ---- per-pixel sums, part 2 (eq. L_mlmc, L_c, L_r) of tile jr (rows j0r .. j0r + 127):
        // four lanes per pixel, each adding a pair of the row buffer's channels over the pixel's
        // rows of this tile in sample order with Kahan compensation (packed FP32 pairs),
        // continuing the carried sums and compensations of a pixel that began in the previous
        // tile: lane g = 0 the cache colours 0 and 1, g = 1 the cache colour 2 and the count
        // (cache rows), g = 2 the residual colours 0 and 1, g = 3 the residual colour 2
        // (residual rows; the other half of its pair is the signature word, summed and
        // dropped).  Pass k takes pixels 32 k .. 32 k + 31 of the tile: pixel qi is lanes
        // 4 (qi % 8) .. 4 (qi % 8) + 3 of warp (qi / 8 + jr) % 4, so a tile of S >= 16 rows per
        // pixel keeps one or two warps busy and the others skip the pass; the busy warp, and
        // with it the scheduler, rotates from tile to tile.  A finished pixel's residual sums
        // reach its cache lanes by warp shuffles and lanes 0 and 1 write it.
        auto reduce_tile = [&](uint32_t jr, uint32_t j0r) {
            const float* rows_r = s_rows2 + 1024u * (jr & 1u);
            const uint32_t pf = div_s(j0r, J.s_magic);
            const uint32_t plast = min(div_s(j0r + 127u, J.s_magic), npix - 1u);
            const uint32_t n_q = plast - pf + 1u;  // pixels with rows in this tile
            const float4* cin = reinterpret_cast<const float4*>(s_carry + 16u * (jr & 1u));  // previous tile's
            float4* cout = reinterpret_cast<float4*>(s_carry + 16u * ((jr + 1u) & 1u));     // next tile's
            const uint32_t lane_t = t & 31u, g = lane_t & 3u;
            const uint32_t wq = ((t >> 5) - jr) & 3u;  // this warp's pixel octet in a pass
            for (uint32_t k = 0; 32u * k < n_q; ++k) {
                if (32u * k + 8u * wq >= n_q) continue;  // warp-uniform: no pixel of this warp in the pass
                const uint32_t qi = 32u * k + 8u * wq + (lane_t >> 2);
                const bool active = qi < n_q;
                const uint32_t q = pf + qi;
                const uint32_t q_lo = q * S, q_hi = q_lo + S;
                const uint32_t lo = max(q_lo, j0r), hi = min(q_hi, j0r + 128u);
                const bool cont_in = q_lo < j0r, cont_out = q_hi > j0r + 128u;
                const uint32_t r_lo = g >= 2u ? max(q_lo + J.N, j0r) : lo;
                const uint32_t r_hi = g >= 2u ? hi : min(q_lo + J.N, hi);
                float2 sum = make_float2(0.f, 0.f), comp = sum;  // comp: what the next add must restore
                if (active) {
                    if (cont_in) {
                        const float4 c = cin[g];
                        sum = make_float2(c.x, c.y);
                        comp = make_float2(c.z, c.w);
                    }
                    const float2* col = reinterpret_cast<const float2*>(rows_r) + g;
#pragma unroll 4
                    for (uint32_t rr = r_lo; rr < r_hi; ++rr) {
                        const float2 y = __fadd2_rn(col[4u * (rr - j0r)], comp);
                        const float2 tt = __fadd2_rn(sum, y);
                        comp = __fadd2_rn(__ffma2_rn(tt, make_float2(-1.f, -1.f), sum), y);  // (sum - tt) + y
                        sum = tt;
                    }
                    if (cont_out) cout[g] = make_float4(sum.x, sum.y, comp.x, comp.y);
                }
                uint64_t sig = kSigInit;
                if (sig_out && active && g == 3u) {
                    // decision signature of the cache samples, in sample order (bit 31 of a
                    // row's word: its pixel's record is valid)
                    if (cont_in) sig = s_sigc[jr & 1u];
                    const uint32_t c_lo = lo, c_hi = min(q_lo + J.N, hi);
                    for (uint32_t rr = c_lo; rr < c_hi; ++rr) {
                        const uint32_t wd = __float_as_uint(rows_r[8u * (rr - j0r) + 7u]);
                        if (wd >> 31) sig = sig_mix(sig, wd & 0x7FFFFFFFu);
                    }
                    if (cont_out) s_sigc[(jr + 1u) & 1u] = sig;
                }
                // cache lane g (0, 1) takes the residual pair of lane g + 2
                const float rx = __shfl_down_sync(0xffffffffu, sum.x, 2);
                const float ry = __shfl_down_sync(0xffffffffu, sum.y, 2);
                if (!active || cont_out) continue;
                const uint32_t gp = p0 + q;
                if (g < 2u) {
                    // the finished pixel: lane 0 colour channels 0 and 1, lane 1 channel 2, alpha and the count
                    const float* bp = base ? reinterpret_cast<const float*>(base + gp) : nullptr;
                    const uint32_t c0 = 2u * g;
                    float2 Lc = make_float2(0.f, 0.f);
                    if (J.N) Lc = make_float2(sum.x * (1.0f / (float)J.N), g ? 0.f : sum.y * (1.0f / (float)J.N));
                    float2 Lr = bp ? make_float2(bp[4 + c0], g ? 0.f : bp[5]) : make_float2(0.f, 0.f);
                    if (J.M && J.N) {  // without a cache level nothing is subtracted
                        Lr.x -= rx * (1.0f / (float)J.M);
                        if (!g) Lr.y -= ry * (1.0f / (float)J.M);
                    }
                    if (beta) {  // the unit's throughput (biased stopping vertex, later vertex of a residual path)
                        const float* bt = reinterpret_cast<const float*>(beta + gp);
                        const float b0 = bt[c0], b1 = g ? 0.f : bt[1];
                        Lc = make_float2(Lc.x * b0, Lc.y * b1);
                        Lr = make_float2(Lr.x * b0, Lr.y * b1);
                    }
                    const float2 le = bp ? make_float2(bp[c0], g ? 0.f : bp[1]) : make_float2(0.f, 0.f);
                    const float2 o = make_float2(le.x + Lc.x + Lr.x, g ? 1.f : le.y + Lc.y + Lr.y);
                    reinterpret_cast<float2*>(out + gp)[g] = o;
                    if (lc_out) {
                        lc_out[3 * (uint64_t)gp + c0] = Lc.x;
                        if (!g) lc_out[3 * (uint64_t)gp + 1] = Lc.y;
                    }
                    if (lr_out) {
                        lr_out[3 * (uint64_t)gp + c0] = Lr.x;
                        if (!g) lr_out[3 * (uint64_t)gp + 1] = Lr.y;
                    }
                    if (g && count) count[gp] += (uint32_t)sum.y;
                } else if (g == 3u && sig_out) {
                    sig_out[2 * (uint64_t)gp + 1] = sig;
                }
            }
        };

        // ------------------------------------------------ pixel stage
        {
            float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
            if (t < npix) {
                const float4* rq = reinterpret_cast<const float4*>(recs + p0 + t);
                r0 = __ldg(rq);
                r1 = __ldg(rq + 1);
                // into L2, what later stages read first: the record's second half and the pixel's
                // residual rows (row tiles), its base and throughput (per-pixel sums)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(rq + 2));
                if (J.M) asm volatile("prefetch.global.L2 [%0];" ::"l"(rows + (uint64_t)(p0 + t) * J.M));
                if (base) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + p0 + t));
                if (beta) asm volatile("prefetch.global.L2 [%0];" ::"l"(beta + p0 + t));
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
                    put_chunk(c, f);
                }
            } else {
                freq4(p.x, f);
                put_chunk(c++, f);
                freq4(p.y, f);
                put_chunk(c++, f);
                freq4(p.z, f);
                put_chunk(c++, f);
            }
            if constexpr (kSh) {
                float ph[16];
                phi_features(n, make_float3(r2.y, r2.z, r2.w), r3.x, ph);
                ph[15] = 0.f;
                put_chunk(c++, ph);
                put_chunk(c++, ph + 8);
            } else {
                freq4(n.x, f);
                put_chunk(c++, f);
                freq4(n.y, f);
                put_chunk(c++, f);
                freq4(n.z, f);
                put_chunk(c++, f);
            }
            for (uint32_t j = 0; j < 8; ++j) f[j] = 0.f;
            for (; c < 8; ++c) put_chunk(c, f);
        }
        tc::tmem_wait_st();
        sync_wg();
        if (t == 0 && !*abort_flag) {
            tc::fence_after_sync();
            mma_ta(0u, w0pix, id64, 4u, false);
            tc::mma_commit(mbar);
        }
        wait_mma();
        if constexpr (kSh) {
            // H pixel-major: row t = h_pix of pixel t = accumulator + b0, 16-bit (+ remainder)
#pragma unroll
            for (uint32_t half = 0; half < 2; ++half) {
                uint32_t v[32];
                tc::tmem_ld32(tDr + 32u * half, v);
                tc::tmem_wait_ld();
#pragma unroll
                for (uint32_t q = 0; q < 4; ++q) {
                    float y[8];
#pragma unroll
                    for (uint32_t j = 0; j < 8; ++j) y[j] = __uint_as_float(v[8 * q + j]) + bias[32 * half + 8 * q + j];
                    if constexpr (kSplit) {
                        uint32_t hi[4], lo[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) split_bf16(y[2 * j], y[2 * j + 1], hi[j], lo[j]);
                        sts_chunk(tH, t, 4 * half + q, hi[0], hi[1], hi[2], hi[3]);
                        sts_chunk(tHlo, t, 4 * half + q, lo[0], lo[1], lo[2], lo[3]);
                    } else {
                        sts_chunk8<AB16>(tH, t, 4 * half + q, y);
                    }
                }
            }
        } else {
            // H operand: element (n = output unit, k = pixel t), h = accumulator + b0 (+ remainder),
            // K-major without swizzling: core matrix (n / 8, t / 8) at (n / 8) * 2048 + (t / 8) * 128,
            // so a K step may start at any multiple of 8 pixels
            const uint32_t hk = (t >> 3) * 128u + (t & 7u) * 2u;
#pragma unroll
            for (uint32_t half = 0; half < 2; ++half) {
                uint32_t v[32];
                tc::tmem_ld32(tDr + 32u * half, v);
                tc::tmem_wait_ld();
#pragma unroll
                for (uint32_t o = 0; o < 32; ++o) {
                    const uint32_t oo = 32u * half + o;
                    const float hv = __uint_as_float(v[o]) + bias[oo];
                    const uint16_t hb = to16<AB16>(hv);
                    const uint32_t off = hk + (oo >> 3) * 2048u + (oo & 7u) * 16u;
                    tc::sts16(tH + off, hb);
                    if constexpr (kSplit) {
                        const float rest = hv - __uint_as_float((uint32_t)hb << 16);
                        tc::sts16(tHlo + off, to16<1>(rest));
                    }
                }
            }
        }
        tc::fence_proxy_async();  // H is an MMA operand (frequency input)
        sync_wg();

        // ------------------------------------------------ row tiles
        const uint32_t R = npix * S;
        uint32_t jt = 0;
        // kCarry: a lane's record for the next tile is loaded while the current tile's output
        // layer runs (16 registers across the output epilogue; the instances whose register
        // budget has no room for them load it at the tile's start)
        constexpr bool kCarry = AB == 0 && !kAmax && !kSh;
        float4 nq0, nq1, nq2, nq3;
        if constexpr (kCarry) {
            const float4* rq = reinterpret_cast<const float4*>(recs + p0 + (t < R ? div_s(t, J.s_magic) : 0u));
            nq0 = __ldg(rq);
            nq1 = __ldg(rq + 1);
            nq2 = __ldg(rq + 2);
            nq3 = __ldg(rq + 3);
        }
        for (uint32_t j0 = 0; j0 < R; j0 += 128u, ++jt) {
            const uint32_t r = j0 + t;
            const bool rin = r < R;
            const uint32_t pl = rin ? div_s(r, J.s_magic) : 0u;
            const uint32_t s = rin ? r - pl * S : 0u;
            const uint32_t pf = div_s(j0, J.s_magic);
            const uint32_t plast = min(div_s(min(j0 + 127u, R_full - 1u), J.s_magic), npix - 1u);
            // one-hot window [kb, kb + 16 n_oh) covers pixels pf..plast and stays inside H's 128
            // columns (1 K step for S >= 16, at most 3 for S >= 4)
            const uint32_t n_oh = (plast - (pf & ~7u) + 16u) >> 4;
            const uint32_t kb = min(pf & ~7u, 128u - 16u * n_oh);

            V3 wi{0.f, 0.f, 1.f};
            float3 w = make_float3(0.f, 0.f, 0.f);
            bool ok = false;
            uint32_t word = 0;
            {
                // all four words of the record at once (one round trip; with kCarry already here)
                float4 q0, q1, q2, q3;
                if constexpr (kCarry) {
                    q0 = nq0;
                    q1 = nq1;
                    q2 = nq2;
                    q3 = nq3;
                } else {
                    const float4* rq = reinterpret_cast<const float4*>(recs + p0 + pl);
                    q0 = __ldg(rq);
                    q1 = __ldg(rq + 1);
                    q2 = __ldg(rq + 2);
                    q3 = __ldg(rq + 3);
                }
                const uint32_t flags = __float_as_uint(q3.z);
                word = (flags & 1u) << 31;  // the pixel's record is valid (signature)
                if (rin && (flags & 1u)) {
                    if (s < J.N) {
                        // Philox counter of the sample: (unit / unit_div, (unit % unit_div) << 16 | s)
                        const uint32_t u = p0 + pl;
                        const uint32_t c0 = J.unit_div == 1u ? u : u / J.unit_div;
                        const uint32_t c1 = J.unit_div == 1u ? s : (((u - c0 * J.unit_div) << 16) | s);
                        const BsdfSample bs =
                            sample_bsdf(V3{q0.w, q1.x, q1.y}, V3{q1.z, q1.w, q2.x}, make_float3(q2.y, q2.z, q2.w),
                                        q3.x, (flags >> 1) & 3u, J.k0, J.k1, c0, c1, J.purpose);
                        wi = bs.wi;
                        w = bs.w;
                        ok = bs.valid;
                        word |= bs.word;
                    } else {
                        const ResidRow* rr = rows + (uint64_t)(p0 + pl) * J.M + (s - J.N);
                        const float4 d = __ldg(&rr->wi), ww = __ldg(&rr->w);
                        wi = V3{d.x, d.y, d.z};
                        w = make_float3(ww.x, ww.y, ww.z);
                        ok = d.w != 0.f;
                    }
                }
            }
            if constexpr (kSh) {
                // columns 0..31 of the row: the 25 spherical harmonics, zero padded (layer 0 reads K = 32)
                float e[32];
                sh_basis25(wi, e);
#pragma unroll
                for (int i = 25; i < 32; ++i) e[i] = 0.f;
#pragma unroll
                for (uint32_t c = 0; c < 4; ++c) put_chunk(c, e + 8 * c);
            } else {
                float e[16];
                dir_features_fast(wi, e);
                put_chunk(0u, e);
                put_chunk(1u, e + 8);
                // one-hot of the row's pixel among K columns 16 .. 16 + 16 n_oh (words 8 .. 8 + 8 n_oh
                // of the row; the MMAs read no further)
                const uint32_t oh = rin ? pl - kb : 0xFFFFu;
                const uint32_t ow = oh >> 1, ov = (uint32_t)one16 << ((oh & 1u) * 16u);
                for (uint32_t qq = 0; qq < n_oh; ++qq) {  // uniform over the warpgroup
                    uint32_t d8[8];
#pragma unroll
                    for (uint32_t j = 0; j < 8; ++j) d8[j] = ow == 8u * qq + j ? ov : 0u;
                    tc::tmem_st8(tAr + 8u + 8u * qq, d8);
                }
            }
            tc::tmem_wait_st();
            sync_wg();
            if (t == 32u * (jt & 3u) && !*abort_flag) {  // the issuing warp rotates from tile to tile
                tc::fence_after_sync();
                if constexpr (kSh) {
                    mma_ta(0u, w0dir, id64, 2u, false);
                } else {
                    mma_ta(0u, w0dir, id64, 1u, false);
                    for (uint32_t qq = 1; qq <= n_oh; ++qq) {
                        const uint32_t hoff = ((kb >> 3) + 2u * (qq - 1)) * 128u;  // K = kb + 16 (qq - 1)
                        tc::mma_f16_ta(tmD, tmA + 8u * qq, tc::sdesc_noswz(tH + hoff, 128u, 2048u), id64, 1);
                        if constexpr (kSplit)
                            tc::mma_f16_ta(tmD, tmA + 8u * qq, tc::sdesc_noswz(tHlo + hoff, 128u, 2048u), id64, 1);
                    }
                }
                tc::mma_commit(mbar);
            }
            if (jt > 0) reduce_tile(jt - 1u, j0 - 128u);  // the previous tile's sums, while layer 0 runs
            wait_mma();
            for (uint32_t l = 0; l < H; ++l) {
                // epilogue of layer l (l = 0: h_pix already holds b0; 16-bit hidden layers: the
                // bias came with the MMA), then the MMAs of layer l + 1
                const float* bl = (l == 0 || !kF8) ? nullptr : bias + 64 + (l - 1) * 64;
                const bool next_hidden = l + 1 < H;
                if (kSh && l == 0) {
                    // layer 0 of the paper's input: + h_pix of the row's pixel (H row pl)
                    if constexpr (kF8) {
                        if (next_hidden)
                            epilogue<0, false, true, false, true, true>(tDr, tAr, nullptr, 1.f, s_inv[0], tA8, t,
                                                                        s_amax, tH, 0u, pl);
                        else
                            epilogue<0, false, false, false, false, true>(tDr, tAr, nullptr, 1.f, 1.f, tA8, t,
                                                                          nullptr, tH, 0u, pl);
                    } else if constexpr (kAmax) {
                        if (next_hidden)
                            epilogue<AB16, kSplit, false, false, true, true>(tDr, tAr, nullptr, 1.f, 1.f, 0u, t,
                                                                             s_amax, tH, tHlo, pl);
                        else
                            epilogue<AB16, kSplit, false, false, false, true>(tDr, tAr, nullptr, 1.f, 1.f, 0u, t,
                                                                              nullptr, tH, tHlo, pl);
                    } else {
                        epilogue<AB16, kSplit, false, false, false, true>(tDr, tAr, nullptr, 1.f, 1.f, 0u, t,
                                                                          nullptr, tH, tHlo, pl);
                    }
                } else if constexpr (kF8) {
                    const float mul = l == 0 ? 1.f : s_mul[l - 1];
                    if (next_hidden) epilogue<0, false, true, true, true>(tDr, tAr, bl, mul, s_inv[l], tA8, t, s_amax + l);
                    else epilogue<0, false, false, true, false>(tDr, tAr, bl, mul, 1.f, tA8, t, nullptr);
                } else if constexpr (kAmax) {
                    if (next_hidden) epilogue<AB16, kSplit, false, false, true>(tDr, tAr, bl, 1.f, 1.f, 0u, t, s_amax + l);
                    else epilogue<AB16, kSplit, false, false, false>(tDr, tAr, bl, 1.f, 1.f, 0u, t, nullptr);
                } else {
                    epilogue<AB16, kSplit, false, false, false>(tDr, tAr, bl, 1.f, 1.f, 0u, t, nullptr);
                }
                if (kF8 && next_hidden) tc::fence_proxy_async();  // E4M3 operand in shared memory
                else tc::tmem_wait_st();                           // 16-bit operand in TMEM
                sync_wg();
                if (next_hidden) {
                    if constexpr (kF8) issue_e4m3(sbase + tcimg::off_wh(l), 32u * ((jt + l + 1u) & 3u));
                    else issue_layer(sbase + tcimg::off_wh(l), id64, l, 32u * ((jt + l + 1u) & 3u));
                } else {
                    issue_layer(wout, id16, H - 1u, 32u * ((jt + l + 1u) & 3u));
                    if constexpr (kCarry) {
                        if (r + 128u < R) {  // the next tile's record of this lane's row (rows past R: unused)
                            const float4* rq =
                                reinterpret_cast<const float4*>(recs + p0 + div_s(r + 128u, J.s_magic));
                            nq0 = __ldg(rq);
                            nq1 = __ldg(rq + 1);
                            nq2 = __ldg(rq + 2);
                            nq3 = __ldg(rq + 3);
                        }
                    }
                }
                wait_mma();
            }
            float3 nv;
            {
                uint32_t v[4];
                tc::tmem_ld4(tDr, v);
                tc::tmem_wait_ld();
                const bool vis = a.s.vis;  // the output bias came with the MMA
                nv.x = out_act_fast(vis, __uint_as_float(v[0]), a.z_clamp);
                nv.y = out_act_fast(vis, __uint_as_float(v[1]), a.z_clamp);
                nv.z = out_act_fast(vis, __uint_as_float(v[2]), a.z_clamp);
                if (J.env_hd && ok) {  // visibility cache: n = V L_env(w)
                    const float3 le = env_radiance(env_from(J.env_hd, J.env_nprims), wi);
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
            // ---- per-pixel sums, part 1: each row's contributions c_r = w_r n_r (cache
            // rows in channels 0-2 with 1 per valid cache sample in 3, residual rows in 4-6)
            // and its signature word (7) go to this tile's row buffer; the sums follow while
            // the next tile's first MMA runs (reduce_tile)
            {
                const bool is_cache = s < J.N;
                const float3 cw = ok ? make_float3(w.x * nv.x, w.y * nv.y, w.z * nv.z) : make_float3(0.f, 0.f, 0.f);
                float4* sr = reinterpret_cast<float4*>(s_rows2 + 1024u * (jt & 1u)) + 2 * t;
                sr[0] = is_cache ? make_float4(cw.x, cw.y, cw.z, (ok ? 1.f : 0.f)) : make_float4(0.f, 0.f, 0.f, 0.f);
                sr[1] = is_cache ? make_float4(0.f, 0.f, 0.f, __uint_as_float(word))
                                 : make_float4(cw.x, cw.y, cw.z, __uint_as_float(word));
            }
        }
        // the last tile's sums (its rows staged by every warp before this barrier)
        tc::named_bar(bar_id, 128);
        reduce_tile(jt - 1u, (jt - 1u) * 128u);
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

template <uint32_t AB>
static size_t tc_smem_bytes(uint32_t img_bytes, uint32_t n_wg) {
    return 1024 + ((img_bytes + 1023) & ~1023u) + (size_t)n_wg * (wg_tile_bytes<AB>() + kSmallStride) + kMiscBytes;
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
           fd.cache_mode == 0 && fd.n_cache + fd.n_resid >= (h->shape.sh ? 1u : 4u) &&
           fd.n_cache + fd.n_resid < 65536u && h->packed_tc != nullptr &&
           (h->shape.n_pos == 24 || h->shape.n_pos == 32);
}

template <uint32_t AB, bool kAmax, bool kSh>
static cudaError_t launch_tc_kernel(uint32_t grid, uint32_t threads, size_t smem, cudaStream_t st, const TcArgs& a,
                                    const TcJobs& jobs, uint32_t* amax) {
    cudaError_t e =
        cudaFuncSetAttribute(k_cache_tc<AB, kAmax, kSh>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_cache_tc<AB, kAmax, kSh><<<grid, threads, smem, st>>>(a, jobs, amax);
    return cudaGetLastError();
}

// The instance for the network input of a.s (frequency or the paper's).
template <uint32_t AB, bool kAmax>
static cudaError_t launch_tc_instance(uint32_t grid, uint32_t threads, size_t smem, cudaStream_t st, const TcArgs& a,
                                      const TcJobs& jobs, uint32_t* amax) {
    if (a.s.sh) return launch_tc_kernel<AB, kAmax, true>(grid, threads, smem, st, a, jobs, amax);
    return launch_tc_kernel<AB, kAmax, false>(grid, threads, smem, st, a, jobs, amax);
}

// Warpgroups per CTA for operand type AB: as many as shared and tensor memory hold (<= 5).
template <uint32_t AB>
static uint32_t tc_warpgroups(uint32_t img_bytes, int max_smem, size_t* smem) {
    uint32_t n_wg = 5;
    while (n_wg > 1 && (tc_smem_bytes<AB>(img_bytes, n_wg) > (size_t)max_smem || n_wg * wg_tmem_cols<AB>() > 512u))
        --n_wg;
    *smem = tc_smem_bytes<AB>(img_bytes, n_wg);
    return n_wg;
}

static TcArgs tc_args(const nirc_handle* h) {
    TcArgs a;
    a.z_clamp = h->cfg.z_clamp;
    a.s = h->shape;
    a.g = h->grid;
    a.img_bytes = h->cfg.precision == NIRC_BF16_TC ? tcimg::bytes_split(h->shape.hidden)
                                                   : tcimg::bytes_hi(h->shape.hidden);
    return a;
}

static TcJob tc_job(const nirc_handle* h, const nirc_frame_desc& fd, const nirc_record* recs, const PixelBase* base,
                    const ResidRow* rows, const float4* beta, float* out_rgba, float* lc, float* lr, uint64_t* sig,
                    uint32_t* count, float* row_n, int* err, CachePass pass, EnvSource env) {
    TcJob j{};
    j.img = reinterpret_cast<const uint8_t*>(h->packed_tc);
    j.hash16 = reinterpret_cast<const __half2*>(h->hash16);
    j.recs = recs;
    j.base = base;
    j.rows = rows;
    j.beta = beta;
    j.out = reinterpret_cast<float4*>(out_rgba);
    j.lc = lc;
    j.lr = lr;
    j.row_n = row_n;
    j.sig = sig;
    j.count = count;
    j.err = err;
    j.env_hd = reinterpret_cast<const SceneHeader*>(env.scene);
    j.env_nprims = env.n_prims;
    j.N = fd.n_cache;
    j.M = fd.n_resid;
    j.k0 = (uint32_t)fd.seed;
    j.k1 = fd.frame;
    j.unit_div = pass.unit_div;
    j.purpose = pass.purpose;
    j.S = fd.n_cache + fd.n_resid;
    j.s_magic = (1ull << 40) / j.S + 1;
    j.P = fd.width * fd.height;
    j.n_blocks = (j.P + 127) / 128;
    return j;
}

static uint32_t tc_launch_shape(const nirc_handle* h, uint32_t img_bytes, size_t* smem) {
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    const nirc_precision p = (nirc_precision)h->cfg.precision;
    const uint32_t n_wg = p == NIRC_BF16_TC ? tc_warpgroups<1>(img_bytes, max_smem, smem)
                                            : (p == NIRC_FP8_E4M3_TC ? tc_warpgroups<2>(img_bytes, max_smem, smem)
                                                                      : tc_warpgroups<0>(img_bytes, max_smem, smem));
    return *smem > (size_t)max_smem ? 0u : n_wg;
}

cudaError_t launch_cache_tc(const nirc_handle* h, const nirc_frame_desc& fd, const nirc_record* recs,
                            const PixelBase* base, const ResidRow* rows, const float4* beta, float* out_rgba,
                            float* lc, float* lr, uint64_t* sig, uint32_t* count, float* row_n, int* err,
                            cudaStream_t st, CachePass pass, EnvSource env) {
    const TcArgs a = tc_args(h);
    TcJobs jobs;
    jobs.n = 1;
    jobs.j[0] = tc_job(h, fd, recs, base, rows, beta, out_rgba, lc, lr, sig, count, row_n, err, pass, env);
    size_t smem = 0;
    const uint32_t n_wg = tc_launch_shape(h, a.img_bytes, &smem);
    if (!n_wg) return cudaErrorInvalidConfiguration;
    uint32_t grid = (jobs.j[0].n_blocks + n_wg - 1) / n_wg;
    if (grid > (uint32_t)h->num_sms) grid = h->num_sms;
    jobs.j[0].cta0 = 0;
    jobs.j[0].n_cta = grid;
    const uint32_t threads = n_wg * 128;
    count_kernels(h);  // the cache kernel; FP8 adds an amax roll (and a calibration pair) below
    if (h->cfg.precision == NIRC_BF16_TC) return launch_tc_instance<1, false>(grid, threads, smem, st, a, jobs, nullptr);
    if (h->cfg.precision != NIRC_FP8_E4M3_TC)
        return launch_tc_instance<0, false>(grid, threads, smem, st, a, jobs, nullptr);
    cudaError_t e = cudaSuccess;
    uint32_t* amax = h->fp8_amax;
    const uint32_t n_slots = h->shape.hidden - 1;
    if (!h->fp8_calibrated) {
        // one FP16 launch records the activation amax (its image is overwritten below); it
        // runs with the FP8 launch's warpgroup count, whose shared memory covers the FP16 layout
        TcJobs cal = jobs;
        cal.j[0].img = reinterpret_cast<const uint8_t*>(h->packed_tc16);
        cal.j[0].lc = cal.j[0].lr = cal.j[0].row_n = nullptr;
        cal.j[0].sig = nullptr;
        cal.j[0].count = nullptr;
        e = launch_tc_instance<0, true>(grid, threads, smem, st, a, cal, amax);
        if (e == cudaSuccess) k_amax_roll<<<1, 32, 0, st>>>(amax, n_slots);
        count_kernels(h, 2);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const_cast<nirc_handle*>(h)->fp8_calibrated = true;
    }
    e = launch_tc_instance<2, true>(grid, threads, smem, st, a, jobs, amax);
    if (e == cudaSuccess) k_amax_roll<<<1, 32, 0, st>>>(amax, n_slots);
    count_kernels(h);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

bool tc_batchable(const nirc_handle* a, const nirc_handle* b) {
    return (a->cfg.precision == NIRC_FP16_TC || a->cfg.precision == NIRC_BF16_TC) &&
           a->cfg.precision == b->cfg.precision && memcmp(&a->shape, &b->shape, sizeof(NetShape)) == 0 &&
           memcmp(&a->grid, &b->grid, sizeof(GridParams)) == 0 && a->cfg.z_clamp == b->cfg.z_clamp;
}

cudaError_t launch_cache_tc_batch(const FrameJob* fj, uint32_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (n > kTcMaxJobs) return cudaErrorInvalidValue;
    const nirc_handle* h0 = fj[0].h;
    const TcArgs a = tc_args(h0);
    size_t smem = 0;
    const uint32_t n_wg = tc_launch_shape(h0, a.img_bytes, &smem);
    if (!n_wg) return cudaErrorInvalidConfiguration;
    TcJobs jobs;
    jobs.n = n;
    uint64_t rows_total = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const FrameJob& f = fj[i];
        if (!tc_batchable(h0, f.h) || !tc_supported(f.h, f.fd)) return cudaErrorInvalidValue;
        jobs.j[i] = tc_job(f.h, f.fd, f.recs, f.base, f.rows, nullptr, f.out, nullptr, nullptr, nullptr, nullptr,
                           nullptr, f.h->dev_err, CachePass{}, EnvSource{});
        rows_total += (uint64_t)jobs.j[i].n_blocks * jobs.j[i].S;
    }
    // CTAs in proportion to each job's row tiles, at least one each and no more than it can use
    const uint32_t grid_max = (uint32_t)h0->num_sms;
    if (grid_max < n) return cudaErrorInvalidConfiguration;
    uint32_t cta = 0;
    for (uint32_t i = 0; i < n; ++i) {
        TcJob& j = jobs.j[i];
        const uint64_t tiles = (uint64_t)j.n_blocks * j.S;
        uint64_t share = tiles * (grid_max - n) / rows_total + 1;  // the shares add up to <= grid_max
        const uint64_t useful = (j.n_blocks + n_wg - 1) / n_wg;
        if (share > useful) share = useful;
        j.cta0 = cta;
        j.n_cta = (uint32_t)share;
        cta += (uint32_t)share;
    }
    const uint32_t threads = n_wg * 128;
    for (uint32_t i = 0; i < n; ++i) count_kernels(fj[i].h);
    if (h0->cfg.precision == NIRC_BF16_TC) return launch_tc_instance<1, false>(cta, threads, smem, st, a, jobs, nullptr);
    return launch_tc_instance<0, false>(cta, threads, smem, st, a, jobs, nullptr);
}

}  // namespace nirc
