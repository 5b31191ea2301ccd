// nirc_cache_simt.cu -- FP32 SIMT evaluation of the cache integral.
//
// One thread per shading point (pixel).  The per-surface part of the
// network input (position and normal encodings) and its first-layer
// product h_pix = W0[:, pix] e_pix + b0 are computed once per pixel and
// shared by its N + M rows (paper: shared surface encodings amortised over
// all requests of a surface, section "Neural Network Architecture").  Each
// row then only encodes its direction (16 features), finishes layer 0,
// runs the hidden layers and the exp output, and adds its term to the
// pixel's two Monte Carlo levels (eq. L_c and L_r) with compensated FP32
// sums; nothing per row is written to global memory.
//
// Weights live in shared memory transposed ([in][64]) so that each input
// reads one row of 64 outputs as broadcast float4 loads; the FMAs are
// packed FP32x2 (fma.rn.f32x2).  Activations round-trip through a per-thread
// shared-memory column (layout [unit][thread], conflict free).
#include "nirc_internal.h"
#include "nirc_simt.cuh"

namespace nirc {

constexpr int kSimtThreads = 128;

struct CacheArgs {
    uint32_t W, H, N, M, k0, k1;
    uint32_t unit_div, purpose;  // Philox counters of the cache samples (CachePass)
    const SceneHeader* env_hd;   // light mode 2 with a visibility cache: cache values times L_env
    uint32_t env_nprims;
    uint32_t cache_mode;
    float cc0, cc1, cc2;
    float z_clamp;
    NetShape s;
    GridParams g;
};

// h_pix = b0 + W0[:, pix] e_pix  (e_pix already in act)
__device__ __forceinline__ void surface_product(const NetShape& s, const float* __restrict__ sw, float* act, int stride,
                                                float2 (&hpix)[32]) {
    load_bias(hpix, sw + s.off_b0);
    for (uint32_t i = 0; i < s.n_pix; ++i) fma_row(hpix, sw + s.off_wpix + i * kWidth, act[i * stride]);
}

// One row: direction features -> layer 0 (with h_pix) -> hidden -> logits.
template <bool kSh>
__device__ __forceinline__ float3 row_mlp(const NetShape& s, const float* __restrict__ sw, float* act, int stride,
                                          const float2 (&hpix)[32], V3 wi, float z_clamp) {
    constexpr int nd = dir_features<kSh>();
    float e[nd];
    dir_encode<kSh>(wi, e);
    float2 acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = hpix[q];
#pragma unroll
    for (int i = 0; i < nd; ++i) fma_row(acc, sw + s.off_wdir + i * kWidth, e[i]);
    for (uint32_t l = 1; l < s.hidden; ++l) {
        store_relu(acc, act, stride);
        const float* Wl = sw + s.off_hidden + (l - 1) * (kWidth * kWidth + kWidth);
        load_bias(acc, Wl + kWidth * kWidth);
#pragma unroll 2
        for (int i = 0; i < (int)kWidth; ++i) fma_row(acc, Wl + i * kWidth, act[i * stride]);
    }
    // output layer straight from registers
    const float* Wo = sw + s.off_out;
    float2 z01 = make_float2(Wo[256], Wo[257]);
    float2 z23 = make_float2(Wo[258], Wo[259]);
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const float a0 = fmaxf(acc[q].x, 0.f), a1 = fmaxf(acc[q].y, 0.f);
        const float4 w0 = *reinterpret_cast<const float4*>(Wo + (2 * q) * 4);
        const float4 w1 = *reinterpret_cast<const float4*>(Wo + (2 * q + 1) * 4);
        z01 = __ffma2_rn(make_float2(w0.x, w0.y), make_float2(a0, a0), z01);
        z23 = __ffma2_rn(make_float2(w0.z, w0.w), make_float2(a0, a0), z23);
        z01 = __ffma2_rn(make_float2(w1.x, w1.y), make_float2(a1, a1), z01);
        z23 = __ffma2_rn(make_float2(w1.z, w1.w), make_float2(a1, a1), z23);
    }
    const bool vis = s.vis;
    return make_float3(out_act(vis, z01.x, z_clamp), out_act(vis, z01.y, z_clamp), out_act(vis, z23.x, z_clamp));
}

template <bool kSh>
__global__ void __launch_bounds__(kSimtThreads, 1)
    k_cache_simt(CacheArgs a, const float* __restrict__ packed, const float* __restrict__ table,
                 const nirc_record* __restrict__ recs, const PixelBase* __restrict__ base,
                 const ResidRow* __restrict__ rows, const float4* __restrict__ beta, float4* __restrict__ out,
                 float* __restrict__ lc_out, float* __restrict__ lr_out, uint64_t* __restrict__ sig_out,
                 uint32_t* __restrict__ count,
                 float* __restrict__ row_n) {
    extern __shared__ __align__(16) float smem[];
    float* sw = smem;
    float* act = smem + a.s.packed_floats + threadIdx.x;
    const int stride = kSimtThreads;
    stage_weights(sw, packed, a.s.packed_floats);
    __syncthreads();

    const uint64_t P = (uint64_t)a.W * a.H;
    const bool network = a.cache_mode == 0;
    const EnvMap env = env_from(a.env_hd, a.env_nprims);
    // Every lane of a block runs the same number of iterations (warp votes below).
    for (uint64_t first = (uint64_t)blockIdx.x * kSimtThreads; first < P; first += (uint64_t)gridDim.x * kSimtThreads) {
        const uint64_t pix64 = first + threadIdx.x;
        const bool in_range = pix64 < P;
        const uint32_t pix = in_range ? (uint32_t)pix64 : 0u;
        const float4* rq = reinterpret_cast<const float4*>(recs + pix);
        const float4 r0 = __ldg(rq), r1 = __ldg(rq + 1), r2 = __ldg(rq + 2), r3 = __ldg(rq + 3);
        const uint32_t flags = in_range ? __float_as_uint(r3.z) : 0u;
        const bool valid = flags & 1u;
        const V3 p{r0.x, r0.y, r0.z}, n{r0.w, r1.x, r1.y}, wo{r1.z, r1.w, r2.x};
        const float3 alb = make_float3(r2.y, r2.z, r2.w);
        const float rough = r3.x;
        const uint32_t mat = (flags >> 1) & 3u;

        float2 hpix[32];
        if (network && __any_sync(0xffffffffu, valid)) {
            encode_surface(a.s, a.g, table, p, n, alb, rough, act, stride);
            surface_product(a.s, sw, act, stride, hpix);
        }
        Kahan3 lc, sub;
        uint64_t sig = kSigInit;
        uint32_t nvalid = 0;
        const uint32_t S = a.N + a.M;
        // Philox counter of cache sample r: (unit / unit_div, (unit % unit_div) << 16 | r)
        const uint32_t sc0 = pix / a.unit_div, sc1 = (pix - sc0 * a.unit_div) << 16;
        for (uint32_t r = 0; r < S; ++r) {
            V3 wi;
            float3 w;
            bool ok;
            if (r < a.N) {
                BsdfSample bs;
                if (valid) {
                    bs = sample_bsdf(n, wo, alb, rough, mat, a.k0, a.k1, sc0, sc1 | r, a.purpose);
                    sig = sig_mix(sig, bs.word);
                } else {
                    bs.valid = false;
                    bs.wi = V3{0.f, 0.f, 1.f};
                    bs.w = make_float3(0.f, 0.f, 0.f);
                }
                wi = bs.wi;
                w = bs.w;
                ok = bs.valid;
            } else {
                const ResidRow* rr = rows + (uint64_t)pix * a.M + (r - a.N);
                const float4 d = __ldg(&rr->wi), ww = __ldg(&rr->w);
                wi = V3{d.x, d.y, d.z};
                w = make_float3(ww.x, ww.y, ww.z);
                ok = valid && d.w != 0.f;
            }
            float3 nv = make_float3(0.f, 0.f, 0.f);
            if (network) {
                if (__any_sync(0xffffffffu, ok)) nv = row_mlp<kSh>(a.s, sw, act, stride, hpix, wi, a.z_clamp);
            } else if (a.cache_mode == 2) {
                nv = make_float3(a.cc0, a.cc1, a.cc2);
            }
            if (a.env_hd && ok) {  // visibility cache: n = V L_env(w)
                const float3 le = env_radiance(env, wi);
                nv = make_float3(nv.x * le.x, nv.y * le.y, nv.z * le.z);
            }
            if (row_n && in_range) {
                float* rn = row_n + 3 * ((uint64_t)pix * S + r);
                rn[0] = ok ? nv.x : 0.f;
                rn[1] = ok ? nv.y : 0.f;
                rn[2] = ok ? nv.z : 0.f;
            }
            if (!ok) continue;
            const float3 t = make_float3(w.x * nv.x, w.y * nv.y, w.z * nv.z);
            if (r < a.N) {
                lc.add(t);
                ++nvalid;
            } else {
                sub.add(t);
            }
        }
        if (!in_range) continue;
        PixelBase b;
        if (base) {
            b = base[pix];
        } else {
            b.le = b.wl = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float3 Lc = make_float3(0.f, 0.f, 0.f), Lr = make_float3(b.wl.x, b.wl.y, b.wl.z);
        if (a.N) {
            const float inv = 1.0f / (float)a.N;
            Lc = make_float3(lc.s.x * inv, lc.s.y * inv, lc.s.z * inv);
        }
        if (a.M && a.N) {  // without a cache level nothing is subtracted
            const float inv = 1.0f / (float)a.M;
            Lr.x -= sub.s.x * inv;
            Lr.y -= sub.s.y * inv;
            Lr.z -= sub.s.z * inv;
        }
        if (beta) {  // the unit's throughput (biased stopping vertex, later vertex of a residual path)
            const float4 bt = beta[pix];
            Lc = make_float3(Lc.x * bt.x, Lc.y * bt.y, Lc.z * bt.z);
            Lr = make_float3(Lr.x * bt.x, Lr.y * bt.y, Lr.z * bt.z);
        }
        out[pix] = make_float4(b.le.x + Lc.x + Lr.x, b.le.y + Lc.y + Lr.y, b.le.z + Lc.z + Lr.z, 1.f);
        if (lc_out) {
            lc_out[3 * (uint64_t)pix] = Lc.x;
            lc_out[3 * (uint64_t)pix + 1] = Lc.y;
            lc_out[3 * (uint64_t)pix + 2] = Lc.z;
        }
        if (lr_out) {
            lr_out[3 * (uint64_t)pix] = Lr.x;
            lr_out[3 * (uint64_t)pix + 1] = Lr.y;
            lr_out[3 * (uint64_t)pix + 2] = Lr.z;
        }
        if (sig_out) sig_out[2 * (uint64_t)pix + 1] = sig;
        if (count) count[pix] += nvalid;
    }
}

template <bool kSh>
__global__ void __launch_bounds__(kSimtThreads, 1)
    k_query_simt(NetShape s, GridParams g, float z_clamp, const float* __restrict__ packed,
                 const float* __restrict__ table, const nirc_record* __restrict__ recs, const float* __restrict__ dirs,
                 uint64_t n_rows, float* __restrict__ out) {
    extern __shared__ __align__(16) float smem[];
    float* sw = smem;
    float* act = smem + s.packed_floats + threadIdx.x;
    const int stride = kSimtThreads;
    stage_weights(sw, packed, s.packed_floats);
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * kSimtThreads + threadIdx.x; i < n_rows;
         i += (uint64_t)gridDim.x * kSimtThreads) {
        const float4* rq = reinterpret_cast<const float4*>(recs + i);
        const float4 r0 = __ldg(rq), r1 = __ldg(rq + 1), r2 = __ldg(rq + 2), r3 = __ldg(rq + 3);
        const V3 p{r0.x, r0.y, r0.z}, n{r0.w, r1.x, r1.y};
        const V3 wi{__ldg(dirs + 3 * i), __ldg(dirs + 3 * i + 1), __ldg(dirs + 3 * i + 2)};
        encode_surface(s, g, table, p, n, make_float3(r2.y, r2.z, r2.w), r3.x, act, stride);
        float2 hpix[32];
        surface_product(s, sw, act, stride, hpix);
        const float3 nv = row_mlp<kSh>(s, sw, act, stride, hpix, wi, z_clamp);
        out[3 * i] = nv.x;
        out[3 * i + 1] = nv.y;
        out[3 * i + 2] = nv.z;
    }
}

// Transpose the FP32 master weights into the SIMT shared-memory image.
__global__ void k_repack_simt(NetShape s, const float* __restrict__ params, float* __restrict__ packed) {
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= s.packed_floats) return;
    const uint32_t n_in = s.n_in;
    float v = 0.f;
    if (idx < s.off_wdir) {
        const uint32_t k = idx / kWidth, o = idx % kWidth;
        const uint32_t col = k < s.n_pos ? k : k + s.n_dir;
        v = params[o * n_in + col];
    } else if (idx < s.off_b0) {
        const uint32_t k = (idx - s.off_wdir) / kWidth, o = (idx - s.off_wdir) % kWidth;
        v = params[o * n_in + s.n_pos + k];
    } else if (idx < s.off_hidden) {
        v = params[kWidth * n_in + (idx - s.off_b0)];
    } else if (idx < s.off_out) {
        const uint32_t l = (idx - s.off_hidden) / (kWidth * kWidth + kWidth);
        const uint32_t r = (idx - s.off_hidden) % (kWidth * kWidth + kWidth);
        const uint64_t base = (uint64_t)kWidth * n_in + kWidth + (uint64_t)l * (kWidth * kWidth + kWidth);
        if (r < kWidth * kWidth) {
            const uint32_t i = r / kWidth, o = r % kWidth;
            v = params[base + o * kWidth + i];
        } else {
            v = params[base + r];
        }
    } else {
        const uint32_t r = idx - s.off_out;
        const uint64_t base = (uint64_t)kWidth * n_in + kWidth + (uint64_t)(s.hidden - 1) * (kWidth * kWidth + kWidth);
        if (r < 4 * kWidth) {
            const uint32_t i = r / 4, c = r % 4;
            v = c < 3 ? params[base + c * kWidth + i] : 0.f;
        } else {
            const uint32_t c = r - 4 * kWidth;
            v = c < 3 ? params[base + 3 * kWidth + c] : 0.f;
        }
    }
    packed[idx] = v;
}

static size_t simt_smem(const NetShape& s) {
    return (size_t)s.packed_floats * 4 + (size_t)kSimtThreads * kWidth * 4;
}

cudaError_t launch_cache_simt(const nirc_handle* h, const nirc_frame_desc& fd, const nirc_record* recs,
                              const PixelBase* base, const ResidRow* rows, const float4* beta, float* out_rgba,
                              float* lc, float* lr, uint64_t* sig, uint32_t* count, float* row_n, cudaStream_t st,
                              CachePass pass, EnvSource env) {
    CacheArgs a;
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
    a.cache_mode = fd.cache_mode;
    a.cc0 = fd.cache_const[0];
    a.cc1 = fd.cache_const[1];
    a.cc2 = fd.cache_const[2];
    a.z_clamp = h->cfg.z_clamp;
    a.s = h->shape;
    a.g = h->grid;
    const size_t smem = simt_smem(h->shape);
    auto kern = h->shape.sh ? k_cache_simt<true> : k_cache_simt<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint64_t P = (uint64_t)fd.width * fd.height;
    uint64_t blocks = (P + kSimtThreads - 1) / kSimtThreads;
    if (blocks > 2ull * h->num_sms) blocks = 2ull * h->num_sms;
    const float* table = h->params + h->shape.hash_off;
    kern<<<(uint32_t)blocks, kSimtThreads, smem, st>>>(a, h->packed, table, recs, base, rows, beta,
                                                       reinterpret_cast<float4*>(out_rgba), lc, lr, sig, count, row_n);
    count_kernels(h);
    return cudaGetLastError();
}

cudaError_t launch_query_simt(const nirc_handle* h, const nirc_record* recs, const float* dirs, uint64_t n, float* out,
                              cudaStream_t st) {
    const size_t smem = simt_smem(h->shape);
    auto kern = h->shape.sh ? k_query_simt<true> : k_query_simt<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    uint64_t blocks = (n + kSimtThreads - 1) / kSimtThreads;
    if (blocks > 2ull * h->num_sms) blocks = 2ull * h->num_sms;
    const float* table = h->params + h->shape.hash_off;
    kern<<<(uint32_t)blocks, kSimtThreads, smem, st>>>(h->shape, h->grid, h->cfg.z_clamp, h->packed, table, recs, dirs,
                                                       n, out);
    count_kernels(h);
    return cudaGetLastError();
}

cudaError_t launch_repack_simt(const nirc_handle* h, cudaStream_t st) {
    const uint32_t n = h->shape.packed_floats;
    k_repack_simt<<<(n + 255) / 256, 256, 0, st>>>(h->shape, h->params, h->packed);
    count_kernels(h);
    return cudaGetLastError();
}

}  // namespace nirc
