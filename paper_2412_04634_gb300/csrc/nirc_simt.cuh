// nirc_simt.cuh -- FP32 SIMT building blocks shared by the cache and
// training kernels: packed FP32x2 FMA rows over transposed weights in
// shared memory, the per-surface encoding and compensated sums.
#pragma once

#include "nirc_internal.h"

namespace nirc {

__device__ __forceinline__ void fma_row(float2 (&acc)[32], const float* __restrict__ wrow, float a) {
    const float4* w4 = reinterpret_cast<const float4*>(wrow);
    const float2 aa = make_float2(a, a);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float4 w = w4[q];
        acc[2 * q] = __ffma2_rn(make_float2(w.x, w.y), aa, acc[2 * q]);
        acc[2 * q + 1] = __ffma2_rn(make_float2(w.z, w.w), aa, acc[2 * q + 1]);
    }
}

__device__ __forceinline__ void load_bias(float2 (&acc)[32], const float* __restrict__ b) {
    const float4* b4 = reinterpret_cast<const float4*>(b);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float4 v = b4[q];
        acc[2 * q] = make_float2(v.x, v.y);
        acc[2 * q + 1] = make_float2(v.z, v.w);
    }
}

__device__ __forceinline__ void store_relu(const float2 (&acc)[32], float* act, int stride) {
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        act[(2 * q) * stride] = fmaxf(acc[q].x, 0.f);
        act[(2 * q + 1) * stride] = fmaxf(acc[q].y, 0.f);
    }
}

// Per-surface features [position (n_pos)][normal frequency (24) or phi (15)]
// into act[k * stride].
__device__ __forceinline__ void encode_surface(const NetShape& s, const GridParams& g, const float* __restrict__ table,
                                               V3 p, V3 n, float3 alb, float rough, float* act, int stride) {
    float e[8];
    uint32_t k = 0;
    if (s.hashgrid) {
        const uint64_t T = (uint64_t)g.mask + 1;
        for (uint32_t l = 0; l < g.n_levels; ++l) {
            uint32_t idx[8];
            float w[8];
            grid_corners(g.level[l], g.mask, p, idx, w);
            const float2* tab = reinterpret_cast<const float2*>(table) + (uint64_t)l * T;
            float f0 = 0.f, f1 = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float2 v = __ldg(tab + idx[c]);
                f0 += w[c] * v.x;
                f1 += w[c] * v.y;
            }
            act[(k++) * stride] = f0;
            act[(k++) * stride] = f1;
        }
    } else {
        const float pv[3] = {p.x, p.y, p.z};
        for (int d = 0; d < 3; ++d) {
            freq4_accurate(pv[d], e);
#pragma unroll
            for (int q = 0; q < 8; ++q) act[(k++) * stride] = e[q];
        }
    }
    if (s.sh) {
        float f[kPhiFeatures];
        phi_features(n, alb, rough, f);
#pragma unroll
        for (int q = 0; q < (int)kPhiFeatures; ++q) act[(k++) * stride] = f[q];
        return;
    }
    const float nv[3] = {n.x, n.y, n.z};
    for (int d = 0; d < 3; ++d) {
        freq4_accurate(nv[d], e);
#pragma unroll
        for (int q = 0; q < 8; ++q) act[(k++) * stride] = e[q];
    }
}

// Direction features of a row: frequency features of (theta/pi, phi/2pi)
// (16) or the spherical harmonics (25).
template <bool kSh>
__device__ __forceinline__ void dir_encode(V3 wi, float* e) {
    if constexpr (kSh) {
        sh_basis25(wi, e);
    } else {
        float th, ph;
        dir_angles(wi, th, ph);
        freq4_accurate(th, e);
        freq4_accurate(ph, e + 8);
    }
}
template <bool kSh>
constexpr int dir_features() {
    return kSh ? (int)kShFeatures : (int)kDirFeatures;
}

__device__ __forceinline__ void stage_weights(float* sw, const float* __restrict__ packed, uint32_t n_floats) {
    const float4* src = reinterpret_cast<const float4*>(packed);
    float4* dst = reinterpret_cast<float4*>(sw);
    for (uint32_t i = threadIdx.x; i < n_floats / 4; i += blockDim.x) dst[i] = __ldg(src + i);
}

// Add (g0, g1) into the two features of table entry idx.  Lanes of the warp
// holding the same entry are summed first; the lowest lane of each group
// issues one 8-byte atomic.  Every lane of the warp must call this together
// (the caller's loop is warp-uniform); lanes with valid == false contribute
// nothing.
__device__ __forceinline__ void scatter_pair(float* __restrict__ gt, uint32_t idx, bool valid, float g0, float g1) {
    const uint32_t key = valid ? idx : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const unsigned groups = __reduce_max_sync(0xffffffffu, valid ? (unsigned)__popc(peers) : 1u);
    float s0 = g0, s1 = g1;
    unsigned rest = peers & ~(1u << lane);
    for (unsigned i = 1; i < groups; ++i) {
        const int src = rest ? __ffs(rest) - 1 : lane;
        rest &= rest - 1u;
        const float a0 = __shfl_sync(0xffffffffu, g0, src);
        const float a1 = __shfl_sync(0xffffffffu, g1, src);
        if (src != lane) {
            s0 += a0;
            s1 += a1;
        }
    }
    if (valid && lane == __ffs(peers) - 1)
        atomicAdd(reinterpret_cast<float2*>(gt + 2 * (uint64_t)idx), make_float2(s0, s1));
}

struct Kahan3 {
    float3 s = make_float3(0.f, 0.f, 0.f);
    float3 c = make_float3(0.f, 0.f, 0.f);
    __device__ __forceinline__ void add(float x, float& sum, float& comp) {
        const float y = x - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    __device__ __forceinline__ void add(float3 v) {
        add(v.x, s.x, c.x);
        add(v.y, s.y, c.y);
        add(v.z, s.z, c.z);
    }
};

}  // namespace nirc
