// nirc_device.cuh -- device building blocks of the NIRC hot path (sm_103a).
//
// Counter-based sampling (Philox4x32-10), strict-IEEE binary32 geometry,
// BSDF importance sampling and the network input encodings.  Everything that
// decides an integer (hits, hit points, sampled directions, disk-rejection
// and Russian-roulette tests, hash-grid cells) uses explicitly rounded
// binary32 intrinsics (__fadd_rn, __fmul_rn, ...), which the compiler never
// contracts into FMAs, in a fixed operation order: the decisions are then
// the same on any IEEE-754 implementation that performs the same operations.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>

#include "nirc.h"

namespace nirc {

// ---------------------------------------------------------------------------
// Binary layouts of the inputs (see nirc.h)
// ---------------------------------------------------------------------------

struct __align__(16) Prim {
    float a[3];
    float radius;
    float u[3];
    float inv_uu;
    float v[3];
    float inv_vv;
    float n[3];
    uint32_t kind;
    float albedo[3];
    float roughness;
    float emission[3];
    uint32_t flags;
};
static_assert(sizeof(Prim) == 96, "primitive layout");

struct __align__(16) SceneHeader {
    uint32_t n_prims;
    uint32_t pad[3];
    float origin[4];
    float top_left[4];
    float horizontal[4];
    float vertical[4];
    uint32_t reserved[4];
};
static_assert(sizeof(SceneHeader) == 96, "scene header layout");
static_assert(sizeof(nirc_record) == 64, "record layout");

// Geometry part of a primitive (first 64 bytes) staged in shared memory.
struct __align__(16) PrimGeom {
    float4 a_r;        // a.xyz, radius
    float4 u_iuu;      // u.xyz, 1/(u.u)
    float4 v_ivv;      // v.xyz, 1/(v.v)
    float4 n_kind;     // n.xyz, kind (bit pattern)
};

enum : uint32_t { MAT_LAMBERT = 0, MAT_GGX = 1, MAT_BLACK = 2 };
enum : uint32_t { KIND_SPHERE = 0, KIND_RECT = 1 };
enum : uint32_t { EMIT_TWO_SIDED = 1u << 8 };

// Philox counter word 3 (purpose of a draw); counter = (pixel or training
// path, sample, call, purpose), key = (seed, frame) or (seed, frame ^ 2^31)
// for the training pass.
enum : uint32_t {
    PURPOSE_CAMERA = 1,
    PURPOSE_CACHE_DIR = 2,
    PURPOSE_RESID_DIR = 3,
    PURPOSE_BOUNCE = 4,  // + 16 * segment
    PURPOSE_RR = 5,      // + 16 * segment
    PURPOSE_TRAIN_PICK = 6,
    PURPOSE_LIGHT = 7,   // + 16 * segment (0: the shading point), light mode 1
    PURPOSE_BTH_DIR = 8, // + 16 * vertex: biased estimator, direction sampled at a camera-path vertex
    PURPOSE_BTH_XI = 9,  // + 16 * vertex: biased estimator, the termination test's uniform
    PURPOSE_VCACHE = 10  // + 16 * vertex (2, 3): multi-vertex estimator, cache samples along a residual path
};

constexpr float kTMin = 1e-4f;
constexpr float kRRContinue = 0.9f;  // Russian roulette terminates with probability 0.1
constexpr float kF0 = 0.04f;
constexpr float kPi = 3.14159265358979f;
constexpr float kInvPi = 0.318309886183791f;
constexpr uint32_t kTrainKeyBit = 0x80000000u;
constexpr uint64_t kSigInit = 0xCBF29CE484222325ull;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------

struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                                     uint32_t c3) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// High 24 bits -> [0, 1), exact.
__device__ __forceinline__ float u01(uint32_t x) {
    return __fmul_rn(__uint2float_rn(x >> 8), 1.0f / 16777216.0f);
}

__device__ __forceinline__ uint64_t sig_mix(uint64_t h, uint32_t w) {
    return (h ^ (uint64_t)w) * 0x100000001B3ull;
}

// ---------------------------------------------------------------------------
// Strict binary32 vector helpers
// ---------------------------------------------------------------------------

struct V3 {
    float x, y, z;
};

__device__ __forceinline__ float sdot(V3 a, V3 b) {
    return __fadd_rn(__fadd_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)), __fmul_rn(a.z, b.z));
}
__device__ __forceinline__ V3 ssub(V3 a, V3 b) {
    return V3{__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z)};
}
__device__ __forceinline__ V3 sneg(V3 a) { return V3{-a.x, -a.y, -a.z}; }
// o + t d
__device__ __forceinline__ V3 smadd(V3 o, float t, V3 d) {
    return V3{__fadd_rn(o.x, __fmul_rn(t, d.x)), __fadd_rn(o.y, __fmul_rn(t, d.y)),
              __fadd_rn(o.z, __fmul_rn(t, d.z))};
}
__device__ __forceinline__ V3 snormalize(V3 v) {
    const float len = __fsqrt_rn(sdot(v, v));
    const float inv = __fdiv_rn(1.0f, len);
    return V3{__fmul_rn(v.x, inv), __fmul_rn(v.y, inv), __fmul_rn(v.z, inv)};
}
// lx t + ly b + lz n, summed left to right per component
__device__ __forceinline__ V3 sframe(float lx, float ly, float lz, V3 t, V3 b, V3 n) {
    return V3{__fadd_rn(__fadd_rn(__fmul_rn(lx, t.x), __fmul_rn(ly, b.x)), __fmul_rn(lz, n.x)),
              __fadd_rn(__fadd_rn(__fmul_rn(lx, t.y), __fmul_rn(ly, b.y)), __fmul_rn(lz, n.y)),
              __fadd_rn(__fadd_rn(__fmul_rn(lx, t.z), __fmul_rn(ly, b.z)), __fmul_rn(lz, n.z))};
}

// ---------------------------------------------------------------------------
// Ray / primitive intersection, nearest hit over shared-memory primitives
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool hit_sphere(const PrimGeom& g, V3 o, V3 d, float& t_out) {
    const V3 oc = ssub(o, V3{g.a_r.x, g.a_r.y, g.a_r.z});
    const float b = sdot(oc, d);
    const float c = __fsub_rn(sdot(oc, oc), __fmul_rn(g.a_r.w, g.a_r.w));
    const float disc = __fsub_rn(__fmul_rn(b, b), c);
    if (!(disc >= 0.0f)) return false;
    const float sq = __fsqrt_rn(disc);
    const float t0 = __fsub_rn(-b, sq);
    const float t1 = __fadd_rn(-b, sq);
    if (t0 > kTMin) {
        t_out = t0;
        return true;
    }
    if (t1 > kTMin) {
        t_out = t1;
        return true;
    }
    return false;
}

__device__ __forceinline__ bool hit_rect(const PrimGeom& g, V3 o, V3 d, float& t_out) {
    const V3 n{g.n_kind.x, g.n_kind.y, g.n_kind.z};
    const float denom = sdot(n, d);
    if (denom == 0.0f) return false;
    const V3 a{g.a_r.x, g.a_r.y, g.a_r.z};
    const float t = __fdiv_rn(sdot(n, ssub(a, o)), denom);
    if (!(t > kTMin)) return false;
    const V3 rel = ssub(smadd(o, t, d), a);
    const float al = __fmul_rn(sdot(rel, V3{g.u_iuu.x, g.u_iuu.y, g.u_iuu.z}), g.u_iuu.w);
    const float be = __fmul_rn(sdot(rel, V3{g.v_ivv.x, g.v_ivv.y, g.v_ivv.z}), g.v_ivv.w);
    if (!(al >= 0.0f && al <= 1.0f && be >= 0.0f && be <= 1.0f)) return false;
    t_out = t;
    return true;
}

// Nearest hit with t > kTMin; ties resolve to the lowest index.
__device__ __forceinline__ int trace_nearest(const PrimGeom* __restrict__ prims, uint32_t n_prims, V3 o, V3 d,
                                             float& t_hit) {
    float best = __int_as_float(0x7f800000);  // +inf
    int idx = -1;
    for (uint32_t i = 0; i < n_prims; ++i) {
        const PrimGeom& g = prims[i];
        float t;
        const bool hit = (__float_as_uint(g.n_kind.w) == KIND_SPHERE) ? hit_sphere(g, o, d, t) : hit_rect(g, o, d, t);
        if (hit && t < best) {
            best = t;
            idx = (int)i;
        }
    }
    t_hit = best;
    return idx;
}

struct Hit {
    V3 p;
    V3 n;       // unit, facing the incoming ray
    bool front; // arrived on the side the stored normal points to
};

__device__ __forceinline__ Hit hit_info(const PrimGeom& g, V3 o, V3 d, float t) {
    Hit h;
    h.p = smadd(o, t, d);
    V3 n;
    if (__float_as_uint(g.n_kind.w) == KIND_SPHERE) {
        n = snormalize(ssub(h.p, V3{g.a_r.x, g.a_r.y, g.a_r.z}));
    } else {
        n = V3{g.n_kind.x, g.n_kind.y, g.n_kind.z};
    }
    const float dn = sdot(n, d);
    h.front = dn < 0.0f;
    if (dn > 0.0f) n = sneg(n);
    h.n = n;
    return h;
}

// Camera ray through pixel (px, py) with jitter (jx, jy).
__device__ __forceinline__ void camera_ray(const SceneHeader& hd, uint32_t W, uint32_t H, uint32_t px, uint32_t py,
                                           float jx, float jy, V3& o, V3& d) {
    const float s = __fdiv_rn(__fadd_rn(__uint2float_rn(px), jx), __uint2float_rn(W));
    const float t = __fdiv_rn(__fadd_rn(__uint2float_rn(py), jy), __uint2float_rn(H));
    o = V3{hd.origin[0], hd.origin[1], hd.origin[2]};
    V3 dd;
    dd.x = __fsub_rn(__fadd_rn(__fadd_rn(hd.top_left[0], __fmul_rn(s, hd.horizontal[0])), __fmul_rn(t, hd.vertical[0])),
                     hd.origin[0]);
    dd.y = __fsub_rn(__fadd_rn(__fadd_rn(hd.top_left[1], __fmul_rn(s, hd.horizontal[1])), __fmul_rn(t, hd.vertical[1])),
                     hd.origin[1]);
    dd.z = __fsub_rn(__fadd_rn(__fadd_rn(hd.top_left[2], __fmul_rn(s, hd.horizontal[2])), __fmul_rn(t, hd.vertical[2])),
                     hd.origin[2]);
    d = snormalize(dd);
}

// Load the geometry of n primitives into shared memory (whole block).
__device__ __forceinline__ void stage_prims(PrimGeom* s_prims, const Prim* __restrict__ g_prims, uint32_t n) {
    const float4* src = reinterpret_cast<const float4*>(g_prims);
    float4* dst = reinterpret_cast<float4*>(s_prims);
    for (uint32_t i = threadIdx.x; i < 4 * n; i += blockDim.x) {
        const uint32_t p = i >> 2, q = i & 3;
        dst[i] = __ldg(src + p * 6 + q);  // the first 4 of each primitive's 6 float4
    }
}

// ---------------------------------------------------------------------------
// BSDF importance sampling (independent sets for L_c and L_r)
// ---------------------------------------------------------------------------

// Orthonormal basis around unit n (Duff et al., JCGT 2017).
__device__ __forceinline__ void onb(V3 n, V3& t, V3& b) {
    const float sign = copysignf(1.0f, n.z);
    const float a = __fdiv_rn(-1.0f, __fadd_rn(sign, n.z));
    const float bb = __fmul_rn(__fmul_rn(n.x, n.y), a);
    t = V3{__fadd_rn(1.0f, __fmul_rn(__fmul_rn(__fmul_rn(sign, n.x), n.x), a)), __fmul_rn(sign, bb),
           __fmul_rn(-sign, n.x)};
    b = V3{bb, __fadd_rn(sign, __fmul_rn(__fmul_rn(n.y, n.y), a)), -n.y};
}

// Uniform point on the unit disk: rejection from the square, 2 candidates per
// Philox call (counter word 2 = call 0..7; `first` is call 0, already drawn).
// Returns the rejected count.
__device__ __forceinline__ uint32_t disk_sample(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c3,
                                                const U4& first, float& a, float& b) {
    uint32_t rejected = 0;
    for (uint32_t call = 0; call < 8; ++call) {
        const U4 r = call == 0 ? first : philox(k0, k1, c0, c1, call, c3);
        float x = __fsub_rn(__fmul_rn(2.0f, u01(r.x)), 1.0f);
        float y = __fsub_rn(__fmul_rn(2.0f, u01(r.y)), 1.0f);
        if (__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)) < 1.0f) {
            a = x;
            b = y;
            return rejected;
        }
        ++rejected;
        x = __fsub_rn(__fmul_rn(2.0f, u01(r.z)), 1.0f);
        y = __fsub_rn(__fmul_rn(2.0f, u01(r.w)), 1.0f);
        if (__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)) < 1.0f) {
            a = x;
            b = y;
            return rejected;
        }
        ++rejected;
    }
    a = 0.0f;
    b = 0.0f;
    return rejected;
}

// GGX visible-normal sampling (Heitz, JCGT 2018) with disk point (t1, t2);
// returns the mirror direction about the sampled normal.
__device__ __forceinline__ V3 ggx_vndf_reflect(V3 wo, V3 t, V3 b, V3 n, float alpha, float t1, float t2) {
    const V3 wl{sdot(wo, t), sdot(wo, b), sdot(wo, n)};
    const V3 vh = snormalize(V3{__fmul_rn(alpha, wl.x), __fmul_rn(alpha, wl.y), wl.z});
    const float lensq = __fadd_rn(__fmul_rn(vh.x, vh.x), __fmul_rn(vh.y, vh.y));
    V3 T1;
    if (lensq > 0.0f) {
        const float il = __fdiv_rn(1.0f, __fsqrt_rn(lensq));
        T1 = V3{__fmul_rn(-vh.y, il), __fmul_rn(vh.x, il), 0.0f};
    } else {
        T1 = V3{1.0f, 0.0f, 0.0f};
    }
    const V3 T2{__fsub_rn(__fmul_rn(vh.y, T1.z), __fmul_rn(vh.z, T1.y)),
                __fsub_rn(__fmul_rn(vh.z, T1.x), __fmul_rn(vh.x, T1.z)),
                __fsub_rn(__fmul_rn(vh.x, T1.y), __fmul_rn(vh.y, T1.x))};
    const float s = __fmul_rn(0.5f, __fadd_rn(1.0f, vh.z));
    const float t2w = __fadd_rn(__fmul_rn(__fsub_rn(1.0f, s), __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(t1, t1)))),
                                __fmul_rn(s, t2));
    const float nz = __fsqrt_rn(fmaxf(0.0f, __fsub_rn(__fsub_rn(1.0f, __fmul_rn(t1, t1)), __fmul_rn(t2w, t2w))));
    const V3 nh{__fadd_rn(__fadd_rn(__fmul_rn(t1, T1.x), __fmul_rn(t2w, T2.x)), __fmul_rn(nz, vh.x)),
                __fadd_rn(__fadd_rn(__fmul_rn(t1, T1.y), __fmul_rn(t2w, T2.y)), __fmul_rn(nz, vh.y)),
                __fadd_rn(__fadd_rn(__fmul_rn(t1, T1.z), __fmul_rn(t2w, T2.z)), __fmul_rn(nz, vh.z))};
    const V3 ne = snormalize(V3{__fmul_rn(alpha, nh.x), __fmul_rn(alpha, nh.y), fmaxf(0.0f, nh.z)});
    const V3 h = sframe(ne.x, ne.y, ne.z, t, b, n);
    const float two_dh = __fmul_rn(2.0f, sdot(wo, h));
    const V3 wi{__fsub_rn(__fmul_rn(two_dh, h.x), wo.x), __fsub_rn(__fmul_rn(two_dh, h.y), wo.y),
                __fsub_rn(__fmul_rn(two_dh, h.z), wo.z)};
    return snormalize(wi);
}

// f_r cos / p of the Lambertian + GGX material under the 1/2 cosine + 1/2
// visible-normal mixture (FP32, continuous).
// sqrt(x) for x >= 0 from the hardware reciprocal square root (a few ulp;
// for continuous quantities only, never for a decision).
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

// a d - b c with one rounding error (Kahan's FMA algorithm).
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
    const float w = b * c;
    const float e = __fmaf_rn(-b, c, w);
    const float f = __fmaf_rn(a, d, -w);
    return f + e;
}

// GGX denominator dd = sin^2 + a2 cos^2 of the angle between n and the
// (unnormalised) half vector s = wo + wi, from the cross and dot products
// normalised by the lengths: no cancellation near the specular peak, where
// 1 - cos^2 (1 - a2) in FP32 loses all accuracy at small roughness.
__device__ __forceinline__ float ggx_dd(V3 n, float sx, float sy, float sz, float a2) {
    const float cx = det2(n.y, n.z, sy, sz), cy = det2(n.z, n.x, sz, sx), cz = det2(n.x, n.y, sx, sy);
    const float ns = n.x * sx + n.y * sy + n.z * sz;
    const float norm = (n.x * n.x + n.y * n.y + n.z * n.z) * (sx * sx + sy * sy + sz * sz);
    return __fdividef(cx * cx + cy * cy + cz * cz + a2 * ns * ns, norm);
}

__device__ __forceinline__ float3 ggx_mix_weight(V3 n, V3 wo, V3 wi, float3 albedo, float rough) {
    const float alpha = __fmul_rn(rough, rough);
    const float a2 = alpha * alpha;
    const float ci = n.x * wi.x + n.y * wi.y + n.z * wi.z;
    const float co = n.x * wo.x + n.y * wo.y + n.z * wo.z;
    const float sx = wo.x + wi.x, sy = wo.y + wi.y, sz = wo.z + wi.z;
    const float hinv = rsqrtf(sx * sx + sy * sy + sz * sz);
    const float oh = fminf(fmaxf((wo.x * sx + wo.y * sy + wo.z * sz) * hinv, 0.0f), 1.0f);
    const float dd = ggx_dd(n, sx, sy, sz, a2);
    const float D = __fdividef(a2, kPi * dd * dd);
    const float lam_o = fast_sqrt(a2 + (1.0f - a2) * co * co);
    const float lam_i = fast_sqrt(a2 + (1.0f - a2) * ci * ci);
    const float m = 1.0f - oh;
    const float m2 = m * m;
    const float F = kF0 + (1.0f - kF0) * (m2 * m2 * m);
    // F D G2 / (4 ci co) with G2 = 2 ci co / (co lam_i + ci lam_o), and the
    // visible-normal pdf G1(wo) D / (4 co) with G1 = 2 co / (co + lam_o)
    const float fs = __fdividef(F * D, 2.0f * (co * lam_i + ci * lam_o));
    const float pdf_s = __fdividef(D, 2.0f * (co + lam_o));
    const float pdf = 0.5f * ci * kInvPi + 0.5f * pdf_s;
    const float k = __fdividef(ci, pdf);
    return make_float3((albedo.x * kInvPi + fs) * k, (albedo.y * kInvPi + fs) * k, (albedo.z * kInvPi + fs) * k);
}

// a . b as if accumulated in twice the precision, then rounded (compensated
// dot product of Ogita, Rump and Oishi 2005: error-free products by FMA,
// error-free sums by TwoSum).  Used for cosines that cancel (grazing light
// samples), where a plain FP32 dot loses most of its relative accuracy.
__device__ __forceinline__ float dot_acc(V3 a, V3 b) {
    float s = __fmul_rn(a.x, b.x);
    float c = __fmaf_rn(a.x, b.x, -s);
    const float qa[2] = {a.y, a.z}, qb[2] = {b.y, b.z};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float p = __fmul_rn(qa[k], qb[k]);
        const float pe = __fmaf_rn(qa[k], qb[k], -p);
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
        s = t;
        c = __fadd_rn(c, __fadd_rn(pe, se));
    }
    return __fadd_rn(s, c);
}

// f_r cos(theta_i) and the sampling density p(wi) (solid angle) of the
// material for an arbitrary direction (next-event estimation and MIS); both
// 0 below the surface.  Same formulas as ggx_mix_weight, which is their
// ratio for sampled directions; the cosines by the compensated dot.
struct BsdfEval {
    float3 fcos;
    float pdf;
};

__device__ __forceinline__ BsdfEval bsdf_eval(V3 n, V3 wo, V3 wi, float3 albedo, float rough, uint32_t mat) {
    BsdfEval r;
    r.fcos = make_float3(0.f, 0.f, 0.f);
    r.pdf = 0.f;
    const float ci = dot_acc(n, wi);
    if (mat == MAT_BLACK || !(ci > 0.f)) return r;
    if (mat == MAT_LAMBERT) {
        const float k = ci * kInvPi;
        r.fcos = make_float3(albedo.x * k, albedo.y * k, albedo.z * k);
        r.pdf = k;
        return r;
    }
    const float alpha = __fmul_rn(rough, rough);
    const float a2 = alpha * alpha;
    const float co = dot_acc(n, wo);
    const float sx = wo.x + wi.x, sy = wo.y + wi.y, sz = wo.z + wi.z;
    const float hinv = rsqrtf(sx * sx + sy * sy + sz * sz);
    const float oh = fminf(fmaxf((wo.x * sx + wo.y * sy + wo.z * sz) * hinv, 0.0f), 1.0f);
    const float dd = ggx_dd(n, sx, sy, sz, a2);
    const float D = __fdividef(a2, kPi * dd * dd);
    const float lam_o = fast_sqrt(a2 + (1.0f - a2) * co * co);
    const float lam_i = fast_sqrt(a2 + (1.0f - a2) * ci * ci);
    const float m = 1.0f - oh;
    const float m2 = m * m;
    const float F = kF0 + (1.0f - kF0) * (m2 * m2 * m);
    const float fs = __fdividef(F * D, 2.0f * (co * lam_i + ci * lam_o));
    r.fcos = make_float3((albedo.x * kInvPi + fs) * ci, (albedo.y * kInvPi + fs) * ci, (albedo.z * kInvPi + fs) * ci);
    r.pdf = 0.5f * ci * kInvPi + 0.5f * __fdividef(D, 2.0f * (co + lam_o));
    return r;
}

struct BsdfSample {
    V3 wi;
    float3 w;        // f_r cos / p, zero when invalid
    bool valid;
    uint32_t word;   // rejected | lobe << 8 | valid << 9 (signature word)
};

// Sample at a shading record (p unused); Philox counter (c0, c1, call, c3).
// The mixture lobe (GGX materials) is the low byte of word 0 of call 0 (< 128:
// cosine lobe), bits the disk candidates, which use the high 24 bits, leave free.
__device__ __forceinline__ BsdfSample sample_bsdf(V3 n, V3 wo, float3 albedo, float rough, uint32_t mat, uint32_t k0,
                                                  uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c3) {
    BsdfSample s;
    s.valid = false;
    s.w = make_float3(0.f, 0.f, 0.f);
    s.wi = n;
    s.word = 0;
    if (mat == MAT_BLACK) return s;
    V3 t, b;
    onb(n, t, b);
    const U4 first = philox(k0, k1, c0, c1, 0u, c3);
    const uint32_t lobe = (mat == MAT_GGX && (first.x & 0xFFu) >= 128u) ? 1u : 0u;
    float da, db;
    const uint32_t rejected = disk_sample(k0, k1, c0, c1, c3, first, da, db);
    if (lobe == 0) {
        const float sq = __fadd_rn(__fmul_rn(da, da), __fmul_rn(db, db));
        const float z = __fsqrt_rn(fmaxf(0.0f, __fsub_rn(1.0f, sq)));
        s.wi = snormalize(sframe(da, db, z, t, b, n));
    } else {
        s.wi = ggx_vndf_reflect(wo, t, b, n, __fmul_rn(rough, rough), da, db);
    }
    s.valid = sdot(s.wi, n) > 0.0f;
    s.word = rejected | (lobe << 8) | ((uint32_t)s.valid << 9);
    if (!s.valid) return s;
    if (mat == MAT_LAMBERT) {
        s.w = albedo;  // (rho/pi) cos / (cos/pi)
    } else {
        s.w = ggx_mix_weight(n, wo, s.wi, albedo, rough);
    }
    return s;
}

__device__ __forceinline__ uint32_t record_material(const nirc_record& r) { return (r.flags >> 1) & 3u; }

// ---------------------------------------------------------------------------
// Encodings
// ---------------------------------------------------------------------------

// sin(2^k pi v), cos(2^k pi v) for k = 0..3 (octave 0 by sincospi, higher
// octaves by the double-angle identities).
__device__ __forceinline__ void freq4(float v, float* e) {
    float s, c;
    sincospif(v, &s, &c);
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

// Same features with one sincospi per octave (argument scaled exactly by
// 2^k): the FP32 reference-accuracy variant used by the SIMT kernels.
__device__ __forceinline__ void freq4_accurate(float v, float* e) {
#pragma unroll
    for (int k = 0; k < 4; ++k) sincospif(ldexpf(v, k), &e[2 * k], &e[2 * k + 1]);
}

// (theta/pi, phi/2pi in [0,1)) of a unit direction.
__device__ __forceinline__ void dir_angles(V3 w, float& th, float& ph) {
    th = acosf(fminf(fmaxf(w.z, -1.0f), 1.0f)) * kInvPi;
    float p = atan2f(w.y, w.x) * (0.5f * kInvPi);
    if (p < 0.0f) p += 1.0f;
    ph = p;
}

// Real spherical harmonics Y_l^m, l = 0..4, of the unit vector w, at index
// l*l + l + m (the paper's direction input, 25 values).  With D_lm the m-th
// derivative of the Legendre polynomial P_l and c_m + i s_m = (x + i y)^m
// (= sin^m t e^{i m p} on the unit sphere):
//   Y_l^0 = A_l0 D_l0(z),  Y_l^m = A_lm D_lm(z) c_m,  Y_l^-m = A_lm D_lm(z) s_m,
// A_l0 = K_l^0, A_lm = sqrt(2) K_l^m, K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
// (orthonormal, no Condon-Shortley phase).
__device__ __forceinline__ void sh_basis25(V3 w, float* e) {
    constexpr float A00 = 0.28209479177387814f, A10 = 0.4886025119029199f, A11 = 0.48860251190292f;
    constexpr float A20 = 0.6307831305050401f, A21 = 0.36418281019735976f, A22 = 0.18209140509867988f;
    constexpr float A30 = 0.7463526651802308f, A31 = 0.3046971996429772f, A32 = 0.09635371475468515f,
                    A33 = 0.03933623932844291f;
    constexpr float A40 = 0.8462843753216345f, A41 = 0.2676186174229157f, A42 = 0.063078313050504f,
                    A43 = 0.016858388283618388f, A44 = 0.005960340337611203f;
    const float x = w.x, y = w.y, z = w.z, z2 = z * z;
    const float c2 = x * x - y * y, s2 = 2.f * x * y;
    const float c3 = x * c2 - y * s2, s3 = x * s2 + y * c2;
    const float c4 = x * c3 - y * s3, s4 = x * s3 + y * c3;
    // A_lm D_lm(z): P_2 = (3z^2 - 1)/2, P_3 = (5z^3 - 3z)/2, P_4 = (35z^4 - 30z^2 + 3)/8 and derivatives
    const float b20 = A20 * (1.5f * z2 - 0.5f), b21 = A21 * 3.f * z, b22 = A22 * 3.f;
    const float b30 = A30 * z * (2.5f * z2 - 1.5f), b31 = A31 * (7.5f * z2 - 1.5f), b32 = A32 * 15.f * z,
                b33 = A33 * 15.f;
    const float b40 = A40 * ((4.375f * z2 - 3.75f) * z2 + 0.375f), b41 = A41 * z * (17.5f * z2 - 7.5f),
                b42 = A42 * (52.5f * z2 - 7.5f), b43 = A43 * 105.f * z, b44 = A44 * 105.f;
    e[0] = A00;
    e[1] = A11 * y;
    e[2] = A10 * z;
    e[3] = A11 * x;
    e[4] = b22 * s2;
    e[5] = b21 * y;
    e[6] = b20;
    e[7] = b21 * x;
    e[8] = b22 * c2;
    e[9] = b33 * s3;
    e[10] = b32 * s2;
    e[11] = b31 * y;
    e[12] = b30;
    e[13] = b31 * x;
    e[14] = b32 * c2;
    e[15] = b33 * c3;
    e[16] = b44 * s4;
    e[17] = b43 * s3;
    e[18] = b42 * s2;
    e[19] = b41 * y;
    e[20] = b40;
    e[21] = b41 * x;
    e[22] = b42 * c2;
    e[23] = b43 * c3;
    e[24] = b44 * c4;
}

// One-blob encoding of s into 4 bins (Mueller et al. 2019): the mass of a
// Gaussian of standard deviation 1/4 centred at s over [i/4, (i+1)/4),
// e_i = (erf((i+1)/4 - s) 4/sqrt 2) - erf((i/4 - s) 4/sqrt 2)) / 2, no wrap-around.
__device__ __forceinline__ void one_blob4(float s, float* e) {
    constexpr float k = 2.8284271247461903f;  // 4 / sqrt(2)
    float g[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) g[i] = erff((0.25f * (float)i - s) * k);
#pragma unroll
    for (int i = 0; i < 4; ++i) e[i] = 0.5f * (g[i + 1] - g[i]);
}

// The paper's per-surface inputs phi (15): albedo, one-blob of the normal's
// (theta/pi, phi/2pi), one-blob of the roughness.
__device__ __forceinline__ void phi_features(V3 n, float3 alb, float rough, float* e) {
    e[0] = alb.x;
    e[1] = alb.y;
    e[2] = alb.z;
    float th, ph;
    dir_angles(n, th, ph);
    one_blob4(th, e + 3);
    one_blob4(ph, e + 7);
    one_blob4(rough, e + 11);
}

// Environment map (light mode 2): a cube map of S x S texels per face after
// the scene's primitives (S = header reserved[0]; 0: none).
struct EnvMap {
    const float4* tex = nullptr;
    uint32_t S = 0;
};

// Texel of direction d: the face of the largest |component| (ties: x, then
// y, then z; face 0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z), column and row from
// the other two components over |major| mapped from [-1, 1] to [0, S),
// clamped.  Strict binary32: it picks an integer.
__device__ __forceinline__ uint32_t env_texel(uint32_t S, V3 d) {
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    uint32_t face;
    float m, a, b;
    if (ax >= ay && ax >= az) {
        face = d.x >= 0.f ? 0u : 1u;
        m = ax;
        a = d.y;
        b = d.z;
    } else if (ay >= az) {
        face = d.y >= 0.f ? 2u : 3u;
        m = ay;
        a = d.x;
        b = d.z;
    } else {
        face = d.z >= 0.f ? 4u : 5u;
        m = az;
        a = d.x;
        b = d.y;
    }
    const float u = __fmul_rn(__fadd_rn(__fdiv_rn(a, m), 1.f), 0.5f);
    const float v = __fmul_rn(__fadd_rn(__fdiv_rn(b, m), 1.f), 0.5f);
    const uint32_t i = min((uint32_t)floorf(__fmul_rn(u, (float)S)), S - 1u);
    const uint32_t j = min((uint32_t)floorf(__fmul_rn(v, (float)S)), S - 1u);
    return face * S * S + j * S + i;
}

// L_env(d): the nearest texel, 0 without a map.
__device__ __forceinline__ float3 env_radiance(const EnvMap& e, V3 d) {
    if (!e.S) return make_float3(0.f, 0.f, 0.f);
    const float4 t = __ldg(e.tex + env_texel(e.S, d));
    return make_float3(t.x, t.y, t.z);
}

// The cube map of a scene blob (NULL header: none).
__device__ __forceinline__ EnvMap env_from(const SceneHeader* hd, uint32_t n_prims) {
    EnvMap e;
    if (hd) {
        e.S = __ldg(&hd->reserved[0]);
        e.tex = reinterpret_cast<const float4*>(reinterpret_cast<const unsigned char*>(hd) + sizeof(SceneHeader) +
                                                (size_t)n_prims * 96u);
    }
    return e;
}

// Output activation of the cache network: visibility V = 1 / (1 + exp(-z))
// (sigmoid), radiance n = exp(min(z, z_clamp)).
__device__ __forceinline__ float out_act(bool vis, float z, float z_clamp) {
    return vis ? 1.0f / (1.0f + expf(-z)) : expf(fminf(z, z_clamp));
}
// The same with the hardware exponential (relative error about 2^-22 + |z| 2^-24,
// results below 2^-126 flushed to zero), for the tensor-core paths, whose
// 16-bit activations dominate their error.
__device__ __forceinline__ float out_act_fast(bool vis, float z, float z_clamp) {
    return vis ? 1.0f / (1.0f + __expf(-z)) : __expf(fminf(z, z_clamp));
}

// Hash-grid level description (precomputed on the host).
struct GridLevel {
    uint32_t res;    // floor(base * growth^l)
    uint32_t dense;  // (res + 1)^3 <= T
    float fres;
    uint32_t pad;
};

// Cell corner indices and trilinear weights of position x at one level.
__device__ __forceinline__ void grid_corners(const GridLevel& L, uint32_t mask, V3 x, uint32_t idx[8], float w[8]) {
    const float xc[3] = {fminf(fmaxf(x.x, 0.0f), 1.0f), fminf(fmaxf(x.y, 0.0f), 1.0f), fminf(fmaxf(x.z, 0.0f), 1.0f)};
    uint32_t cell[3];
    float fr[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float ps = __fmul_rn(xc[d], L.fres);
        float fl = floorf(ps);
        if (fl >= L.fres) fl = __fsub_rn(L.fres, 1.0f);
        cell[d] = (uint32_t)fl;
        fr[d] = __fsub_rn(ps, fl);
    }
    const uint32_t side = L.res + 1;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t v0 = cell[0] + (c & 1), v1 = cell[1] + ((c >> 1) & 1), v2 = cell[2] + ((c >> 2) & 1);
        idx[c] = L.dense ? v0 + v1 * side + v2 * side * side
                         : ((v0 * 1u) ^ (v1 * 2654435761u) ^ (v2 * 805459861u)) & mask;
        const float wx = (c & 1) ? fr[0] : 1.0f - fr[0];
        const float wy = ((c >> 1) & 1) ? fr[1] : 1.0f - fr[1];
        const float wz = ((c >> 2) & 1) ? fr[2] : 1.0f - fr[2];
        w[c] = wx * wy * wz;
    }
}

}  // namespace nirc
