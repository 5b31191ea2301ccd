// nirc_bvh.cuh -- per-CTA bounding-volume hierarchy over the scene's
// primitives, built in shared memory and used for nearest-hit queries.
//
// Primitives whose box spans more than half of the scene (walls, floors) are
// kept in a short list tested by brute force first; they would overlap every
// node of a hierarchy.  The others get a binary radix tree: conservative
// AABBs, 30-bit Morton codes of the centroids made unique with the primitive
// index, a rank sort, the topology of Karras (HPG 2012), then boxes
// bottom-up.  Each internal node stores the boxes of its two children (64
// bytes: one visit is four 16-byte shared loads), a leaf child being one
// primitive.  A query tests the large list, then walks the tree in near-first
// order with a stack, testing a leaf child's primitive as soon as its box is
// hit and entering an internal child only when a ray could hit its box no
// later than the best hit so far (with slack).  Primitives are tested with
// the same strict binary32 routines as the brute-force loop, keeping the
// smallest (t, primitive index): boxes are expanded and pruning is
// conservative, so the result equals the brute-force nearest hit exactly.
#pragma once

#include "nirc_device.cuh"

namespace nirc {

// Internal node i of the tree is 16 floats at nodes[4 i]: the two children's
// boxes component by component, child 0 then child 1 (min x, min y, min z,
// max x, max y, max z: floats 2 c + k for component c of child k), so that
// both children's slab parameters come from packed FP32 pairs; then the
// child bits (floats 12, 13).  Child bits: bit 31 set = leaf, low bits =
// primitive; otherwise the internal node's index.
struct Bvh {
    const float4* nodes;
    const uint32_t* large;  // primitives tested by brute force
    uint32_t n_large;
    uint32_t n_tree;        // leaves of the tree
    uint32_t root;          // node index, or kLeafBit | primitive when n_tree == 1
};

constexpr uint32_t kLeafBit = 0x80000000u;
constexpr int kBvhStack = 64;  // >= tree depth (at most 62 for 64-bit unique keys)

// Shared-memory bytes the build needs for n primitives.
__host__ __device__ inline size_t bvh_smem_bytes(uint32_t n) {
    uint32_t np2 = 1;
    while (np2 < n) np2 <<= 1;
    return (size_t)(n > 1 ? n - 1 : 1) * 64 + (size_t)np2 * 8 + (size_t)n * 32 + (size_t)n * 4 * 3 + 16;
}

__device__ __forceinline__ uint32_t expand_bits10(uint32_t v) {
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

__device__ __forceinline__ int lcp_delta(const unsigned long long* keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    return __clzll(keys[i] ^ keys[j]);
}

// All threads of the CTA call it; `mem` holds bvh_smem_bytes(n) bytes, 16-byte aligned.
__device__ inline Bvh bvh_build(const PrimGeom* __restrict__ prims, uint32_t n, unsigned char* mem) {
    uint32_t np2 = 1;
    while (np2 < n) np2 <<= 1;
    float4* nodes = reinterpret_cast<float4*>(mem);
    float* nodef = reinterpret_cast<float*>(mem);  // the same, by component
    unsigned char* p = mem + (size_t)(n > 1 ? n - 1 : 1) * 64;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(p);
    p += (size_t)np2 * 8;
    float4* box = reinterpret_cast<float4*>(p);  // 2 per primitive: lo, hi
    p += (size_t)n * 32;
    uint32_t* large = reinterpret_cast<uint32_t*>(p);
    p += (size_t)n * 4;
    int* done = reinterpret_cast<int*>(p);  // internal node state
    p += (size_t)n * 4;
    uint32_t* parent = reinterpret_cast<uint32_t*>(p);  // internal node -> parent * 2 + side (root: ~0)
    p += (size_t)n * 4;
    float* scal = reinterpret_cast<float*>(p);  // [centroid min, 1/extent, n_large, n_small]
    const uint32_t tid = threadIdx.x, nt = blockDim.x;

    // 1. conservative primitive boxes
    for (uint32_t i = tid; i < n; i += nt) {
        const PrimGeom& g = prims[i];
        float3 lo, hi;
        if (__float_as_uint(g.n_kind.w) == KIND_SPHERE) {
            const float r = g.a_r.w;
            lo = make_float3(g.a_r.x - r, g.a_r.y - r, g.a_r.z - r);
            hi = make_float3(g.a_r.x + r, g.a_r.y + r, g.a_r.z + r);
        } else {
            const float ax = g.a_r.x, ay = g.a_r.y, az = g.a_r.z;
            const float ux = g.u_iuu.x, uy = g.u_iuu.y, uz = g.u_iuu.z;
            const float vx = g.v_ivv.x, vy = g.v_ivv.y, vz = g.v_ivv.z;
            lo = make_float3(fminf(fminf(ax, ax + ux), fminf(ax + vx, ax + ux + vx)),
                             fminf(fminf(ay, ay + uy), fminf(ay + vy, ay + uy + vy)),
                             fminf(fminf(az, az + uz), fminf(az + vz, az + uz + vz)));
            hi = make_float3(fmaxf(fmaxf(ax, ax + ux), fmaxf(ax + vx, ax + ux + vx)),
                             fmaxf(fmaxf(ay, ay + uy), fmaxf(ay + vy, ay + uy + vy)),
                             fmaxf(fmaxf(az, az + uz), fmaxf(az + vz, az + uz + vz)));
        }
        const float m = fmaxf(fmaxf(fmaxf(fabsf(lo.x), fabsf(lo.y)), fmaxf(fabsf(lo.z), fabsf(hi.x))),
                              fmaxf(fabsf(hi.y), fabsf(hi.z)));
        const float e = 1e-5f + 1e-5f * m;  // far above the rounding of the intersection routines
        box[2 * i] = make_float4(lo.x - e, lo.y - e, lo.z - e, 0.f);
        box[2 * i + 1] = make_float4(hi.x + e, hi.y + e, hi.z + e, 0.f);
    }
    __syncthreads();
    // 2. large / small split and centroid bounds of the small primitives (warp 0; the large
    // list in index order by ballot compaction)
    if (tid < 32) {
        float3 slo = make_float3(3e38f, 3e38f, 3e38f), shi = make_float3(-3e38f, -3e38f, -3e38f);
        for (uint32_t i = tid; i < n; i += 32) {
            const float4 l = box[2 * i], h = box[2 * i + 1];
            slo = make_float3(fminf(slo.x, l.x), fminf(slo.y, l.y), fminf(slo.z, l.z));
            shi = make_float3(fmaxf(shi.x, h.x), fmaxf(shi.y, h.y), fmaxf(shi.z, h.z));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            slo.x = fminf(slo.x, __shfl_xor_sync(0xffffffffu, slo.x, off));
            slo.y = fminf(slo.y, __shfl_xor_sync(0xffffffffu, slo.y, off));
            slo.z = fminf(slo.z, __shfl_xor_sync(0xffffffffu, slo.z, off));
            shi.x = fmaxf(shi.x, __shfl_xor_sync(0xffffffffu, shi.x, off));
            shi.y = fmaxf(shi.y, __shfl_xor_sync(0xffffffffu, shi.y, off));
            shi.z = fmaxf(shi.z, __shfl_xor_sync(0xffffffffu, shi.z, off));
        }
        const float scene = fmaxf(fmaxf(shi.x - slo.x, shi.y - slo.y), shi.z - slo.z);
        uint32_t nl = 0;
        float mn = 3e38f, mx = -3e38f;
        for (uint32_t i0 = 0; i0 < n; i0 += 32) {
            const uint32_t i = i0 + tid;
            bool lg = false;
            if (i < n) {
                const float4 l = box[2 * i], h = box[2 * i + 1];
                const float ext = fmaxf(fmaxf(h.x - l.x, h.y - l.y), h.z - l.z);
                lg = ext > 0.5f * scene;
                if (lg) {
                    box[2 * i].w = 1.f;  // marks a large primitive
                } else {
                    const float c[3] = {0.5f * (l.x + h.x), 0.5f * (l.y + h.y), 0.5f * (l.z + h.z)};
                    for (int d = 0; d < 3; ++d) {
                        mn = fminf(mn, c[d]);
                        mx = fmaxf(mx, c[d]);
                    }
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, lg);
            if (lg) large[nl + __popc(m & ((1u << tid) - 1u))] = i;
            nl += __popc(m);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        }
        if (tid == 0) {
            scal[0] = mn;
            scal[1] = mx > mn ? 1.0f / (mx - mn) : 1.0f;
            scal[2] = __uint_as_float(nl);
            scal[3] = __uint_as_float(n - nl);
        }
    }
    __syncthreads();
    const float cmin = scal[0], cinv = scal[1];
    Bvh out;
    out.nodes = nodes;
    out.large = large;
    out.n_large = __float_as_uint(scal[2]);
    out.n_tree = __float_as_uint(scal[3]);
    out.root = 0;
    for (uint32_t i = tid; i < np2; i += nt) {
        unsigned long long k = ~0ull;  // padding and large primitives sort to the end
        if (i < n && box[2 * i].w == 0.f) {
            const float4 l = box[2 * i], h = box[2 * i + 1];
            const float c[3] = {0.5f * (l.x + h.x), 0.5f * (l.y + h.y), 0.5f * (l.z + h.z)};
            uint32_t q[3];
            for (int d = 0; d < 3; ++d) {
                const float u = fminf(fmaxf((c[d] - cmin) * cinv, 0.f), 1.f);
                q[d] = min((uint32_t)(u * 1023.0f), 1023u);
            }
            const uint32_t morton = (expand_bits10(q[0]) << 2) | (expand_bits10(q[1]) << 1) | expand_bits10(q[2]);
            k = ((unsigned long long)morton << 32) | i;
        }
        keys[i] = k;
    }
    __syncthreads();
    // 3. sort: each small primitive's key goes to its rank, the number of smaller keys (the
    // primitive index in the low bits makes those keys unique; the ~0 keys of large primitives
    // and padding are never smaller and are not placed: nothing reads keys past the small
    // ones).  Four lanes count one key's rank over interleaved quarters of the keys (four
    // consecutive words per load, no bank conflict) and add their counts by shuffles; the
    // sorted keys are staged in done[] (high words) and parent[] (low words), unused until 4.
    {
        uint32_t* hiw = reinterpret_cast<uint32_t*>(done);
        const uint32_t span = (4u * n + 31u) & ~31u;  // whole warps, so every shuffle sees all lanes
        for (uint32_t u = tid; u < span; u += nt) {
            const uint32_t i = u >> 2, q = u & 3u;
            const unsigned long long ki = i < n ? keys[i] : ~0ull;
            uint32_t c = 0;
            for (uint32_t j = q; j < n; j += 4u) c += keys[j] < ki ? 1u : 0u;
            c += __shfl_xor_sync(0xffffffffu, c, 1);
            c += __shfl_xor_sync(0xffffffffu, c, 2);
            if (q == 0u && ki != ~0ull) {
                hiw[c] = (uint32_t)(ki >> 32);
                parent[c] = (uint32_t)ki;
            }
        }
        __syncthreads();
        for (uint32_t i = tid; i < out.n_tree; i += nt) keys[i] = ((unsigned long long)hiw[i] << 32) | parent[i];
        __syncthreads();
    }
    const uint32_t m = out.n_tree;
    if (m <= 1) {
        out.root = m == 1 ? (kLeafBit | (uint32_t)(keys[0] & 0x3FFu)) : 0u;
        return out;
    }
    // 4. radix-tree topology over the m small primitives (sorted keys 0..m-1)
    for (uint32_t ii = tid; ii + 1 < m; ii += nt) {
        const int i = (int)ii, nn = (int)m;
        const int d = (lcp_delta(keys, nn, i, i + 1) - lcp_delta(keys, nn, i, i - 1)) >= 0 ? 1 : -1;
        const int dmin = lcp_delta(keys, nn, i, i - d);
        int lmax = 2;
        while (lcp_delta(keys, nn, i, i + lmax * d) > dmin) lmax <<= 1;
        int l = 0;
        for (int t = lmax >> 1; t >= 1; t >>= 1)
            if (lcp_delta(keys, nn, i, i + (l + t) * d) > dmin) l += t;
        const int j = i + l * d;
        const int dnode = lcp_delta(keys, nn, i, j);
        int s = 0;
        for (int t = (l + 1) >> 1;; t = (t + 1) >> 1) {
            if (lcp_delta(keys, nn, i, i + (s + t) * d) > dnode) s += t;
            if (t == 1) break;
        }
        const int gamma = i + s * d + min(d, 0);
        const int lo = min(i, j), hi = max(i, j);
        const uint32_t left = lo == gamma ? (kLeafBit | (uint32_t)(keys[gamma] & 0x3FFu)) : (uint32_t)gamma;
        const uint32_t right = hi == gamma + 1 ? (kLeafBit | (uint32_t)(keys[gamma + 1] & 0x3FFu)) : (uint32_t)(gamma + 1);
        // child bits, and the box of a leaf child in its slot; an internal child writes its
        // own box into the slot when it is finished (step 5)
        nodef[16 * i + 12] = __uint_as_float(left);
        nodef[16 * i + 13] = __uint_as_float(right);
        const uint32_t ch[2] = {left, right};
        for (int k = 0; k < 2; ++k) {
            if (ch[k] & kLeafBit) {
                const uint32_t q = ch[k] & ~kLeafBit;
                const float4 l = box[2 * q], h = box[2 * q + 1];
                float* slot = nodef + 16 * i + k;  // component c at slot[2 c]
                slot[0] = l.x;
                slot[2] = l.y;
                slot[4] = l.z;
                slot[6] = h.x;
                slot[8] = h.y;
                slot[10] = h.z;
            } else {
                parent[ch[k]] = 2u * (uint32_t)i + (uint32_t)k;
            }
        }
        done[i] = (int)((left & kLeafBit) == 0u) + (int)((right & kLeafBit) == 0u);  // internal children pending
    }
    if (tid == 0) parent[0] = ~0u;  // node 0 is the root
    __syncthreads();
    // 5. boxes bottom-up (the atomic scheme of Karras): a finished node writes the union of its
    // two slots into its parent's slot and counts itself off the parent's pending children;
    // the child that finishes a parent goes on with it.  Walks start at the nodes whose
    // children are both leaves, marked (-1) before any walk runs.
    for (uint32_t i = tid; i + 1 < m; i += nt)
        if (done[i] == 0) done[i] = -1;
    __syncthreads();
    for (uint32_t i0 = tid; i0 + 1 < m; i0 += nt) {
        if (done[i0] != -1) continue;
        uint32_t i = i0;
        for (int steps = 0; steps < 64; ++steps) {
            const uint32_t pa = parent[i];
            if (pa == ~0u || (pa >> 1) + 1 >= m) break;  // the root (or a malformed link)
            const volatile float* nd = nodef + 16 * i;
            volatile float* slot = nodef + 16 * (pa >> 1) + (pa & 1u);  // component c at slot[2 c]
            slot[0] = fminf(nd[0], nd[1]);
            slot[2] = fminf(nd[2], nd[3]);
            slot[4] = fminf(nd[4], nd[5]);
            slot[6] = fmaxf(nd[6], nd[7]);
            slot[8] = fmaxf(nd[8], nd[9]);
            slot[10] = fmaxf(nd[10], nd[11]);
            __threadfence_block();
            if (atomicSub(&done[pa >> 1], 1) != 1) break;  // its other child is not finished yet
            __threadfence_block();
            i = pa >> 1;
        }
    }
    __syncthreads();
    return out;
}

// Slab test of a box against the ray from its slab parameters t = fma(x,
// 1/d, -o/d) for its min (l) and max (h) planes per axis.  The roundings
// move a slab plane by about (|o| + L) 2^-24 along its axis for a box at
// distance L along the ray; since |o| <= m + L (m the box's largest
// coordinate), that stays far inside the box's expansion 1e-5 (1 + m) plus
// the 1e-5 L relative slack below, so the test is conservative,
// axis-parallel rays (|1/d| up to 1e30) included.  tcap: the best hit with
// slack.
__device__ __forceinline__ bool slab_entry(float lx, float hx, float ly, float hy, float lz, float hz, float tcap,
                                           float& tnear) {
    const float tmin = fmaxf(fmaxf(fminf(lx, hx), fminf(ly, hy)), fminf(lz, hz));
    const float tmax = fminf(fminf(fmaxf(lx, hx), fmaxf(ly, hy)), fmaxf(lz, hz));
    tnear = tmin;
    // conservative: slack on both ends (boxes are expanded as well)
    return tmax * 1.00001f + 1e-6f >= fmaxf(tmin, 0.f) && tmin <= tcap;
}

// 1 / d for the slab tests, |d| raised to at least 1e-30 (sign kept), by the
// fast reciprocal: its few-ulp error moves slab planes by far less than the
// boxes' expansion and the tests' slack.
__device__ __forceinline__ float safe_inv(float d) {
    const float dd = fabsf(d) < 1e-30f ? copysignf(1e-30f, d) : d;
    return __fdividef(1.0f, dd);
}

// hit_rect for a caller that only needs hits no farther than `best`: a
// rectangle whose plane lies behind the ray or beyond best is rejected on the
// fast quotient (a few ulp; rejection only outside a 0.1 % margin, so no
// hit that hit_rect would report at t <= best is lost); the others take
// hit_rect's exact steps, so an accepted t is hit_rect's.
__device__ __forceinline__ bool hit_rect_within(const PrimGeom& g, V3 o, V3 d, float best, float& t_out) {
    const V3 n{g.n_kind.x, g.n_kind.y, g.n_kind.z};
    const float denom = sdot(n, d);
    if (denom == 0.0f) return false;
    const V3 a{g.a_r.x, g.a_r.y, g.a_r.z};
    const float num = sdot(n, ssub(a, o));
    const float ta = __fdividef(num, denom);
    if (!(ta > 0.999f * kTMin) || ta > 1.001f * best) return false;
    const float t = __fdiv_rn(num, denom);
    if (!(t > kTMin)) return false;
    const V3 rel = ssub(smadd(o, t, d), a);
    const float al = __fmul_rn(sdot(rel, V3{g.u_iuu.x, g.u_iuu.y, g.u_iuu.z}), g.u_iuu.w);
    const float be = __fmul_rn(sdot(rel, V3{g.v_ivv.x, g.v_ivv.y, g.v_ivv.z}), g.v_ivv.w);
    if (!(al >= 0.0f && al <= 1.0f && be >= 0.0f && be <= 1.0f)) return false;
    t_out = t;
    return true;
}

__device__ __forceinline__ void test_prim(const PrimGeom* __restrict__ prims, uint32_t pi, V3 o, V3 d, float& best,
                                          int& idx) {
    const PrimGeom& g = prims[pi];
    float t;
    const bool hit =
        (__float_as_uint(g.n_kind.w) == KIND_SPHERE) ? hit_sphere(g, o, d, t) : hit_rect_within(g, o, d, best, t);
    if (hit && (t < best || (t == best && (int)pi < idx))) {
        best = t;
        idx = (int)pi;
    }
}

// The walk behind both queries: the large list, then the tree, keeping the
// smallest (t, index) starting from (best, idx); kFirstCloser stops as soon
// as anything beats the starting pair.  Child indices are range-checked and
// the walk is capped at 4n + 64 visits, so a malformed tree yields a wrong
// answer (caught by the parity tests) rather than an out-of-range read or an
// endless loop.
template <bool kFirstCloser>
__device__ inline int bvh_walk(const Bvh& b, const PrimGeom* __restrict__ prims, uint32_t n, V3 o, V3 d,
                               float& best, int idx) {
    const int idx0 = idx;
    for (uint32_t k = 0; k < b.n_large; ++k) {
        test_prim(prims, b.large[k], o, d, best, idx);
        if (kFirstCloser && idx != idx0) return idx;
    }
    if (b.n_tree == 1) {
        if ((b.root & ~kLeafBit) < n) test_prim(prims, b.root & ~kLeafBit, o, d, best, idx);
    } else if (b.n_tree >= 2) {
        const float3 inv = make_float3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
        const float3 ooi = make_float3(-o.x * inv.x, -o.y * inv.y, -o.z * inv.z);
        const float2 ix2 = make_float2(inv.x, inv.x), iy2 = make_float2(inv.y, inv.y), iz2 = make_float2(inv.z, inv.z);
        const float2 ox2 = make_float2(ooi.x, ooi.x), oy2 = make_float2(ooi.y, ooi.y), oz2 = make_float2(ooi.z, ooi.z);
        const uint32_t m = b.n_tree;
        uint32_t stack[kBvhStack];
        int sp = 0;
        uint32_t node = b.root;
        for (uint32_t visits = 0; visits < 4 * n + 64; ++visits) {
            const float4* q = b.nodes + 4 * node;
            const float4 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
            const uint32_t c0 = __float_as_uint(q3.x), c1 = __float_as_uint(q3.y);
            // slab parameters of both children, one packed FMA per plane pair
            const float2 tlx = __ffma2_rn(make_float2(q0.x, q0.y), ix2, ox2);
            const float2 tly = __ffma2_rn(make_float2(q0.z, q0.w), iy2, oy2);
            const float2 tlz = __ffma2_rn(make_float2(q1.x, q1.y), iz2, oz2);
            const float2 thx = __ffma2_rn(make_float2(q1.z, q1.w), ix2, ox2);
            const float2 thy = __ffma2_rn(make_float2(q2.x, q2.y), iy2, oy2);
            const float2 thz = __ffma2_rn(make_float2(q2.z, q2.w), iz2, oz2);
            float t0 = 0.f, t1 = 0.f;
            const float tcap = best * 1.00001f + 1e-6f;
            bool h0 = slab_entry(tlx.x, thx.x, tly.x, thy.x, tlz.x, thz.x, tcap, t0);
            bool h1 = slab_entry(tlx.y, thx.y, tly.y, thy.y, tlz.y, thz.y, tcap, t1);
            // leaf children: their primitive right away (the second against the updated best)
            if (h0 && (c0 & kLeafBit)) {
                if ((c0 & ~kLeafBit) < n) test_prim(prims, c0 & ~kLeafBit, o, d, best, idx);
                h0 = false;
            }
            if (h1 && (c1 & kLeafBit)) {
                if ((c1 & ~kLeafBit) < n && t1 <= best * 1.00001f + 1e-6f)
                    test_prim(prims, c1 & ~kLeafBit, o, d, best, idx);
                h1 = false;
            }
            if (kFirstCloser && idx != idx0) break;
            h0 = h0 && c0 + 1 < m;
            h1 = h1 && c1 + 1 < m;
            if (h0 && h1) {
                const bool first0 = t0 <= t1;
                if (sp < kBvhStack) stack[sp++] = first0 ? c1 : c0;
                node = first0 ? c0 : c1;
                continue;
            }
            if (h0 || h1) {
                node = h0 ? c0 : c1;
                continue;
            }
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    return idx;
}

// Nearest hit: same (t, index) result as trace_nearest.
__device__ inline int bvh_nearest(const Bvh& b, const PrimGeom* __restrict__ prims, uint32_t n, V3 o, V3 d,
                                  float& t_hit) {
    float best = __int_as_float(0x7f800000);
    const int idx = bvh_walk<false>(b, prims, n, o, d, best, -1);
    t_hit = best;
    return idx;
}

// Whether a primitive other than li comes before (t_l, li) in the (t, index)
// order along the ray: with (t_l, li) li's own hit, the same decision as
// "the nearest hit is not li", but the walk prunes everything beyond t_l and
// stops at the first primitive in front.
__device__ inline bool bvh_occluded(const Bvh& b, const PrimGeom* __restrict__ prims, uint32_t n, V3 o, V3 d,
                                    float t_l, int li) {
    float best = t_l;
    return bvh_walk<true>(b, prims, n, o, d, best, li) != li;
}

}  // namespace nirc
