// nirc_pt.cu -- path-tracing kernels of the two-level estimator.
//
// k_camera, then k_resid: per pixel, the camera ray (1 spp, Philox jitter)
//   and the shading record of the first hit (paper: surface parameter
//   buffer), traced by the camera pass with consecutive pixels on
//   consecutive lanes; then the residual level's M BSDF-sampled directions
//   with their path-traced incident radiance L_j (eq. L_r, the L_i term),
//   Russian roulette with termination probability 0.1 (paper: section
//   "Results", implementation paragraph), by the residual pass from the
//   records.  In the residual pass lanes regenerate work: one ray per busy
//   lane per iteration, new pixels from a work counter as old ones finish.
// k_gen_train: the separate training pass (section "Cache application"):
//   T paths from uniformly drawn pixels, one record per path, organised the
//   same way.
//
// k_primary_bth: the biased estimator's camera path (Balanced Termination
//   Heuristic), see below.
// Multi-vertex estimator: k_resid also hands the cache kernels the
//   records, throughputs and continuation rows of each residual path's
//   second and third vertex (MvOut).
//
// The kernels are persistent: each CTA stages the primitives' geometry in
// shared memory and, for scenes of more than 16 primitives, builds its own
// bounding-volume hierarchy there once, then loops over pixels (paths).
//
// Light mode 1 (template kNee; eq. Lsplit): L_i = L_ind + L_nee.  At the
// shading point one light sample (uniform emitting rectangle, uniform point,
// shadow ray) is combined by the power heuristic with the M residual
// directions as the BSDF technique, whose first-hit emission joins the
// direct part; along paths every vertex takes a light sample against the
// continuation direction, and emission reached by a continuation is
// weighted the same way.  The residual paths and the training targets then
// carry L_ind, which is what the cache learns.  Shadow-ray decisions are
// strict binary32, like every other decision.
#include "nirc_bvh.cuh"
#include "nirc_internal.h"

namespace nirc {

// Threads per CTA.  One CTA per SM, so that each SM holds one copy of the
// geometry and hierarchy in shared memory and the rest of the unified cache
// serves as L1 (the traversal stacks and register spills live in local
// memory).  The traversal is latency-bound: 32 warps at 64 registers (some
// spilled to L1) beat 20 at 96 (residual pass at 1080p: 1.00 vs 1.11 ms;
// light mode 1 3.09 vs 3.33 ms at 16 warps; the biased camera path 0.33 vs
// 0.44 ms).  The training pass keeps 512-thread CTAs: its 65,536 paths would
// fill only 64 CTAs of 1024.
constexpr int kPtThreads = 1024;      // k_camera, k_resid and their batched forms
constexpr int kPtThreadsBth = 1024;   // k_primary_bth
constexpr int kPtThreadsTrain = 512;  // k_gen_train
constexpr uint32_t kBvhMinPrims = 17;

struct FrameArgs {
    uint32_t W, H, N, M, D, n_prims;
    uint32_t k0, k1;
    uint32_t env_mode;  // light mode 2: residual rows are one visibility ray times L_env
    unsigned long long* rays;  // optional: gains the rays traced
};

// The scene's cube map (header reserved[0] = face size, texels after the primitives).
__device__ __forceinline__ EnvMap scene_env(const SceneHeader& hd, const Prim* __restrict__ gp, uint32_t n_prims) {
    EnvMap e;
    e.S = hd.reserved[0];
    e.tex = reinterpret_cast<const float4*>(gp + n_prims);
    return e;
}

// Emitting rectangles in primitive order (the light technique's choices).
struct Lights {
    const uint16_t* idx;
    uint32_t n;
};

// Multi-vertex estimator: per residual path (unit u = pixel * M + j) the
// record of its vertices 2 and 3 ([k - 2][P M]), the throughput to each
// (w_j / M included) and the continuation row (direction, weight w / q
// relative to that throughput; w = 0 in .wi when the path stops there).
struct MvOut {
    nirc_record* rec;
    float4* beta;
    ResidRow* row;
    uint64_t PM;
};

// Nearest-hit queries over the CTA's primitives (brute force or hierarchy).
struct Tracer {
    const PrimGeom* prims;
    uint32_t n;
    Bvh tree;
    bool bvh;
    mutable uint32_t rays = 0;  // nearest-hit queries of this thread
    __device__ __forceinline__ int nearest(V3 o, V3 d, float& t) const {
        ++rays;
        return bvh ? bvh_nearest(tree, prims, n, o, d, t) : trace_nearest(prims, n, o, d, t);
    }
    // Whether the nearest hit along (o, d) is another primitive than li, given
    // li's own hit at t_l (shadow rays).
    __device__ __forceinline__ bool occluded(V3 o, V3 d, float t_l, int li) const {
        ++rays;
        if (bvh) return bvh_occluded(tree, prims, n, o, d, t_l, li);
        float t;
        return trace_nearest(prims, n, o, d, t) != li;
    }
};

// Add the threads' ray counts to *out (one atomic per converged group).
__device__ __forceinline__ void add_rays(unsigned long long* out, uint32_t r) {
    const unsigned m = __activemask();
    const uint32_t s = __reduce_add_sync(m, r);
    if ((threadIdx.x & 31u) == (uint32_t)(__ffs(m) - 1)) atomicAdd(out, (unsigned long long)s);
}

// Shared bytes of the staged geometry and hierarchy (the light list follows, 16-byte aligned).
__host__ __device__ __forceinline__ size_t pt_geom_bytes(uint32_t n_prims) {
    const size_t b = (size_t)n_prims * sizeof(PrimGeom) + (n_prims >= kBvhMinPrims ? bvh_smem_bytes(n_prims) : 0);
    return (b + 15) & ~(size_t)15;
}

// Stage the scene header and primitive geometry, build the hierarchy.
__device__ __forceinline__ Tracer setup_scene(const SceneHeader* __restrict__ hd_g, const Prim* __restrict__ gp,
                                              uint32_t n_prims, unsigned char* smem, SceneHeader* hd) {
    PrimGeom* sp = reinterpret_cast<PrimGeom*>(smem);
    stage_prims(sp, gp, n_prims);
    if (threadIdx.x < sizeof(SceneHeader) / 16)
        reinterpret_cast<float4*>(hd)[threadIdx.x] = __ldg(reinterpret_cast<const float4*>(hd_g) + threadIdx.x);
    __syncthreads();
    Tracer tr;
    tr.prims = sp;
    tr.n = n_prims;
    tr.tree = Bvh{nullptr, nullptr, 0u, 0u, 0u};
    tr.bvh = n_prims >= kBvhMinPrims;
    if (tr.bvh) {
        tr.tree = bvh_build(sp, n_prims, smem + (size_t)n_prims * sizeof(PrimGeom));
        __syncthreads();
    }
    return tr;
}

__device__ __forceinline__ bool rect_emitter(const Prim* __restrict__ Q) {
    return __ldg(&Q->kind) == KIND_RECT &&
           (__ldg(&Q->emission[0]) > 0.f || __ldg(&Q->emission[1]) > 0.f || __ldg(&Q->emission[2]) > 0.f);
}

// Thread 0 lists the emitting rectangles in primitive order (the order the
// light choice indexes); every thread of the CTA calls it.
__device__ __forceinline__ Lights collect_lights(const Prim* __restrict__ gp, uint32_t n_prims, uint16_t* s_idx,
                                                 uint32_t* s_n) {
    if (threadIdx.x == 0) {
        uint32_t k = 0;
        for (uint32_t i = 0; i < n_prims; ++i)
            if (rect_emitter(gp + i)) s_idx[k++] = (uint16_t)i;
        *s_n = k;
    }
    __syncthreads();
    return Lights{s_idx, *s_n};
}

__device__ __forceinline__ float rect_area(const PrimGeom& g) {
    const float cx = g.u_iuu.y * g.v_ivv.z - g.u_iuu.z * g.v_ivv.y;
    const float cy = g.u_iuu.z * g.v_ivv.x - g.u_iuu.x * g.v_ivv.z;
    const float cz = g.u_iuu.x * g.v_ivv.y - g.u_iuu.y * g.v_ivv.x;
    return sqrtf(cx * cx + cy * cy + cz * cz);
}

// Solid-angle density of the light technique for direction d toward a point
// at distance t on emitting rectangle g.
__device__ __forceinline__ float light_pdf(const PrimGeom& g, V3 d, float t, uint32_t n_lights) {
    const float cl = fabsf(dot_acc(V3{g.n_kind.x, g.n_kind.y, g.n_kind.z}, d));
    return t * t / (cl * rect_area(g) * (float)n_lights);
}

__device__ __forceinline__ float power_weight(float na_pa, float nb_pb) {
    const float a = na_pa * na_pa, b = nb_pb * nb_pb;
    return a + b > 0.f ? a / (a + b) : 0.f;
}

// One light sample at a shading point (p, n, wo, material), MIS against n_b
// BSDF samples; adds into out and returns the decision word
// (emitter | geometry ok << 16 | visible << 17).
__device__ __forceinline__ uint32_t nee_sample(const Tracer& tr, const Prim* __restrict__ gp, const Lights& lt, V3 p,
                                               V3 n, V3 wo, float3 alb, float rough, uint32_t mat, uint32_t n_b,
                                               uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c3,
                                               float3& out) {
    if (lt.n == 0 || mat == MAT_BLACK) return 0u;
    const U4 r = philox(k0, k1, c0, c1, 0u, c3);
    const uint32_t e = __umulhi(r.x, lt.n);
    const uint32_t li = lt.idx[e];
    const PrimGeom& g = tr.prims[li];
    const float u1 = u01(r.y), u2 = u01(r.z);
    const V3 pt{__fadd_rn(__fadd_rn(g.a_r.x, __fmul_rn(u1, g.u_iuu.x)), __fmul_rn(u2, g.v_ivv.x)),
                __fadd_rn(__fadd_rn(g.a_r.y, __fmul_rn(u1, g.u_iuu.y)), __fmul_rn(u2, g.v_ivv.y)),
                __fadd_rn(__fadd_rn(g.a_r.z, __fmul_rn(u1, g.u_iuu.z)), __fmul_rn(u2, g.v_ivv.z))};
    const V3 v = ssub(pt, p);
    const float dist2 = sdot(v, v);
    const float dist = __fsqrt_rn(dist2);
    const V3 w = snormalize(v);
    const float cx = sdot(n, w);
    const float cl = -sdot(V3{g.n_kind.x, g.n_kind.y, g.n_kind.z}, w);
    const Prim* L = gp + li;
    const bool ok = cx > 0.f && (cl > 0.f || ((__ldg(&L->flags) & EMIT_TWO_SIDED) && cl < 0.f));
    uint32_t word = e | ((uint32_t)ok << 16);
    if (!ok) return word;
    // visible: the nearest hit along w is the light, at the sampled distance (the light's own
    // hit first, then an occlusion walk that prunes everything beyond it)
    float t = 0.f;
    const bool visible = hit_rect(g, p, w, t) && fabsf(__fsub_rn(t, dist)) <= __fmul_rn(1e-3f, dist) &&
                         !tr.occluded(p, w, t, (int)li);
    word |= (uint32_t)visible << 17;
    if (!visible) return word;
    const BsdfEval be = bsdf_eval(n, wo, w, alb, rough, mat);
    const float pl = light_pdf(g, w, dist, lt.n);
    const float k = power_weight(pl, (float)n_b * be.pdf) / pl;
    out.x += be.fcos.x * __ldg(&L->emission[0]) * k;
    out.y += be.fcos.y * __ldg(&L->emission[1]) * k;
    out.z += be.fcos.z * __ldg(&L->emission[2]) * k;
    return word;
}

__device__ __forceinline__ void write_record(nirc_record* dst, const Hit& h, V3 d, const Prim* P, uint32_t prim,
                                             uint32_t flags) {
    float4* q = reinterpret_cast<float4*>(dst);
    q[0] = make_float4(h.p.x, h.p.y, h.p.z, h.n.x);
    q[1] = make_float4(h.n.y, h.n.z, -d.x, -d.y);
    q[2] = make_float4(-d.z, __ldg(&P->albedo[0]), __ldg(&P->albedo[1]), __ldg(&P->albedo[2]));
    q[3] = make_float4(__ldg(&P->roughness), __uint_as_float(prim), __uint_as_float(flags), 0.f);
}

// Vertex k = seg + 1 (seg 1, 2) of a residual path: its record and throughput;
// the continuation row is invalid until mv_continue_row sets it.
__device__ __forceinline__ void mv_vertex(const MvOut* mv, uint32_t seg, uint64_t unit, const Hit& h, V3 d,
                                          const Prim* Q, uint32_t prim, uint32_t flags, float3 pre, float3 beta) {
    const uint64_t slot = (uint64_t)(seg - 1) * mv->PM + unit;
    write_record(mv->rec + slot, h, d, Q, prim, 1u | ((flags & 3u) << 1));
    mv->beta[slot] = make_float4(pre.x * beta.x, pre.y * beta.y, pre.z * beta.z, 0.f);
    mv->row[slot].wi = make_float4(0.f, 0.f, 1.f, 0.f);
    mv->row[slot].w = make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void mv_continue_row(const MvOut* mv, uint32_t seg, uint64_t unit, V3 wi, float3 w) {
    const uint64_t slot = (uint64_t)(seg - 1) * mv->PM + unit;
    mv->row[slot].wi = make_float4(wi.x, wi.y, wi.z, 1.f);
    mv->row[slot].w = make_float4(w.x / kRRContinue, w.y / kRRContinue, w.z / kRRContinue, 0.f);
}
// Both later vertices of a unit not reached (yet): zero records (flags 0).
__device__ __forceinline__ void mv_clear(const MvOut* mv, uint64_t unit) {
    for (uint32_t k = 0; k < 2; ++k) {
        const uint64_t slot = (uint64_t)k * mv->PM + unit;
        float4* q = reinterpret_cast<float4*>(mv->rec + slot);
        q[0] = q[1] = q[2] = q[3] = make_float4(0.f, 0.f, 0.f, 0.f);
        mv->beta[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
        mv->row[slot].wi = make_float4(0.f, 0.f, 1.f, 0.f);
        mv->row[slot].w = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// One segment of an L_ind path (light mode 1) after its ray was traced:
// emission found by the continuation (MIS weighted; the first hit's goes to
// first_emit, weighted against nb0 BSDF samples of density pb at the
// shading point), a light sample at the vertex, Russian roulette, the next
// direction and its density.  Returns true when the path ends.
__device__ __forceinline__ bool path_segment_nee(const Tracer& tr, const Prim* __restrict__ gp, const Lights& lt,
                                                 int prim, float t, V3& o, V3& d, float3& beta, float3& L,
                                                 uint32_t& seg, uint32_t max_depth, uint32_t k0, uint32_t k1,
                                                 uint32_t c0, uint32_t c1, uint64_t& sig, float& pb, uint32_t nb0,
                                                 float3& first_emit, const MvOut* mv, uint64_t unit, float3 pre) {
    sig = sig_mix(sig, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
    if (prim < 0) return true;
    const Hit h = hit_info(tr.prims[prim], o, d, t);
    const Prim* Q = gp + prim;
    const uint32_t flags = __ldg(&Q->flags);
    if (h.front || (flags & EMIT_TWO_SIDED)) {
        const float3 le = make_float3(__ldg(&Q->emission[0]), __ldg(&Q->emission[1]), __ldg(&Q->emission[2]));
        if (le.x > 0.f || le.y > 0.f || le.z > 0.f) {
            float wb = 1.f;
            if (__ldg(&Q->kind) == KIND_RECT && lt.n)
                wb = power_weight((float)(seg == 1 ? nb0 : 1u) * pb, light_pdf(tr.prims[prim], d, t, lt.n));
            if (seg == 1) {
                first_emit = make_float3(le.x * wb, le.y * wb, le.z * wb);
            } else {
                L.x += beta.x * le.x * wb;
                L.y += beta.y * le.y * wb;
                L.z += beta.z * le.z * wb;
            }
        }
    }
    const float3 alb = make_float3(__ldg(&Q->albedo[0]), __ldg(&Q->albedo[1]), __ldg(&Q->albedo[2]));
    const float rough = __ldg(&Q->roughness);
    const V3 wo = sneg(d);
    float3 dl = make_float3(0.f, 0.f, 0.f);
    sig = sig_mix(sig, nee_sample(tr, gp, lt, h.p, h.n, wo, alb, rough, flags & 3u, seg < max_depth ? 1u : 0u, k0,
                                  k1, c0, c1, PURPOSE_LIGHT + 16u * seg, dl));
    L.x += beta.x * dl.x;
    L.y += beta.y * dl.y;
    L.z += beta.z * dl.z;
    const bool mv_here = mv && seg <= 2u;
    if (mv_here) mv_vertex(mv, seg, unit, h, d, Q, (uint32_t)prim, flags, pre, beta);
    if (seg == max_depth) return true;
    const U4 r = philox(k0, k1, c0, c1, 0u, PURPOSE_RR + 16u * seg);
    const bool cont = u01(r.x) < kRRContinue;
    sig = sig_mix(sig, (uint32_t)cont);
    if (!cont) return true;
    beta.x /= kRRContinue;
    beta.y /= kRRContinue;
    beta.z /= kRRContinue;
    const BsdfSample s = sample_bsdf(h.n, wo, alb, rough, flags & 3u, k0, k1, c0, c1, PURPOSE_BOUNCE + 16u * seg);
    sig = sig_mix(sig, s.word);
    if (!s.valid) return true;
    beta.x *= s.w.x;
    beta.y *= s.w.y;
    beta.z *= s.w.z;
    if (mv_here) mv_continue_row(mv, seg, unit, s.wi, s.w);
    pb = bsdf_eval(h.n, wo, s.wi, alb, rough, flags & 3u).pdf;
    o = h.p;
    d = s.wi;
    ++seg;
    return false;
}

// One segment of a path (residual or training) after its ray was traced:
// emission of the hit, then Russian roulette and the next BSDF direction.
// Counters (c0, c1) identify the path, `seg` its segment (1-based).  Returns
// true when the path ends; otherwise (o, d) is the next ray and seg + 1.
__device__ __forceinline__ bool path_segment(const Tracer& tr, const Prim* __restrict__ gp, int prim, float t, V3& o,
                                             V3& d, float3& beta, float3& L, uint32_t& seg, uint32_t max_depth,
                                             uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint64_t& sig,
                                             const MvOut* mv = nullptr, uint64_t unit = 0,
                                             float3 pre = make_float3(0.f, 0.f, 0.f)) {
    sig = sig_mix(sig, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
    if (prim < 0) return true;
    const Hit h = hit_info(tr.prims[prim], o, d, t);
    const Prim* Q = gp + prim;
    const uint32_t flags = __ldg(&Q->flags);
    if (h.front || (flags & EMIT_TWO_SIDED)) {
        L.x += beta.x * __ldg(&Q->emission[0]);
        L.y += beta.y * __ldg(&Q->emission[1]);
        L.z += beta.z * __ldg(&Q->emission[2]);
    }
    const bool mv_here = mv && seg <= 2u;
    if (mv_here) mv_vertex(mv, seg, unit, h, d, Q, (uint32_t)prim, flags, pre, beta);
    if (seg == max_depth) return true;
    const U4 r = philox(k0, k1, c0, c1, 0u, PURPOSE_RR + 16u * seg);
    const bool cont = u01(r.x) < kRRContinue;
    sig = sig_mix(sig, (uint32_t)cont);
    if (!cont) return true;
    beta.x /= kRRContinue;
    beta.y /= kRRContinue;
    beta.z /= kRRContinue;
    const float3 alb = make_float3(__ldg(&Q->albedo[0]), __ldg(&Q->albedo[1]), __ldg(&Q->albedo[2]));
    const BsdfSample s =
        sample_bsdf(h.n, sneg(d), alb, __ldg(&Q->roughness), flags & 3u, k0, k1, c0, c1, PURPOSE_BOUNCE + 16u * seg);
    sig = sig_mix(sig, s.word);
    if (!s.valid) return true;
    beta.x *= s.w.x;
    beta.y *= s.w.y;
    beta.z *= s.w.z;
    if (mv_here) mv_continue_row(mv, seg, unit, s.wi, s.w);
    o = h.p;
    d = s.wi;
    ++seg;
    return false;
}

// Take `need` lanes' next work items from the counter (one atomic per warp);
// returns the lane's item (or a value >= limit when none is left).
__device__ __forceinline__ uint64_t fetch_work(unsigned long long* work, bool need) {
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned needm = __ballot_sync(0xffffffffu, need);
    if (!needm) return ~0ull;
    const int leader = __ffs(needm) - 1;
    unsigned long long first = 0;
    if ((int)lane == leader) first = atomicAdd(work, (unsigned long long)__popc(needm));
    first = __shfl_sync(0xffffffffu, first, leader);
    return first + (uint64_t)__popc(needm & ((1u << lane) - 1u));
}

// Lane state of the residual pass and the training pass: which pixel (path),
// which ray is in flight.
enum : uint32_t { kNeedPixel = 0, kCameraRay = 1, kResidRay = 2, kNoMoreWork = 3 };

// Residual pass: per pixel the camera pass hit (its record, emission and
// signature so far), for j = 0..M-1 a residual direction and its path (eq.
// L_r's L_j), exactly in the order and with the Philox counters of a
// sequential loop.  The loop is organised as a per-lane state machine so
// that every iteration traces one ray per busy lane: a lane whose pixel is
// done takes the next pixel from a work counter (one atomic per warp), so
// lanes do not idle while others finish long paths.  kExtra compiles in the
// multi-vertex outputs and light mode 2 (environment visibility); frames
// with neither run the instance without that code, which keeps the loop
// smaller in the instruction cache.
template <bool kNee, bool kExtra>
__device__ __forceinline__ void resid_pass(const SceneHeader* __restrict__ hd_g, const Prim* __restrict__ gp,
                                              const FrameArgs& a, nirc_record* __restrict__ recs,
                                              PixelBase* __restrict__ base, ResidRow* __restrict__ rows,
                                              uint64_t* __restrict__ sig_out, uint32_t* __restrict__ count,
                                              unsigned long long* __restrict__ work, const MvOut& mvo) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SceneHeader hd;
    __shared__ uint32_t s_nlights;
    const Tracer tr = setup_scene(hd_g, gp, a.n_prims, smem_raw, &hd);
    Lights lt{nullptr, 0u};
    if constexpr (kNee)
        lt = collect_lights(gp, a.n_prims, reinterpret_cast<uint16_t*>(smem_raw + pt_geom_bytes(a.n_prims)),
                            &s_nlights);
    // multi-vertex estimator: later-vertex data per residual path (kExtra instances only)
    const MvOut* mv = (kExtra && mvo.rec) ? &mvo : nullptr;
    const float invM = a.M ? 1.0f / (float)a.M : 0.f;

    const uint64_t P = (uint64_t)a.W * a.H;
    uint32_t stage = kNeedPixel;
    uint32_t pix = 0, j = 0, seg = 0, nvalid = 0;
    V3 o{0.f, 0.f, 0.f}, d{0.f, 0.f, 1.f};
    V3 sp{0.f, 0.f, 0.f}, sn{0.f, 0.f, 1.f}, swo{0.f, 0.f, 1.f};  // shading point, normal, wo
    float3 salb = make_float3(0.f, 0.f, 0.f), le = salb, wl = salb, L = salb, beta = salb, sw = salb;
    float srough = 1.f;
    uint32_t smat = 0;
    uint64_t sig = kSigInit;
    float pb = 0.f;                                  // light mode 1: density of the current direction
    float3 first_emit = make_float3(0.f, 0.f, 0.f);  // light mode 1: first hit's weighted emission

    // Next residual sample of the current pixel: the first valid one becomes
    // the ray in flight; with none left the pixel's outputs are written.
    auto next_residual = [&]() -> uint32_t {
        ResidRow* my_rows = rows + (uint64_t)pix * a.M;
        for (; j < a.M; ++j) {
            if (mv) mv_clear(mv, (uint64_t)pix * a.M + j);
            const BsdfSample s = sample_bsdf(sn, swo, salb, srough, smat, a.k0, a.k1, pix, j, PURPOSE_RESID_DIR);
            sig = sig_mix(sig, s.word);
            my_rows[j].wi = make_float4(s.wi.x, s.wi.y, s.wi.z, s.valid ? 1.f : 0.f);
            my_rows[j].w = make_float4(s.w.x, s.w.y, s.w.z, 0.f);
            if (s.valid) {
                o = sp;
                d = s.wi;
                sw = s.w;
                beta = make_float3(1.f, 1.f, 1.f);
                L = make_float3(0.f, 0.f, 0.f);
                seg = 1;
                if constexpr (kNee) {
                    pb = bsdf_eval(sn, swo, s.wi, salb, srough, smat).pdf;
                    first_emit = make_float3(0.f, 0.f, 0.f);
                }
                return kResidRay;
            }
        }
        float3 w = wl;
        if (a.M) {
            const float inv = 1.0f / (float)a.M;
            w.x *= inv;
            w.y *= inv;
            w.z *= inv;
        }
        base[pix].le = make_float4(le.x, le.y, le.z, 0.f);
        base[pix].wl = make_float4(w.x, w.y, w.z, 0.f);
        if (sig_out) sig_out[2 * (uint64_t)pix] = sig;
        if (count) count[pix] = nvalid;
        return kNeedPixel;
    };

    while (true) {
        // lanes without a pixel take the next ones (warp-aggregated)
        const bool need = stage == kNeedPixel;
        const uint64_t mine = fetch_work(work, need);
        if (need) {
            if (mine >= P) {
                stage = kNoMoreWork;
            } else {
                // the camera pass traced the pixel: its record, emission and signature so far
                pix = (uint32_t)mine;
                const float4* q = reinterpret_cast<const float4*>(recs + pix);
                const float4 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
                const uint32_t rflags = __float_as_uint(q3.z);
                stage = kNeedPixel;  // a camera miss: the camera pass wrote the whole pixel
                if (rflags & 1u) {
                    sp = V3{q0.x, q0.y, q0.z};
                    sn = V3{q0.w, q1.x, q1.y};
                    swo = V3{q1.z, q1.w, q2.x};
                    salb = make_float3(q2.y, q2.z, q2.w);
                    srough = q3.x;
                    smat = (rflags >> 1) & 3u;
                    const float4 b = base[pix].le;
                    le = make_float3(b.x, b.y, b.z);
                    sig = sig_out ? sig_out[2 * (uint64_t)pix] : kSigInit;
                    wl = make_float3(0.f, 0.f, 0.f);
                    nvalid = 0;
                    j = 0;
                    stage = next_residual();
                }
            }
        }
        if (__all_sync(0xffffffffu, stage == kNoMoreWork)) break;

        float t = 0.f;
        int prim = -1;
        if (stage == kResidRay) prim = tr.nearest(o, d, t);

        if (stage == kResidRay) {
            bool end;
            if (kExtra && a.env_mode) {  // light mode 2: V(x, w_j) L_env(w_j), one ray
                sig = sig_mix(sig, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
                L = prim < 0 ? env_radiance(scene_env(hd, gp, a.n_prims), d) : make_float3(0.f, 0.f, 0.f);
                end = true;
            } else if constexpr (kNee)
                end = path_segment_nee(tr, gp, lt, prim, t, o, d, beta, L, seg, a.D, a.k0, a.k1, pix, j, sig, pb, a.M,
                                       first_emit, mv, (uint64_t)pix * a.M + j,
                                       make_float3(sw.x * invM, sw.y * invM, sw.z * invM));
            else
                end = path_segment(tr, gp, prim, t, o, d, beta, L, seg, a.D, a.k0, a.k1, pix, j, sig, mv,
                                   (uint64_t)pix * a.M + j, make_float3(sw.x * invM, sw.y * invM, sw.z * invM));
            if (end) {
                if constexpr (kNee) {
                    const float inv = 1.0f / (float)a.M;
                    le.x += sw.x * first_emit.x * inv;
                    le.y += sw.y * first_emit.y * inv;
                    le.z += sw.z * first_emit.z * inv;
                }
                wl.x += sw.x * L.x;
                wl.y += sw.y * L.y;
                wl.z += sw.z * L.z;
                ++nvalid;
                ++j;
                stage = next_residual();
            }
        }
    }
    if (a.rays) add_rays(a.rays, tr.rays);
}

// Camera pass: one camera ray per pixel, consecutive pixels on consecutive
// lanes (a warp's rays are nearly parallel and walk the hierarchy alike).  A
// hit writes the shading record, the emission seen (plus, in light mode 1,
// the light sample at the shading point) and the signature so far, which the
// residual pass continues; a miss writes the whole pixel.
template <bool kNee>
__device__ __forceinline__ void camera_pass(const SceneHeader* __restrict__ hd_g, const Prim* __restrict__ gp,
                                            const FrameArgs& a, nirc_record* __restrict__ recs,
                                            PixelBase* __restrict__ base, ResidRow* __restrict__ rows,
                                            uint64_t* __restrict__ sig_out, uint32_t* __restrict__ count,
                                            const MvOut& mvo, uint32_t cta, uint32_t n_cta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SceneHeader hd;
    __shared__ uint32_t s_nlights;
    const Tracer tr = setup_scene(hd_g, gp, a.n_prims, smem_raw, &hd);
    Lights lt{nullptr, 0u};
    if constexpr (kNee)
        lt = collect_lights(gp, a.n_prims, reinterpret_cast<uint16_t*>(smem_raw + pt_geom_bytes(a.n_prims)),
                            &s_nlights);
    const MvOut* mv = mvo.rec ? &mvo : nullptr;
    const uint64_t P = (uint64_t)a.W * a.H;
    const uint64_t stride = (uint64_t)n_cta * blockDim.x;  // CTAs [0, n_cta) of the frame, this one cta
    for (uint64_t q = (uint64_t)cta * blockDim.x + threadIdx.x; q < P; q += stride) {
        const uint32_t pix = (uint32_t)q;
        const U4 r = philox(a.k0, a.k1, pix, 0u, 0u, PURPOSE_CAMERA);
        V3 o, d;
        camera_ray(hd, a.W, a.H, pix % a.W, pix / a.W, u01(r.x), u01(r.y), o, d);
        float t = 0.f;
        const int prim = tr.nearest(o, d, t);
        uint64_t sig = sig_mix(kSigInit, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
        if (prim < 0) {
            float4* qr = reinterpret_cast<float4*>(recs + pix);
            qr[0] = qr[1] = qr[2] = qr[3] = make_float4(0.f, 0.f, 0.f, 0.f);
            base[pix].le = make_float4(0.f, 0.f, 0.f, 0.f);
            base[pix].wl = make_float4(0.f, 0.f, 0.f, 0.f);
            ResidRow* my_rows = rows + (uint64_t)pix * a.M;
            for (uint32_t jj = 0; jj < a.M; ++jj) {
                my_rows[jj].wi = make_float4(0.f, 0.f, 1.f, 0.f);
                my_rows[jj].w = make_float4(0.f, 0.f, 0.f, 0.f);
                if (mv) mv_clear(mv, (uint64_t)pix * a.M + jj);
            }
            if (sig_out) sig_out[2 * (uint64_t)pix] = sig;
            if (count) count[pix] = 0;
            continue;
        }
        const Hit h = hit_info(tr.prims[prim], o, d, t);
        const Prim* Pp = gp + prim;
        const uint32_t pflags = __ldg(&Pp->flags);
        const uint32_t smat = pflags & 3u;
        write_record(recs + pix, h, d, Pp, (uint32_t)prim, 1u | (smat << 1));
        float3 le = make_float3(0.f, 0.f, 0.f);
        if (h.front || (pflags & EMIT_TWO_SIDED))
            le = make_float3(__ldg(&Pp->emission[0]), __ldg(&Pp->emission[1]), __ldg(&Pp->emission[2]));
        if constexpr (kNee) {
            // direct light at the shading point: one light sample against the M residual directions
            const float3 salb = make_float3(__ldg(&Pp->albedo[0]), __ldg(&Pp->albedo[1]), __ldg(&Pp->albedo[2]));
            sig = sig_mix(sig, nee_sample(tr, gp, lt, h.p, h.n, sneg(d), salb, __ldg(&Pp->roughness), smat, a.M,
                                          a.k0, a.k1, pix, 0u, PURPOSE_LIGHT, le));
        }
        base[pix].le = make_float4(le.x, le.y, le.z, 0.f);
        if (sig_out) sig_out[2 * (uint64_t)pix] = sig;
    }
    if (a.rays) add_rays(a.rays, tr.rays);
}

template <bool kNee>
__global__ void __launch_bounds__(kPtThreads, 1)
    k_camera(const SceneHeader* __restrict__ hd_g, const Prim* __restrict__ gp, FrameArgs a,
             nirc_record* __restrict__ recs, PixelBase* __restrict__ base, ResidRow* __restrict__ rows,
             uint64_t* __restrict__ sig_out, uint32_t* __restrict__ count, MvOut mvo) {
    camera_pass<kNee>(hd_g, gp, a, recs, base, rows, sig_out, count, mvo, blockIdx.x, gridDim.x);
}

// Residual pass: the residual paths of the pixels the camera pass hit.
template <bool kNee, bool kExtra>
__global__ void __launch_bounds__(kPtThreads, 1)
    k_resid(const SceneHeader* __restrict__ hd_g, const Prim* __restrict__ gp, FrameArgs a,
            nirc_record* __restrict__ recs, PixelBase* __restrict__ base, ResidRow* __restrict__ rows,
            uint64_t* __restrict__ sig_out, uint32_t* __restrict__ count, unsigned long long* __restrict__ work,
            MvOut mvo) {
    resid_pass<kNee, kExtra>(hd_g, gp, a, recs, base, rows, sig_out, count, work, mvo);
}

// Several frames in one launch of each pass (the frame-request server's
// batches): CTAs [cta0, cta0 + n_cta) trace job j's frame, staging its scene
// once; the residual pass takes its pixels from the job's own counter.
struct PtJob {
    const SceneHeader* hd;
    const Prim* gp;
    FrameArgs a;
    nirc_record* recs;
    PixelBase* base;
    ResidRow* rows;
    unsigned long long* work;
    uint32_t cta0, n_cta;
};
struct PtJobs {
    uint32_t n;
    PtJob j[kMaxFrameJobs];
};

__device__ __forceinline__ const PtJob& pt_job(const PtJobs& jobs) {
    uint32_t ji = 0;
    while (ji + 1 < jobs.n && blockIdx.x >= jobs.j[ji + 1].cta0) ++ji;
    return jobs.j[ji];
}

template <bool kNee>
__global__ void __launch_bounds__(kPtThreads, 1) k_camera_batch(const __grid_constant__ PtJobs jobs) {
    const PtJob& J = pt_job(jobs);
    camera_pass<kNee>(J.hd, J.gp, J.a, J.recs, J.base, J.rows, nullptr, nullptr, MvOut{nullptr, nullptr, nullptr, 0},
                      blockIdx.x - J.cta0, J.n_cta);
}

template <bool kNee>
__global__ void __launch_bounds__(kPtThreads, 1) k_resid_batch(const __grid_constant__ PtJobs jobs) {
    const PtJob& J = pt_job(jobs);
    // batched frames are light mode 0 or 1 with the two-level estimator (their FrameArgs carry
    // env_mode 0, and no multi-vertex outputs), so the instance without those paths serves them
    resid_pass<kNee, false>(J.hd, J.gp, J.a, J.recs, J.base, J.rows, nullptr, nullptr, J.work,
                     MvOut{nullptr, nullptr, nullptr, 0});
}

// ---------------------------------------------------------------------------
// Biased estimator: path termination (Balanced Termination Heuristic and
// NRC's footprint test).  These quantities decide whether a path goes on,
// so they are strict binary32 in a fixed operation order.
// ---------------------------------------------------------------------------

// Density of the BSDF sampler at wi: cos/pi (Lambertian), or the one-sample
// mixture 1/2 cos/pi + 1/2 G1(wo) D / (4 cos_o) with D = a2 / (pi dd^2),
// dd = |n x h|^2 + a2 (n.h)^2, a = roughness^2.
__device__ __forceinline__ float sampler_pdf32(V3 n, V3 wo, V3 wi, float rough, uint32_t mat) {
    const float ci = sdot(n, wi);
    if (mat == MAT_BLACK || !(ci > 0.f)) return 0.f;
    if (mat == MAT_LAMBERT) return __fmul_rn(ci, kInvPi);
    const float co = sdot(n, wo);
    const V3 h = snormalize(V3{__fadd_rn(wo.x, wi.x), __fadd_rn(wo.y, wi.y), __fadd_rn(wo.z, wi.z)});
    const float a = __fmul_rn(rough, rough), a2 = __fmul_rn(a, a);
    const float cnh = sdot(n, h);
    const V3 cx{__fsub_rn(__fmul_rn(n.y, h.z), __fmul_rn(n.z, h.y)), __fsub_rn(__fmul_rn(n.z, h.x), __fmul_rn(n.x, h.z)),
                __fsub_rn(__fmul_rn(n.x, h.y), __fmul_rn(n.y, h.x))};
    const float dd = __fadd_rn(sdot(cx, cx), __fmul_rn(a2, __fmul_rn(cnh, cnh)));
    const float D = __fdiv_rn(a2, __fmul_rn(__fmul_rn(kPi, dd), dd));
    const float lam = __fsqrt_rn(__fadd_rn(a2, __fmul_rn(__fsub_rn(1.f, a2), __fmul_rn(co, co))));
    const float g1 = __fdiv_rn(__fmul_rn(2.f, co), __fadd_rn(co, lam));
    return __fadd_rn(__fmul_rn(0.5f, __fmul_rn(ci, kInvPi)),
                     __fmul_rn(0.5f, __fdiv_rn(__fmul_rn(g1, D), __fmul_rn(4.f, co))));
}

// Balanced Termination Heuristic: continuation probability p / (p + N_c / pi).
__device__ __forceinline__ float bth_continue_prob(float p, uint32_t n_c) {
    return __fdiv_rn(p, __fadd_rn(p, __fmul_rn((float)n_c, kInvPi)));
}

// Footprint term sqrt(t^2 / (p cos_in)) of one segment (NRC's spread heuristic).
__device__ __forceinline__ float spread_term(float t, float p, float cos_in) {
    return __fsqrt_rn(__fdiv_rn(__fmul_rn(t, t), __fmul_rn(p, cos_in)));
}

// Emission of primitive q seen along d at distance t from a vertex whose
// BSDF technique sampled d with density pb (light mode 1: power heuristic
// against the light technique for emitting rectangles).
template <bool kNee>
__device__ __forceinline__ float3 weighted_emission(const Tracer& tr, const Prim* __restrict__ gp, const Lights& lt,
                                                    int q, bool front, V3 d, float t, float pb) {
    const Prim* Q = gp + q;
    if (!(front || (__ldg(&Q->flags) & EMIT_TWO_SIDED))) return make_float3(0.f, 0.f, 0.f);
    const float3 le = make_float3(__ldg(&Q->emission[0]), __ldg(&Q->emission[1]), __ldg(&Q->emission[2]));
    if (!(le.x > 0.f || le.y > 0.f || le.z > 0.f)) return make_float3(0.f, 0.f, 0.f);
    float wb = 1.f;
    if constexpr (kNee) {
        if (__ldg(&Q->kind) == KIND_RECT && lt.n) wb = power_weight(pb, light_pdf(tr.prims[q], d, t, lt.n));
    }
    return make_float3(le.x * wb, le.y * wb, le.z * wb);
}

// Per pixel, the camera path of the biased estimator: from vertex x_i it
// continues along the BSDF-sampled w_i unless xi_i > P_s(w_i), or (i > 1)
// the footprint a exceeds 0.01 a_0, or i = max_depth.  Emission found along
// the path (and in light mode 1 a light sample at every vertex, with w_i as
// the one-sample BSDF technique, traced at the stopping vertex for its
// emission) goes into base.le; the stopping vertex's record and the
// throughput up to it are what the cache kernel completes.  One pixel per
// lane, pixels from the work counter.
template <bool kNee>
__global__ void __launch_bounds__(kPtThreadsBth, 1) k_primary_bth(const SceneHeader* __restrict__ hd_g,
                                                                const Prim* __restrict__ gp, FrameArgs a,
                                                                nirc_record* __restrict__ recs,
                                                                PixelBase* __restrict__ base,
                                                                float4* __restrict__ beta_out,
                                                                uint64_t* __restrict__ sig_out,
                                                                uint32_t* __restrict__ count,
                                                                unsigned long long* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SceneHeader hd;
    __shared__ uint32_t s_nlights;
    const Tracer tr = setup_scene(hd_g, gp, a.n_prims, smem_raw, &hd);
    Lights lt{nullptr, 0u};
    if constexpr (kNee)
        lt = collect_lights(gp, a.n_prims, reinterpret_cast<uint16_t*>(smem_raw + pt_geom_bytes(a.n_prims)),
                            &s_nlights);
    const uint64_t P = (uint64_t)a.W * a.H;
    while (true) {
        const uint64_t mine = fetch_work(work, true);
        if (__all_sync(0xffffffffu, mine >= P)) break;
        if (mine >= P) continue;
        const uint32_t pix = (uint32_t)mine;
        uint64_t sig = kSigInit;
        float3 le = make_float3(0.f, 0.f, 0.f), beta = make_float3(1.f, 1.f, 1.f);
        uint32_t stop_at = 0;
        const U4 rc = philox(a.k0, a.k1, pix, 0u, 0u, PURPOSE_CAMERA);
        V3 o, d;
        camera_ray(hd, a.W, a.H, pix % a.W, pix / a.W, u01(rc.x), u01(rc.y), o, d);
        float t = 0.f;
        int prim = tr.nearest(o, d, t);
        sig = sig_mix(sig, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
        if (prim >= 0) {
            Hit h = hit_info(tr.prims[prim], o, d, t);
            le = weighted_emission<false>(tr, gp, lt, prim, h.front, d, t, 0.f);
            const float c_a0 =
                __fmul_rn(0.01f, __fdiv_rn(__fmul_rn(t, t), __fmul_rn(__fmul_rn(4.f, kPi), fabsf(sdot(h.n, d)))));
            float spread = 0.f;
            for (uint32_t i = 1;; ++i) {
                const Prim* Q = gp + prim;
                const uint32_t mat = __ldg(&Q->flags) & 3u;
                const float3 alb = make_float3(__ldg(&Q->albedo[0]), __ldg(&Q->albedo[1]), __ldg(&Q->albedo[2]));
                const float rough = __ldg(&Q->roughness);
                const V3 wo = sneg(d);
                if constexpr (kNee) {
                    float3 dl = make_float3(0.f, 0.f, 0.f);
                    sig = sig_mix(sig, nee_sample(tr, gp, lt, h.p, h.n, wo, alb, rough, mat, 1u, a.k0, a.k1, pix, 0u,
                                                  PURPOSE_LIGHT + 16u * i, dl));
                    le.x += beta.x * dl.x;
                    le.y += beta.y * dl.y;
                    le.z += beta.z * dl.z;
                }
                const BsdfSample s =
                    sample_bsdf(h.n, wo, alb, rough, mat, a.k0, a.k1, pix, 0u, PURPOSE_BTH_DIR + 16u * i);
                sig = sig_mix(sig, s.word);
                const float p = s.valid ? sampler_pdf32(h.n, wo, s.wi, rough, mat) : 0.f;
                const U4 rx = philox(a.k0, a.k1, pix, 0u, 0u, PURPOSE_BTH_XI + 16u * i);
                uint32_t stop = u01(rx.x) > bth_continue_prob(p, a.N) ? 1u : 0u;
                if (i > 1 && __fmul_rn(spread, spread) > c_a0) stop |= 2u;
                if (i == a.D) stop |= 4u;
                sig = sig_mix(sig, stop);
                if (stop) {
                    write_record(recs + pix, h, d, Q, (uint32_t)prim, 1u | (mat << 1));
                    stop_at = i;
                    if constexpr (kNee) {
                        if (s.valid) {  // the BSDF technique of the direct light at the stopping vertex
                            float tq = 0.f;
                            const int q = tr.nearest(h.p, s.wi, tq);
                            sig = sig_mix(sig, q < 0 ? 0xFFFFFFFFu : (uint32_t)q);
                            if (q >= 0) {
                                const Hit hq = hit_info(tr.prims[q], h.p, s.wi, tq);
                                const float pb = bsdf_eval(h.n, wo, s.wi, alb, rough, mat).pdf;
                                const float3 e = weighted_emission<true>(tr, gp, lt, q, hq.front, s.wi, tq, pb);
                                le.x += beta.x * s.w.x * e.x;
                                le.y += beta.y * s.w.y * e.y;
                                le.z += beta.z * s.w.z * e.z;
                            }
                        }
                    }
                    break;
                }
                float pb = 0.f;
                if constexpr (kNee) pb = bsdf_eval(h.n, wo, s.wi, alb, rough, mat).pdf;
                beta.x *= s.w.x;
                beta.y *= s.w.y;
                beta.z *= s.w.z;
                o = h.p;
                d = s.wi;
                prim = tr.nearest(o, d, t);
                sig = sig_mix(sig, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
                if (prim < 0) break;
                h = hit_info(tr.prims[prim], o, d, t);
                const float3 e = weighted_emission<kNee>(tr, gp, lt, prim, h.front, d, t, pb);
                le.x += beta.x * e.x;
                le.y += beta.y * e.y;
                le.z += beta.z * e.z;
                spread = __fadd_rn(spread, spread_term(t, p, fabsf(sdot(h.n, d))));
            }
        }
        if (!stop_at) {
            float4* q = reinterpret_cast<float4*>(recs + pix);
            q[0] = q[1] = q[2] = q[3] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        base[pix].le = make_float4(le.x, le.y, le.z, 0.f);
        base[pix].wl = make_float4(0.f, 0.f, 0.f, 0.f);
        beta_out[pix] = make_float4(beta.x, beta.y, beta.z, 0.f);
        if (sig_out) sig_out[2 * (uint64_t)pix] = sig;
        if (count) count[pix] = 0;
    }
    if (a.rays) add_rays(a.rays, tr.rays);
}

// Training paths, organised like the residual pass: per path index the pixel
// pick, camera ray, record and first direction, then the path's segments;
// one ray per busy lane per iteration.
template <bool kNee>
__global__ void __launch_bounds__(kPtThreadsTrain, 1) k_gen_train(const SceneHeader* __restrict__ hd_g,
                                                          const Prim* __restrict__ gp, uint32_t n_prims, uint32_t W,
                                                          uint32_t H, uint64_t T, uint32_t k0, uint32_t k1,
                                                          uint32_t max_depth, nirc_record* __restrict__ recs,
                                                          float* __restrict__ dirs, float* __restrict__ targets,
                                                          unsigned long long* __restrict__ work, uint32_t env_mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SceneHeader hd;
    __shared__ uint32_t s_nlights;
    const Tracer tr = setup_scene(hd_g, gp, n_prims, smem_raw, &hd);
    Lights lt{nullptr, 0u};
    if constexpr (kNee)
        lt = collect_lights(gp, n_prims, reinterpret_cast<uint16_t*>(smem_raw + pt_geom_bytes(n_prims)), &s_nlights);
    float pb = 0.f;
    float3 first_emit = make_float3(0.f, 0.f, 0.f);
    const uint32_t P = W * H;
    uint32_t stage = kNeedPixel;
    uint32_t ti = 0, seg = 0;
    V3 o{0.f, 0.f, 0.f}, d{0.f, 0.f, 1.f};
    float3 beta = make_float3(0.f, 0.f, 0.f), L = beta;
    uint64_t sig = 0;
    while (true) {
        const bool need = stage == kNeedPixel;
        const uint64_t mine = fetch_work(work, need);
        if (need) {
            if (mine < T) {
                ti = (uint32_t)mine;
                const U4 r = philox(k0, k1, ti, 0u, 0u, PURPOSE_TRAIN_PICK);
                const uint32_t pix = __umulhi(r.x, P);
                camera_ray(hd, W, H, pix % W, pix / W, u01(r.y), u01(r.z), o, d);
                stage = kCameraRay;
            } else {
                stage = kNoMoreWork;
            }
        }
        if (__all_sync(0xffffffffu, stage == kNoMoreWork)) break;

        float t = 0.f;
        int prim = -1;
        if (stage == kCameraRay || stage == kResidRay) prim = tr.nearest(o, d, t);

        if (stage == kCameraRay) {
            float* dir = dirs + 3 * (uint64_t)ti;
            float* tg = targets + 3 * (uint64_t)ti;
            if (prim < 0) {
                float4* q = reinterpret_cast<float4*>(recs + ti);
                q[0] = q[1] = q[2] = q[3] = make_float4(0.f, 0.f, 0.f, 0.f);
                dir[0] = dir[1] = dir[2] = 0.f;
                tg[0] = tg[1] = tg[2] = 0.f;
                stage = kNeedPixel;
            } else {
                const Hit h = hit_info(tr.prims[prim], o, d, t);
                const Prim* Pp = gp + prim;
                const uint32_t mat = __ldg(&Pp->flags) & 3u;
                const float3 alb = make_float3(__ldg(&Pp->albedo[0]), __ldg(&Pp->albedo[1]), __ldg(&Pp->albedo[2]));
                const BsdfSample s =
                    sample_bsdf(h.n, sneg(d), alb, __ldg(&Pp->roughness), mat, k0, k1, ti, 0u, PURPOSE_RESID_DIR);
                write_record(recs + ti, h, d, Pp, (uint32_t)prim, (s.valid ? 1u : 0u) | (mat << 1));
                if (!s.valid) {
                    dir[0] = dir[1] = dir[2] = 0.f;
                    tg[0] = tg[1] = tg[2] = 0.f;
                    stage = kNeedPixel;
                } else {
                    dir[0] = s.wi.x;
                    dir[1] = s.wi.y;
                    dir[2] = s.wi.z;
                    o = h.p;
                    d = s.wi;
                    beta = make_float3(1.f, 1.f, 1.f);
                    L = make_float3(0.f, 0.f, 0.f);
                    seg = 1;
                    stage = kResidRay;
                }
            }
        } else if (stage == kResidRay) {
            bool end;
            if (env_mode) {  // light mode 2: one ray; target V L_env (1) or V (2, visibility cache)
                sig = sig_mix(sig, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
                L = make_float3(0.f, 0.f, 0.f);
                if (prim < 0) L = env_mode == 2 ? make_float3(1.f, 1.f, 1.f) : env_radiance(scene_env(hd, gp, n_prims), d);
                end = true;
            } else if constexpr (kNee)  // target = L_ind: the first hit's emission is direct light (discarded)
                end = path_segment_nee(tr, gp, lt, prim, t, o, d, beta, L, seg, max_depth, k0, k1, ti, 0u, sig, pb, 0u,
                                       first_emit, nullptr, 0, make_float3(0.f, 0.f, 0.f));
            else
                end = path_segment(tr, gp, prim, t, o, d, beta, L, seg, max_depth, k0, k1, ti, 0u, sig);
            if (end) {
                float* tg = targets + 3 * (uint64_t)ti;
                tg[0] = L.x;
                tg[1] = L.y;
                tg[2] = L.z;
                stage = kNeedPixel;
            }
        }
    }
}

static size_t pt_smem(uint32_t n_prims) {
    // geometry | hierarchy | light list (2 bytes per primitive)
    return pt_geom_bytes(n_prims) + (size_t)n_prims * 2 + 16;
}

template <typename K>
static cudaError_t persistent_grid(K kernel, int threads, size_t smem, uint64_t work, int num_sms, uint32_t* grid) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint64_t need = (work + threads - 1) / threads;
    uint64_t g = (uint64_t)per_sm * (uint64_t)num_sms;
    if (g > need) g = need;
    *grid = (uint32_t)(g < 1 ? 1 : g);
    return cudaSuccess;
}

template <bool kNee>
static cudaError_t launch_primary_resid_t(const nirc_handle* h, const SceneHeader* hd, const Prim* gp,
                                          const FrameArgs& a, uint64_t P, nirc_record* recs, PixelBase* base,
                                          ResidRow* rows, uint64_t* sig, uint32_t* count, const MvOut& mv,
                                          cudaStream_t st) {
    const size_t smem = pt_smem(a.n_prims);
    uint32_t grid = 1;
    cudaError_t e = persistent_grid(k_camera<kNee>, kPtThreads, smem, P, h->num_sms, &grid);
    if (e != cudaSuccess) return e;
    k_camera<kNee><<<grid, kPtThreads, smem, st>>>(hd, gp, a, recs, base, rows, sig, count, mv);
    count_kernels(h);
    e = cudaMemsetAsync(h->work_counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (mv.rec || a.env_mode) {  // the multi-vertex outputs or light mode 2: the instance with those paths
        e = persistent_grid(k_resid<kNee, true>, kPtThreads, smem, P, h->num_sms, &grid);
        if (e != cudaSuccess) return e;
        k_resid<kNee, true><<<grid, kPtThreads, smem, st>>>(hd, gp, a, recs, base, rows, sig, count, h->work_counter, mv);
    } else {
        e = persistent_grid(k_resid<kNee, false>, kPtThreads, smem, P, h->num_sms, &grid);
        if (e != cudaSuccess) return e;
        k_resid<kNee, false><<<grid, kPtThreads, smem, st>>>(hd, gp, a, recs, base, rows, sig, count, h->work_counter, mv);
    }
    count_kernels(h);
    return cudaGetLastError();
}

cudaError_t launch_primary_resid(const nirc_handle* h, const void* scene, const nirc_frame_desc& fd,
                                 nirc_record* recs, PixelBase* base, ResidRow* rows, uint64_t* sig, uint32_t* count,
                                 cudaStream_t st, nirc_record* mv_rec, float4* mv_beta, ResidRow* mv_row,
                                 unsigned long long* rays) {
    FrameArgs a{fd.width, fd.height, fd.n_cache,  fd.n_resid, fd.max_depth,
                fd.n_prims, (uint32_t)fd.seed, fd.frame, fd.light_mode == 2 ? 1u : 0u, rays};
    const uint64_t P = (uint64_t)fd.width * fd.height;
    const MvOut mv{mv_rec, mv_beta, mv_row, P * fd.n_resid};
    const auto* hd = reinterpret_cast<const SceneHeader*>(scene);
    const auto* gp = reinterpret_cast<const Prim*>(reinterpret_cast<const char*>(scene) + sizeof(SceneHeader));
    if (fd.light_mode == 1)
        return launch_primary_resid_t<true>(h, hd, gp, a, P, recs, base, rows, sig, count, mv, st);
    return launch_primary_resid_t<false>(h, hd, gp, a, P, recs, base, rows, sig, count, mv, st);
}

template <bool kNee>
static cudaError_t launch_primary_resid_batch_t(const FrameJob* fj, uint32_t n, cudaStream_t st) {
    const nirc_handle* h0 = fj[0].h;
    uint32_t max_prims = 0;
    uint64_t work_total = 0;
    for (uint32_t i = 0; i < n; ++i) {
        max_prims = max_prims > fj[i].fd.n_prims ? max_prims : fj[i].fd.n_prims;
        work_total += (uint64_t)fj[i].fd.width * fj[i].fd.height * (1u + fj[i].fd.n_resid);
    }
    const size_t smem = pt_smem(max_prims);
    cudaError_t e = cudaFuncSetAttribute(k_camera_batch<kNee>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_resid_batch<kNee>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, per_sm_r = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_camera_batch<kNee>, kPtThreads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_r, k_resid_batch<kNee>, kPtThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = per_sm < per_sm_r ? per_sm : per_sm_r;
    const uint64_t grid_max = (uint64_t)(per_sm < 1 ? 1 : per_sm) * (uint64_t)h0->num_sms;
    if (grid_max < n) return cudaErrorInvalidConfiguration;
    // CTAs in proportion to each frame's rays (camera + residual paths), at least one
    // each and no more than one per CTA-width of pixels
    PtJobs jobs;
    jobs.n = n;
    uint32_t cta = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const FrameJob& f = fj[i];
        const uint64_t P = (uint64_t)f.fd.width * f.fd.height;
        uint64_t share = P * (1u + f.fd.n_resid) * (grid_max - n) / work_total + 1;  // the shares add up to <= grid_max
        const uint64_t useful = (P + kPtThreads - 1) / kPtThreads;
        if (share > useful) share = useful;
        PtJob& j = jobs.j[i];
        j.hd = reinterpret_cast<const SceneHeader*>(f.scene);
        j.gp = reinterpret_cast<const Prim*>(reinterpret_cast<const char*>(f.scene) + sizeof(SceneHeader));
        j.a = FrameArgs{f.fd.width, f.fd.height, f.fd.n_cache, f.fd.n_resid, f.fd.max_depth, f.fd.n_prims,
                        (uint32_t)f.fd.seed, f.fd.frame, 0u, nullptr};
        j.recs = f.recs;
        j.base = f.base;
        j.rows = f.rows;
        j.work = f.work;
        j.cta0 = cta;
        j.n_cta = (uint32_t)share;
        cta += (uint32_t)share;
        count_kernels(f.h, 2);  // its share of the two launches
    }
    k_camera_batch<kNee><<<cta, kPtThreads, smem, st>>>(jobs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_resid_batch<kNee><<<cta, kPtThreads, smem, st>>>(jobs);
    return cudaGetLastError();
}

cudaError_t launch_primary_resid_batch(const FrameJob* fj, uint32_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (n > kMaxFrameJobs) return cudaErrorInvalidValue;
    for (uint32_t i = 1; i < n; ++i)
        if (fj[i].fd.light_mode != fj[0].fd.light_mode) return cudaErrorInvalidValue;
    if (fj[0].fd.light_mode == 1) return launch_primary_resid_batch_t<true>(fj, n, st);
    if (fj[0].fd.light_mode == 0) return launch_primary_resid_batch_t<false>(fj, n, st);
    return cudaErrorInvalidValue;
}

template <bool kNee>
static cudaError_t launch_primary_bth_t(const nirc_handle* h, const SceneHeader* hd, const Prim* gp,
                                        const FrameArgs& a, uint64_t P, nirc_record* recs, PixelBase* base,
                                        float4* beta, uint64_t* sig, uint32_t* count, cudaStream_t st) {
    const size_t smem = pt_smem(a.n_prims);
    uint32_t grid = 1;
    cudaError_t e = persistent_grid(k_primary_bth<kNee>, kPtThreadsBth, smem, P, h->num_sms, &grid);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(h->work_counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_primary_bth<kNee><<<grid, kPtThreadsBth, smem, st>>>(hd, gp, a, recs, base, beta, sig, count, h->work_counter);
    count_kernels(h);
    return cudaGetLastError();
}

cudaError_t launch_primary_bth(const nirc_handle* h, const void* scene, const nirc_frame_desc& fd, nirc_record* recs,
                               PixelBase* base, float4* beta, uint64_t* sig, uint32_t* count, cudaStream_t st,
                               unsigned long long* rays) {
    FrameArgs a{fd.width, fd.height, fd.n_cache, fd.n_resid, fd.max_depth, fd.n_prims, (uint32_t)fd.seed, fd.frame, 0u,
                rays};
    const uint64_t P = (uint64_t)fd.width * fd.height;
    const auto* hd = reinterpret_cast<const SceneHeader*>(scene);
    const auto* gp = reinterpret_cast<const Prim*>(reinterpret_cast<const char*>(scene) + sizeof(SceneHeader));
    if (fd.light_mode == 1) return launch_primary_bth_t<true>(h, hd, gp, a, P, recs, base, beta, sig, count, st);
    return launch_primary_bth_t<false>(h, hd, gp, a, P, recs, base, beta, sig, count, st);
}

template <bool kNee>
static cudaError_t launch_gen_train_t(const nirc_handle* h, const SceneHeader* hd, const Prim* gp, uint32_t n_prims,
                                      uint32_t W, uint32_t H, uint64_t T, uint32_t frame, uint64_t seed,
                                      uint32_t max_depth, nirc_record* recs, float* dirs, float* targets,
                                      uint32_t env_mode, cudaStream_t st) {
    const size_t smem = pt_smem(n_prims);
    uint32_t grid = 1;
    cudaError_t e = persistent_grid(k_gen_train<kNee>, kPtThreadsTrain, smem, T, h->num_sms, &grid);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(h->work_counter + 1, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_gen_train<kNee><<<grid, kPtThreadsTrain, smem, st>>>(hd, gp, n_prims, W, H, T, (uint32_t)seed, frame ^ kTrainKeyBit,
                                                      max_depth, recs, dirs, targets, h->work_counter + 1,
                                                      env_mode);
    count_kernels(h);
    return cudaGetLastError();
}

cudaError_t launch_gen_train(const nirc_handle* h, const void* scene, uint32_t n_prims, uint32_t W, uint32_t H,
                             uint64_t T, uint32_t frame, uint64_t seed, uint32_t max_depth, uint32_t light_mode,
                             nirc_record* recs, float* dirs, float* targets, cudaStream_t st) {
    const auto* hd = reinterpret_cast<const SceneHeader*>(scene);
    const auto* gp = reinterpret_cast<const Prim*>(reinterpret_cast<const char*>(scene) + sizeof(SceneHeader));
    if (light_mode == 1)
        return launch_gen_train_t<true>(h, hd, gp, n_prims, W, H, T, frame, seed, max_depth, recs, dirs, targets, 0u,
                                        st);
    const uint32_t env_mode = light_mode == 2 ? (h->shape.vis ? 2u : 1u) : 0u;
    return launch_gen_train_t<false>(h, hd, gp, n_prims, W, H, T, frame, seed, max_depth, recs, dirs, targets,
                                     env_mode, st);
}

}  // namespace nirc
