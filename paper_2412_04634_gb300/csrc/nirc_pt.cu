// nirc_pt.cu -- path-tracing kernels of the two-level estimator.
//
// k_primary_resid: per pixel, the camera ray (1 spp, Philox jitter), the
//   shading record of the first hit (paper: surface parameter buffer), and
//   the residual level's M BSDF-sampled directions with their path-traced
//   incident radiance L_j (eq. L_r, the L_i term), Russian roulette with
//   termination probability 0.1 (paper: section "Results", implementation
//   paragraph).  Lanes regenerate work: one ray per busy lane per iteration,
//   new pixels from a work counter as old ones finish.
// k_gen_train: the separate training pass (section "Cache application"):
//   T paths from uniformly drawn pixels, one record per path, organised the
//   same way.
//
// Both kernels are persistent: each CTA stages the primitives' geometry in
// shared memory and, for scenes of more than 16 primitives, builds its own
// bounding-volume hierarchy there once, then loops over pixels (paths).
#include "nirc_bvh.cuh"
#include "nirc_internal.h"

namespace nirc {

constexpr int kPtThreads = 128;
constexpr uint32_t kBvhMinPrims = 17;

struct FrameArgs {
    uint32_t W, H, N, M, D, n_prims;
    uint32_t k0, k1;
};

// Nearest-hit queries over the CTA's primitives (brute force or hierarchy).
struct Tracer {
    const PrimGeom* prims;
    uint32_t n;
    Bvh tree;
    bool bvh;
    __device__ __forceinline__ int nearest(V3 o, V3 d, float& t) const {
        return bvh ? bvh_nearest(tree, prims, n, o, d, t) : trace_nearest(prims, n, o, d, t);
    }
};

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
    tr.tree = Bvh{nullptr, nullptr, nullptr, 0u, 0u, 0u};
    tr.bvh = n_prims >= kBvhMinPrims;
    if (tr.bvh) {
        tr.tree = bvh_build(sp, n_prims, smem + (size_t)n_prims * sizeof(PrimGeom));
        __syncthreads();
    }
    return tr;
}

// One segment of a path (residual or training) after its ray was traced:
// emission of the hit, then Russian roulette and the next BSDF direction.
// Counters (c0, c1) identify the path, `seg` its segment (1-based).  Returns
// true when the path ends; otherwise (o, d) is the next ray and seg + 1.
__device__ __forceinline__ bool path_segment(const Tracer& tr, const Prim* __restrict__ gp, int prim, float t, V3& o,
                                             V3& d, float3& beta, float3& L, uint32_t& seg, uint32_t max_depth,
                                             uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint64_t& sig) {
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

__device__ __forceinline__ void write_record(nirc_record* dst, const Hit& h, V3 d, const Prim* P, uint32_t prim,
                                             uint32_t flags) {
    float4* q = reinterpret_cast<float4*>(dst);
    q[0] = make_float4(h.p.x, h.p.y, h.p.z, h.n.x);
    q[1] = make_float4(h.n.y, h.n.z, -d.x, -d.y);
    q[2] = make_float4(-d.z, __ldg(&P->albedo[0]), __ldg(&P->albedo[1]), __ldg(&P->albedo[2]));
    q[3] = make_float4(__ldg(&P->roughness), __uint_as_float(prim), __uint_as_float(flags), 0.f);
}

// Lane state of k_primary_resid: which pixel, which ray is in flight.
enum : uint32_t { kNeedPixel = 0, kCameraRay = 1, kResidRay = 2, kNoMoreWork = 3 };

// Per pixel: the camera ray, the shading record, then for j = 0..M-1 a
// residual direction and its path (eq. L_r's L_j), exactly in the order and
// with the Philox counters of a sequential loop.  The loop is organised as a
// per-lane state machine so that every iteration traces one ray per busy
// lane: a lane whose pixel is done takes the next pixel from a work counter
// (one atomic per warp), so lanes do not idle while others finish long paths.
__global__ void __launch_bounds__(kPtThreads) k_primary_resid(const SceneHeader* __restrict__ hd_g,
                                                              const Prim* __restrict__ gp, FrameArgs a,
                                                              nirc_record* __restrict__ recs,
                                                              PixelBase* __restrict__ base,
                                                              ResidRow* __restrict__ rows,
                                                              uint64_t* __restrict__ sig_out,
                                                              uint32_t* __restrict__ count,
                                                              unsigned long long* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SceneHeader hd;
    const Tracer tr = setup_scene(hd_g, gp, a.n_prims, smem_raw, &hd);

    const uint64_t P = (uint64_t)a.W * a.H;
    uint32_t stage = kNeedPixel;
    uint32_t pix = 0, j = 0, seg = 0, nvalid = 0;
    V3 o{0.f, 0.f, 0.f}, d{0.f, 0.f, 1.f};
    V3 sp{0.f, 0.f, 0.f}, sn{0.f, 0.f, 1.f}, swo{0.f, 0.f, 1.f};  // shading point, normal, wo
    float3 salb = make_float3(0.f, 0.f, 0.f), le = salb, wl = salb, L = salb, beta = salb, sw = salb;
    float srough = 1.f;
    uint32_t smat = 0;
    uint64_t sig = kSigInit;

    // Next residual sample of the current pixel: the first valid one becomes
    // the ray in flight; with none left the pixel's outputs are written.
    auto next_residual = [&]() -> uint32_t {
        ResidRow* my_rows = rows + (uint64_t)pix * a.M;
        for (; j < a.M; ++j) {
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
            if (mine < P) {
                pix = (uint32_t)mine;
                const U4 r = philox(a.k0, a.k1, pix, 0u, 0u, PURPOSE_CAMERA);
                camera_ray(hd, a.W, a.H, pix % a.W, pix / a.W, u01(r.x), u01(r.y), o, d);
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
            sig = sig_mix(kSigInit, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
            if (prim < 0) {
                float4* q = reinterpret_cast<float4*>(recs + pix);
                q[0] = q[1] = q[2] = q[3] = make_float4(0.f, 0.f, 0.f, 0.f);
                base[pix].le = make_float4(0.f, 0.f, 0.f, 0.f);
                base[pix].wl = make_float4(0.f, 0.f, 0.f, 0.f);
                ResidRow* my_rows = rows + (uint64_t)pix * a.M;
                for (uint32_t jj = 0; jj < a.M; ++jj) {
                    my_rows[jj].wi = make_float4(0.f, 0.f, 1.f, 0.f);
                    my_rows[jj].w = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                if (sig_out) sig_out[2 * (uint64_t)pix] = sig;
                if (count) count[pix] = 0;
                stage = kNeedPixel;
            } else {
                const Hit h = hit_info(tr.prims[prim], o, d, t);
                const Prim* Pp = gp + prim;
                const uint32_t pflags = __ldg(&Pp->flags);
                smat = pflags & 3u;
                write_record(recs + pix, h, d, Pp, (uint32_t)prim, 1u | (smat << 1));
                le = make_float3(0.f, 0.f, 0.f);
                if (h.front || (pflags & EMIT_TWO_SIDED))
                    le = make_float3(__ldg(&Pp->emission[0]), __ldg(&Pp->emission[1]), __ldg(&Pp->emission[2]));
                salb = make_float3(__ldg(&Pp->albedo[0]), __ldg(&Pp->albedo[1]), __ldg(&Pp->albedo[2]));
                srough = __ldg(&Pp->roughness);
                sp = h.p;
                sn = h.n;
                swo = sneg(d);
                wl = make_float3(0.f, 0.f, 0.f);
                nvalid = 0;
                j = 0;
                stage = next_residual();
            }
        } else if (stage == kResidRay) {
            const bool end = path_segment(tr, gp, prim, t, o, d, beta, L, seg, a.D, a.k0, a.k1, pix, j, sig);
            if (end) {
                wl.x += sw.x * L.x;
                wl.y += sw.y * L.y;
                wl.z += sw.z * L.z;
                ++nvalid;
                ++j;
                stage = next_residual();
            }
        }
    }
}

// Training paths, organised like k_primary_resid: per path index the pixel
// pick, camera ray, record and first direction, then the path's segments;
// one ray per busy lane per iteration.
__global__ void __launch_bounds__(kPtThreads) k_gen_train(const SceneHeader* __restrict__ hd_g,
                                                          const Prim* __restrict__ gp, uint32_t n_prims, uint32_t W,
                                                          uint32_t H, uint64_t T, uint32_t k0, uint32_t k1,
                                                          uint32_t max_depth, nirc_record* __restrict__ recs,
                                                          float* __restrict__ dirs, float* __restrict__ targets,
                                                          unsigned long long* __restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SceneHeader hd;
    const Tracer tr = setup_scene(hd_g, gp, n_prims, smem_raw, &hd);
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
            if (path_segment(tr, gp, prim, t, o, d, beta, L, seg, max_depth, k0, k1, ti, 0u, sig)) {
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
    return (size_t)n_prims * sizeof(PrimGeom) + (n_prims >= kBvhMinPrims ? bvh_smem_bytes(n_prims) : 0);
}

template <typename K>
static cudaError_t persistent_grid(K kernel, size_t smem, uint64_t work, int num_sms, uint32_t* grid) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPtThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint64_t need = (work + kPtThreads - 1) / kPtThreads;
    uint64_t g = (uint64_t)per_sm * (uint64_t)num_sms;
    if (g > need) g = need;
    *grid = (uint32_t)(g < 1 ? 1 : g);
    return cudaSuccess;
}

cudaError_t launch_primary_resid(const nirc_handle* h, const void* scene, const nirc_frame_desc& fd,
                                 nirc_record* recs, PixelBase* base, ResidRow* rows, uint64_t* sig, uint32_t* count,
                                 cudaStream_t st) {
    FrameArgs a{fd.width, fd.height, fd.n_cache, fd.n_resid, fd.max_depth, fd.n_prims, (uint32_t)fd.seed, fd.frame};
    const uint64_t P = (uint64_t)fd.width * fd.height;
    const size_t smem = pt_smem(fd.n_prims);
    const auto* hd = reinterpret_cast<const SceneHeader*>(scene);
    const auto* gp = reinterpret_cast<const Prim*>(reinterpret_cast<const char*>(scene) + sizeof(SceneHeader));
    uint32_t grid = 1;
    cudaError_t e = persistent_grid(k_primary_resid, smem, P, h->num_sms, &grid);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(h->work_counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_primary_resid<<<grid, kPtThreads, smem, st>>>(hd, gp, a, recs, base, rows, sig, count, h->work_counter);
    return cudaGetLastError();
}

cudaError_t launch_gen_train(const nirc_handle* h, const void* scene, uint32_t n_prims, uint32_t W, uint32_t H,
                             uint64_t T, uint32_t frame, uint64_t seed, uint32_t max_depth, nirc_record* recs,
                             float* dirs, float* targets, cudaStream_t st) {
    const size_t smem = pt_smem(n_prims);
    const auto* hd = reinterpret_cast<const SceneHeader*>(scene);
    const auto* gp = reinterpret_cast<const Prim*>(reinterpret_cast<const char*>(scene) + sizeof(SceneHeader));
    uint32_t grid = 1;
    cudaError_t e = persistent_grid(k_gen_train, smem, T, h->num_sms, &grid);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(h->work_counter + 1, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_gen_train<<<grid, kPtThreads, smem, st>>>(hd, gp, n_prims, W, H, T, (uint32_t)seed, frame ^ kTrainKeyBit,
                                                max_depth, recs, dirs, targets, h->work_counter + 1);
    return cudaGetLastError();
}

}  // namespace nirc
