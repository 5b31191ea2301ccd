// nirc_capi.cu -- the extern "C" boundary of libnirc.so (declared in nirc.h).
//
// Validates arguments, owns device state of a cache handle, sizes scratch,
// and enqueues the kernels on the caller's stream.  Every entry point
// returns a status; failures record a thread-local message.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "nirc_internal.h"

namespace nirc {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

nirc_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return NIRC_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? NIRC_ERR_OOM : NIRC_ERR_CUDA;
}

NetShape make_shape(const nirc_config& cfg) {
    NetShape s{};
    s.hashgrid = cfg.pos_encoding == NIRC_POS_HASHGRID;
    s.levels = s.hashgrid ? cfg.hash_levels : 0;
    s.log2_table = cfg.log2_table;
    s.n_pos = s.hashgrid ? cfg.hash_levels * cfg.feats_per_level : 3 * 2 * cfg.freq_octaves;
    s.sh = cfg.input_encoding == NIRC_INPUT_SH ? 1u : 0u;
    s.vis = cfg.output == NIRC_OUT_VISIBILITY ? 1u : 0u;
    s.n_dir = s.sh ? kShFeatures : kDirFeatures;
    s.n_surf = s.sh ? kPhiFeatures : kNrmFeatures;
    s.n_in = s.n_pos + s.n_dir + s.n_surf;
    s.n_pix = s.n_pos + s.n_surf;
    s.hidden = cfg.hidden_layers;
    s.n_mlp = (uint64_t)kWidth * s.n_in + kWidth + (uint64_t)(s.hidden - 1) * (kWidth * kWidth + kWidth) +
              3ull * kWidth + 3;
    s.n_hash = s.hashgrid ? (uint64_t)cfg.hash_levels * (1ull << cfg.log2_table) * cfg.feats_per_level : 0;
    s.hash_off = (s.n_mlp + 3) & ~3ull;
    s.n_dev = s.hash_off + s.n_hash;
    s.off_wpix = 0;
    s.off_wdir = s.n_pix * kWidth;
    s.off_b0 = s.off_wdir + s.n_dir * kWidth;
    s.off_hidden = s.off_b0 + kWidth;
    s.off_out = s.off_hidden + (s.hidden - 1) * (kWidth * kWidth + kWidth);
    s.packed_floats = s.off_out + 4 * kWidth + 4;
    return s;
}

GridParams make_grid(const nirc_config& cfg) {
    GridParams g{};
    if (cfg.pos_encoding != NIRC_POS_HASHGRID) return g;
    g.n_levels = cfg.hash_levels;
    const uint64_t T = 1ull << cfg.log2_table;
    g.mask = (uint32_t)(T - 1);
    for (uint32_t l = 0; l < cfg.hash_levels; ++l) {
        const uint32_t res = (uint32_t)std::floor((double)cfg.base_res * std::pow((double)cfg.growth, (double)l));
        const uint64_t side = (uint64_t)res + 1;
        g.level[l].res = res;
        g.level[l].dense = side * side * side <= T ? 1u : 0u;
        g.level[l].fres = (float)res;
        g.level[l].pad = 0;
    }
    return g;
}

static nirc_status check_config(const nirc_config* c) {
    if (!c) {
        set_error("config is NULL");
        return NIRC_ERR_INVALID;
    }
    if (c->width != kWidth) {
        set_error("width %u unsupported (only 64)", c->width);
        return NIRC_ERR_UNSUPPORTED;
    }
    if (c->hidden_layers < 1 || c->hidden_layers > kMaxHidden) {
        set_error("hidden_layers %u outside 1..%u", c->hidden_layers, kMaxHidden);
        return NIRC_ERR_UNSUPPORTED;
    }
    if (c->freq_octaves != 4) {
        set_error("freq_octaves %u unsupported (only 4)", c->freq_octaves);
        return NIRC_ERR_UNSUPPORTED;
    }
    if (c->pos_encoding == NIRC_POS_HASHGRID) {
        if (c->feats_per_level != 2 || c->hash_levels < 1 || c->hash_levels > kMaxLevels || c->log2_table < 4 ||
            c->log2_table > 24 || c->base_res < 1 || !(c->growth >= 1.0f) ||
            std::floor((double)c->base_res * std::pow((double)c->growth, (double)(c->hash_levels - 1))) > 1e7) {
            set_error("hash grid configuration unsupported (2 features, 1..16 levels, log2_table 4..24)");
            return NIRC_ERR_UNSUPPORTED;
        }
    } else if (c->pos_encoding != NIRC_POS_FREQ) {
        set_error("pos_encoding %u unknown", c->pos_encoding);
        return NIRC_ERR_INVALID;
    }
    if (c->input_encoding > NIRC_INPUT_SH) {
        set_error("input_encoding %u unknown", c->input_encoding);
        return NIRC_ERR_INVALID;
    }
    if (c->output > NIRC_OUT_VISIBILITY) {
        set_error("output %u unknown", c->output);
        return NIRC_ERR_INVALID;
    }
    {
        const uint32_t n_pos = c->pos_encoding == NIRC_POS_HASHGRID ? c->hash_levels * 2 : 24;
        if (n_pos + (c->input_encoding == NIRC_INPUT_SH ? kPhiFeatures : kNrmFeatures) > kWidth) {
            set_error("too many per-surface features (position + surface features must fit in 64)");
            return NIRC_ERR_UNSUPPORTED;
        }
    }
    if (c->precision > NIRC_FP8_E4M3_TC) {
        set_error("precision %u unknown", c->precision);
        return NIRC_ERR_INVALID;
    }
    return NIRC_OK;
}

static nirc_status ensure(void** buf, size_t* cap, size_t bytes, const char* what) {
    if (*cap >= bytes) return NIRC_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) {
        *buf = nullptr;
        cudaGetLastError();
        set_error("cannot allocate %zu bytes of %s scratch: %s", bytes, what, cudaGetErrorString(e));
        return NIRC_ERR_BUDGET;
    }
    *cap = bytes;
    return NIRC_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

constexpr int kMaxPending = 2048;

static void resolve_pending(nirc_handle* h) {
    for (int i = 0; i < h->n_pending; ++i) {
        const auto& p = h->pending[i];
        float ms = 0.f;
        if (cudaEventSynchronize(p.stop) == cudaSuccess && cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            h->timing_ms[p.cls] += ms;
            h->timing_launches[p.cls] += p.kernels;
        }
    }
    h->n_pending = 0;
}

void timer_begin(const nirc_handle* hc, int cls, cudaStream_t st) {
    auto* h = const_cast<nirc_handle*>(hc);
    if (!h->timing || !h->pending) return;
    if (h->n_pending >= kMaxPending) resolve_pending(h);
    auto& p = h->pending[h->n_pending];
    p.cls = cls;
    p.k0 = h->n_kernels;
    p.start = h->event_pool[2 * h->n_pending];
    p.stop = h->event_pool[2 * h->n_pending + 1];
    cudaEventRecord(p.start, st);
}

void timer_end(const nirc_handle* hc, int cls, cudaStream_t st) {
    (void)cls;
    auto* h = const_cast<nirc_handle*>(hc);
    if (!h->timing || !h->pending) return;
    auto& p = h->pending[h->n_pending];
    cudaEventRecord(p.stop, st);
    p.kernels = h->n_kernels - p.k0;
    h->n_pending += 1;
}

static size_t round256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

// Later-vertex data of the multi-vertex estimator, per residual path (unit)
// and vertex: record, throughput, continuation row; and per unit the two
// vertex passes' outputs.
static size_t mv_bytes(uint64_t PM) {
    return round256(2 * PM * sizeof(nirc_record)) + round256(2 * PM * sizeof(float4)) +
           round256(2 * PM * sizeof(ResidRow)) + 2 * round256(PM * sizeof(float4));
}

size_t frame_scratch_bytes(uint64_t P, uint32_t M, uint32_t estimator) {
    // records | per-pixel bases | residual rows (two-level) or path throughputs (biased) | later vertices
    const size_t third = estimator == NIRC_EST_BIASED_BTH ? P * sizeof(float4) : P * M * sizeof(ResidRow);
    return round256(P * sizeof(nirc_record)) + round256(P * sizeof(PixelBase)) + round256(third) +
           (estimator == NIRC_EST_MULTI_VERTEX ? mv_bytes(P * M) : 0);
}

nirc_status check_frame_args(const char* who, const void* scene, const nirc_frame_desc& fd, const float* out,
                             const nirc_frame_aux* aux) {
    const uint64_t P = (uint64_t)fd.width * fd.height;
    if (!scene || (!out && fd.phase != NIRC_PHASE_TRACE) || !aligned16(scene) || (out && !aligned16(out)) ||
        fd.phase > NIRC_PHASE_CACHE) {
        set_error("%s: NULL or misaligned scene/output pointer, or phase > 2", who);
        return NIRC_ERR_INVALID;
    }
    if (fd.n_prims < 1 || fd.n_prims > NIRC_MAX_PRIMS || fd.n_cache > 1024 || fd.n_resid > 64 || fd.max_depth < 1 ||
        fd.max_depth > 64 || fd.cache_mode > 2 || fd.light_mode > 2 || P > 0xFFFFFFFFull ||
        (fd.light_mode == 2 && fd.estimator != NIRC_EST_TWO_LEVEL) ||
        fd.estimator > NIRC_EST_MULTI_VERTEX || (fd.estimator == NIRC_EST_BIASED_BTH && fd.n_resid != 0) ||
        (fd.estimator == NIRC_EST_MULTI_VERTEX &&
         (fd.n_cache2 > 1024 || fd.n_cache3 > 1024 || P * fd.n_resid > 0xFFFFFFFFull))) {
        set_error("%s: argument out of range (n_prims 1..%u, N, N2, N3 <= 1024, M <= 64, depth 1..64, "
                  "light_mode 0..2, estimator 0..2, M = 0 for the biased estimator, light mode 2 two-level only)",
                  who, NIRC_MAX_PRIMS);
        return NIRC_ERR_INVALID;
    }
    if (aux && ((aux->lc && ((uintptr_t)aux->lc & 3u)) || (aux->lr && ((uintptr_t)aux->lr & 3u)) ||
                (aux->sig && ((uintptr_t)aux->sig & 7u)) || (aux->count && ((uintptr_t)aux->count & 3u)) ||
                (aux->row_n && ((uintptr_t)aux->row_n & 3u)) || (aux->rays && ((uintptr_t)aux->rays & 7u)))) {
        set_error("%s: misaligned aux pointer", who);
        return NIRC_ERR_INVALID;
    }
    return NIRC_OK;
}

nirc_status enqueue_frame(const char* who, const nirc_handle* h, const void* scene, const nirc_frame_desc& fd,
                          float* out, const nirc_frame_aux* aux, void* scratch, cudaStream_t st) {
    const uint64_t P = (uint64_t)fd.width * fd.height;
    char* sp = reinterpret_cast<char*>(scratch);
    const size_t rec_bytes = round256(P * sizeof(nirc_record));
    const size_t base_bytes = round256(P * sizeof(PixelBase));
    // The path-tracing kernel writes every record, base and residual row that
    // the cache kernel reads, so no part of the scratch has to start at zero.
    nirc_record* recs = reinterpret_cast<nirc_record*>(sp);
    PixelBase* base = reinterpret_cast<PixelBase*>(sp + rec_bytes);
    const bool biased = fd.estimator == NIRC_EST_BIASED_BTH;
    ResidRow* rows = biased ? nullptr : reinterpret_cast<ResidRow*>(sp + rec_bytes + base_bytes);
    float4* beta = biased ? reinterpret_cast<float4*>(sp + rec_bytes + base_bytes) : nullptr;
    uint64_t* sig = aux ? aux->sig : nullptr;
    uint32_t* count = aux ? aux->count : nullptr;
    // multi-vertex estimator: later-vertex data after the residual rows
    const bool multi = fd.estimator == NIRC_EST_MULTI_VERTEX && fd.n_resid > 0 && (fd.n_cache2 || fd.n_cache3);
    const uint64_t PM = P * fd.n_resid;
    nirc_record* mv_rec = nullptr;
    float4 *mv_beta = nullptr, *mv_out = nullptr;
    ResidRow* mv_row = nullptr;
    if (multi) {
        char* q = sp + rec_bytes + base_bytes + round256(PM * sizeof(ResidRow));
        mv_rec = reinterpret_cast<nirc_record*>(q);
        q += round256(2 * PM * sizeof(nirc_record));
        mv_beta = reinterpret_cast<float4*>(q);
        q += round256(2 * PM * sizeof(float4));
        mv_row = reinterpret_cast<ResidRow*>(q);
        q += round256(2 * PM * sizeof(ResidRow));
        mv_out = reinterpret_cast<float4*>(q);  // [2][PM], each part round256
    }
    cudaError_t e = cudaSuccess;
    if (fd.phase != NIRC_PHASE_CACHE) {
        timer_begin(h, NIRC_K_PATH_TRACE, st);
        unsigned long long* rays = aux ? reinterpret_cast<unsigned long long*>(aux->rays) : nullptr;
        e = biased ? launch_primary_bth(h, scene, fd, recs, base, beta, sig, count, st, rays)
                   : launch_primary_resid(h, scene, fd, recs, base, rows, sig, count, st, mv_rec, mv_beta, mv_row,
                                          rays);
        timer_end(h, NIRC_K_PATH_TRACE, st);
        if (e != cudaSuccess) {
            set_error("%s (path tracing): %s", who, cudaGetErrorString(e));
            return NIRC_ERR_CUDA;
        }
        if (fd.phase == NIRC_PHASE_TRACE) return NIRC_OK;
    }
    timer_begin(h, NIRC_K_CACHE, st);
    const bool tc = tc_supported(h, fd);
    EnvSource env;  // light mode 2 with a visibility cache: n = V L_env
    if (fd.light_mode == 2 && h->shape.vis) {
        env.scene = scene;
        env.n_prims = fd.n_prims;
    }
    if (tc) {
        e = launch_cache_tc(h, fd, recs, base, rows, beta, out, aux ? aux->lc : nullptr, aux ? aux->lr : nullptr, sig,
                            count, aux ? aux->row_n : nullptr, h->dev_err, st, CachePass{}, env);
    } else {
        e = launch_cache_simt(h, fd, recs, base, rows, beta, out, aux ? aux->lc : nullptr, aux ? aux->lr : nullptr, sig,
                              count, aux ? aux->row_n : nullptr, st, CachePass{}, env);
    }
    bool tc_any = tc;
    if (multi && e == cudaSuccess) {
        // vertices 2 and 3 of every residual path: one cache pass each over the
        // P M units (N_k cache rows + the continuation row), then the sums
        const size_t part = round256(PM * sizeof(float4)) / sizeof(float4);
        float4* outs[2] = {nullptr, nullptr};
        for (uint32_t k = 2; k <= 3 && e == cudaSuccess; ++k) {
            const uint32_t nk = k == 2 ? fd.n_cache2 : fd.n_cache3;
            if (!nk) continue;
            nirc_frame_desc dk = fd;
            dk.width = (uint32_t)PM;
            dk.height = 1;
            dk.n_cache = nk;
            dk.n_resid = 1;
            dk.estimator = NIRC_EST_TWO_LEVEL;
            const uint64_t off = (uint64_t)(k - 2) * PM;
            float4* ok = mv_out + (k - 2) * part;
            const CachePass pass{fd.n_resid, PURPOSE_VCACHE + 16u * k};
            const bool tck = tc_supported(h, dk);
            tc_any = tc_any || tck;
            if (tck)
                e = launch_cache_tc(h, dk, mv_rec + off, nullptr, mv_row + off, mv_beta + off,
                                    reinterpret_cast<float*>(ok), nullptr, nullptr, nullptr, nullptr, nullptr,
                                    h->dev_err, st, pass);
            else
                e = launch_cache_simt(h, dk, mv_rec + off, nullptr, mv_row + off, mv_beta + off,
                                      reinterpret_cast<float*>(ok), nullptr, nullptr, nullptr, nullptr, nullptr, st,
                                      pass);
            outs[k - 2] = ok;
        }
        if (e == cudaSuccess) {
            e = launch_mv_accumulate(out, aux ? aux->lr : nullptr, outs[0], outs[1], P, fd.n_resid, st);
            count_kernels(h);
        }
    }
    timer_end(h, NIRC_K_CACHE, st);
    if (e == cudaSuccess && tc_any)
        e = cudaMemcpyAsync(h->host_err, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
        set_error("%s (cache integral): %s", who, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? NIRC_ERR_OOM : NIRC_ERR_CUDA;
    }
    return NIRC_OK;
}

nirc_status reserve_train_scratch(nirc_handle* h, uint64_t n) {
    return ensure(&h->train_scratch, &h->train_scratch_bytes, train_scratch_bytes(h, n), "training");
}

}  // namespace nirc

using namespace nirc;

extern "C" {

const char* nirc_last_error(void) { return g_err; }

nirc_status nirc_timing_enable(nirc_handle* h, int enable) {
    if (!h) {
        set_error("nirc_timing_enable: handle is NULL");
        return NIRC_ERR_INVALID;
    }
    if (enable && !h->pending) {
        h->pending = new (std::nothrow) nirc_handle::Pending[kMaxPending];
        h->event_pool = new (std::nothrow) cudaEvent_t[2 * kMaxPending];
        if (!h->pending || !h->event_pool) {
            set_error("nirc_timing_enable: host allocation failed");
            return NIRC_ERR_OOM;
        }
        for (int i = 0; i < 2 * kMaxPending; ++i) {
            cudaError_t e = cudaEventCreate(&h->event_pool[i]);
            if (e != cudaSuccess) return cuda_status(e, "nirc_timing_enable");
            h->n_pool = i + 1;
        }
    }
    resolve_pending(h);
    for (int c = 0; c < NIRC_K_CLASSES; ++c) {
        h->timing_ms[c] = 0.0;
        h->timing_launches[c] = 0;
    }
    h->timing = enable != 0;
    return NIRC_OK;
}

nirc_status nirc_sync(nirc_handle* h, void* stream) {
    if (!h) {
        set_error("nirc_sync: handle is NULL");
        return NIRC_ERR_INVALID;
    }
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e, "nirc_sync");
    if (*h->host_err) {
        *h->host_err = 0;
        cudaMemset(h->dev_err, 0, sizeof(int));
        set_error("a tensor-core kernel gave up waiting for an MMA (bounded wait ran out); its output is invalid");
        return NIRC_ERR_TIMEOUT;
    }
    return NIRC_OK;
}

nirc_status nirc_timing_read(nirc_handle* h, nirc_timing* out) {
    if (!h || !out) {
        set_error("nirc_timing_read: NULL argument");
        return NIRC_ERR_INVALID;
    }
    resolve_pending(h);
    for (int c = 0; c < NIRC_K_CLASSES; ++c) {
        out->ms[c] = h->timing_ms[c];
        out->launches[c] = h->timing_launches[c];
    }
    return cuda_status(cudaGetLastError(), "nirc_timing_read");
}

uint64_t nirc_param_count(const nirc_config* cfg) {
    if (check_config(cfg) != NIRC_OK) return 0;
    const NetShape s = make_shape(*cfg);
    return s.n_mlp + s.n_hash;
}

nirc_status nirc_create(const nirc_config* cfg, nirc_handle** out) {
    if (!out) {
        set_error("out is NULL");
        return NIRC_ERR_INVALID;
    }
    *out = nullptr;
    nirc_status st = check_config(cfg);
    if (st != NIRC_OK) return st;
    nirc_handle* h = new (std::nothrow) nirc_handle();
    if (!h) {
        set_error("host allocation failed");
        return NIRC_ERR_OOM;
    }
    h->cfg = *cfg;
    h->shape = make_shape(*cfg);
    h->grid = make_grid(*cfg);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    const uint64_t np = h->shape.n_dev;
    if (e == cudaSuccess) e = cudaMalloc(&h->params, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->adam_m, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->adam_v, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->grad, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->packed, h->shape.packed_floats * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->loss_accum, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->work_counter, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->dev_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->dev_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&h->host_err, sizeof(int));
    if (e == cudaSuccess) *h->host_err = 0;
    h->packed_tc_bytes = tc_image_bytes(h->shape.hidden);
    if (e == cudaSuccess) e = cudaMalloc(&h->packed_tc, h->packed_tc_bytes);
    if (e == cudaSuccess) e = cudaMemset(h->packed_tc, 0, h->packed_tc_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->packed_tc16, h->packed_tc_bytes);
    if (e == cudaSuccess) e = cudaMemset(h->packed_tc16, 0, h->packed_tc_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->fp8_amax, 16 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(h->fp8_amax, 0, 16 * sizeof(uint32_t));
    if (e == cudaSuccess && h->shape.n_hash) e = cudaMalloc(&h->hash16, h->shape.n_hash * sizeof(__half));
    if (e == cudaSuccess) e = cudaMemset(h->params, 0, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(h->adam_m, 0, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(h->adam_v, 0, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(h->grad, 0, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(h->packed, 0, h->shape.packed_floats * sizeof(float));
    if (e == cudaSuccess && h->hash16) e = cudaMemset(h->hash16, 0, h->shape.n_hash * sizeof(__half));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        st = cuda_status(e, "nirc_create");
        nirc_destroy(h);
        return st;
    }
    *out = h;
    return NIRC_OK;
}

nirc_status nirc_destroy(nirc_handle* h) {
    if (!h) return NIRC_OK;
    cudaFree(h->params);
    cudaFree(h->adam_m);
    cudaFree(h->adam_v);
    cudaFree(h->grad);
    cudaFree(h->packed);
    cudaFree(h->loss_accum);
    cudaFree(h->dev_err);
    cudaFree(h->work_counter);
    if (h->host_err) cudaFreeHost(h->host_err);
    cudaFree(h->hash16);
    cudaFree(h->packed_tc);
    cudaFree(h->packed_tc16);
    cudaFree(h->packed_train);
    cudaFree(h->fp8_amax);
    cudaFree(h->scratch);
    cudaFree(h->train_scratch);
    for (int i = 0; i < h->n_pool; ++i) cudaEventDestroy(h->event_pool[i]);
    delete[] h->event_pool;
    delete[] h->pending;
    delete h;
    return NIRC_OK;
}

nirc_status nirc_set_params(nirc_handle* h, const float* params, int on_device, void* stream) {
    if (!h || !params) {
        set_error("nirc_set_params: NULL argument");
        return NIRC_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t np = h->shape.n_dev;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // flat [mlp | hash] input -> device [mlp | pad | hash] with the table 16-byte aligned
    cudaError_t e = cudaMemsetAsync(h->params, 0, np * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->params, params, h->shape.n_mlp * sizeof(float), kind, st);
    if (e == cudaSuccess && h->shape.n_hash)
        e = cudaMemcpyAsync(h->params + h->shape.hash_off, params + h->shape.n_mlp, h->shape.n_hash * sizeof(float),
                            kind, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->adam_m, 0, np * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->adam_v, 0, np * sizeof(float), st);
    if (e == cudaSuccess) e = launch_repack_simt(h, st);
    if (e == cudaSuccess) e = launch_hash_to_half(h, st);
    if (e == cudaSuccess) e = launch_repack_tc(h, st);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(st);  // host buffer may be freed on return
    if (e != cudaSuccess) return cuda_status(e, "nirc_set_params");
    h->step = 0;
    h->fp8_calibrated = false;
    return NIRC_OK;
}

nirc_status nirc_load_params(nirc_handle* h, const float* params, int on_device, void* stream) {
    if (!h || !params) {
        set_error("nirc_load_params: NULL argument");
        return NIRC_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(h->params, params, h->shape.n_mlp * sizeof(float), kind, st);
    if (e == cudaSuccess && h->shape.n_hash)
        e = cudaMemcpyAsync(h->params + h->shape.hash_off, params + h->shape.n_mlp, h->shape.n_hash * sizeof(float),
                            kind, st);
    if (e == cudaSuccess) e = launch_repack_simt(h, st);
    if (e == cudaSuccess) e = launch_hash_to_half(h, st);
    if (e == cudaSuccess) e = launch_repack_tc(h, st);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(st);
    h->fp8_calibrated = false;
    return cuda_status(e, "nirc_load_params");
}

static nirc_status copy_out(const nirc_handle* h, const float* src, float* out, int on_device, void* stream,
                            const char* what) {
    cudaStream_t st = (cudaStream_t)stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpyAsync(out, src, h->shape.n_mlp * sizeof(float), kind, st);
    if (e == cudaSuccess && h->shape.n_hash)
        e = cudaMemcpyAsync(out + h->shape.n_mlp, src + h->shape.hash_off, h->shape.n_hash * sizeof(float), kind, st);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(st);
    return cuda_status(e, what);
}

namespace {
struct StateHeader {
    char magic[8];
    uint32_t version;
    uint32_t step;
    nirc_config cfg;
    uint64_t n_params;
    uint64_t pad;
};
constexpr uint32_t kStateVersion = 3;

bool same_shape(const nirc_config& a, const nirc_config& b) {
    return a.pos_encoding == b.pos_encoding && a.hash_levels == b.hash_levels &&
           a.feats_per_level == b.feats_per_level && a.log2_table == b.log2_table && a.base_res == b.base_res &&
           a.growth == b.growth && a.freq_octaves == b.freq_octaves && a.width == b.width &&
           a.hidden_layers == b.hidden_layers && a.input_encoding == b.input_encoding && a.output == b.output;
}
}  // namespace

uint64_t nirc_state_bytes(const nirc_handle* h) {
    if (!h) return 0;
    return sizeof(StateHeader) + 3ull * (h->shape.n_mlp + h->shape.n_hash) * sizeof(float);
}

nirc_status nirc_save_state(nirc_handle* h, void* host_buf, uint64_t bytes, void* stream) {
    if (!h || !host_buf || bytes < nirc_state_bytes(h)) {
        set_error("nirc_save_state: NULL argument or buffer smaller than nirc_state_bytes()");
        return NIRC_ERR_INVALID;
    }
    StateHeader hd{};
    memcpy(hd.magic, "NIRCSTAT", 8);
    hd.version = kStateVersion;
    hd.step = h->step;
    hd.cfg = h->cfg;
    hd.n_params = h->shape.n_mlp + h->shape.n_hash;
    char* out = static_cast<char*>(host_buf);
    memcpy(out, &hd, sizeof(hd));
    float* body = reinterpret_cast<float*>(out + sizeof(hd));
    nirc_status st = copy_out(h, h->params, body, 0, stream, "nirc_save_state");
    if (st == NIRC_OK) st = copy_out(h, h->adam_m, body + hd.n_params, 0, stream, "nirc_save_state");
    if (st == NIRC_OK) st = copy_out(h, h->adam_v, body + 2 * hd.n_params, 0, stream, "nirc_save_state");
    return st;
}

nirc_status nirc_load_state(nirc_handle* h, const void* host_buf, uint64_t bytes, void* stream) {
    if (!h || !host_buf || bytes < sizeof(StateHeader)) {
        set_error("nirc_load_state: NULL argument or truncated buffer");
        return NIRC_ERR_INVALID;
    }
    StateHeader hd;
    memcpy(&hd, host_buf, sizeof(hd));
    const uint64_t np = h->shape.n_mlp + h->shape.n_hash;
    if (memcmp(hd.magic, "NIRCSTAT", 8) != 0 || hd.version != kStateVersion || hd.n_params != np ||
        !same_shape(hd.cfg, h->cfg) || bytes < nirc_state_bytes(h)) {
        set_error("nirc_load_state: not a state of this configuration (magic, version, shape or size differ)");
        return NIRC_ERR_INVALID;
    }
    const float* body = reinterpret_cast<const float*>(static_cast<const char*>(host_buf) + sizeof(hd));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t mlp_b = h->shape.n_mlp * sizeof(float), hash_b = h->shape.n_hash * sizeof(float);
    float* dst[3] = {h->params, h->adam_m, h->adam_v};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        e = cudaMemsetAsync(dst[k], 0, h->shape.n_dev * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst[k], body + k * np, mlp_b, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && hash_b)
            e = cudaMemcpyAsync(dst[k] + h->shape.hash_off, body + k * np + h->shape.n_mlp, hash_b,
                                cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = launch_repack_simt(h, st);
    if (e == cudaSuccess) e = launch_hash_to_half(h, st);
    if (e == cudaSuccess) e = launch_repack_tc(h, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host buffer may be freed on return
    if (e != cudaSuccess) return cuda_status(e, "nirc_load_state");
    h->step = hd.step;
    h->fp8_calibrated = false;
    return NIRC_OK;
}

nirc_status nirc_get_params(nirc_handle* h, float* out, int on_device, void* stream) {
    if (!h || !out) {
        set_error("nirc_get_params: NULL argument");
        return NIRC_ERR_INVALID;
    }
    return copy_out(h, h->params, out, on_device, stream, "nirc_get_params");
}

nirc_status nirc_get_grads(nirc_handle* h, float* out, int on_device, void* stream) {
    if (!h || !out) {
        set_error("nirc_get_grads: NULL argument");
        return NIRC_ERR_INVALID;
    }
    return copy_out(h, h->grad, out, on_device, stream, "nirc_get_grads");
}

nirc_status nirc_set_precision(nirc_handle* h, uint32_t precision) {
    if (!h || precision > NIRC_FP8_E4M3_TC) {
        set_error("nirc_set_precision: bad argument");
        return NIRC_ERR_INVALID;
    }
    const uint32_t old = h->cfg.precision;
    h->cfg.precision = precision;
    h->fp8_calibrated = false;
    // the tensor-core weight image depends on the operand type
    cudaError_t e = launch_repack_tc(h, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        h->cfg.precision = old;
        return cuda_status(e, "nirc_set_precision");
    }
    return NIRC_OK;
}

nirc_status nirc_query(nirc_handle* h, const nirc_record* d_records, const float* d_dirs, uint64_t n,
                       float* d_out_rgb, void* stream) {
    if (!h) {
        set_error("nirc_query: handle is NULL");
        return NIRC_ERR_INVALID;
    }
    if (n == 0) return NIRC_OK;
    if (!d_records || !d_dirs || !d_out_rgb || !aligned16(d_records)) {
        set_error("nirc_query: NULL or misaligned pointer");
        return NIRC_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    timer_begin(h, NIRC_K_QUERY, st);
    cudaError_t e = launch_query_simt(h, d_records, d_dirs, n, d_out_rgb, st);
    timer_end(h, NIRC_K_QUERY, st);
    return cuda_status(e, "nirc_query");
}

nirc_status nirc_estimate_frame(nirc_handle* h, const void* d_scene, const nirc_frame_desc* desc, float* d_out_rgba,
                                const nirc_frame_aux* aux, void* stream) {
    if (!h || !desc) {
        set_error("nirc_estimate_frame: NULL handle or descriptor");
        return NIRC_ERR_INVALID;
    }
    const nirc_frame_desc& fd = *desc;
    const uint64_t P = (uint64_t)fd.width * fd.height;
    if (P == 0) return NIRC_OK;
    nirc_status s = check_frame_args("nirc_estimate_frame", d_scene, fd, d_out_rgba, aux);
    if (s != NIRC_OK) return s;
    if (fd.phase == NIRC_PHASE_CACHE) {
        // the scratch must hold this frame's traced data: same descriptor apart from the phase
        nirc_frame_desc a = fd, b = h->traced_desc;
        a.phase = b.phase = 0;
        if (!h->traced || std::memcmp(&a, &b, sizeof(a)) != 0) {
            set_error("nirc_estimate_frame: NIRC_PHASE_CACHE without a NIRC_PHASE_TRACE call of the same frame");
            return NIRC_ERR_INVALID;
        }
    } else {
        h->traced = false;
        s = ensure(&h->scratch, &h->scratch_bytes, frame_scratch_bytes(P, fd.n_resid, fd.estimator), "frame");
        if (s != NIRC_OK) return s;
    }
    s = enqueue_frame("nirc_estimate_frame", h, d_scene, fd, d_out_rgba, aux, h->scratch, (cudaStream_t)stream);
    if (s == NIRC_OK && fd.phase == NIRC_PHASE_TRACE) {
        h->traced = true;
        h->traced_desc = fd;
    }
    return s;
}

nirc_status nirc_gen_train(nirc_handle* h, const void* d_scene, uint32_t n_prims, uint32_t width, uint32_t height,
                           uint64_t T, uint32_t frame, uint64_t seed, uint32_t max_depth, uint32_t light_mode,
                           nirc_record* d_records, float* d_dirs, float* d_targets, void* stream) {
    if (!h) {
        set_error("nirc_gen_train: handle is NULL");
        return NIRC_ERR_INVALID;
    }
    if (T == 0) return NIRC_OK;
    if (!d_scene || !d_records || !d_dirs || !d_targets || !aligned16(d_scene) || !aligned16(d_records)) {
        set_error("nirc_gen_train: NULL or misaligned pointer");
        return NIRC_ERR_INVALID;
    }
    if (n_prims < 1 || n_prims > NIRC_MAX_PRIMS || width == 0 || height == 0 ||
        (uint64_t)width * height > 0xFFFFFFFFull || max_depth < 1 || max_depth > 64 || T > 0xFFFFFFFFull ||
        light_mode > 2) {
        set_error("nirc_gen_train: argument out of range");
        return NIRC_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    timer_begin(h, NIRC_K_TRAIN_RECORDS, st);
    cudaError_t e = launch_gen_train(h, d_scene, n_prims, width, height, T, frame, seed, max_depth, light_mode,
                                     d_records, d_dirs, d_targets, st);
    timer_end(h, NIRC_K_TRAIN_RECORDS, st);
    return cuda_status(e, "nirc_gen_train");
}

nirc_status nirc_train_step(nirc_handle* h, const nirc_record* d_records, const float* d_dirs, const float* d_targets,
                            uint64_t n, float* d_loss, void* stream) {
    if (!h) {
        set_error("nirc_train_step: handle is NULL");
        return NIRC_ERR_INVALID;
    }
    if (n == 0) return NIRC_OK;
    if (!d_records || !d_dirs || !d_targets || !aligned16(d_records) || n > 0xFFFFFFFFull) {
        set_error("nirc_train_step: NULL/misaligned pointer or n too large");
        return NIRC_ERR_INVALID;
    }
    nirc_status s = ensure(&h->train_scratch, &h->train_scratch_bytes, train_scratch_bytes(h, n), "training");
    if (s != NIRC_OK) return s;
    return cuda_status(launch_train_step(h, d_records, d_dirs, d_targets, n, d_loss, (cudaStream_t)stream),
                       "nirc_train_step");
}

nirc_status nirc_set_train_mode(nirc_handle* h, int store_activations, uint64_t recompute_chunk) {
    if (!h || (!store_activations && (recompute_chunk < 1024 || recompute_chunk > (1ull << 26)))) {
        set_error("nirc_set_train_mode: NULL handle or recompute_chunk outside 1024..2^26");
        return NIRC_ERR_INVALID;
    }
    h->store_activations = store_activations ? 1 : 0;
    if (!store_activations) h->recompute_chunk = recompute_chunk;
    return NIRC_OK;
}

nirc_status nirc_set_train_precision(nirc_handle* h, uint32_t precision) {
    if (!h || (precision != NIRC_FP32_SIMT && precision != NIRC_FP16_TC)) {
        set_error("nirc_set_train_precision: NULL handle or precision not NIRC_FP32_SIMT / NIRC_FP16_TC");
        return NIRC_ERR_INVALID;
    }
    if (precision == NIRC_FP32_SIMT) {
        if (h->packed_train) {
            cudaError_t e = cudaDeviceSynchronize();
            cudaFree(h->packed_train);
            h->packed_train = nullptr;
            if (e != cudaSuccess) return cuda_status(e, "nirc_set_train_precision");
        }
        return NIRC_OK;
    }
    if (!train_tc_shape_ok(h->shape)) {
        set_error("nirc_set_train_precision: tensor-core training covers 1..8 hidden layers and 24 or 32 "
                  "position features");
        return NIRC_ERR_UNSUPPORTED;
    }
    cudaError_t e = cudaSuccess;
    if (!h->packed_train) e = cudaMalloc(&h->packed_train, train_tc_image_bytes(h->shape.hidden));
    if (e == cudaSuccess) e = cudaMemset(h->packed_train, 0, train_tc_image_bytes(h->shape.hidden));
    if (e == cudaSuccess) e = launch_repack_train(h, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        cudaFree(h->packed_train);
        h->packed_train = nullptr;
        return cuda_status(e, "nirc_set_train_precision");
    }
    return NIRC_OK;
}

nirc_status nirc_set_deterministic(nirc_handle* h, int on) {
    if (!h) {
        set_error("nirc_set_deterministic: NULL handle");
        return NIRC_ERR_INVALID;
    }
    h->deterministic = on ? 1 : 0;
    return NIRC_OK;
}

nirc_status nirc_query_bwd(nirc_handle* h, const nirc_record* d_records, const float* d_dirs,
                           const float* d_grad_out, uint64_t n, float* d_grad_params, float* d_value, void* stream) {
    if (!h) {
        set_error("nirc_query_bwd: handle is NULL");
        return NIRC_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(h->grad, 0, h->shape.n_dev * sizeof(float), st);
        if (e == cudaSuccess && d_value) e = cudaMemsetAsync(d_value, 0, sizeof(float), st);
        if (e == cudaSuccess && d_grad_params) {
            e = cudaMemsetAsync(d_grad_params, 0, (h->shape.n_mlp + h->shape.n_hash) * sizeof(float), st);
        }
        return cuda_status(e, "nirc_query_bwd");
    }
    if (!d_records || !d_dirs || !d_grad_out || !aligned16(d_records) || n > 0xFFFFFFFFull) {
        set_error("nirc_query_bwd: NULL/misaligned pointer or n too large");
        return NIRC_ERR_INVALID;
    }
    nirc_status s = ensure(&h->train_scratch, &h->train_scratch_bytes, train_scratch_bytes(h, n), "training");
    if (s != NIRC_OK) return s;
    cudaError_t e = launch_query_bwd(h, d_records, d_dirs, d_grad_out, n, d_value, st);
    if (e != cudaSuccess) return cuda_status(e, "nirc_query_bwd");
    if (!d_grad_params) return NIRC_OK;
    return copy_out(h, h->grad, d_grad_params, 1, stream, "nirc_query_bwd");
}

nirc_status nirc_frame_mrse(const float* d_img_rgba, const float* d_ref_rgba, uint64_t n_pixels, float eps,
                            double* d_out, void* stream) {
    if (!d_out) {
        set_error("nirc_frame_mrse: output is NULL");
        return NIRC_ERR_INVALID;
    }
    if (n_pixels && (!d_img_rgba || !d_ref_rgba || !aligned16(d_img_rgba) || !aligned16(d_ref_rgba))) {
        set_error("nirc_frame_mrse: NULL or misaligned image");
        return NIRC_ERR_INVALID;
    }
    return cuda_status(launch_mrse(d_img_rgba, d_ref_rgba, n_pixels, eps, d_out, (cudaStream_t)stream),
                       "nirc_frame_mrse");
}

}  // extern "C"
