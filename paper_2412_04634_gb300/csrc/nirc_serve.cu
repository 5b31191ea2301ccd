// nirc_serve.cu -- frame-request server (include/nirc_serve.h): continuous
// batching of render requests over resident scene caches.
//
// Host-side runtime only; the GPU work of a request is the library's own
// frame, training-pass and training-step kernels, enqueued exactly as the
// single-renderer entry points enqueue them.
//
//  Arena      first-fit allocator over one cudaMalloc'd block, 256-byte
//             granules, neighbours coalesced on release
//  scheduler  forms a batch from the FIFO (arrival order, skipping requests
//             whose scene is busy, stopping at the first that does not fit),
//             captures the batch into a CUDA graph, re-uses the batch
//             slot's executable graph via cudaGraphExecUpdate when it can,
//             and launches it.  In the graph the frames of all requests are
//             one launch of each path-tracing pass (camera, residual; per
//             light mode) and one cache-integral launch over the union of
//             their pixels, CTAs shared out in proportion to each
//             request's work; then each request's training pass and step
//             run as their own branch (fork/join over worker streams).  A batch that cannot share launches (another
//             precision, network shape or light mode 2 among its caches)
//             runs each request's whole chain as its own branch.
//  completer  polls the in-flight batches' events, stamps completion times,
//             returns frame scratch to the arena and frees the scenes
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nirc_internal.h"
#include "nirc_serve.h"

namespace nirc {

constexpr uint32_t kMaxSlots = 16;
constexpr uint32_t kMaxBatches = 4;

static uint64_t granule(uint64_t b) { return (b + 255) & ~255ull; }

class Arena {
   public:
    void init(uint64_t size) {
        size_ = size;
        free_.clear();
        free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(uint64_t bytes, uint64_t* off) {
        bytes = granule(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const uint64_t o = it->first, rem = it->second - bytes;
            free_.erase(it);
            if (rem) free_[o + bytes] = rem;
            *off = o;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = granule(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    uint64_t size() const { return size_; }
    uint64_t used() const { return used_; }
    uint64_t peak() const { return peak_; }

   private:
    uint64_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<uint64_t, uint64_t> free_;  // offset -> length
};

struct SceneSlot {
    nirc_handle* h = nullptr;
    const char* frames = nullptr;
    uint32_t n_frames = 0;
    uint64_t stride = 0;
    uint32_t n_prims = 0;
    uint64_t seed = 0;
    nirc_record* trecs = nullptr;
    float* tdirs = nullptr;
    float* ttgts = nullptr;
    uint64_t resident = 0;
    bool busy = false;
};

struct Req {
    nirc_request r{};
    double t_submit = 0, t_launch = 0, t_done = 0;
    uint64_t img_off = 0, img_bytes = 0, scr_off = 0, scr_bytes = 0;
    int status = NIRC_OK;
    uint32_t batch_size = 0;
};

struct Batch {
    std::vector<Req*> reqs;
    int slot = 0;
};

static double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace nirc

using namespace nirc;

struct nirc_server {
    nirc_server_config cfg{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    char* arena_base = nullptr;
    Arena arena;
    std::vector<SceneSlot> scenes;

    std::mutex mu;
    std::condition_variable cv;       // scheduler wake-ups
    std::condition_variable cv_done;  // completer wake-ups
    std::condition_variable cv_user;  // poll / drain wake-ups
    std::deque<Req*> queue;
    std::deque<Req*> completed;                 // finished, not yet polled
    std::unordered_map<uint64_t, Req*> active;  // submitted and not released
    std::vector<Batch*> inflight;
    int launching = 0;
    bool stalled = false;  // queue non-empty, nothing running, head does not fit
    uint64_t gen = 0;      // bumped by every event that can unblock admission
    bool stop = false, stop_done = false;

    std::vector<cudaStream_t> launch_st;               // one per batch slot
    std::vector<std::vector<cudaStream_t>> worker_st;  // [slot][request]
    std::vector<cudaEvent_t> fork_ev, done_ev;         // per batch slot
    std::vector<std::vector<cudaEvent_t>> join_ev;     // [slot][request]
    std::vector<std::vector<cudaGraphExec_t>> execs;   // [slot][batch size]
    std::vector<bool> slot_busy;
    unsigned long long* work_counters = nullptr;       // [slot][request]: path-tracing pixel counters

    nirc_server_stats stats{};
    std::thread scheduler, completer;

    void run_scheduler();
    void run_completer();
    nirc_status enqueue_request(Req* q, cudaStream_t st);
    nirc_status enqueue_training(Req* q, cudaStream_t st);
    bool shares_launches(const Batch* b) const;
    nirc_status enqueue_batch_frames(Batch* b, cudaStream_t st);
    nirc_status launch_batch(Batch* b);
};

nirc_status nirc_server::enqueue_request(Req* q, cudaStream_t st) {
    SceneSlot& sc = scenes[q->r.scene];
    nirc_frame_desc fd{};
    fd.width = q->r.width;
    fd.height = q->r.height;
    fd.n_cache = q->r.n_cache;
    fd.n_resid = q->r.n_resid;
    fd.max_depth = q->r.max_depth;
    fd.frame = q->r.frame;
    fd.seed = sc.seed;
    fd.n_prims = sc.n_prims;
    fd.cache_mode = 0;
    fd.light_mode = q->r.light_mode;
    const void* blob = sc.frames + (uint64_t)(q->r.frame % sc.n_frames) * sc.stride;
    float* img = reinterpret_cast<float*>(arena_base + q->img_off);
    void* scratch = arena_base + q->scr_off;
    nirc_status s = enqueue_frame("nirc_server", sc.h, blob, fd, img, nullptr, scratch, st);
    if (s == NIRC_OK) {
        std::lock_guard<std::mutex> lk(mu);
        stats.frame_launches += 3;  // camera pass, residual pass, cache integral
    }
    if (s != NIRC_OK) return s;
    return enqueue_training(q, st);
}

nirc_status nirc_server::enqueue_training(Req* q, cudaStream_t st) {
    SceneSlot& sc = scenes[q->r.scene];
    if (cfg.train_samples == 0) return NIRC_OK;
    if (sc.h->train_scratch_bytes < train_scratch_bytes(sc.h, cfg.train_samples)) {
        set_error("nirc_server: scene %u needs more training scratch than was reserved at registration "
                  "(set the handle's training modes before nirc_server_add_scene)", q->r.scene);
        return NIRC_ERR_BUDGET;
    }
    const void* blob = sc.frames + (uint64_t)(q->r.frame % sc.n_frames) * sc.stride;
    cudaError_t e = launch_gen_train(sc.h, blob, sc.n_prims, q->r.width, q->r.height, cfg.train_samples, q->r.frame,
                                     sc.seed, q->r.max_depth, q->r.light_mode, sc.trecs, sc.tdirs, sc.ttgts, st);
    if (e == cudaSuccess) e = launch_train_step(sc.h, sc.trecs, sc.tdirs, sc.ttgts, cfg.train_samples, nullptr, st);
    return cuda_status(e, "nirc_server (training)");
}

// Whether the batch's frames can share one launch per path-tracing pass
// and light mode and one cache-integral launch.
bool nirc_server::shares_launches(const Batch* b) const {
    const nirc_handle* h0 = scenes[b->reqs[0]->r.scene].h;
    for (const Req* q : b->reqs) {
        const nirc_handle* h = scenes[q->r.scene].h;
        nirc_frame_desc fd{};
        fd.width = q->r.width;
        fd.height = q->r.height;
        fd.n_cache = q->r.n_cache;
        fd.n_resid = q->r.n_resid;
        if (q->r.light_mode > 1 || h->timing || !tc_batchable(h0, h) || !tc_supported(h, fd)) return false;
    }
    return true;
}

nirc_status nirc_server::enqueue_batch_frames(Batch* b, cudaStream_t st) {
    const uint32_t n = (uint32_t)b->reqs.size();
    FrameJob fj[kMaxFrameJobs];
    unsigned long long* counters = work_counters + (uint64_t)b->slot * kMaxSlots;
    for (uint32_t i = 0; i < n; ++i) {
        const Req* q = b->reqs[i];
        const SceneSlot& sc = scenes[q->r.scene];
        FrameJob& f = fj[i];
        f.h = sc.h;
        f.fd = nirc_frame_desc{};
        f.fd.width = q->r.width;
        f.fd.height = q->r.height;
        f.fd.n_cache = q->r.n_cache;
        f.fd.n_resid = q->r.n_resid;
        f.fd.max_depth = q->r.max_depth;
        f.fd.frame = q->r.frame;
        f.fd.seed = sc.seed;
        f.fd.n_prims = sc.n_prims;
        f.fd.light_mode = q->r.light_mode;
        f.scene = sc.frames + (uint64_t)(q->r.frame % sc.n_frames) * sc.stride;
        // frame scratch as enqueue_frame carves it: records | per-pixel bases | residual rows
        const uint64_t P = (uint64_t)q->r.width * q->r.height;
        char* sp = arena_base + q->scr_off;
        f.recs = reinterpret_cast<nirc_record*>(sp);
        f.base = reinterpret_cast<PixelBase*>(sp + granule(P * sizeof(nirc_record)));
        f.rows = reinterpret_cast<ResidRow*>(sp + granule(P * sizeof(nirc_record)) + granule(P * sizeof(PixelBase)));
        f.out = reinterpret_cast<float*>(arena_base + q->img_off);
        f.work = counters + i;
    }
    cudaError_t e = cudaMemsetAsync(counters, 0, n * sizeof(unsigned long long), st);
    uint32_t launches = 0;
    for (uint32_t lm = 0; lm <= 1 && e == cudaSuccess; ++lm) {
        FrameJob sub[kMaxFrameJobs];
        uint32_t m = 0;
        for (uint32_t i = 0; i < n; ++i)
            if (fj[i].fd.light_mode == lm) sub[m++] = fj[i];
        if (m) {
            e = launch_primary_resid_batch(sub, m, st);
            launches += 2;  // camera and residual passes
        }
    }
    if (e == cudaSuccess) {
        e = launch_cache_tc_batch(fj, n, st);
        ++launches;
    }
    for (uint32_t i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(fj[i].h->host_err, fj[i].h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(mu);
        stats.frame_launches += launches;
    }
    return cuda_status(e, "nirc_server (batched frames)");
}

nirc_status nirc_server::launch_batch(Batch* b) {
    const int k = b->slot;
    cudaStream_t ls = launch_st[k];
    const size_t n = b->reqs.size();
    bool graphs = cfg.use_graphs != 0;
    for (Req* q : b->reqs) graphs = graphs && !scenes[q->r.scene].h->timing;
    cudaError_t e = cudaSuccess;
    if (graphs) e = cudaStreamBeginCapture(ls, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_status(e, "nirc_server (begin capture)");
    nirc_status s = NIRC_OK;
    const bool shared = shares_launches(b);
    if (shared) s = enqueue_batch_frames(b, ls);  // every frame of the batch: one launch per kernel
    if (s == NIRC_OK) e = cudaEventRecord(fork_ev[k], ls);
    for (size_t i = 0; i < n && e == cudaSuccess && s == NIRC_OK; ++i) {
        cudaStream_t ws = worker_st[k][i];
        e = cudaStreamWaitEvent(ws, fork_ev[k], 0);
        if (e != cudaSuccess) break;
        s = shared ? enqueue_training(b->reqs[i], ws) : enqueue_request(b->reqs[i], ws);
        if (s != NIRC_OK) break;
        e = cudaEventRecord(join_ev[k][i], ws);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ls, join_ev[k][i], 0);
    }
    if (graphs) {
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(ls, &g);
        if (e == cudaSuccess) e = ec;
        if (e == cudaSuccess && s == NIRC_OK) {
            cudaGraphExec_t& ex = execs[k][n];
            bool updated = false;
            if (ex) {
                cudaGraphExecUpdateResultInfo info{};
                if (cudaGraphExecUpdate(ex, g, &info) == cudaSuccess) {
                    updated = true;
                } else {
                    cudaGetLastError();
                    cudaGraphExecDestroy(ex);
                    ex = nullptr;
                }
            }
            if (!updated) e = cudaGraphInstantiate(&ex, g, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ex, ls);
            std::lock_guard<std::mutex> lk(mu);
            if (updated) stats.graph_updates += 1;
            else stats.graph_instantiations += 1;
        }
        if (g) cudaGraphDestroy(g);
    }
    if (s != NIRC_OK) return s;
    if (e == cudaSuccess) e = cudaEventRecord(done_ev[k], ls);
    return cuda_status(e, "nirc_server (batch launch)");
}

void nirc_server::run_scheduler() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    uint64_t seen = ~0ull;
    while (true) {
        cv.wait(lk, [&] { return stop || (gen != seen && !queue.empty()); });
        if (stop) break;
        seen = gen;
        int slot = -1;
        for (uint32_t i = 0; i < cfg.max_batches; ++i)
            if (!slot_busy[i]) {
                slot = (int)i;
                break;
            }
        if (slot < 0) continue;  // a completion bumps gen
        Batch* b = new (std::nothrow) Batch();
        if (!b) continue;
        b->slot = slot;
        for (auto it = queue.begin(); it != queue.end() && b->reqs.size() < cfg.slots;) {
            Req* q = *it;
            SceneSlot& sc = scenes[q->r.scene];
            if (sc.busy) {
                ++it;
                continue;
            }
            if (!arena.alloc(q->img_bytes, &q->img_off)) break;
            if (!arena.alloc(q->scr_bytes, &q->scr_off)) {
                arena.release(q->img_off, q->img_bytes);
                break;
            }
            sc.busy = true;
            b->reqs.push_back(q);
            it = queue.erase(it);
        }
        if (b->reqs.empty()) {
            delete b;
            stalled = inflight.empty() && launching == 0;
            if (stalled) cv_user.notify_all();
            continue;
        }
        stalled = false;
        slot_busy[slot] = true;
        launching += 1;
        const double t = now_s(t0);
        for (Req* q : b->reqs) {
            q->t_launch = t;
            q->batch_size = (uint32_t)b->reqs.size();
        }
        stats.batches += 1;
        stats.max_batch_seen = std::max<uint32_t>(stats.max_batch_seen, (uint32_t)b->reqs.size());
        lk.unlock();
        const nirc_status s = launch_batch(b);
        lk.lock();
        launching -= 1;
        if (s != NIRC_OK) {
            // nothing of the batch is known to run: drain the slot's streams
            // before the buffers go back to the arena
            lk.unlock();
            cudaStreamSynchronize(launch_st[slot]);
            for (size_t i = 0; i < b->reqs.size(); ++i) cudaStreamSynchronize(worker_st[slot][i]);
            lk.lock();
            const double td = now_s(t0);
            for (Req* q : b->reqs) {
                q->status = s;
                q->t_done = td;
                arena.release(q->scr_off, q->scr_bytes);
                scenes[q->r.scene].busy = false;
                completed.push_back(q);
                stats.failed += 1;
            }
            slot_busy[slot] = false;
            delete b;
            gen += 1;
            cv_user.notify_all();
            continue;
        }
        inflight.push_back(b);
        gen += 1;  // the rest of the queue may fill another batch slot now
        cv_done.notify_all();
        cv_user.notify_all();
    }
}

void nirc_server::run_completer() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        cv_done.wait(lk, [&] { return stop_done || !inflight.empty(); });
        if (inflight.empty()) {
            if (stop_done) break;
            continue;
        }
        std::vector<Batch*> snap = inflight;
        lk.unlock();
        std::vector<std::pair<Batch*, cudaError_t>> fin;
        for (Batch* b : snap) {
            const cudaError_t q = cudaEventQuery(done_ev[b->slot]);
            if (q != cudaErrorNotReady) fin.emplace_back(b, q);
        }
        if (fin.empty()) {
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
            continue;
        }
        const double t = now_s(t0);
        lk.lock();
        for (auto& [b, q] : fin) {
            inflight.erase(std::find(inflight.begin(), inflight.end(), b));
            for (Req* r : b->reqs) {
                SceneSlot& sc = scenes[r->r.scene];
                r->t_done = t;
                if (q != cudaSuccess) {
                    r->status = NIRC_ERR_CUDA;
                } else if (*sc.h->host_err) {
                    *sc.h->host_err = 0;
                    cudaMemsetAsync(sc.h->dev_err, 0, sizeof(int), launch_st[b->slot]);
                    r->status = NIRC_ERR_TIMEOUT;
                }
                if (r->status == NIRC_OK) stats.completed += 1;
                else stats.failed += 1;
                arena.release(r->scr_off, r->scr_bytes);
                sc.busy = false;
                completed.push_back(r);
            }
            slot_busy[b->slot] = false;
            delete b;
        }
        gen += 1;
        cv.notify_all();
        cv_user.notify_all();
    }
}

static nirc_status server_fail(nirc_server* s, nirc_status st) {
    nirc_server_destroy(s);
    return st;
}

extern "C" {

nirc_status nirc_server_create(const nirc_server_config* cfg, nirc_server** out) {
    if (!cfg || !out) {
        set_error("nirc_server_create: NULL argument");
        return NIRC_ERR_INVALID;
    }
    *out = nullptr;
    if (cfg->budget_bytes < (1ull << 20) || cfg->slots < 1 || cfg->slots > kMaxSlots || cfg->max_batches < 1 ||
        cfg->max_batches > kMaxBatches || cfg->train_samples > (1u << 24)) {
        set_error("nirc_server_create: budget >= 1 MiB, slots 1..%u, max_batches 1..%u, train_samples <= 2^24",
                  kMaxSlots, kMaxBatches);
        return NIRC_ERR_INVALID;
    }
    nirc_server* s = new (std::nothrow) nirc_server();
    if (!s) {
        set_error("nirc_server_create: host allocation failed");
        return NIRC_ERR_OOM;
    }
    s->cfg = *cfg;
    s->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->arena_base, cfg->budget_bytes);
    if (e != cudaSuccess) {
        s->arena_base = nullptr;
        return server_fail(s, cuda_status(e, "nirc_server_create (arena)"));
    }
    e = cudaMalloc(&s->work_counters, (size_t)kMaxBatches * kMaxSlots * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        s->work_counters = nullptr;
        return server_fail(s, cuda_status(e, "nirc_server_create (work counters)"));
    }
    s->arena.init(cfg->budget_bytes);
    const uint32_t B = cfg->max_batches, S = cfg->slots;
    s->launch_st.assign(B, nullptr);
    s->fork_ev.assign(B, nullptr);
    s->done_ev.assign(B, nullptr);
    s->worker_st.assign(B, std::vector<cudaStream_t>(S, nullptr));
    s->join_ev.assign(B, std::vector<cudaEvent_t>(S, nullptr));
    s->execs.assign(B, std::vector<cudaGraphExec_t>(S + 1, nullptr));
    s->slot_busy.assign(B, false);
    for (uint32_t k = 0; k < B && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&s->launch_st[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork_ev[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->done_ev[k], cudaEventDisableTiming);
        for (uint32_t i = 0; i < S && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&s->worker_st[k][i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->join_ev[k][i], cudaEventDisableTiming);
        }
    }
    if (e != cudaSuccess) return server_fail(s, cuda_status(e, "nirc_server_create (streams)"));
    try {
        s->scheduler = std::thread([s] { s->run_scheduler(); });
        s->completer = std::thread([s] { s->run_completer(); });
    } catch (...) {
        set_error("nirc_server_create: cannot start threads");
        return server_fail(s, NIRC_ERR_OOM);
    }
    *out = s;
    return NIRC_OK;
}

nirc_status nirc_server_add_scene(nirc_server* s, nirc_handle* cache, const void* d_frames, uint32_t n_frames,
                                  uint64_t frame_stride, uint32_t n_prims, uint64_t seed, uint32_t* scene_out) {
    if (!s || !cache || !d_frames || !scene_out || n_frames == 0 || ((uintptr_t)d_frames & 15u) ||
        (n_frames > 1 && (frame_stride & 15u)) || n_prims < 1 || n_prims > NIRC_MAX_PRIMS) {
        set_error("nirc_server_add_scene: NULL/misaligned argument or bad frame/primitive count");
        return NIRC_ERR_INVALID;
    }
    if (cache->timing) {
        set_error("nirc_server_add_scene: the handle's kernel timers must be off");
        return NIRC_ERR_INVALID;
    }
    SceneSlot sc;
    sc.h = cache;
    sc.frames = static_cast<const char*>(d_frames);
    sc.n_frames = n_frames;
    sc.stride = frame_stride;
    sc.n_prims = n_prims;
    sc.seed = seed;
    const uint64_t T = s->cfg.train_samples;
    cudaError_t e = cudaSuccess;
    if (T) {
        e = cudaMalloc(&sc.trecs, T * sizeof(nirc_record));
        if (e == cudaSuccess) e = cudaMalloc(&sc.tdirs, T * 3 * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&sc.ttgts, T * 3 * sizeof(float));
        if (e == cudaSuccess) {
            const nirc_status r = reserve_train_scratch(cache, T);
            if (r != NIRC_OK) {
                cudaFree(sc.trecs);
                cudaFree(sc.tdirs);
                cudaFree(sc.ttgts);
                return r;
            }
        }
    }
    if (e != cudaSuccess) {
        cudaFree(sc.trecs);
        cudaFree(sc.tdirs);
        cudaFree(sc.ttgts);
        return cuda_status(e, "nirc_server_add_scene");
    }
    // blobs and parameters uploaded on other streams must be in place before
    // the server's non-blocking streams read them
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(sc.trecs);
        cudaFree(sc.tdirs);
        cudaFree(sc.ttgts);
        return cuda_status(e, "nirc_server_add_scene");
    }
    const NetShape& sh = cache->shape;
    sc.resident = sh.n_dev * 4 * sizeof(float) + sh.n_hash * sizeof(__half) + cache->packed_tc_bytes +
                  sh.packed_floats * sizeof(float) + cache->train_scratch_bytes + cache->scratch_bytes +
                  T * (sizeof(nirc_record) + 6 * sizeof(float));
    std::lock_guard<std::mutex> lk(s->mu);
    for (const SceneSlot& o : s->scenes)
        if (o.h == cache) {
            cudaFree(sc.trecs);
            cudaFree(sc.tdirs);
            cudaFree(sc.ttgts);
            set_error("nirc_server_add_scene: handle already registered");
            return NIRC_ERR_INVALID;
        }
    *scene_out = (uint32_t)s->scenes.size();
    s->scenes.push_back(sc);
    s->stats.resident_bytes += sc.resident;
    return NIRC_OK;
}

nirc_status nirc_server_submit(nirc_server* s, const nirc_request* req) {
    if (!s || !req) {
        set_error("nirc_server_submit: NULL argument");
        return NIRC_ERR_INVALID;
    }
    const nirc_request& r = *req;
    if (r.width < 1 || r.width > 8192 || r.height < 1 || r.height > 8192 || r.n_cache > 1024 || r.n_resid > 64 ||
        r.max_depth < 1 || r.max_depth > 64 || r.light_mode > 1) {
        set_error("nirc_server_submit: size out of range (W, H 1..8192, N <= 1024, M <= 64, depth 1..64, "
                  "light_mode 0..1)");
        return NIRC_ERR_INVALID;
    }
    Req* q = new (std::nothrow) Req();
    if (!q) {
        set_error("nirc_server_submit: host allocation failed");
        return NIRC_ERR_OOM;
    }
    q->r = r;
    const uint64_t P = (uint64_t)r.width * r.height;
    q->img_bytes = granule(P * 16);
    q->scr_bytes = granule(frame_scratch_bytes(P, r.n_resid, NIRC_EST_TWO_LEVEL));
    std::lock_guard<std::mutex> lk(s->mu);
    if (r.scene >= s->scenes.size()) {
        delete q;
        set_error("nirc_server_submit: scene %u not registered", r.scene);
        return NIRC_ERR_INVALID;
    }
    if (q->img_bytes + q->scr_bytes > s->arena.size()) {
        delete q;
        set_error("nirc_server_submit: request needs %llu bytes, the arena holds %llu",
                  (unsigned long long)(q->img_bytes + q->scr_bytes), (unsigned long long)s->arena.size());
        return NIRC_ERR_BUDGET;
    }
    if (s->active.count(r.id)) {
        delete q;
        set_error("nirc_server_submit: id %llu is still in use", (unsigned long long)r.id);
        return NIRC_ERR_INVALID;
    }
    q->t_submit = now_s(s->t0);
    s->active[r.id] = q;
    s->queue.push_back(q);
    s->stats.submitted += 1;
    s->gen += 1;
    s->cv.notify_all();
    return NIRC_OK;
}

nirc_status nirc_server_poll(nirc_server* s, nirc_completion* out, uint32_t max, uint32_t* n_out, int wait) {
    if (!s || !n_out || (max && !out)) {
        set_error("nirc_server_poll: NULL argument");
        return NIRC_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (wait) {
        s->cv_user.wait(lk, [&] {
            return !s->completed.empty() || s->stalled ||
                   (s->queue.empty() && s->inflight.empty() && s->launching == 0);
        });
    }
    uint32_t n = 0;
    while (n < max && !s->completed.empty()) {
        Req* q = s->completed.front();
        s->completed.pop_front();
        nirc_completion& c = out[n++];
        c.id = q->r.id;
        c.status = q->status;
        c.batch_size = q->batch_size;
        c.d_image = reinterpret_cast<float*>(s->arena_base + q->img_off);
        c.t_submit = q->t_submit;
        c.t_launch = q->t_launch;
        c.t_done = q->t_done;
    }
    *n_out = n;
    if (n == 0 && wait && s->stalled) {
        set_error("nirc_server_poll: queued requests do not fit in the arena while completed images are unreleased");
        return NIRC_ERR_BUDGET;
    }
    return NIRC_OK;
}

nirc_status nirc_server_copy_image(nirc_server* s, uint64_t id, float* d_dst, void* stream) {
    if (!s || !d_dst) {
        set_error("nirc_server_copy_image: NULL argument");
        return NIRC_ERR_INVALID;
    }
    const void* src = nullptr;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->active.find(id);
        if (it == s->active.end() || it->second->t_done == 0.0 ||
            std::find(s->completed.begin(), s->completed.end(), it->second) != s->completed.end()) {
            set_error("nirc_server_copy_image: id %llu is not a polled request", (unsigned long long)id);
            return NIRC_ERR_INVALID;
        }
        src = s->arena_base + it->second->img_off;
        bytes = (size_t)it->second->r.width * it->second->r.height * 16;
    }
    return cuda_status(cudaMemcpyAsync(d_dst, src, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
                       "nirc_server_copy_image");
}

nirc_status nirc_server_release(nirc_server* s, uint64_t id) {
    if (!s) {
        set_error("nirc_server_release: NULL server");
        return NIRC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->active.find(id);
    if (it == s->active.end() ||
        std::find(s->completed.begin(), s->completed.end(), it->second) != s->completed.end() ||
        it->second->t_done == 0.0) {
        set_error("nirc_server_release: id %llu is not a polled request", (unsigned long long)id);
        return NIRC_ERR_INVALID;
    }
    Req* q = it->second;
    s->arena.release(q->img_off, q->img_bytes);
    s->active.erase(it);
    delete q;
    s->stalled = false;
    s->gen += 1;
    s->cv.notify_all();
    return NIRC_OK;
}

nirc_status nirc_server_drain(nirc_server* s) {
    if (!s) {
        set_error("nirc_server_drain: NULL server");
        return NIRC_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_user.wait(lk, [&] { return s->stalled || (s->queue.empty() && s->inflight.empty() && s->launching == 0); });
    if (!s->queue.empty()) {
        set_error("nirc_server_drain: queued requests do not fit in the arena while completed images are unreleased");
        return NIRC_ERR_BUDGET;
    }
    return NIRC_OK;
}

nirc_status nirc_server_stats_read(nirc_server* s, nirc_server_stats* out) {
    if (!s || !out) {
        set_error("nirc_server_stats_read: NULL argument");
        return NIRC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->arena_bytes = s->arena.used();
    out->arena_peak_bytes = s->arena.peak();
    out->queued = (uint32_t)s->queue.size();
    uint32_t inf = 0;
    for (Batch* b : s->inflight) inf += (uint32_t)b->reqs.size();
    out->in_flight = inf;
    return NIRC_OK;
}

double nirc_server_clock(nirc_server* s) { return s ? now_s(s->t0) : 0.0; }

nirc_status nirc_server_destroy(nirc_server* s) {
    if (!s) return NIRC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->scheduler.joinable()) s->scheduler.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop_done = true;
        s->cv_done.notify_all();
    }
    if (s->completer.joinable()) s->completer.join();  // returns once nothing is in flight
    for (Req* q : s->queue) {
        s->active.erase(q->r.id);
        delete q;
    }
    for (auto& kv : s->active) delete kv.second;
    for (auto& row : s->execs)
        for (cudaGraphExec_t ex : row)
            if (ex) cudaGraphExecDestroy(ex);
    for (auto& row : s->worker_st)
        for (cudaStream_t st : row)
            if (st) cudaStreamDestroy(st);
    for (auto& row : s->join_ev)
        for (cudaEvent_t ev : row)
            if (ev) cudaEventDestroy(ev);
    for (cudaStream_t st : s->launch_st)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->fork_ev)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : s->done_ev)
        if (ev) cudaEventDestroy(ev);
    for (SceneSlot& sc : s->scenes) {
        cudaFree(sc.trecs);
        cudaFree(sc.tdirs);
        cudaFree(sc.ttgts);
    }
    cudaFree(s->arena_base);
    cudaFree(s->work_counters);
    delete s;
    return NIRC_OK;
}

}  // extern "C"
