// nirc_noalloc.cu -- nirc_estimate_frame_noalloc: the frame estimate for
// callers that cannot allocate device memory at call time.
//
// nirc_estimate_frame keeps its per-frame scratch (shading records, per-pixel
// bases, residual rows) in handle-owned buffers that it grows with cudaMalloc
// the first time a larger frame arrives.  Some callers cannot let a call do
// that: a renderer that has reserved all device memory up front, a real-time
// frame loop that must not pay cudaMalloc/cudaFree's implicit device-wide
// synchronisation in the middle of a frame, or an embedding application whose
// allocation policy forbids allocations outside its own allocator.  This
// entry point runs the same two kernels on a fixed scratch area compiled into
// the library instead, so it never calls cudaMalloc, cudaFree or any
// allocating routine.
//
// The scratch is one file-scope device array of kNoAllocScratchBytes (4 MiB)
// that every GPU loading the library holds until the process exits.  Host
// code never uses the array's name as an address: the first call on each
// device looks the device address up with cudaGetSymbolAddress (with that
// device current) and later calls reuse it.  All calls on a device share the
// array; calls that overlap on the GPU (different streams, or different
// handles, without ordering between them) race on it.
#include <mutex>

#include "nirc_internal.h"

namespace nirc {

constexpr size_t kNoAllocScratchBytes = 4u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_frame_scratch[kNoAllocScratchBytes];

// Device address of g_frame_scratch on the current device (set up once per device).
static nirc_status scratch_address(int device, unsigned char** out) {
    static std::mutex mu;
    static unsigned char* addr[kMaxDevices] = {};
    if (device < 0 || device >= kMaxDevices) {
        set_error("nirc_estimate_frame_noalloc: device ordinal %d out of range", device);
        return NIRC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_frame_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error("nirc_estimate_frame_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return NIRC_ERR_CUDA;
        }
        addr[device] = static_cast<unsigned char*>(p);
    }
    *out = addr[device];
    return NIRC_OK;
}

static size_t round256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

}  // namespace nirc

using namespace nirc;

extern "C" nirc_status nirc_estimate_frame_noalloc(nirc_handle* h, const void* d_scene, const nirc_frame_desc* desc,
                                                   float* d_out_rgba, const nirc_frame_aux* aux, void* stream) {
    if (!h || !desc) {
        set_error("nirc_estimate_frame_noalloc: NULL handle or descriptor");
        return NIRC_ERR_INVALID;
    }
    const nirc_frame_desc& fd = *desc;
    const uint64_t P = (uint64_t)fd.width * fd.height;
    if (P == 0) return NIRC_OK;
    if (!d_scene || !d_out_rgba || ((uintptr_t)d_scene & 15u) || ((uintptr_t)d_out_rgba & 15u)) {
        set_error("nirc_estimate_frame_noalloc: NULL or misaligned scene/output pointer");
        return NIRC_ERR_INVALID;
    }
    if (fd.n_prims < 1 || fd.n_prims > NIRC_MAX_PRIMS || fd.n_cache > 1024 || fd.n_resid > 64 || fd.max_depth < 1 ||
        fd.max_depth > 64 || fd.cache_mode > 2 || P > 0xFFFFFFFFull) {
        set_error("nirc_estimate_frame_noalloc: argument out of range (n_prims 1..%u, N <= 1024, M <= 64, depth 1..64)",
                  NIRC_MAX_PRIMS);
        return NIRC_ERR_INVALID;
    }
    if (aux && ((aux->lc && ((uintptr_t)aux->lc & 3u)) || (aux->lr && ((uintptr_t)aux->lr & 3u)) ||
                (aux->sig && ((uintptr_t)aux->sig & 7u)) || (aux->count && ((uintptr_t)aux->count & 3u)) ||
                (aux->row_n && ((uintptr_t)aux->row_n & 3u)))) {
        set_error("nirc_estimate_frame_noalloc: misaligned aux pointer");
        return NIRC_ERR_INVALID;
    }
    const size_t rec_bytes = round256(P * sizeof(nirc_record));
    const size_t base_bytes = round256(P * sizeof(PixelBase));
    const size_t rows_bytes = round256(P * fd.n_resid * sizeof(ResidRow));
    const size_t need = rec_bytes + base_bytes + rows_bytes;
    if (need > kNoAllocScratchBytes) {
        set_error("nirc_estimate_frame_noalloc: frame needs %zu bytes of scratch (W*H*(96 + 32*M) rounded), more than "
                  "the fixed %zu-byte area; use nirc_estimate_frame or a smaller tile",
                  need, kNoAllocScratchBytes);
        return NIRC_ERR_BUDGET;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "nirc_estimate_frame_noalloc");
    unsigned char* sp = nullptr;
    const nirc_status st = scratch_address(dev, &sp);
    if (st != NIRC_OK) return st;
    // The path-tracing kernel writes every record, base and residual row that
    // the cache kernel reads, so no part of the array has to start at zero.
    nirc_record* recs = reinterpret_cast<nirc_record*>(sp);
    PixelBase* base = reinterpret_cast<PixelBase*>(sp + rec_bytes);
    ResidRow* rows = reinterpret_cast<ResidRow*>(sp + rec_bytes + base_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* sig = aux ? aux->sig : nullptr;
    uint32_t* count = aux ? aux->count : nullptr;
    timer_begin(h, NIRC_K_PATH_TRACE, s);
    e = launch_primary_resid(h, d_scene, fd, recs, base, rows, sig, count, s);
    timer_end(h, NIRC_K_PATH_TRACE, s);
    if (e != cudaSuccess) return cuda_status(e, "nirc_estimate_frame_noalloc (path tracing)");
    timer_begin(h, NIRC_K_CACHE, s);
    const bool tc = tc_supported(h, fd);
    if (tc) {
        e = launch_cache_tc(h, fd, recs, base, rows, d_out_rgba, aux ? aux->lc : nullptr, aux ? aux->lr : nullptr, sig,
                            count, aux ? aux->row_n : nullptr, h->dev_err, s);
    } else {
        e = launch_cache_simt(h, fd, recs, base, rows, d_out_rgba, aux ? aux->lc : nullptr, aux ? aux->lr : nullptr,
                              sig, count, aux ? aux->row_n : nullptr, s);
    }
    timer_end(h, NIRC_K_CACHE, s);
    if (e == cudaSuccess && tc) e = cudaMemcpyAsync(h->host_err, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    return cuda_status(e, "nirc_estimate_frame_noalloc (cache integral)");
}
