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
// device current) and later calls reuse it for the life of the process (a
// cudaDeviceReset invalidates it, as it invalidates every handle's device
// memory).  All calls on a device share the
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
    nirc_status st = check_frame_args("nirc_estimate_frame_noalloc", d_scene, fd, d_out_rgba, aux);
    if (st != NIRC_OK) return st;
    if (fd.phase != NIRC_PHASE_ALL) {
        set_error("nirc_estimate_frame_noalloc: split frames (phase != 0) are not supported here");
        return NIRC_ERR_INVALID;
    }
    const size_t need = frame_scratch_bytes(P, fd.n_resid, fd.estimator);
    if (need > kNoAllocScratchBytes) {
        static const char* const names[3] = {"two-level, W*H*(96 + 32*M)", "biased BTH, W*H*112",
                                             "multi-vertex, W*H*(96 + 288*M)"};
        set_error("nirc_estimate_frame_noalloc: a %ux%u frame (estimator %u: %s, M = %u) needs %zu bytes of scratch, "
                  "more than the fixed %zu-byte area; use nirc_estimate_frame or a smaller tile",
                  fd.width, fd.height, fd.estimator, fd.estimator < 3 ? names[fd.estimator] : "?", fd.n_resid, need,
                  kNoAllocScratchBytes);
        return NIRC_ERR_BUDGET;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "nirc_estimate_frame_noalloc");
    unsigned char* sp = nullptr;
    st = scratch_address(dev, &sp);
    if (st != NIRC_OK) return st;
    return enqueue_frame("nirc_estimate_frame_noalloc", h, d_scene, fd, d_out_rgba, aux, sp, (cudaStream_t)stream);
}
