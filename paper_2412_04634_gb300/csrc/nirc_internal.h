// nirc_internal.h -- state of a cache handle and the kernel launchers the
// C-ABI layer (nirc_capi.cu) drives.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <string>

#include "nirc.h"
#include "nirc_device.cuh"

namespace nirc {

constexpr uint32_t kWidth = 64;
constexpr uint32_t kMaxHidden = 8;
constexpr uint32_t kMaxLevels = 16;
constexpr uint32_t kDirFeatures = 16;  // (theta, phi) x 4 octaves x (sin, cos)
constexpr uint32_t kNrmFeatures = 24;  // normal (3) x 4 octaves x (sin, cos)
constexpr uint32_t kShFeatures = 25;   // real spherical harmonics, degree <= 4
constexpr uint32_t kPhiFeatures = 15;  // albedo (3), one-blob normal angles (8), one-blob roughness (4)

// Per-pixel data the path-tracing kernel hands to the cache kernel.
struct __align__(16) PixelBase {
    float4 le;  // L_e(x, wo) of the camera hit (w unused)
    float4 wl;  // (1/M) sum_j w_j L_j: the path-traced part of L_r (w unused)
};

// One residual direction of a pixel.
struct __align__(16) ResidRow {
    float4 wi;  // direction, w = 1 if valid else 0
    float4 w;   // f_r cos / p (w unused)
};

// Network shape derived from a config.
struct NetShape {
    uint32_t n_pos;     // position features
    uint32_t n_dir;     // direction features: 16 (frequency) or 25 (spherical harmonics)
    uint32_t n_surf;    // per-surface features after the position: 24 (normal frequency) or 15 (phi)
    uint32_t sh;        // 1 = the paper's input (spherical harmonics + phi)
    uint32_t vis;       // 1 = visibility output (sigmoid, L2 loss)
    uint32_t n_in;      // network inputs = n_pos + n_dir + n_surf, in the order [pos][dir][surf]
    uint32_t n_pix;     // per-pixel features = n_pos + n_surf
    uint32_t hidden;    // hidden layers (>= 1)
    uint64_t n_mlp;     // MLP parameters in the master vector
    uint64_t n_hash;    // hash-table parameters
    uint64_t hash_off;  // device offset (floats) of the hash table: n_mlp rounded up to 4 (16-byte aligned)
    uint64_t n_dev;     // device floats of params / moments / gradients = hash_off + n_hash
    uint32_t log2_table;
    uint32_t levels;
    uint32_t hashgrid;  // 1 = hash grid, 0 = frequency encoding of x
    // Offsets (floats) in the packed FP32 SIMT weights:
    uint32_t off_wpix, off_wdir, off_b0, off_hidden, off_out, packed_floats;
};

struct GridParams {
    GridLevel level[kMaxLevels];
    uint32_t n_levels;
    uint32_t mask;  // T - 1
};

}  // namespace nirc

struct nirc_handle {
    nirc_config cfg;
    int device = 0;
    int num_sms = 0;
    nirc::NetShape shape{};
    nirc::GridParams grid{};
    float* params = nullptr;        // FP32 master parameters
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* grad = nullptr;
    float* packed = nullptr;        // transposed FP32 weights for the SIMT kernels
    __half* hash16 = nullptr;       // FP16 copy of the hash table (tensor-core path)
    void* packed_tc = nullptr;      // tensor-core operand images of the weights
    size_t packed_tc_bytes = 0;
    void* packed_tc16 = nullptr;    // FP16 image used to calibrate FP8 activation scales
    void* packed_train = nullptr;   // tensor-core training image (FP16 forward and backward); NULL: FP32 training
    uint32_t* fp8_amax = nullptr;   // [0,8) activation amax history, [8,16) current launch (float bits)
    bool fp8_calibrated = false;    // history valid for the current weights
    uint32_t step = 0;              // Adam steps taken
    void* scratch = nullptr;        // estimate_frame intermediates
    size_t scratch_bytes = 0;
    void* train_scratch = nullptr;  // training activations
    size_t train_scratch_bytes = 0;
    int store_activations = 1;      // 0: recompute activations chunk by chunk
    int deterministic = 0;          // 1: order-independent gradient sums
    uint64_t recompute_chunk = 1ull << 15;
    float* loss_accum = nullptr;    // one float
    unsigned long long* work_counter = nullptr;  // pixel counter of the path-tracing kernel
    int* dev_err = nullptr;         // device flag: a bounded wait ran out (1)
    int* host_err = nullptr;        // pinned copy of dev_err, refreshed after tensor-core launches
    // kernel timers (nirc_timing_enable / nirc_timing_read)
    bool timing = false;
    struct Pending {
        int cls;
        cudaEvent_t start, stop;
        uint64_t k0, kernels;  // n_kernels at the start; kernels launched in the interval
    };
    Pending* pending = nullptr;     // recorded, not yet read
    mutable uint64_t n_kernels = 0; // kernels launched by the handle so far
    // split frames (nirc_frame_desc.phase): the descriptor of the last traced frame
    bool traced = false;
    nirc_frame_desc traced_desc{};
    int n_pending = 0;
    cudaEvent_t* event_pool = nullptr;
    int n_pool = 0;
    double timing_ms[NIRC_K_CLASSES] = {};
    uint64_t timing_launches[NIRC_K_CLASSES] = {};
};

namespace nirc {

void set_error(const char* fmt, ...);
nirc_status cuda_status(cudaError_t e, const char* what);

// Bracket one kernel launch with timer events when timing is enabled.
// Every kernel launch of the library is followed by count_kernels (the
// timers report kernels per class, not intervals).
inline void count_kernels(const nirc_handle* h, uint32_t k = 1) { h->n_kernels += k; }
void timer_begin(const nirc_handle* h, int cls, cudaStream_t st);
void timer_end(const nirc_handle* h, int cls, cudaStream_t st);

NetShape make_shape(const nirc_config& cfg);
GridParams make_grid(const nirc_config& cfg);

// nirc_pt.cu
// mv_* (multi-vertex estimator, else NULL): [2][W H M] records, throughputs and continuation rows
cudaError_t launch_primary_resid(const nirc_handle* h, const void* scene, const nirc_frame_desc& fd,
                                 nirc_record* recs, PixelBase* base, ResidRow* rows, uint64_t* sig,
                                 uint32_t* count, cudaStream_t st, nirc_record* mv_rec = nullptr,
                                 float4* mv_beta = nullptr, ResidRow* mv_row = nullptr,
                                 unsigned long long* rays = nullptr);
// Multi-vertex estimator: out (RGBA) and lr (RGB, may be NULL) of pixel p gain
// sum over j of o2[p M + j] + o3[p M + j] (either may be NULL).
cudaError_t launch_mv_accumulate(float* out_rgba, float* lr, const float4* o2, const float4* o3, uint64_t P,
                                 uint32_t M, cudaStream_t st);
cudaError_t launch_primary_bth(const nirc_handle* h, const void* scene, const nirc_frame_desc& fd, nirc_record* recs,
                               PixelBase* base, float4* beta, uint64_t* sig, uint32_t* count, cudaStream_t st,
                               unsigned long long* rays = nullptr);
cudaError_t launch_gen_train(const nirc_handle* h, const void* scene, uint32_t n_prims, uint32_t W, uint32_t H,
                             uint64_t T, uint32_t frame, uint64_t seed, uint32_t max_depth, uint32_t light_mode,
                             nirc_record* recs, float* dirs, float* targets, cudaStream_t st);

// nirc_cache_simt.cu
// Which cache samples a launch of the cache integral draws: unit u's row i
// takes Philox counter (u / unit_div, ((u % unit_div) << 16) | i) and
// purpose `purpose`.  The shading-point pass: {1, PURPOSE_CACHE_DIR}; the
// later-vertex passes of the multi-vertex estimator: {M, PURPOSE_VCACHE + 16 k}.
struct CachePass {
    uint32_t unit_div = 1;
    uint32_t purpose = PURPOSE_CACHE_DIR;
};

// beta (biased and multi-vertex estimators, else NULL): per-unit throughput
// applied to both levels; base NULL: zero emission and path-traced part.
// env (light mode 2 with a visibility cache, else empty): the scene whose
// cube map multiplies every cache value (L_env of the row's direction).
struct EnvSource {
    const void* scene = nullptr;
    uint32_t n_prims = 0;
};
cudaError_t launch_cache_simt(const nirc_handle* h, const nirc_frame_desc& fd, const nirc_record* recs,
                              const PixelBase* base, const ResidRow* rows, const float4* beta, float* out_rgba,
                              float* lc, float* lr, uint64_t* sig, uint32_t* count, float* row_n, cudaStream_t st,
                              CachePass pass = CachePass{}, EnvSource env = EnvSource{});
cudaError_t launch_query_simt(const nirc_handle* h, const nirc_record* recs, const float* dirs, uint64_t n,
                              float* out, cudaStream_t st);
cudaError_t launch_repack_simt(const nirc_handle* h, cudaStream_t st);

// nirc_cache_tc.cu
size_t tc_image_bytes(uint32_t hidden);
cudaError_t launch_repack_tc(const nirc_handle* h, cudaStream_t st);
bool tc_supported(const nirc_handle* h, const nirc_frame_desc& fd);
cudaError_t launch_cache_tc(const nirc_handle* h, const nirc_frame_desc& fd, const nirc_record* recs,
                            const PixelBase* base, const ResidRow* rows, const float4* beta, float* out_rgba,
                            float* lc, float* lr, uint64_t* sig, uint32_t* count, float* row_n, int* err,
                            cudaStream_t st, CachePass pass = CachePass{}, EnvSource env = EnvSource{});

// nirc_cache_tc.cu: the FP16 cache image (forward part of the training image)
cudaError_t launch_repack_fwd16(const nirc_handle* h, uint8_t* img, cudaStream_t st);

// nirc_train_tc.cu: the training step's forward and backward on the tensor cores
// Training buffers of one chunk: encodings, activations and deltas as
// [feature][ld] columns, dL/dz as [3][dz_ld].
struct TrainPtrs {
    float* e;      // [n_in][ld]
    float* act;    // [hidden][64][ld]
    float* delta;  // [hidden][64][ld]
    uint64_t ld;
    float* dz;     // [3][dz_ld]
    uint64_t dz_ld;
};
size_t train_tc_image_bytes(uint32_t hidden);
bool train_tc_shape_ok(const NetShape& s);
bool train_tc_supported(const nirc_handle* h);
cudaError_t launch_repack_train(const nirc_handle* h, cudaStream_t st);
cudaError_t launch_train_tc(const nirc_handle* h, const nirc_record* recs, const float* dirs, const float* targets,
                            uint64_t m, float scale, const TrainPtrs& tp, float* grad_table, float* loss_accum,
                            cudaStream_t st);

// nirc_train.cu
size_t train_scratch_bytes(const nirc_handle* h, uint64_t n);
cudaError_t launch_train_step(nirc_handle* h, const nirc_record* recs, const float* dirs, const float* targets,
                              uint64_t n, float* d_loss, cudaStream_t st);
cudaError_t launch_query_bwd(nirc_handle* h, const nirc_record* recs, const float* dirs, const float* grad_out,
                             uint64_t n, float* d_value, cudaStream_t st);
cudaError_t launch_hash_to_half(const nirc_handle* h, cudaStream_t st);

// nirc_capi.cu: shared by the public frame entry points and the server.
// Frame scratch = records | per-pixel bases | residual rows, each part
// rounded up to 256 bytes.
size_t frame_scratch_bytes(uint64_t P, uint32_t M, uint32_t estimator);
// Argument checks of a frame call (message prefixed with `who`).
nirc_status check_frame_args(const char* who, const void* scene, const nirc_frame_desc& fd, const float* out,
                             const nirc_frame_aux* aux);
// Enqueue the path-tracing and cache-integral kernels of one frame on `st`
// with the given scratch (frame_scratch_bytes bytes).
nirc_status enqueue_frame(const char* who, const nirc_handle* h, const void* scene, const nirc_frame_desc& fd,
                          float* out, const nirc_frame_aux* aux, void* scratch, cudaStream_t st);
// Grow the handle's training scratch for batches of n (cudaMalloc).
nirc_status reserve_train_scratch(nirc_handle* h, uint64_t n);

// Frames of several caches in one launch per kernel (the frame-request
// server's batches): two-level estimator, whole frames, light modes 0 and 1
// (one light mode per path-tracing launch), one tensor-core precision and
// network shape across the cache launch (tc_batchable).
constexpr uint32_t kMaxFrameJobs = 16;
struct FrameJob {
    const nirc_handle* h;
    nirc_frame_desc fd;
    const void* scene;
    nirc_record* recs;          // frame scratch, as enqueue_frame carves it
    PixelBase* base;
    ResidRow* rows;
    float* out;                 // RGBA image
    unsigned long long* work;   // the path tracer's pixel counter, zeroed before the launch
};
cudaError_t launch_primary_resid_batch(const FrameJob* fj, uint32_t n, cudaStream_t st);  // nirc_pt.cu
bool tc_batchable(const nirc_handle* a, const nirc_handle* b);                             // nirc_cache_tc.cu
cudaError_t launch_cache_tc_batch(const FrameJob* fj, uint32_t n, cudaStream_t st);       // nirc_cache_tc.cu

// nirc_metrics.cu
cudaError_t launch_mrse(const float* img, const float* ref, uint64_t n, float eps, double* out, cudaStream_t st);

}  // namespace nirc
