/*
 * nirc.h -- C ABI of libnirc.so, the GB300 (sm_103a) implementation of the
 * Neural Incident Radiance Cache (NIRC) two-level Monte Carlo hot path of
 * "Neural Two-Level Monte Carlo Real-Time Rendering" (arXiv 2412.04634).
 *
 * The method (paper section "Neural Incident Radiance Cache"): split the
 * rendering equation's integral into a cache level and a residual level,
 *   L_o = L_e + L_c + L_r                                         (eq. L_mlmc)
 *   L_c = 1/N sum_i n(x, w_i) f_r cos / p(w_i)                    (eq. L_c)
 *   L_r = 1/M sum_j (L_i(x, w_j) - n(x, w_j)) f_r cos / p(w_j)    (eq. L_r)
 * where n is a small MLP over encodings of position, incident direction and
 * surface features (the cache, eq. 11), the two direction sets are drawn
 * independently by BSDF importance sampling (section "Cache application"),
 * and the cache is trained on-line with the relative L2 loss (eq. 12) by
 * Adam on paths from a separate training pass.
 *
 * Conventions for every call:
 *  - Pointers named d_* are DEVICE memory owned by the caller; the library
 *    never frees them and keeps no reference after the call returns.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and is stream-ordered; calls return before the GPU finishes.
 *  - Every call returns a status and never aborts the process.  On error
 *    nirc_last_error() gives a message (thread-local); a failing call leaves
 *    the handle's parameters and optimiser state unchanged unless the
 *    failure is a CUDA error raised by already-enqueued work.
 *  - Calls on one handle are not re-entrant; separate handles are
 *    independent.
 *  - Sizes of 0 are valid no-ops.
 */
#ifndef NIRC_H
#define NIRC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nirc_status {
    NIRC_OK = 0,
    NIRC_ERR_INVALID = 1,     /* bad argument (null pointer, size, config) */
    NIRC_ERR_OOM = 2,         /* device allocation failed */
    NIRC_ERR_BUDGET = 3,      /* request exceeds a documented size limit */
    NIRC_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    NIRC_ERR_TIMEOUT = 5,     /* a bounded device wait ran out */
    NIRC_ERR_UNSUPPORTED = 6  /* configuration not implemented on this path */
} nirc_status;

/* Arithmetic of the network layers (section "Neural Network Architecture").
 * FP32_SIMT: plain FP32 FMA kernels.  FP16_TC: tcgen05 tensor-core MMAs with
 * FP16 operands and FP32 accumulation in tensor memory.  BF16_TC: the same
 * with every operand carried as two BF16 values, hi = bf16(x) and lo =
 * bf16(x - hi), and each product formed as hi*hi + lo*hi + hi*lo (about 16
 * significant bits, three MMAs per product; BF16's own 8 bits do not meet
 * 2e-2 on n = exp(z) for trained logits).  FP8_E4M3_TC: the hidden 64x64 layers
 * take E4M3 operands (kind::f8f6f4) with per-layer scales, weights scaled
 * by amax|W| / 448 and activations by the amax of the previous launch / 448
 * (delayed scaling; the first launch after new weights or a precision change
 * runs one extra FP16 pass to measure it), FP32 accumulation; the first
 * layer and the output layer stay FP16.  Encodings, sampling, pdfs and the
 * Kahan-compensated per-pixel sums are FP32 in every mode. */
typedef enum nirc_precision {
    NIRC_FP32_SIMT = 0,
    NIRC_FP16_TC = 1,
    NIRC_BF16_TC = 2,
    NIRC_FP8_E4M3_TC = 3
} nirc_precision;

typedef enum nirc_pos_encoding {
    NIRC_POS_FREQ = 0,     /* 4-octave sin/cos of x (the 64x64 workload) */
    NIRC_POS_HASHGRID = 1  /* multiresolution hash grid of x (paper: section
                              "Neural Network Architecture", first bullet) */
} nirc_pos_encoding;

typedef enum nirc_output {
    NIRC_OUT_RADIANCE = 0,   /* n = exp(min(z, z_clamp)), relative L2 loss (eq. 12) */
    NIRC_OUT_VISIBILITY = 1  /* the Neural Visibility Cache: V = 1 / (1 + exp(-z))
                                per channel (a sigmoid on the output neurons),
                                loss mean (f - V)^2 over records and channels */
} nirc_output;

typedef enum nirc_input_encoding {
    NIRC_INPUT_FREQ = 0,  /* direction (theta/pi, phi/2pi) and normal by
                             frequency features (the 64x64 and 1080p workloads) */
    NIRC_INPUT_SH = 1     /* the paper's input (section "Neural Network
                             Architecture", encoding bullets and the system
                             figure's 24 + 25 + 15 inputs): direction by the 25
                             real spherical harmonics of degree <= 4, and
                             phi = albedo (3), one-blob normal angles (2 x 4)
                             and one-blob roughness (4) */
} nirc_input_encoding;

/* Cache hyper-parameters.  Network input, in order: position features
 * (3 dims x 2 x freq_octaves, or hash_levels x feats_per_level), then
 * direction and per-surface features by `input_encoding`:
 *  NIRC_INPUT_FREQ: the incident direction as (theta/pi, phi/2pi) with
 *   2 x 2 x freq_octaves features, and the shading normal with
 *   3 x 2 x freq_octaves features.  Frequency features of a scalar v are
 *   sin(2^k pi v), cos(2^k pi v).
 *  NIRC_INPUT_SH: Y_l^m(w), l = 0..4, at index l*l + l + m (orthonormal
 *   real harmonics: sqrt(2) K_l^m P_l^m(cos t) cos(m p) for m > 0, sin(|m| p)
 *   for m < 0, no Condon-Shortley phase); then albedo, the one-blob
 *   encodings of the normal's theta/pi and phi/2pi and of the roughness, each
 *   4 bins holding the mass of a Gaussian of standard deviation 1/4 centred
 *   at the value over [i/4, (i+1)/4) (no wrap-around).  Needs
 *   position features + 15 <= 64.
 * Hidden layers: `hidden_layers` ReLU layers of `width` (only 64 is
 * supported), output 3 logits z, cache value n = exp(min(z, z_clamp)). */
typedef struct nirc_config {
    uint32_t pos_encoding;     /* nirc_pos_encoding */
    uint32_t hash_levels;      /* L, e.g. 16 */
    uint32_t feats_per_level;  /* F, only 2 supported */
    uint32_t log2_table;       /* T = 2^log2_table entries per level, e.g. 19 */
    uint32_t base_res;         /* N_min, e.g. 16 */
    float growth;              /* b: level resolution floor(N_min * b^l) */
    uint32_t freq_octaves;     /* only 4 supported */
    uint32_t width;            /* only 64 supported */
    uint32_t hidden_layers;    /* 1..8 */
    uint32_t precision;        /* nirc_precision */
    float lr;                  /* Adam learning rate (paper: 0.01) */
    float beta1, beta2;        /* Adam moments, e.g. 0.9, 0.99 */
    float adam_eps;            /* e.g. 1e-15 */
    float loss_eps;            /* eps of eq. 12, e.g. 0.01 */
    float z_clamp;             /* e.g. 15 */
    uint32_t input_encoding;   /* nirc_input_encoding */
    uint32_t output;           /* nirc_output */
} nirc_config;

/* Shading record: one surface point (paper: "surface parameter buffer",
 * section "Memory consumption").  64 bytes, 16-byte aligned.
 * flags bit 0 = valid, bits 1-2 = material (0 Lambertian, 1 Lambertian +
 * GGX, 2 black/non-scattering).  n is the unit shading normal facing wo. */
typedef struct nirc_record {
    float p[3];
    float n[3];
    float wo[3];
    float albedo[3];
    float roughness;
    uint32_t prim;
    uint32_t flags;
    uint32_t pad;
} nirc_record;

/* One frame of the two-level estimator.
 * Scene blob (device): 96-byte header {u32 n_prims, u32 pad[3],
 * f32 cam_origin[4], f32 cam_top_left[4], f32 cam_horizontal[4],
 * f32 cam_vertical[4], u32 reserved[4]} followed by n_prims 96-byte
 * primitives {f32 a[3], radius, u[3], inv_uu, v[3], inv_vv, n[3], u32 kind,
 * f32 albedo[3], roughness, emission[3], u32 flags}; kind 0 sphere (centre
 * a), 1 rectangle (corner a, perpendicular edges u, v, unit normal n);
 * flags bits 0-1 material, bit 8 two-sided emission.  The blob must be
 * 16-byte aligned and hold at least n_prims primitives.  Environment map
 * (light mode 2): header word reserved[0] = cube face size S (0: none) and
 * 6 S S texels {f32 rgb[3], pad} after the primitives, face-major (0 +x,
 * 1 -x, 2 +y, 3 -y, 4 +z, 5 -z), then row, then column; direction d picks
 * the face of its largest |component| (ties: x, then y, then z) and, with
 * (a, b) its other two components in axis order, column
 * floor((a / |major| + 1) / 2 * S) and row floor((b / |major| + 1) / 2 * S)
 * (clamped to S - 1), in binary32; L_env(d) is that texel (nearest). */
typedef struct nirc_frame_desc {
    uint32_t width, height;  /* W, H; pixel index = y * W + x, row 0 at top */
    uint32_t n_cache;        /* N cache-level samples per pixel (0..1024) */
    uint32_t n_resid;        /* M residual samples per pixel (0..64) */
    uint32_t max_depth;      /* path segments of a residual path (1..64) */
    uint32_t frame;          /* Philox key word 1 */
    uint64_t seed;           /* Philox key word 0 = low 32 bits */
    uint32_t n_prims;        /* primitives in the scene blob (1..NIRC_MAX_PRIMS) */
    uint32_t cache_mode;     /* 0 network, 1 zero cache (n = 0: plain path
                                tracing), 2 constant cache n = cache_const */
    float cache_const[3];
    uint32_t light_mode;     /* 0: the cache and the residual paths carry the
                                full incident radiance, pure BSDF paths.
                                1: L_i = L_ind + L_nee (eq. Lsplit): direct
                                light by next-event estimation on emitting
                                rectangles (one light sample at the shading
                                point and at every path vertex) combined with
                                BSDF sampling by the power heuristic (the M
                                residual directions are the BSDF technique at
                                the shading point); cache, residual paths and
                                training targets carry L_ind.  Spherical
                                emitters are reached by BSDF sampling only.
                                2: direct environment light (section
                                "Neural Visibility Cache"): the frame is
                                L_e(x) + the two levels of
                                f cos V(x, w) L_env(w): residual rows trace
                                one ray (V = 1 when it leaves the scene), the
                                cache value is V^(x, w) L_env(w) for a
                                visibility cache (NIRC_OUT_VISIBILITY) or the
                                network's radiance otherwise (the generic
                                NIRC on the same task); two-level estimator
                                only. */
    uint32_t estimator;      /* nirc_estimator */
    uint32_t n_cache2;       /* NIRC_EST_MULTI_VERTEX: cache samples at the */
    uint32_t n_cache3;       /* second and third vertex (0..1024) */
    uint32_t phase;          /* NIRC_PHASE_ALL (0): the whole estimate.
                                NIRC_PHASE_TRACE (1): only the path-tracing
                                pass (camera hits, shading records, residual
                                paths) into the handle's frame scratch;
                                d_out_rgba may be NULL and is not written.
                                NIRC_PHASE_CACHE (2): only the cache integral
                                and the per-pixel sums, over the scratch of
                                the handle's last NIRC_PHASE_TRACE call,
                                whose descriptor must equal this one apart
                                from the phase (else NIRC_ERR_INVALID); pass
                                the same scene and aux.  The path-tracing
                                pass reads no cache weights, so a caller can
                                trace frame f + 1 while training on frame f
                                (on another stream, after frame f's cache
                                pass, which reads the scratch).  A
                                NIRC_PHASE_ALL call ends the traced state.
                                nirc_estimate_frame_noalloc and the server
                                take NIRC_PHASE_ALL only. */
} nirc_frame_desc;

enum { NIRC_PHASE_ALL = 0, NIRC_PHASE_TRACE = 1, NIRC_PHASE_CACHE = 2 };

/* Estimator of nirc_frame_desc.estimator.
 * NIRC_EST_TWO_LEVEL: eq. L_mlmc at the first camera hit (N cache samples,
 *   M residual paths): unbiased.  With N = 0 there is no cache level and no
 *   cache value is subtracted (plain path tracing).
 * NIRC_EST_MULTI_VERTEX: the paper's unbiased variant ("Biased and unbiased
 *   variants": NIRC at the first three vertices, the neural samples
 *   redistributed between them): the same at the shading point x_1, and
 *   along each residual path at its vertices x_2 and x_3 the path's
 *   incident-radiance estimate gains beta_k C_k - beta_{k+1} n(x_k, w_k):
 *   C_k = 1/N_k sum_i (f cos / p)_i n(x_k, w_i) over N_k = n_cache2 /
 *   n_cache3 BSDF-sampled directions (Philox purpose 10 + 16 k, counter
 *   (pixel, j << 16 | i) for residual path j), minus the cache value of the
 *   path's continuation direction w_k (only when it continues; beta_{k+1}
 *   includes the continuation weight and Russian roulette), beta_k the
 *   path's throughput to x_k times w_j / M.  Zero mean for any cache;
 *   vertices with N_k = 0 use no cache.  The terms count in lr; count,
 *   sig[1] and row_n describe x_1's cache samples.
 * NIRC_EST_BIASED_BTH: the paper's biased variant (section "Path
 *   Termination Heuristics", paragraph "Biased and unbiased variants"): the
 *   camera path continues from vertex x_i with its BSDF-sampled direction
 *   w_i (Philox purpose 8 + 16 i) unless xi_i (purpose 9 + 16 i) > P_s =
 *   p / (p + N / pi), p the sampler's density of w_i (Balanced Termination
 *   Heuristic), or, for i > 1, NRC's footprint
 *   a = (sum_k sqrt(|x_{k-1} - x_k|^2 / (p_{k-1} cos_k)))^2 exceeds
 *   0.01 |x_0 - x_1|^2 / (4 pi cos_1), or i = max_depth.  At the stopping
 *   vertex N cache samples complete the outgoing radiance, times the path
 *   throughput; emission found along the path is added; light mode 1 adds a
 *   light sample at every vertex and uses w_i as the BSDF technique (one
 *   sample, traced at the stopping vertex for its emission only).  No
 *   Russian roulette, no residual level: requires n_resid = 0.  The
 *   decisions (p, P_s, the footprint) are strict binary32.  lc = throughput
 *   x cache level at the stopping vertex, lr = 0. */
typedef enum nirc_estimator {
    NIRC_EST_TWO_LEVEL = 0,
    NIRC_EST_BIASED_BTH = 1,
    NIRC_EST_MULTI_VERTEX = 2
} nirc_estimator;

#define NIRC_MAX_PRIMS 1024u

/* Optional per-pixel outputs of nirc_estimate_frame (device pointers, any
 * may be NULL): lc, lr = the two levels (W*H x 3 floats); sig = two 64-bit
 * FNV-1a signatures per pixel of the discrete decisions (path: primary hit,
 * residual directions, hits, Russian roulette; cache: cache-direction
 * rejection counts and lobes); count = valid (active) samples per pixel;
 * row_n = the cache value n of every row, W*H*(N+M) x 3 floats in pixel-major,
 * sample-minor order (cache samples first), 0 for rows whose sample is
 * invalid (network mode only); rays (one device uint64, not cleared) gains
 * the number of rays the path-tracing pass traced (camera rays, path
 * segments, shadow and visibility rays). */
typedef struct nirc_frame_aux {
    float* lc;
    float* lr;
    uint64_t* sig;
    uint32_t* count;
    float* row_n;
    uint64_t* rays;
} nirc_frame_aux;

typedef struct nirc_handle nirc_handle;

/* Number of parameters of a configuration: for each layer W (fan_out x
 * fan_in, row-major) then b (fan_out), input layer first, then the hash
 * table [level][entry][feature] (hash-grid configs only). */
uint64_t nirc_param_count(const nirc_config* cfg);

/* Create a cache with zero parameters on the current CUDA device.  The
 * handle owns the FP32 master parameters, their FP16/BF16 copies, the Adam
 * moments, gradients and scratch.  Returns NIRC_ERR_UNSUPPORTED for widths
 * other than 64, more than 8 hidden layers or other feature counts. */
nirc_status nirc_create(const nirc_config* cfg, nirc_handle** out);
nirc_status nirc_destroy(nirc_handle* h);

/* Copy nirc_param_count() floats in (host or device pointer per
 * `on_device`), refresh the low-precision copies and reset Adam (step 0,
 * zero moments). */
nirc_status nirc_set_params(nirc_handle* h, const float* params, int on_device, void* stream);
/* Copy nirc_param_count() floats in and refresh the low-precision copies,
 * keeping the Adam moments and step (for callers that update the weights
 * with their own optimiser, e.g. through the autograd wrapper).  Host input
 * synchronises `stream`. */
nirc_status nirc_load_params(nirc_handle* h, const float* params, int on_device, void* stream);
/* Copy the FP32 master parameters out. Synchronises `stream` for host output. */
nirc_status nirc_get_params(nirc_handle* h, float* out, int on_device, void* stream);
/* Copy out the gradient of the last nirc_train_step (same layout). */
nirc_status nirc_get_grads(nirc_handle* h, float* out, int on_device, void* stream);
/* Checkpoint / resume of a cache: nirc_state_bytes() bytes of host memory
 * hold a header (magic "NIRCSTAT", format version, the nirc_config, the
 * Adam step count) followed by the FP32 master parameters, Adam m and v in
 * the nirc_param_count() layout.  nirc_save_state synchronises `stream`
 * and writes `host_buf`; nirc_load_state reads it back (the handle must
 * have the same configuration apart from precision and learning-rate
 * fields: NIRC_ERR_INVALID otherwise, handle unchanged), restores weights,
 * moments and step exactly and refreshes the low-precision copies.
 * Training after a load continues bit for bit as it would have without the
 * save (deterministic mode). */
uint64_t nirc_state_bytes(const nirc_handle* h);
nirc_status nirc_save_state(nirc_handle* h, void* host_buf, uint64_t bytes, void* stream);
nirc_status nirc_load_state(nirc_handle* h, const void* host_buf, uint64_t bytes, void* stream);

/* Select the layer arithmetic for later calls (nirc_precision).  The
 * tensor-core modes apply to the cache integral of nirc_estimate_frame when
 * the network is used (cache_mode 0) and N + M >= 4 (N + M >= 1 with
 * NIRC_INPUT_SH); other work (queries,
 * training, the other cache modes) runs the FP32 kernels.  Synchronises the
 * legacy default stream. */
nirc_status nirc_set_precision(nirc_handle* h, uint32_t precision);

/* Wait for `stream` and report device-side failures of the handle's
 * kernels: NIRC_ERR_TIMEOUT if a tensor-core kernel's bounded wait for an
 * MMA ran out (about 2 s; that launch's output is invalid). */
nirc_status nirc_sync(nirc_handle* h, void* stream);

/* Bare cache queries (eq. 11's n_i): d_out_rgb[i] = n(record_i, dir_i),
 * n rows, d_dirs = n x 3 unit world directions, d_out_rgb = n x 3. */
nirc_status nirc_query(nirc_handle* h, const nirc_record* d_records, const float* d_dirs, uint64_t n,
                       float* d_out_rgb, void* stream);

/* One frame of the two-level estimator (eq. L_mlmc, L_c, L_r) at one shading
 * point per pixel (the first camera hit, 1 spp): camera ray, N cache samples
 * and M residual samples drawn independently by BSDF sampling, M residual
 * paths traced with Russian roulette (continue with probability 0.9) up to
 * max_depth segments, cache evaluated at all N + M directions.
 * d_out_rgba = W*H float4 (alpha = 1).  Returns NIRC_ERR_BUDGET when the
 * scratch for W*H*(N+M) rows cannot be allocated. */
nirc_status nirc_estimate_frame(nirc_handle* h, const void* d_scene, const nirc_frame_desc* desc,
                                float* d_out_rgba, const nirc_frame_aux* aux, void* stream);

/* nirc_estimate_frame for callers that cannot allocate device memory during
 * the call (the paper has no counterpart: it is an interface addition).
 * nirc_estimate_frame grows handle-owned scratch with cudaMalloc the first
 * time a larger frame arrives; callers that have reserved all device memory
 * up front, real-time frame loops that must not pay cudaMalloc/cudaFree's
 * implicit synchronisation, or applications whose allocation policy forbids
 * it use this entry point instead.  It runs the same kernels, with the same
 * arguments and results, on a fixed 4 MiB scratch area compiled into the
 * library, and calls no cudaMalloc, cudaFree or other allocating routine.
 * Limit, per estimator (P = W * H; each part rounded up to 256 bytes; the
 * sum must fit in 4 MiB, larger frames return NIRC_ERR_BUDGET and the error
 * string names the estimator and the bytes needed):
 *   NIRC_EST_TWO_LEVEL     P * (96 + 32 M)   e.g. 32,768 pixels at M = 1
 *   NIRC_EST_BIASED_BTH    P * 112           e.g. about 37,400 pixels
 *   NIRC_EST_MULTI_VERTEX  P * (96 + 288 M)  e.g. about 10,900 pixels at M = 1
 * The first call on each device looks up the area's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process; make that first call before any stream capture, and do
 * not use the library across a cudaDeviceReset (which invalidates the
 * address, as it does every handle's device memory).  Every call on a device
 * shares the area and it keeps the last call's contents: calls that overlap
 * on the GPU race on it, so order them on one stream.  Every GPU that loads
 * the library holds the 4 MiB until the process exits. */
nirc_status nirc_estimate_frame_noalloc(nirc_handle* h, const void* d_scene, const nirc_frame_desc* desc,
                                        float* d_out_rgba, const nirc_frame_aux* aux, void* stream);

/* Training records from a separate path-tracing pass (section "Cache
 * application"): T paths, each from a uniformly drawn pixel, one record per
 * path at its first hit with the BSDF-sampled direction and the path-traced
 * incident radiance as target.  Records whose path has no usable direction
 * get flags bit 0 cleared (excluded from the loss).  Philox key word 1 is
 * frame ^ 0x80000000 so training draws never repeat rendering draws.
 * light_mode as in nirc_frame_desc (1: targets are L_ind estimates with NEE
 * + MIS along the path; 2: one ray, target V L_env along it, or V in all
 * three channels for a visibility cache).  d_records = T x 64 B,
 * d_dirs = T x 3, d_targets = T x 3. */
nirc_status nirc_gen_train(nirc_handle* h, const void* d_scene, uint32_t n_prims, uint32_t width,
                           uint32_t height, uint64_t T, uint32_t frame, uint64_t seed, uint32_t max_depth,
                           uint32_t light_mode, nirc_record* d_records, float* d_dirs, float* d_targets,
                           void* stream);

/* One Adam step on the relative L2 loss of eq. 12 with p_r = 1:
 *   L = 1/(3n) sum_t sum_rgb valid_t (f - n)^2 / (sg(n)^2 + loss_eps)
 * over n records (forward, backward through the MLP and the encoding, hash
 * table gradient scatter, dense bias-corrected Adam over all parameters).
 * d_loss (optional, device float) receives L. */
nirc_status nirc_train_step(nirc_handle* h, const nirc_record* d_records, const float* d_dirs,
                            const float* d_targets, uint64_t n, float* d_loss, void* stream);

/* Activation memory of nirc_train_step and nirc_query_bwd.  store != 0
 * (default): the forward stores every layer's output for the whole batch,
 * n * (n_in + 128 * hidden_layers) floats.  store == 0: the forward keeps
 * only dL/dz (3 floats per sample) and the backward walks the batch in
 * chunks of `recompute_chunk` samples (1024..2^26), running each chunk's
 * forward again into a chunk-sized buffer before its backward, one extra
 * forward in exchange for O(chunk) memory.  Results agree up to the order of
 * the float atomics in the gradient sums. */
nirc_status nirc_set_train_mode(nirc_handle* h, int store_activations, uint64_t recompute_chunk);

/* Arithmetic of nirc_train_step's forward and backward through the MLP.
 * NIRC_FP32_SIMT (default): FP32 on the CUDA cores.  NIRC_FP16_TC: one
 * tensor-core kernel per chunk runs the forward (FP16 operands, FP32
 * accumulation in tensor memory, the same weight image as the FP16 frame
 * path), the loss of eq. 12, and the backward of every layer (FP16
 * operands; each record's delta row is scaled by an exact power of two
 * into FP16's range and scaled back after the MMA); the hash-table scatter
 * (warp-aggregated atomics) and Adam stay FP32, and the weight and bias
 * gradients of every layer are one more tensor-core kernel (BF16 operands
 * rounded from the stored FP32 activations and deltas, FP32 accumulation,
 * a row of ones giving the bias sums).  The hash-grid features come from the FP16 copy of the
 * table, as in the FP16 frame path.  Weight gradients agree with the FP32
 * ones to about 1e-3 of their maximum; the hash-table gradient to about
 * 1e-3 (relative L2 norm) for records whose pre-activations are not within
 * FP16 rounding of a ReLU kink, and a few percent over batches where many
 * are (such a record's ReLU can switch, which moves the few table entries
 * around it).  NIRC_K_TRAIN_FWD times the kernel (forward and backward).
 * Applies to the relative L2
 * loss only: nirc_query_bwd and deterministic training keep FP32.  Any
 * other value returns NIRC_ERR_INVALID; NIRC_ERR_UNSUPPORTED for a network
 * the kernel does not cover (hidden_layers > 8, or position features other
 * than 24 or 32: the frequency encoding, or 12 or 16 hash-grid levels).
 * Allocates the training weight image (about 100 KB) on first use. */
nirc_status nirc_set_train_precision(nirc_handle* h, uint32_t precision);

/* Deterministic training (on != 0): nirc_train_step and nirc_query_bwd give
 * bit-identical losses, gradients and weights for identical inputs and
 * state, however the GPU schedules the work (the default sums gradients with
 * float atomics, whose order varies; with Adam's sign-like first steps that
 * moves near-zero-gradient parameters by +-lr between runs).  Weight
 * gradients and the loss are summed from per-block partials in a fixed
 * order; the hash-table gradient is accumulated in 64-bit fixed point with a
 * power-of-two scale per level (2^61 / (8 n max|dL/de|) rounded down), so
 * each contribution keeps FP32 relative precision and the sum is exact.
 * Costs extra scratch (2 x levels floats per sample, 8 bytes per table
 * entry) and one more pass over the table gradient. */
nirc_status nirc_set_deterministic(nirc_handle* h, int on);

/* Backward of the bare query (for a torch.autograd.Function around
 * nirc_query): with d_grad_out = dL/dn (n x 3 floats, device) it computes
 * d_grad_params = sum_i dL/dn_i . dn_i/dparams over every row (the valid flag
 * is ignored, as in nirc_query), through the output exp and clamp, the ReLU
 * layers, the frequency encodings and the trilinear hash-grid interpolation
 * (table gradient scattered with warp-aggregated atomics).  The gradient is
 * left in the handle's gradient buffer (nirc_get_grads; it replaces the last
 * training gradient) and, when d_grad_params != NULL, copied there in the
 * nirc_param_count() layout (device pointer).  d_value (optional, device
 * float) receives sum dL/dn * n.  Same FP32 arithmetic as nirc_query. */
nirc_status nirc_query_bwd(nirc_handle* h, const nirc_record* d_records, const float* d_dirs,
                           const float* d_grad_out, uint64_t n, float* d_grad_params, float* d_value, void* stream);

/* Mean relative squared error over pixels and RGB (paper: MRSE),
 * mean (I - R)^2 / (R^2 + eps); each term in binary32, the sum accumulated
 * with about 48 significant bits (per-thread compensated binary32 pairs,
 * combined in FP64); images are float4 per pixel (alpha ignored); d_out =
 * one device double. */
nirc_status nirc_frame_mrse(const float* d_img_rgba, const float* d_ref_rgba, uint64_t n_pixels, float eps,
                            double* d_out, void* stream);

/* Kernel timers.  While enabled, each phase of the handle's work (one or
 * more kernels) is bracketed by CUDA events on its stream; nirc_timing_read
 * waits for the recorded events and returns, per kernel class since the
 * last enable, the summed device time of its phases and the number of the
 * library's own kernels they launched (every kernel of a phase is the
 * library's own).  Classes: */
enum {
    NIRC_K_PATH_TRACE = 0,   /* camera hits, records, residual paths */
    NIRC_K_CACHE = 1,        /* cache integral (encodings, MLP, per-pixel sums) */
    NIRC_K_TRAIN_RECORDS = 2,/* training-path pass */
    NIRC_K_TRAIN_FWD = 3,    /* training forward + loss (tensor-core training: + backward) */
    NIRC_K_TRAIN_BWD = 4,    /* backward through the MLP + hash scatter */
    NIRC_K_TRAIN_GRADW = 5,  /* weight-gradient reduction */
    NIRC_K_ADAM = 6,         /* Adam + weight repacking */
    NIRC_K_QUERY = 7,        /* bare cache queries */
    NIRC_K_CLASSES = 8
};
typedef struct nirc_timing {
    double ms[NIRC_K_CLASSES];
    uint64_t launches[NIRC_K_CLASSES];
} nirc_timing;
nirc_status nirc_timing_enable(nirc_handle* h, int enable);
nirc_status nirc_timing_read(nirc_handle* h, nirc_timing* out);

/* Message of the last failing call on this thread ("" if none). */
const char* nirc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NIRC_H */
