/*
 * nirc_serve.h -- frame-request server on top of libnirc.so (same library).
 *
 * The paper renders one view per frame with a cache trained on-line from
 * that frame's own paths (section "Cache application").  This server runs
 * that frame loop for many independent render requests at once; it has no
 * counterpart in the paper, which studies a single renderer.  Every request
 * is one frame of the two-level estimator (nirc_estimate_frame) followed by
 * one training pass and one Adam step of the scene's cache
 * (nirc_gen_train + nirc_train_step), exactly as a single renderer would run
 * them; the server only decides when, and next to which other requests, the
 * GPU does that work.
 *
 * Scheduling (continuous batching at frame granularity):
 *  - Each scene is a cache handle that stays resident on the device with its
 *    FP32 master weights, low-precision copies, Adam moments and hash table,
 *    plus the server's training buffers for that scene.
 *  - Submitted requests wait in a FIFO.  A scheduler thread forms a batch
 *    from the queue whenever a batch slot is free: requests are taken in
 *    arrival order, skipping (not dropping) a request whose scene already has
 *    a request in flight (a scene's frames and training steps stay in order),
 *    up to `slots` requests, while their buffers fit into the arena.  A
 *    request that does not fit stops the scan (no overtaking on memory, so
 *    large frames are not starved).
 *  - A batch is launched as ONE CUDA graph.  In it the frames of all its
 *    requests are one launch of each path-tracing pass (camera, residual;
 *    per light mode) and one cache-integral launch over the union of their
 *    pixels (each request's
 *    CTAs in proportion to its work, so requests of different resolution
 *    and N share the GPU inside one kernel); then each request's training
 *    pass and step run as their own branch of the graph.  When the caches
 *    of a batch differ in precision or network shape, or a request uses
 *    light mode 2, each request's chain runs as its own branch instead.  Up to
 *    `max_batches` batches are in flight at once on their own streams, so a
 *    request that arrives while others run is admitted as soon as a batch
 *    slot and memory are free, without waiting for the running batches.
 *  - A completion thread polls the batches' events and stamps each request
 *    with the server clock when its batch finishes on the device.
 *
 * Memory: `budget_bytes` of device memory is reserved at creation for the
 * per-request buffers (the output image, W*H*16 bytes, and the frame
 * scratch, W*H*(96 + 32*M) bytes rounded) and managed by a first-fit arena.
 * A request is admitted only when both buffers fit; the scratch returns to
 * the arena when the request completes, the image when the caller releases
 * it.  A request that could never fit fails at submission with
 * NIRC_ERR_BUDGET.  Resident scene state is allocated by the handles and
 * reported separately (nirc_server_stats).
 *
 * Threading: all nirc_server_* calls are thread-safe.  Handles registered
 * with a server must not be used by the caller while the server runs work
 * on them (between registration and nirc_server_drain); their kernel timers
 * must be off.  Destroy the server before its handles.
 */
#ifndef NIRC_SERVE_H
#define NIRC_SERVE_H

#include "nirc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nirc_server nirc_server;

typedef struct nirc_server_config {
    uint64_t budget_bytes;   /* arena for per-request buffers (>= 1 MiB) */
    uint32_t slots;          /* requests per batch, 1..16 */
    uint32_t max_batches;    /* batches in flight at once, 1..4 */
    uint32_t train_samples;  /* training paths + one Adam step per served frame (0 = no training) */
    uint32_t use_graphs;     /* 1: capture each batch into one CUDA graph; 0: plain stream launches */
} nirc_server_config;

typedef struct nirc_request {
    uint64_t id;                 /* caller's tag, unique among unreleased requests */
    uint32_t scene;              /* index from nirc_server_add_scene */
    uint32_t width, height;      /* 1..8192 each */
    uint32_t n_cache, n_resid;   /* N (0..1024), M (0..64) */
    uint32_t max_depth;          /* 1..64 */
    uint32_t frame;              /* frame index: Philox key word 1 and scene key frame (mod n_frames) */
    uint32_t light_mode;         /* as in nirc_frame_desc (frame and training pass) */
} nirc_request;

typedef struct nirc_completion {
    uint64_t id;
    int32_t status;              /* nirc_status of the request */
    uint32_t batch_size;         /* requests in the batch it ran in */
    float* d_image;              /* W*H float4 (device), valid until nirc_server_release */
    double t_submit;             /* server clock (s) at nirc_server_submit */
    double t_launch;             /* server clock (s) when its batch was launched */
    double t_done;               /* server clock (s) when its batch was seen complete */
} nirc_completion;

typedef struct nirc_server_stats {
    uint64_t submitted, completed, failed, batches, graph_instantiations, graph_updates;
    uint64_t arena_bytes, arena_peak_bytes, resident_bytes;
    uint32_t queued, in_flight, max_batch_seen, pad;
    uint64_t frame_launches;     /* path-tracing (camera, residual) + cache-integral launches for frames */
} nirc_server_stats;

/* Create a server on the current CUDA device: reserves budget_bytes of device
 * memory and starts the scheduler and completion threads. */
nirc_status nirc_server_create(const nirc_server_config* cfg, nirc_server** out);

/* Register a resident scene: `cache` (owned by the caller, kept alive until
 * the server is destroyed), n_frames scene blobs (nirc.h layout) at d_frames
 * + k * frame_stride (device, 16-byte aligned; request frame f uses key
 * frame f mod n_frames), n_prims primitives, Philox seed.  Reserves the
 * scene's training buffers and scratch for train_samples paths (allocated
 * here, counted in resident_bytes). */
nirc_status nirc_server_add_scene(nirc_server* s, nirc_handle* cache, const void* d_frames, uint32_t n_frames,
                                  uint64_t frame_stride, uint32_t n_prims, uint64_t seed, uint32_t* scene_out);

/* Queue a request (copied).  NIRC_ERR_INVALID for a bad scene or size,
 * NIRC_ERR_BUDGET when its buffers exceed the whole arena. */
nirc_status nirc_server_submit(nirc_server* s, const nirc_request* req);

/* Move up to `max` finished requests into `out` (oldest first); *n_out gets
 * the count.  wait != 0 blocks until at least one is available or nothing
 * is queued or in flight. */
nirc_status nirc_server_poll(nirc_server* s, nirc_completion* out, uint32_t max, uint32_t* n_out, int wait);

/* Copy a polled request's image (W*H float4) to d_dst (device) on `stream`. */
nirc_status nirc_server_copy_image(nirc_server* s, uint64_t id, float* d_dst, void* stream);

/* Return a completed request's image to the arena. */
nirc_status nirc_server_release(nirc_server* s, uint64_t id);

/* Block until nothing is queued or in flight. */
nirc_status nirc_server_drain(nirc_server* s);

nirc_status nirc_server_stats_read(nirc_server* s, nirc_server_stats* out);

/* Seconds since the server was created (the clock of nirc_completion). */
double nirc_server_clock(nirc_server* s);

/* Stop the threads after in-flight work finishes (queued requests are
 * dropped), free the arena and the scenes' training buffers. */
nirc_status nirc_server_destroy(nirc_server* s);

#ifdef __cplusplus
}
#endif

#endif /* NIRC_SERVE_H */
