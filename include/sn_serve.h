/*
 * sn_serve.h -- serving runtime of libsn.so: continuous batching of frames
 * from several cameras of different resolutions on one GPU.
 *
 * The paper has no serving layer (each frame is one shader dispatch,
 * Sec. IV); this runtime feeds the per-frame chain of sn.h (sn_run_frame)
 * from many cameras at once.
 *
 * Model.  A server owns, per camera, one sn_ctx and a set of request slots:
 * device-resident input and output buffers (and, optionally, pinned host
 * copies of the outputs), each with one CUDA graph instantiated at creation
 * that runs the whole chain for that slot.  Slots are allocated at creation,
 * round-robin over the cameras, until the device-memory budget is used up;
 * admission is therefore by memory: a request starts as soon as a slot of
 * its camera is free.  A scheduler thread admits waiting requests, issues
 * the host->device copy of the frame and the slot's graph on one of several
 * streams (so frames of different cameras overlap on the device), and
 * detects completion by polling events.  Latency is measured from the
 * request's arrival to the moment its result is ready (outputs on the
 * device, or on the host when results_to_host is set).
 *
 * Ownership.  Host frames handed to sn_server_submit must stay valid until
 * the request's result is polled; they should be pinned (page-locked) for
 * the copy to be asynchronous.  The server owns all device buffers.
 *
 * Threads.  sn_server_submit, sn_server_poll, sn_server_release and
 * sn_server_simulate may be called from one client thread; the scheduler
 * thread is internal.  Errors: SN_EBUSY when a camera's waiting queue is
 * full; SN_EINVAL for bad arguments; SN_ENOMEM when the budget does not give
 * every camera at least one slot.
 */
#ifndef SN_SERVE_H
#define SN_SERVE_H

#include "sn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sn_server sn_server;

typedef struct {
    int W, H;
    sn_camera cam;
    sn_params params;  /* in_dtype, normal_fmt and learned select the form per camera */
    double rate_hz;    /* mean frame rate for sn_server_simulate */
    /* params.learned = 1: the gate weights (the blob sn_load_gate_weights
     * takes, HOST memory, read during sn_server_create only); ignored
     * otherwise.  A learned camera without weights fails with SN_EINVAL. */
    const void *gate_weights;
    size_t gate_weights_bytes;
} sn_server_camera;

typedef struct {
    int n_cameras;
    const sn_server_camera *cameras;
    size_t memory_budget;     /* bytes of device memory for request slots */
    int max_slots_per_camera; /* upper bound on slots per camera (>= 1) */
    int n_streams;            /* concurrent device streams (1..16) */
    int results_to_host;      /* 1: each result is copied to pinned host buffers */
    int queue_depth;          /* waiting requests per camera before SN_EBUSY */
} sn_server_config;

typedef struct {
    uint64_t tag;
    int camera;
    int slot;
    double latency_ms;       /* arrival -> result ready */
    /* results_to_host = 1: host copies, valid until sn_server_release(slot) */
    const void *normals;     /* layout of the camera's normal_fmt, W-dense rows */
    const float *points;     /* 3 planes, W-dense rows */
    const int32_t *labels;
    const uint8_t *mask;
    int32_t num_components;
} sn_serve_result;

typedef struct {
    double duration_s;        /* emission window */
    double rate_scale;        /* multiplies every camera's rate_hz */
    uint64_t seed;            /* Poisson inter-arrival times */
    const void *const *frames; /* frames[cam * max_pool + i], pinned host frames */
    const int *pool_size;     /* per camera, 1..max_pool */
    int max_pool;
    const size_t *frame_pitch; /* per camera, bytes */
} sn_serve_sim;

typedef struct {
    double offered_mpix_s;   /* pixels emitted / duration */
    double sustained_mpix_s; /* pixels completed / (last completion - first arrival) */
    double p50_ms, p99_ms, max_ms;
    long long submitted, completed, refused;
    double wall_s;
} sn_serve_stats;

sn_status sn_server_create(const sn_server_config *cfg, sn_server **out);
sn_status sn_server_destroy(sn_server *s);
/* Number of slots the memory budget gave camera `cam`. */
int sn_server_slots(const sn_server *s, int cam);
sn_status sn_server_submit(sn_server *s, int cam, const void *host_disp, size_t pitch, uint64_t tag);
/* Writes up to max completed results (oldest first); returns how many. */
int sn_server_poll(sn_server *s, sn_serve_result *out, int max);
/* Returns a completed slot to the pool (results_to_host = 1 only; with 0 a
 * slot is reused as soon as its result is ready). */
sn_status sn_server_release(sn_server *s, int cam, int slot);
/* Emits Poisson arrivals from the frame pools for duration_s, waits until
 * every admitted request has completed, and reports latency percentiles and
 * throughput.  Results are not handed to the client. */
sn_status sn_server_simulate(sn_server *s, const sn_serve_sim *sim, sn_serve_stats *out);
/* Device error bits collected from the cameras' contexts (see sn_check_device). */
sn_status sn_server_check(sn_server *s);

#ifdef __cplusplus
}
#endif
#endif /* SN_SERVE_H */
