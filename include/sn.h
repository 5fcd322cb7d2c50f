/*
 * sn.h -- C ABI of the GB300 stereo surface-normal library (libsn.so).
 *
 * The library estimates, for every pixel of a rectified stereo disparity
 * map, a camera-facing unit surface normal from the local affine
 * transformation between the two views, together with a denoised
 * disparity, a triangulated point, a connected-surface-component label and a
 * status mask.  Method: "Robust and Real-time Surface Normal Estimation from
 * Stereo Disparities using Affine Transformations" (arXiv 2504.15121).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * u is the column, v the row; both 0-based, pixel centres at integer
 *    (u, v).  Images are row-major with a row pitch in BYTES.
 *  * Disparity is positive: d = u_left - u_right = fx * B / z (pixels).  The
 *    paper's signed disparity (Sec. III-B) is the negative of this.
 *  * Every discrete decision is taken on the integer grid D = rint(256 d)
 *    (ties to even).  A pixel is valid iff d is finite, d > 0 and
 *    1 <= D <= 131071; pixels outside the image are invalid.
 *  * Device buffers: every pointer passed to a compute entry point is a
 *    device pointer, 16-byte aligned, and every pitch is a multiple of 16
 *    bytes and at least W * element size.  Multi-plane outputs (normals in
 *    SN_NORMALS_F32X3, points) hold their planes back to back, plane k at
 *    byte offset k * H * pitch.
 *  * Ownership: the caller owns every input and output buffer and keeps it
 *    alive until the stream has reached the call.  The context owns only its
 *    own workspace (allocated once by sn_create, freed by sn_destroy).
 *  * Execution: compute entry points only enqueue work on `stream` (NULL =
 *    the legacy default stream) and return; they do not allocate, copy
 *    host<->device or synchronise.  Argument errors are detected on the host
 *    and returned before anything is enqueued.
 *  * Errors: no exception crosses the ABI.  SN_ECUDA reports a launch error
 *    (the message is kept in the context, see sn_last_error).  A context is
 *    not thread-safe: use one context per host thread.
 */
#ifndef SN_H
#define SN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sn_stream; /* same type as cudaStream_t */
typedef struct sn_ctx sn_ctx;

typedef enum {
    SN_OK = 0,
    SN_EINVAL = 1,   /* null pointer, misaligned pointer or pitch, bad size or parameter */
    SN_ENOMEM = 2,   /* device workspace allocation failed (sn_create only) */
    SN_ECUDA = 3,    /* CUDA launch or runtime error; see sn_last_error */
    SN_ETIMEOUT = 4, /* a bounded device wait gave up; outputs of that call are undefined */
    SN_EBUSY = 5,    /* admission refused (serving) */
    SN_ENOTSUP = 6   /* parameter combination not built into this library */
} sn_status;

/* Rectified pinhole pair (Sec. II, "Rectified stereo images"): focal lengths
 * and principal point in pixels, baseline B in metres (right camera at +B
 * along x). */
typedef struct {
    double fx, fy, cx, cy, baseline;
} sn_camera;

enum { SN_SUPPORT_FIXED = 0, SN_SUPPORT_STARFILL_CD = 1, SN_SUPPORT_STARFILL_ST = 2 };
enum { SN_IN_F32 = 0, SN_IN_F16 = 1, SN_IN_U16X256 = 2 };
enum { SN_NORMALS_F32X3 = 0, SN_NORMALS_SNORM16X4 = 1 };

/* Bits of the per-pixel status mask (uint8). */
enum {
    SN_MASK_VALID = 1,    /* input disparity valid */
    SN_MASK_NORMAL = 2,   /* normal (and affine fit) valid */
    SN_MASK_FP64 = 4,     /* conditioning flag tripped: affine solve done in FP64 */
    SN_MASK_LEARNED = 8,  /* learned gate certified the full window (fast path) */
    SN_MASK_DENOISED = 16 /* the 3-parameter denoise fit was determined */
};

/* Method parameters, frozen at sn_create.
 *  r_denoise  radius of the denoise window (1..4), default 2 (5x5)
 *  r_affine   radius of the fixed affine window (1..15), default 4 (9x9;
 *             the paper's main setting, Tables perf-disc/perf-disc2)
 *  support    SN_SUPPORT_FIXED, SN_SUPPORT_STARFILL_CD (default) or
 *             SN_SUPPORT_STARFILL_ST (Sec. III-D: rays stop at depth edges)
 *  dirs,steps star-fill directions M (4..16) and steps s (1..30), default 8, 10
 *  k_cd       covered-depth threshold k (Sec. III-D), default 0.1
 *  k_pair     relative disparity step that still joins two 4-neighbours into
 *             one surface component, default 0.05
 *  k_range    relative range gate of the denoise window, default 0.05
 *  tau        confidence threshold of the learned gate, default 0.9
 *  in_dtype   SN_IN_F32 (float d), SN_IN_F16 (half d), SN_IN_U16X256 (uint16
 *             rint(256 d), 0 = invalid)
 *  normal_fmt SN_NORMALS_F32X3 (3 float planes) or SN_NORMALS_SNORM16X4
 *             (int16 x4 per pixel: rint(32767 n), 4th lane 0)
 *  learned    1 = use the learned gate (weights via sn_load_gate_weights);
 *             needs the default star (support, dirs 8, steps 10, r_denoise 2,
 *             r_affine 4), else SN_ENOTSUP.  A small network gives each pixel
 *             the probability q that the 5x5 patch centred there shows one
 *             surface; a valid pixel whose q values at the lattice points
 *             (pixels with both coordinates even, outside the image
 *             included) within SN_LEARNED_RADIUS - 1 of it are all >= tau is
 *             certified (SN_MASK_LEARNED; the 5x5 patches centred there cover
 *             its full window):
 *             its denoise fit takes every valid sample of the 5x5 window (no
 *             range gate) and its affine fit every valid sample of the
 *             (2 SN_LEARNED_RADIUS + 1)^2 window but the centre (no
 *             star-fill).  Other pixels take the plain chain.
 *  st_t       ST threshold t (metres), default 0.1: a pixel is a depth edge
 *             iff one of its 4-neighbours is invalid or its 5-point depth
 *             Laplacian ((z_l + z_r) + (z_u + z_d)) - 4 z_c, z = 256 fx B / D,
 *             exceeds t in magnitude (decided as in FP64 evaluated in that
 *             order without fused multiply-adds); an ST ray stops before the
 *             first invalid or edge pixel
 * Every k is used as the integer K = rint(65536 k).
 */
#define SN_LEARNED_RADIUS 6
typedef struct {
    int r_denoise;
    int r_affine;
    int support;
    int dirs;
    int steps;
    float k_cd;
    float k_pair;
    float k_range;
    float tau;
    int in_dtype;
    int normal_fmt;
    int learned;
    float st_t;
} sn_params;

/* Fills *p with the defaults listed above. */
void sn_default_params(sn_params *p);

/* Creates a context for W x H frames (1 <= W, H <= 16384) on the current CUDA
 * device, validates the parameters (SN_EINVAL / SN_ENOTSUP), tabulates the
 * star-fill offsets and allocates the device workspace (SN_ENOMEM).
 * p == NULL selects the defaults.  On failure *out is NULL. */
sn_status sn_create(const sn_camera *cam, int W, int H, const sn_params *p, sn_ctx **out);

/* Frees the context and its workspace; waits for nothing (the caller must
 * have synchronised the streams that used it).  NULL is accepted. */
sn_status sn_destroy(sn_ctx *ctx);

/* Denoise (abstract: noise reduction "inspired by convolutional
 * operations"; least squares of Sec. III-B written as the convolution of
 * Sec. III-C).  For every valid pixel p, fits the plane
 * d(p + o) = c + g . o by least squares over
 *   W_d = { o in [-r_denoise, r_denoise]^2 : p + o valid,
 *           2^16 |D(p+o) - D(p)| <= K_range D(p) }
 * and writes den = c (pixels).  Where the 3x3 normal matrix is singular or
 * c <= 0, den = D(p) / 256.  Invalid pixels get den = 0.
 *   disp   [H][disp_pitch] input in the context's in_dtype
 *   den    [H][den_pitch] float output
 *   mask   [H][mask_pitch] uint8 output: SN_MASK_VALID | SN_MASK_DENOISED */
sn_status sn_denoise(sn_ctx *ctx, const void *disp, size_t disp_pitch, float *den, size_t den_pitch,
                     uint8_t *mask, size_t mask_pitch, sn_stream stream);

/* Affine parameters and normals (Sec. III-A..III-D).  For every valid pixel:
 * the support is the fixed (2 r_affine + 1)^2 window without invalid pixels,
 * or the star-fill union of M rays stopped by the covered-depth rule
 *   (Dmax - Dmin) D(p) 2^16 > K_cd Dmin Dmax  (exact integer form of
 *   z_max - z_min > k z_centre)
 * before the first failing or invalid pixel.  Pass 1 forms alpha, beta,
 * gamma; pass 2 the gradient g = S (d_i - d~_p) anchored at the denoised
 * centre den[p] (eqs. convprep/convprep2).  The normal is the unit vector
 * -m / |m| with m = (g_u, g_v fy / fx, (d~ - g_u (u - cx) - g_v (v - cy)) / fx),
 * which equals the cross product of Sec. III-A (sign of its printed b term
 * corrected) turned towards the camera.  Valid iff >= 3 support pixels and
 * det = alpha gamma - beta^2 > 0; if 1024 det < alpha gamma the solve runs in
 * FP64 (SN_MASK_FP64).  Invalid normals are 0.
 *   den      denoised disparity from sn_denoise on the same disp
 *   normals  SN_NORMALS_F32X3: 3 float planes; SN_NORMALS_SNORM16X4: int16x4
 *   mask     uint8 output: SN_MASK_VALID | SN_MASK_NORMAL | SN_MASK_FP64 */
sn_status sn_affine_normals(sn_ctx *ctx, const void *disp, size_t disp_pitch, const float *den,
                            size_t den_pitch, void *normals, size_t normals_pitch, uint8_t *mask,
                            size_t mask_pitch, sn_stream stream);

/* Comparison estimators of the paper's experiments (Sec. IV, "Implemented
 * algorithms"), on the same ingest; not part of sn_run_frame.  Points are
 * X = B (u - cx, fx/fy (v - cy), fx) / (D / 256) of the valid pixels.
 * sn_cross_normals ("Cross"): n = t_u x t_v with t_u = X(u+1, v) - X(u, v),
 *   or X(u, v) - X(u-1, v) when the right neighbour is invalid, and t_v the
 *   same downwards / upwards; a normal iff the centre and both tangents
 *   exist.
 * sn_pca_normals ("PCA n x n", n = 2r + 1, 1 <= r <= 7 else SN_EINVAL): the
 *   eigenvector of the smallest eigenvalue of the covariance of the valid
 *   points of the window (centre included), closed form in FP32; a normal
 *   iff the centre is valid and the window holds >= 3 valid pixels that
 *   are not all on one image line (exact integer test).
 * Both turn the normal towards the camera (n . X < 0).
 *   disp     [H][disp_pitch] input in the context's in_dtype
 *   normals  the context's normal_fmt
 *   mask     uint8 output: SN_MASK_VALID | SN_MASK_NORMAL */
sn_status sn_cross_normals(sn_ctx *ctx, const void *disp, size_t disp_pitch, void *normals,
                           size_t normals_pitch, uint8_t *mask, size_t mask_pitch, sn_stream stream);
sn_status sn_pca_normals(sn_ctx *ctx, const void *disp, size_t disp_pitch, int r, void *normals,
                         size_t normals_pitch, uint8_t *mask, size_t mask_pitch, sn_stream stream);

/* Connected surface components (abstract: "detecting connected surface
 * components"; adaptive relative threshold as in the covered-depth rule of
 * Sec. III-D).  Two 4-neighbours p, q are joined iff both are valid and
 * 2^16 |D(p) - D(q)| <= K_pair min(D(p), D(q)).  labels[p] = the smallest
 * row-major index v * W + u of p's component, -1 for invalid pixels
 * (bit-exact, unique).  If num_components is not NULL it receives (device
 * int32) the number of components.
 *   labels  [H][labels_pitch] int32 output */
sn_status sn_components(sn_ctx *ctx, const void *disp, size_t disp_pitch, int32_t *labels,
                        size_t labels_pitch, int32_t *num_components, sn_stream stream);

/* Oriented point cloud (abstract; projection of Sec. II): for pixels with
 * SN_MASK_VALID, X = B (u - cx, fx / fy (v - cy), fx) / den; 0 elsewhere.
 *   points  3 float planes (X, Y, Z) */
sn_status sn_pointcloud(sn_ctx *ctx, const float *den, size_t den_pitch, const uint8_t *mask,
                        size_t mask_pitch, float *points, size_t points_pitch, sn_stream stream);

typedef struct {
    const void *disp;
    size_t disp_pitch;
} sn_frame_in;

typedef struct {
    float *den; /* may be NULL: the denoised disparity is then not written */
    size_t den_pitch;
    void *normals;
    size_t normals_pitch;
    float *points;
    size_t points_pitch;
    int32_t *labels;
    size_t labels_pitch;
    uint8_t *mask;
    size_t mask_pitch;
    int32_t *num_components; /* device int32, may be NULL */
} sn_frame_out;

/* The whole chain on one frame: the results of sn_denoise, sn_affine_normals,
 * sn_components and sn_pointcloud on the same input, with the mask carrying
 * all their bits.  Four kernel launches, ordered after earlier work on
 * `stream` and before later work on it: the fused frame kernel on `stream`,
 * and the three component passes (which read only the disparity) on one of
 * the context's side streams, forked from `stream` and joined back to it by
 * events, so that they run concurrently with the frame kernel.  Legal under
 * CUDA stream capture (the fork and join become graph edges).  While
 * profiling is on (sn_set_profiling), all four launches stay on `stream`. */
sn_status sn_run_frame(sn_ctx *ctx, const sn_frame_in *in, sn_frame_out *out, sn_stream stream);

/* The learned gate's probability map (no counterpart in the paper: the
 * gate is this library's own addition, see `learned` above).  For every
 * pixel p, q[p] = sigmoid(z . W3 + b3) of the gate network: features of the
 * codes (the FP32 differences of the FP32 log2 of the codes of p's right and
 * lower neighbours and of p, 0 where either is invalid; p's validity), two
 * 3x3 convolutions with ReLU in BF16 with FP32 accumulation, a 1x1 head.
 * The gate reads q only at the lattice points (pixels with both
 * coordinates even), and this call evaluates it there: q[p] at pixels with
 * both coordinates even, NaN at the others.  Needs a learned context with
 * weights loaded (else SN_EINVAL).
 *   disp  [H][disp_pitch] input in the context's in_dtype
 *   q     [H][q_pitch] float output */
sn_status sn_gate_q(sn_ctx *ctx, const void *disp, size_t disp_pitch, float *q, size_t q_pitch, sn_stream stream);

/* The table of log2 D for every disparity code D = 0..131071 that the gate's
 * features read (FP32, the correctly rounded FP32 value of log2 D; NaN for
 * D = 0, the invalid code), copied to HOST memory `out` (n >= 131072
 * floats), for inspection and tests.  Fills the table on the current device
 * first if no learned context did (a one-time kernel and a synchronisation).
 * SN_EINVAL for a NULL pointer or n < 131072, SN_ECUDA on a CUDA error. */
sn_status sn_gate_log2_table(float *out, int n);

/* The FP32 reciprocal 1/D of every disparity code D = 0..131071 as the
 * kernels compute it (the 1/D of the (D, 1/D) tiles that the covered-depth
 * stop of Sec. III-D reads, and the depths F / D of the ST edge test: PTX
 * rcp.approx; +inf for D = 0, the invalid code), copied to HOST memory `out`
 * (n >= 131072 floats), so that tests can check the error bound the
 * kernels' exact-decision bands assume.  A one-time kernel and a
 * synchronisation on the current device.  SN_EINVAL for a NULL pointer or
 * n < 131072, SN_ECUDA on a CUDA error. */
sn_status sn_rcp_table(float *out, int n);

/* sn_run_frame on HOST buffers: copies the disparity (in->disp, host) to
 * the device, runs sn_run_frame, and copies normals, points, labels, mask
 * and, if out->num_components is not NULL, the component count (host
 * int32) back into the host buffers of `out`; everything is enqueued on
 * `stream` (the results are in place once `stream` has passed the call).
 * Host buffers have the layout of sn_run_frame's outputs with any pitch
 * >= W x element size and no alignment requirement; page-locked (pinned)
 * host memory makes the copies asynchronous, pageable memory makes them
 * synchronous.  out->den must be NULL.  The context cycles through 4 sets
 * of device staging buffers (frames on up to 4 streams in flight at once);
 * a set is reused only after its previous frame's copies are done (event
 * wait on `stream`).  The first call allocates the staging buffers (not
 * under stream capture); later calls allocate nothing.  Errors as
 * sn_run_frame, plus SN_EINVAL for a NULL host pointer or a short pitch and
 * SN_ENOMEM if the staging buffers cannot be allocated. */
sn_status sn_run_frame_host(sn_ctx *ctx, const sn_frame_in *in, sn_frame_out *out, sn_stream stream);

/* Allocation-free denoise + normals.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc -- a plugin whose host application
 * owns all device memory through its own pool, or a real-time loop that must
 * not call it because it can synchronise the device and take unbounded time.
 * It needs no context (sn_create allocates): camera, parameters (NULL =
 * defaults) and size are passed directly, and the results are those of
 * sn_denoise followed by sn_affine_normals on the same input (normals and
 * mask with SN_MASK_VALID | SN_MASK_NORMAL | SN_MASK_FP64).
 * The denoised plane lives in a static device array of the library, sized for
 * frames with H * (W rounded up to a multiple of 4) <= 2048 * 1024 elements
 * (8 MiB, held on every GPU that loads the library until the process exits);
 * larger frames return SN_EINVAL before anything is enqueued.  Nothing is
 * allocated by this call.  The first call on a device resolves the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls on a device share the
 * array: calls whose work overlaps on the GPU (different streams without
 * ordering) race and give undefined results.  Buffers follow the rules at the
 * top of this header. */
sn_status sn_normals_noalloc(const sn_camera *cam, const sn_params *p, int W, int H, const void *disp,
                             size_t disp_pitch, void *normals, size_t normals_pitch, uint8_t *mask,
                             size_t mask_pitch, sn_stream stream);

/* Error status of the allocation-free path (no counterpart in the paper).
 * The kernels of sn_normals_noalloc bound every wait for an asynchronous
 * tile copy; one that gives up sets a bit in a static device error word of
 * the library (its frame's outputs are then undefined, and the call that
 * enqueued it has already returned SN_OK).  This call waits for `stream`,
 * reads that word on the current device and clears it: SN_OK if no wait gave
 * up since the previous check, SN_ETIMEOUT if one did, SN_ECUDA on a CUDA
 * error.  It allocates nothing (two synchronous copies between the word and
 * a host variable). */
sn_status sn_noalloc_check_device(sn_stream stream);

/* Loads the learned gate's weights (format version, BF16 weights, FP32
 * biases; see the package's gate module).  Copies synchronously. */
sn_status sn_load_gate_weights(sn_ctx *ctx, const void *blob, size_t bytes);

/* Star-fill offset table (host only, needs no GPU): direction j at angle
 * 2 pi j / M, step k at (round(k cos), round(k sin)) with halves rounded away
 * from zero; entry j * steps + k - 1.  Returns M * steps, or -1 if out of
 * range. */
int sn_star_offsets(int dirs, int steps, int8_t *ou, int8_t *ov);

/* Fault-detection hook (for tests): bounds every union-find walk of the
 * component passes (k_ccl_merge, k_ccl_flatten) of this context to `steps`
 * parent steps; steps <= 0 restores the default 4194304, more than any chain
 * of a 16384 x 16384 frame.  A walk that runs out stops there and sets the
 * device error word: sn_check_device then returns SN_ETIMEOUT and that
 * frame's labels and component count are undefined; the context stays
 * usable.  Takes effect for calls enqueued after it (not for graphs already
 * captured). */
sn_status sn_set_walk_limit(sn_ctx *ctx, int steps);

/* Reads and clears the context's device error word (synchronous on the
 * context's internal stream only after `stream` completes).  Returns SN_OK,
 * or SN_ETIMEOUT if a bounded device wait gave up since the last call. */
sn_status sn_check_device(sn_ctx *ctx, sn_stream stream);

/* Stage timing, for benchmarks and serving statistics.  While profiling is
 * on, sn_run_frame enqueues all its launches on its stream and records a
 * CUDA event before its first and after each of them (stage i = the i-th launch, named by
 * sn_stage_name).  sn_stage_times waits for the recorded events, writes the
 * summed milliseconds of each stage since the previous call into ms[0..n-1]
 * (n >= sn_stage_count), the number of frames into *frames, the duration of
 * each frame (first to last event) into frame_ms[0..cap-1] if frame_ms is not
 * NULL, and starts a new accumulation.  Up to 4096 frames are recorded between two calls; later
 * frames are not recorded (*frames says how many were).  sn_set_profiling
 * creates the events on first use (not a hot call). */
sn_status sn_set_profiling(sn_ctx *ctx, int on);
int sn_stage_count(const sn_ctx *ctx);
const char *sn_stage_name(const sn_ctx *ctx, int i);
sn_status sn_stage_times(sn_ctx *ctx, double *ms, int n, int *frames, double *frame_ms, int cap);

/* Number of kernels this context has launched since sn_create. */
uint64_t sn_launch_count(const sn_ctx *ctx);

const char *sn_status_string(sn_status s);
const char *sn_last_error(const sn_ctx *ctx);

/* Library version, (major << 16) | minor. */
int sn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SN_H */
