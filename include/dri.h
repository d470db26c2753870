/*
 * dri.h -- C ABI of the GB300 dense RGB-D-inertial tracking library.
 *
 * The library tracks camera streams with the tightly coupled photometric +
 * point-to-plane ICP + inertial Gauss-Newton of Laidlow et al., "Dense
 * RGB-D-Inertial SLAM with Map Deformations" (IROS 2017), Sec. IV: per frame it
 * estimates the current state x1 and refines the previous state x0 (Sec. IV-A),
 * over a coarse-to-fine image pyramid (Sec. IV-D), and marginalises x0 into a
 * prior for the next frame (Sec. IV-E, Eq. 8-9).  Every step of a frame runs in
 * the library's CUDA kernels on one GPU; the host only copies inputs in and
 * results out.
 *
 * Conventions (Sec. II).  Frames: W world (= first camera frame), I inertial
 * (gravity aligned, z up, shares W's origin), C camera, S IMU sensor.  Poses
 * T_AB map B coordinates into A.  Quaternions are Hamilton, stored (w, x, y, z).
 * Images are row-major FP32, depth in metres (<= 0 or outside
 * [depth_min, depth_max] is invalid), intensity in [0, 1].
 *
 * Errors.  Every call returns an int status (DRI_OK = 0 or a negative DRI_E*
 * code).  No call throws across the ABI.  On error the stream's state is left
 * as it was before the call unless the description says otherwise.
 *
 * Threads.  A stream handle is used by one host thread at a time.  Different
 * streams may be driven from different threads.
 */
#ifndef DRI_H
#define DRI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define DRI_OK          0
#define DRI_EINVAL    (-1)   /* bad size, pointer, configuration or IMU order   */
#define DRI_ENOMEM    (-2)   /* device or host allocation failed; workspace too small */
#define DRI_EADMIT    (-3)   /* over the server's HBM budget                     */
#define DRI_ENOTREADY (-4)   /* no frame uploaded, or IMU does not cover [t0, t1] */
#define DRI_ELOST     (-5)   /* tracking failure; the stream keeps its last good state */
#define DRI_ETIMEDOUT (-6)   /* a bounded wait expired                           */
#define DRI_ECUDA     (-7)   /* a CUDA runtime call failed                       */

/* ---- memory kinds for uploads ------------------------------------------ */
#define DRI_HOST   0
#define DRI_DEVICE 1

/* ---- precision flags (dri_stream_config.precision_flags) --------------- */
#define DRI_FP16_MAPS     1  /* normal and intensity-gradient maps stored in FP16 */
#define DRI_FP32_PARTIALS 2  /* per-block partial sums in FP32 instead of FP64     */

/* ---- IMU term per Gauss-Newton iteration (dri_stream_config.imu_mode) ---
 * The paper pre-integrates the IMU samples between frames (Sec. IV-C, after
 * Forster et al.).  DRI_IMU_REINTEGRATE repeats the integration at x0's current
 * biases every iteration (exact).  DRI_IMU_FIRST_ORDER integrates once per
 * frame at x0's biases when the frame starts and updates that pre-integration
 * to first order in the bias change every iteration (dR Exp(Phi_g db_g),
 * dv + V_g db_g + V_a db_a, dp + P_g db_g + P_a db_a), re-integrating and
 * moving the linearisation point to the current biases once |db_g| exceeds
 * bias_relin_g or |db_a| exceeds bias_relin_a. */
#define DRI_IMU_REINTEGRATE 0
#define DRI_IMU_FIRST_ORDER 1

/* ---- what a stream tracks (dri_stream_config.track_mode) ----------------
 * DRI_TRACK_INERTIAL: the paper's joint RGB-D-inertial tracker (Eq. 6-9).
 * DRI_TRACK_RGBD_ONLY: the vision-only baseline it compares with (Sec. III,
 * ElasticFusion's tracking): Gauss-Newton on the current pose only, x1 starting
 * at the previous result x0, which stays fixed (the photometric term warps
 * with it), over H_icp + rgbd_lambda H_rgb with the per-pixel weights kept; no
 * IMU term, prior or marginalisation, and no IMU samples are needed.  Velocity,
 * biases and gravity are carried over unchanged. */
#define DRI_TRACK_INERTIAL  0
#define DRI_TRACK_RGBD_ONLY 1
/* DRI_TRACK_GYRO_ONLY: the paper's gyroscope-only setup (Sec. VII, Fig. 5 and
 * Table VI: the accelerometer-related residuals ignored).  The joint tracker
 * of Eq. 6-9 with the IMU term reduced to its rotation rows and the gyro-bias
 * random walk, weighted by the inverse of their own covariance block; the
 * velocity, accelerometer bias and gravity direction of both states are held
 * (not estimated: they keep x_init's values, and the marginalisation prior
 * carries no information on them).  x1 starts at x0's position with the
 * gyro's rotation prediction.  IMU samples are needed as for the inertial
 * mode; their accelerometer readings do not affect the result. */
#define DRI_TRACK_GYRO_ONLY 2

/* Depth-dependent ICP weight (dri_stream_config.icp_depth_weight = 1; the
 * paper weighs each term by its noise covariance, Sec. III, and a structured-
 * light or stereo sensor's axial noise grows with the square of the depth):
 * sigma_d(z) = sigma_d (z / 1 m)^2, so a pixel's ICP weight is W_ICP / z^4 with
 * z its live depth in metres.  Streams tracked in one batch or served together
 * must agree on this option and on whether occlusion_thr is > 0. */

/* Occlusion test (dri_stream_config.occlusion_thr > 0; the paper has none,
 * the readings add it as an option): a photometric residual (Eq. 3) is used
 * only where the warped point's depth in x0's camera agrees within
 * occlusion_thr metres with the reference depth at the nearest reference pixel
 * (when that depth is valid); elsewhere the point changed visibility between
 * the frames and its intensity belongs to another surface. */

/* Gravity direction in the state (dri_stream_config.gravity_dof).  The paper
 * keeps q_IW with three degrees of freedom (Sec. II, IV-A) although two fix
 * gravity's direction; the third, the turn about gravity, is a gauge freedom
 * that no measurement sees.  DRI_GRAVITY_2DOF perturbs q_IW about I's x and y
 * axes only (17 tangent dimensions per state; the turn about gravity is fixed
 * and its freedom taken up by v_I).  DRI_GRAVITY_3D perturbs it about all three
 * (18 per state, the paper's parameterisation): the first-frame prior holds
 * all three axes, each Gauss-Newton step is damped on the gravity components of
 * both states, (H + D_g) dx = b with D_g the identity there (the damping is not
 * part of the cost; marginalisation takes the Schur complement of the undamped
 * system), and the prior of dri_get_state / dri_set_state is 18 x 18.  Only
 * for DRI_TRACK_INERTIAL; dri_linearise does not serve it (DRI_EINVAL). */
#define DRI_GRAVITY_2DOF 2
#define DRI_GRAVITY_3D   3

#define DRI_MAX_LEVELS 4

typedef struct dri_stream_s* dri_stream;

/* Per-stream configuration.  dri_config_default fills every field with the
 * values of the synthetic-dataset column of Table I (Sec. VI) and the readings
 * documented beside each field. */
typedef struct {
    double fx, fy, cx, cy;         /* level-0 intrinsics, pixels                     */
    int32_t width, height;         /* level-0 image size (>= 8 x 8, <= 8192 x 8192)  */
    int32_t levels;                /* pyramid levels, 1..DRI_MAX_LEVELS (Sec. IV-D)  */
    int32_t iters[DRI_MAX_LEVELS]; /* Gauss-Newton iterations per level, [0] finest  */
    double T_CS[7];                /* IMU in camera: r_CS (3), q_CS (w, x, y, z)      */
    double sigma_I;                /* photometric noise, W_RGB = 1/sigma_I^2 (Eq. 6)  */
    double sigma_d;                /* point-to-plane noise, W_ICP = 1/sigma_d^2       */
    double gyr_nd, acc_nd;         /* IMU white-noise densities (Table I)            */
    double gyr_rw, acc_rw;         /* bias random-walk densities (Table I)           */
    double g;                      /* gravity magnitude (Table I)                     */
    double sigma_grav_rw;          /* gravity-direction noise between frames, rad     */
    double prior_sigma[5];         /* first-frame prior: pose, v, b_g, b_a, gravity   */
    double icp_dist_thr;           /* ICP association distance threshold, m           */
    double icp_angle_thr_deg;      /* ICP normal-angle threshold, degrees, in (0, 90) */
    double depth_min, depth_max;   /* valid depth range, m                            */
    int32_t min_valid;             /* level-0 correspondences below this: DRI_ELOST   */
    int32_t precision_flags;       /* DRI_FP16_MAPS | DRI_FP32_PARTIALS               */
    int32_t max_imu;               /* IMU samples one frame interval may span         */
    int32_t imu_mode;              /* DRI_IMU_REINTEGRATE (default) | _FIRST_ORDER    */
    double bias_relin_g;           /* first order: re-integrate past |db_g|, rad/s    */
    double bias_relin_a;           /* first order: re-integrate past |db_a|, m/s^2    */
    int32_t track_mode;            /* DRI_TRACK_INERTIAL (default) | _RGBD_ONLY | _GYRO_ONLY */
    int32_t count_margins;         /* 1: fill dri_track_result.n_margin (the pixel kernel
                                      of each level's last iteration counts them: ~2% of a
                                      batched frame's pixel-kernel time); 0 (default): zeros */
    double rgbd_lambda;            /* RGB-D-only: photometric weight (default 1)      */
    double occlusion_thr;          /* > 0: photometric depth-consistency test, m; 0 off */
    int32_t icp_depth_weight;      /* 1: ICP weight W_ICP / z^4 (sigma_d at 1 m); 0 off */
    int32_t gravity_dof;           /* DRI_GRAVITY_2DOF (0, default) | DRI_GRAVITY_3D    */
} dri_stream_config;

/* One IMU sample: time (s), gyro (rad/s) and accelerometer (m/s^2) in S. */
typedef struct { double t; double gyr[3]; double acc[3]; } dri_imu_sample;

/* State x of Eq. 1: r_WC, q_WC, v_IS (in I), b_g, b_a, q_IW, and its time. */
typedef struct {
    double r_WC[3];
    double q_WC[4];
    double v_I[3];
    double bg[3];
    double ba[3];
    double q_IW[4];
    double t;
} dri_state;

/* Result of one tracked frame.  n_icp / n_rgb are the valid correspondence
 * counts of the last iteration at each level.  n_margin counts, for that
 * iteration, the pixel decisions of the ICP term plus those of the photometric
 * term that lay within the rounding margins of FP32 arithmetic: a projection
 * within 1e-4 px of a rounding or image-bound boundary, or a depth-range, z > 0,
 * distance, normal-angle or occlusion test within a relative 1e-5 of its
 * threshold (normal angle with FP16 maps: 4 * 2^-11 in cos).  Such a pixel may
 * be decided either way by implementations that round differently; decisions
 * made while the maps were built (the normals' own tests) are not counted.
 * Counted when the stream's config has count_margins = 1 (in a batch: when any
 * of its streams has), else zero.  cost is Eq. 6 at the last linearisation (data + IMU terms, prior excluded);
 * status is the frame's DRI_* code (DRI_OK, or DRI_ELOST with x1 = the
 * previous state). */
typedef struct {
    dri_state x1;
    dri_state x0;
    int32_t n_icp[DRI_MAX_LEVELS];
    int32_t n_rgb[DRI_MAX_LEVELS];
    int32_t n_margin[DRI_MAX_LEVELS];
    double cost;
    int32_t status;
    int32_t initialised;           /* 1 if this call only initialised the stream     */
} dri_track_result;

/* Debug / parity output of dri_linearise: every term of Eq. 6 linearised at
 * one (x0, x1) on one pyramid level, in world coordinates, with H dx = b and
 * b = -sum J^T W e (Eq. 7).  Matrices are row-major. */
typedef struct {
    double H[34 * 34];             /* assembled joint system over [dx0; dx1]          */
    double b[34];
    double H_icp[36], b_icp[6];    /* ICP term on x1's pose (dr1, da1)                */
    double H_rgb[36], b_rgb[6];    /* photometric term, x1 pose block                 */
    double cost_icp, cost_rgb, cost_imu;
    double e_imu[18];              /* IMU error x^1(x0) boxminus x1                   */
    int64_t n_icp, n_rgb;
    int64_t n_margin_icp, n_margin_rgb;  /* margin decisions per term (see dri_track_result) */
} dri_linearisation;

/* Fills *cfg with defaults for a width x height stream: intrinsics scaled from
 * 277 px focal per 320 px width with the principal point at the image centre,
 * 3 levels with 10/5/4 iterations, identity T_CS, Table I noise (synthetic),
 * sigma_I 0.01, sigma_d 0.002 m, ICP thresholds 0.10 m / 20 deg, depth range
 * [0.3, 8] m.  Returns DRI_EINVAL for a NULL cfg or a size out of range. */
int dri_config_default(int32_t width, int32_t height, dri_stream_config* cfg);

/* Device bytes one stream needs for its maps, partials and state (the
 * workspace passed to dri_create_stream).  DRI_EINVAL for a bad config. */
int dri_stream_workspace_bytes(const dri_stream_config* cfg, size_t* bytes);

/* Creates a stream.  cfg and x_init are copied.  cuda_stream is the
 * cudaStream_t every operation of this stream is ordered on (NULL = legacy
 * default stream).  workspace is caller-owned device memory of at least
 * dri_stream_workspace_bytes(cfg) bytes, 256-byte aligned, kept alive until
 * dri_destroy_stream; if NULL the library allocates (and frees) it.  The first
 * dri_track call only initialises: x1 := x_init, the first-frame prior, and the
 * frame becomes the reference (W = first camera frame, Sec. II). */
int dri_create_stream(const dri_stream_config* cfg, const dri_state* x_init, void* cuda_stream,
                      void* workspace, size_t workspace_bytes, dri_stream* out);

/* Waits for the stream's work, frees what the library allocated. */
int dri_destroy_stream(dri_stream s);

/* Uploads the live frame at time t (seconds, strictly increasing): depth and
 * intensity, height rows of width floats, rows pitch_bytes apart (0 = packed,
 * a multiple of 4).  DRI_HOST: host memory.  Pageable memory is copied into the
 * stream's workspace, stream-ordered on the stream's cuda_stream, before this
 * call returns.  Pinned (page-locked) memory is not copied here: the GPU reads
 * it directly over the host link in the first kernel of the next dri_track /
 * dri_track_batch of this stream (one pass, no copy-engine transfer), so, as
 * for DRI_DEVICE, the caller keeps it unchanged until that work has run.
 * DRI_DEVICE: device memory, not copied here: the first kernel
 * of the next dri_track / dri_track_batch of this stream reads it, so the
 * caller keeps it unchanged until that work has run on cuda_stream, and work
 * that produces it on another stream is ordered before the track call (e.g.
 * with an event).  The caller keeps ownership. */
int dri_upload_frame(dri_stream s, double t, const float* depth, const float* intensity,
                     size_t pitch_bytes, int32_t mem_kind);

/* Replaces the reference the next frame is tracked against with a model
 * prediction rendered at T_WC_ref (r_WC (3), q_WC (w, x, y, z)), as the paper
 * tracks against its surfel model's prediction (Sec. IV-B): vertex_W and
 * normal_W hold an (x, y, z) FP32 triple per pixel in W, intensity one float;
 * height rows of width pixels, pitch_px pixels apart (0 = width) in all three.
 * A pixel with a zero normal has no surface.  Level 0 keeps, for each pixel
 * with a surface, the depth of its vertex in the reference camera (the vertex
 * of a prediction rendered from T_WC_ref lies on its pixel's ray) and its
 * normal where that depth is in [depth_min, depth_max]; coarser levels average
 * the depth over samples > 0, the intensity, and the non-zero normals
 * (renormalised).  Only the next tracked frame uses it: that frame then becomes
 * the reference, unless another prediction is uploaded.
 * DRI_HOST: copied through a device staging buffer that the library allocates
 * on first use (28 bytes per pixel, freed with the stream); DRI_DEVICE: read by
 * this call's kernels, stream-ordered on the stream's cuda_stream.
 * DRI_ENOTREADY before the stream's first (initialising) frame. */
int dri_upload_reference(dri_stream s, const float* vertex_W, const float* normal_W,
                         const float* intensity, const double* T_WC_ref, size_t pitch_px,
                         int32_t mem_kind);

/* Appends IMU samples (host memory, n >= 0) with strictly increasing times,
 * later than every sample already pushed.  DRI_EINVAL otherwise. */
int dri_push_imu(dri_stream s, const dri_imu_sample* samples, size_t n);

/* Tracks the uploaded frame (Sec. IV): IMU pre-integration, coarse-to-fine
 * Gauss-Newton over x0 and x1 with the photometric, ICP, IMU and prior terms,
 * marginalisation of x0 and the swap of the reference to this frame.
 * out != NULL: waits and fills *out, returning DRI_OK or the frame's error.
 * out == NULL: returns after enqueuing; read the state with dri_get_state.
 * DRI_ENOTREADY when no new frame is uploaded or the IMU samples do not cover
 * [t_previous_frame, t_frame]. */
int dri_track(dri_stream s, dri_track_result* out);

/* Tracks the uploaded frame of each of n streams (Sec. IV, as dri_track) in
 * one batched launch sequence: every kernel of a frame (maps, frame start, each
 * Gauss-Newton iteration's pixel kernel and solve, marginalisation, gradients)
 * is one launch over the pixels or states of all n streams.  The paper tracks
 * one camera; batching independent streams is this library's throughput mode.
 *
 * streams: n (1..4096) distinct handles created on the same cuda_stream with
 * the same levels, iterations and precision flags (sizes and intrinsics may
 * differ), otherwise DRI_EINVAL.  The first call with a given list (same
 * handles, same order) builds a plan: device tables, a staging ring and
 * buffers for the n result blocks (allocated; freed when one of the streams
 * is destroyed).  On the first call that tracks a frame the plan times the
 * pixel kernel at rows-per-thread 2, 4, 8, 16, 32 on each level and keeps the
 * fastest (this call waits); later calls replay the sequence as one CUDA graph
 * (launched directly on the legacy default stream or while profiling).
 *
 * With n = 1 the call tracks through the stream's own plan, as dri_track does.
 * A stream without an uploaded frame, or whose IMU samples do not yet cover
 * [t_previous_frame, t_frame], sits the call out (its frame stays pending).
 * out == NULL: returns after enqueuing; out != NULL: waits and fills out[i]
 * for every stream (status DRI_ENOTREADY for one that sat out).  Returns
 * DRI_OK when the batch ran, DRI_ENOTREADY when no stream had work. */
int dri_track_batch(const dri_stream* streams, int32_t n, dri_track_result* out);

/* Launch options of a plan (the stream's own for n = 1, else the batch plan of
 * the list):
 *   rows_per_thread  pixel-kernel rows per thread on each level (tile = 32
 *                    columns x 4 * rows); 0 past the last level
 *   groups           the Gauss-Newton loop runs as this many groups of slots,
 *                    each on its own CUDA stream forked from and joined to the
 *                    plan's stream, so one group's FP64 solves overlap another
 *                    group's pixel kernels (1 .. min(n, 8); default n / 16
 *                    clamped to 1 .. 4; a stream's own plan has 1); 0 in
 *                    dri_batch_set_options keeps the plan's current groups
 *   autotune         1: the next tracked frame times rows per thread
 *                    2, 4, 8, 16, 32 per level and keeps the fastest (batch
 *                    plans start with it on); 0: rows_per_thread as given, so
 *                    repeated runs sum pixels in the same order (identical bits) */
typedef struct {
    int32_t rows_per_thread[DRI_MAX_LEVELS];
    int32_t groups;
    int32_t autotune;
} dri_batch_options;

/* Reads the options of the plan for this stream list; DRI_ENOTREADY if no
 * batch plan exists for it yet. */
int dri_batch_get_options(const dri_stream* streams, int32_t n, dri_batch_options* out);

/* Sets them (creating the batch plan if needed, as dri_track_batch would).
 * Waits for the streams' work.  rows_per_thread is ignored when autotune is 1.
 * DRI_EINVAL for a bad list or value. */
int dri_batch_set_options(const dri_stream* streams, int32_t n, const dri_batch_options* opt);

/* ---- serving loop --------------------------------------------------------
 * A server tracks many independent camera streams on one GPU by continuous
 * batching (the paper tracks one camera; this is the library's serving mode).
 * Streams are admitted while the device bytes of all admitted streams
 * (workspace + 64 KB of plan state each) stay within hbm_budget_bytes;
 * all of a server's streams share levels, iterations and precision flags.
 * Requests (a frame with the IMU samples since the stream's previous frame)
 * are submitted from any thread; a worker thread takes the oldest request of
 * each stream, at most max_batch streams per tick, and tracks them in one
 * batched launch sequence (dri_track_batch's plan over all the server's
 * streams; streams without a request sit the tick out).  Two ticks may be on
 * the GPU at once: requests that arrive while one runs go into the next. */
typedef struct dri_server_s* dri_server;

/* Creates a server; cuda_stream orders all its work (NULL = legacy default
 * stream: no CUDA-graph replay).  DRI_EINVAL for a zero budget or max_batch
 * outside 1..4096. */
int dri_server_create(size_t hbm_budget_bytes, int32_t max_batch, void* cuda_stream, dri_server* out);

/* Finishes every submitted request, closes every stream, frees the server. */
int dri_server_destroy(dri_server srv);

/* Admits and creates a stream (as dri_create_stream, library-allocated
 * workspace, the server's cuda_stream).  DRI_EADMIT if it would exceed the
 * budget; DRI_EINVAL if its levels, iterations or precision flags differ from
 * the server's first stream.  The handle is driven by the server only: use
 * it with dri_server_submit / dri_server_close_stream, and for reads
 * (dri_get_state) only while none of its requests is pending. */
int dri_server_open_stream(dri_server srv, const dri_stream_config* cfg, const dri_state* x_init,
                           dri_stream* out);

/* Waits until the stream's submitted requests are done, then destroys it and
 * returns its bytes to the budget. */
int dri_server_close_stream(dri_server srv, dri_stream s);

/* Queues the frame at time t of stream s (images as in dri_upload_frame; they
 * are read when the request's tick runs, so the caller keeps them unchanged
 * until the ticket is done) with the n_imu samples (copied here) that extend
 * the stream's IMU record to t.  *ticket identifies the request. */
int dri_server_submit(dri_server srv, dri_stream s, double t, const float* depth,
                      const float* intensity, size_t pitch_bytes, int32_t mem_kind,
                      const dri_imu_sample* imu, size_t n_imu, uint64_t* ticket);

/* Waits up to timeout_ms (< 0: without limit; 0: just checks) for the
 * request; returns DRI_ETIMEDOUT if it is not done, else fills *out (nullable)
 * and returns the request's status (DRI_OK, DRI_ELOST, DRI_ENOTREADY when its
 * IMU samples did not cover the frame, or the upload's error); a done ticket
 * is released by this call. */
int dri_server_poll(dri_server srv, uint64_t ticket, dri_track_result* out, int32_t timeout_ms);

typedef struct {
    int64_t submitted, completed, failed, ticks;
    double mean_batch;             /* requests per tick                              */
    double p50_ms, p99_ms, max_ms; /* submit-to-done latency of completed requests   */
    double frames_per_s;           /* completed / (last done - first submit)         */
    size_t hbm_used, hbm_budget;
    int32_t streams;
    int32_t reserved;
} dri_server_stats;

/* Counters since creation or the last reset (reset = 1 clears them and the
 * tick trace). */
int dri_server_stats_read(dri_server srv, int32_t reset, dri_server_stats* out);

/* Host timestamps of one tick of the serving loop (a tracing aid, not part of
 * the paper): milliseconds since dri_server_create on the host's steady clock. */
typedef struct {
    int64_t tick;                  /* tick number since creation                      */
    int32_t requests;              /* requests the tick took                          */
    int32_t status;                /* DRI_OK or the error of the tick's launch        */
    double dequeue_ms;             /* the worker took the tick's requests             */
    double staged_ms;              /* their IMU samples and frame uploads were enqueued */
    double launched_ms;            /* the tick's batched frame was enqueued           */
    double done_ms;                /* the worker saw the tick's results complete      */
    double device_ms;              /* device time of the tick's launch sequence (CUDA
                                      events around it on the server's stream; -1 if
                                      unavailable): the uploads read in its first
                                      kernel, the batched frame, the result copy       */
} dri_server_tick;

/* Copies the most recent min(cap, recorded) ticks (the server keeps the last
 * 65536 since creation or the last stats reset), oldest first, into out[0 .. *n). */
int dri_server_trace_read(dri_server srv, dri_server_tick* out, int32_t cap, int32_t* n);

/* Waits for the stream and copies out x1 and, when non-NULL, the prior
 * H* (n x n, row-major) and b* (n) that the next frame will use: n = 17, or
 * 18 for a stream with gravity_dof = DRI_GRAVITY_3D. */
int dri_get_state(dri_stream s, dri_state* x1, double* H_prior, double* b_prior);

/* Replaces x1 and, when non-NULL, the prior (checkpoint / resume; sizes as
 * dri_get_state).  The prior mean becomes x1. */
int dri_set_state(dri_stream s, const dri_state* x1, const double* H_prior, const double* b_prior);

/* Parity / debug entry: linearises every term of Eq. 6 at the given (x0, x1)
 * on pyramid level `level` of the uploaded frame against the stream's
 * reference, prior and IMU, without changing the stream.  W_IMU is taken at x0.
 * flags (nullable, host, width_l * height_l bytes) receives per pixel
 * bit 0 = ICP correspondence valid, bit 1 = photometric valid, for a valid
 * ICP correspondence its reference pixel (x_i, y_i) as x_i mod 4 in bits 2-3
 * and y_i mod 4 in bits 4-5, bit 6 = the ICP term's decision was a margin
 * decision, bit 7 = the photometric term's (as counted by
 * dri_track_result.n_margin).  The terms are evaluated by the same pixel
 * kernel (and rows per thread) that dri_track runs for the stream. */
int dri_linearise(dri_stream s, int32_t level, const dri_state* x0, const dri_state* x1,
                  dri_linearisation* out, uint8_t* flags);

/* Static description of a status code. */
const char* dri_status_string(int code);

/* Kernel launches this stream has issued since creation (all kernels of the
 * library, counted on the host at launch). */
int dri_launch_count(dri_stream s, int64_t* count);

/* Waits for the stream's frames and returns how many tracked frames (the
 * initialising one included) finished with DRI_OK and how many failed
 * (DRI_ELOST, or DRI_ENOTREADY for a frame queued behind a failed one). */
int dri_frame_counts(dri_stream s, int64_t* ok, int64_t* failed);

/* Host<->device bytes the library copied for the last frame: the uploaded
 * images (host uploads only) plus the staged IMU samples, and the result block
 * copied back by dri_track. */
int dri_io_bytes(dri_stream s, int64_t* h2d, int64_t* d2h);

/* Per-kernel-class device time, measured with CUDA events recorded on the
 * stream around each launch while profiling is enabled (tracing aid; adds two
 * event records per launch).  Classes: */
#define DRI_KC_MAPS     0   /* level-0 copy, pyramid downsample, normal maps      */
#define DRI_KC_TRACK    1   /* fused photometric + ICP linearisation and reduction */
#define DRI_KC_SOLVE    2   /* Gauss-Newton step (IMU, assembly, Cholesky, update) */
#define DRI_KC_FRAME    3   /* frame begin / end / init (IMU weight, Schur)        */
#define DRI_KC_GRAD     4   /* reference intensity-gradient maps                   */
#define DRI_KC_COUNT    8
typedef struct {
    int64_t launches[DRI_KC_COUNT];
    double ms[DRI_KC_COUNT];       /* summed device time per class                     */
    double pixels[DRI_KC_COUNT];   /* pixels processed per class (track: pixel-iterations) */
} dri_profile;

/* Starts (enable = 1) or stops (0) recording; starting clears the counters. */
int dri_profile_enable(dri_stream s, int32_t enable);

/* Waits for the stream and returns the counters recorded since profiling was
 * enabled (up to 65536 launches are timed; later ones are counted only). */
int dri_profile_read(dri_stream s, dri_profile* out);

/* Linearisation of one image pair without any allocation.  The paper has no
 * counterpart: this entry exists for callers that may not allocate device
 * memory when they call the library (a host framework that owns all device
 * memory and forbids allocation in its per-frame callback, a real-time thread
 * that must not block in the allocator, work recorded during CUDA stream
 * capture).  Creating a stream allocates, so such code cannot use the stream
 * API on the fly; this call needs only the caller's buffers.
 *
 * Inputs: cfg (intrinsics of the images, sigma_I, sigma_d, ICP thresholds, the
 * depth range, precision_flags, occlusion_thr and icp_depth_weight, each with
 * the meaning it has for a stream; levels, iterations and IMU fields are
 * ignored); the
 * reference and live depth / intensity images, width * height FP32 each,
 * row-major, packed, in device memory; the pose the reference images were taken
 * at (x_ref) and the states x0, x1 to linearise at.  Output (device memory):
 * *out receives the ICP and photometric fields of dri_linearisation exactly as
 * dri_linearise fills them for a one-level stream (H_icp, b_icp, H_rgb, b_rgb,
 * cost_icp, cost_rgb, n_icp, n_rgb, n_margin_icp, n_margin_rgb; H, b, e_imu and
 * cost_imu are zeroed);
 * flags (nullable, device, width * height bytes) the per-pixel validity,
 * association and margin bits, encoded as by dri_linearise.
 * Work is enqueued on cuda_stream; the call does not wait.
 *
 * DRI_EINVAL for a NULL argument, an option value a stream would reject, or a
 * state that is not finite or whose q_WC is zero.
 *
 * Every intermediate (normal and gradient maps, per-block partial sums, the
 * block counter and per-call transforms) lives in one static device array of
 * the library (about 4.0 MB per GPU, held until the process exits), sized for
 * at most 320 x 240 pixels: larger images return DRI_EINVAL.  The CUDA runtime
 * reserves the array when it loads the library's device code on a GPU; with
 * lazy module loading (the default since CUDA 12.2) that is the first call made
 * with that GPU current, so the first call reserves it and later calls reserve
 * nothing.  The array is shared by all calls on a device and keeps the last
 * call's contents; each call clears what must start at zero.  Calls whose GPU
 * work overlaps race on it: order them on one stream.  The first call made with
 * a device current looks up the array's device address for that device
 * (cudaGetSymbolAddress); make that first call before any stream capture. */
int dri_linearise_pair_noalloc(const dri_stream_config* cfg, const float* ref_depth,
                               const float* ref_intensity, const float* live_depth,
                               const float* live_intensity, const dri_state* x_ref,
                               const dri_state* x0, const dri_state* x1,
                               dri_linearisation* out, uint8_t* flags, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DRI_H */
