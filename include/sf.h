/*
 * sf.h -- C ABI of libsf, a B300 (sm_103a) implementation of the per-frame
 * predictor-update loop of "Real-time Structure Flow" (Adarve & Mahony,
 * arXiv 2406.18031, Sec. 4 and Fig. 3).
 *
 * The filter estimates, at every pixel, the structure flow w (the scene's
 * 3-D velocity relative to the camera scaled by inverse range, rad/s;
 * Sec. 3.1, Eq. 10) and the inverse depth rho = lambda_ref / lambda (Eq. 8)
 * from a stream of grayscale images and range maps.  Each frame:
 *   prediction   -- upwind finite-difference transport of the previous
 *                   state over N sub-iterations (Sec. 4.4, Sec. 4.6);
 *   update       -- brightness and inverse-depth model fits (Sec. 4.2,
 *                   4.3), a per-pixel 3x3 least-squares solve (Sec. 4.5,
 *                   Eqs. 42-50), inverse-depth blend (Eq. 52) and 5x5
 *                   smoothing, on every level of an image pyramid;
 *   reconstruct  -- w_h = up(w_{h+1}) + dw_h down to full resolution
 *                   (Eq. 26).
 *
 * Conventions
 *   - Images are H x W, row-major, contiguous float32.  Pixel (i, j) is row
 *     i, column j.  The camera is a pinhole (fx, fy, cx, cy in pixels); the
 *     ray of pixel (i, j) passes through ((j + 0.5 - cx)/fx, (i + 0.5 -
 *     cy)/fy, 1).  Level h (1 = full resolution) is the pinhole grid with
 *     the intrinsics divided by 2^(h-1).
 *   - All pointers marked "device" must be CUDA device (or managed) memory
 *     on the current device; "host" pointers are ordinary host memory
 *     (pinned memory makes the copies asynchronous).  The library never
 *     frees memory it did not allocate.
 *   - Every call returns SF_OK (0), a negative error code, or a positive
 *     warning.  Nothing throws across the ABI.  Calls that take a stream
 *     enqueue work on it and return without waiting unless stated.
 *   - Calls on one context must not run concurrently from several host
 *     threads; different contexts are independent.
 */
#ifndef SF_H
#define SF_H

#ifdef __cplusplus
extern "C" {
#endif

#define SF_MAX_LEVELS 4

/* return codes */
#define SF_OK 0
#define SF_EINVAL (-1)      /* invalid argument or configuration            */
#define SF_ENOMEM (-2)      /* device or host allocation failed             */
#define SF_ECUDA (-3)       /* a CUDA runtime call failed                   */
#define SF_ETIMEOUT (-4)    /* a bounded device wait gave up                */
#define SF_ENONFINITE (-5)  /* the state became NaN or infinite             */
#define SF_WARN_CFL 1       /* a prediction broke dt*max|speed| <= 1 (Eq. 67) */

/* sf_params.flags */
#define SF_DOMINANT_LITERAL 1 /* dominant speed = neighbour of SMALLER |u|, the
                                 literal text of Eqs. 55-56 (default: larger) */
#define SF_SOURCE_SPLIT 2     /* apply the source term -f<eta,w> with dt/2 in
                                 each axis pass (once per sub-iteration, as in
                                 Eq. 53) instead of dt in both printed passes */
#define SF_CHECK_CFL 4        /* record SF_WARN_CFL when Eq. 67 is violated   */
#define SF_CHECK_FINITE 8     /* record SF_ENONFINITE for NaN/Inf output flow */
#define SF_IMU 32             /* add the inertial source terms to the prediction:
                                 the terms the paper drops by its assumption in
                                 Sec. 4.4, -Omega x w + a_w of the total-derivative
                                 equation of Sec. 3 with a_w = -rho a_c -
                                 Omega x (w + Omega x eta) (acceleration sign from
                                 the camera's equation of motion dv_c/dt =
                                 -Omega x v_c + a_c; the derivation prints
                                 +rho a_c), integrated once per sub-iteration after
                                 the two axis passes; lower levels turn their
                                 increment by -2 Omega x dw.  Omega and a_c come
                                 from sf_set_motion / sf_batch_motion.          */
#define SF_AUTOTUNE 16        /* at creation, time the propagation launches of one
                                 frame for each nf_max in {8, 6, 4, 3, 2} that
                                 splits the N_h differently and keep the fastest
                                 (overrides sf_params.nf_max; see sf_nf_max);
                                 then, with update_mode 0 and/or solve_tile 0,
                                 time whole frames for every update mode and
                                 solve tile edge left open and keep the fastest
                                 (see sf_update_mode, sf_solve_tile)          */

typedef struct sf_params {
    float fx, fy, cx, cy;          /* level-1 pinhole intrinsics, pixels              */
    int iters[SF_MAX_LEVELS];      /* N_h, propagation sub-iterations of level h (index
                                      0 = level 1); 0 selects ceil(max_flow / 2^(h-1)) */
    float max_flow;                /* largest expected flow, px/frame at level 1      */
    int smooth_iters[SF_MAX_LEVELS]; /* S_h, 5x5 smoothing passes after each solve    */
    float gamma[5];                /* gains gamma1..gamma5 of Eqs. 42, 47, 51; the
                                      prior weight of level h is gamma[2] * (2^(h-1)/fx)^2 */
    float lambda_ref;              /* reference range of Eq. 8, metres (1.0)          */
    int flags;                     /* SF_* flags above                                */
    int nf_max;                    /* sub-iterations fused in one propagation launch,
                                      1..8; 0 selects 8.  Level h then runs
                                      ceil(N_h / nf_max) launches of about equal
                                      length (a launch of nf sub-iterations
                                      recomputes an nf-pixel halo around each
                                      (64 - 2 nf)^2 output tile)                   */
    int update_mode;               /* how the smoothing and reconstruction of Sec. 4.5
                                      and Eq. 26 are launched: 1 = one launch per
                                      pyramid depth, top first, each smoothing a level
                                      and reconstructing it from the coarser level's
                                      result; 2 = one launch smoothing every level,
                                      then one light reconstruction launch per lower
                                      depth (fewer dependent launches, more traffic);
                                      0 = 1, or the autotuner's choice under SF_AUTOTUNE */
    int solve_tile;                /* edge of the square pixel tiles of the solve launch
                                      (Eqs. 30-52 per pixel): 16 or 32; 0 = 16 when the
                                      levels' 32-pixel tiles number at most 5 per SM
                                      (about one wave: short CTAs overlap the
                                      propagation launch before them), else 32, or the
                                      autotuner's choice under SF_AUTOTUNE.  Results
                                      are the same up to rounding order            */
} sf_params;

typedef struct sf_ctx sf_ctx;      /* opaque; owns all device state of one stream     */

/* Fill *p with defaults for an H x W image with `levels` pyramid levels:
 * fx = fy = W/2 (90 degree field of view), principal point at the centre,
 * max_flow = 1, iters = 0 (derive from max_flow), smooth = 2 at level 1 and
 * 4 above (Tables 2-4), gamma = (1, 1, 1e-2, 1, 1), lambda_ref = 1,
 * flags = SF_CHECK_CFL.  Returns SF_EINVAL for a NULL pointer. */
int sf_params_default(sf_params* p, int H, int W, int levels);

/* Create a filter for H x W frames with `levels` levels (1..SF_MAX_LEVELS = 4;
 * the coarse levels are built on the fly, 4^(h-1) input reads per pixel).
 * H and W must be divisible by 2^(levels-1); every level must be at least
 * 8 x 8; H x W at most 2^30.  Allocates all device state on the current device (about 128 bytes
 * per level-1 pixel, the coarser levels adding a third).  *out receives the
 * context; on error *out is NULL. */
int sf_create(int H, int W, int levels, const sf_params* p, sf_ctx** out);

/* Forget the state: the next sf_step initialises (Sec. 5.2: zero initial
 * flow) and returns zero flow. */
int sf_reset(sf_ctx* c);

/* One frame k -> k+1 on `stream` (a cudaStream_t; NULL = legacy default).
 *   image        device, H x W float32, brightness (any affine scale; [0, 1] typical)
 *   range        device, H x W float32, range lambda along the ray in metres;
 *                lambda <= 0, NaN or Inf means "no measurement" at that pixel
 *   dt           frame time in seconds (> 0); a change of dt between frames
 *                rescales the state, which is kept in rad/frame
 *   flow_out     device, 3 x H x W float32 (x, y, z planes) structure flow in
 *                rad/s, or NULL
 *   invdepth_out device, H x W float32 inverse depth, or NULL
 * Inputs must stay valid, and outputs untouched, until the stream reaches
 * the step.  Asynchronous: no host synchronisation. */
int sf_step(sf_ctx* c, const float* image, const float* range, float dt,
            float* flow_out, float* invdepth_out, void* stream);

/* sf_step on HOST buffers: copies image and range to the device, runs the
 * step and copies the outputs back, then waits for `stream` and for the
 * library's own copy stream.  The input copies run on that internal stream,
 * after the work already queued on `stream`, beside the propagation (which
 * reads only the state); the update waits for them, and the output copies run
 * on `stream`.  Pinned host buffers make the copies run at full speed.  image
 * and range hold H x W floats each.  SF_EINVAL for a null context, image or
 * range, or a dt that is not finite and positive (before any copy). */
int sf_step_host(sf_ctx* c, const float* image, const float* range, float dt,
                 float* flow_out, float* invdepth_out, void* stream);

/* Pipelined sf_step on HOST buffers, for a stream of frames: enqueues the
 * copy of image and range to a device staging slot (on a copy stream of the
 * context), the step (on `stream`) and the copy of the outputs back to
 * flow_out / invdepth_out (on a second copy stream), then returns without
 * waiting.  Frame k's input copy, frame k-1's step and frame k-2's output
 * copy can so run at the same time; three staging slots, reused in turn
 * (about 72 bytes per level-1 pixel, allocated by the first call).  Same
 * arguments and meaning as sf_step_host (host pointers; dt > 0 and finite,
 * else SF_EINVAL).  *ticket (if not NULL) receives the frame's number, 0 for
 * the first call, -1 on error.  The caller keeps image and range unchanged,
 * and flow_out / invdepth_out unread and alive, until sf_wait_host(c, ticket)
 * returns.  Pinned host memory (cudaHostAlloc / cudaHostRegister) lets the
 * call return at once; with pageable memory the CUDA runtime may wait inside
 * the copies.  Frames are processed in submission order; mixing with sf_step
 * on the same stream keeps that order. */
int sf_submit_host(sf_ctx* c, const float* image, const float* range, float dt,
                   float* flow_out, float* invdepth_out, void* stream, long long* ticket);

/* Wait until the outputs of frame `ticket` (from sf_submit_host; -1 = every
 * frame submitted so far) are in host memory, and its inputs are no longer
 * read.  SF_EINVAL for a NULL context or a ticket not yet issued; SF_ECUDA
 * if the wait failed. */
int sf_wait_host(sf_ctx* c, long long ticket);

/* Synchronise the device and return the sticky status recorded since the
 * last call (and clear it): SF_ENONFINITE, then SF_WARN_CFL, else SF_OK. */
int sf_status(sf_ctx* c);

/* Checkpoint access to level h (0-based) on `stream`.  dst/src are device
 * buffers of 8 x H_h x W_h float32 planes: w (3), rho, dw (3), Y-hat.  At
 * the top level w is the state; below it w is the reconstructed flow.
 * Flow planes are in rad/frame at frame time *dt_prev (get: written if not
 * NULL; set: read, must be > 0).  sf_set_state marks the context as
 * initialised. */
int sf_get_state(sf_ctx* c, int level, float* dst, float* dt_prev, void* stream);
int sf_set_state(sf_ctx* c, int level, const float* src, float dt_prev, void* stream);

/* Number of kernel launches one sf_step enqueues after the first frame (the
 * propagation launches, the solve launch and one smoothing/reconstruction
 * launch per pyramid level); a negative code for a NULL context. */
int sf_kernels_per_step(const sf_ctx* c);

/* Camera motion over the next frame interval for SF_IMU: omega = angular
 * velocity (rad/s, 3 floats), accel = linear acceleration with respect to an
 * inertial frame (m/s^2, 3 floats), both in the camera frame (Sec. 3; an IMU
 * measures them).  Host pointers; NULL means zero.  Copied to the device on
 * `stream` (pageable copy: the call returns once the values are staged);
 * the next sf_step calls on that stream use them, converted to frame units
 * with that step's dt (Omega dt, a dt^2).  SF_EINVAL for a NULL context or a
 * non-finite value.  Without SF_IMU the values are not read. */
int sf_set_motion(sf_ctx* c, const float* omega, const float* accel, void* stream);

/* The nf_max the context runs with (sf_params.nf_max, or the autotuner's
 * choice under SF_AUTOTUNE); a negative code for a NULL context.  The paper
 * has no such setting: it is how the N sub-iterations of Sec. 4.6 are cut
 * into launches. */
int sf_nf_max(const sf_ctx* c);

/* The update_mode the context runs with (1 or 2; see sf_params). */
int sf_update_mode(const sf_ctx* c);

/* The solve tile edge the context runs with (16 or 32; see sf_params). */
int sf_solve_tile(const sf_ctx* c);

/* Per-launch device timing.  sf_profile(c, 1) makes every following sf_step
 * record a CUDA event pair around each of its kernel launches, on the
 * step's stream; sf_profile(c, 0) stops it.  sf_profile_read waits for the
 * recorded work, writes for each launch slot of a step (the propagation
 * launches, the update, the reconstruction launches; n slots at most) the
 * summed milliseconds into ms[slot] and the number of timed launches into
 * *count, forgets the records, and returns the number of slots. */
int sf_profile(sf_ctx* c, int enable);
int sf_profile_read(sf_ctx* c, float* ms, int* count, int n);

/* Release everything the context owns.  NULL is a no-op. */
void sf_destroy(sf_ctx* c);

/* Static description of a return code. */
const char* sf_strerror(int code);

/* ------------------------------------------------------------------------
 * Batched streams.  One sf_batch holds n independent filters (camera
 * streams) of possibly different sizes and level counts and runs a frame of
 * all of them with one set of launches (the propagation launches, one
 * update launch and the reconstruction cascade), so that many small streams
 * fill the GPU; each stream computes exactly what its own sf_step would.
 * In steady state (same dt as the previous frame, a non-default stream) the
 * frame is replayed from a CUDA graph captured on an earlier frame.
 * ---------------------------------------------------------------------- */

typedef struct sf_batch sf_batch;

/* Create n streams: stream s is H[s] x W[s] with levels[s] levels and the
 * parameters params[s] (validated as in sf_create; all streams must use the
 * same SF_DOMINANT_LITERAL / SF_SOURCE_SPLIT choice; nf_max, update_mode,
 * solve_tile and SF_AUTOTUNE are taken from params[0]).  The batch owns one
 * device input slot (image, range) and one output slot (flow 3 x H x W,
 * inverse depth) per stream, zero-filled; see sf_batch_buffers. */
int sf_batch_create(int n, const int* H, const int* W, const int* levels, const sf_params* params,
                    sf_batch** out);

/* Device pointers of stream s's slots (any may be NULL): the caller writes
 * the frame's image and range there (on the step's stream or before it) and
 * reads the flow (rad/s) and inverse depth there after the step.  The
 * pointers stay valid until sf_batch_destroy. */
int sf_batch_buffers(sf_batch* b, int s, float** image, float** range, float** flow, float** invdepth);

/* One frame of every stream on `stream` (asynchronous; dt in seconds is the
 * same for every stream of the batch; the first step initialises). */
int sf_batch_step(sf_batch* b, float dt, void* stream);

/* As sf_status, for the whole batch. */
int sf_batch_status(sf_batch* b);

/* Kernel launches of one steady-state sf_batch_step. */
int sf_batch_launches_per_step(const sf_batch* b);

/* As sf_nf_max, for the whole batch (every stream uses params[0].nf_max and
 * params[0].flags' SF_AUTOTUNE). */
int sf_batch_nf_max(const sf_batch* b);
int sf_batch_update_mode(const sf_batch* b);
int sf_batch_solve_tile(const sf_batch* b);

/* Stream s's motion slot for SF_IMU (the batch takes SF_IMU from
 * params[0].flags): *motion receives a device pointer to 6 floats, Omega
 * (rad/s) then a_c (m/s^2), camera frame, zero at creation and owned by the
 * batch.  Write it on the stepping stream before sf_batch_step; the step
 * reads it on the device (so graph replays see new values) and converts it
 * with dt as sf_set_motion does. */
int sf_batch_motion(sf_batch* b, int s, float** motion);

/* As sf_profile / sf_profile_read for a batch; while profiling, steps run as
 * plain launches (no graph replay) so each launch can be timed. */
int sf_batch_profile(sf_batch* b, int enable);
int sf_batch_profile_read(sf_batch* b, float* ms, int* count, int n);

void sf_batch_destroy(sf_batch* b);

/* ------------------------------------------------------------------------
 * Stage entry points.  Each runs one stage of the frame on caller-owned
 * device buffers with the same kernels that sf_step uses, so that every
 * stage can be checked on its own.  They upload a small launch descriptor
 * and wait for `stream` once to do so; the kernels themselves stay
 * asynchronous.  State planes are interleaved
 * H x W x 4 float32 ("float4"): s0 = (w_x, w_y, w_z, rho), s1 = (dw_x, dw_y,
 * dw_z, Y).  w and dw are in rad/frame.
 * ---------------------------------------------------------------------- */

typedef struct sf_grid {
    int H, W;                /* level size                                   */
    float fx, fy, cx, cy;    /* level intrinsics (level-1 values / 2^(h-1))  */
} sf_grid;

/* Prediction of one level (Sec. 4.4, Sec. 4.6, Eqs. 53-66): N sub-iterations
 * with dt = 1/N.  Top level: s1_in and s1_out are NULL; w and rho are
 * transported by w (Eqs. 36-37).  Lower level: w, dw, rho and Y are
 * transported by w (Eqs. 38-41).  wscale multiplies w and dw on load (frame
 * time change).  status (device int, may be NULL) receives bit 1 when
 * Eq. 67 is violated.  Inputs and outputs must not overlap.  When N is
 * larger than one launch can fuse, the sub-iterations are split over several
 * launches that pass the fields through stream-ordered scratch memory
 * (cudaMallocAsync). */
int sf_propagate(const sf_grid* g, int N, int flags, float wscale,
                 const float* s0_in, const float* s1_in, float* s0_out, float* s1_out,
                 int* status, void* stream);

/* sf_propagate with the inertial source terms of SF_IMU (set or not in
 * flags): imu = host pointer to 6 floats in frame units, Omega dt (rad per
 * frame) then a_c dt^2 (m per frame^2); the source step runs once per
 * sub-iteration with dt = 1/N.  SF_EINVAL for a NULL or non-finite imu. */
int sf_propagate_imu(const sf_grid* g, int N, int flags, float wscale, const float* imu,
                     const float* s0_in, const float* s1_in, float* s0_out, float* s1_out,
                     int* status, void* stream);

/* sf_propagate without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory --
 * real-time loops that must not touch the allocator (cudaMalloc and
 * cudaFree can block and synchronise the device), hosts whose memory pools
 * belong to another framework, code that has been handed a fixed memory
 * budget.  It computes exactly what sf_propagate computes,
 * with the same arguments, but keeps the fields passed between launches and
 * the launch descriptors in a file-scope device array of 33 MiB that every
 * GPU using this library holds until the process exits; it calls no
 * cudaMalloc, cudaMallocAsync or cudaFree.
 *   - H * W must not exceed 1,048,576 pixels (e.g. 1024 x 1024); larger
 *     grids return SF_EINVAL (use sf_propagate).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the array, which keeps the last call's contents (every
 *     value a call reads there it has written first).  Calls whose work
 *     overlaps on the GPU -- on different streams or different host threads
 *     without ordering between them -- race on the array.
 *   - The call enqueues two small descriptor kernels ahead of each
 *     propagation launch (which is then an ordinary, fully stream-ordered
 *     launch, since its descriptors come from those kernels) and returns
 *     without waiting for the stream. */
int sf_propagate_noalloc(const sf_grid* g, int N, int flags, float wscale,
                         const float* s0_in, const float* s1_in, float* s0_out, float* s1_out,
                         int* status, void* stream);

/* Update of one level (Sec. 4.2, 4.3, 4.5; Eqs. 30-34, 42-52) with S
 * smoothing passes.  `level` is 1-based; the level's image and inverse
 * depth are built from the level-1 inputs (H1 x W1 device arrays) by 2x2
 * means (no-measurement children excluded from the depth mean).
 *   top: the unknown is w (prior p0.xyz; temporal terms use Y-hat = s1_cur.w
 *        and rho = s0_cur.w); writes s0_new = (w, rho), s1_new = (0, Y-hat).
 *   lower: the unknown is dw (prior p1.xyz; temporal terms use p1.w and
 *        p0.w); writes s1_new = (dw, Y-hat) and s0_new.w = rho; s0_new.xyz is
 *        left for sf_reconstruct.
 *   init != 0: the first frame (w = dw = 0, rho = rho-hat, Y-hat = model);
 *        s0_cur, s1_cur, p0, p1 are not read.
 * gamma[2] is the level's prior weight as used (already scaled).  diag (may
 * be NULL): H x W x 12 float32 per pixel: Y-hat, d_eta Y-hat (3), rho-hat
 * (0 = none), d_eta rho-hat (3), unsmoothed solution (3), 0. */
int sf_update(const sf_grid* g, int level, int top, int S, int init, const float* gamma,
              float lambda_ref, const float* image, const float* range, int H1, int W1,
              const float* s0_cur, const float* s1_cur, const float* p0, const float* p1,
              float* s0_new, float* s1_new, float* diag, void* stream);

/* Reconstruction (Eq. 26) of levels < top from new states: for h = top-1 ..
 * 1, w_h = bilinear x2 up(w_{h+1}) + dw_h written to s0[h].xyz; then the
 * outputs of level 1: flow_out = w_1 / dt (3 x H x W) and invdepth_out =
 * rho_1, either may be NULL.  s0[h], s1[h] are the levels' device planes
 * (index 0 = level 1); grids[h] their sizes.  status bit 2 (device int, may
 * be NULL) is set when check_finite and a flow value is not finite. */
int sf_reconstruct(int levels, const sf_grid* grids, float* const* s0, const float* const* s1,
                   float dt, float* flow_out, float* invdepth_out, int check_finite,
                   int* status, void* stream);

/* ----------------------------------------------------------------------
 * Mapping camera data onto the filter's grid.  The paper maps its panoramic
 * renders and camera frames onto its grid before filtering and counts that
 * step in its runtime (Sec. 6, "Urban Canyon" and "ZED" experiments); the
 * resampling itself is not described there.  Every grid pixel (i, j) of
 * `dst` (the level-1 sf_grid of a filter) casts the ray through its centre,
 * ((j + 0.5 - cx)/fx, (i + 0.5 - cy)/fy, 1), rotated into the source's frame
 * by R (3 x 3 row-major, source <- grid; x right, y down, z forward).
 * Brightness: bilinear between source pixel centres, edges replicated.
 * Range: the value of the source pixel containing the projected point (no
 * interpolation across occlusion edges).  A source pixel k covers [k, k+1).
 * src_image, src_range: device Hs x Ws float32; out_image, out_range: device
 * dst->H x dst->W float32; src_range and out_range are both NULL or both
 * set.  SF_EINVAL for bad sizes, pointers or non-finite R / intrinsics
 * (checked before any device call).  Asynchronous on `stream`.
 * ---------------------------------------------------------------------- */

/* A pinhole frame with intrinsics cam = (fx, fy, cx, cy) (pixels): rays
 * behind the camera or projecting outside [0, Ws] x [0, Hs] get brightness 0
 * and range 0 (no measurement). */
int sf_remap_pinhole(const sf_grid* dst, const float* R, int Hs, int Ws, const float* cam,
                     const float* src_image, const float* src_range, float* out_image,
                     float* out_range, void* stream);

/* An equirectangular panorama: column u spans longitude 2 pi u / Ws - pi
 * (0 = forward, +x to the right), row v latitude pi/2 - pi v / Hs (up
 * first); the direction of (longitude phi, latitude th) is
 * (cos th sin phi, -sin th, cos th cos phi); longitude wraps around. */
int sf_remap_equirect(const sf_grid* dst, const float* R, int Hs, int Ws, const float* src_image,
                      const float* src_range, float* out_image, float* out_range, void* stream);

/* ----------------------------------------------------------------------
 * Learned propagation surrogate (no counterpart in the paper: a small
 * convolutional network trained on the plain propagation's own output).
 * ---------------------------------------------------------------------- */

/* One 3x3 convolution layer, stride 1, zero padding 1, on the tensor cores
 * (BF16 operands, FP32 accumulation):
 *   y[n,i,j,co] = act(bias[co] + sum_{dy,dx,ci} w[3 dy + dx][co][ci] x[n, i+dy-1, j+dx-1, ci])
 * act = ReLU when relu != 0, else identity.  x: device N x H x W x Cin
 * bfloat16 (NHWC); w: device 9 x Cout x Cin bfloat16; bias: device Cout
 * float32 or NULL; y: device N x H x W x Cout bfloat16 or NULL; y32: the
 * same in float32 or NULL (at least one of y, y32).  Cin and Cout are 16 or
 * 32; pointers 16-byte aligned.  status (device int, may be NULL) gets bit 4
 * if a bounded wait for the tensor cores gave up.  SF_EINVAL for bad
 * shapes or pointers (checked before any device call). */
int sf_conv3x3(int N, int H, int W, int Cin, int Cout, const void* x, const void* w,
               const float* bias, int relu, void* y, float* y32, int* status, void* stream);

/* Weight and bias gradients of one 3x3 layer (the contraction over pixels
 * of the surrogate's training step):
 *   dw[3 dy + dx][co][ci] = sum_{n,i,j} g[n,i,j,co] x[n, i+dy-1, j+dx-1, ci]
 *   db[co] = sum_{n,i,j} g[n,i,j,co]
 * with x outside the frame read as zero.  x: device N x H x W x Cin
 * bfloat16 (NHWC); dy = g: device N x H x W x Cout bfloat16; dw: device
 * 9 x Cout x Cin float32 and db: device Cout float32, both overwritten
 * (FP32 accumulation).  Cin and Cout are 16 or 32; pointers 16-byte
 * aligned.  SF_EINVAL for bad shapes or pointers (checked before any device
 * call).  Asynchronous on `stream`. */
int sf_conv3x3_wgrad(int N, int H, int W, int Cin, int Cout, const void* x, const void* dy,
                     float* dw, float* db, void* stream);

/* Self-test of the convolution's bounded wait: runs one tile whose MMAs are
 * never issued, so its mbarrier wait cannot complete; the kernel gives up
 * after a short poll limit, sets the timeout bit, frees its tensor memory and
 * returns.  Returns SF_ETIMEOUT when that happened (the expected outcome),
 * SF_OK when the wait somehow completed, another code on a CUDA error.  The
 * device stays usable afterwards.  Waits for `stream`. */
int sf_selftest_conv_timeout(void* stream);

/* The same self-test for the fused surrogate network (sf_surrogate_forward's
 * kernel): one 16 x 16 frame whose MMAs are never issued, so the epilogue's,
 * the producer's and the MMA thread's bounded waits give up; the kernel sets
 * the timeout bit, frees its tensor memory and returns.  Returns SF_ETIMEOUT
 * when that happened (the expected outcome), SF_OK when a wait somehow
 * completed, another code on a CUDA error.  Waits for `stream`. */
int sf_selftest_net_timeout(void* stream);

/* The surrogate network: 4 such layers, 16 -> 32 -> 32 -> 32 -> 16 channels,
 * ReLU after the first three.  Input features of a pixel of the top level:
 * w / (4 dmu) (3 channels, px/frame over 4), rho, eta_x, eta_y, 10 zeros;
 * output channels 0..3: the change over one frame in the same units, so the
 * prediction is w + 4 dmu o[0..2], rho + o[3].  It replaces the N
 * sub-iterations of the top-level propagation (Sec. 4.6) once trained on
 * (state, plain prediction) pairs.  Parameters: per layer the weights
 * 9 x Cout x Cin (tap-major) then Cout biases, FP32 master copy; BF16 copies
 * feed the tensor cores. */
typedef struct sf_surrogate sf_surrogate;

/* Seeded He-normal initialisation (a small last layer: nearly no change). */
int sf_surrogate_create(unsigned long long seed, sf_surrogate** out);
void sf_surrogate_destroy(sf_surrogate* s);
/* Number of FP32 parameters (a negative code for NULL). */
int sf_surrogate_num_params(const sf_surrogate* s);
/* Copy the FP32 parameters to (set = 0) or from (set != 0) host memory;
 * setting rebuilds the BF16 copies; non-finite values give SF_EINVAL. */
int sf_surrogate_params(sf_surrogate* s, float* host, int set);
/* Gradient of the last training step's loss (FP32, parameter layout). */
int sf_surrogate_grads(sf_surrogate* s, float* host);
/* Predict: s0 = n frames of the grid g's top-level state (device
 * n x H x W float4 (w_x, w_y, w_z, rho), w in rad/frame) -> p0 (same layout).
 * The features, the four layers and the head run in one tensor-core kernel
 * that keeps the features and the hidden activations in shared memory (only
 * the state and the prediction touch HBM); it allocates nothing.  Up to 64
 * frames per launch. */
int sf_surrogate_forward(sf_surrogate* s, const sf_grid* g, int n, const float* s0, float* p0,
                         void* stream);
/* The same prediction computed layer by layer (the forward pass of
 * sf_surrogate_train_step): every hidden activation goes to HBM as BF16 and
 * back.  The same arithmetic at the same rounding points as
 * sf_surrogate_forward; kept for comparison and measurement. */
int sf_surrogate_forward_layered(sf_surrogate* s, const sf_grid* g, int n, const float* s0, float* p0,
                                 void* stream);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) on the mean squared error, over
 * the 4 used output channels in the network's units, between the
 * prediction from s0 and `target` (the plain propagation's p0 of the same
 * states).  *loss_out (host, may be NULL) receives the loss before the step
 * (the call then waits for the stream).  SF_ETIMEOUT if a tensor-core wait
 * gave up. */
int sf_surrogate_train_step(sf_surrogate* s, const sf_grid* g, int n, const float* s0,
                            const float* target, float lr, float* loss_out, void* stream);
/* The surrogate as the top-level prediction with its fallback: p0 = the
 * surrogate's prediction of s0, checked against one plain step (the plain
 * propagation with N = 1): if the largest flow difference over all pixels
 * and frames exceeds threshold_px (px/frame; NaN always does), p0 is
 * recomputed by the plain propagation with N sub-iterations.
 * *residual_px and *used_plain (host, may be NULL) receive the largest
 * difference and whether the fallback ran.  Waits for the stream (the
 * decision is taken on the host). */
int sf_surrogate_propagate(sf_surrogate* s, const sf_grid* g, int n, int N, const float* s0, float* p0,
                           float threshold_px, float* residual_px, int* used_plain, void* stream);
/* Let a filter's top level (every stream's, for a batch) be predicted by the
 * surrogate instead of the plain propagation (NULL restores the plain one).
 * The lower levels keep the plain propagation.  The surrogate's buffers are
 * sized here; it serves one filter or batch at a time and must outlive the
 * attachment.  Steady-state batch steps re-capture their graphs.
 * Every frame then checks each stream's prediction on the device, with no
 * host decision (so the frame stays one captured graph): one plain
 * sub-iteration (N = 1) of the top level, the largest flow difference to the
 * surrogate's prediction over the stream's pixels (px/frame), and the plain
 * propagation of the Sec. 4.6 scheme with the level's N sub-iterations
 * replacing the prediction of every stream whose difference exceeds its
 * threshold (default 1 px/frame) or is NaN. */
int sf_set_surrogate(sf_ctx* c, sf_surrogate* s);
int sf_batch_set_surrogate(sf_batch* b, sf_surrogate* s);

/* NVTX ranges (one per frame and one per stage launch: propagation,
 * surrogate, its fallback check, solve, smoothing and reconstruction of each
 * pyramid depth) for a system trace: enable != 0 turns them on for every
 * filter and batch of the process, 0 (the default) off.  They mark the host
 * side of each launch; with a tracing tool attached each costs microseconds
 * of host time, so they are off unless asked for.  Always SF_OK. */
int sf_set_trace(int enable);

/* Threshold (px/frame, >= 0; +inf: never fall back) of the surrogate's
 * fallback: for a filter, or for batch stream s (s = -1: every stream, and
 * the default of later attachments).  Synchronous copy to the device; takes
 * effect from the next frame, captured graphs included.  SF_EINVAL for a
 * negative or NaN threshold, a bad s, or s >= 0 before any attachment. */
int sf_set_surrogate_threshold(sf_ctx* c, float threshold_px);
int sf_batch_set_surrogate_threshold(sf_batch* b, int s, float threshold_px);

/* Waits for the device, then returns per stream (the first n of a batch; a
 * filter has one) the last frame's largest difference between the
 * surrogate's prediction and one plain step (px/frame) and the number of
 * frames whose prediction fell back to the plain propagation since the
 * attachment.  Either output may be NULL.  SF_EINVAL before any attachment. */
int sf_surrogate_stats(sf_ctx* c, float* residual_px, int* fallbacks);
int sf_batch_surrogate_stats(sf_batch* b, float* residual_px, int* fallbacks, int n);

#ifdef __cplusplus
}
#endif
#endif /* SF_H */
