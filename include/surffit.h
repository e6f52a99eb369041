/*
 * surffit.h -- C ABI of the GB300 dense RGBD plane-fitting library (libsurffit.so).
 *
 * Method: "Real-Time Surface Fitting to RGBD Sensor Data" (Papadakis & Willis).
 * For every pixel p of a depth image and a k x k window centred on it, the
 * library fits the plane n.P + d = 0 (|n| = 1, d > 0) to the window's valid
 * 3D points and returns the unit normal n, the offset d (metres, the distance
 * of the plane from the camera centre) and the curvature
 * lambda0 / (lambda0 + lambda1 + lambda2) of the fit's 3x3 scatter matrix.
 *
 *   - SF_METHOD_DISPARITY: the implicit fit in RGBD space, Eq. 12 and Eq. 14:
 *     monomials [tan(theta_x), tan(theta_y), 1, 1/Z].  Only the four 1/Z
 *     entries of the scatter matrix depend on the depth (Section II.A).
 *   - SF_METHOD_STANDARD: the implicit algebraic fit of Eq. 3-6 with monomials
 *     [X, Y, Z, 1], X and Y from Eq. 1 -- the comparison fit.
 *   - SF_METHOD_EXPLICIT_DISPARITY / SF_METHOD_EXPLICIT_STANDARD: the explicit
 *     fits of Eq. 15-16 (1/Z = a tan(theta_x) + b tan(theta_y) + c) and
 *     Eq. 7-9 (Z = a X + b Y + c), least squares over the same exact window
 *     sums; the plane is returned as n.P + d = 0 like the implicit fits.  Their
 *     third output is the mean squared residual in the fit's own units (1/m^2
 *     and m^2) instead of the curvature.  A window whose valid pixels are
 *     collinear in the image has no unique explicit fit and gets NaN.
 *
 * Rays follow Eq. 10: tan(theta_x) = (x + dx - cx)/fx, tan(theta_y) =
 * (y + dy - cy)/fy, with x the column and y the row, both 0-based.
 * A pixel is missing when its depth is not finite or <= 0 (uint16: raw == 0).
 * Windows are clipped at the image border.  The fit is written for p when at
 * least min_valid window pixels are valid and (if require_center_valid) p
 * itself is; otherwise normal, offset and curvature are NaN.
 *
 * The implicit fits use the constraint |(a, b, c)| = 1: the offset is
 * eliminated (Schur complement of the 4x4 scatter matrix) and the normal is
 * the eigenvector of the smallest eigenvalue of the remaining 3x3 matrix
 * (Eq. 4-5).
 *
 * Conventions for every call:
 *   - Device pointers are CUDA device memory of the device current at
 *     sf_create; host pointers are ordinary host memory.  Images are dense,
 *     row-major, pitch = W elements; normals are [H][W][3] float.
 *   - The caller owns every buffer it passes.  A context owns its scratch and
 *     tables and frees them in sf_destroy.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device calls
 *     enqueue work and return without synchronising the host.
 *   - Every call returns SF_OK or an error status; argument errors are found
 *     before any launch and leave the outputs untouched.  sf_last_error()
 *     returns a message for the calling thread's last failure.
 *   - A context is not safe for concurrent use from several streams: its
 *     scratch is shared by all its calls.
 */
#ifndef SURFFIT_H_
#define SURFFIT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SF_OK = 0,
    SF_ERR_INVALID_ARG = 1, /* null pointer, bad size, even or too large window ... */
    SF_ERR_UNSUPPORTED = 2, /* a valid request this build does not implement     */
    SF_ERR_ALLOC = 3,       /* device or host allocation failed                  */
    SF_ERR_CUDA = 4,        /* a CUDA runtime call failed                         */
    SF_ERR_TIMEOUT = 5      /* a bounded device-side wait gave up                 */
} sf_status;

/* SF_DEPTH_DISPARITY_U16: raw sensor disparity D (uint16, 0 = missing) with
 * 1/Z = alpha D + beta (sf_set_disparity_model); the disparity form then
 * fits the measured disparity directly, without any Z -> 1/Z conversion
 * (the future work of the paper's conclusion). */
typedef enum { SF_DEPTH_F32 = 0, SF_DEPTH_U16 = 1, SF_DEPTH_DISPARITY_U16 = 2 } sf_depth_type;

typedef enum {
    SF_METHOD_DISPARITY = 0,
    SF_METHOD_STANDARD = 1,
    SF_METHOD_EXPLICIT_DISPARITY = 2,
    SF_METHOD_EXPLICIT_STANDARD = 3
} sf_method;

/* Pinhole intrinsics of Eq. 1: focal lengths and principal point in pixels,
 * (dx, dy) the constant pixel-coordinate adjustment. */
typedef struct {
    double fx, fy, cx, cy, dx, dy;
} sf_intrinsics;

typedef struct sf_ctx sf_ctx;

/* Largest supported window: k <= SF_MAX_WINDOW (the exact integer window sums
 * are sized for at most 31 x 31 = 961 pixels). */
#define SF_MAX_WINDOW 31

/*
 * sf_create -- precompute the calibration tables for one camera, image size
 * and window (Section II.A: the ray terms depend only on the intrinsics, so
 * they are computed once, before any depth is seen) and allocate scratch.
 *   K        intrinsics (host pointer, read during the call)
 *   W, H     image size in pixels, >= 1
 *   window   odd k, 1 <= k <= SF_MAX_WINDOW
 *   out      receives the new context
 * Defaults: disparity method, float32 metres, min_valid 3, centre required.
 * Synchronises the device once.  Errors: SF_ERR_INVALID_ARG, SF_ERR_ALLOC,
 * SF_ERR_CUDA.
 */
sf_status sf_create(const sf_intrinsics* K, int W, int H, int window, sf_ctx** out);

/*
 * sf_set_params -- choose the fit and the depth encoding.
 *   method        an sf_method value
 *   depth_type    SF_DEPTH_F32 (metres), SF_DEPTH_U16 (raw units, 0 = missing) or
 *                 SF_DEPTH_DISPARITY_U16 (raw disparity, model from sf_set_disparity_model)
 *   depth_scale   metres per raw unit for SF_DEPTH_U16 (ignored for f32), > 0
 *   min_valid     minimum number of valid window pixels, >= 1
 *   require_center_valid  nonzero: the centre pixel must be valid
 */
sf_status sf_set_params(sf_ctx* ctx, int method, int depth_type, float depth_scale, int min_valid,
                        int require_center_valid);

/*
 * sf_set_disparity_model -- the sensor model of SF_DEPTH_DISPARITY_U16 input,
 * 1/Z = alpha D + beta (1/metres; e.g. alpha = 1/(f b s) for a stereo pair of
 * baseline b and focal length f reporting disparity in 1/s pixel, beta = 0).
 * The library holds the model as 1/Z = (|alpha| / 128) (sign(alpha) 128 D + B + f)
 * with B + f = 128 beta / |alpha| (B an integer, f in [0, 1) stored as a
 * float32): the exact window sums hold the integers sign(alpha) 128 D + B,
 * and the fraction f, common to every pixel, enters the solve through the
 * mean disparity.  The model is therefore reproduced to float32 rounding of
 * |alpha| / 128 (a common scale, which moves no normal) and of f.  A pixel is
 * missing when D == 0 or its 1/Z <= 0.
 * Errors: SF_ERR_INVALID_ARG unless alpha is finite and nonzero and
 * |128 beta / alpha| <= 2^23; a later disparity-form fit rejects a model
 * whose largest value 128 * 65535 + |B| + 1 times the window size k reaches 2^31.
 * Default: alpha = 1, beta = 0.
 */
sf_status sf_set_disparity_model(sf_ctx* ctx, double alpha, double beta);

/*
 * Normalisation of the implicit fits (Eq. 4).  Section I.C's Euclidean
 * invariance holds for |(a, b, c)| = 1, the default: the offset is eliminated
 * and the normal is the smallest eigenvector of the 3x3 Schur complement.  The
 * literal constraint of Eq. 4, |(a, b, c, d)| = 1, takes the smallest
 * eigenvector alpha of the whole 4x4 scatter matrix in metric units (metres,
 * 1/metres): n = alpha[0:3] / |alpha[0:3]|, d = alpha[3] / |alpha[0:3]|,
 * curvature = lambda0 / trace of the 4x4.  Its result depends on the units.
 */
typedef enum { SF_CONSTRAINT_UNIT3 = 0, SF_CONSTRAINT_UNIT4 = 1 } sf_constraint;

/*
 * sf_set_constraint -- choose the normalisation for the implicit fits of this
 * context (SF_CONSTRAINT_UNIT3 default).  With SF_CONSTRAINT_UNIT4, sf_fit,
 * sf_fit_ex and sf_fit_host solve the 4x4 problem (explicit methods:
 * SF_ERR_UNSUPPORTED at fit time); sf_fit_backward and sf_quadtree return
 * SF_ERR_UNSUPPORTED.  sf_set_precision applies to both constraints.
 */
sf_status sf_set_constraint(sf_ctx* ctx, int constraint);

/*
 * sf_set_precision -- precision of the per-pixel solve (Eq. 4-5: the normal is
 * the eigenvector of the smallest eigenvalue of R, whose error under a
 * perturbation dR is about |dR| / (lambda1 - lambda0)).  The window sums are
 * exact integers of the depth (or disparity) in fixed point, 26-28 bits per
 * frame; the modes differ in the solve and in how the fixed-point rounding of
 * the depth is treated:
 *   0  float32 solve (default).  Normal error ~ 3e-8 / gamma rad against an
 *      FP64 fit of the same data, gamma = (lambda1 - lambda0) / lambda2, plus
 *      the effect of the rounding.
 *   1  float32 solve, then every window with gamma < tau, or whose rounding
 *      could move its normal by more than 3e-5 rad (an estimate from the
 *      float32 eigenvalues), is queued: its normal is refined in double-float
 *      (pairs of float32) from the same exact moments, and where the
 *      refined estimate of the rounding's effect (5.5 standard deviations)
 *      still exceeds 3e-5 rad the window's depth is re-summed without the
 *      rounding before refining again; the queued windows' outputs are
 *      overwritten.  The estimate treats the pixels' rounding errors as
 *      independent, which holds unless many depths of a window repeat exactly
 *      (depths quantised coarsely at the source).  Measured on 1080p frames at
 *      k = 31: within 3e-5 rad of the FP64 fit of the unrounded depth on
 *      every window with gamma >= 1e-6.
 *   2  the refinement and the re-summing for every window (slow: every
 *      window reads its k x k depth again): agreement with the FP64 fit to
 *      ~1e-7 rad, whatever the data.
 * tau in (0, 1] (mode 1; default 1e-3).  Modes 1 and 2 allocate on the next fit
 * a queue of 8 bytes per pixel plus the queued windows' moments (80 bytes for
 * a quarter of the pixels in mode 1, for every pixel in mode 2).  The explicit
 * fits and the |(a,b,c,d)| = 1 constraint are re-solved in FP64 from the exact
 * moments instead (mode 1 leaves the explicit fits in float32).
 */
sf_status sf_set_precision(sf_ctx* ctx, int mode, float tau);

/*
 * sf_precision_stats -- for the context's most recent fit pass (the last group
 * of up to 64 frames of its last sf_fit / sf_fit_ex / sf_fit_host call) in
 * precision mode 1 or 2: the number of windows queued for refinement and the
 * number among them re-summed from the depth (both 0 in mode 0).  Waits for
 * the context's device to finish its queued work.
 */
sf_status sf_precision_stats(sf_ctx* ctx, unsigned long long* queued, unsigned long long* resummed);

/*
 * sf_fit -- fit every pixel of one frame.
 *   depth      device [H][W] float32 metres or uint16 raw (per sf_set_params)
 *   normals    device [H][W][3] float32, out
 *   offsets    device [H][W] float32, out
 *   curvature  device [H][W] float32, out (mean squared residual for explicit fits)
 * Every buffer must be aligned to its element size (SF_ERR_INVALID_ARG
 * otherwise; CUDA allocations always are).  Asynchronous on `stream`.
 */
sf_status sf_fit(sf_ctx* ctx, const void* depth, float* normals, float* offsets, float* curvature, void* stream);

/*
 * sf_fit_ex -- sf_fit for n_frames frames of the context's size stored back to
 * back ([n_frames][H][W] in, [n_frames][H][W][3] / [n_frames][H][W] out), with
 * optional per-pixel valid-window counts (device int32 [n_frames][H][W] or NULL).
 */
sf_status sf_fit_ex(sf_ctx* ctx, int n_frames, const void* depth, float* normals, float* offsets, float* curvature,
                    int32_t* counts, void* stream);

/*
 * sf_fit_host -- sf_fit_ex on HOST buffers (pageable or page-locked memory;
 * page-locked buffers let the copies run as DMA in both directions): the
 * frames go through in up to four chunks on two context-owned streams, the
 * copy-out of one chunk overlapping the copy-in and fit of the next, with
 * copies straight between the caller's buffers and two device staging
 * buffers owned by the context.  Work already queued on `stream` runs first;
 * the call returns when every result is in the caller's buffers.  Same
 * layouts as sf_fit_ex; counts may be NULL.
 */
sf_status sf_fit_host(sf_ctx* ctx, int n_frames, const void* depth, float* normals, float* offsets, float* curvature,
                      int32_t* counts, void* stream);

/*
 * sf_fit_backward -- gradient of L = sum_p (g_normals_p . n_p + g_offsets_p d_p
 * + g_curvature_p kappa_p) with respect to the depth, for the implicit fits
 * (SF_METHOD_DISPARITY, SF_METHOD_STANDARD).  The fit is differentiated as the
 * paper defines it: the Schur complement of the scatter matrix (Eq. 6 / Eq. 14
 * with the offset eliminated), its smallest eigenvector (Eq. 4-5), the offset
 * and the curvature; dL/dZ at a pixel collects the contributions of every
 * window containing it.  Invalid windows contribute nothing; missing pixels
 * get 0.  The normal's sign is treated as locally constant (the orientation
 * rule), and the gradient is undefined where lambda0 == lambda1.
 *   depth                      device, as for sf_fit_ex ([n_frames][H][W])
 *   g_normals                  device float [n_frames][H][W][3] (NaN-free)
 *   g_offsets, g_curvature     device float [n_frames][H][W]
 *   g_depth                    device float [n_frames][H][W], out: dL/dZ with Z in metres
 *                              (for uint16 input, times depth_scale gives dL/d(raw))
 * Errors: SF_ERR_UNSUPPORTED for the explicit fits.  Asynchronous on `stream`.
 */
sf_status sf_fit_backward(sf_ctx* ctx, int n_frames, const void* depth, const float* g_normals, const float* g_offsets,
                          const float* g_curvature, float* g_depth, void* stream);

/*
 * sf_fit_backward_ex -- sf_fit_backward with flags.  SF_BACKWARD_AFTER_FIT:
 * the caller promises that `depth` holds the same values as when the last
 * sf_fit_ex call on this context fitted it (that call ordered before this
 * one on the device); the backward then reuses that fit's quantum and row
 * sums (the forward's range and row passes, Section II.C's window sums)
 * instead of computing them again.  The library itself checks the rest: the
 * same buffer, frame count and settings, at most 64 frames (one pass), no
 * per-pixel delta table and no call on the context in between that wrote its
 * scratch (another fit, sf_fit_host, a backward of other frames,
 * sf_quadtree); when any of that fails the row pass runs as without the flag
 * (results are the same either way).  The promise itself cannot be checked:
 * a depth changed in between gives the gradient of a mixture.  flags = 0 is
 * sf_fit_backward.  Errors as sf_fit_backward.
 */
#define SF_BACKWARD_AFTER_FIT 1u
sf_status sf_fit_backward_ex(sf_ctx* ctx, int n_frames, const void* depth, const float* g_normals,
                             const float* g_offsets, const float* g_curvature, float* g_depth, unsigned flags,
                             void* stream);
/* sf_backward_reuses -- how many backward calls on this context reused the last fit's row pass. */
sf_status sf_backward_reuses(const sf_ctx* ctx, long long* n);

/*
 * Mixed-resolution batches.  One frame of a batch: its size, window and
 * intrinsics, its device buffers (layouts as for sf_fit), and optionally its
 * tile shape (0 = default): hseg in {32, 64, 128} columns per horizontal
 * tile, vband in [8, 1024] rows per vertical band.
 */
typedef struct {
    int W, H, window;
    sf_intrinsics K;
    const void* depth;
    float* normals;
    float* offsets;
    float* curvature;
    int hseg, vband;
} sf_batch_frame;

typedef struct sf_batch sf_batch;

/*
 * sf_batch_create -- prepare the fit of n_frames frames of any sizes and
 * windows as one pass (the per-frame fit of Eq. 12-14 / Eq. 3-6 with the
 * window sums of Section II.C): a table of per-frame descriptors and of work
 * items is uploaded once, and every pass is ONE persistent kernel launch
 * whose CTAs claim items with an atomic counter, in this order: the quantum
 * chunks of every frame, its horizontal tiles, its column bands.  A tile
 * waits for its frame's quantum, a band for its frame's tiles; each wait
 * polls a counter at most a set number of times (sf_batch_set_wait_limit),
 * and one that gives up records it for sf_batch_check and skips its item.
 * With use_graph != 0 the pass (two counter resets and the launch) is
 * captured once in a CUDA graph and sf_batch_run replays it.  The device
 * buffers named in `frames` are bound for the life of the batch: refill them
 * and run again.  Method, depth type and validity rule are shared by all
 * frames (disparity or standard implicit fit; SF_ERR_UNSUPPORTED for the
 * explicit fits).  Synchronises once.
 */
sf_status sf_batch_create(const sf_batch_frame* frames, int n_frames, int method, int depth_type, float depth_scale,
                          int min_valid, int require_center_valid, int use_graph, sf_batch** out);
/* sf_batch_run -- one pass of the batch on `stream` (asynchronous). */
sf_status sf_batch_run(sf_batch* batch, void* stream);
/*
 * sf_batch_check -- waits for the last pass to finish and returns
 * SF_ERR_TIMEOUT if one of its waits gave up (that pass's outputs are then
 * incomplete; the batch stays usable), else SF_OK.
 */
sf_status sf_batch_check(sf_batch* batch);
/*
 * sf_batch_set_wait_limit -- polls per wait of the following passes (default
 * 2^22, about a second; 0: every wait that has something to wait for gives
 * up at once).  Waits for the last pass to finish first.
 */
sf_status sf_batch_set_wait_limit(sf_batch* batch, unsigned polls);
/* sf_batch_info -- total pixels (plane fits) per pass and kernel launches per pass (1). */
sf_status sf_batch_info(const sf_batch* batch, long long* pixels, int* launches);
/* sf_batch_destroy -- free the batch (NULL is a no-op). */
sf_status sf_batch_destroy(sf_batch* batch);

/*
 * sf_set_delta_table -- per-pixel ray adjustments (Eq. 1 and Eq. 10 add an
 * adjustment (dx, dy) to a pixel's coordinates before its ray is formed; this
 * gives every pixel its own, added to the intrinsics' dx, dy):
 *   ddx, ddy   host float [H][W] in pixels, |value| < 16, finite; read during
 *              the call and stored on the device rounded to 1/2^18 pixel
 *              (both NULL: remove the table)
 * With a table, sf_fit / sf_fit_ex / sf_fit_host of SF_METHOD_DISPARITY (either
 * constraint, every precision mode) use the per-pixel rays; every other
 * method, sf_fit_backward and sf_quadtree return SF_ERR_UNSUPPORTED while a
 * table is set.  In precision modes 1 and 2 the windows that the float32
 * solve queues (mode 1: gap below tau or a rounding estimate above 3e-5 rad;
 * mode 2: every window) are solved again in FP64 from the unrounded depth and
 * the stored rays, one warp per window: exact to FP64 rounding, at the cost
 * of one k x k re-read per queued window.  The table takes 8 B per pixel and
 * its scratch 84 B per pixel instead of 20.  Synchronous: waits for the
 * context's device to finish its queued work before replacing a table; do not
 * call it while a stream capture is in progress on that device.
 * Errors: SF_ERR_INVALID_ARG (one table NULL, entry out of range),
 * SF_ERR_ALLOC, SF_ERR_CUDA.
 */
sf_status sf_set_delta_table(sf_ctx* ctx, const float* ddx, const float* ddy);

/*
 * sf_set_tiles -- tile shape of a context: hseg in {8, 16, 32, 64, 128}
 * output columns per thread of the horizontal pass (0, the default: 32, or
 * 16 / 8 for calls with too few rows to fill the GPU), vband rows per
 * vertical band (0 = chosen from the grid size, else 2..1024).  Results do
 * not depend on the tiles: the window sums are exact.  SF_ERR_INVALID_ARG
 * for any other value.
 */
sf_status sf_set_tiles(sf_ctx* ctx, int hseg, int vband);


/* sf_destroy -- free the context and everything it owns (NULL is a no-op). */
sf_status sf_destroy(sf_ctx* ctx);

/* Message for the calling thread's most recent error ("" if none). */
const char* sf_last_error(void);

/*
 * sf_channel_counts -- how many per-pixel depth-dependent channels the
 * method's window sums carry, and how many depend on the validity mask only
 * (the paper's calibration-only terms, Section II.D).  Host-only, no device
 * work.  Returns SF_ERR_INVALID_ARG for an unknown method.
 */
sf_status sf_channel_counts(int method, int* depth_channels, int* mask_channels);

/*
 * sf_profile_enable / sf_profile_read -- per-stage CUDA-event timing of the
 * context's own launches, for benchmarks.  While enabled, every kernel launch
 * of the context is bracketed by two events on its stream.  sf_profile_read
 * waits for the recorded events, writes for each stage s < n_stages the
 * summed milliseconds ms[s] and the launch count launches[s], and clears the
 * record.  Stages: 0 range (quantum), 1 horizontal moments, 2 vertical
 * moments + solve, 3 precision fallback (modes 1-2: refinement, re-sums and
 * FP64 re-solves of the queued windows).  Enabling again
 * clears the record.
 */
sf_status sf_profile_enable(sf_ctx* ctx, int on);
sf_status sf_profile_read(sf_ctx* ctx, int n_stages, double* ms, int* launches);

#define SF_NUM_STAGES 4

/*
 * sf_fit_static -- the fit of sf_fit for one frame, without a context and
 * without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate when they need a fit
 * (work recorded while a CUDA graph is being captured, real-time loops that
 * forbid allocator calls after start-up, hosts whose own allocator owns the
 * GPU's memory).  Its scratch lives in one device array of
 * SF_STATIC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library holds until the process exits.
 *   K, W, H, window          as for sf_create
 *   method                   SF_METHOD_DISPARITY or SF_METHOD_STANDARD
 *   depth_type, depth_scale, min_valid, require_center_valid   as for sf_set_params
 *   depth, normals, offsets, curvature, stream                 as for sf_fit
 * Limits and errors: the frame's scratch (about 20 B per pixel for the
 * disparity form, 44 B for the standard form, plus the ray tables) must fit
 * in SF_STATIC_SCRATCH_BYTES, e.g. 1280x720 disparity or 640x480 standard;
 * larger frames are rejected with SF_ERR_INVALID_ARG and a message, before
 * any device work.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) and sets kernel attributes; make that
 * first call before any stream capture.  All calls on a device share the one
 * array and it keeps the previous call's contents (the kernels clear what
 * must start at zero), so calls whose work overlaps on the GPU -- on
 * different streams, or from several host threads -- race and corrupt each
 * other's results: serialise them.
 */
#define SF_STATIC_SCRATCH_BYTES (32u << 20)
sf_status sf_fit_static(const sf_intrinsics* K, int W, int H, int window, int method, int depth_type,
                        float depth_scale, int min_valid, int require_center_valid, const void* depth,
                        float* normals, float* offsets, float* curvature, void* stream);

/*
 * Planar segmentation by tile subdivision (Section III, planar segmentation
 * application): the image is cut into square root tiles from the top-left
 * corner (clipped at the right and bottom borders); each tile's plane is fitted
 * over all its valid pixels with the context's method; a tile whose fit error
 * is above the threshold is split into four children of half its width and
 * height (left/top halves floor(w/2), floor(h/2)), down to max_level
 * subdivisions.  The fit error is the root mean square of the residual the
 * method minimises, sqrt(residual / n): for the implicit fits lambda0 of the
 * Schur complement (the disparity form's residual is the point-to-plane
 * distance divided by the depth, unitless; the standard form's is the
 * point-to-plane distance in metres); for the explicit fits the residual of
 * their regression.  Every node is solved in FP64 from exact integer sums.
 * Clustering the plane coefficients (the paper's K-means step) is not part of
 * the library.
 */
typedef struct {
    int tile;               /* root tile side in pixels, 2..64 */
    int max_level;          /* subdivisions below the roots, 0..6 */
    float tau;              /* split threshold on the rms fit error (> 0, method units) */
    int min_valid_permille; /* a node needs >= max(min_valid, ceil(permille * area / 1000))
                               valid pixels, else it is SF_QUAD_INVALID; 0..1000 */
} sf_quad_params;

typedef enum {
    SF_QUAD_FIT = 0,        /* leaf: rms <= tau */
    SF_QUAD_SPLIT = 1,      /* inner node: rms > tau, its four children follow at level + 1 */
    SF_QUAD_HIGH_ERROR = 2, /* leaf: rms > tau at max_level (or a side of 1 pixel) */
    SF_QUAD_INVALID = 3     /* leaf: too few valid pixels, or valid pixels collinear in the image
                               (no surface fit with any method); fit fields NaN */
} sf_quad_status;

typedef struct {
    int32_t frame, x0, y0, w, h, level, status, count; /* rectangle [x0, x0+w) x [y0, y0+h) of frame */
    float normal[3], offset, curvature, rms;            /* fit (curvature: as for sf_fit) */
} sf_quad_node;

/*
 * sf_quadtree -- the segmentation of n_frames frames of the context's size.
 *   depth     device, as for sf_fit_ex ([n_frames][H][W])
 *   params    host pointer, read during the call
 *   nodes     device array of `capacity` sf_quad_node, out: every evaluated
 *             node (inner nodes included), in no particular order
 *   n_nodes   device int32, out: the number of nodes evaluated; when it
 *             exceeds `capacity` only `capacity` were stored
 * The context's method, depth type and min_valid apply (its window and
 * require_center_valid do not).  Asynchronous on `stream`; scratch (node
 * queues, sized for the deepest level) is owned by the context.
 * Errors: SF_ERR_INVALID_ARG for parameters out of range or null pointers.
 */
sf_status sf_quadtree(sf_ctx* ctx, int n_frames, const void* depth, const sf_quad_params* params, sf_quad_node* nodes,
                      int capacity, int32_t* n_nodes, void* stream);

/* Library version as a static string. */
const char* sf_version(void);

/*
 * sf_debug_fail_allocs -- test hook for the error paths: the next `after`
 * device allocations of the library succeed and every later one fails as if
 * the device were out of memory (SF_ERR_ALLOC, every partial allocation
 * freed), until called again with a negative value (the default: no limit).
 * Process-wide; not for concurrent use with working contexts.
 */
sf_status sf_debug_fail_allocs(long long after);
/*
 * sf_graph_replays -- the number of sf_fit_ex calls on this context that were
 * served by replaying its captured CUDA graph (a call that repeats the
 * previous one's frames, buffers and settings is captured, and later such
 * calls replay it); the other calls launched their kernels one by one.
 */
sf_status sf_graph_replays(const sf_ctx* ctx, long long* n);
/* sf_debug_live_allocs -- the number of the library's device allocations not yet freed (all contexts and batches). */
sf_status sf_debug_live_allocs(long long* n);

/*
 * sf_eval_acos -- diagnostics: the float32 arccos that the per-pixel solve's
 * trigonometric eigenvalue estimate uses (the closed-form roots of the 3x3
 * characteristic polynomial behind Eq. 4-5), evaluated on the device for n
 * values:
 *   x   device float [n], each in [-1, 1]
 *   y   device float [n], out
 * Errors: SF_ERR_INVALID_ARG (null pointer, n < 0, misaligned buffer).
 * Asynchronous on `stream`.
 */
sf_status sf_eval_acos(const float* x, float* y, int n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SURFFIT_H_ */
