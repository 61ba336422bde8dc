/*
 * ssvp.h - C ABI of the GB300 scene-space gather-and-filter library (libssvp.so).
 *
 * Method (Klose et al., "Sampling Based Scene-Space Video Processing"):
 *   every output pixel p of frame O is unprojected by its depth and camera (the reference
 *   sample s_ref, Sec. "Denoising"), projected into every frame J of a temporal window, and a
 *   k x k neighbourhood around the projection is tested: a candidate q is gathered when its own
 *   unprojection lies within radius r of the reference point (the back-projection test of
 *   Sec. "Sample Gathering", Eq. 2, seeded by the output depth).  The gathered set S(p) is
 *   reduced by the weighted mean of Eq. 3 with the weights of Eq. 4 (denoising) or of Eq. 13-14
 *   (virtual aperture), fused into the same CUDA kernel.
 *
 * Conventions (all entry points)
 *   - Every call returns an ssvp_status; nothing aborts.  ssvp_last_error() gives the text.
 *   - Work is queued on the context's CUDA stream.  Errors raised by queued work surface at a
 *     later call or at ssvp_sync().
 *   - Pixel (x, y) with integer coordinates is the pixel centre.  Depth is camera-space z.
 *     Depth values that are not finite or not > 0 are invalid and never gathered.
 *   - Images are row-major, frame-major: colour F*H*W*3 floats interleaved (r, g, b), depth
 *     F*H*W floats, output F*H*W*3 floats.
 *   - Inputs are copied; the caller keeps ownership of its buffers.  The library owns its
 *     device buffers until ssvp_destroy().
 *   - Caller buffers are checked for where they live before any work touches them: one given
 *     as device memory (SSVP_MEM_DEVICE, or documented as a device buffer) must be device
 *     memory of the context's device or managed memory, one given as or documented as host
 *     memory (cameras, shutter table, box, network weights, host outputs) must not be device
 *     memory; otherwise the call returns SSVP_EINVAL and queues nothing.
 *   - A context is not thread-safe: one host thread per context at a time.
 */
#ifndef SSVP_H
#define SSVP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssvp_ctx ssvp_ctx;

typedef enum {
    SSVP_OK = 0,
    SSVP_EINVAL = -1,    /* bad argument: shape, k, window, unsupported camera, null pointer */
    SSVP_ENOMEM = -2,    /* device or pinned host allocation failed */
    SSVP_ECUDA = -3,     /* a CUDA call failed (text in ssvp_last_error) */
    SSVP_ENOCLIP = -4,   /* clip id not loaded */
    SSVP_ENOCAM = -5,    /* cameras not set for the clip */
    SSVP_ETIMEOUT = -6,  /* a bounded device-side wait gave up */
    SSVP_EDEVICE = -7    /* no usable CUDA device */
} ssvp_status;

enum { SSVP_MEM_HOST = 0, SSVP_MEM_DEVICE = 1 };
enum { SSVP_COLOUR_F32 = 0, SSVP_COLOUR_F16 = 1 };
enum {
    SSVP_MODE_DENOISE = 0,   /* Eq. 4 weights (Sec. "Denoising") */
    SSVP_MODE_APERTURE = 1,  /* Eq. 13-14 (Sec. "Virtual aperture") */
    SSVP_MODE_LEARNED = 2,   /* per-sample weights from a small MLP, plain Eq. 4 as fallback */
    SSVP_MODE_MEAN = 3,      /* w = 1 (the plain average of Sec. "Denoising") */
    SSVP_MODE_DEBLUR = 4,    /* Eq. 5: Eq. 4 times the sample frame's gradient-magnitude sum
                                (Sec. "Deblurring"; see ssvp_frame_sharpness) */
    SSVP_MODE_SHUTTER = 5,   /* Eq. 10: w = xi(J - O) alone, xi from ssvp_set_shutter
                                (Sec. "Computational scene-space shutters") */
    SSVP_MODE_INPAINT = 6,   /* Eq. 8-9 with the frustum gather: masked pixels are replaced
                                (Sec. "Inpainting and semi-transparency"; see ssvp_set_mask) */
    SSVP_MODE_SEMI = 7       /* semi-transparency: Eq. 8-9 plus, in the second Eq. 9 step, the
                                Eq. 4 weight of every sample around the pixel's own sample (the
                                same section, after Eq. 9; see ssvp_set_mask) */
};
enum {
    SSVP_GATHER_WINDOW = 0,  /* depth-seeded k x k window + radius (or the aperture cone) */
    SSVP_GATHER_FRUSTUM = 1, /* the pixel frustum of Sec. "Sample Gathering", Eq. 1-2 */
    SSVP_GATHER_WINDOW_TMA = 2 /* the window gather of SSVP_GATHER_WINDOW, same samples and
                                results, with each warp's window footprint in frame J copied into
                                shared memory by a TMA tensor copy before its radius tests */
};

#define SSVP_MAX_CLIPS 64
#define SSVP_MAX_K 31
#define SSVP_MAX_HALF_WINDOW 127

/*
 * Parameters of one gather-and-filter call.  Fill with ssvp_params_default() first.
 *   mode          SSVP_MODE_*
 *   k             window width in pixels, odd, 1 <= k <= 31
 *   half_window   T: frames J = O-T .. O+T (clipped to the clip) are gathered, 0 <= T <= 127
 *   frame_begin, frame_end   output frames [frame_begin, frame_end) of each clip
 *   crop_*        output pixel rectangle; crop_w == 0 or crop_h == 0 means the full frame
 *   radius        gather radius r: > 0 absolute scene units, < 0 means |radius| times the
 *                 clip's lower-median valid input depth (computed at load)
 *   sigma_rgb, sigma_xyz, sigma_f   Eq. 4 standard deviations (colour units, scene units,
 *                 frames); sigma_xyz <= 0 means "equal to r"
 *   aperture, focal_depth, a0, lens_samples, cap   virtual aperture (Eq. 13-14): lens radius A,
 *                 focal depth z0 (<= 0: clip median depth), cone waist a0 (<= 0: 0.5 z0 / fx),
 *                 lens seed points (1..64), footprint cap per axis (odd, <= 63)
 *   max_samples, conf_threshold     learned filter: sample cap (<= 64), fallback threshold
 *   gather        SSVP_GATHER_WINDOW, or SSVP_GATHER_FRUSTUM: the paper's own gather (Sec.
 *                 "Sample Gathering", Eq. 1-2).  Every pixel q of every window frame J whose
 *                 back-projection into O has O depth in (near_plane, far_plane) and lands within
 *                 L1 distance frustum_l / 2 of the output pixel (|u - u'| + |v - v'| < l / 2,
 *                 strict) is a sample, whatever its depth; the output depth is not used to
 *                 gather, only for s_ref in Eq. 4 (an invalid output depth still gives c_ref).
 *                 Denoise, mean, deblur, shutter and inpaint modes; k is ignored and the radius
 *                 serves only as the default sigma_xyz.  Not available in batched plans.
 *                 SSVP_GATHER_WINDOW_TMA: the window gather with the candidate depths of each
 *                 warp (32 output pixels of a row) staged, frame by frame, into shared memory by
 *                 TMA tensor copies (a 48 x 12 box of frame J around the warp's windows, two
 *                 buffers, frame J + 1 copied while J is tested); lanes whose window is not
 *                 inside the box read the global plane.  Same samples and outputs as
 *                 SSVP_GATHER_WINDOW.  Denoise, mean, deblur and shutter modes, k <= 7; not in
 *                 batched plans.
 *   frustum_l, near_plane, far_plane   frustum size l in pixels (0 < l <= 64; the paper uses 3)
 *                 and its O depth range (0 < near < far; the paper uses 0.01 and 1000)
 *   sigma_area    ssvp_superres only: length scale of Eq. 7's area term (scene units); <= 0 means
 *                 one input-pixel footprint at the median depth (median depth / fx of O)
 *   test_skip_mma 0 normally.  1 (a test of the time-out paths): in learned mode the learned
 *                 inference issues none of its tensor-core products, so its bounded waits for
 *                 them run out (within about 1 s each); ssvp_sync then returns SSVP_ETIMEOUT, the
 *                 outputs of the call are not valid, and the context stays usable.  With
 *                 SSVP_GATHER_WINDOW_TMA the gather issues none of its tensor copies: each warp's
 *                 first wait runs out (about 1 s, then up to 2 s more waiting for copies that
 *                 might be in flight), the warp reads the global planes, ssvp_sync returns
 *                 SSVP_ETIMEOUT and the outputs are those of SSVP_GATHER_WINDOW.  Ignored otherwise.
 *   membership_out   optional device buffer (debug): per crop pixel (row-major) and per slot
 *                 j = 0..2T (J = O-T+j) a record of 3 + ceil(k*k/32) int32 words:
 *                 status (-2 invalid reference depth, -1 J outside the clip, 0 J skipped: the
 *                 reference point is behind camera J, 1 gathered, 2 no window pixel inside the
 *                 image), window centre x, y, then the accepted bits of the k x k window
 *                 (bit dy*k+dx).  In aperture mode the record is 5 + ceil(cap*cap/32) words:
 *                 status, the scanned box x0, y0, x1, y1 (inclusive, before clipping to the
 *                 image), then the accepted bits of the box (bit (y-y0)*cap + (x-x0)).  With
 *                 the frustum gather it is 4 words: status (-2, -1 as above, -2 also for an
 *                 unmasked pixel in inpainting, 0 the frustum
 *                 misses J's depth range or image, 1 scanned), the number of samples from J,
 *                 and the low and high words of the wrapping 64-bit sum over them of
 *                 SplitMix64's output function of qy*W + qx + 1 (an order-free checksum).
 *                 Only valid with a single output frame.
 *   pixel_stats_out  optional device buffer (debug): per crop pixel 3 words: int32 accepted,
 *                 int32 examined (window pixels inside the image), float sum of weights.
 */
typedef struct ssvp_params {
    int32_t mode;
    int32_t k;
    int32_t half_window;
    int32_t frame_begin;
    int32_t frame_end;
    int32_t crop_x, crop_y, crop_w, crop_h;
    float radius;
    float sigma_rgb;
    float sigma_xyz;
    float sigma_f;
    float aperture;
    float focal_depth;
    float a0;
    int32_t lens_samples;
    int32_t cap;
    int32_t max_samples;
    float conf_threshold;
    int32_t gather;
    float frustum_l;
    float near_plane;
    float far_plane;
    float sigma_area;
    int32_t test_skip_mma;
    void *membership_out;
    void *pixel_stats_out;
} ssvp_params;

/*
 * Super-resolution (Sec. "Super resolution", Eq. 6-7) of output frames [frame_begin, frame_end)
 * of clip `clip_id` on a grid of `scale` (1..8) times the input resolution per axis.  Output
 * pixel (U, V) sits at input coordinates ((U + 0.5) / scale - 0.5, (V + 0.5) / scale - 0.5);
 * its camera is K_O with fx, fy scaled and the principal point mapped the same way.  s_ref is
 * the bilinear interpolation of the input colour and depth there (coordinates clamped to the
 * image; an invalid depth among the four pixels makes the reference invalid and the output
 * the interpolated colour).  Samples are gathered from the output pixel's own frustum (the
 * frustum gather of Eq. 1-2 with frustum_l in output pixels, near_plane, far_plane) over the
 * window [O - half_window, O + half_window] and weighted by Eq. 7: Eq. 4 (sigma_rgb, sigma_xyz,
 * sigma_f; the paper uses sigma_rgb = 50 on a 0-255 scale) times exp(-s_area / (2
 * sigma_area^2)) with s_area = (d_q / fx_J)^2, the squared scene length of one pixel edge of the
 * sample at its depth (Eq. 6); SSVP_MODE_MEAN uses w = 1.  params.gather and k are ignored.
 * out: a device buffer of (frame_end - frame_begin) x (H scale) x (W scale) x 3 floats owned by
 * the caller (with a crop, in output-grid pixels, only the crop is written).  Debug outputs as
 * for the frustum gather, per output-grid crop pixel.  Queued on the context's stream.
 */
int ssvp_superres(ssvp_ctx *ctx, const ssvp_params *params, int clip_id, int scale, float *out);

/*
 * Inpainting mask of clip `clip_id` (Sec. "Inpainting and semi-transparency", Eq. 8-9): F*H*W
 * bytes, nonzero = the pixel shows something to remove, on the host (SSVP_MEM_HOST) or device
 * (SSVP_MEM_DEVICE), copied.  SSVP_MODE_INPAINT (with gather = SSVP_GATHER_FRUSTUM) replaces every
 * masked output pixel: it gathers the pixel's frustum S(p) (its own depth is not used), starts
 * from the mean colour of all of S(p) (Eq. 8) and takes two steps of the weighted mean with
 * w = exp(-|c_ref - c|^2 / (2 sigma_rgb^2)) over the unmasked samples (masked ones weigh 0,
 * Eq. 9), each step's result being the next step's c_ref; a step whose weights are all 0 keeps
 * its reference, an empty S(p) keeps the input colour.  Unmasked pixels keep their input colour.
 * The paper uses sigma_rgb = 55 on a 0-255 scale.  The mask lives until the clip is unloaded or
 * reloaded with another shape or colour format (a reload with the same ones keeps it).
 *
 * SSVP_MODE_SEMI (semi-transparency, same gather and mask) makes the masked region see-through
 * instead: its second step also gives every sample s of S(p), masked or not, the Eq. 4 weight
 * exp(-|I(p) - c_s|^2 / (2 sigma_rgb^2) - |x_ref - X_s|^2 / (2 sigma_xyz^2) - (J - O)^2 /
 * (2 sigma_f^2)) around the pixel's own sample (I(p), x_ref = D(p) K_O^-1 (u, v, 1), O), added to
 * its Eq. 9 weight, so the object's samples near x_ref blend with the background's estimate.  A
 * masked pixel without a valid depth gets the inpainting result.  The paper uses sigma_rgb = 80.
 */
int ssvp_set_mask(ssvp_ctx *ctx, int clip_id, const uint8_t *mask, int mem_kind);

/*
 * The same mask from a scene-space region (the paper's alternative to painted masks): box =
 * {xmin, ymin, zmin, xmax, ymax, zmax} in world coordinates (inclusive).  A pixel of any frame is
 * masked when its depth, unprojected with its frame's camera (FP64), gives a world point inside
 * the box; invalid depths are not masked.  Needs the clip's cameras; queued on the stream (the
 * cameras are copied before the call returns).
 */
int ssvp_mask_from_box(ssvp_ctx *ctx, int clip_id, const double *box);

/* Copy the clip's mask (F*H*W bytes, 0 or 1 for box masks) to host memory; waits for the stream. */
int ssvp_read_mask(ssvp_ctx *ctx, int clip_id, uint8_t *out);

/*
 * Shutter function xi of Eq. 10 (Sec. "Computational scene-space shutters") for
 * SSVP_MODE_SHUTTER: xi[j] weighs every sample from frame J = O - half_window + j,
 * j = 0 .. 2 half_window (host array, copied).  Values must be finite and >= 0; 0 drops a frame
 * from the average.  A box (all ones) is a long exposure, a single non-zero entry projects one
 * frame, a decaying tail leaves motion trails.  Shutter-mode calls must use this half_window.
 * The weight has no colour, position or frame-distance term; a pixel whose samples all weigh 0
 * keeps its input colour.  SSVP_EINVAL for a NULL table, a bad half_window or a bad value.
 */
int ssvp_set_shutter(ssvp_ctx *ctx, const float *xi, int half_window);

/*
 * Eq. 5's blurriness measure (Sec. "Deblurring") of every frame of clip `clip_id`: the sum over
 * the pixels that have a right and a lower neighbour of the forward-difference gradient
 * magnitude, the L2 norm over the three colour channels and both axes.  Computed on the device
 * when the clip is loaded, from the stored colour (FP16-rounded with SSVP_COLOUR_F16), with a
 * deterministic FP64 reduction.  SSVP_MODE_DEBLUR multiplies the Eq. 4 weight of a sample from J
 * by out[J] / max(out) (the common scale cancels in Eq. 3).  out: F doubles on the host; the
 * call waits for the context's stream.
 */
int ssvp_frame_sharpness(ssvp_ctx *ctx, int clip_id, double *out);

/* Defaults: denoise, k = 7, T = 15, radius = 0.5 % of the median depth, sigma_rgb = 40/255
 * (the paper's 40 on a 0-255 scale, Sec. "Denoising"), sigma_xyz = r, sigma_f = 6, all frames
 * of the clip, full frame; aperture 0.05, focal depth = median, 16 lens points, cap 31;
 * learned cap 64, threshold 0.5; window gather, frustum l = 3, near 0.01, far 1000; no debug
 * outputs. */
void ssvp_params_default(ssvp_params *p);

/* Create a context on CUDA device `cuda_device`, queuing work on `cuda_stream` (a cudaStream_t;
 * NULL means the legacy default stream).  *out receives the context.  SSVP_EDEVICE when no
 * usable device exists. */
int ssvp_create(ssvp_ctx **out, int cuda_device, void *cuda_stream);

/* Release every device and host resource of the context (waits for queued work).  NULL is a no-op. */
void ssvp_destroy(ssvp_ctx *ctx);

/* Text of the last error on this context (or of the last failed ssvp_create when ctx is NULL). */
const char *ssvp_last_error(const ssvp_ctx *ctx);

/* Change the stream later calls queue work on. */
int ssvp_set_stream(ssvp_ctx *ctx, void *cuda_stream);

/*
 * Load clip `clip_id` (0 <= id < SSVP_MAX_CLIPS), replacing any clip with that id.
 * Inputs I and D of Sec. "Method overview": rgb F*H*W*3 floats (linear colour), depth F*H*W
 * floats (camera z), on the host (mem_kind = SSVP_MEM_HOST, pinned memory is fastest) or on
 * this context's device (SSVP_MEM_DEVICE).  colour_fmt selects the stored colour precision
 * (SSVP_COLOUR_F32 or SSVP_COLOUR_F16, round to nearest even); depth is always stored as FP32.
 * The lower-median valid depth is computed on the device for relative radii.
 * Sizes: 1 <= W, H <= 16384, 1 <= F <= 65535.  The copy is queued: the caller's buffers may be
 * reused once the context's stream has passed this call (ssvp_sync() waits for it).  The load
 * itself runs on the context's internal stream of the device's highest priority, after the
 * work queued on the context's stream before the call; the context's stream waits for it, so
 * work queued after the call sees the new clip.  (Its kernels are short: at high priority they
 * overlap a long gather another context runs on another stream.)  Host inputs up to 4 GB go to
 * the device in one copy through a staging buffer the context keeps.  Reloading
 * an id with the same W, H, F and colour_fmt reuses its device planes (and keeps its inpainting
 * mask, if one is set) without allocating; work already queued on the stream still sees the old
 * contents.
 * Any reload invalidates batched plans that include the id.
 */
int ssvp_load_clip(ssvp_ctx *ctx, int clip_id, int W, int H, int F, const float *rgb, const float *depth,
                   int mem_kind, int colour_fmt);

/* Drop a clip and free its device memory. */
int ssvp_unload_clip(ssvp_ctx *ctx, int clip_id);

/*
 * Slide a loaded clip's frames forward for streaming video: frames n .. F-1 become frames
 * 0 .. F-n-1 and the n new frames become frames F-n .. F-1, with their cameras (K: one shared 3x3
 * or n per-frame ones as in ssvp_set_cameras; w2c: n x 3 x 4).  rgb (n x H x W x 3) and depth
 * (n x H x W) as in ssvp_load_clip, on the host or the device; 1 <= n <= F.  Only the n new
 * frames cross to the device: the kept frames are copied on the device into a second window the
 * clip keeps (allocated by the first call: a second set of planes), which then becomes current.
 * The work runs on the context's load stream after the work queued before the previous append
 * (every gather that read the second window) and before the work queued after this call: it
 * overlaps gathers of the current window queued since the previous append (device inputs are
 * packed only after all work queued before this call, which may produce them).  The clip's median
 * and per-frame values are those of the new window; its output frames are not cleared.  Needs
 * the cameras set and no inpainting mask; invalidates batched plans that include the clip.
 */
int ssvp_append_frames(ssvp_ctx *ctx, int clip_id, int n, const float *rgb, const float *depth, int mem_kind,
                       const double *K, int per_frame_K, const double *w2c);

/*
 * Cameras C of Sec. "Method overview" for clip `clip_id`, in double precision on the host:
 * K intrinsics (3x3 row-major, shared: per_frame_K = 0, or F of them: per_frame_K = 1), upper
 * triangular with zero skew and K[2][2] = 1; w2c world->camera [R|t] (F x 3x4 row-major, R a
 * rotation).  The library composes the per-(O, J) transforms in FP64 (C_O C_J^-1 of Eq. 2).
 */
int ssvp_set_cameras(ssvp_ctx *ctx, int clip_id, const double *K, int per_frame_K, const double *w2c);

/*
 * Gather and filter output frames [frame_begin, frame_end) of each listed clip with the same
 * parameters (Sec. "Sample Gathering" + Eq. 3).  Results go to the clip's output buffer, read
 * with ssvp_read_output().  Statistics of this call (examined and accepted samples, sum of
 * weights) replace the previous ones; read them with ssvp_read_stats().  Queued on the stream.
 */
int ssvp_gather_filter(ssvp_ctx *ctx, const ssvp_params *params, const int *clip_ids, int n_clips);

/* Copy output frames [frame_begin, frame_end) of a clip (full frames, F*H*W*3 layout) to `dst`
 * on the host (mem_kind = SSVP_MEM_HOST; waits for completion) or device (SSVP_MEM_DEVICE;
 * queued).  Pixels no gather call has written since the clip was loaded hold 0 (a reload with the
 * same shape clears the frames written before it). */
int ssvp_read_output(ssvp_ctx *ctx, int clip_id, int frame_begin, int frame_end, float *dst, int mem_kind);

/* Device pointer of a clip's output buffer (F*H*W*3 floats, owned by the library).  The caller
 * may write it; the next same-shape reload then clears the whole buffer. */
int ssvp_output_device_ptr(ssvp_ctx *ctx, int clip_id, void **dev_ptr);

/*
 * Kernel timing (no counterpart in the paper; a measurement aid).  While tracing is on
 * (ssvp_trace_enable(ctx, 1); off when a context is created), each gather, learned-filter
 * (extraction, inference, training, Adam), mask and batched-plan launch the context queues is
 * bracketed by a pair of CUDA timing events on its stream and recorded under one of the kinds
 * below; so is the whole of each ssvp_load_clip / ssvp_append_frames (copies and kernels on the
 * load stream: one SSVP_TRACE_LOAD entry per call) and the per-frame values a call computes the
 * first time it needs them after one (the frames' depth ranges for the frustum gathers, the Eq. 5
 * gradient sums for deblurring and ssvp_frame_sharpness: one more SSVP_TRACE_LOAD entry), and a
 * batched plan's launch (one CUDA graph) is one SSVP_TRACE_BATCH entry.  Not traced: the autotuner's trial launches, the expansion of
 * ssvp_learned_samples and the weight conversion of ssvp_set_mlp.  ssvp_trace_read waits for the
 * traced work; for each kind with launches since the last read, in increasing kind order and at
 * most max_kinds of them, it writes the kind, the launch count and the summed device time in
 * milliseconds, sets *n_kinds to the number written, and clears the record (kinds beyond
 * max_kinds are dropped).  The times are those of the bracketed stream intervals: work that
 * overlaps on other streams shares the device and is not subtracted.  Arrays are host memory,
 * owned by the caller; any of kind, launches, ms, n_kinds may be NULL.  Errors: SSVP_EINVAL (NULL
 * ctx, max_kinds < 0), SSVP_ECUDA.
 */
enum {
    SSVP_TRACE_GATHER = 0,    /* window gather and filter (denoise, mean, deblur, shutter) */
    SSVP_TRACE_APERTURE = 1,  /* virtual-aperture gather (Eq. 13-14) */
    SSVP_TRACE_FRUSTUM = 2,   /* frustum gather (Eq. 1-2): filter, inpainting, semi-transparency */
    SSVP_TRACE_SUPERRES = 3,  /* frustum gather on the super-resolution grid (Eq. 6-7) */
    SSVP_TRACE_EXTRACT = 4,   /* learned filter: capped sample sets (extraction gather) */
    SSVP_TRACE_INFER = 5,     /* learned filter: tensor-core inference */
    SSVP_TRACE_TRAIN = 6,     /* learned filter: forward and backward pass on a batch */
    SSVP_TRACE_ADAM = 7,      /* learned filter: Adam step */
    SSVP_TRACE_BATCH = 8,     /* one launch of a batched plan */
    SSVP_TRACE_LOAD = 9,      /* pack, median, depth ranges and gradient sums of a load or append */
    SSVP_TRACE_MASK = 10,     /* inpainting mask from a scene-space box */
    SSVP_TRACE_KINDS = 11
};
int ssvp_trace_enable(ssvp_ctx *ctx, int on);
int ssvp_trace_read(ssvp_ctx *ctx, int max_kinds, int *kind, int *launches, double *ms, int *n_kinds);
/* A short name of a trace kind ("gather", "infer", ...), or "" for an unknown kind. */
const char *ssvp_trace_kind_name(int kind);

/* Statistics of the last ssvp_gather_filter call (waits for it): examined candidates (window
 * pixels inside the image), accepted samples |S| summed over pixels, and the sum of weights W
 * (Sec. "Filtering" reports W / |S|).  Any pointer may be NULL. */
int ssvp_read_stats(ssvp_ctx *ctx, unsigned long long *examined, unsigned long long *accepted, double *sum_w);

/*
 * Batched plans (persistent launch of several clips, captured in a CUDA graph).
 * A plan fixes the parameters, the clip list and their cameras: it composes every per-(O, J)
 * transform once, numbers the work items (clip, output-frame chunk, 32 x tile_rows tile),
 * sizes a persistent grid from the kernel's occupancy, and captures "reset counters + launch"
 * as a CUDA graph that ssvp_plan_launch replays on the context's stream.  Denoise and mean
 * modes, full frames, no debug outputs; all clips must share one colour format.  After any of
 * its clips is reloaded or unloaded the plan's launch fails with SSVP_ENOCLIP until the plan is
 * updated (ssvp_plan_update, for reloads with the same shapes) or re-created; after
 * ssvp_set_cameras it must be updated or re-created too.
 */
typedef struct ssvp_plan ssvp_plan;
typedef struct ssvp_plan_config {
    int32_t tile_rows;    /* output rows per CTA: 4 or 8 */
    int32_t frame_chunk;  /* consecutive output frames per work item: 1 .. 16 */
} ssvp_plan_config;

/* Autotuner: times every (tile_rows, frame_chunk) candidate on a sample of the plan's work (the
 * first 8 output frames of every listed clip: tile_rows 4 or 8 x frame_chunk 1, 2, 4 or 8) and
 * keeps the fastest in the context for later plans with the same k, half window, mode and
 * colour format; *best (may be NULL) receives it. */
int ssvp_autotune(ssvp_ctx *ctx, const ssvp_params *params, const int *clip_ids, int n_clips, ssvp_plan_config *best);

/* Create a plan.  config NULL: the context's tuned shape for these parameters if any, else
 * tile_rows = 8, frame_chunk = 1.  Allocates device memory and synchronises the stream. */
int ssvp_plan_create(ssvp_ctx *ctx, const ssvp_params *params, const int *clip_ids, int n_clips,
                     const ssvp_plan_config *config, ssvp_plan **out);

/* Replay the plan's graph on the context's stream (asynchronous); statistics as for
 * ssvp_gather_filter. */
int ssvp_plan_launch(ssvp_plan *plan);

/* Refresh a plan for its clips' current contents and cameras, keeping its captured graph: valid
 * after reloads with the same W, H, F and colour format (which keep the clips' planes) and after
 * ssvp_set_cameras.  Recomposes every per-(O, J) transform from the current cameras into the
 * plan's table (a copy queued on the context's stream after the plan's earlier launches; does
 * not wait).  SSVP_ENOCLIP / SSVP_ENOCAM for a clip not loaded / without cameras, SSVP_EINVAL if a
 * clip's planes moved (another shape or format, or ssvp_append_frames): make a new plan. */
int ssvp_plan_update(ssvp_plan *plan);

/* Shape, number of work items and persistent grid size of a plan (any pointer may be NULL). */
int ssvp_plan_get_config(const ssvp_plan *plan, ssvp_plan_config *config, long long *n_items, int *grid);

/* Free a plan (waits for its launches).  NULL is a no-op.  Destroy plans before their context. */
void ssvp_plan_destroy(ssvp_plan *plan);

/*
 * Learned per-sample weights (SSVP_MODE_LEARNED).  Per output pixel the first n <= 64 gathered
 * samples in canonical order (frames O, O-1, O+1, ..., then window raster order) get 16 features
 * [colour (3), colour - reference (3), distance / r, (J - O) / T, depth residual in the sample's
 * frame / r, log of the Eq. 4 weight, 1, size of the whole gathered set / 64, colour - the plain
 * Eq. 4 result (3), 0] (BF16); a
 * 16 -> 64 -> 2 MLP (BF16 tensor cores,
 * FP32 accumulation) gives per-sample weights softplus(z_w) and a confidence mean sigmoid(z_c);
 * the output is the weighted mean of the samples' colours when the confidence is at least
 * params.conf_threshold, else the plain Eq. 3/4 result.
 */

/* Set the network (FP32 host arrays: W1 64x16 hidden x feature row-major, b1 64, W2 2x64, b2 2).
 * W1 and W2 are used rounded to BF16, b1 and b2 in FP32.  Resets the training state. */
int ssvp_set_mlp(ssvp_ctx *ctx, const float *W1, const float *b1, const float *W2, const float *b2);

/* Copy the current FP32 weights to the host (waits). */
int ssvp_get_mlp(ssvp_ctx *ctx, float *W1, float *b1, float *W2, float *b2);

/* Capped sample sets of one output frame's crop (params.frame_begin; crop_* as for gather) written
 * to caller device buffers: feat (crop pixels x 64 x 16 BF16 bits), col (x 64 x 3 floats), nsamp
 * (int32 per pixel) and plain (3 floats per pixel, the Eq. 3/4 result).  Slots beyond nsamp are
 * left as they were. */
int ssvp_learned_samples(ssvp_ctx *ctx, const ssvp_params *params, int clip_id, unsigned short *feat, float *col,
                         int32_t *nsamp, float *plain);

typedef struct ssvp_train_config {
    int32_t steps;         /* optimiser steps */
    int32_t batch_pixels;  /* pixels per step, drawn uniformly from one frame of one clip */
    float lr;              /* Adam learning rate */
    float bce_weight;      /* weight of the confidence BCE term */
    uint64_t seed;         /* frame/pixel draws and the He initialisation */
    int32_t init;          /* 1: He-initialise from seed first, 0: continue from the current weights */
    int32_t pad_;
} ssvp_train_config;

/*
 * Train the network on the GPU (forward, loss, backward on the tensor cores; Adam on FP32 master
 * weights).  Each step draws a clip and an output frame, extracts that frame's capped sample sets
 * with params (mode is ignored; the gather and the plain fallback use params' k, T, radius and
 * sigmas), draws batch_pixels pixels, and minimises mean (learned - clean)^2 + bce_weight *
 * BCE(confidence, [learned error <= plain error]).  clean[i] is a device pointer to clip i's
 * target frames (F x H x W x 3 floats).  loss_out (host, steps floats, may be NULL) receives the
 * per-step batch losses (waits).
 */
int ssvp_train(ssvp_ctx *ctx, const ssvp_params *params, const int *clip_ids, const float *const *clean, int n_clips,
               const ssvp_train_config *cfg, float *loss_out);

/* Loss and gradient at the current weights over listed pixels (crop-of-full-frame indices
 * y * W + x) of output frame params.frame_begin of a clip; grad_out (host) receives the flat
 * gradient W1 | b1 | W2 | b2 followed by the loss (1219 floats).  Waits. */
int ssvp_mlp_grad(ssvp_ctx *ctx, const ssvp_params *params, int clip_id, const int32_t *pixels, int n_pixels,
                  const float *clean, float *grad_out);

/* Lower-median valid input depth of a loaded clip (waits for the load). */
int ssvp_clip_median_depth(ssvp_ctx *ctx, int clip_id, float *median);

/* Wait for all work queued on the context's stream; returns the first pending error, or
 * SSVP_ETIMEOUT when a kernel's bounded device-side wait gave up since the last call: the learned
 * inference waits for its tensor-core products on an MMA-completion barrier with a limit of about
 * 1 s (the outputs of that launch are then not valid); the staged window gather
 * (SSVP_GATHER_WINDOW_TMA) waits for its tensor copies with the same limit (a warp whose wait gave
 * up tests the rest of its frames from the global planes, so its outputs stay valid).  The
 * time-out is reported once. */
int ssvp_sync(ssvp_ctx *ctx);

/*
 * Lower-median valid depth of a caller-owned device array, without allocating any memory.
 *
 * The paper has no counterpart: this is a service for callers that may not allocate device
 * memory themselves or through this library -- for example a plug-in inside a video host that
 * owns every GPU buffer through its own pool, or a per-frame real-time callback, where a
 * cudaMalloc/cudaFree would synchronise the device and stall the host's pipeline.  It computes
 * the same value as ssvp_clip_median_depth (the element of rank floor((m-1)/2) among the m
 * finite, positive values) with the same radix-select kernels, but keeps their scratch (8,208
 * bytes of histogram and bookkeeping) in a fixed array in the library's device memory, which
 * every GPU that loads the library holds until the process exits.  No context is needed.
 *
 *   depth_dev   n floats in device (or managed) memory of the current CUDA device (any layout;
 *               invalid values are ignored); a host address returns SSVP_EINVAL
 *   n           1 <= n <= 4294967295 (the scratch counts in 32-bit words); other sizes return
 *               SSVP_EINVAL with a message in ssvp_last_error(NULL)
 *   median_dev  one float in device (or managed) memory: the median, or NaN when no value is
 *               valid; a host address returns SSVP_EINVAL
 *   cuda_stream stream to queue the work on (NULL: legacy default stream); asynchronous
 *
 * The first call on a device looks up the scratch array's device address for that device (the
 * device must be current); make that first call before any stream capture.  The address is kept
 * for the life of the process, so the library must not be used on a device after a
 * cudaDeviceReset of it.  All calls share the one array: each call clears it before use, and
 * calls whose work overlaps on the GPU (for example on two streams at once) race on it and give
 * wrong results.
 */
int ssvp_median_depth_noalloc(const float *depth_dev, unsigned long long n, float *median_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SSVP_H */
