// ssvp_internal.h - device data layout shared by the host runtime (ssvp_api.cpp) and the CUDA
// kernels (ssvp_gather.cu, ssvp_pack.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ssvp {

// Every packed plane has kPad pixels of padding on each side.  A k x k window whose centre is
// within h pixels of the image reaches at most 2h <= 30 pixels beyond it, so window loads never
// leave the allocation and need no bounds test: padding depth is NaN, which fails the radius test.
constexpr int kPad = 32;
constexpr int kMaxSlots = 2 * 127 + 1;

// One loaded clip on the device.
struct Planes {
    int W, H, F;
    int pitch;             // elements per padded row, multiple of 32 (128-byte rows for depth)
    int rows;              // H + 2 * kPad
    long long fstride;     // pitch * rows: elements per frame
    float *depth;          // F * fstride floats; pixel (x, y) at (y + kPad) * pitch + x + kPad
    void *colour;          // F * fstride texels: float4 (r, g, b, 0) or 4 x half (r, g, b, 0)
    int colour_fmt;        // 0 FP32, 1 FP16
    float *median;         // device scalar: lower-median valid depth
    unsigned int *zrange;  // F x 2 words: valid depth range of each frame as bit patterns,
                           // complement of the minimum's bits and the maximum's bits (0: none)
    double *grad_sum;      // F: Eq. 5 blurriness measure (sum of gradient magnitudes) per frame
    float *grad_log2;      // F: log2(grad_sum / max over frames), the Eq. 5 factor in log2 units
    double *grad_partial;  // F x grad_partial_words(1): partial sums of grad_sum
    unsigned char *mask;   // inpainting mask (Eq. 8-9), same indexing as depth, pads 0; null until set
    float *out;            // F * H * W * 3 output floats (row-major, interleaved)
};

// Host-composed geometry of one (output frame O, window slot j) pair, J = O - T + j.
// M = K_J R_JO K_O^-1 and e = K_J t_JO map (u d, v d, d) of O to homogeneous pixel coordinates
// of J; they are stored as unevaluated FP32 pairs (hi + lo) of their FP64 values.
struct __align__(16) PairGeom {
    float M_hi[9], M_lo[9];
    float e_hi[3], e_lo[3];
    float ifx, ify, cx, cy;   // intrinsics of J (zero skew): 1/fx, 1/fy, cx, cy
    float beta;               // (J - O)^2 / (2 sigma_f^2)
    int32_t J;                // input frame, or -1 when outside the clip
    int32_t same;             // J == O
    int32_t pad_;
};
static_assert(sizeof(PairGeom) == 128, "PairGeom layout");

// Capped sample sets of the learned filter, per crop pixel up to 64 samples in canonical order,
// stored compactly; the MLP kernels rebuild the 16 BF16 features of a sample from them:
// [colour (3), colour - c_ref (3), dist / r, (J - O) / T, depth residual / r, log w, 1,
//  |S(p)| / 64, colour - plain (3), 0].
struct SampleSets {
    float4 *col;     // pixel x 64: FP32 colour (x, y, z); w holds the BF16 pair (dist / r, (J - O) / T)
    unsigned *f89;   // pixel x 64: the BF16 pair (depth residual / r, log w)
    float4 *info;    // pixel: c_ref (x, y, z) and |S(p)| / 64
    int32_t *n;      // pixel: samples kept (<= 64)
    float *plain;    // pixel x 3: the plain Eq. 3/4 result over the whole set
};

// Arguments of one gather launch (one clip, a range of output frames).
struct GatherArgs {
    Planes clip;
    const PairGeom *geom;     // n_out * n_slots entries
    int frame_begin, n_out, n_slots, T;
    int x0, y0, cw, ch;       // output crop
    int k, mode;
    float radius;             // > 0 absolute, < 0 relative to *clip.median
    float sigma_rgb, sigma_xyz, sigma_f;  // sigma_xyz <= 0: equal to the radius
    // virtual aperture (mode 1)
    float aperture;           // A, lens radius
    float focal_depth;        // z0; <= 0: *clip.median
    float a0;                 // cone waist; <= 0: 0.5 z0 / fx_O
    int lens_n;               // seed points
    int cap;                  // box cap per axis (odd)
    float lens_xy[128];       // seed lens points (x, y) on the unit-radius disc, scaled by A in the kernel
    // learned filter: the capped sample sets of the crop (set when extracting them)
    SampleSets sets;
    // per-frame weights in log2 units, subtracted from the exponent of every sample from J:
    // frame_log2w[J] (Eq. 5, indexed by input frame) and slot_log2w[j] (Eq. 10, by window slot)
    const float *frame_log2w;
    const float *slot_log2w;
    // frustum gather (Eq. 1-2): back maps G_{O<-J} (same indexing as geom), frustum size and depths
    const PairGeom *geom_back;
    float frustum_l, near_plane, far_plane;
    // super-resolution (Eq. 6-7): output grid scale, Eq. 7's sigma_area (<= 0: median / fx_O) and
    // the caller's output, n_out x (H scale) x (W scale) x 3 floats; null for the other gathers
    int sr_scale;
    float sigma_area;
    float *sr_out;
    int32_t *membership;      // debug record per (crop pixel, slot) or null
    int32_t *pixel_stats;     // debug record per crop pixel or null
    unsigned long long *stat_counts;  // [0] examined, [1] accepted
    double *stat_sumw;
    // window gather: 1 stages the candidate depths into shared memory by tensor copies (k <= 7);
    // 2 as 1 but issues no copies, so that the waits run out (a test of the time-out path)
    int stage;
    int *err;                 // error word: bit 1 set when a staging wait timed out
};

// One clip of a batched launch (A10).  Work items are (clip, output-frame chunk, tile) triples
// numbered from item_begin; tiles are 32 x tile_rows output pixels.
struct BatchClip {
    Planes p;
    const PairGeom *geom;     // n_out * n_slots entries
    int frame_begin, n_out, tiles_x, tiles_y;
    long long item_begin;
};

constexpr int kMaxBatchClips = 64;  // SSVP_MAX_CLIPS

struct BatchArgs {
    int n_clips, frame_chunk;
    long long n_items;
    unsigned long long *counter;  // work counter, zero before the launch
    // the clip table itself travels in the kernel's parameter space: read-only constant-bank data
    // that the compiler may reload at will instead of holding it in registers
    BatchClip clip[kMaxBatchClips];
};

// ---------------------------------------------------------------- learned per-sample weights
// Flat parameter vector: W1 (64 x 16, hidden x feature) | b1 (64) | W2 (2 x 64) | b2 (2).
constexpr int kMlpParams = 64 * 16 + 64 + 2 * 64 + 2;
constexpr int kMlpB1 = 64 * 16, kMlpW2 = kMlpB1 + 64, kMlpB2 = kMlpW2 + 128;

struct MlpWeights {           // what the tensor-core kernels read
    const unsigned short *W1; // BF16 bits
    const float *b1;          // FP32
    const float *W2;          // FP32 holding BF16-rounded values
    const float *b2;          // FP32
};

struct MlpState {             // training state on the device
    float *master, *m, *v;    // kMlpParams each
    float *grad;              // kMlpParams + 1 (the batch loss last)
    unsigned short *W1_bf16;  // 1024
    float *W2_r;              // 128
};

struct MlpArgs {
    MlpWeights w;
    SampleSets sets;              // the crop's capped sample sets (read only)
    long long n_px;               // crop pixels
    int O, W, H, x0, y0, cw;      // output frame and crop (pixel px = (x0 + px % cw, y0 + px / cw))
    float tau;                    // confidence threshold
    float *out;                   // clip output buffer (inference)
    float *conf_out;              // optional per crop pixel confidence
    const int32_t *batch;         // training: crop pixel indices
    long long n_batch;
    const float *clean;           // training: target frames (F x H x W x 3, FP32)
    float bce_w;
    float *grad;                  // training: kMlpParams + 1 accumulators
    int skip_mma;                 // inference: issue no tensor-core products (test of the time-out path)
};

// learned inference on the tcgen05 tensor cores; err (device word) is raised if one of its bounded
// waits for MMA completion times out
cudaError_t launch_mlp_infer_tc(const MlpArgs &m, int *err, cudaStream_t s);
// training on the tcgen05 tensor cores (forward, loss, backward; gradients accumulated into
// m.grad); err as for the inference
cudaError_t launch_mlp_train_tc(const MlpArgs &m, int *err, cudaStream_t s);
cudaError_t launch_adam(const MlpState &st, float lr, int step, cudaStream_t s);
cudaError_t launch_mlp_refresh(const MlpState &st, cudaStream_t s);
// expand compact sample sets into 64 x 16 BF16 features, 64 x 3 colours, counts and plain results
cudaError_t launch_expand_sets(const SampleSets &sets, unsigned short *feat, float *col, int32_t *nsamp, float *plain,
                               long long n_px, cudaStream_t s);

cudaError_t launch_pack(const float *rgb, const float *depth, int W, int H, int nF, const Planes &dst, int frame0,
                        cudaStream_t s);
cudaError_t launch_median(const Planes &p, unsigned int *scratch, cudaStream_t s);
size_t median_scratch_words();
cudaError_t launch_gather(const GatherArgs &a, cudaStream_t s);
cudaError_t launch_aperture(const GatherArgs &a, cudaStream_t s);
cudaError_t launch_frustum(const GatherArgs &a, cudaStream_t s);
cudaError_t launch_grad_sum(const Planes &p, cudaStream_t s);
cudaError_t launch_mask_box(const Planes &p, const double *cam, const double *box, cudaStream_t s);
size_t grad_partial_words(int F);
cudaError_t launch_zrange(const Planes &p, cudaStream_t s);
// persistent batched gather; grid = batch_grid(...) CTAs
cudaError_t launch_batch(const GatherArgs &a, const BatchArgs &b, int tile_rows, int colour_fmt, int grid,
                         cudaStream_t s);
int batch_grid(int k, int tile_rows, int colour_fmt, int n_slots);

// largest input of ssvp_median_depth_noalloc: its fixed scratch counts values in 32-bit words
constexpr unsigned long long kMedianNoallocMax = 0xffffffffull;
// error text for entry points that have no context (read with ssvp_last_error(NULL))
void set_global_error(const char *fmt, ...);

}  // namespace ssvp
