// ssvp_api.cpp - host runtime behind the C ABI of include/ssvp.h: context and device buffers,
// input upload and packing, FP64 camera composition (step A1), argument checks, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ssvp.h"
#include "ssvp_internal.h"

using ssvp::GatherArgs;
using ssvp::PairGeom;
using ssvp::Planes;

namespace {

struct Clip {
    bool loaded = false;
    bool has_cams = false;
    unsigned generation = 0;  // bumped on every load and unload
    Planes p{};
    std::vector<double> K;    // F * 9
    std::vector<double> w2c;  // F * 12
    // ssvp_append_frames: the spare window (depth and colour planes and the per-window values:
    // median, depth ranges, gradient sums) the next window is built in while queued gathers still
    // read the current one, and the event recorded on the context's stream by the previous
    // append: every read of the spare window precedes it
    Planes spare{};
    cudaEvent_t ev_append = nullptr;
    // per-frame values of the current window that only some calls need, computed on first use:
    // the valid depth range of each frame (the frustum gathers) and the Eq. 5 gradient sums
    bool zrange_ready = false, grad_ready = false;
    // output frames [out_lo, out_hi) may hold values written since the buffer was last cleared
    // (a reload with the same shape clears only these)
    int out_lo = 0, out_hi = 0;
    void mark_out(int b, int e) {
        if (e <= b) return;
        if (out_hi <= out_lo) {
            out_lo = b;
            out_hi = e;
        } else {
            out_lo = std::min(out_lo, b);
            out_hi = std::max(out_hi, e);
        }
    }
};

// the arrays of one window of a clip (the rest of Planes, such as the output and the mask, is shared)
void swap_window(Planes &a, Planes &b) {
    std::swap(a.depth, b.depth);
    std::swap(a.colour, b.colour);
    std::swap(a.median, b.median);
    std::swap(a.zrange, b.zrange);
    std::swap(a.grad_sum, b.grad_sum);
    std::swap(a.grad_log2, b.grad_log2);
    std::swap(a.grad_partial, b.grad_partial);
}

char g_create_error[512] = "";

}  // namespace

struct ssvp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    Clip clips[SSVP_MAX_CLIPS];
    char err[512] = "";
    // device scratch
    unsigned long long *stat_counts = nullptr;  // [2]
    double *stat_sumw = nullptr;
    unsigned int *median_scratch = nullptr;
    int *d_kerr = nullptr;  // set by a kernel whose bounded device-side wait gave up; read by ssvp_sync
    PairGeom *geom = nullptr;
    size_t geom_cap = 0;  // entries
    void *staging = nullptr;
    size_t staging_bytes = 0;
    // Loads run on an internal stream of the device's highest priority, ordered after the work
    // already queued on the context's stream and before everything queued after the load: their
    // short kernels (pack, median, depth ranges, gradient sums) then start as soon as SMs free up,
    // instead of queueing behind a long gather launched on another stream
    cudaStream_t load_stream = nullptr;
    cudaEvent_t ev_load_in = nullptr, ev_load_out = nullptr;
    std::vector<PairGeom> host_geom;
    unsigned clip_generation[SSVP_MAX_CLIPS] = {};
    // learned filter: weights and training state, scratch of one frame's capped sample sets
    ssvp::MlpState mlp{};
    float *mlp_buf = nullptr;        // master | m | v | grad (+ loss) | W2_r
    unsigned short *mlp_w1 = nullptr;
    bool mlp_set = false;
    int mlp_step = 0;
    ssvp::SampleSets l_sets{};  // compact capped sample sets of one frame's crop
    float *l_loss = nullptr;
    int32_t *l_batch = nullptr;
    size_t l_cap = 0, l_batch_cap = 0, l_loss_cap = 0;
    // tuned batch shapes: key (k, half window, mode, colour format) -> config
    struct Tuned {
        int k, T, mode, cfmt;
        ssvp_plan_config cfg;
    };
    std::vector<Tuned> tuned;
    // Eq. 10 shutter function (host copy) and its per-slot log2 weights on the device
    std::vector<float> shutter;
    float *d_shutter_log2 = nullptr;
    // kernel timing (ssvp_trace_enable): the event pairs of traced launches, and spare events
    struct TraceRec {
        int kind;
        cudaEvent_t a, b;
    };
    bool trace_on = false;
    std::vector<TraceRec> trace_pending;
    std::vector<cudaEvent_t> trace_free;
    // ssvp_mask_from_box: the per-frame cameras (K^-1, R, t; 21 doubles a frame) on the device
    double *mask_cam = nullptr;
    size_t mask_cam_cap = 0;  // doubles
};

struct ssvp_plan {
    ssvp_ctx *ctx = nullptr;
    ssvp_params params{};
    std::vector<int> clip_ids;
    std::vector<unsigned> generations;
    // what the captured graph holds of each clip: its plane pointers and the shape they have
    struct Frozen {
        const void *depth, *colour, *out, *median;
        int W, H, F, fmt;
        bool operator==(const Frozen &o) const {
            return depth == o.depth && colour == o.colour && out == o.out && median == o.median && W == o.W &&
                   H == o.H && F == o.F && fmt == o.fmt;
        }
    };
    static Frozen frozen(const Planes &p) {
        return Frozen{p.depth, p.colour, p.out, p.median, p.W, p.H, p.F, p.colour_fmt};
    }
    std::vector<Frozen> planes;
    ssvp_plan_config cfg{8, 1};
    long long n_items = 0;
    int grid = 0;
    PairGeom *d_geom = nullptr;
    unsigned long long *d_counter = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int fail(ssvp_ctx *c, int code, const char *fmt, ...) {
    char *dst = c ? c->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(ssvp_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(c, SSVP_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(c, SSVP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Where a caller's buffer really lives, before any work touches it.  A buffer given as device memory
// must be device memory of the context's device (or managed memory): a kernel handed a host address
// faults, or, where the GPU can reach host memory, reads and writes the wrong memory.  A buffer
// given as host memory must not be device memory: the copy would name the wrong direction, and a
// host loop reading it would crash.
int check_mem(ssvp_ctx *ctx, const void *ptr, int mem_kind, const char *what) {
    cudaPointerAttributes at{};
    const cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SSVP_EINVAL, "%s: not an address CUDA can classify (%s)", what, cudaGetErrorString(e));
    }
    if (mem_kind == SSVP_MEM_DEVICE) {
        if (at.type == cudaMemoryTypeManaged) return SSVP_OK;
        if (at.type != cudaMemoryTypeDevice) return fail(ctx, SSVP_EINVAL, "%s is not device memory", what);
        if (at.device != ctx->device)
            return fail(ctx, SSVP_EINVAL, "%s is memory of device %d, not of the context's device %d", what, at.device,
                        ctx->device);
    } else if (at.type == cudaMemoryTypeDevice) {
        return fail(ctx, SSVP_EINVAL, "%s is device memory but was given as host memory", what);
    }
    return SSVP_OK;
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

cudaEvent_t trace_event(ssvp_ctx *ctx) {
    if (!ctx->trace_free.empty()) {
        cudaEvent_t e = ctx->trace_free.back();
        ctx->trace_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// While tracing is on, brackets the work queued on stream s during its lifetime with a pair of
// timing events, recorded under `kind` (never used on a capturing stream)
struct TraceScope {
    ssvp_ctx *ctx;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    TraceScope(ssvp_ctx *c, int k, cudaStream_t st) : ctx(c), kind(k), s(st) {
        if (!c->trace_on || !(a = trace_event(c))) return;
        if (cudaEventRecord(a, s) != cudaSuccess) {
            cudaGetLastError();
            c->trace_free.push_back(a);
            a = nullptr;
        }
    }
    ~TraceScope() {
        if (!a) return;
        cudaEvent_t b = trace_event(ctx);
        if (b && cudaEventRecord(b, s) == cudaSuccess) {
            ctx->trace_pending.push_back({kind, a, b});
            return;
        }
        cudaGetLastError();
        ctx->trace_free.push_back(a);
        if (b) ctx->trace_free.push_back(b);
    }
    TraceScope(const TraceScope &) = delete;
    TraceScope &operator=(const TraceScope &) = delete;
};

// The per-frame values some calls need, the first time a call needs them for this window: like
// the load's kernels, on the load stream of the device's highest priority (so that they start
// as soon as SMs free up instead of queueing behind another context's gather), after the work
// queued on the context's stream and before the work queued after them
int ensure_frame_values(ssvp_ctx *ctx, Clip &c, bool zrange, bool grad) {
    zrange = zrange && !c.zrange_ready;
    grad = grad && !c.grad_ready;
    if (!zrange && !grad) return SSVP_OK;
    cudaStream_t ls = ctx->load_stream;
    CK(cudaEventRecord(ctx->ev_load_in, ctx->stream), "cudaEventRecord");
    CK(cudaStreamWaitEvent(ls, ctx->ev_load_in, 0), "cudaStreamWaitEvent");
    {
        TraceScope ts(ctx, SSVP_TRACE_LOAD, ls);
        if (zrange) {
            CK(ssvp::launch_zrange(c.p, ls), "depth range kernel");
            c.zrange_ready = true;
        }
        if (grad) {
            CK(ssvp::launch_grad_sum(c.p, ls), "gradient sum kernels");
            c.grad_ready = true;
        }
    }
    CK(cudaEventRecord(ctx->ev_load_out, ls), "cudaEventRecord");
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_load_out, 0), "cudaStreamWaitEvent");
    return SSVP_OK;
}

void free_clip(Clip &c) {
    if (c.p.depth) cudaFree(c.p.depth);
    if (c.p.colour) cudaFree(c.p.colour);
    if (c.p.out) cudaFree(c.p.out);
    if (c.p.median) cudaFree(c.p.median);
    if (c.p.zrange) cudaFree(c.p.zrange);
    if (c.p.grad_sum) cudaFree(c.p.grad_sum);
    if (c.p.grad_log2) cudaFree(c.p.grad_log2);
    if (c.p.grad_partial) cudaFree(c.p.grad_partial);
    if (c.p.mask) cudaFree(c.p.mask);
    for (void *q : {(void *)c.spare.depth, (void *)c.spare.colour, (void *)c.spare.median, (void *)c.spare.zrange,
                    (void *)c.spare.grad_sum, (void *)c.spare.grad_log2, (void *)c.spare.grad_partial})
        if (q) cudaFree(q);
    if (c.ev_append) cudaEventDestroy(c.ev_append);
    c = Clip();
}

bool finite_all(const double *v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// ---------------------------------------------------------------- A1: camera composition (FP64)

void split(double x, float &hi, float &lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

void mat3_mul(const double *A, const double *B, double *C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// M = K_J R_JO K_O^-1, e = K_J t_JO with R_JO = R_J R_O^T, t_JO = t_J - R_JO t_O: maps
// d (u, v, 1) of frame O to homogeneous pixel coordinates of frame J (C_J C_O^-1 of Eq. 2).
void compose_pair(const double *KO, const double *wO, const double *KJ, const double *wJ, bool same, int dJ,
                  double sigma_f, PairGeom &g) {
    double M[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, e[3] = {0, 0, 0};
    if (!same) {
        double RO[9], RJ[9], tO[3], tJ[3];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) { RO[3 * i + j] = wO[4 * i + j]; RJ[3 * i + j] = wJ[4 * i + j]; }
            tO[i] = wO[4 * i + 3];
            tJ[i] = wJ[4 * i + 3];
        }
        double RJO[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                RJO[3 * i + j] = RJ[3 * i] * RO[3 * j] + RJ[3 * i + 1] * RO[3 * j + 1] + RJ[3 * i + 2] * RO[3 * j + 2];
        double tJO[3];
        for (int i = 0; i < 3; ++i) tJO[i] = tJ[i] - (RJO[3 * i] * tO[0] + RJO[3 * i + 1] * tO[1] + RJO[3 * i + 2] * tO[2]);
        // K_O^-1 of an upper-triangular, zero-skew K
        const double KOi[9] = {1.0 / KO[0], 0.0, -KO[2] / KO[0], 0.0, 1.0 / KO[4], -KO[5] / KO[4], 0.0, 0.0, 1.0};
        double T[9];
        mat3_mul(KJ, RJO, T);
        mat3_mul(T, KOi, M);
        for (int i = 0; i < 3; ++i) e[i] = KJ[3 * i] * tJO[0] + KJ[3 * i + 1] * tJO[1] + KJ[3 * i + 2] * tJO[2];
    }
    for (int i = 0; i < 9; ++i) split(M[i], g.M_hi[i], g.M_lo[i]);
    for (int i = 0; i < 3; ++i) split(e[i], g.e_hi[i], g.e_lo[i]);
    g.ifx = (float)(1.0 / KJ[0]);
    g.ify = (float)(1.0 / KJ[4]);
    g.cx = (float)KJ[2];
    g.cy = (float)KJ[5];
    g.beta = (float)((double)dJ * dJ / (2.0 * sigma_f * sigma_f));
    g.same = same ? 1 : 0;
    g.pad_ = 0;
}

// A1 for output frames [fb, fb + n_out) of a clip: n_out * (2T + 1) entries, slot j <-> J = O - T + j.
void compose_table(const Clip &c, int fb, int n_out, int T, double sigma_f, PairGeom *out) {
    const int ns = 2 * T + 1;
    for (int oi = 0; oi < n_out; ++oi) {
        const int O = fb + oi;
        for (int j = 0; j < ns; ++j) {
            const int J = O - T + j;
            PairGeom &g = out[(size_t)oi * ns + j];
            if (J < 0 || J >= c.p.F) {
                std::memset(&g, 0, sizeof(g));
                g.J = -1;
                continue;
            }
            compose_pair(&c.K[9 * (size_t)O], &c.w2c[12 * (size_t)O], &c.K[9 * (size_t)J], &c.w2c[12 * (size_t)J],
                         J == O, J - O, sigma_f, g);
            g.J = J;
        }
    }
}

// Back maps of the frustum gather: G_{O<-J} for every (O, slot), composed like the forward maps
// with the roles of O and J exchanged (M = K_O R_OJ K_J^-1, e = K_O t_OJ; intrinsics of O).
void compose_table_back(const Clip &c, int fb, int n_out, int T, double sigma_f, PairGeom *out) {
    const int ns = 2 * T + 1;
    for (int oi = 0; oi < n_out; ++oi) {
        const int O = fb + oi;
        for (int j = 0; j < ns; ++j) {
            const int J = O - T + j;
            PairGeom &g = out[(size_t)oi * ns + j];
            if (J < 0 || J >= c.p.F) {
                std::memset(&g, 0, sizeof(g));
                g.J = -1;
                continue;
            }
            compose_pair(&c.K[9 * (size_t)J], &c.w2c[12 * (size_t)J], &c.K[9 * (size_t)O], &c.w2c[12 * (size_t)O],
                         J == O, J - O, sigma_f, g);
            g.J = J;
        }
    }
}

// Super-resolution (Eq. 6-7): forward and back maps of every (O, slot) with the output-grid
// camera of O (fx, fy scaled, principal point c -> scale (c + 0.5) - 0.5) in place of K_O.
void compose_tables_sr(const Clip &c, int fb, int n_out, int T, double sigma_f, int scale, PairGeom *fwd,
                       PairGeom *back) {
    const int ns = 2 * T + 1;
    for (int oi = 0; oi < n_out; ++oi) {
        const int O = fb + oi;
        double Ks[9];
        std::memcpy(Ks, &c.K[9 * (size_t)O], sizeof(Ks));
        Ks[0] *= scale;
        Ks[2] = scale * (Ks[2] + 0.5) - 0.5;
        Ks[4] *= scale;
        Ks[5] = scale * (Ks[5] + 0.5) - 0.5;
        for (int j = 0; j < ns; ++j) {
            const int J = O - T + j;
            PairGeom &g = fwd[(size_t)oi * ns + j], &h = back[(size_t)oi * ns + j];
            if (J < 0 || J >= c.p.F) {
                std::memset(&g, 0, sizeof(g));
                std::memset(&h, 0, sizeof(h));
                g.J = h.J = -1;
                continue;
            }
            // the two cameras of O differ unless scale = 1, so J = O is exact only then
            const bool same = J == O && scale == 1;
            compose_pair(Ks, &c.w2c[12 * (size_t)O], &c.K[9 * (size_t)J], &c.w2c[12 * (size_t)J], same, J - O, sigma_f, g);
            compose_pair(&c.K[9 * (size_t)J], &c.w2c[12 * (size_t)J], Ks, &c.w2c[12 * (size_t)O], same, J - O, sigma_f, h);
            g.J = h.J = J;
        }
    }
}

int check_params(ssvp_ctx *ctx, const ssvp_params *p) {
    if (!p) return fail(ctx, SSVP_EINVAL, "params is NULL");
    if (p->mode != SSVP_MODE_DENOISE && p->mode != SSVP_MODE_MEAN && p->mode != SSVP_MODE_APERTURE &&
        p->mode != SSVP_MODE_LEARNED && p->mode != SSVP_MODE_DEBLUR && p->mode != SSVP_MODE_SHUTTER &&
        p->mode != SSVP_MODE_INPAINT && p->mode != SSVP_MODE_SEMI)
        return fail(ctx, SSVP_EINVAL, "mode %d is not available in this build", p->mode);
    if (p->mode == SSVP_MODE_LEARNED && !(std::isfinite(p->conf_threshold)))
        return fail(ctx, SSVP_EINVAL, "conf_threshold must be finite");
    if (p->mode == SSVP_MODE_APERTURE) {
        if (p->cap < 1 || p->cap > 63 || (p->cap & 1) == 0) return fail(ctx, SSVP_EINVAL, "cap=%d must be odd in [1, 63]", p->cap);
        if (p->lens_samples < 1 || p->lens_samples > 64)
            return fail(ctx, SSVP_EINVAL, "lens_samples=%d must be in [1, 64]", p->lens_samples);
        if (!(p->aperture >= 0.0f && std::isfinite(p->aperture))) return fail(ctx, SSVP_EINVAL, "aperture must be >= 0");
        if (!std::isfinite(p->focal_depth) || !std::isfinite(p->a0))
            return fail(ctx, SSVP_EINVAL, "focal_depth and a0 must be finite");
    }
    if (p->gather != SSVP_GATHER_WINDOW && p->gather != SSVP_GATHER_FRUSTUM && p->gather != SSVP_GATHER_WINDOW_TMA)
        return fail(ctx, SSVP_EINVAL, "gather %d is not available in this build", p->gather);
    if (p->gather == SSVP_GATHER_WINDOW_TMA &&
        (p->mode == SSVP_MODE_APERTURE || p->mode == SSVP_MODE_LEARNED || p->k > 7))
        return fail(ctx, SSVP_EINVAL, "the staged window gather supports the denoise, mean, deblur and shutter modes "
                                      "with k <= 7");
    if (p->gather == SSVP_GATHER_WINDOW_TMA && p->test_skip_mma != 0 && p->test_skip_mma != 1)
        return fail(ctx, SSVP_EINVAL, "test_skip_mma must be 0 or 1");
    if ((p->mode == SSVP_MODE_INPAINT || p->mode == SSVP_MODE_SEMI) && p->gather != SSVP_GATHER_FRUSTUM)
        return fail(ctx, SSVP_EINVAL, "inpainting gathers the pixel frustum: set gather = SSVP_GATHER_FRUSTUM");
    if (p->gather == SSVP_GATHER_FRUSTUM) {
        if (p->mode == SSVP_MODE_APERTURE || p->mode == SSVP_MODE_LEARNED)
            return fail(ctx, SSVP_EINVAL, "the frustum gather supports the denoise, mean, deblur and shutter modes");
        if (!(p->frustum_l > 0.0f && p->frustum_l <= 64.0f)) return fail(ctx, SSVP_EINVAL, "frustum_l must be in (0, 64]");
        if (!(p->near_plane > 0.0f && p->far_plane > p->near_plane && std::isfinite(p->far_plane)))
            return fail(ctx, SSVP_EINVAL, "need 0 < near_plane < far_plane < inf");
    }
    if (p->k < 1 || p->k > SSVP_MAX_K || (p->k & 1) == 0) return fail(ctx, SSVP_EINVAL, "k=%d must be odd in [1, 31]", p->k);
    if (p->half_window < 0 || p->half_window > SSVP_MAX_HALF_WINDOW)
        return fail(ctx, SSVP_EINVAL, "half_window=%d must be in [0, 127]", p->half_window);
    if (!(std::isfinite(p->radius) && p->radius != 0.0f)) return fail(ctx, SSVP_EINVAL, "radius must be finite and non-zero");
    if (!(p->sigma_rgb > 0.0f && std::isfinite(p->sigma_rgb))) return fail(ctx, SSVP_EINVAL, "sigma_rgb must be > 0");
    if (!(p->sigma_f > 0.0f && std::isfinite(p->sigma_f))) return fail(ctx, SSVP_EINVAL, "sigma_f must be > 0");
    if (!std::isfinite(p->sigma_xyz)) return fail(ctx, SSVP_EINVAL, "sigma_xyz must be finite");
    if (p->crop_w < 0 || p->crop_h < 0) return fail(ctx, SSVP_EINVAL, "negative crop size");
    int rc;
    if (p->membership_out && (rc = check_mem(ctx, p->membership_out, SSVP_MEM_DEVICE, "membership_out")) != SSVP_OK)
        return rc;
    if (p->pixel_stats_out && (rc = check_mem(ctx, p->pixel_stats_out, SSVP_MEM_DEVICE, "pixel_stats_out")) != SSVP_OK)
        return rc;
    return SSVP_OK;
}


// ---------------------------------------------------------------- batched plans (A10)

struct BatchSetup {
    std::vector<ssvp::BatchClip> clips;
    std::vector<PairGeom> geom;
    std::vector<size_t> geom_off;
    long long n_items = 0;
    int cfmt = 0, ns = 0;
};

int batch_check(ssvp_ctx *ctx, const ssvp_params *p, const int *ids, int n, int &cfmt) {
    int rc = check_params(ctx, p);
    if (rc != SSVP_OK) return rc;
    if (p->mode != SSVP_MODE_DENOISE && p->mode != SSVP_MODE_MEAN)
        return fail(ctx, SSVP_EINVAL, "batched plans support the denoise and mean modes");
    if (p->crop_w != 0 || p->crop_h != 0) return fail(ctx, SSVP_EINVAL, "batched plans gather full frames (crop_w = crop_h = 0)");
    if (p->membership_out || p->pixel_stats_out) return fail(ctx, SSVP_EINVAL, "batched plans have no debug outputs");
    if (p->gather != SSVP_GATHER_WINDOW) return fail(ctx, SSVP_EINVAL, "batched plans use the window gather");
    if (!ids || n < 1 || n > SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "bad clip list");
    for (int i = 0; i < n; ++i) {
        if (ids[i] < 0 || ids[i] >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", ids[i]);
        const Clip &c = ctx->clips[ids[i]];
        if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", ids[i]);
        if (!c.has_cams) return fail(ctx, SSVP_ENOCAM, "clip %d has no cameras", ids[i]);
        if (i == 0) cfmt = c.p.colour_fmt;
        else if (c.p.colour_fmt != cfmt) return fail(ctx, SSVP_EINVAL, "all clips of a plan must share one colour format");
        int b = p->frame_begin, e = p->frame_end < 0 ? c.p.F : p->frame_end;
        if (b < 0 || e > c.p.F || b > e) return fail(ctx, SSVP_EINVAL, "frame range [%d, %d) outside clip %d (F=%d)", b, e, ids[i], c.p.F);
    }
    return SSVP_OK;
}

// host tables of every clip, output frames [fb, fb + min(n_out, max_out))
void batch_tables(ssvp_ctx *ctx, const ssvp_params &p, const int *ids, int n, int max_out, BatchSetup &bs) {
    const int T = p.half_window;
    bs.ns = 2 * T + 1;
    bs.clips.assign(n, ssvp::BatchClip{});
    bs.geom_off.assign(n, 0);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        const Clip &c = ctx->clips[ids[i]];
        const int b = p.frame_begin, e = p.frame_end < 0 ? c.p.F : p.frame_end;
        ssvp::BatchClip &bc = bs.clips[i];
        bc.p = c.p;
        bc.frame_begin = b;
        bc.n_out = std::min(e - b, max_out);
        bs.geom_off[i] = total;
        total += (size_t)bc.n_out * bs.ns;
    }
    bs.geom.resize(std::max<size_t>(total, 1));
    for (int i = 0; i < n; ++i)
        compose_table(ctx->clips[ids[i]], bs.clips[i].frame_begin, bs.clips[i].n_out, T, p.sigma_f, &bs.geom[bs.geom_off[i]]);
}

// number the work items for a shape; geometry pointers into d_geom
void batch_items(BatchSetup &bs, const ssvp_plan_config &cfg, PairGeom *d_geom) {
    long long item = 0;
    for (size_t i = 0; i < bs.clips.size(); ++i) {
        ssvp::BatchClip &bc = bs.clips[i];
        bc.geom = d_geom + bs.geom_off[i];
        bc.tiles_x = (bc.p.W + 31) / 32;
        bc.tiles_y = (bc.p.H + cfg.tile_rows - 1) / cfg.tile_rows;
        bc.item_begin = item;
        const long long chunks = (bc.n_out + cfg.frame_chunk - 1) / cfg.frame_chunk;
        item += chunks * bc.tiles_x * bc.tiles_y;
    }
    bs.n_items = item;
}

GatherArgs batch_gather_args(ssvp_ctx *ctx, const ssvp_params &p) {
    GatherArgs a{};
    a.n_slots = 2 * p.half_window + 1;
    a.T = p.half_window;
    a.k = p.k;
    a.mode = p.mode;
    a.radius = p.radius;
    a.sigma_rgb = p.sigma_rgb;
    a.sigma_xyz = p.sigma_xyz;
    a.sigma_f = p.sigma_f;
    a.stat_counts = ctx->stat_counts;
    a.stat_sumw = ctx->stat_sumw;
    return a;
}

bool valid_config(const ssvp_plan_config &c) {
    return (c.tile_rows == 4 || c.tile_rows == 8) && c.frame_chunk >= 1 && c.frame_chunk <= 16;
}

const ssvp_plan_config *find_tuned(const ssvp_ctx *ctx, const ssvp_params &p, int cfmt) {
    for (const auto &t : ctx->tuned)
        if (t.k == p.k && t.T == p.half_window && t.mode == p.mode && t.cfmt == cfmt) return &t.cfg;
    return nullptr;
}


// ---------------------------------------------------------------- learned filter (A8/A9)

int mlp_alloc(ssvp_ctx *ctx) {
    if (ctx->mlp_buf) return SSVP_OK;
    const size_t nf = 4 * (size_t)ssvp::kMlpParams + 1 + 128;
    CK(cudaMalloc(&ctx->mlp_buf, nf * sizeof(float)), "cudaMalloc (mlp)");
    CK(cudaMalloc(&ctx->mlp_w1, 1024 * sizeof(unsigned short)), "cudaMalloc (mlp)");
    ssvp::MlpState &st = ctx->mlp;
    st.master = ctx->mlp_buf;
    st.m = st.master + ssvp::kMlpParams;
    st.v = st.m + ssvp::kMlpParams;
    st.grad = st.v + ssvp::kMlpParams;
    st.W2_r = st.grad + ssvp::kMlpParams + 1;
    st.W1_bf16 = ctx->mlp_w1;
    return SSVP_OK;
}

ssvp::MlpWeights mlp_weights(const ssvp_ctx *ctx) {
    ssvp::MlpWeights w;
    w.W1 = ctx->mlp.W1_bf16;
    w.b1 = ctx->mlp.master + ssvp::kMlpB1;
    w.W2 = ctx->mlp.W2_r;
    w.b2 = ctx->mlp.master + ssvp::kMlpB2;
    return w;
}

// scratch for the capped sample sets of n_px crop pixels
void free_sets(ssvp::SampleSets &S) {
    for (void *q : {(void *)S.col, (void *)S.f89, (void *)S.info, (void *)S.n, (void *)S.plain})
        if (q) cudaFree(q);
    S = ssvp::SampleSets{};
}

int learned_scratch(ssvp_ctx *ctx, size_t n_px) {
    // the kernels address a crop's sets with one 32-bit sample index (pixel * 64 + slot)
    if (n_px * 64 > 0xffffffffull)
        return fail(ctx, SSVP_EINVAL, "the learned filter takes crops of at most 67,108,863 pixels (have %zu)", n_px);
    if (n_px <= ctx->l_cap) return SSVP_OK;
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    free_sets(ctx->l_sets);
    ctx->l_cap = 0;
    ssvp::SampleSets &S = ctx->l_sets;
    CK(cudaMalloc(&S.col, n_px * 64 * sizeof(float4)), "cudaMalloc (learned scratch)");
    CK(cudaMalloc(&S.f89, n_px * 64 * sizeof(unsigned)), "cudaMalloc (learned scratch)");
    CK(cudaMalloc(&S.info, n_px * sizeof(float4)), "cudaMalloc (learned scratch)");
    CK(cudaMalloc(&S.n, n_px * sizeof(int32_t)), "cudaMalloc (learned scratch)");
    CK(cudaMalloc(&S.plain, n_px * 3 * sizeof(float)), "cudaMalloc (learned scratch)");
    ctx->l_cap = n_px;
    return SSVP_OK;
}

// capped sample sets of output frame O of a clip over a crop, into the context's scratch
int extract_samples(ssvp_ctx *ctx, const ssvp_params &p, int clip_id, int O, int x0, int y0, int cw, int ch) {
    Clip &c = ctx->clips[clip_id];
    const int T = p.half_window, ns = 2 * T + 1;
    if ((size_t)ns > ctx->geom_cap) {
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        if (ctx->geom) cudaFree(ctx->geom);
        ctx->geom = nullptr;
        ctx->geom_cap = 0;
        CK(cudaMalloc(&ctx->geom, std::max<size_t>(ns, 4096) * sizeof(PairGeom)), "cudaMalloc (geometry)");
        ctx->geom_cap = std::max<size_t>(ns, 4096);
    }
    ctx->host_geom.resize(ns);
    compose_table(c, O, 1, T, p.sigma_f, ctx->host_geom.data());
    CK(cudaMemcpyAsync(ctx->geom, ctx->host_geom.data(), ns * sizeof(PairGeom), cudaMemcpyHostToDevice, ctx->stream),
       "cudaMemcpyAsync (geometry)");
    GatherArgs a{};
    a.clip = c.p;
    a.geom = ctx->geom;
    a.frame_begin = O;
    a.n_out = 1;
    a.n_slots = ns;
    a.T = T;
    a.x0 = x0; a.y0 = y0; a.cw = cw; a.ch = ch;
    a.k = p.k;
    a.mode = SSVP_MODE_DENOISE;
    a.radius = p.radius;
    a.sigma_rgb = p.sigma_rgb;
    a.sigma_xyz = p.sigma_xyz;
    a.sigma_f = p.sigma_f;
    a.sets = ctx->l_sets;
    a.stat_counts = ctx->stat_counts;
    a.stat_sumw = ctx->stat_sumw;
    TraceScope ts(ctx, SSVP_TRACE_EXTRACT, ctx->stream);
    CK(ssvp::launch_gather(a, ctx->stream), "gather kernel (learned samples)");
    return SSVP_OK;
}

// splitmix64 draws for training (frame and pixel sampling, He initialisation)
struct Rng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uniform() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return std::sqrt(-2.0 * std::log(uniform())) * std::cos(6.283185307179586 * uniform()); }
};

}  // namespace

namespace ssvp {
void set_global_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_create_error, sizeof(g_create_error), fmt, ap);
    va_end(ap);
}
}  // namespace ssvp

extern "C" {

void ssvp_params_default(ssvp_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->mode = SSVP_MODE_DENOISE;
    p->k = 7;
    p->half_window = 15;
    p->frame_begin = 0;
    p->frame_end = -1;  // all frames
    p->radius = -0.005f;
    p->sigma_rgb = 40.0f / 255.0f;
    p->sigma_xyz = 0.0f;
    p->sigma_f = 6.0f;
    p->aperture = 0.05f;
    p->focal_depth = 0.0f;
    p->a0 = 0.0f;
    p->lens_samples = 16;
    p->cap = 31;
    p->max_samples = 64;
    p->conf_threshold = 0.5f;
    p->gather = SSVP_GATHER_WINDOW;
    p->frustum_l = 3.0f;
    p->near_plane = 0.01f;
    p->far_plane = 1000.0f;
    p->sigma_area = 0.0f;
}

int ssvp_create(ssvp_ctx **out, int cuda_device, void *cuda_stream) {
    if (!out) return fail(nullptr, SSVP_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return fail(nullptr, SSVP_EDEVICE, "no CUDA device: %s", e == cudaSuccess ? "count is 0" : cudaGetErrorString(e));
    }
    if (cuda_device < 0 || cuda_device >= n) return fail(nullptr, SSVP_EINVAL, "device %d out of range [0, %d)", cuda_device, n);
    if ((e = cudaSetDevice(cuda_device)) != cudaSuccess) return fail(nullptr, SSVP_EDEVICE, "cudaSetDevice: %s", cudaGetErrorString(e));
    ssvp_ctx *ctx = new (std::nothrow) ssvp_ctx();
    if (!ctx) return fail(nullptr, SSVP_ENOMEM, "host allocation failed");
    ctx->device = cuda_device;
    ctx->stream = (cudaStream_t)cuda_stream;
    int prio_least = 0, prio_greatest = 0;
    if ((e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest)) != cudaSuccess ||
        (e = cudaStreamCreateWithPriority(&ctx->load_stream, cudaStreamNonBlocking, prio_greatest)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ctx->ev_load_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ctx->ev_load_out, cudaEventDisableTiming)) != cudaSuccess) {
        int rc = fail(nullptr, SSVP_ECUDA, "load stream: %s", cudaGetErrorString(e));
        ssvp_destroy(ctx);
        return rc;
    }
    if ((e = cudaMalloc(&ctx->stat_counts, 2 * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->stat_sumw, sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->median_scratch, ssvp::median_scratch_words() * sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->d_kerr, sizeof(int))) != cudaSuccess) {
        int rc = fail(nullptr, e == cudaErrorMemoryAllocation ? SSVP_ENOMEM : SSVP_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
        ssvp_destroy(ctx);
        return rc;
    }
    cudaMemsetAsync(ctx->stat_counts, 0, 2 * sizeof(unsigned long long), ctx->stream);
    cudaMemsetAsync(ctx->stat_sumw, 0, sizeof(double), ctx->stream);
    cudaMemsetAsync(ctx->d_kerr, 0, sizeof(int), ctx->stream);
    *out = ctx;
    return SSVP_OK;
}

void ssvp_destroy(ssvp_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->load_stream) cudaStreamSynchronize(ctx->load_stream);
    for (auto &c : ctx->clips) free_clip(c);  // plans of this context must be destroyed first
    if (ctx->stat_counts) cudaFree(ctx->stat_counts);
    if (ctx->stat_sumw) cudaFree(ctx->stat_sumw);
    if (ctx->median_scratch) cudaFree(ctx->median_scratch);
    if (ctx->d_kerr) cudaFree(ctx->d_kerr);
    if (ctx->geom) cudaFree(ctx->geom);
    if (ctx->staging) cudaFree(ctx->staging);
    if (ctx->d_shutter_log2) cudaFree(ctx->d_shutter_log2);
    if (ctx->mask_cam) cudaFree(ctx->mask_cam);
    free_sets(ctx->l_sets);
    for (void *q : {(void *)ctx->mlp_buf, (void *)ctx->mlp_w1, (void *)ctx->l_loss, (void *)ctx->l_batch})
        if (q) cudaFree(q);
    for (auto &r : ctx->trace_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : ctx->trace_free) cudaEventDestroy(e);
    if (ctx->ev_load_in) cudaEventDestroy(ctx->ev_load_in);
    if (ctx->ev_load_out) cudaEventDestroy(ctx->ev_load_out);
    if (ctx->load_stream) cudaStreamDestroy(ctx->load_stream);
    delete ctx;
}

const char *ssvp_last_error(const ssvp_ctx *ctx) { return ctx ? ctx->err : g_create_error; }

int ssvp_set_stream(ssvp_ctx *ctx, void *cuda_stream) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    ctx->stream = (cudaStream_t)cuda_stream;
    return SSVP_OK;
}

int ssvp_load_clip(ssvp_ctx *ctx, int clip_id, int W, int H, int F, const float *rgb, const float *depth, int mem_kind,
                   int colour_fmt) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    if (W < 1 || H < 1 || F < 1 || W > 16384 || H > 16384 || F > 65535)
        return fail(ctx, SSVP_EINVAL, "bad clip shape W=%d H=%d F=%d", W, H, F);
    if (!rgb || !depth) return fail(ctx, SSVP_EINVAL, "rgb and depth must not be NULL");
    if (mem_kind != SSVP_MEM_HOST && mem_kind != SSVP_MEM_DEVICE) return fail(ctx, SSVP_EINVAL, "bad mem_kind %d", mem_kind);
    if (colour_fmt != SSVP_COLOUR_F32 && colour_fmt != SSVP_COLOUR_F16)
        return fail(ctx, SSVP_EINVAL, "bad colour_fmt %d", colour_fmt);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc;
    if ((rc = check_mem(ctx, rgb, mem_kind, "rgb")) != SSVP_OK || (rc = check_mem(ctx, depth, mem_kind, "depth")) != SSVP_OK)
        return rc;
    Clip &c = ctx->clips[clip_id];
    // a reload with the same shape and format keeps the planes (and the inpainting mask, if one is
    // set): the work queued on the context's stream that still reads them runs before the upload
    const bool reuse = c.loaded && c.p.W == W && c.p.H == H && c.p.F == F && c.p.colour_fmt == colour_fmt;
    if (c.loaded && !reuse) {
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        CK(cudaStreamSynchronize(ctx->load_stream), "cudaStreamSynchronize");
        free_clip(c);
    }
    Planes &p = c.p;
    p.W = W;
    p.H = H;
    p.F = F;
    p.pitch = ((W + 2 * ssvp::kPad) + 31) / 32 * 32;
    p.rows = H + 2 * ssvp::kPad;
    p.fstride = (long long)p.pitch * p.rows;
    p.colour_fmt = colour_fmt;
    const size_t texel = colour_fmt == SSVP_COLOUR_F32 ? 16 : 8;
    const size_t nplane = (size_t)F * (size_t)p.fstride;
    const size_t nout = (size_t)F * H * W * 3;
    cudaError_t e = cudaSuccess;
    if (!reuse && ((e = cudaMalloc(&p.depth, nplane * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&p.colour, nplane * texel)) != cudaSuccess ||
        (e = cudaMalloc(&p.out, nout * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&p.median, sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&p.zrange, 2 * sizeof(unsigned int) * (size_t)F)) != cudaSuccess ||
        (e = cudaMalloc(&p.grad_sum, sizeof(double) * (size_t)F)) != cudaSuccess ||
        (e = cudaMalloc(&p.grad_log2, sizeof(float) * (size_t)F)) != cudaSuccess ||
        (e = cudaMalloc(&p.grad_partial, sizeof(double) * ssvp::grad_partial_words(F))) != cudaSuccess)) {
        free_clip(c);
        return cuda_fail(ctx, e, "cudaMalloc (clip planes)");
    }
    // the load's work goes to the high-priority load stream, after everything already queued on
    // the context's stream (which may still read the planes being replaced)
    cudaStream_t ls = ctx->load_stream;
    CK(cudaEventRecord(ctx->ev_load_in, ctx->stream), "cudaEventRecord");
    CK(cudaStreamWaitEvent(ls, ctx->ev_load_in, 0), "cudaStreamWaitEvent");
    {
        TraceScope ts(ctx, SSVP_TRACE_LOAD, ls);
        // padding and invalid depth: NaN (all bits set); colour 0; output 0.  A reload keeps the
        // padding of the planes it reuses (the packing rewrites every pixel inside them)
        if (!reuse) {
            CK(cudaMemsetAsync(p.depth, 0xff, nplane * sizeof(float), ls), "cudaMemsetAsync");
            CK(cudaMemsetAsync(p.colour, 0, nplane * texel, ls), "cudaMemsetAsync");
        }
        if (!reuse) {
            CK(cudaMemsetAsync(p.out, 0, nout * sizeof(float), ls), "cudaMemsetAsync");
        } else if (c.out_hi > c.out_lo) {
            const size_t per = (size_t)W * H * 3;
            CK(cudaMemsetAsync(p.out + per * (size_t)c.out_lo, 0, per * (size_t)(c.out_hi - c.out_lo) * sizeof(float), ls),
               "cudaMemsetAsync");
        }
        c.out_lo = c.out_hi = 0;
        const size_t frame_px = (size_t)W * H;
        if (mem_kind == SSVP_MEM_DEVICE) {
            CK(ssvp::launch_pack(rgb, depth, W, H, F, p, 0, ls), "pack kernel");
        } else {
            // stage the frames through a device buffer: the whole clip in one copy up to 4 GB (the
            // copy engines then run without waiting for a pack kernel between chunks), larger clips
            // in chunks of that size
            const size_t per_frame = frame_px * 16;
            int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)F, ((size_t)4 << 30) / per_frame));
            const size_t need = per_frame * (size_t)chunk;
            if (ctx->staging_bytes < need) {
                CK(cudaStreamSynchronize(ls), "cudaStreamSynchronize");
                if (ctx->staging) cudaFree(ctx->staging);
                ctx->staging = nullptr;
                ctx->staging_bytes = 0;
                if ((e = cudaMalloc(&ctx->staging, need)) != cudaSuccess) {
                    free_clip(c);
                    return cuda_fail(ctx, e, "cudaMalloc (staging)");
                }
                ctx->staging_bytes = need;
            }
            float *srgb = (float *)ctx->staging;
            float *sdep = srgb + frame_px * 3 * (size_t)chunk;
            for (int f0 = 0; f0 < F; f0 += chunk) {
                int nf = std::min(chunk, F - f0);
                CK(cudaMemcpyAsync(srgb, rgb + frame_px * 3 * (size_t)f0, frame_px * 3 * nf * sizeof(float),
                    cudaMemcpyHostToDevice, ls), "cudaMemcpyAsync (rgb)");
                CK(cudaMemcpyAsync(sdep, depth + frame_px * (size_t)f0, frame_px * nf * sizeof(float), cudaMemcpyHostToDevice,
                    ls), "cudaMemcpyAsync (depth)");
                CK(ssvp::launch_pack(srgb, sdep, W, H, nf, p, f0, ls), "pack kernel");
            }
        }
        CK(ssvp::launch_median(p, ctx->median_scratch, ls), "median kernels");
    }
    c.zrange_ready = c.grad_ready = false;
    // everything queued on the context's stream from here on runs after the load
    CK(cudaEventRecord(ctx->ev_load_out, ls), "cudaEventRecord");
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_load_out, 0), "cudaStreamWaitEvent");
    c.loaded = true;
    c.has_cams = false;
    c.generation = ++ctx->clip_generation[clip_id];
    return SSVP_OK;
}

int ssvp_unload_clip(ssvp_ctx *ctx, int clip_id) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    if (!ctx->clips[clip_id].loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    free_clip(ctx->clips[clip_id]);
    ++ctx->clip_generation[clip_id];
    return SSVP_OK;
}

// F frames of cameras: per-frame (or one shared) K and world->camera [R|t], checked (finite, zero
// skew, orthonormal R) and expanded to per-frame arrays
static int checked_cameras(ssvp_ctx *ctx, int F, const double *K, int per_frame_K, const double *w2c,
                           std::vector<double> &Kv, std::vector<double> &Wv) {
    Kv.assign((size_t)F * 9, 0.0);
    Wv.assign(w2c, w2c + (size_t)F * 12);
    for (int f = 0; f < F; ++f) std::memcpy(&Kv[9 * (size_t)f], K + (per_frame_K ? 9 * (size_t)f : 0), 9 * sizeof(double));
    if (!finite_all(Kv.data(), Kv.size()) || !finite_all(Wv.data(), Wv.size()))
        return fail(ctx, SSVP_EINVAL, "cameras must be finite");
    for (int f = 0; f < F; ++f) {
        const double *k = &Kv[9 * (size_t)f];
        if (!(k[0] > 0 && k[4] > 0) || k[1] != 0.0 || k[3] != 0.0 || k[6] != 0.0 || k[7] != 0.0 || k[8] != 1.0)
            return fail(ctx, SSVP_EINVAL, "frame %d: K must be [[fx,0,cx],[0,fy,cy],[0,0,1]] with fx, fy > 0", f);
        const double *R = &Wv[12 * (size_t)f];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double d = R[4 * i] * R[4 * j] + R[4 * i + 1] * R[4 * j + 1] + R[4 * i + 2] * R[4 * j + 2];
                if (std::fabs(d - (i == j ? 1.0 : 0.0)) > 1e-6)
                    return fail(ctx, SSVP_EINVAL, "frame %d: w2c rotation is not orthonormal", f);
            }
    }
    return SSVP_OK;
}

int ssvp_set_cameras(ssvp_ctx *ctx, int clip_id, const double *K, int per_frame_K, const double *w2c) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    Clip &c = ctx->clips[clip_id];
    if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    if (!K || !w2c) return fail(ctx, SSVP_EINVAL, "K and w2c must not be NULL");
    int rc;
    if ((rc = check_mem(ctx, K, SSVP_MEM_HOST, "K")) != SSVP_OK || (rc = check_mem(ctx, w2c, SSVP_MEM_HOST, "w2c")) != SSVP_OK)
        return rc;
    std::vector<double> Kv, Wv;
    rc = checked_cameras(ctx, c.p.F, K, per_frame_K, w2c, Kv, Wv);
    if (rc != SSVP_OK) return rc;
    c.K.swap(Kv);
    c.w2c.swap(Wv);
    c.has_cams = true;
    return SSVP_OK;
}

int ssvp_append_frames(ssvp_ctx *ctx, int clip_id, int n, const float *rgb, const float *depth, int mem_kind,
                       const double *K, int per_frame_K, const double *w2c) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    Clip &c = ctx->clips[clip_id];
    if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    if (!c.has_cams) return fail(ctx, SSVP_ENOCAM, "clip %d has no cameras", clip_id);
    if (c.p.mask)
        return fail(ctx, SSVP_EINVAL, "clip %d has an inpainting mask: unload and load it to append frames", clip_id);
    const int W = c.p.W, H = c.p.H, F = c.p.F;
    if (n < 1 || n > F) return fail(ctx, SSVP_EINVAL, "n=%d must be in [1, %d] (the clip's frame count)", n, F);
    if (!rgb || !depth || !K || !w2c) return fail(ctx, SSVP_EINVAL, "rgb, depth, K and w2c must not be NULL");
    if (mem_kind != SSVP_MEM_HOST && mem_kind != SSVP_MEM_DEVICE) return fail(ctx, SSVP_EINVAL, "bad mem_kind %d", mem_kind);
    int rc;
    if ((rc = check_mem(ctx, K, SSVP_MEM_HOST, "K")) != SSVP_OK || (rc = check_mem(ctx, w2c, SSVP_MEM_HOST, "w2c")) != SSVP_OK)
        return rc;
    std::vector<double> Kn, Wn;
    rc = checked_cameras(ctx, n, K, per_frame_K, w2c, Kn, Wn);
    if (rc != SSVP_OK) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if ((rc = check_mem(ctx, rgb, mem_kind, "rgb")) != SSVP_OK || (rc = check_mem(ctx, depth, mem_kind, "depth")) != SSVP_OK)
        return rc;
    Planes &p = c.p;
    const size_t texel = p.colour_fmt == SSVP_COLOUR_F32 ? 16 : 8;
    const size_t nplane = (size_t)F * (size_t)p.fstride;
    cudaError_t e = cudaSuccess;
    Planes &sp = c.spare;
    if (!sp.depth) {
        // the spare window, its planes padded like the current ones (padding is never written again)
        if ((e = cudaMalloc(&sp.depth, nplane * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&sp.colour, nplane * texel)) != cudaSuccess ||
            (e = cudaMalloc(&sp.median, sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&sp.zrange, 2 * sizeof(unsigned int) * (size_t)F)) != cudaSuccess ||
            (e = cudaMalloc(&sp.grad_sum, sizeof(double) * (size_t)F)) != cudaSuccess ||
            (e = cudaMalloc(&sp.grad_log2, sizeof(float) * (size_t)F)) != cudaSuccess ||
            (e = cudaMalloc(&sp.grad_partial, sizeof(double) * ssvp::grad_partial_words(F))) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&c.ev_append, cudaEventDisableTiming)) != cudaSuccess) {
            for (void *q : {(void *)sp.depth, (void *)sp.colour, (void *)sp.median, (void *)sp.zrange,
                            (void *)sp.grad_sum, (void *)sp.grad_log2, (void *)sp.grad_partial})
                if (q) cudaFree(q);
            sp = Planes{};
            return cuda_fail(ctx, e, "cudaMalloc (spare window)");
        }
        CK(cudaMemsetAsync(sp.depth, 0xff, nplane * sizeof(float), ctx->stream), "cudaMemsetAsync");
        CK(cudaMemsetAsync(sp.colour, 0, nplane * texel, ctx->stream), "cudaMemsetAsync");
        CK(cudaEventRecord(c.ev_append, ctx->stream), "cudaEventRecord");
    }
    // the new window is built in the spare planes on the load stream.  It must follow every read of
    // them, and those were all queued before the previous append (which made the current planes
    // current): the load stream waits for that point only, not for the gathers queued since,
    // which read the current planes, so building the next window overlaps them
    cudaStream_t ls = ctx->load_stream;
    CK(cudaStreamWaitEvent(ls, c.ev_append, 0), "cudaStreamWaitEvent");
    CK(cudaEventRecord(c.ev_append, ctx->stream), "cudaEventRecord");
    Planes q = p;  // the next window: the shared fields of p with the spare window's arrays
    q.depth = sp.depth;
    q.colour = sp.colour;
    q.median = sp.median;
    q.zrange = sp.zrange;
    q.grad_sum = sp.grad_sum;
    q.grad_log2 = sp.grad_log2;
    q.grad_partial = sp.grad_partial;
    {
        TraceScope ts(ctx, SSVP_TRACE_LOAD, ls);
        const size_t keep = (size_t)(F - n) * (size_t)p.fstride;
        if (keep) {
            CK(cudaMemcpyAsync(q.depth, p.depth + (size_t)n * p.fstride, keep * sizeof(float), cudaMemcpyDeviceToDevice, ls),
                "cudaMemcpyAsync (window)");
            CK(cudaMemcpyAsync(q.colour, (const char *)p.colour + (size_t)n * p.fstride * texel, keep * texel,
                cudaMemcpyDeviceToDevice, ls),
                "cudaMemcpyAsync (window)");
        }
        const size_t frame_px = (size_t)W * H;
        if (mem_kind == SSVP_MEM_DEVICE) {
            // device inputs may be produced by work queued on the context's stream up to this call
            CK(cudaStreamWaitEvent(ls, c.ev_append, 0), "cudaStreamWaitEvent");
            CK(ssvp::launch_pack(rgb, depth, W, H, n, q, F - n, ls), "pack kernel");
        } else {
            const size_t need = frame_px * 16 * (size_t)n;
            if (ctx->staging_bytes < need) {
                CK(cudaStreamSynchronize(ls), "cudaStreamSynchronize");
                if (ctx->staging) cudaFree(ctx->staging);
                ctx->staging = nullptr;
                ctx->staging_bytes = 0;
                if ((e = cudaMalloc(&ctx->staging, need)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc (staging)");
                ctx->staging_bytes = need;
            }
            float *srgb = (float *)ctx->staging;
            float *sdep = srgb + frame_px * 3 * (size_t)n;
            CK(cudaMemcpyAsync(srgb, rgb, frame_px * 3 * n * sizeof(float), cudaMemcpyHostToDevice, ls), "cudaMemcpyAsync (rgb)");
            CK(cudaMemcpyAsync(sdep, depth, frame_px * n * sizeof(float), cudaMemcpyHostToDevice, ls), "cudaMemcpyAsync (depth)");
            CK(ssvp::launch_pack(srgb, sdep, W, H, n, q, F - n, ls), "pack kernel");
        }
        CK(ssvp::launch_median(q, ctx->median_scratch, ls), "median kernels");
    }
    CK(cudaEventRecord(ctx->ev_load_out, ls), "cudaEventRecord");
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_load_out, 0), "cudaStreamWaitEvent");
    // the spare window becomes current; the cameras slide with the frames
    swap_window(p, sp);
    c.zrange_ready = c.grad_ready = false;
    c.K.erase(c.K.begin(), c.K.begin() + 9 * (size_t)n);
    c.K.insert(c.K.end(), Kn.begin(), Kn.end());
    c.w2c.erase(c.w2c.begin(), c.w2c.begin() + 12 * (size_t)n);
    c.w2c.insert(c.w2c.end(), Wn.begin(), Wn.end());
    c.generation = ++ctx->clip_generation[clip_id];
    return SSVP_OK;
}

int ssvp_gather_filter(ssvp_ctx *ctx, const ssvp_params *params, const int *clip_ids, int n_clips) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    int rc = check_params(ctx, params);
    if (rc != SSVP_OK) return rc;
    if (!clip_ids || n_clips < 1 || n_clips > SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "bad clip list");
    const ssvp_params &p = *params;
    const int T = p.half_window, ns = 2 * T + 1;
    // resolve ranges and compose the geometry of every (clip, O, slot)
    std::vector<int> fb(n_clips), nout(n_clips), cx0(n_clips), cy0(n_clips), cw(n_clips), chh(n_clips);
    size_t total = 0;
    for (int i = 0; i < n_clips; ++i) {
        int id = clip_ids[i];
        if (id < 0 || id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", id);
        Clip &c = ctx->clips[id];
        if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", id);
        if (!c.has_cams) return fail(ctx, SSVP_ENOCAM, "clip %d has no cameras", id);
        int b = p.frame_begin, e = p.frame_end < 0 ? c.p.F : p.frame_end;
        if (b < 0 || e > c.p.F || b > e) return fail(ctx, SSVP_EINVAL, "frame range [%d, %d) outside clip %d (F=%d)", b, e, id, c.p.F);
        int x0 = p.crop_x, y0 = p.crop_y, w = p.crop_w, h = p.crop_h;
        if (w == 0 || h == 0) { x0 = 0; y0 = 0; w = c.p.W; h = c.p.H; }
        if (x0 < 0 || y0 < 0 || x0 + w > c.p.W || y0 + h > c.p.H)
            return fail(ctx, SSVP_EINVAL, "crop (%d, %d, %d, %d) outside clip %d (%dx%d)", x0, y0, w, h, id, c.p.W, c.p.H);
        fb[i] = b; nout[i] = e - b; cx0[i] = x0; cy0[i] = y0; cw[i] = w; chh[i] = h;
        c.mark_out(b, e);
        total += (size_t)(e - b) * ns;
    }
    if ((p.membership_out || p.pixel_stats_out) && (n_clips != 1 || nout[0] > 1))
        return fail(ctx, SSVP_EINVAL, "debug outputs need exactly one clip and at most one output frame");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (p.mode == SSVP_MODE_LEARNED) {
        // per output frame: capped sample sets into scratch, then the tensor-core MLP
        if (!ctx->mlp_set) return fail(ctx, SSVP_EINVAL, "learned mode needs a network (ssvp_set_mlp or ssvp_train)");
        if (p.k > 7) return fail(ctx, SSVP_EINVAL, "the learned filter supports k <= 7");
        if (p.membership_out || p.pixel_stats_out) return fail(ctx, SSVP_EINVAL, "learned mode has no debug outputs");
        if (p.test_skip_mma != 0 && p.test_skip_mma != 1) return fail(ctx, SSVP_EINVAL, "test_skip_mma must be 0 or 1");
        CK(cudaMemsetAsync(ctx->stat_counts, 0, 2 * sizeof(unsigned long long), ctx->stream), "cudaMemsetAsync");
        CK(cudaMemsetAsync(ctx->stat_sumw, 0, sizeof(double), ctx->stream), "cudaMemsetAsync");
        for (int i = 0; i < n_clips; ++i) {
            Clip &c = ctx->clips[clip_ids[i]];
            const size_t npx = (size_t)cw[i] * chh[i];
            if ((rc = learned_scratch(ctx, npx)) != SSVP_OK) return rc;
            for (int oi = 0; oi < nout[i]; ++oi) {
                const int O = fb[i] + oi;
                if ((rc = extract_samples(ctx, p, clip_ids[i], O, cx0[i], cy0[i], cw[i], chh[i])) != SSVP_OK)
                    return rc;
                ssvp::MlpArgs m{};
                m.w = mlp_weights(ctx);
                m.sets = ctx->l_sets;
                m.n_px = (long long)npx;
                m.O = O; m.W = c.p.W; m.H = c.p.H; m.x0 = cx0[i]; m.y0 = cy0[i]; m.cw = cw[i];
                m.tau = p.conf_threshold;
                m.out = c.p.out;
                m.skip_mma = p.test_skip_mma;
                TraceScope ts(ctx, SSVP_TRACE_INFER, ctx->stream);
                CK(ssvp::launch_mlp_infer_tc(m, ctx->d_kerr, ctx->stream), "mlp inference kernel");
            }
        }
        return SSVP_OK;
    }
    // Eq. 10: the shutter table must cover the window; its log2 weights go to the device per call
    const bool shutter = p.mode == SSVP_MODE_SHUTTER;
    if (shutter) {
        if ((int)ctx->shutter.size() != ns)
            return fail(ctx, SSVP_EINVAL, "shutter mode needs ssvp_set_shutter with half_window %d (have %d values)", T,
                        (int)ctx->shutter.size());
        if (!ctx->d_shutter_log2) CK(cudaMalloc(&ctx->d_shutter_log2, sizeof(float) * ssvp::kMaxSlots), "cudaMalloc (shutter)");
        std::vector<float> lg(ns);
        for (int j = 0; j < ns; ++j) lg[j] = (float)std::log2((double)ctx->shutter[j]);  // log2(0) = -inf: weight 0
        CK(cudaMemcpyAsync(ctx->d_shutter_log2, lg.data(), sizeof(float) * ns, cudaMemcpyHostToDevice, ctx->stream),
           "cudaMemcpyAsync (shutter)");
    }
    if (p.mode == SSVP_MODE_INPAINT || p.mode == SSVP_MODE_SEMI)
        for (int i = 0; i < n_clips; ++i)
            if (!ctx->clips[clip_ids[i]].p.mask)
                return fail(ctx, SSVP_EINVAL, "inpainting needs a mask for clip %d (ssvp_set_mask or ssvp_mask_from_box)",
                            clip_ids[i]);
    // the shutter and inpainting weights have no frame-distance term: sigma_f = infinity (beta = 0);
    // semi-transparency keeps it for its Eq. 4 term (the kernel leaves it out of the Eq. 9 term)
    const double sigma_f = shutter || p.mode == SSVP_MODE_INPAINT ? INFINITY : (double)p.sigma_f;
    // the frustum gather also needs the back maps: a second table of the same shape after the first
    const bool frustum = p.gather == SSVP_GATHER_FRUSTUM;
    const size_t entries = frustum ? 2 * total : total;
    if (entries > ctx->geom_cap) {
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        if (ctx->geom) cudaFree(ctx->geom);
        ctx->geom = nullptr;
        ctx->geom_cap = 0;
        size_t cap = std::max<size_t>(entries, 4096);
        CK(cudaMalloc(&ctx->geom, cap * sizeof(PairGeom)), "cudaMalloc (geometry)");
        ctx->geom_cap = cap;
    }
    ctx->host_geom.resize(std::max<size_t>(entries, 1));
    size_t off = 0;
    for (int i = 0; i < n_clips; ++i) {
        compose_table(ctx->clips[clip_ids[i]], fb[i], nout[i], T, sigma_f, &ctx->host_geom[off]);
        if (frustum) compose_table_back(ctx->clips[clip_ids[i]], fb[i], nout[i], T, sigma_f, &ctx->host_geom[total + off]);
        off += (size_t)nout[i] * ns;
    }
    // pageable source: the call returns once the table is staged, so host_geom may be reused
    if (entries)
        CK(cudaMemcpyAsync(ctx->geom, ctx->host_geom.data(), entries * sizeof(PairGeom), cudaMemcpyHostToDevice, ctx->stream),
           "cudaMemcpyAsync (geometry)");
    CK(cudaMemsetAsync(ctx->stat_counts, 0, 2 * sizeof(unsigned long long), ctx->stream), "cudaMemsetAsync");
    CK(cudaMemsetAsync(ctx->stat_sumw, 0, sizeof(double), ctx->stream), "cudaMemsetAsync");
    off = 0;
    for (int i = 0; i < n_clips; ++i) {
        Clip &c = ctx->clips[clip_ids[i]];
        GatherArgs a{};
        a.clip = c.p;
        a.geom = ctx->geom + off;
        a.frame_begin = fb[i];
        a.n_out = nout[i];
        a.n_slots = ns;
        a.T = T;
        a.x0 = cx0[i]; a.y0 = cy0[i]; a.cw = cw[i]; a.ch = chh[i];
        a.k = p.k;
        a.mode = p.mode;
        a.radius = p.radius;
        a.sigma_rgb = p.sigma_rgb;
        a.sigma_xyz = p.sigma_xyz;
        a.sigma_f = p.sigma_f;
        a.aperture = p.aperture;
        a.focal_depth = p.focal_depth;
        a.a0 = p.a0;
        a.cap = p.cap;
        a.lens_n = p.mode == SSVP_MODE_APERTURE ? p.lens_samples : 0;
        for (int i = 0; i < a.lens_n; ++i) {
            // Vogel (golden-angle) disc of unit radius; the kernel scales it by the lens radius
            const double rho = std::sqrt((i + 0.5) / a.lens_n), th = 2.399963229728653 * i;
            a.lens_xy[2 * i] = (float)(rho * std::cos(th));
            a.lens_xy[2 * i + 1] = (float)(rho * std::sin(th));
        }
        a.membership = (int32_t *)p.membership_out;
        a.pixel_stats = (int32_t *)p.pixel_stats_out;
        a.stage = p.gather == SSVP_GATHER_WINDOW_TMA ? (p.test_skip_mma ? 2 : 1) : 0;
        a.err = ctx->d_kerr;
        a.stat_counts = ctx->stat_counts;
        a.stat_sumw = ctx->stat_sumw;
        a.geom_back = frustum ? ctx->geom + total + off : nullptr;
        if ((rc = ensure_frame_values(ctx, c, frustum, p.mode == SSVP_MODE_DEBLUR)) != SSVP_OK) return rc;
        a.frame_log2w = p.mode == SSVP_MODE_DEBLUR ? c.p.grad_log2 : nullptr;
        a.slot_log2w = shutter ? ctx->d_shutter_log2 : nullptr;
        a.frustum_l = p.frustum_l;
        a.near_plane = p.near_plane;
        a.far_plane = p.far_plane;
        TraceScope ts(ctx, frustum ? SSVP_TRACE_FRUSTUM : p.mode == SSVP_MODE_APERTURE ? SSVP_TRACE_APERTURE
                                                                                       : SSVP_TRACE_GATHER,
                      ctx->stream);
        if (frustum) CK(ssvp::launch_frustum(a, ctx->stream), "frustum kernel");
        else if (p.mode == SSVP_MODE_APERTURE) CK(ssvp::launch_aperture(a, ctx->stream), "aperture kernel");
        else CK(ssvp::launch_gather(a, ctx->stream), "gather kernel");
        off += (size_t)nout[i] * ns;
    }
    return SSVP_OK;
}

int ssvp_superres(ssvp_ctx *ctx, const ssvp_params *params, int clip_id, int scale, float *out) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    int rc = check_params(ctx, params);
    if (rc != SSVP_OK) return rc;
    const ssvp_params &p = *params;
    if (p.mode != SSVP_MODE_DENOISE && p.mode != SSVP_MODE_MEAN)
        return fail(ctx, SSVP_EINVAL, "super-resolution weights are Eq. 7 (SSVP_MODE_DENOISE) or w = 1 (SSVP_MODE_MEAN)");
    if (scale < 1 || scale > 8) return fail(ctx, SSVP_EINVAL, "scale=%d must be in [1, 8]", scale);
    if (!out) return fail(ctx, SSVP_EINVAL, "out is NULL");
    if ((rc = check_mem(ctx, out, SSVP_MEM_DEVICE, "out")) != SSVP_OK) return rc;
    if (!(p.frustum_l > 0.0f && p.frustum_l <= 64.0f)) return fail(ctx, SSVP_EINVAL, "frustum_l must be in (0, 64]");
    if (!(p.near_plane > 0.0f && p.far_plane > p.near_plane && std::isfinite(p.far_plane)))
        return fail(ctx, SSVP_EINVAL, "need 0 < near_plane < far_plane < inf");
    if (!std::isfinite(p.sigma_area)) return fail(ctx, SSVP_EINVAL, "sigma_area must be finite");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    Clip &c = ctx->clips[clip_id];
    if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    if (!c.has_cams) return fail(ctx, SSVP_ENOCAM, "clip %d has no cameras", clip_id);
    const int b = p.frame_begin, e = p.frame_end < 0 ? c.p.F : p.frame_end;
    if (b < 0 || e > c.p.F || b > e) return fail(ctx, SSVP_EINVAL, "frame range [%d, %d) outside the clip", b, e);
    const long long Wo = (long long)c.p.W * scale, Ho = (long long)c.p.H * scale;
    if (Wo > 65535 || Ho > 65535) return fail(ctx, SSVP_EINVAL, "output grid %lldx%lld too large", Wo, Ho);
    int x0 = p.crop_x, y0 = p.crop_y, w = p.crop_w, h = p.crop_h;
    if (w == 0 || h == 0) { x0 = 0; y0 = 0; w = (int)Wo; h = (int)Ho; }
    if (x0 < 0 || y0 < 0 || x0 + w > Wo || y0 + h > Ho)
        return fail(ctx, SSVP_EINVAL, "crop (%d, %d, %d, %d) outside the %lldx%lld output grid", x0, y0, w, h, Wo, Ho);
    const int n_out = e - b, T = p.half_window, ns = 2 * T + 1;
    if ((p.membership_out || p.pixel_stats_out) && n_out > 1)
        return fail(ctx, SSVP_EINVAL, "debug outputs need at most one output frame");
    if (n_out == 0) return SSVP_OK;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if ((rc = ensure_frame_values(ctx, c, true, p.mode == SSVP_MODE_DEBLUR)) != SSVP_OK) return rc;
    const size_t total = (size_t)n_out * ns;
    if (2 * total > ctx->geom_cap) {
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        if (ctx->geom) cudaFree(ctx->geom);
        ctx->geom = nullptr;
        ctx->geom_cap = 0;
        const size_t cap = std::max<size_t>(2 * total, 4096);
        CK(cudaMalloc(&ctx->geom, cap * sizeof(PairGeom)), "cudaMalloc (geometry)");
        ctx->geom_cap = cap;
    }
    ctx->host_geom.resize(2 * total);
    compose_tables_sr(c, b, n_out, T, p.sigma_f, scale, ctx->host_geom.data(), ctx->host_geom.data() + total);
    CK(cudaMemcpyAsync(ctx->geom, ctx->host_geom.data(), 2 * total * sizeof(PairGeom), cudaMemcpyHostToDevice, ctx->stream),
       "cudaMemcpyAsync (geometry)");
    CK(cudaMemsetAsync(ctx->stat_counts, 0, 2 * sizeof(unsigned long long), ctx->stream), "cudaMemsetAsync");
    CK(cudaMemsetAsync(ctx->stat_sumw, 0, sizeof(double), ctx->stream), "cudaMemsetAsync");
    GatherArgs a{};
    a.clip = c.p;
    a.geom = ctx->geom;
    a.geom_back = ctx->geom + total;
    a.frame_begin = b;
    a.n_out = n_out;
    a.n_slots = ns;
    a.T = T;
    a.x0 = x0; a.y0 = y0; a.cw = w; a.ch = h;
    a.k = 1;
    a.mode = p.mode;
    a.radius = p.radius;
    a.sigma_rgb = p.sigma_rgb;
    a.sigma_xyz = p.sigma_xyz;
    a.sigma_f = p.sigma_f;
    a.frustum_l = p.frustum_l;
    a.near_plane = p.near_plane;
    a.far_plane = p.far_plane;
    a.sr_scale = scale;
    a.sigma_area = p.sigma_area;
    a.sr_out = out;
    a.membership = (int32_t *)p.membership_out;
    a.pixel_stats = (int32_t *)p.pixel_stats_out;
    a.stat_counts = ctx->stat_counts;
    a.stat_sumw = ctx->stat_sumw;
    TraceScope ts(ctx, SSVP_TRACE_SUPERRES, ctx->stream);
    CK(ssvp::launch_frustum(a, ctx->stream), "super-resolution kernel");
    return SSVP_OK;
}

// the clip's mask plane (padded like depth, pads 0), allocated and cleared on first use
static int ensure_mask(ssvp_ctx *ctx, Clip &c) {
    if (c.p.mask) return SSVP_OK;
    const size_t bytes = (size_t)c.p.F * (size_t)c.p.fstride;
    CK(cudaMalloc(&c.p.mask, bytes), "cudaMalloc (mask)");
    CK(cudaMemsetAsync(c.p.mask, 0, bytes, ctx->stream), "cudaMemsetAsync (mask)");
    return SSVP_OK;
}

static int mask_clip(ssvp_ctx *ctx, int clip_id, Clip **out) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    Clip &c = ctx->clips[clip_id];
    if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    *out = &c;
    return SSVP_OK;
}

int ssvp_set_mask(ssvp_ctx *ctx, int clip_id, const uint8_t *mask, int mem_kind) {
    Clip *c = nullptr;
    int rc = mask_clip(ctx, clip_id, &c);
    if (rc != SSVP_OK) return rc;
    if (!mask) return fail(ctx, SSVP_EINVAL, "mask is NULL");
    if (mem_kind != SSVP_MEM_HOST && mem_kind != SSVP_MEM_DEVICE) return fail(ctx, SSVP_EINVAL, "bad mem_kind %d", mem_kind);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if ((rc = check_mem(ctx, mask, mem_kind, "mask")) != SSVP_OK) return rc;
    if ((rc = ensure_mask(ctx, *c)) != SSVP_OK) return rc;
    const Planes &p = c->p;
    for (int f = 0; f < p.F; ++f)
        CK(cudaMemcpy2DAsync(p.mask + (size_t)f * p.fstride + (size_t)ssvp::kPad * p.pitch + ssvp::kPad, (size_t)p.pitch,
                             mask + (size_t)f * p.W * p.H, (size_t)p.W, (size_t)p.W, (size_t)p.H,
                             mem_kind == SSVP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream),
           "cudaMemcpy2DAsync (mask)");
    return SSVP_OK;
}

int ssvp_mask_from_box(ssvp_ctx *ctx, int clip_id, const double *box) {
    Clip *c = nullptr;
    int rc = mask_clip(ctx, clip_id, &c);
    if (rc != SSVP_OK) return rc;
    if (!c->has_cams) return fail(ctx, SSVP_ENOCAM, "clip %d has no cameras", clip_id);
    if (!box) return fail(ctx, SSVP_EINVAL, "box is NULL");
    if ((rc = check_mem(ctx, box, SSVP_MEM_HOST, "box")) != SSVP_OK) return rc;
    if (!finite_all(box, 6)) return fail(ctx, SSVP_EINVAL, "box must hold 6 finite values");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if ((rc = ensure_mask(ctx, *c)) != SSVP_OK) return rc;
    const int F = c->p.F;
    std::vector<double> cam((size_t)F * 21);
    for (int f = 0; f < F; ++f) {
        const double *K = &c->K[9 * (size_t)f], *w = &c->w2c[12 * (size_t)f];
        double *o = &cam[21 * (size_t)f];
        // K^-1 of an upper-triangular, zero-skew K; then R and t of the pose
        const double Ki[9] = {1.0 / K[0], 0.0, -K[2] / K[0], 0.0, 1.0 / K[4], -K[5] / K[4], 0.0, 0.0, 1.0};
        for (int i = 0; i < 9; ++i) o[i] = Ki[i];
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) o[9 + 3 * r + k] = w[4 * r + k];
            o[18 + r] = w[4 * r + 3];
        }
    }
    // the camera table goes to a device buffer the context keeps: the next call's copy into it is
    // queued after this call's kernel on the same stream (a pageable source is staged before the
    // copy call returns)
    if (ctx->mask_cam_cap < cam.size()) {
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        if (ctx->mask_cam) cudaFree(ctx->mask_cam);
        ctx->mask_cam = nullptr;
        ctx->mask_cam_cap = 0;
        CK(cudaMalloc(&ctx->mask_cam, cam.size() * sizeof(double)), "cudaMalloc (cameras)");
        ctx->mask_cam_cap = cam.size();
    }
    CK(cudaMemcpyAsync(ctx->mask_cam, cam.data(), cam.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
       "cudaMemcpyAsync (cameras)");
    TraceScope ts(ctx, SSVP_TRACE_MASK, ctx->stream);
    CK(ssvp::launch_mask_box(c->p, ctx->mask_cam, box, ctx->stream), "mask from box");
    return SSVP_OK;
}

int ssvp_read_mask(ssvp_ctx *ctx, int clip_id, uint8_t *out) {
    Clip *c = nullptr;
    int rc = mask_clip(ctx, clip_id, &c);
    if (rc != SSVP_OK) return rc;
    if (!out) return fail(ctx, SSVP_EINVAL, "out is NULL");
    if ((rc = check_mem(ctx, out, SSVP_MEM_HOST, "out")) != SSVP_OK) return rc;
    if (!c->p.mask) return fail(ctx, SSVP_EINVAL, "clip %d has no mask", clip_id);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const Planes &p = c->p;
    for (int f = 0; f < p.F; ++f)
        CK(cudaMemcpy2DAsync(out + (size_t)f * p.W * p.H, (size_t)p.W,
                             p.mask + (size_t)f * p.fstride + (size_t)ssvp::kPad * p.pitch + ssvp::kPad, (size_t)p.pitch,
                             (size_t)p.W, (size_t)p.H, cudaMemcpyDeviceToHost, ctx->stream),
           "cudaMemcpy2DAsync (mask)");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    return SSVP_OK;
}

int ssvp_set_shutter(ssvp_ctx *ctx, const float *xi, int half_window) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (!xi) return fail(ctx, SSVP_EINVAL, "xi is NULL");
    if (int rc = check_mem(ctx, xi, SSVP_MEM_HOST, "xi"); rc != SSVP_OK) return rc;
    if (half_window < 0 || half_window > SSVP_MAX_HALF_WINDOW)
        return fail(ctx, SSVP_EINVAL, "half_window=%d must be in [0, 127]", half_window);
    const int n = 2 * half_window + 1;
    for (int j = 0; j < n; ++j)
        if (!(std::isfinite(xi[j]) && xi[j] >= 0.0f)) return fail(ctx, SSVP_EINVAL, "xi[%d] must be finite and >= 0", j);
    ctx->shutter.assign(xi, xi + n);
    return SSVP_OK;
}

int ssvp_frame_sharpness(ssvp_ctx *ctx, int clip_id, double *out) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    Clip &c = ctx->clips[clip_id];
    if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    if (!out) return fail(ctx, SSVP_EINVAL, "out is NULL");
    int rc = check_mem(ctx, out, SSVP_MEM_HOST, "out");
    if (rc != SSVP_OK) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    rc = ensure_frame_values(ctx, c, false, true);
    if (rc != SSVP_OK) return rc;
    CK(cudaMemcpyAsync(out, c.p.grad_sum, sizeof(double) * (size_t)c.p.F, cudaMemcpyDeviceToHost, ctx->stream),
       "cudaMemcpyAsync (gradient sums)");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    return SSVP_OK;
}

int ssvp_read_output(ssvp_ctx *ctx, int clip_id, int frame_begin, int frame_end, float *dst, int mem_kind) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    Clip &c = ctx->clips[clip_id];
    if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    if (!dst) return fail(ctx, SSVP_EINVAL, "dst is NULL");
    if (frame_begin < 0 || frame_end > c.p.F || frame_begin > frame_end)
        return fail(ctx, SSVP_EINVAL, "frame range [%d, %d) outside the clip", frame_begin, frame_end);
    if (mem_kind != SSVP_MEM_HOST && mem_kind != SSVP_MEM_DEVICE) return fail(ctx, SSVP_EINVAL, "bad mem_kind %d", mem_kind);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc = check_mem(ctx, dst, mem_kind, "dst");
    if (rc != SSVP_OK) return rc;
    const size_t per = (size_t)c.p.W * c.p.H * 3;
    const size_t bytes = per * (size_t)(frame_end - frame_begin) * sizeof(float);
    if (bytes) {
        CK(cudaMemcpyAsync(dst, c.p.out + per * (size_t)frame_begin, bytes,
                           mem_kind == SSVP_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->stream),
           "cudaMemcpyAsync (output)");
    }
    if (mem_kind == SSVP_MEM_HOST) CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    return SSVP_OK;
}

int ssvp_output_device_ptr(ssvp_ctx *ctx, int clip_id, void **dev_ptr) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    if (!ctx->clips[clip_id].loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    if (!dev_ptr) return fail(ctx, SSVP_EINVAL, "dev_ptr is NULL");
    Clip &c = ctx->clips[clip_id];
    c.mark_out(0, c.p.F);  // the caller may write the buffer: a reload clears all of it
    *dev_ptr = c.p.out;
    return SSVP_OK;
}

int ssvp_read_stats(ssvp_ctx *ctx, unsigned long long *examined, unsigned long long *accepted, double *sum_w) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    unsigned long long cnt[2];
    double sw;
    CK(cudaMemcpyAsync(cnt, ctx->stat_counts, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->stream), "cudaMemcpyAsync");
    CK(cudaMemcpyAsync(&sw, ctx->stat_sumw, sizeof(sw), cudaMemcpyDeviceToHost, ctx->stream), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    if (examined) *examined = cnt[0];
    if (accepted) *accepted = cnt[1];
    if (sum_w) *sum_w = sw;
    return SSVP_OK;
}

int ssvp_clip_median_depth(ssvp_ctx *ctx, int clip_id, float *median) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    if (!ctx->clips[clip_id].loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    if (!median) return fail(ctx, SSVP_EINVAL, "median is NULL");
    if (int rc = check_mem(ctx, median, SSVP_MEM_HOST, "median"); rc != SSVP_OK) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(median, ctx->clips[clip_id].p.median, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    return SSVP_OK;
}

// Kernel arguments of a batched launch: the clip table goes by value into the parameter space
ssvp::BatchArgs batch_args(const BatchSetup &bs, int n_clips, int frame_chunk, unsigned long long *counter) {
    ssvp::BatchArgs b{};
    b.n_clips = n_clips;
    b.frame_chunk = frame_chunk;
    b.n_items = bs.n_items;
    b.counter = counter;
    for (int i = 0; i < n_clips && i < ssvp::kMaxBatchClips; ++i) b.clip[i] = bs.clips[i];
    return b;
}

int ssvp_autotune(ssvp_ctx *ctx, const ssvp_params *params, const int *clip_ids, int n_clips, ssvp_plan_config *best) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    int cfmt = 0;
    int rc = batch_check(ctx, params, clip_ids, n_clips, cfmt);
    if (rc != SSVP_OK) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    BatchSetup bs;
    batch_tables(ctx, *params, clip_ids, n_clips, 8, bs);
    for (int i = 0; i < n_clips; ++i)  // the trial launches write these output frames
        ctx->clips[clip_ids[i]].mark_out(bs.clips[i].frame_begin, bs.clips[i].frame_begin + bs.clips[i].n_out);
    PairGeom *d_geom = nullptr;
    unsigned long long *d_counter = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaSuccess;
    ssvp_plan_config winner{8, 1};
    float best_ms = 3.0e38f;
    const ssvp_plan_config cands[] = {{4, 1}, {4, 2}, {4, 4}, {4, 8}, {8, 1}, {8, 2}, {8, 4}, {8, 8}};
    GatherArgs a = batch_gather_args(ctx, *params);
    do {
        if ((e = cudaMalloc(&d_geom, bs.geom.size() * sizeof(PairGeom))) != cudaSuccess) break;
        if ((e = cudaMalloc(&d_counter, sizeof(unsigned long long))) != cudaSuccess) break;
        if ((e = cudaMemcpy(d_geom, bs.geom.data(), bs.geom.size() * sizeof(PairGeom), cudaMemcpyHostToDevice)) != cudaSuccess) break;
        if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) break;
        for (const auto &cfg : cands) {
            batch_items(bs, cfg, d_geom);
            const int grid = ssvp::batch_grid(params->k, cfg.tile_rows, cfmt, bs.ns);
            const ssvp::BatchArgs b = batch_args(bs, n_clips, cfg.frame_chunk, d_counter);
            float ms = 0.0f;
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                if (rep == 1 && (e = cudaEventRecord(e0, ctx->stream)) != cudaSuccess) break;
                if ((e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), ctx->stream)) != cudaSuccess) break;
                e = ssvp::launch_batch(a, b, cfg.tile_rows, cfmt, grid, ctx->stream);
            }
            if (e != cudaSuccess) break;
            if ((e = cudaEventRecord(e1, ctx->stream)) != cudaSuccess) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
            if (ms < best_ms) { best_ms = ms; winner = cfg; }
        }
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(ctx->stream);
    if (d_geom) cudaFree(d_geom);
    if (d_counter) cudaFree(d_counter);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
    bool stored = false;
    for (auto &t : ctx->tuned)
        if (t.k == params->k && t.T == params->half_window && t.mode == params->mode && t.cfmt == cfmt) {
            t.cfg = winner;
            stored = true;
        }
    if (!stored) ctx->tuned.push_back({params->k, params->half_window, params->mode, cfmt, winner});
    if (best) *best = winner;
    return SSVP_OK;
}

void ssvp_plan_destroy(ssvp_plan *plan) {
    if (!plan) return;
    if (plan->ctx) {
        cudaSetDevice(plan->ctx->device);
        cudaStreamSynchronize(plan->ctx->stream);
    }
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
    if (plan->d_geom) cudaFree(plan->d_geom);
    if (plan->d_counter) cudaFree(plan->d_counter);
    delete plan;
}

int ssvp_plan_create(ssvp_ctx *ctx, const ssvp_params *params, const int *clip_ids, int n_clips,
                     const ssvp_plan_config *config, ssvp_plan **out) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (!out) return fail(ctx, SSVP_EINVAL, "out is NULL");
    *out = nullptr;
    int cfmt = 0;
    int rc = batch_check(ctx, params, clip_ids, n_clips, cfmt);
    if (rc != SSVP_OK) return rc;
    ssvp_plan_config cfg{8, 1};
    if (config) cfg = *config;
    else if (const ssvp_plan_config *t = find_tuned(ctx, *params, cfmt)) cfg = *t;
    if (!valid_config(cfg)) return fail(ctx, SSVP_EINVAL, "plan shape: tile_rows must be 4 or 8, frame_chunk 1..16");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    ssvp_plan *plan = new (std::nothrow) ssvp_plan();
    if (!plan) return fail(ctx, SSVP_ENOMEM, "host allocation failed");
    plan->ctx = ctx;
    plan->params = *params;
    plan->clip_ids.assign(clip_ids, clip_ids + n_clips);
    for (int i = 0; i < n_clips; ++i) {
        plan->generations.push_back(ctx->clips[clip_ids[i]].generation);
        plan->planes.push_back(ssvp_plan::frozen(ctx->clips[clip_ids[i]].p));
    }
    plan->cfg = cfg;
    BatchSetup bs;
    batch_tables(ctx, *params, clip_ids, n_clips, 1 << 30, bs);
    cudaError_t e = cudaSuccess;
    const char *what = "plan";
    do {
        what = "cudaMalloc (plan)";
        if ((e = cudaMalloc(&plan->d_geom, bs.geom.size() * sizeof(PairGeom))) != cudaSuccess) break;
        if ((e = cudaMalloc(&plan->d_counter, sizeof(unsigned long long))) != cudaSuccess) break;
        batch_items(bs, cfg, plan->d_geom);
        plan->n_items = bs.n_items;
        what = "cudaMemcpy (plan)";
        if ((e = cudaMemcpy(plan->d_geom, bs.geom.data(), bs.geom.size() * sizeof(PairGeom), cudaMemcpyHostToDevice)) != cudaSuccess) break;
        plan->grid = ssvp::batch_grid(params->k, cfg.tile_rows, cfmt, bs.ns);
        what = "occupancy";
        if (plan->grid <= 0) { e = cudaErrorInvalidConfiguration; break; }
        what = "graph capture";
        if ((e = cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        GatherArgs a = batch_gather_args(ctx, *params);
        const ssvp::BatchArgs b = batch_args(bs, n_clips, cfg.frame_chunk, plan->d_counter);
        cudaError_t e1 = cudaMemsetAsync(plan->d_counter, 0, sizeof(unsigned long long), plan->cap_stream);
        cudaError_t e2 = cudaMemsetAsync(ctx->stat_counts, 0, 2 * sizeof(unsigned long long), plan->cap_stream);
        cudaError_t e3 = cudaMemsetAsync(ctx->stat_sumw, 0, sizeof(double), plan->cap_stream);
        cudaError_t e4 = ssvp::launch_batch(a, b, cfg.tile_rows, cfmt, plan->grid, plan->cap_stream);
        e = cudaStreamEndCapture(plan->cap_stream, &plan->graph);
        if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3 != cudaSuccess ? e3 : e4;
        if (e != cudaSuccess) break;
        if ((e = cudaGraphInstantiate(&plan->exec, plan->graph, 0)) != cudaSuccess) break;
    } while (0);
    if (e != cudaSuccess) {
        int code = cuda_fail(ctx, e, what);
        ssvp_plan_destroy(plan);
        return code;
    }
    *out = plan;
    return SSVP_OK;
}

int ssvp_plan_launch(ssvp_plan *plan) {
    if (!plan) return fail(nullptr, SSVP_EINVAL, "plan is NULL");
    ssvp_ctx *ctx = plan->ctx;
    for (size_t i = 0; i < plan->clip_ids.size(); ++i) {
        const Clip &c = ctx->clips[plan->clip_ids[i]];
        if (!c.loaded || c.generation != plan->generations[i])
            return fail(ctx, SSVP_ENOCLIP, "clip %d was reloaded or unloaded after the plan was made", plan->clip_ids[i]);
    }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    for (int id : plan->clip_ids) {
        Clip &c = ctx->clips[id];
        c.mark_out(plan->params.frame_begin, plan->params.frame_end < 0 ? c.p.F : plan->params.frame_end);
    }
    TraceScope ts(ctx, SSVP_TRACE_BATCH, ctx->stream);
    CK(cudaGraphLaunch(plan->exec, ctx->stream), "cudaGraphLaunch");
    return SSVP_OK;
}

int ssvp_plan_update(ssvp_plan *plan) {
    if (!plan) return fail(nullptr, SSVP_EINVAL, "plan is NULL");
    ssvp_ctx *ctx = plan->ctx;
    const int n = (int)plan->clip_ids.size();
    for (int i = 0; i < n; ++i) {
        const int id = plan->clip_ids[i];
        const Clip &c = ctx->clips[id];
        if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", id);
        if (!c.has_cams) return fail(ctx, SSVP_ENOCAM, "clip %d has no cameras", id);
        // the captured graph holds the clip's plane pointers and strides: a reload with another
        // shape or format, or an append (which swaps windows), changed them
        if (!(ssvp_plan::frozen(c.p) == plan->planes[i]))
            return fail(ctx, SSVP_EINVAL, "clip %d's planes changed since the plan was made (another shape, format or "
                                          "an append): make a new plan", id);
    }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    BatchSetup bs;
    batch_tables(ctx, plan->params, plan->clip_ids.data(), n, 1 << 30, bs);
    // queued after the plan's earlier launches on the same stream; a pageable source is staged
    // before the call returns
    CK(cudaMemcpyAsync(plan->d_geom, bs.geom.data(), bs.geom.size() * sizeof(PairGeom), cudaMemcpyHostToDevice,
                       ctx->stream),
       "cudaMemcpyAsync (plan geometry)");
    for (int i = 0; i < n; ++i) plan->generations[i] = ctx->clips[plan->clip_ids[i]].generation;
    return SSVP_OK;
}

int ssvp_plan_get_config(const ssvp_plan *plan, ssvp_plan_config *config, long long *n_items, int *grid) {
    if (!plan) return fail(nullptr, SSVP_EINVAL, "plan is NULL");
    if (config) *config = plan->cfg;
    if (n_items) *n_items = plan->n_items;
    if (grid) *grid = plan->grid;
    return SSVP_OK;
}

int ssvp_set_mlp(ssvp_ctx *ctx, const float *W1, const float *b1, const float *W2, const float *b2) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (!W1 || !b1 || !W2 || !b2) return fail(ctx, SSVP_EINVAL, "weights must not be NULL");
    int rc;
    if ((rc = check_mem(ctx, W1, SSVP_MEM_HOST, "W1")) != SSVP_OK || (rc = check_mem(ctx, b1, SSVP_MEM_HOST, "b1")) != SSVP_OK ||
        (rc = check_mem(ctx, W2, SSVP_MEM_HOST, "W2")) != SSVP_OK || (rc = check_mem(ctx, b2, SSVP_MEM_HOST, "b2")) != SSVP_OK)
        return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    rc = mlp_alloc(ctx);
    if (rc != SSVP_OK) return rc;
    std::vector<float> flat(ssvp::kMlpParams);
    std::memcpy(flat.data(), W1, 1024 * sizeof(float));
    std::memcpy(flat.data() + ssvp::kMlpB1, b1, 64 * sizeof(float));
    std::memcpy(flat.data() + ssvp::kMlpW2, W2, 128 * sizeof(float));
    std::memcpy(flat.data() + ssvp::kMlpB2, b2, 2 * sizeof(float));
    for (float x : flat)
        if (!std::isfinite(x)) return fail(ctx, SSVP_EINVAL, "weights must be finite");
    CK(cudaMemcpy(ctx->mlp.master, flat.data(), flat.size() * sizeof(float), cudaMemcpyHostToDevice), "cudaMemcpy (mlp)");
    CK(cudaMemsetAsync(ctx->mlp.m, 0, 2 * ssvp::kMlpParams * sizeof(float), ctx->stream), "cudaMemsetAsync");
    CK(ssvp::launch_mlp_refresh(ctx->mlp, ctx->stream), "mlp refresh");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    ctx->mlp_set = true;
    ctx->mlp_step = 0;
    return SSVP_OK;
}

int ssvp_get_mlp(ssvp_ctx *ctx, float *W1, float *b1, float *W2, float *b2) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (!ctx->mlp_set) return fail(ctx, SSVP_EINVAL, "no network has been set or trained");
    {
        const float *outs[4] = {W1, b1, W2, b2};
        const char *names[4] = {"W1", "b1", "W2", "b2"};
        for (int i = 0; i < 4; ++i)
            if (outs[i])
                if (int rc = check_mem(ctx, outs[i], SSVP_MEM_HOST, names[i]); rc != SSVP_OK) return rc;
    }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::vector<float> flat(ssvp::kMlpParams);
    CK(cudaMemcpyAsync(flat.data(), ctx->mlp.master, flat.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream),
       "cudaMemcpyAsync (mlp)");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    if (W1) std::memcpy(W1, flat.data(), 1024 * sizeof(float));
    if (b1) std::memcpy(b1, flat.data() + ssvp::kMlpB1, 64 * sizeof(float));
    if (W2) std::memcpy(W2, flat.data() + ssvp::kMlpW2, 128 * sizeof(float));
    if (b2) std::memcpy(b2, flat.data() + ssvp::kMlpB2, 2 * sizeof(float));
    return SSVP_OK;
}

int ssvp_learned_samples(ssvp_ctx *ctx, const ssvp_params *params, int clip_id, unsigned short *feat, float *col,
                         int32_t *nsamp, float *plain) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    int rc = check_params(ctx, params);
    if (rc != SSVP_OK) return rc;
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    Clip &c = ctx->clips[clip_id];
    if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    if (!c.has_cams) return fail(ctx, SSVP_ENOCAM, "clip %d has no cameras", clip_id);
    if (!feat || !col || !nsamp || !plain) return fail(ctx, SSVP_EINVAL, "output buffers must not be NULL");
    if ((rc = check_mem(ctx, feat, SSVP_MEM_DEVICE, "feat")) != SSVP_OK ||
        (rc = check_mem(ctx, col, SSVP_MEM_DEVICE, "col")) != SSVP_OK ||
        (rc = check_mem(ctx, nsamp, SSVP_MEM_DEVICE, "nsamp")) != SSVP_OK ||
        (rc = check_mem(ctx, plain, SSVP_MEM_DEVICE, "plain")) != SSVP_OK)
        return rc;
    const ssvp_params &p = *params;
    if (p.frame_begin < 0 || p.frame_begin >= c.p.F) return fail(ctx, SSVP_EINVAL, "frame %d outside the clip", p.frame_begin);
    if (p.k > 7) return fail(ctx, SSVP_EINVAL, "the learned filter supports k <= 7");
    int x0 = p.crop_x, y0 = p.crop_y, w = p.crop_w, h = p.crop_h;
    if (w == 0 || h == 0) { x0 = 0; y0 = 0; w = c.p.W; h = c.p.H; }
    if (x0 < 0 || y0 < 0 || x0 + w > c.p.W || y0 + h > c.p.H) return fail(ctx, SSVP_EINVAL, "crop outside the clip");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if ((rc = learned_scratch(ctx, (size_t)w * h)) != SSVP_OK) return rc;
    if ((rc = extract_samples(ctx, p, clip_id, p.frame_begin, x0, y0, w, h)) != SSVP_OK) return rc;
    // the kernels keep the sets compact; this caller gets the full feature layout
    CK(ssvp::launch_expand_sets(ctx->l_sets, feat, col, nsamp, plain, (long long)w * h, ctx->stream), "sample set expansion kernel");
    return SSVP_OK;
}

int ssvp_mlp_grad(ssvp_ctx *ctx, const ssvp_params *params, int clip_id, const int32_t *pixels, int n_pixels,
                  const float *clean, float *grad_out) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    int rc = check_params(ctx, params);
    if (rc != SSVP_OK) return rc;
    if (!ctx->mlp_set) return fail(ctx, SSVP_EINVAL, "no network has been set or trained");
    if (clip_id < 0 || clip_id >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id %d out of range", clip_id);
    Clip &c = ctx->clips[clip_id];
    if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_id);
    if (!c.has_cams) return fail(ctx, SSVP_ENOCAM, "clip %d has no cameras", clip_id);
    if (!pixels || n_pixels < 1 || !clean || !grad_out) return fail(ctx, SSVP_EINVAL, "bad pixel list or buffers");
    if ((rc = check_mem(ctx, pixels, SSVP_MEM_HOST, "pixels")) != SSVP_OK ||
        (rc = check_mem(ctx, clean, SSVP_MEM_DEVICE, "clean")) != SSVP_OK ||
        (rc = check_mem(ctx, grad_out, SSVP_MEM_HOST, "grad_out")) != SSVP_OK)
        return rc;
    if (params->k > 7) return fail(ctx, SSVP_EINVAL, "the learned filter supports k <= 7");
    const int O = params->frame_begin;
    if (O < 0 || O >= c.p.F) return fail(ctx, SSVP_EINVAL, "frame %d outside the clip", O);
    const size_t npx = (size_t)c.p.W * c.p.H;
    for (int i = 0; i < n_pixels; ++i)
        if (pixels[i] < 0 || (size_t)pixels[i] >= npx) return fail(ctx, SSVP_EINVAL, "pixel index out of range");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if ((rc = learned_scratch(ctx, npx)) != SSVP_OK) return rc;
    if ((size_t)n_pixels > ctx->l_batch_cap) {
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        if (ctx->l_batch) cudaFree(ctx->l_batch);
        ctx->l_batch = nullptr;
        CK(cudaMalloc(&ctx->l_batch, n_pixels * sizeof(int32_t)), "cudaMalloc (batch)");
        ctx->l_batch_cap = n_pixels;
    }
    if ((rc = extract_samples(ctx, *params, clip_id, O, 0, 0, c.p.W, c.p.H)) != SSVP_OK)
        return rc;
    CK(cudaMemcpyAsync(ctx->l_batch, pixels, n_pixels * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream), "cudaMemcpyAsync");
    CK(cudaMemsetAsync(ctx->mlp.grad, 0, (ssvp::kMlpParams + 1) * sizeof(float), ctx->stream), "cudaMemsetAsync");
    ssvp::MlpArgs m{};
    m.w = mlp_weights(ctx);
    m.sets = ctx->l_sets;
    m.n_px = (long long)npx;
    m.O = O; m.W = c.p.W; m.H = c.p.H; m.x0 = 0; m.y0 = 0; m.cw = c.p.W;
    m.batch = ctx->l_batch;
    m.n_batch = n_pixels;
    m.clean = clean;
    m.bce_w = 0.1f;
    m.grad = ctx->mlp.grad;
    {
        TraceScope ts(ctx, SSVP_TRACE_TRAIN, ctx->stream);
        CK(ssvp::launch_mlp_train_tc(m, ctx->d_kerr, ctx->stream), "mlp train kernel");
    }
    CK(cudaMemcpyAsync(grad_out, ctx->mlp.grad, (ssvp::kMlpParams + 1) * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream),
       "cudaMemcpyAsync");
    return ssvp_sync(ctx);  // also reports a timed-out tensor-core wait
}

int ssvp_train(ssvp_ctx *ctx, const ssvp_params *params, const int *clip_ids, const float *const *clean, int n_clips,
               const ssvp_train_config *cfg, float *loss_out) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    int rc = check_params(ctx, params);
    if (rc != SSVP_OK) return rc;
    if (!cfg || cfg->steps < 0 || cfg->batch_pixels < 1 || !(cfg->lr > 0.0f) || !(cfg->bce_weight >= 0.0f))
        return fail(ctx, SSVP_EINVAL, "bad training configuration");
    if (!clip_ids || !clean || n_clips < 1) return fail(ctx, SSVP_EINVAL, "bad clip list");
    if (params->k > 7) return fail(ctx, SSVP_EINVAL, "the learned filter supports k <= 7");
    if (loss_out && (rc = check_mem(ctx, loss_out, SSVP_MEM_HOST, "loss_out")) != SSVP_OK) return rc;
    size_t max_px = 0;
    for (int i = 0; i < n_clips; ++i) {
        if (clip_ids[i] < 0 || clip_ids[i] >= SSVP_MAX_CLIPS) return fail(ctx, SSVP_EINVAL, "clip_id out of range");
        const Clip &c = ctx->clips[clip_ids[i]];
        if (!c.loaded) return fail(ctx, SSVP_ENOCLIP, "clip %d is not loaded", clip_ids[i]);
        if (!c.has_cams) return fail(ctx, SSVP_ENOCAM, "clip %d has no cameras", clip_ids[i]);
        if (!clean[i]) return fail(ctx, SSVP_EINVAL, "clean target of clip %d is NULL", clip_ids[i]);
        if ((rc = check_mem(ctx, clean[i], SSVP_MEM_DEVICE, "clean target")) != SSVP_OK) return rc;
        max_px = std::max(max_px, (size_t)c.p.W * c.p.H);
    }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if ((rc = mlp_alloc(ctx)) != SSVP_OK) return rc;
    Rng rng{cfg->seed};
    if (cfg->init || !ctx->mlp_set) {
        // He-normal W1 (15 non-zero inputs), W2; zero biases
        std::vector<float> W1(1024), b1(64, 0.0f), W2(128), b2(2, 0.0f);
        for (auto &x : W1) x = (float)(rng.normal() * std::sqrt(2.0 / 15.0));
        for (auto &x : W2) x = (float)(rng.normal() * std::sqrt(2.0 / 64.0));
        if ((rc = ssvp_set_mlp(ctx, W1.data(), b1.data(), W2.data(), b2.data())) != SSVP_OK) return rc;
    }
    if ((rc = learned_scratch(ctx, max_px)) != SSVP_OK) return rc;
    const size_t nb = (size_t)cfg->batch_pixels;
    if (nb > ctx->l_batch_cap) {
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        if (ctx->l_batch) cudaFree(ctx->l_batch);
        ctx->l_batch = nullptr;
        CK(cudaMalloc(&ctx->l_batch, nb * sizeof(int32_t)), "cudaMalloc (batch)");
        ctx->l_batch_cap = nb;
    }
    if ((size_t)cfg->steps > ctx->l_loss_cap) {
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        if (ctx->l_loss) cudaFree(ctx->l_loss);
        ctx->l_loss = nullptr;
        CK(cudaMalloc(&ctx->l_loss, std::max(cfg->steps, 1) * sizeof(float)), "cudaMalloc (loss)");
        ctx->l_loss_cap = std::max(cfg->steps, 1);
    }
    std::vector<int32_t> batch(nb);
    for (int step = 0; step < cfg->steps; ++step) {
        const int ci = (int)(rng.next() % (uint64_t)n_clips);
        const Clip &c = ctx->clips[clip_ids[ci]];
        const int O = (int)(rng.next() % (uint64_t)c.p.F);
        const uint64_t npx = (uint64_t)c.p.W * c.p.H;
        for (auto &b : batch) b = (int32_t)(rng.next() % npx);
        if ((rc = extract_samples(ctx, *params, clip_ids[ci], O, 0, 0, c.p.W, c.p.H)) != SSVP_OK)
            return rc;
        // pageable source: the copy is staged before the call returns, so batch may be rewritten
        CK(cudaMemcpyAsync(ctx->l_batch, batch.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream),
           "cudaMemcpyAsync");
        CK(cudaMemsetAsync(ctx->mlp.grad, 0, (ssvp::kMlpParams + 1) * sizeof(float), ctx->stream), "cudaMemsetAsync");
        ssvp::MlpArgs m{};
        m.w = mlp_weights(ctx);
        m.sets = ctx->l_sets;
        m.n_px = (long long)npx;
        m.O = O; m.W = c.p.W; m.H = c.p.H; m.x0 = 0; m.y0 = 0; m.cw = c.p.W;
        m.batch = ctx->l_batch;
        m.n_batch = (long long)nb;
        m.clean = clean[ci];
        m.bce_w = cfg->bce_weight;
        m.grad = ctx->mlp.grad;
        {
            TraceScope ts(ctx, SSVP_TRACE_TRAIN, ctx->stream);
            CK(ssvp::launch_mlp_train_tc(m, ctx->d_kerr, ctx->stream), "mlp train kernel");
        }
        {
            TraceScope ts(ctx, SSVP_TRACE_ADAM, ctx->stream);
            CK(ssvp::launch_adam(ctx->mlp, cfg->lr, ++ctx->mlp_step, ctx->stream), "adam kernel");
        }
        CK(cudaMemcpyAsync(ctx->l_loss + step, ctx->mlp.grad + ssvp::kMlpParams, sizeof(float), cudaMemcpyDeviceToDevice,
                           ctx->stream), "cudaMemcpyAsync");
    }
    if (loss_out && cfg->steps > 0)
        CK(cudaMemcpyAsync(loss_out, ctx->l_loss, cfg->steps * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream),
           "cudaMemcpyAsync");
    return ssvp_sync(ctx);  // also reports a timed-out tensor-core wait
}

int ssvp_trace_enable(ssvp_ctx *ctx, int on) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    ctx->trace_on = on != 0;
    return SSVP_OK;
}

int ssvp_trace_read(ssvp_ctx *ctx, int max_kinds, int *kind, int *launches, double *ms, int *n_kinds) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    if (max_kinds < 0) return fail(ctx, SSVP_EINVAL, "max_kinds %d < 0", max_kinds);
    if (n_kinds) *n_kinds = 0;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int cnt[SSVP_TRACE_KINDS] = {};
    double tot[SSVP_TRACE_KINDS] = {};
    cudaError_t err = cudaSuccess;
    for (auto &r : ctx->trace_pending) {
        float t = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e == cudaSuccess) {
            ++cnt[r.kind];
            tot[r.kind] += t;
        } else if (err == cudaSuccess) {
            err = e;
        }
        ctx->trace_free.push_back(r.a);
        ctx->trace_free.push_back(r.b);
    }
    ctx->trace_pending.clear();
    if (err != cudaSuccess) return cuda_fail(ctx, err, "trace events");
    int w = 0;
    for (int k = 0; k < SSVP_TRACE_KINDS && w < max_kinds; ++k) {
        if (!cnt[k]) continue;
        if (kind) kind[w] = k;
        if (launches) launches[w] = cnt[k];
        if (ms) ms[w] = tot[k];
        ++w;
    }
    if (n_kinds) *n_kinds = w;
    return SSVP_OK;
}

const char *ssvp_trace_kind_name(int kind) {
    static const char *const names[SSVP_TRACE_KINDS] = {"gather", "aperture", "frustum", "superres", "extract", "infer",
                                                        "train", "adam", "batch", "load", "mask"};
    return kind >= 0 && kind < SSVP_TRACE_KINDS ? names[kind] : "";
}

int ssvp_sync(ssvp_ctx *ctx) {
    if (!ctx) return fail(nullptr, SSVP_EINVAL, "ctx is NULL");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    CK(cudaGetLastError(), "pending CUDA error");
    int kerr = 0;
    CK(cudaMemcpy(&kerr, ctx->d_kerr, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy (kernel error word)");
    if (kerr) {
        CK(cudaMemset(ctx->d_kerr, 0, sizeof(int)), "cudaMemset (kernel error word)");
        if (kerr & 1) return fail(ctx, SSVP_ETIMEOUT, "a tensor-core completion wait of the learned filter timed out");
        return fail(ctx, SSVP_ETIMEOUT, "a tensor-copy wait of the staged window gather timed out");
    }
    return SSVP_OK;
}

}  // extern "C"
