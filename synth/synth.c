/*
 * synth.c - seeded procedural scene generator for test and benchmark inputs.
 *
 * Renders clips of a static Lambertian scene (infinite planes, rectangles and oriented boxes
 * with value-noise or constant albedo) seen by a moving pinhole camera, and applies the
 * workloads' noise model: multiplicative depth noise and additive Gaussian image noise.
 * It casts primary rays only.  It holds none of the gather-and-filter arithmetic and is
 * shared, as an input source, by the CPU oracle and the CUDA path alike.
 *
 * Conventions
 *   camera coordinates: x right, y down, z forward; world->camera x_c = R X_w + t
 *   pixel (u, v) with integer coordinates is the pixel centre
 *   K = [[fx, s, cx], [0, fy, cy], [0, 0, 1]] (upper triangular)
 *   depth = camera-space z of the first hit
 *
 * Random numbers: splitmix64 keyed by (seed, stream, frame, index), Box-Muller for normals.
 * Built with -ffp-contract=off so results do not depend on FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define SYNTH_PLANE 0
#define SYNTH_RECT 1
#define SYNTH_BOX 2

typedef struct {
    int32_t kind;       /* SYNTH_PLANE, SYNTH_RECT or SYNTH_BOX */
    int32_t textured;   /* 1: value-noise albedo, 0: constant albedo */
    double c[3];        /* point on plane / rectangle centre / box centre (world) */
    double ax[9];       /* rows: U, V, N (plane, rect; N faces the camera side) or box axes */
    double half[3];     /* rect half extents along U, V; box half extents along its axes */
    double albedo[3];   /* constant albedo (also used as tint weight when textured) */
    double tex_freq;    /* value-noise lattice cells per scene unit */
    uint64_t tex_seed;  /* per-object texture seed */
} synth_object;

/* ---------------------------------------------------------------- random numbers */

static uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t key4(uint64_t seed, uint64_t stream, uint64_t frame, uint64_t index) {
    uint64_t h = mix64(seed);
    h = mix64(h ^ stream);
    h = mix64(h ^ frame);
    return mix64(h ^ index);
}

static double u01(uint64_t h) { return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

/* standard normal from one key (Box-Muller, cosine branch) */
static double normal_key(uint64_t k) {
    double a = u01(k);
    double b = u01(mix64(k ^ 0xD1B54A32D192ED03ULL));
    return sqrt(-2.0 * log(a)) * cos(6.283185307179586 * b);
}

double synth_normal(uint64_t seed, uint64_t stream, uint64_t frame, uint64_t index) {
    return normal_key(key4(seed, stream, frame, index));
}

/* ---------------------------------------------------------------- value noise */

static double lattice(uint64_t s, int64_t ix, int64_t iy) {
    uint64_t h = mix64(s ^ mix64((uint64_t)ix * 0x9E3779B97F4A7C15ULL) ^
                       mix64((uint64_t)iy * 0xC2B2AE3D27D4EB4FULL + 0x165667B19E3779F9ULL));
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

static double smooth(double t) { return t * t * (3.0 - 2.0 * t); }

static double vnoise(uint64_t s, double x, double y) {
    double fx = floor(x), fy = floor(y);
    int64_t ix = (int64_t)fx, iy = (int64_t)fy;
    double tx = smooth(x - fx), ty = smooth(y - fy);
    double a = lattice(s, ix, iy), b = lattice(s, ix + 1, iy);
    double c = lattice(s, ix, iy + 1), d = lattice(s, ix + 1, iy + 1);
    double ab = a + (b - a) * tx, cd = c + (d - c) * tx;
    return ab + (cd - ab) * ty;
}

/* three octaves, normalised to [0, 1] */
static double fbm(uint64_t s, double x, double y) {
    double sum = 0.0, amp = 1.0, norm = 0.0, f = 1.0;
    for (int o = 0; o < 3; ++o) {
        sum += amp * vnoise(mix64(s + (uint64_t)o), x * f, y * f);
        norm += amp;
        amp *= 0.5;
        f *= 2.0;
    }
    return sum / norm;
}

/* ---------------------------------------------------------------- geometry */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Ray (o, d), d not normalised.  On a hit nearer than *tbest, updates tbest, normal, (a, b)
 * texture coordinates and face id. */
static void hit_object(const synth_object *ob, const double *o, const double *d, double *tbest,
                       double *nrm, double *ta, double *tb, int *face) {
    if (ob->kind == SYNTH_PLANE || ob->kind == SYNTH_RECT) {
        const double *U = ob->ax, *V = ob->ax + 3, *N = ob->ax + 6;
        double den = dot3(N, d);
        if (fabs(den) < 1e-15) return;
        double pc[3] = {ob->c[0] - o[0], ob->c[1] - o[1], ob->c[2] - o[2]};
        double t = dot3(N, pc) / den;
        if (!(t > 1e-9) || t >= *tbest) return;
        double x[3] = {o[0] + t * d[0] - ob->c[0], o[1] + t * d[1] - ob->c[1], o[2] + t * d[2] - ob->c[2]};
        double a = dot3(U, x), b = dot3(V, x);
        if (ob->kind == SYNTH_RECT && (fabs(a) > ob->half[0] || fabs(b) > ob->half[1])) return;
        *tbest = t;
        nrm[0] = N[0]; nrm[1] = N[1]; nrm[2] = N[2];
        *ta = a; *tb = b; *face = 0;
        return;
    }
    /* oriented box: slab test in local coordinates */
    double ol[3], dl[3], oc[3] = {o[0] - ob->c[0], o[1] - ob->c[1], o[2] - ob->c[2]};
    for (int i = 0; i < 3; ++i) { ol[i] = dot3(ob->ax + 3 * i, oc); dl[i] = dot3(ob->ax + 3 * i, d); }
    double tn = -1e300, tf = 1e300;
    int axn = -1; double sgn = 0.0;
    for (int i = 0; i < 3; ++i) {
        if (fabs(dl[i]) < 1e-15) {
            if (fabs(ol[i]) > ob->half[i]) return;
            continue;
        }
        double t1 = (-ob->half[i] - ol[i]) / dl[i], t2 = (ob->half[i] - ol[i]) / dl[i];
        double s = -1.0;
        if (t1 > t2) { double tmp = t1; t1 = t2; t2 = tmp; s = 1.0; }
        if (t1 > tn) { tn = t1; axn = i; sgn = s; }
        if (t2 < tf) tf = t2;
    }
    if (axn < 0 || tn > tf || !(tn > 1e-9) || tn >= *tbest) return;
    *tbest = tn;
    for (int j = 0; j < 3; ++j) nrm[j] = sgn * ob->ax[3 * axn + j];
    int i1 = (axn + 1) % 3, i2 = (axn + 2) % 3;
    *ta = ol[i1] + tn * dl[i1];
    *tb = ol[i2] + tn * dl[i2];
    *face = 1 + 2 * axn + (sgn > 0.0 ? 1 : 0);
}

static void shade(const synth_object *ob, const double *nrm, double a, double b, int face,
                  const double *light, float *rgb) {
    double lam = dot3(nrm, light);
    double s = 0.45 + 0.55 * (lam > 0.0 ? lam : 0.0);
    for (int ch = 0; ch < 3; ++ch) {
        double alb;
        if (ob->textured) {
            uint64_t ts = mix64(ob->tex_seed + 977u * (uint64_t)face);
            double lum = fbm(ts, a * ob->tex_freq, b * ob->tex_freq);
            double chroma = fbm(mix64(ts ^ (0x51ULL + (uint64_t)ch)), a * ob->tex_freq * 0.5, b * ob->tex_freq * 0.5);
            alb = 0.1 + 0.8 * (0.65 * lum + 0.35 * chroma * ob->albedo[ch]);
        } else {
            alb = ob->albedo[ch];
        }
        rgb[ch] = (float)(alb * s);
    }
}

/* Casts one ray; returns the hit parameter (camera z when d has camera-space z = 1) or +inf. */
static double trace(const synth_object *objs, int n_obj, const double *light, const double *o,
                    const double *d, float *rgb, int *obj_id) {
    double tbest = INFINITY, nrm[3] = {0, 0, 0}, ta = 0, tb = 0;
    int face = 0, best = -1;
    for (int i = 0; i < n_obj; ++i) {
        double before = tbest;
        hit_object(objs + i, o, d, &tbest, nrm, &ta, &tb, &face);
        if (tbest < before) best = i;
    }
    if (best < 0) { rgb[0] = rgb[1] = rgb[2] = 0.0f; *obj_id = -1; return INFINITY; }
    shade(objs + best, nrm, ta, tb, face, light, rgb);
    *obj_id = best;
    return tbest;
}

/* inverse of upper-triangular K applied to (u, v, 1) */
static void kinv_pixel(const double *K, double u, double v, double *r) {
    double fx = K[0], s = K[1], cx = K[2], fy = K[4], cy = K[5];
    double y = (v - cy) / fy;
    r[0] = (u - cx - s * y) / fx;
    r[1] = y;
    r[2] = 1.0;
}

/*
 * Pinhole render of frames [0, nF).  K: nF*9, R: nF*9 (world->camera rotation, row-major),
 * t: nF*3.  Outputs (row-major, frame-major): rgb nF*H*W*3, depth nF*H*W (camera z; +inf on a
 * miss), optional world nF*H*W*3 hit points and obj nF*H*W object ids (NULL to skip).
 */
void synth_render(const synth_object *objs, int n_obj, const double *light, int W, int H, int nF,
                  const double *K, const double *R, const double *t, float *rgb, float *depth,
                  double *world, int32_t *obj) {
    long long total = (long long)nF * H;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long fr = 0; fr < total; ++fr) {
        int f = (int)(fr / H), v = (int)(fr % H);
        const double *Kf = K + 9 * f, *Rf = R + 9 * f, *tf = t + 3 * f;
        double C[3];
        for (int j = 0; j < 3; ++j) C[j] = -(Rf[j] * tf[0] + Rf[3 + j] * tf[1] + Rf[6 + j] * tf[2]);
        for (int u = 0; u < W; ++u) {
            double rc[3], dw[3];
            kinv_pixel(Kf, (double)u, (double)v, rc);
            for (int j = 0; j < 3; ++j) dw[j] = Rf[j] * rc[0] + Rf[3 + j] * rc[1] + Rf[6 + j] * rc[2];
            size_t pix = ((size_t)f * H + v) * W + u;
            int id;
            double th = trace(objs, n_obj, light, C, dw, rgb + 3 * pix, &id);
            depth[pix] = (float)th;
            if (world) for (int j = 0; j < 3; ++j) world[3 * pix + j] = C[j] + th * dw[j];
            if (obj) obj[pix] = id;
        }
    }
}

/*
 * Thin-lens render (reference image for the virtual-aperture workload).  For each pixel,
 * n_lens rays start at points of a disc of radius `aperture` in the camera's z = 0 plane
 * (concentric Vogel spiral) and pass through the in-focus point z_focus * K^-1 [u, v, 1].
 * The pixel colour is the mean of the ray colours.
 */
void synth_render_thinlens(const synth_object *objs, int n_obj, const double *light, int W, int H,
                           int nF, const double *K, const double *R, const double *t,
                           double aperture, double z_focus, int n_lens, float *rgb) {
    long long total = (long long)nF * H;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long fr = 0; fr < total; ++fr) {
        int f = (int)(fr / H), v = (int)(fr % H);
        const double *Kf = K + 9 * f, *Rf = R + 9 * f, *tf = t + 3 * f;
        double C[3];
        for (int j = 0; j < 3; ++j) C[j] = -(Rf[j] * tf[0] + Rf[3 + j] * tf[1] + Rf[6 + j] * tf[2]);
        for (int u = 0; u < W; ++u) {
            double rc[3];
            kinv_pixel(Kf, (double)u, (double)v, rc);
            double F[3] = {z_focus * rc[0], z_focus * rc[1], z_focus};
            double acc[3] = {0, 0, 0};
            for (int i = 0; i < n_lens; ++i) {
                double rho = aperture * sqrt((i + 0.5) / n_lens);
                double th = 2.399963229728653 * i;
                double L[3] = {rho * cos(th), rho * sin(th), 0.0};
                double dc[3] = {F[0] - L[0], F[1] - L[1], F[2] - L[2]}, o[3], dw[3];
                for (int j = 0; j < 3; ++j) {
                    o[j] = C[j] + Rf[j] * L[0] + Rf[3 + j] * L[1] + Rf[6 + j] * L[2];
                    dw[j] = Rf[j] * dc[0] + Rf[3 + j] * dc[1] + Rf[6 + j] * dc[2];
                }
                float c[3];
                int id;
                trace(objs, n_obj, light, o, dw, c, &id);
                for (int j = 0; j < 3; ++j) acc[j] += c[j];
            }
            size_t pix = ((size_t)f * H + v) * W + u;
            for (int j = 0; j < 3; ++j) rgb[3 * pix + j] = (float)(acc[j] / n_lens);
        }
    }
}

/*
 * Noise model.  frame0 is the absolute index of the first frame in the buffers, so clips
 * rendered in pieces get the same noise.  depth_out = depth * (1 + sigma_depth * n1),
 * rgb_out = rgb + sigma_img * n2 (no clipping).  Either output may be NULL.
 */
void synth_add_noise(int W, int H, int nF, int frame0, uint64_t seed, double sigma_img,
                     double sigma_depth, const float *rgb, const float *depth, float *rgb_out,
                     float *depth_out) {
    long long total = (long long)nF * H;
#pragma omp parallel for schedule(static)
    for (long long fr = 0; fr < total; ++fr) {
        int f = (int)(fr / H), v = (int)(fr % H);
        uint64_t fabs_idx = (uint64_t)(frame0 + f);
        for (int u = 0; u < W; ++u) {
            size_t pix = ((size_t)f * H + v) * W + u;
            uint64_t pidx = (uint64_t)v * (uint64_t)W + (uint64_t)u;
            if (depth_out) {
                double n = sigma_depth != 0.0 ? normal_key(key4(seed, 1, fabs_idx, pidx)) : 0.0;
                depth_out[pix] = (float)((double)depth[pix] * (1.0 + sigma_depth * n));
            }
            if (rgb_out) {
                for (int ch = 0; ch < 3; ++ch) {
                    double n = sigma_img != 0.0 ? normal_key(key4(seed, 2, fabs_idx, 3 * pidx + ch)) : 0.0;
                    rgb_out[3 * pix + ch] = (float)((double)rgb[3 * pix + ch] + sigma_img * n);
                }
            }
        }
    }
}

/* n standard normals for (seed, stream, frame, 0..n-1): used for pose noise and jitter */
void synth_normals(uint64_t seed, uint64_t stream, uint64_t frame, int n, double *out) {
    for (int i = 0; i < n; ++i) out[i] = normal_key(key4(seed, stream, frame, (uint64_t)i));
}
