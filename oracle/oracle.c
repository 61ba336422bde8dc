/*
 * oracle.c - FP64 CPU oracle of the scene-space gather-and-filter.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may call it.  It shares no code with the CUDA path and is not a fallback for it.
 *
 * It is the plain definition, written out in double precision, one output pixel at a time:
 *
 *   A1  camera composition (Sec. "Sample Gathering", Eq. 2 uses C_O * C_J^-1):
 *         P_{J<-O} = K_J [R_J R_O^T | t_J - R_J R_O^T t_O]          O-camera point -> J pixel (homog.)
 *         G_{O<-J} = [R_O R_J^T K_J^-1 | t_O - R_O R_J^T t_J]       (q_x d, q_y d, d, 1) in J -> O camera
 *       with P = [K_O | 0] and G = [K_O^-1 | 0] set directly when J = O.
 *   A3  reference sample s_ref (Sec. "Denoising"): x_ref = D_O(p) K_O^-1 [u, v, 1], c_ref = I_O(p).
 *   A4  project x_ref into every frame J of the temporal window [O-T, O+T]; the k x k window is
 *       centred on (floor(x'/z' + 0.5), floor(y'/z' + 0.5)); frames with z' <= 1e-6 d_ref are
 *       skipped, window pixels outside the image are skipped.
 *   A5  candidate q with valid depth d_q (finite, > 0): X_q = G (q_x d_q, q_y d_q, d_q, 1);
 *       accepted into S(p) iff |X_q - x_ref|^2 < r^2 (strict).
 *   A6  weight w(s) of Eq. 4 with diagonal covariance: exp(-sum over the 7 dimensions of the
 *       squared difference to s_ref over 2 sigma_d^2), sigma_rgb on colour, sigma_xyz on scene
 *       position, sigma_f on frame time; mode "mean" uses w = 1 (the averaging of Sec. "Denoising").
 *   A7  Eq. 3: O(p) = sum_s w(s) s_rgb / sum_s w(s).  An invalid reference depth gives c_ref.
 *
 * Virtual aperture (Sec. "Virtual aperture", Eq. 13-14) with the thin-lens footprint reading:
 *   the cone's axis is the viewing ray of p (from the O camera centre along K_O^-1 [u, v, 1]);
 *   for a sample X_q (O camera coordinates) t = O-camera depth of its foot point on the axis and
 *   q_perp = its distance to the axis (|X_q x ray| / |ray|);
 *   a(t) = a0 + A |z0 - t| / z0 (Eq. 13: focal plane at depth z0, slope A / z0 of a thin lens of
 *   radius A);
 *   per frame J the scanned box is the bounding box of the projections of the n_lens seed points
 *   (lens point L_i on a Vogel disc of radius A in the camera's z = 0 plane, ray L_i -> focus
 *   point z0 K_O^-1 [u, v, 1], seed point where that ray reaches depth d_ref), rounded with
 *   floor(x + 0.5), grown by h on each side and capped at `cap` pixels per axis around the rounded
 *   centroid, then clipped to the image; accepted iff q_perp < a(t); weight s_area / (pi a(t)^2)
 *   with s_area the squared scene length of one pixel edge of q at its depth (Eq. 6), which is
 *   (d_q / fx_J)^2 for a camera without skew.  Output sum w c / sum w (c_ref if nothing is
 *   accepted).
 *
 * Frustum gather (Sec. "Sample Gathering", Eq. 1-2), the paper's own gather:
 *   pixel (u, v) of O owns the frustum V of Eq. 1, the square of side l around the pixel swept
 *   from O-camera depth near to far.  A pixel q of frame J (in the temporal window) with valid
 *   depth d_q is a sample when X_q = G_{O<-J} (q_x d_q, q_y d_q, d_q, 1) has O depth in
 *   (near, far) and its O pixel (u', v') satisfies |u - u'| + |v - v'| < l / 2 (Eq. 2 as
 *   printed: the L1 distance, strict).  Every pixel of every window frame is tested; the paper's
 *   rasterised hull V_J only skips pixels that fail.  The same Eq. 4 weights and Eq. 3 mean
 *   follow (an invalid reference depth gives c_ref, as in the window gather).
 *
 * Per-frame weights (Sec. "Deblurring", Eq. 5; Sec. "Computational scene-space shutters", Eq. 10):
 *   mode 4 multiplies the Eq. 4 weight by the sum over frame J of the gradient magnitudes
 *   |grad I_J(q)| (forward differences, the L2 norm over the three colour channels and both
 *   axes, summed over the pixels that have a right and a lower neighbour); mode 5 replaces the
 *   weight by the shutter function xi(J - O).  Both apply to either gather.
 *
 * Super-resolution (Sec. "Super resolution", Eq. 6-7): the output grid has `scale` times the
 *   input resolution per axis; output pixel (U, V) sits at input coordinates
 *   u = (U + 0.5) / scale - 0.5 (and v alike), and its camera is K_O with fx, fy scaled and the
 *   principal point mapped the same way.  s_ref is the bilinear interpolation of colour and
 *   depth at (u, v) (coordinates clamped to the image; an invalid depth among the four makes
 *   the reference invalid, which outputs the interpolated colour).  Samples are gathered from
 *   the output pixel's own frustum (Eq. 1-2 in output pixels) and weighted by Eq. 4 times
 *   exp(-s_area / (2 sigma_area^2)) with s_area = (d_q / fx_J)^2, the squared scene length of
 *   one pixel edge of the sample at its depth (Eq. 6 for a camera without skew); mode 3 uses
 *   w = 1.
 *
 * Inpainting (Sec. "Inpainting and semi-transparency", Eq. 8-9): a per-frame mask M marks the
 *   pixels to remove; from a scene-space box, M_J(q) = 1 when q's world point (its depth
 *   unprojected with the camera of J) lies inside the box.  A pixel with M_O(p) = 0 keeps its
 *   input colour.  A masked pixel gathers its frustum S(p) (Eq. 1-2; its own depth is not used)
 *   and starts from the mean colour of all of S(p) (Eq. 8); two steps of the weighted mean of
 *   Eq. 9 follow, each with w = exp(-|c_ref - c|^2 / (2 sigma_rgb^2)) for unmasked samples and 0
 *   for masked ones, the result of a step being the next step's reference (a step whose weights
 *   are all 0 keeps the reference).  An empty S(p) keeps the input colour.
 *
 * Semi-transparency (same section, the sentence after Eq. 9: the standard multivariate weighting
 *   is added, for the input frame's own sample, with sigma_rgb = 80 on the 0-255 scale): the
 *   masked pixel's own sample s_I = (I_O(p), x_ref, O), x_ref from its depth as in denoising,
 *   serves as a second reference.  The mean of Eq. 8 and the first step of Eq. 9 are those of
 *   inpainting; in the second step every sample s of S(p), masked or not, additionally weighs
 *   the Eq. 4 weight w(s; s_I) (colour, scene position and frame terms), so a sample's weight is
 *   [M(s) = 0] exp(-|c_ref - c_s|^2 / (2 sigma_rgb^2)) + w_Eq4(s; s_I) and the output is Eq. 3
 *   with it: the object's own samples near x_ref blend with the background's mean-shift estimate.
 *   A masked pixel without a valid depth has no x_ref and gets the inpainting result.
 *
 * Built with -ffp-contract=off: every product and sum is rounded on its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t W, H, F, pad_;
    const float *rgb;    /* F*H*W*3, interleaved, row-major */
    const float *depth;  /* F*H*W camera z */
    const double *K;     /* F*9 intrinsics, row-major */
    const double *w2c;   /* F*12 world->camera [R|t], row-major */
} oc_clip;

typedef struct {
    int32_t mode;        /* 0 denoise (Eq. 4), 1 virtual aperture (Eq. 13-14), 3 mean (w = 1) */
    int32_t k;           /* odd window width */
    int32_t T;           /* temporal half window */
    int32_t lens_samples;
    double radius;       /* absolute radius r */
    double sigma_rgb, sigma_xyz, sigma_f;
    double band_rel;     /* |dist - r| <= band_rel * r marks a candidate as "in band" */
    double tie_band;     /* |frac(x) - 0.5| < tie_band marks a window centre as ambiguous */
    double aperture;     /* A: lens radius (scene units) */
    double focal_depth;  /* z0 */
    double a0;           /* cone waist */
    int32_t cap;         /* aperture footprint cap per axis (pixels) */
    int32_t gather;      /* 0 depth-seeded window (or the aperture cone), 1 frustum (Eq. 1-2) */
    double frustum_l;    /* frustum size l in pixels (Eq. 1) */
    double near_plane, far_plane;  /* frustum depth range (Eq. 1) */
    const double *frame_w;  /* mode 4: per input frame J the blurriness factor of Eq. 5 (F values) */
    const double *slot_w;   /* mode 5: the shutter function xi(J - O) of Eq. 10 at J = O-T+j (2T+1 values) */
    double sigma_area;      /* super-resolution (Eq. 7): length scale of the s_area term */
} oc_params;

/* membership codes (low 3 bits) and band flag */
#define OC_OUT 0       /* window pixel outside the image */
#define OC_INVALID 1   /* invalid depth */
#define OC_REJECT 2
#define OC_ACCEPT 3
#define OC_BAND 8      /* or-ed in when |dist - r| <= band_rel * r (or the cone analogue) */

/* ------------------------------------------------------------------ small linear algebra */

static void mat3_inverse(const double *A, double *B) {
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    B[0] = c00 / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = c01 / det;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = c02 / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

static void mat3_mul(const double *A, const double *B, double *C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

static void mat3_vec(const double *A, const double *x, double *y) {
    for (int i = 0; i < 3; ++i) y[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
}

static void split_rt(const double *w2c, double *R, double *t) {
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) R[3 * i + j] = w2c[4 * i + j];
        t[i] = w2c[4 * i + 3];
    }
}

/* apply a 3x4 matrix to (x, 1) */
static void apply34(const double *M, const double *x, double *y) {
    for (int i = 0; i < 3; ++i) y[i] = M[4 * i] * x[0] + M[4 * i + 1] * x[1] + M[4 * i + 2] * x[2] + M[4 * i + 3];
}

/* A1: P_{J<-O} and G_{O<-J} (both 3x4 row-major). */
void oc_compose(const double *K_O, const double *w2c_O, const double *K_J, const double *w2c_J, int same,
                double *P, double *G) {
    if (same) {
        double Ki[9];
        mat3_inverse(K_O, Ki);
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) { P[4 * i + j] = K_O[3 * i + j]; G[4 * i + j] = Ki[3 * i + j]; }
            P[4 * i + 3] = 0.0;
            G[4 * i + 3] = 0.0;
        }
        return;
    }
    double RO[9], tO[3], RJ[9], tJ[3], ROt[9], RJt[9], RJO[9], ROJ[9], KJi[9], M[9], tmp[3];
    split_rt(w2c_O, RO, tO);
    split_rt(w2c_J, RJ, tJ);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { ROt[3 * i + j] = RO[3 * j + i]; RJt[3 * i + j] = RJ[3 * j + i]; }
    /* P = K_J [R_J R_O^T | t_J - R_J R_O^T t_O] */
    mat3_mul(RJ, ROt, RJO);
    mat3_vec(RJO, tO, tmp);
    double tJO[3] = {tJ[0] - tmp[0], tJ[1] - tmp[1], tJ[2] - tmp[2]};
    mat3_mul(K_J, RJO, M);
    double KtJO[3];
    mat3_vec(K_J, tJO, KtJO);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) P[4 * i + j] = M[3 * i + j];
        P[4 * i + 3] = KtJO[i];
    }
    /* G = [R_O R_J^T K_J^-1 | t_O - R_O R_J^T t_J] */
    mat3_mul(RO, RJt, ROJ);
    mat3_inverse(K_J, KJi);
    mat3_mul(ROJ, KJi, M);
    mat3_vec(ROJ, tJ, tmp);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) G[4 * i + j] = M[3 * i + j];
        G[4 * i + 3] = tO[i] - tmp[i];
    }
}

/* ------------------------------------------------------------------ weights and filter */

/* Eq. 4 with diagonal covariance: s = (r, g, b, x, y, z, f). */
double oc_weight_denoise(const double *s, const double *sref, double sigma_rgb, double sigma_xyz, double sigma_f) {
    double e = 0.0;
    for (int i = 0; i < 3; ++i) e += (sref[i] - s[i]) * (sref[i] - s[i]) / (2.0 * sigma_rgb * sigma_rgb);
    for (int i = 3; i < 6; ++i) e += (sref[i] - s[i]) * (sref[i] - s[i]) / (2.0 * sigma_xyz * sigma_xyz);
    e += (sref[6] - s[6]) * (sref[6] - s[6]) / (2.0 * sigma_f * sigma_f);
    return exp(-e);
}

/* Eq. 3 over an explicit sample set S (n x 7) with Eq. 4 weights (mode 0) or w = 1 (mode 3).
 * Writes the colour and returns W = sum of weights. */
double oc_filter(const double *S, int n, const double *sref, int mode, double sigma_rgb, double sigma_xyz,
                 double sigma_f, double *out) {
    double acc[3] = {0, 0, 0}, W = 0.0;
    for (int i = 0; i < n; ++i) {
        double w = mode == 3 ? 1.0 : oc_weight_denoise(S + 7 * i, sref, sigma_rgb, sigma_xyz, sigma_f);
        for (int c = 0; c < 3; ++c) acc[c] += w * S[7 * i + c];
        W += w;
    }
    for (int c = 0; c < 3; ++c) out[c] = acc[c] / W;
    return W;
}

static int valid_depth(float d) { return isfinite(d) && d > 0.0f; }

/* Weight of an accepted sample s (7-vector) against s_ref from window frame J (slot j) for the
 * Eq. 4 based modes: 0 denoise, 3 mean, 4 deblurring (Eq. 5), 5 computational shutter (Eq. 10). */
static double sample_weight(const oc_params *p, const double *s, const double *sr, int J, int j) {
    switch (p->mode) {
    case 3: return 1.0;
    case 5: return p->slot_w ? p->slot_w[j] : 1.0;
    case 4: return oc_weight_denoise(s, sr, p->sigma_rgb, p->sigma_xyz, p->sigma_f) * (p->frame_w ? p->frame_w[J] : 1.0);
    default: return oc_weight_denoise(s, sr, p->sigma_rgb, p->sigma_xyz, p->sigma_f);
    }
}

/* Eq. 5's blurriness measure: per frame the sum of the gradient magnitudes (see above); out F values. */
void oc_frame_sharpness(const oc_clip *c, double *out) {
    const int W = c->W, H = c->H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int f = 0; f < c->F; ++f) {
        double sum = 0.0;
        for (int y = 0; y + 1 < H; ++y)
            for (int x = 0; x + 1 < W; ++x) {
                const float *a = c->rgb + 3 * (((size_t)f * H + y) * W + x);
                const float *r = a + 3, *d = a + 3 * (size_t)W;
                double g2 = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    const double gx = (double)r[ch] - a[ch], gy = (double)d[ch] - a[ch];
                    g2 += gx * gx + gy * gy;
                }
                sum += sqrt(g2);
            }
        out[f] = sum;
    }
}

/* ------------------------------------------------------------------ gather + filter, one pixel */

typedef struct {
    int32_t *status;  /* per slot: -2 invalid reference, -1 frame outside clip, 0 skipped (behind), 1 gathered */
    int32_t *centre;  /* per slot: window centre (x, y) */
    uint8_t *amb;     /* per slot: 1 if the window centre is within tie_band of a rounding tie */
    uint8_t *codes;   /* per slot: k*k membership codes (row-major window) */
    int32_t *box;     /* aperture: per slot window box (x0, y0, x1, y1) inclusive */
} oc_member;

/* Vogel-disc lens point i of n, radius A */
static void lens_point(int i, int n, double A, double *L) {
    double rho = A * sqrt((i + 0.5) / n);
    double th = 2.399963229728653 * i;
    L[0] = rho * cos(th);
    L[1] = rho * sin(th);
}

static void pixel(const oc_clip *c, const oc_params *p, int O, int u, int v, const double *Pt, const double *Gt,
                  double *out, double *sumw, int64_t *nacc, int64_t *nexam, oc_member *mem, size_t mi) {
    const int W = c->W, H = c->H, F = c->F, k = p->k, h = (k - 1) / 2, ns = 2 * p->T + 1;
    size_t pix = ((size_t)O * H + v) * W + u;
    float dref_f = c->depth[pix];
    double cref[3] = {c->rgb[3 * pix], c->rgb[3 * pix + 1], c->rgb[3 * pix + 2]};
    *nacc = 0;
    *nexam = 0;
    *sumw = 0.0;
    if (!valid_depth(dref_f)) {
        for (int ch = 0; ch < 3; ++ch) out[ch] = cref[ch];
        if (mem) for (int j = 0; j < ns; ++j) mem->status[mi * ns + j] = -2;
        return;
    }
    double dref = dref_f;
    double KOi[9], ray[3], xref[3];
    mat3_inverse(c->K + 9 * O, KOi);
    double uv1[3] = {u, v, 1.0};
    mat3_vec(KOi, uv1, ray);
    for (int i = 0; i < 3; ++i) xref[i] = dref * ray[i];

    /* aperture: seed points where the lens rays through the focus point reach depth d_ref */
    double rr = ray[0] * ray[0] + ray[1] * ray[1] + ray[2] * ray[2], seeds[64][3];
    int nl = p->lens_samples > 64 ? 64 : p->lens_samples;
    if (p->mode == 1) {
        double Fp[3] = {p->focal_depth * ray[0], p->focal_depth * ray[1], p->focal_depth * ray[2]};
        for (int i = 0; i < nl; ++i) {
            double L[2];
            lens_point(i, nl, p->aperture, L);
            double s = dref / p->focal_depth;
            seeds[i][0] = L[0] + s * (Fp[0] - L[0]);
            seeds[i][1] = L[1] + s * (Fp[1] - L[1]);
            seeds[i][2] = dref;
        }
    }

    double acc[3] = {0, 0, 0}, Wsum = 0.0;
    for (int j = 0; j < ns; ++j) {
        int J = O - p->T + j;
        if (J < 0 || J >= F) {
            if (mem) mem->status[mi * ns + j] = -1;
            continue;
        }
        const double *P = Pt + 12 * j, *G = Gt + 12 * j;
        int bx0, by0, bx1, by1, amb = 0;
        if (p->mode != 1) {
            double xp[3];
            apply34(P, xref, xp);
            if (xp[2] <= 1e-6 * dref) {
                if (mem) mem->status[mi * ns + j] = 0;
                continue;
            }
            double up = xp[0] / xp[2], vp = xp[1] / xp[2];
            double fu = up - floor(up), fv = vp - floor(vp);
            amb = fabs(fu - 0.5) < p->tie_band || fabs(fv - 0.5) < p->tie_band;
            double cxd = floor(up + 0.5), cyd = floor(vp + 0.5);
            /* a centre this far out cannot reach the image: clamp it far outside */
            if (cxd < -(double)(4 * k + 8)) cxd = -(double)(4 * k + 8);
            if (cxd > (double)(W + 4 * k + 8)) cxd = (double)(W + 4 * k + 8);
            if (cyd < -(double)(4 * k + 8)) cyd = -(double)(4 * k + 8);
            if (cyd > (double)(H + 4 * k + 8)) cyd = (double)(H + 4 * k + 8);
            bx0 = (int)cxd - h; bx1 = (int)cxd + h; by0 = (int)cyd - h; by1 = (int)cyd + h;
            if (mem) { mem->centre[2 * (mi * ns + j)] = (int)cxd; mem->centre[2 * (mi * ns + j) + 1] = (int)cyd; }
        } else {
            /* footprint: bbox of projected seed points, grown by h, capped around the centroid */
            double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300, sx = 0, sy = 0;
            int nin = 0;
            for (int i = 0; i < nl; ++i) {
                double xp[3];
                apply34(P, seeds[i], xp);
                if (xp[2] <= 1e-6 * dref) continue;
                double up = xp[0] / xp[2], vp = xp[1] / xp[2];
                if (fabs(up - floor(up) - 0.5) < p->tie_band || fabs(vp - floor(vp) - 0.5) < p->tie_band) amb = 1;
                if (up < mnx) mnx = up;
                if (up > mxx) mxx = up;
                if (vp < mny) mny = vp;
                if (vp > mxy) mxy = vp;
                sx += up; sy += vp; ++nin;
            }
            if (nin < nl) {  /* a seed behind the J camera: skip the frame */
                if (mem) mem->status[mi * ns + j] = 0;
                continue;
            }
            double lim = (double)(W + H + 4 * p->cap + 8);
            double mx = sx / nl, my = sy / nl;
            if (fabs(mx - floor(mx) - 0.5) < p->tie_band || fabs(my - floor(my) - 0.5) < p->tie_band) amb = 1;
            if (mx < -lim) mx = -lim;
            if (mx > lim) mx = lim;
            if (my < -lim) my = -lim;
            if (my > lim) my = lim;
            int ccx = (int)floor(mx + 0.5), ccy = (int)floor(my + 0.5), hc = (p->cap - 1) / 2;
            double fx0 = floor(mnx + 0.5) - h, fx1 = floor(mxx + 0.5) + h;
            double fy0 = floor(mny + 0.5) - h, fy1 = floor(mxy + 0.5) + h;
            bx0 = fx0 < ccx - hc ? ccx - hc : (int)fx0;
            bx1 = fx1 > ccx + hc ? ccx + hc : (int)fx1;
            by0 = fy0 < ccy - hc ? ccy - hc : (int)fy0;
            by1 = fy1 > ccy + hc ? ccy + hc : (int)fy1;
            if (mem) {
                int32_t *b = mem->box + 4 * (mi * ns + j);
                b[0] = bx0; b[1] = by0; b[2] = bx1; b[3] = by1;
            }
        }
        if (mem) { mem->status[mi * ns + j] = 1; mem->amb[mi * ns + j] = (uint8_t)amb; }
        double fxJ = c->K[9 * J + 0];
        const int win = p->mode == 1 ? p->cap : k;
        for (int qy = by0; qy <= by1; ++qy) {
            for (int qx = bx0; qx <= bx1; ++qx) {
                int slot = (qy - by0) * win + (qx - bx0);
                uint8_t code;
                if (qx < 0 || qx >= W || qy < 0 || qy >= H) {
                    code = OC_OUT;
                } else {
                    ++*nexam;
                    size_t qi = ((size_t)J * H + qy) * W + qx;
                    float dq = c->depth[qi];
                    if (!valid_depth(dq)) {
                        code = OC_INVALID;
                    } else {
                        double q3[3] = {qx * (double)dq, qy * (double)dq, (double)dq}, X[3];
                        apply34(G, q3, X);
                        double dx = X[0] - xref[0], dy = X[1] - xref[1], dz = X[2] - xref[2];
                        double w = 0.0;
                        int acc_ok;
                        if (p->mode != 1) {
                            double d2 = dx * dx + dy * dy + dz * dz;
                            acc_ok = d2 < p->radius * p->radius;
                            code = acc_ok ? OC_ACCEPT : OC_REJECT;
                            if (fabs(sqrt(d2) - p->radius) <= p->band_rel * p->radius) code |= OC_BAND;
                            if (acc_ok) {
                                double s[7] = {c->rgb[3 * qi], c->rgb[3 * qi + 1], c->rgb[3 * qi + 2], X[0], X[1], X[2], J};
                                double sr[7] = {cref[0], cref[1], cref[2], xref[0], xref[1], xref[2], O};
                                w = sample_weight(p, s, sr, J, j);
                            }
                        } else {
                            /* foot point depth t and distance to the axis (textbook point-line distance) */
                            double xr = X[0] * ray[0] + X[1] * ray[1] + X[2] * ray[2];
                            double t = xr / rr;
                            double cr0 = X[1] * ray[2] - X[2] * ray[1], cr1 = X[2] * ray[0] - X[0] * ray[2],
                                   cr2 = X[0] * ray[1] - X[1] * ray[0];
                            double qperp = sqrt((cr0 * cr0 + cr1 * cr1 + cr2 * cr2) / rr);
                            double a = p->a0 + p->aperture * fabs(p->focal_depth - t) / p->focal_depth;
                            acc_ok = qperp < a;
                            code = acc_ok ? OC_ACCEPT : OC_REJECT;
                            if (fabs(qperp - a) <= p->band_rel * a) code |= OC_BAND;
                            if (acc_ok) {
                                double e = (double)dq / fxJ;
                                double s_area = e * e;
                                w = s_area / (3.141592653589793 * a * a);
                            }
                        }
                        if (acc_ok) {
                            for (int ch = 0; ch < 3; ++ch) acc[ch] += w * c->rgb[3 * qi + ch];
                            Wsum += w;
                            ++*nacc;
                        }
                    }
                }
                if (mem) mem->codes[(mi * ns + j) * (size_t)(win * win) + slot] = code;
            }
        }
    }
    *sumw = Wsum;
    if (Wsum > 0.0) {
        for (int ch = 0; ch < 3; ++ch) out[ch] = acc[ch] / Wsum;
    } else {
        for (int ch = 0; ch < 3; ++ch) out[ch] = cref[ch];
    }
}

/*
 * Gather and filter the crop [x0, x0+cw) x [y0, y0+ch) of output frame O.
 * Outputs (row-major over the crop): out_rgb cw*ch*3, sumw, nacc, nexam.  mem_* may be NULL;
 * otherwise they hold per (pixel, slot) records for slots J = O-T .. O+T.
 */
int oc_gather_filter(const oc_clip *c, const oc_params *p, int O, int x0, int y0, int cw, int ch, double *out_rgb,
                     double *out_sumw, int64_t *out_nacc, int64_t *out_nexam, int32_t *mem_status,
                     int32_t *mem_centre, uint8_t *mem_amb, uint8_t *mem_codes, int32_t *mem_box) {
    if (p->k < 1 || (p->k & 1) == 0 || p->T < 0 || O < 0 || O >= c->F) return -1;
    int ns = 2 * p->T + 1;
    double *Pt = (double *)malloc(sizeof(double) * 12 * ns), *Gt = (double *)malloc(sizeof(double) * 12 * ns);
    if (!Pt || !Gt) { free(Pt); free(Gt); return -2; }
    for (int j = 0; j < ns; ++j) {
        int J = O - p->T + j;
        if (J < 0 || J >= c->F) continue;
        oc_compose(c->K + 9 * O, c->w2c + 12 * O, c->K + 9 * J, c->w2c + 12 * J, J == O, Pt + 12 * j, Gt + 12 * j);
    }
    oc_member mem = {mem_status, mem_centre, mem_amb, mem_codes, mem_box};
    oc_member *mp = mem_status ? &mem : NULL;
    long long n = (long long)cw * ch;
#pragma omp parallel for schedule(dynamic, 8)
    for (long long i = 0; i < n; ++i) {
        int u = x0 + (int)(i % cw), v = y0 + (int)(i / cw);
        pixel(c, p, O, u, v, Pt, Gt, out_rgb + 3 * i, out_sumw + i, out_nacc + i, out_nexam + i, mp, (size_t)i);
    }
    free(Pt);
    free(Gt);
    return 0;
}

/* ================================================================== frustum gather (Eq. 1-2) */

/* SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014): an order-independent
 * membership checksum sums it over the linear indices qy * W + qx + 1 of a sample set. */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* Is X (O-camera coordinates) inside the frustum of pixel (u, v)?  *band is set when X lies
 * within tie_band pixels of the L1 bound or within band_rel of the near or far depth. */
static int in_frustum(const double *KO, const double *X, int u, int v, const oc_params *p, int *band) {
    const double z = X[2];
    *band = fabs(z - p->near_plane) <= p->band_rel * p->near_plane || fabs(z - p->far_plane) <= p->band_rel * p->far_plane;
    if (!(z > p->near_plane && z < p->far_plane)) return 0;
    const double up = (KO[0] * X[0] + KO[1] * X[1] + KO[2] * X[2]) / z;
    const double vp = (KO[4] * X[1] + KO[5] * X[2]) / z;
    const double l1 = fabs((double)u - up) + fabs((double)v - vp);
    if (fabs(l1 - 0.5 * p->frustum_l) <= p->tie_band) *band = 1;
    return l1 < 0.5 * p->frustum_l;
}

/*
 * Frustum gather and filter of the crop [x0, x0+cw) x [y0, y0+ch) of output frame O.
 * Outputs (row-major over the crop): out_rgb cw*ch*3, sumw, nacc.  mem_count, mem_hash and
 * mem_band may be NULL; otherwise per (pixel, slot J = O-T+j): the number of samples from J,
 * the wrapping sum of mix64(qy * W + qx + 1) over them, and 1 when any tested pixel of J lies in
 * the tie band.  A pixel with an invalid reference depth gets c_ref and empty records.
 */
int oc_frustum_filter(const oc_clip *c, const oc_params *p, int O, int x0, int y0, int cw, int ch, double *out_rgb,
                      double *out_sumw, int64_t *out_nacc, int32_t *mem_count, uint64_t *mem_hash, uint8_t *mem_band) {
    if (p->T < 0 || O < 0 || O >= c->F || !(p->frustum_l > 0) || !(p->near_plane > 0) ||
        !(p->far_plane > p->near_plane))
        return -1;
    const int ns = 2 * p->T + 1, W = c->W, H = c->H;
    double *Gt = (double *)malloc(sizeof(double) * 12 * ns);
    if (!Gt) return -2;
    for (int j = 0; j < ns; ++j) {
        int J = O - p->T + j;
        double P[12];
        if (J < 0 || J >= c->F) continue;
        oc_compose(c->K + 9 * O, c->w2c + 12 * O, c->K + 9 * J, c->w2c + 12 * J, J == O, P, Gt + 12 * j);
    }
    const double *KO = c->K + 9 * O;
    double KOi[9];
    mat3_inverse(KO, KOi);
    long long n = (long long)cw * ch;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long i = 0; i < n; ++i) {
        const int u = x0 + (int)(i % cw), v = y0 + (int)(i / cw);
        const size_t pix = ((size_t)O * H + v) * W + u;
        const float dref = c->depth[pix];
        double sref[7], acc[3] = {0, 0, 0}, sw = 0.0;
        int64_t cnt = 0;
        for (int ch3 = 0; ch3 < 3; ++ch3) sref[ch3] = c->rgb[3 * pix + ch3];
        if (mem_count)
            for (int j = 0; j < ns; ++j) {
                mem_count[i * ns + j] = 0;
                mem_hash[i * ns + j] = 0;
                mem_band[i * ns + j] = 0;
            }
        if (valid_depth(dref)) {
            double uv1[3] = {u, v, 1.0}, ray[3];
            mat3_vec(KOi, uv1, ray);
            for (int a = 0; a < 3; ++a) sref[3 + a] = (double)dref * ray[a];
            sref[6] = O;
            for (int j = 0; j < ns; ++j) {
                const int J = O - p->T + j;
                if (J < 0 || J >= c->F) continue;
                const double *G = Gt + 12 * j;
                int32_t mc = 0;
                uint64_t mh = 0;
                uint8_t mb = 0;
                for (int qy = 0; qy < H; ++qy)
                    for (int qx = 0; qx < W; ++qx) {
                        const size_t qi = ((size_t)J * H + qy) * W + qx;
                        const float dq = c->depth[qi];
                        if (!valid_depth(dq)) continue;
                        double q3[3] = {qx * (double)dq, qy * (double)dq, (double)dq}, X[3];
                        apply34(G, q3, X);
                        int band;
                        const int in = in_frustum(KO, X, u, v, p, &band);
                        mb |= (uint8_t)band;
                        if (!in) continue;
                        double s[7] = {c->rgb[3 * qi], c->rgb[3 * qi + 1], c->rgb[3 * qi + 2], X[0], X[1], X[2], (double)J};
                        const double w = sample_weight(p, s, sref, J, j);
                        for (int a = 0; a < 3; ++a) acc[a] += w * s[a];
                        sw += w;
                        ++mc;
                        mh += mix64((uint64_t)qy * (uint64_t)W + (uint64_t)qx + 1u);
                    }
                cnt += mc;
                if (mem_count) {
                    mem_count[i * ns + j] = mc;
                    mem_hash[i * ns + j] = mh;
                    mem_band[i * ns + j] = mb;
                }
            }
        }
        for (int a = 0; a < 3; ++a) out_rgb[3 * i + a] = sw > 0.0 ? acc[a] / sw : sref[a];
        out_sumw[i] = sw;
        out_nacc[i] = cnt;
    }
    free(Gt);
    return 0;
}

/* Eq. 7's weight of sample s (7-vector, depth d_q in frame J with focal length fx_J) against sref */
double oc_weight_superres(const double *s, const double *sref, double dq, double fxJ, double sigma_rgb,
                          double sigma_xyz, double sigma_f, double sigma_area) {
    const double e = dq / fxJ;
    const double s_area = e * e;
    return oc_weight_denoise(s, sref, sigma_rgb, sigma_xyz, sigma_f) * exp(-s_area / (2.0 * sigma_area * sigma_area));
}

/* Output-grid intrinsics of super-resolution: K with fx, fy scaled and c -> scale (c + 0.5) - 0.5 */
static void scaled_K(const double *K, int scale, double *Ks) {
    memcpy(Ks, K, 9 * sizeof(double));
    Ks[0] = K[0] * scale;
    Ks[1] = K[1] * scale;
    Ks[2] = scale * (K[2] + 0.5) - 0.5;
    Ks[4] = K[4] * scale;
    Ks[5] = scale * (K[5] + 0.5) - 0.5;
}

/* Bilinear value of a (H, W, nc) float image at (x, y), coordinates clamped to the image */
static void bilinear(const float *img, int W, int H, int nc, double x, double y, double *out) {
    x = x < 0 ? 0 : (x > W - 1 ? W - 1 : x);
    y = y < 0 ? 0 : (y > H - 1 ? H - 1 : y);
    int x0 = (int)floor(x), y0 = (int)floor(y);
    int x1 = x0 + 1 < W ? x0 + 1 : W - 1, y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    double fx = x - x0, fy = y - y0;
    for (int c = 0; c < nc; ++c) {
        double a = img[((size_t)y0 * W + x0) * nc + c], b = img[((size_t)y0 * W + x1) * nc + c];
        double d = img[((size_t)y1 * W + x0) * nc + c], e = img[((size_t)y1 * W + x1) * nc + c];
        out[c] = (1.0 - fy) * ((1.0 - fx) * a + fx * b) + fy * ((1.0 - fx) * d + fx * e);
    }
}

/*
 * Super-resolution gather and filter of output frame O on the `scale`-times grid, over the
 * output crop [X0, X0+CW) x [Y0, Y0+CH) (output-grid pixels).  Outputs as oc_frustum_filter.
 */
int oc_superres_filter(const oc_clip *c, const oc_params *p, int O, int scale, int X0, int Y0, int CW, int CH,
                       double *out_rgb, double *out_sumw, int64_t *out_nacc, int32_t *mem_count, uint64_t *mem_hash,
                       uint8_t *mem_band) {
    if (p->T < 0 || O < 0 || O >= c->F || scale < 1 || !(p->frustum_l > 0) || !(p->near_plane > 0) ||
        !(p->far_plane > p->near_plane) || !(p->sigma_area > 0))
        return -1;
    const int ns = 2 * p->T + 1, W = c->W, H = c->H;
    double KOs[9], KOsi[9];
    scaled_K(c->K + 9 * O, scale, KOs);
    mat3_inverse(KOs, KOsi);
    double *Gt = (double *)malloc(sizeof(double) * 12 * ns);
    if (!Gt) return -2;
    for (int j = 0; j < ns; ++j) {
        int J = O - p->T + j;
        double P[12];
        if (J < 0 || J >= c->F) continue;
        /* G_{O<-J} maps J pixels to O camera coordinates; the output grid only enters the test */
        oc_compose(c->K + 9 * O, c->w2c + 12 * O, c->K + 9 * J, c->w2c + 12 * J, J == O, P, Gt + 12 * j);
    }
    long long n = (long long)CW * CH;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long i = 0; i < n; ++i) {
        const int U = X0 + (int)(i % CW), V = Y0 + (int)(i / CW);
        const double u = (U + 0.5) / scale - 0.5, v = (V + 0.5) / scale - 0.5;
        double sref[7], dref, acc[3] = {0, 0, 0}, sw = 0.0;
        int64_t cnt = 0;
        bilinear(c->rgb + (size_t)O * H * W * 3, W, H, 3, u, v, sref);
        bilinear(c->depth + (size_t)O * H * W, W, H, 1, u, v, &dref);
        if (mem_count)
            for (int j = 0; j < ns; ++j) {
                mem_count[i * ns + j] = 0;
                mem_hash[i * ns + j] = 0;
                mem_band[i * ns + j] = 0;
            }
        /* an invalid depth among the four (NaN, inf or <= 0 before mixing) invalidates s_ref */
        int ok = 1;
        {
            const double xc = u < 0 ? 0 : (u > W - 1 ? W - 1 : u), yc = v < 0 ? 0 : (v > H - 1 ? H - 1 : v);
            const int x0 = (int)floor(xc), y0 = (int)floor(yc);
            const int x1 = x0 + 1 < W ? x0 + 1 : W - 1, y1 = y0 + 1 < H ? y0 + 1 : H - 1;
            const float *D = c->depth + (size_t)O * H * W;
            ok = valid_depth(D[(size_t)y0 * W + x0]) && valid_depth(D[(size_t)y0 * W + x1]) &&
                 valid_depth(D[(size_t)y1 * W + x0]) && valid_depth(D[(size_t)y1 * W + x1]);
        }
        if (ok) {
            double UV1[3] = {U, V, 1.0}, ray[3];
            mat3_vec(KOsi, UV1, ray);
            for (int a = 0; a < 3; ++a) sref[3 + a] = dref * ray[a];
            sref[6] = O;
            for (int j = 0; j < ns; ++j) {
                const int J = O - p->T + j;
                if (J < 0 || J >= c->F) continue;
                const double *G = Gt + 12 * j;
                const double fxJ = c->K[9 * J];
                int32_t mc = 0;
                uint64_t mh = 0;
                uint8_t mb = 0;
                for (int qy = 0; qy < H; ++qy)
                    for (int qx = 0; qx < W; ++qx) {
                        const size_t qi = ((size_t)J * H + qy) * W + qx;
                        const float dq = c->depth[qi];
                        if (!valid_depth(dq)) continue;
                        double q3[3] = {qx * (double)dq, qy * (double)dq, (double)dq}, X[3];
                        apply34(G, q3, X);
                        int band;
                        const int in = in_frustum(KOs, X, U, V, p, &band);
                        mb |= (uint8_t)band;
                        if (!in) continue;
                        double s[7] = {c->rgb[3 * qi], c->rgb[3 * qi + 1], c->rgb[3 * qi + 2], X[0], X[1], X[2], (double)J};
                        const double w = p->mode == 3 ? 1.0
                                                      : oc_weight_superres(s, sref, dq, fxJ, p->sigma_rgb, p->sigma_xyz,
                                                                           p->sigma_f, p->sigma_area);
                        for (int a = 0; a < 3; ++a) acc[a] += w * s[a];
                        sw += w;
                        ++mc;
                        mh += mix64((uint64_t)qy * (uint64_t)W + (uint64_t)qx + 1u);
                    }
                cnt += mc;
                if (mem_count) {
                    mem_count[i * ns + j] = mc;
                    mem_hash[i * ns + j] = mh;
                    mem_band[i * ns + j] = mb;
                }
            }
        }
        for (int a = 0; a < 3; ++a) out_rgb[3 * i + a] = sw > 0.0 ? acc[a] / sw : sref[a];
        out_sumw[i] = sw;
        out_nacc[i] = cnt;
    }
    free(Gt);
    return 0;
}

/* Eq. 8-9's mask from a scene-space axis-aligned box = {xmin, ymin, zmin, xmax, ymax, zmax} (world
 * coordinates, inclusive): mask F*H*W bytes, 1 inside, 0 outside or for an invalid depth. */
void oc_mask_from_box(const oc_clip *c, const double *box, uint8_t *mask) {
    const int W = c->W, H = c->H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int f = 0; f < c->F; ++f) {
        double Ki[9], R[9], t[3];
        mat3_inverse(c->K + 9 * f, Ki);
        split_rt(c->w2c + 12 * f, R, t);
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const size_t i = ((size_t)f * H + y) * W + x;
                const float d = c->depth[i];
                uint8_t m = 0;
                if (valid_depth(d)) {
                    double q[3] = {x, y, 1.0}, ray[3], Xc[3], Xw[3];
                    mat3_vec(Ki, q, ray);
                    for (int a = 0; a < 3; ++a) Xc[a] = (double)d * ray[a] - t[a];
                    for (int a = 0; a < 3; ++a) Xw[a] = R[a] * Xc[0] + R[3 + a] * Xc[1] + R[6 + a] * Xc[2];  /* R^T */
                    m = Xw[0] >= box[0] && Xw[1] >= box[1] && Xw[2] >= box[2] && Xw[0] <= box[3] && Xw[1] <= box[4] &&
                        Xw[2] <= box[5];
                }
                mask[i] = m;
            }
    }
}

/*
 * Inpainting (semi = 0) or semi-transparency (semi = 1) of the crop [x0, x0+cw) x [y0, y0+ch) of
 * output frame O (see the header comment).  mask: F*H*W bytes (nonzero = remove).  Outputs as
 * oc_frustum_filter (nacc = |S(p)| of masked pixels, sumw = the last step's sum of weights);
 * records only for masked pixels.
 */
static int inpaint_body(const oc_clip *c, const oc_params *p, const uint8_t *mask, int O, int x0, int y0, int cw,
                        int ch, int semi, double *out_rgb, double *out_sumw, int64_t *out_nacc, int32_t *mem_count,
                        uint64_t *mem_hash, uint8_t *mem_band) {
    if (p->T < 0 || O < 0 || O >= c->F || !(p->frustum_l > 0) || !(p->near_plane > 0) ||
        !(p->far_plane > p->near_plane) || !(p->sigma_rgb > 0))
        return -1;
    const int ns = 2 * p->T + 1, W = c->W, H = c->H;
    double *Gt = (double *)malloc(sizeof(double) * 12 * ns);
    if (!Gt) return -2;
    for (int j = 0; j < ns; ++j) {
        int J = O - p->T + j;
        double P[12];
        if (J < 0 || J >= c->F) continue;
        oc_compose(c->K + 9 * O, c->w2c + 12 * O, c->K + 9 * J, c->w2c + 12 * J, J == O, P, Gt + 12 * j);
    }
    const double *KO = c->K + 9 * O;
    long long n = (long long)cw * ch;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long i = 0; i < n; ++i) {
        const int u = x0 + (int)(i % cw), v = y0 + (int)(i / cw);
        const size_t pix = ((size_t)O * H + v) * W + u;
        double ref[3] = {c->rgb[3 * pix], c->rgb[3 * pix + 1], c->rgb[3 * pix + 2]}, sw = 0.0;
        int64_t cnt = 0;
        if (mem_count)
            for (int j = 0; j < ns; ++j) {
                mem_count[i * ns + j] = 0;
                mem_hash[i * ns + j] = 0;
                mem_band[i * ns + j] = 0;
            }
        if (mask[pix]) {
            /* S(p): colours, mask flags, O-camera positions and frames of every sample */
            size_t cap = 1024, m = 0;
            double *col = (double *)malloc(sizeof(double) * 3 * cap);
            double *pos = (double *)malloc(sizeof(double) * 4 * cap);
            uint8_t *msk = (uint8_t *)malloc(cap);
            for (int j = 0; j < ns && col && pos && msk; ++j) {
                const int J = O - p->T + j;
                if (J < 0 || J >= c->F) continue;
                const double *G = Gt + 12 * j;
                int32_t mc = 0;
                uint64_t mh = 0;
                uint8_t mb = 0;
                for (int qy = 0; qy < H; ++qy)
                    for (int qx = 0; qx < W; ++qx) {
                        const size_t qi = ((size_t)J * H + qy) * W + qx;
                        const float dq = c->depth[qi];
                        if (!valid_depth(dq)) continue;
                        double q3[3] = {qx * (double)dq, qy * (double)dq, (double)dq}, X[3];
                        apply34(G, q3, X);
                        int band;
                        const int in = in_frustum(KO, X, u, v, p, &band);
                        mb |= (uint8_t)band;
                        if (!in) continue;
                        if (m == cap) {
                            cap *= 2;
                            double *c2 = (double *)realloc(col, sizeof(double) * 3 * cap);
                            double *p2 = (double *)realloc(pos, sizeof(double) * 4 * cap);
                            uint8_t *m2 = (uint8_t *)realloc(msk, cap);
                            if (!c2 || !p2 || !m2) {
                                free(c2 ? c2 : col);
                                free(p2 ? p2 : pos);
                                free(m2 ? m2 : msk);
                                col = NULL;
                                pos = NULL;
                                msk = NULL;
                                break;
                            }
                            col = c2;
                            pos = p2;
                            msk = m2;
                        }
                        for (int a = 0; a < 3; ++a) col[3 * m + a] = c->rgb[3 * qi + a];
                        for (int a = 0; a < 3; ++a) pos[4 * m + a] = X[a];
                        pos[4 * m + 3] = J;
                        msk[m] = mask[qi] != 0;
                        ++m;
                        ++mc;
                        mh += mix64((uint64_t)qy * (uint64_t)W + (uint64_t)qx + 1u);
                    }
                if (mem_count) {
                    mem_count[i * ns + j] = mc;
                    mem_hash[i * ns + j] = mh;
                    mem_band[i * ns + j] = mb;
                }
                if (!col) break;
            }
            if (!col || !pos || !msk) {
#pragma omp atomic write
                err = 1;
            } else if (m > 0) {
                /* semi-transparency: the pixel's own sample s_I = (I_O(p), x_ref, O) */
                double sI[7] = {ref[0], ref[1], ref[2], 0.0, 0.0, 0.0, (double)O};
                const float dp = c->depth[pix];
                const int has_sI = semi && valid_depth(dp);
                if (has_sI) {
                    double KOi[9], uv1[3] = {u, v, 1.0}, ray[3];
                    mat3_inverse(KO, KOi);
                    mat3_vec(KOi, uv1, ray);
                    for (int a = 0; a < 3; ++a) sI[3 + a] = (double)dp * ray[a];
                }
                /* Eq. 8: the mean of all samples */
                double acc[3] = {0, 0, 0};
                for (size_t k = 0; k < m; ++k)
                    for (int a = 0; a < 3; ++a) acc[a] += col[3 * k + a];
                for (int a = 0; a < 3; ++a) ref[a] = acc[a] / (double)m;
                /* Eq. 9, two steps (the second with the added Eq. 4 weight for semi-transparency) */
                for (int step = 0; step < 2; ++step) {
                    const int add4 = has_sI && step == 1;
                    double num[3] = {0, 0, 0}, den = 0.0;
                    for (size_t k = 0; k < m; ++k) {
                        if (msk[k] && !add4) continue;
                        double w = 0.0;
                        if (!msk[k]) {
                            double d2 = 0.0;
                            for (int a = 0; a < 3; ++a) d2 += (col[3 * k + a] - ref[a]) * (col[3 * k + a] - ref[a]);
                            w = exp(-d2 / (2.0 * p->sigma_rgb * p->sigma_rgb));
                        }
                        if (add4) {
                            const double sk[7] = {col[3 * k], col[3 * k + 1], col[3 * k + 2], pos[4 * k], pos[4 * k + 1],
                                                  pos[4 * k + 2], pos[4 * k + 3]};
                            w += oc_weight_denoise(sk, sI, p->sigma_rgb, p->sigma_xyz, p->sigma_f);
                        }
                        for (int a = 0; a < 3; ++a) num[a] += w * col[3 * k + a];
                        den += w;
                    }
                    sw = den;
                    if (den > 0.0)
                        for (int a = 0; a < 3; ++a) ref[a] = num[a] / den;
                }
            }
            cnt = (int64_t)m;
            free(col);
            free(pos);
            free(msk);
        }
        for (int a = 0; a < 3; ++a) out_rgb[3 * i + a] = ref[a];
        out_sumw[i] = sw;
        out_nacc[i] = cnt;
    }
    free(Gt);
    return err ? -2 : 0;
}

int oc_inpaint_filter(const oc_clip *c, const oc_params *p, const uint8_t *mask, int O, int x0, int y0, int cw, int ch,
                      double *out_rgb, double *out_sumw, int64_t *out_nacc, int32_t *mem_count, uint64_t *mem_hash,
                      uint8_t *mem_band) {
    return inpaint_body(c, p, mask, O, x0, y0, cw, ch, 0, out_rgb, out_sumw, out_nacc, mem_count, mem_hash, mem_band);
}

int oc_semitransparent_filter(const oc_clip *c, const oc_params *p, const uint8_t *mask, int O, int x0, int y0, int cw,
                              int ch, double *out_rgb, double *out_sumw, int64_t *out_nacc, int32_t *mem_count,
                              uint64_t *mem_hash, uint8_t *mem_band) {
    if (!(p->sigma_xyz > 0) || !(p->sigma_f > 0)) return -1;
    return inpaint_body(c, p, mask, O, x0, y0, cw, ch, 1, out_rgb, out_sumw, out_nacc, mem_count, mem_hash, mem_band);
}

/*
 * Brute force: test EVERY pixel of frame J against the radius around x_ref of pixel (u, v) of
 * frame O, against its aperture cone in mode 1 (no window, no box), or against its frustum when
 * gather = 1.  accept is H*W bytes (1 accepted, 0 not); returns the count.
 */
long long oc_bruteforce(const oc_clip *c, const oc_params *p, int O, int u, int v, int J, uint8_t *accept) {
    const int W = c->W, H = c->H;
    double P[12], G[12], KOi[9], ray[3], xref[3];
    oc_compose(c->K + 9 * O, c->w2c + 12 * O, c->K + 9 * J, c->w2c + 12 * J, J == O, P, G);
    float dref = c->depth[((size_t)O * H + v) * W + u];
    memset(accept, 0, (size_t)W * H);
    if (!valid_depth(dref)) return 0;
    mat3_inverse(c->K + 9 * O, KOi);
    double uv1[3] = {u, v, 1.0};
    mat3_vec(KOi, uv1, ray);
    for (int i = 0; i < 3; ++i) xref[i] = (double)dref * ray[i];
    double rr = ray[0] * ray[0] + ray[1] * ray[1] + ray[2] * ray[2];
    long long cnt = 0;
    for (int qy = 0; qy < H; ++qy) {
        for (int qx = 0; qx < W; ++qx) {
            float dq = c->depth[((size_t)J * H + qy) * W + qx];
            if (!valid_depth(dq)) continue;
            double q3[3] = {qx * (double)dq, qy * (double)dq, (double)dq}, X[3];
            apply34(G, q3, X);
            int ok;
            if (p->gather == 1) {
                int band;
                ok = in_frustum(c->K + 9 * O, X, u, v, p, &band);
            } else if (p->mode == 1) {
                double xr = X[0] * ray[0] + X[1] * ray[1] + X[2] * ray[2];
                double t = xr / rr;
                double cr0 = X[1] * ray[2] - X[2] * ray[1], cr1 = X[2] * ray[0] - X[0] * ray[2],
                       cr2 = X[0] * ray[1] - X[1] * ray[0];
                double qperp = sqrt((cr0 * cr0 + cr1 * cr1 + cr2 * cr2) / rr);
                ok = qperp < p->a0 + p->aperture * fabs(p->focal_depth - t) / p->focal_depth;
            } else {
                double d2 = (X[0] - xref[0]) * (X[0] - xref[0]) + (X[1] - xref[1]) * (X[1] - xref[1]) +
                            (X[2] - xref[2]) * (X[2] - xref[2]);
                ok = d2 < p->radius * p->radius;
            }
            if (ok) { accept[(size_t)qy * W + qx] = 1; ++cnt; }
        }
    }
    return cnt;
}

/* ================================================================== learned per-sample weights
 *
 * Samples (the capped set): the first n <= 64 accepted samples of S(p) in canonical order --
 * frames J = O, O-1, O+1, O-2, O+2, ... (the earlier frame first on ties), then the k x k window
 * in raster order.  Features of a sample s gathered from pixel q of frame J (16 per sample):
 *   [c_s (3), c_s - c_ref (3), |X_q - x_ref| / r, (J - O) / max(T, 1), (d_q - z'_J) / r,
 *    log w_denoise(s) (Eq. 4, natural log), 1, |S(p)| / 64, c_s - plain (3), 0]
 * (|S(p)| the size of the whole gathered set, which the plain fallback averages, and plain the
 * Eq. 4 result over it: the network sees each sample against the robust estimate it may replace)
 * with z'_J the depth of the reference point in camera J.  Network: h = ReLU(W1 f + b1) (64),
 * (z_w, z_c) = W2 h + b2; w_s = softplus(z_w); conf = mean_s sigmoid(z_c);
 * learned output = sum w_s c_s / sum w_s; final output = learned if conf >= tau else the plain
 * Eq. 4 result.  With round_bf16 = 1 the features, W1, W2 and the hidden activations (after the
 * ReLU) are rounded to BF16 -- the input precision of the tensor-core products of both layers --
 * and b1, b2 to FP32 before use, as on the GPU.  The backward pass treats that rounding of h as
 * the identity (the gradient of W2 uses the rounded h).
 */
#define OC_MAXS 64
#define OC_NF 16
#define OC_NH 64

static double bf16_round(double x) {
    float f = (float)x;
    uint32_t b;
    memcpy(&b, &f, 4);
    if ((b & 0x7f800000u) != 0x7f800000u) {
        b += 0x7fffu + ((b >> 16) & 1u);
        b &= 0xffff0000u;
    }
    memcpy(&f, &b, 4);
    return (double)f;
}

/* Capped sample set, features and colours of pixel (u, v) of frame O; *n receives the count.
 * plain receives the Eq. 4 output over the whole S(p).  Returns 0, or -1 for an invalid
 * reference depth (then n = 0 and plain = c_ref). */
int oc_learned_samples(const oc_clip *c, const oc_params *p, int O, int u, int v, double *feat, double *col,
                       int *n, double *plain) {
    const int W = c->W, H = c->H, F = c->F, k = p->k, h = (k - 1) / 2;
    double sumw;
    int64_t nacc, nexam;
    double Pt[12], Gt[12];
    *n = 0;
    memset(feat, 0, sizeof(double) * OC_MAXS * OC_NF);
    memset(col, 0, sizeof(double) * OC_MAXS * 3);
    /* the plain result over all of S(p) */
    {
        int ns = 2 * p->T + 1;
        double *PP = (double *)malloc(sizeof(double) * 12 * ns), *GG = (double *)malloc(sizeof(double) * 12 * ns);
        for (int j = 0; j < ns; ++j) {
            int J = O - p->T + j;
            if (J < 0 || J >= F) continue;
            oc_compose(c->K + 9 * O, c->w2c + 12 * O, c->K + 9 * J, c->w2c + 12 * J, J == O, PP + 12 * j, GG + 12 * j);
        }
        oc_params pd = *p;
        pd.mode = 0;
        pixel(c, &pd, O, u, v, PP, GG, plain, &sumw, &nacc, &nexam, NULL, 0);
        free(PP);
        free(GG);
    }
    size_t pix = ((size_t)O * H + v) * W + u;
    float dref_f = c->depth[pix];
    if (!valid_depth(dref_f)) return -1;
    double dref = dref_f, cref[3] = {c->rgb[3 * pix], c->rgb[3 * pix + 1], c->rgb[3 * pix + 2]};
    double KOi[9], ray[3], xref[3], uv1[3] = {u, v, 1.0};
    mat3_inverse(c->K + 9 * O, KOi);
    mat3_vec(KOi, uv1, ray);
    for (int i = 0; i < 3; ++i) xref[i] = dref * ray[i];
    const double r = p->radius, Tn = p->T > 0 ? p->T : 1, ntot = (double)nacc / 64.0;
    for (int t = 0; t <= 2 * p->T && *n < OC_MAXS; ++t) {
        /* canonical frame order: O, O-1, O+1, O-2, O+2, ... */
        int J = O + (t == 0 ? 0 : ((t & 1) ? -(t + 1) / 2 : t / 2));
        if (J < 0 || J >= F) continue;
        oc_compose(c->K + 9 * O, c->w2c + 12 * O, c->K + 9 * J, c->w2c + 12 * J, J == O, Pt, Gt);
        double xp[3];
        apply34(Pt, xref, xp);
        if (xp[2] <= 1e-6 * dref) continue;
        double up = xp[0] / xp[2], vp = xp[1] / xp[2];
        double cxd = floor(up + 0.5), cyd = floor(vp + 0.5);
        if (cxd < -(double)(4 * k + 8) || cxd > (double)(W + 4 * k + 8) || cyd < -(double)(4 * k + 8) ||
            cyd > (double)(H + 4 * k + 8))
            continue;
        const double zJ = xp[2];
        for (int dy = -h; dy <= h && *n < OC_MAXS; ++dy) {
            for (int dx = -h; dx <= h && *n < OC_MAXS; ++dx) {
                int qx = (int)cxd + dx, qy = (int)cyd + dy;
                if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
                size_t qi = ((size_t)J * H + qy) * W + qx;
                float dq = c->depth[qi];
                if (!valid_depth(dq)) continue;
                double q3[3] = {qx * (double)dq, qy * (double)dq, (double)dq}, X[3];
                apply34(Gt, q3, X);
                double d2 = (X[0] - xref[0]) * (X[0] - xref[0]) + (X[1] - xref[1]) * (X[1] - xref[1]) +
                            (X[2] - xref[2]) * (X[2] - xref[2]);
                if (!(d2 < r * r)) continue;
                double *f = feat + (size_t)*n * OC_NF, cs[3] = {c->rgb[3 * qi], c->rgb[3 * qi + 1], c->rgb[3 * qi + 2]};
                double s[7] = {cs[0], cs[1], cs[2], X[0], X[1], X[2], J};
                double sr[7] = {cref[0], cref[1], cref[2], xref[0], xref[1], xref[2], O};
                for (int i = 0; i < 3; ++i) { f[i] = cs[i]; f[3 + i] = cs[i] - cref[i]; col[3 * *n + i] = cs[i]; }
                f[6] = sqrt(d2) / r;
                f[7] = (J - O) / Tn;
                f[8] = ((double)dq - zJ) / r;
                f[9] = log(oc_weight_denoise(s, sr, p->sigma_rgb, p->sigma_xyz, p->sigma_f));
                f[10] = 1.0;
                f[11] = ntot;
                /* the sample against the plain Eq. 4 estimate of the whole set */
                for (int i = 0; i < 3; ++i) f[12 + i] = cs[i] - plain[i];
                ++*n;
            }
        }
    }
    return 0;
}

static double softplus(double z) { return z > 0 ? z + log1p(exp(-z)) : log1p(exp(z)); }
static double sigm(double z) { return z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z)); }

/* Forward pass of one pixel: z (n x 2) and h (n x 64) may be NULL.  Returns conf. */
double oc_mlp_pixel(const double *feat, const double *col, int n, const double *W1, const double *b1,
                    const double *W2, const double *b2, int round_bf16, double tau, const double *plain,
                    double *out_learned, double *out_final, double *z, double *hid) {
    double acc[3] = {0, 0, 0}, Wsum = 0.0, csum = 0.0;
    for (int s = 0; s < n; ++s) {
        double f[OC_NF], hh[OC_NH], zz[2];
        for (int i = 0; i < OC_NF; ++i) f[i] = round_bf16 ? bf16_round(feat[s * OC_NF + i]) : feat[s * OC_NF + i];
        for (int j = 0; j < OC_NH; ++j) {
            double a = round_bf16 ? (double)(float)b1[j] : b1[j];
            for (int i = 0; i < OC_NF; ++i) a += (round_bf16 ? bf16_round(W1[j * OC_NF + i]) : W1[j * OC_NF + i]) * f[i];
            hh[j] = a > 0 ? (round_bf16 ? bf16_round(a) : a) : 0.0;
        }
        for (int o = 0; o < 2; ++o) {
            double a = round_bf16 ? (double)(float)b2[o] : b2[o];
            for (int j = 0; j < OC_NH; ++j) a += (round_bf16 ? bf16_round(W2[o * OC_NH + j]) : W2[o * OC_NH + j]) * hh[j];
            zz[o] = a;
        }
        if (z) { z[2 * s] = zz[0]; z[2 * s + 1] = zz[1]; }
        if (hid) memcpy(hid + (size_t)s * OC_NH, hh, sizeof(hh));
        double w = softplus(zz[0]);
        for (int ch = 0; ch < 3; ++ch) acc[ch] += w * col[3 * s + ch];
        Wsum += w;
        csum += sigm(zz[1]);
    }
    double conf = n > 0 ? csum / n : 0.0;
    for (int ch = 0; ch < 3; ++ch) {
        out_learned[ch] = Wsum > 0 ? acc[ch] / Wsum : plain[ch];
        out_final[ch] = (n > 0 && conf >= tau) ? out_learned[ch] : plain[ch];
    }
    return conf;
}

/*
 * Training loss and gradients over n_px pixels (feature blocks of 64 x 16, colours 64 x 3):
 *   L = (1/n_px) sum_p [ mean_c (o_p - y_p)^2 + bce_w BCE(clamp(conf_p), t_p) ],
 *   t_p = 1 if mean_c (o_p - y_p)^2 <= mean_c (plain_p - y_p)^2 else 0 (a constant target),
 * o_p the learned output, conf clamped to [1e-6, 1 - 1e-6].  Gradients (same layout as the
 * weights) are overwritten.  Returns L.
 *
 * aW1, ab1, aW2, ab2 (each may be NULL) receive, per gradient entry, the same sum taken over the
 * absolute values of its terms (|dh_j fr_i|, |dh_j|, |dz_o h_j|, |dz_o|, divided by n_px): the
 * scale against which a rounding error in the terms of that entry is measured.
 */
double oc_mlp_loss_grad(int n_px, const double *feat, const double *col, const int *nsamp, const double *plain,
                        const double *clean, const double *W1, const double *b1, const double *W2, const double *b2,
                        int round_bf16, double bce_w, double *gW1, double *gb1, double *gW2, double *gb2,
                        double *aW1, double *ab1, double *aW2, double *ab2) {
    memset(gW1, 0, sizeof(double) * OC_NH * OC_NF);
    memset(gb1, 0, sizeof(double) * OC_NH);
    memset(gW2, 0, sizeof(double) * 2 * OC_NH);
    memset(gb2, 0, sizeof(double) * 2);
    if (aW1) memset(aW1, 0, sizeof(double) * OC_NH * OC_NF);
    if (ab1) memset(ab1, 0, sizeof(double) * OC_NH);
    if (aW2) memset(aW2, 0, sizeof(double) * 2 * OC_NH);
    if (ab2) memset(ab2, 0, sizeof(double) * 2);
    double L = 0.0;
    double *z = (double *)malloc(sizeof(double) * OC_MAXS * 2), *hid = (double *)malloc(sizeof(double) * OC_MAXS * OC_NH);
    for (int p = 0; p < n_px; ++p) {
        const double *f = feat + (size_t)p * OC_MAXS * OC_NF, *cl = col + (size_t)p * OC_MAXS * 3, *y = clean + 3 * p;
        int n = nsamp[p];
        if (n <= 0) continue;
        double ol[3], of[3];
        double conf = oc_mlp_pixel(f, cl, n, W1, b1, W2, b2, round_bf16, 0.5, plain + 3 * p, ol, of, z, hid);
        double el = 0, ep = 0;
        for (int ch = 0; ch < 3; ++ch) {
            el += (ol[ch] - y[ch]) * (ol[ch] - y[ch]) / 3.0;
            ep += (plain[3 * p + ch] - y[ch]) * (plain[3 * p + ch] - y[ch]) / 3.0;
        }
        double t = el <= ep ? 1.0 : 0.0;
        double cc = conf < 1e-6 ? 1e-6 : (conf > 1 - 1e-6 ? 1 - 1e-6 : conf);
        L += el - bce_w * (t * log(cc) + (1 - t) * log(1 - cc));
        /* d/d o_c and d/d conf (the clamp passes the gradient through only inside the interval) */
        double dO[3], Wsum = 0.0;
        for (int ch = 0; ch < 3; ++ch) dO[ch] = 2.0 * (ol[ch] - y[ch]) / 3.0;
        double dconf = (conf > 1e-6 && conf < 1 - 1e-6) ? bce_w * (cc - t) / (cc * (1 - cc)) : 0.0;
        for (int s = 0; s < n; ++s) Wsum += softplus(z[2 * s]);
        for (int s = 0; s < n; ++s) {
            double dw = 0.0;
            for (int ch = 0; ch < 3; ++ch) dw += dO[ch] * (cl[3 * s + ch] - ol[ch]) / Wsum;
            double dz[2] = {dw * sigm(z[2 * s]), dconf * sigm(z[2 * s + 1]) * (1 - sigm(z[2 * s + 1])) / n};
            const double *hh = hid + (size_t)s * OC_NH;
            double fr[OC_NF];
            for (int i = 0; i < OC_NF; ++i) fr[i] = round_bf16 ? bf16_round(f[s * OC_NF + i]) : f[s * OC_NF + i];
            for (int o = 0; o < 2; ++o) {
                gb2[o] += dz[o];
                if (ab2) ab2[o] += fabs(dz[o]);
                for (int j = 0; j < OC_NH; ++j) {
                    gW2[o * OC_NH + j] += dz[o] * hh[j];
                    if (aW2) aW2[o * OC_NH + j] += fabs(dz[o] * hh[j]);
                }
            }
            for (int j = 0; j < OC_NH; ++j) {
                if (hh[j] <= 0.0) continue;
                double w20 = round_bf16 ? bf16_round(W2[j]) : W2[j], w21 = round_bf16 ? bf16_round(W2[OC_NH + j]) : W2[OC_NH + j];
                double dh = dz[0] * w20 + dz[1] * w21;
                gb1[j] += dh;
                if (ab1) ab1[j] += fabs(dh);
                for (int i = 0; i < OC_NF; ++i) {
                    gW1[j * OC_NF + i] += dh * fr[i];
                    if (aW1) aW1[j * OC_NF + i] += fabs(dh * fr[i]);
                }
            }
        }
    }
    free(z);
    free(hid);
    double inv = n_px > 0 ? 1.0 / n_px : 0.0;
    for (int i = 0; i < OC_NH * OC_NF; ++i) gW1[i] *= inv;
    for (int i = 0; i < OC_NH; ++i) gb1[i] *= inv;
    for (int i = 0; i < 2 * OC_NH; ++i) gW2[i] *= inv;
    for (int i = 0; i < 2; ++i) gb2[i] *= inv;
    for (int i = 0; aW1 && i < OC_NH * OC_NF; ++i) aW1[i] *= inv;
    for (int i = 0; ab1 && i < OC_NH; ++i) ab1[i] *= inv;
    for (int i = 0; aW2 && i < 2 * OC_NH; ++i) aW2[i] *= inv;
    for (int i = 0; ab2 && i < 2; ++i) ab2[i] *= inv;
    return L * inv;
}

/* oc_learned_samples over a crop (row-major): feat cw*ch*64*16, col cw*ch*64*3, nsamp, plain cw*ch*3 */
void oc_learned_crop(const oc_clip *c, const oc_params *p, int O, int x0, int y0, int cw, int ch, double *feat,
                     double *col, int32_t *nsamp, double *plain) {
    long long n = (long long)cw * ch;
#pragma omp parallel for schedule(dynamic, 8)
    for (long long i = 0; i < n; ++i) {
        int cnt = 0;
        oc_learned_samples(c, p, O, x0 + (int)(i % cw), y0 + (int)(i / cw), feat + i * OC_MAXS * OC_NF,
                           col + i * OC_MAXS * 3, &cnt, plain + 3 * i);
        nsamp[i] = cnt;
    }
}
