// ssvp_frustum.cu - the paper's frustum gather (Sec. "Sample Gathering", Eq. 1-2) fused with the
// Eq. 3/4 filter.  One thread per output pixel, window frames in order.
//
// Per (pixel p, frame J):
//   1. The frustum V of Eq. 1 (the l x l square around p swept over O depths [near, far]) is
//      clipped to frame J's valid-depth slab [zlo_J, zhi_J] (no pixel of J has a depth outside
//      it, so nothing is lost) and projected into J: the 12 edges of V are clipped in O depth
//      and their end points projected.  A parallelogram along the projected central ray bounds
//      that hull (grown by a rounding margin); only its pixels are tested.
//   2. Each pixel q in it with depth d is back-projected into O through the homogeneous map
//      h = M_{O<-J} (q_x d, q_y d, d) + e_{O<-J}; it is a sample when near < h_3 < far and
//      |h_1 - u h_3| + |h_2 - v h_3| < (l / 2) h_3, which is Eq. 2's L1 test multiplied by the
//      positive O depth h_3.
//   3. Samples are weighted by Eq. 4 around s_ref (times the per-frame factors of Eq. 5, or by
//      Eq. 10's shutter function alone) and reduced by Eq. 3, as in the window gather.
#include <cuda_fp16.h>

#include <algorithm>

#include "../../include/ssvp.h"
#include "ssvp_df.cuh"
#include "ssvp_internal.h"

namespace ssvp {
namespace {

constexpr int kFrTileX = 32, kFrTileY = 8, kFrThreads = kFrTileX * kFrTileY;

// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014); debug records sum it over the
// linear indices qy * W + qx + 1 of a sample set, an order-independent membership checksum.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Bound of the projected hull: minor = b * major + [lo, hi], major in [mlo, mhi].
struct HullBound {
    float b, lo, hi, mlo, mhi;
    bool xmajor, any;
};

__device__ __forceinline__ void bound_add(HullBound &hb, float px, float py) {
    const float maj = hb.xmajor ? px : py, mnr = hb.xmajor ? py : px;
    const float ic = fmaf(-hb.b, maj, mnr);
    hb.lo = fminf(hb.lo, ic);
    hb.hi = fmaxf(hb.hi, ic);
    hb.mlo = fminf(hb.mlo, maj);
    hb.mhi = fmaxf(hb.mhi, maj);
    hb.any = true;
}

// Interval of t in [t0, t1] where w(t) = w0 + t dw lies in [zlo, zhi]; false when empty.
__device__ __forceinline__ bool slab_interval(float w0, float dw, float zlo, float zhi, float t0, float t1, float &ta,
                                              float &tb) {
    if (dw != 0.0f) {
        const float sa = (zlo - w0) / dw, sb = (zhi - w0) / dw;
        ta = fmaxf(t0, fminf(sa, sb));
        tb = fminf(t1, fmaxf(sa, sb));
    } else {
        if (!(w0 >= zlo && w0 <= zhi)) return false;
        ta = t0;
        tb = t1;
    }
    return ta <= tb;
}

// Lateral edge of V through the O pixel point (cu, cv): h(z) = z A + e for O depth z.
__device__ __forceinline__ void lateral_edge(const float *M, const float *e, float cu, float cv, float nearp,
                                             float farp, float zlo, float zhi, HullBound &hb) {
    const float A0 = fmaf(M[0], cu, fmaf(M[1], cv, M[2]));
    const float A1 = fmaf(M[3], cu, fmaf(M[4], cv, M[5]));
    const float A2 = fmaf(M[6], cu, fmaf(M[7], cv, M[8]));
    float za, zb;
    // J depth along the edge: A2 z + e2
    if (!slab_interval(e[2], A2, zlo, zhi, nearp, farp, za, zb)) return;
    // the interval above is in units of z (w0 = e2 at z = 0), clipped to [near, far]
    const float wa = fmaf(A2, za, e[2]), wb = fmaf(A2, zb, e[2]);
    if (wa > 0.0f) bound_add(hb, fmaf(A0, za, e[0]) / wa, fmaf(A1, za, e[1]) / wa);
    if (wb > 0.0f) bound_add(hb, fmaf(A0, zb, e[0]) / wb, fmaf(A1, zb, e[1]) / wb);
}

// Edge of the near or far face of V at O depth z0, from O pixel point (cu, cv) to (cu', cv').
__device__ __forceinline__ void face_edge(const float *M, const float *e, float z0, float cu, float cv, float du,
                                          float dv, float zlo, float zhi, HullBound &hb) {
    // h(s) = z0 M (cu + s du, cv + s dv, 1) + e, s in [0, 1]
    const float P0 = fmaf(z0, fmaf(M[0], cu, fmaf(M[1], cv, M[2])), e[0]);
    const float P1 = fmaf(z0, fmaf(M[3], cu, fmaf(M[4], cv, M[5])), e[1]);
    const float P2 = fmaf(z0, fmaf(M[6], cu, fmaf(M[7], cv, M[8])), e[2]);
    const float D0 = z0 * fmaf(M[0], du, M[1] * dv), D1 = z0 * fmaf(M[3], du, M[4] * dv),
                D2 = z0 * fmaf(M[6], du, M[7] * dv);
    float sa, sb;
    if (!slab_interval(P2, D2, zlo, zhi, 0.0f, 1.0f, sa, sb)) return;
    const float wa = fmaf(D2, sa, P2), wb = fmaf(D2, sb, P2);
    if (wa > 0.0f) bound_add(hb, fmaf(D0, sa, P0) / wa, fmaf(D1, sa, P1) / wa);
    if (wb > 0.0f) bound_add(hb, fmaf(D0, sb, P0) / wb, fmaf(D1, sb, P1) / wb);
}

// SR: super-resolution (Sec. "Super resolution", Eq. 6-7) on the a.sr_scale-times output grid;
// the maps use the output-grid camera of O, s_ref is bilinear in the input frame, and the
// exponent gains Eq. 7's area term.
// INP: inpainting (Sec. "Inpainting and semi-transparency", Eq. 8-9): only pixels with a mask
// gather; three passes over S(p): the mean of all samples (Eq. 8), then two steps of the
// colour-weighted mean over unmasked samples (Eq. 9), each around the previous result.
// INP == 2: semi-transparency (the same section, after Eq. 9): in the last pass every sample,
// masked or not, also weighs the Eq. 4 weight around the pixel's own sample (I(p), x_ref, O),
// so the object's samples near x_ref blend with the background's mean-shift estimate.
// Fast path of the hull: the 4 lateral rays of the frustum, h(z) = z A + e, clipped to the slab
// alone.  Valid (returns true) when every ray's depth in J grows (or every one falls) with z and
// every clipped interval lies strictly inside (near, far): then no face of V touches the slab,
// every point of V in the slab has its O depth inside (near, far), and the hull is that of the
// 8 end points, which are projected here with approximate reciprocals (the bound's margin
// covers their error).
// corner c = 0..3 of the l x l square around (u, v), counter-clockwise from (u - L, v - L)
__device__ __forceinline__ float corner_u(int c, float u, float L) { return (c == 1 || c == 2) ? u + L : u - L; }
__device__ __forceinline__ float corner_v(int c, float v, float L) { return c >= 2 ? v + L : v - L; }

__device__ __forceinline__ bool lateral_fast(const float *M, const float *e, float u, float v, float L, float nearp,
                                             float farp, float zlo, float zhi, HullBound &hb) {
    float sgn = 0.0f;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float cu = corner_u(c, u, L), cv = corner_v(c, v, L);
        const float A0 = fmaf(M[0], cu, fmaf(M[1], cv, M[2]));
        const float A1 = fmaf(M[3], cu, fmaf(M[4], cv, M[5]));
        const float A2 = fmaf(M[6], cu, fmaf(M[7], cv, M[8]));
        const float s = A2 > 0.0f ? 1.0f : (A2 < 0.0f ? -1.0f : 0.0f);
        ok = ok && s != 0.0f && (c == 0 || s == sgn);
        sgn = s;
        const float r = rcp_approx(A2);
        const float sa = (zlo - e[2]) * r, sb = (zhi - e[2]) * r;
        const float za = fminf(sa, sb), zb = fmaxf(sa, sb);
        ok = ok && za > nearp * 1.0001f && zb < farp * 0.9999f;
        const float wa = fmaf(A2, za, e[2]), wb = fmaf(A2, zb, e[2]);
        const float ra = rcp_approx(wa), rb = rcp_approx(wb);
        ok = ok && wa > 0.0f && wb > 0.0f;
        bound_add(hb, fmaf(A0, za, e[0]) * ra, fmaf(A1, za, e[1]) * ra);
        bound_add(hb, fmaf(A0, zb, e[0]) * rb, fmaf(A1, zb, e[1]) * rb);
    }
    return ok;
}

template <int CFMT, bool DEBUG, bool SR, int INP>
__global__ void __launch_bounds__(kFrThreads, 3) frustum_kernel(const GatherArgs a) {
    __shared__ float s_const[4];
    __shared__ unsigned long long s_cnt[2][kFrThreads / 32];
    __shared__ float s_w[kFrThreads / 32];
    const Planes &P = a.clip;
    const int oi = blockIdx.z;
    const int O = a.frame_begin + oi;
    if (threadIdx.x == 0) {
        const float r = a.radius > 0.0f ? a.radius : -a.radius * *P.median;
        const float sx = a.sigma_xyz > 0.0f ? a.sigma_xyz : r;
        // the shutter weight of Eq. 10 replaces Eq. 4: no colour and no position term
        const bool shutter = a.mode == SSVP_MODE_SHUTTER;
        s_const[0] = shutter ? 0.0f : kLog2e / (2.0f * a.sigma_rgb * a.sigma_rgb);
        s_const[1] = shutter || INP == 1 ? 0.0f : kLog2e / (2.0f * sx * sx);
        s_const[2] = a.mode == SSVP_MODE_MEAN ? 0.0f : 1.0f;
        if (SR) {
            // sigma_area <= 0: one input-pixel footprint at the median depth (median / fx_O); the
            // back map of slot T (J = O) carries the output-grid 1 / fx of O
            const float ifx_grid = a.geom_back[(long long)oi * a.n_slots + a.T].ifx;
            const float sa = a.sigma_area > 0.0f ? a.sigma_area : *P.median * ifx_grid * (float)a.sr_scale;
            s_const[3] = kLog2e / (2.0f * sa * sa);
        }
    }
    __syncthreads();
    const float a_rgb = s_const[0], a_xyz = s_const[1], a_area = SR ? s_const[3] : 0.0f;
    const bool weighted = s_const[2] != 0.0f;
    const int Wo = SR ? P.W * a.sr_scale : P.W;
    const int Ho = SR ? P.H * a.sr_scale : P.H;

    const int u = a.x0 + blockIdx.x * kFrTileX + (threadIdx.x % kFrTileX);
    const int v = a.y0 + blockIdx.y * kFrTileY + (threadIdx.x / kFrTileX);
    const bool active = u < a.x0 + a.cw && v < a.y0 + a.ch;
    const long long crop_idx = (long long)(v - a.y0) * a.cw + (u - a.x0);
    const float L = 0.5f * a.frustum_l, nearp = a.near_plane, farp = a.far_plane;
    const float zmid = 0.5f * (nearp + farp), zhalf = 0.5f * (farp - nearp);
    const int ns = a.n_slots;

    float3 cref = make_float3(0.f, 0.f, 0.f);
    float dref = 0.0f;
    if (active && !SR) {
        const long long pix = (long long)O * P.fstride + (long long)(v + kPad) * P.pitch + (u + kPad);
        dref = __ldg(P.depth + pix);
        cref = load_colour<CFMT>(P.colour, pix);
    }
    if (active && SR) {
        // bilinear s_ref at input coordinates ((u, v) + 0.5) / scale - 0.5, clamped to the image; an
        // invalid (NaN) depth among the four propagates and invalidates the reference
        const float is = 1.0f / (float)a.sr_scale;
        const float xc = fminf(fmaxf(((float)u + 0.5f) * is - 0.5f, 0.0f), (float)(P.W - 1));
        const float yc = fminf(fmaxf(((float)v + 0.5f) * is - 0.5f, 0.0f), (float)(P.H - 1));
        const int x0 = (int)floorf(xc), y0 = (int)floorf(yc);
        const int x1 = min(x0 + 1, P.W - 1), y1 = min(y0 + 1, P.H - 1);
        const float fx = xc - (float)x0, fy = yc - (float)y0;
        const long long fb = (long long)O * P.fstride;
        const long long p00 = fb + (long long)(y0 + kPad) * P.pitch + (x0 + kPad), p10 = p00 + (x1 - x0);
        const long long p01 = fb + (long long)(y1 + kPad) * P.pitch + (x0 + kPad), p11 = p01 + (x1 - x0);
        const float3 c00 = load_colour<CFMT>(P.colour, p00), c10 = load_colour<CFMT>(P.colour, p10);
        const float3 c01 = load_colour<CFMT>(P.colour, p01), c11 = load_colour<CFMT>(P.colour, p11);
        const float d00 = __ldg(P.depth + p00), d10 = __ldg(P.depth + p10), d01 = __ldg(P.depth + p01),
                    d11 = __ldg(P.depth + p11);
        const float gx = 1.0f - fx, gy = 1.0f - fy;
        cref.x = gy * (gx * c00.x + fx * c10.x) + fy * (gx * c01.x + fx * c11.x);
        cref.y = gy * (gx * c00.y + fx * c10.y) + fy * (gx * c01.y + fx * c11.y);
        cref.z = gy * (gx * c00.z + fx * c10.z) + fy * (gx * c01.z + fx * c11.z);
        dref = gy * (gx * d00 + fx * d10) + fy * (gx * d01 + fx * d11);
    }
    // inpainting gathers for masked pixels only and does not need their depth; the others need
    // a valid reference depth (NaN fails)
    const long long pix_o = (long long)O * P.fstride + (long long)(v + kPad) * P.pitch + (u + kPad);
    const bool gather = INP ? active && __ldg(P.mask + pix_o) != 0 : active && dref > 0.0f;
    if (INP && active) cref = load_colour<CFMT>(P.colour, pix_o);
    // semi-transparency: the pixel's own sample (I(p), x_ref, O) needs a valid depth (NaN fails)
    const float3 c_in = cref;
    const bool own = INP == 2 && dref > 0.0f;
    // Accumulators carry the common factor 2^-m, m the largest log2 weight so far: without the
    // reference sample (outside near / far) every weight can be far below FP32's range while
    // Eq. 3 is still well defined.  The start, -1e30, is below every finite exponent, and a
    // weight of exactly 0 (an exponent of -inf) stays 0.
    constexpr float kNoWeight = -1e30f;
    float acc_r = 0.0f, acc_g = 0.0f, acc_b = 0.0f, acc_w = 0.0f, m_log2 = 0.0f, sw_true = 0.0f;
    long long n_exam = 0;
    int n_acc = 0;
    if (DEBUG && active && !gather && a.membership)
        for (int j = 0; j < ns; ++j) {
            int32_t *rec = a.membership + (crop_idx * ns + j) * 4;
            rec[0] = -2; rec[1] = 0; rec[2] = 0; rec[3] = 0;
        }

    constexpr int kPasses = INP ? 3 : 1;
    for (int pass = 0; pass < kPasses; ++pass) {
    const bool wpass = INP ? pass > 0 : weighted;
    acc_r = acc_g = acc_b = acc_w = 0.0f;
    m_log2 = wpass ? kNoWeight : 0.0f;
    if (gather) {
        for (int j = 0; j < ns; ++j) {
            const PairGeom &gf = a.geom[(long long)oi * ns + j];
            const int J = __ldg(&gf.J);
            int32_t *rec = DEBUG && a.membership && pass == 0 ? a.membership + (crop_idx * ns + j) * 4 : nullptr;
            if (J < 0) {
                if (DEBUG && rec) { rec[0] = -1; rec[1] = 0; rec[2] = 0; rec[3] = 0; }
                continue;
            }
            const PairGeom &gb = a.geom_back[(long long)oi * ns + j];
            // J's valid depth range (order-preserving bit patterns; 0 words: no valid depth)
            const unsigned int zmin_w = __ldg(P.zrange + 2 * J), zmax_w = __ldg(P.zrange + 2 * J + 1);
            const float zlo = zmin_w ? __uint_as_float(~zmin_w) : __int_as_float(0x7f800000);
            const float zhi = __uint_as_float(zmax_w);
            float Mf[9], ef[3];
#pragma unroll
            for (int i = 0; i < 9; ++i) Mf[i] = __ldg(&gf.M_hi[i]);
#pragma unroll
            for (int i = 0; i < 3; ++i) ef[i] = __ldg(&gf.e_hi[i]);
            // ---- 1. bound of the projected frustum, clipped to the slab
            HullBound hb;
            hb.any = false;
            hb.xmajor = true;
            hb.b = 0.0f;
            {
                // direction of the projected central ray (its clipped end points), for the slope
                const float A0 = fmaf(Mf[0], (float)u, fmaf(Mf[1], (float)v, Mf[2]));
                const float A1 = fmaf(Mf[3], (float)u, fmaf(Mf[4], (float)v, Mf[5]));
                const float A2 = fmaf(Mf[6], (float)u, fmaf(Mf[7], (float)v, Mf[8]));
                float za, zb;
                if (zlo <= zhi && slab_interval(ef[2], A2, zlo, zhi, nearp, farp, za, zb)) {
                    const float wa = fmaf(A2, za, ef[2]), wb = fmaf(A2, zb, ef[2]);
                    const float xa = fmaf(A0, za, ef[0]) / wa, ya = fmaf(A1, za, ef[1]) / wa;
                    const float xb = fmaf(A0, zb, ef[0]) / wb, yb = fmaf(A1, zb, ef[1]) / wb;
                    const float dx = xb - xa, dy = yb - ya;
                    if (isfinite(dx) && isfinite(dy)) {
                        hb.xmajor = fabsf(dx) >= fabsf(dy);
                        const float den = hb.xmajor ? dx : dy;
                        if (fabsf(den) > 1e-6f) hb.b = (hb.xmajor ? dy : dx) / den;
                    }
                }
            }
            hb.lo = hb.mlo = __int_as_float(0x7f800000);
            hb.hi = hb.mhi = -__int_as_float(0x7f800000);
            bool check_nf = true;  // per-candidate near / far test needed
            if (zlo <= zhi) {
                if (lateral_fast(Mf, ef, (float)u, (float)v, L, nearp, farp, zlo, zhi, hb)) {
                    check_nf = false;
                } else {
                    // general case: all 12 edges of V clipped to the slab and to [near, far]
                    hb.any = false;
                    hb.lo = hb.mlo = __int_as_float(0x7f800000);
                    hb.hi = hb.mhi = -__int_as_float(0x7f800000);
#pragma unroll 1
                    for (int c = 0; c < 4; ++c) {
                        const float cu = corner_u(c, (float)u, L), cv = corner_v(c, (float)v, L);
                        const int c2 = (c + 1) & 3;
                        const float du = corner_u(c2, (float)u, L) - cu, dv = corner_v(c2, (float)v, L) - cv;
                        lateral_edge(Mf, ef, cu, cv, nearp, farp, zlo, zhi, hb);
                        face_edge(Mf, ef, nearp, cu, cv, du, dv, zlo, zhi, hb);
                        face_edge(Mf, ef, farp, cu, cv, du, dv, zlo, zhi, hb);
                    }
                }
            }
            if (DEBUG && rec) { rec[0] = 0; rec[1] = 0; rec[2] = 0; rec[3] = 0; }
            if (!hb.any) continue;
            // rounding margin: FP32 end points are off by far less than 0.02 px + 1e-5 relative
            const float mg = 0.02f;
            const float lo = hb.lo - (mg + 1e-5f * fabsf(hb.lo)), hi = hb.hi + (mg + 1e-5f * fabsf(hb.hi));
            const float mlo = hb.mlo - (mg + 1e-5f * fabsf(hb.mlo)), mhi = hb.mhi + (mg + 1e-5f * fabsf(hb.mhi));
            const int nmaj = hb.xmajor ? P.W : P.H, nmin = hb.xmajor ? P.H : P.W;
            // NaN bounds (degenerate projections) scan the whole image: fmaxf/fminf drop NaN; the
            // clamps on both sides keep every float -> int conversion in range
            const int m0 = (int)fminf(fmaxf(ceilf(mlo), 0.0f), (float)nmaj);
            const int m1 = (int)fmaxf(fminf(floorf(mhi), (float)(nmaj - 1)), -1.0f);
            if (m0 > m1) continue;
            if (DEBUG && rec) rec[0] = 1;

            // ---- 2. back-projection test rows, centred on p: val = d (R q~) + E
            float R1[3], R2[3], R3[3], E1, E2, E3;
            {
                float Mb[9], eb[3];
#pragma unroll
                for (int i = 0; i < 9; ++i) Mb[i] = __ldg(&gb.M_hi[i]);
#pragma unroll
                for (int i = 0; i < 3; ++i) eb[i] = __ldg(&gb.e_hi[i]);
                const float fu = (float)u, fv = (float)v;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    R1[i] = fmaf(-fu, Mb[6 + i], Mb[i]);
                    R2[i] = fmaf(-fv, Mb[6 + i], Mb[3 + i]);
                    R3[i] = Mb[6 + i];
                }
                E1 = fmaf(-fu, eb[2], eb[0]);
                E2 = fmaf(-fv, eb[2], eb[1]);
                E3 = eb[2];
            }
            // O intrinsics (the back map's target camera) for the metric offset to x_ref
            const float ifxO = __ldg(&gb.ifx), ifyO = __ldg(&gb.ify);
            const float ux = (float)u - __ldg(&gb.cx), vy = (float)v - __ldg(&gb.cy);
            const float ifxJ = SR ? __ldg(&gf.ifx) : 0.0f;  // 1 / fx of J for Eq. 7's area term
            // frame term of Eq. 4 plus the per-frame weights of Eq. 5 / Eq. 10, in log2 units
            float beta = __ldg(&gf.beta) * kLog2e;
            if (a.frame_log2w) beta -= __ldg(a.frame_log2w + J);
            if (a.slot_log2w) beta -= __ldg(a.slot_log2w + j);
            const long long fbase = (long long)J * P.fstride;
            int mc = 0;
            unsigned long long mh = 0ull;
            // The band is walked row by row of its minor axis (|b| <= 1 by the choice of the major
            // axis), each row a run along the major axis: runs are long for the flat epipolar
            // bands of a sideways-moving camera, and every candidate of the parallelogram
            // b m + lo <= n <= b m + hi, m in [m0, m1], is visited once.
            const float fb0 = fmaf(hb.b, (float)m0, 0.0f), fb1 = fmaf(hb.b, (float)m1, 0.0f);
            const int r0 = (int)fminf(fmaxf(ceilf(fminf(fb0, fb1) + lo), 0.0f), (float)nmin);
            const int r1 = (int)fmaxf(fminf(floorf(fmaxf(fb0, fb1) + hi), (float)(nmin - 1)), -1.0f);
            const bool flat = fabsf(hb.b) < 1e-6f;
            const float ib = flat ? 0.0f : 1.0f / hb.b;
            // major / minor shares of R q~ and the memory stride along the major axis
            const float sm1 = hb.xmajor ? R1[0] : R1[1], sm2 = hb.xmajor ? R2[0] : R2[1], sm3 = hb.xmajor ? R3[0] : R3[1];
            const float sn1 = hb.xmajor ? R1[1] : R1[0], sn2 = hb.xmajor ? R2[1] : R2[0], sn3 = hb.xmajor ? R3[1] : R3[0];
            const long long mstep = hb.xmajor ? 1ll : (long long)P.pitch;
            const long long nstep = hb.xmajor ? (long long)P.pitch : 1ll;
            const float *plane = P.depth + fbase + (long long)kPad * P.pitch + kPad;
            // The test in the form |h1 + h2| < L h3 and |h1 - h2| < L h3 (|h1| + |h2| is the larger of
            // |h1 + h2| and |h1 - h2|), with the sums and differences of the coefficients taken once,
            // so that two candidates share each packed FP32x2 operation and the comparisons keep
            // their free absolute values
            const f32x2 sp2 = f2_pack(sm1 + sm2, sm1 + sm2), sq2 = f2_pack(sm1 - sm2, sm1 - sm2),
                        s32 = f2_pack(sm3, sm3);
            const f32x2 Ep2 = f2_pack(E1 + E2, E1 + E2), Eq2 = f2_pack(E1 - E2, E1 - E2), E32 = f2_pack(E3, E3);
            const f32x2 L2 = f2_pack(L, L), off01 = f2_pack(0.0f, 1.0f), off23 = f2_pack(2.0f, 3.0f);
            for (int n = r0; n <= r1; ++n) {
                const float fn = (float)n;
                int ma = m0, mb = m1;
                if (!flat) {
                    // rounding of ta, tb is far below the 0.02 px margin already in lo and hi
                    const float ta = (fn - hi) * ib, tb = (fn - lo) * ib;
                    ma = max(m0, (int)fminf(fmaxf(ceilf(fminf(ta, tb) - 1e-3f), -1.0f), (float)nmaj));
                    mb = min(m1, (int)fmaxf(fminf(floorf(fmaxf(ta, tb) + 1e-3f), (float)nmaj), -1.0f));
                }
                if (ma > mb) continue;
                if (pass == 0) n_exam += mb - ma + 1;
                const float b1 = fmaf(sn1, fn, R1[2]), b2 = fmaf(sn2, fn, R2[2]), b3 = fmaf(sn3, fn, R3[2]);
                const f32x2 bp2 = f2_pack(b1 + b2, b1 + b2), bq2 = f2_pack(b1 - b2, b1 - b2), b32 = f2_pack(b3, b3);
                const float *rowp = plane + (long long)n * nstep;
                // test up to 32 candidates of the run into a hit mask (no branch per candidate),
                // then take the hits (their h1, h2, h3 for the weights are computed again in FP32)
                for (int mc0 = ma; mc0 <= mb; mc0 += 32) {
                    const int cnt = min(mb - mc0, 31);
                    const float *dp = rowp + (long long)mc0 * mstep;
                    float fm = (float)mc0;
                    unsigned int hit = 0u;
                    // four candidates per step, their loads in flight together; the last step may
                    // read up to 3 pixels past the run, inside the image or its 32-pixel padding,
                    // and their bits are dropped
                    for (int k = 0; k <= cnt; k += 4, dp += 4 * mstep, fm += 4.0f) {
                        float dq[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) dq[i] = __ldg(dp + i * mstep);
                        unsigned int bits = 0u;
                        const f32x2 fm2 = f2_pack(fm, fm);
#pragma unroll
                        for (int pr = 0; pr < 2; ++pr) {
                            const f32x2 fmp = f2_add(fm2, pr == 0 ? off01 : off23);
                            const f32x2 d2 = f2_pack(dq[2 * pr], dq[2 * pr + 1]);
                            const f32x2 sv = f2_fma(d2, f2_fma(sp2, fmp, bp2), Ep2);  // h1 + h2
                            const f32x2 tv = f2_fma(d2, f2_fma(sq2, fmp, bq2), Eq2);  // h1 - h2
                            const f32x2 h3 = f2_fma(d2, f2_fma(s32, fmp, b32), E32);
                            const f32x2 cv = f2_mul(L2, h3);
                            float sa, sb, ta, tb, ca, cb;
                            f2_unpack(sv, sa, sb);
                            f2_unpack(tv, ta, tb);
                            f2_unpack(cv, ca, cb);
                            // NaN depth fails the comparisons
                            bool t0 = fabsf(sa) < ca && fabsf(ta) < ca, t1 = fabsf(sb) < cb && fabsf(tb) < cb;
                            if (check_nf) {
                                float h3a, h3b;
                                f2_unpack(h3, h3a, h3b);
                                t0 = t0 && fabsf(h3a - zmid) < zhalf;
                                t1 = t1 && fabsf(h3b - zmid) < zhalf;
                            }
                            bits |= ((unsigned int)t0 << (2 * pr)) | ((unsigned int)t1 << (2 * pr + 1));
                        }
                        // keep the bits of candidates inside the run (k + i <= cnt)
                        bits &= (2u << min(cnt - k, 3)) - 1u;
                        hit |= bits << k;
                    }
                    while (hit) {
                        const int k = __ffs((int)hit) - 1;
                        hit &= hit - 1u;
                        const int m = mc0 + k;
                        const int qx = hb.xmajor ? m : n, qy = hb.xmajor ? n : m;
                        const long long off = fbase + (long long)(qy + kPad) * P.pitch + (qx + kPad);
                        float d;
                        float3 c;
                        load_sample<CFMT>(P.depth, P.colour, off, d, c);
                        const float fmk = (float)m;
                        const float h1 = fmaf(d, fmaf(sm1, fmk, b1), E1);
                        const float h2 = fmaf(d, fmaf(sm2, fmk, b2), E2);
                        const float h3 = fmaf(d, fmaf(sm3, fmk, b3), E3);
                        // Eq. 9: masked samples weigh 0 in the mean-shift steps (semi-transparency:
                        // except for their Eq. 4 term in the last pass)
                        const bool masked = INP && pass > 0 && __ldg(P.mask + off) != 0;
                        const bool add4 = INP == 2 && pass == 2 && own;
                        if (masked && !add4) continue;
                        const float er = c.x - cref.x, eg = c.y - cref.y, eb = c.z - cref.z;
                        float w = 1.0f;
                        if (wpass) {
                            const float dz = h3 - dref;
                            const float ex = fmaf(ux, dz, h1) * ifxO, ey = fmaf(vy, dz, h2) * ifyO;
                            const float d2 = fmaf(ex, ex, fmaf(ey, ey, dz * dz));
                            // inpainting's colour term has no position or frame term
                            float x = INP ? -a_rgb * fmaf(er, er, fmaf(eg, eg, eb * eb))
                                          : -fmaf(a_rgb, fmaf(er, er, fmaf(eg, eg, eb * eb)), fmaf(a_xyz, d2, beta));
                            float w_rel = 1.0f;  // the sample's weight relative to 2^x
                            if (add4) {
                                // the two weights of the semi-transparency step, relative to the larger
                                const float fr = c.x - c_in.x, fg = c.y - c_in.y, fb = c.z - c_in.z;
                                const float x4 = -fmaf(a_rgb, fmaf(fr, fr, fmaf(fg, fg, fb * fb)), fmaf(a_xyz, d2, beta));
                                const float xi = masked ? -__int_as_float(0x7f800000) : x;
                                x = fmaxf(xi, x4);
                                w_rel = ex2(xi - x) + ex2(x4 - x);
                            }
                            if (SR) {  // Eq. 7: s_area = (d / fx_J)^2, the sample's pixel edge squared
                                const float edge = d * ifxJ;
                                x = fmaf(-a_area, edge * edge, x);
                            }
                            if (x > m_log2) {  // new largest weight: rescale what was summed so far
                                const float sc = ex2(m_log2 - x);
                                acc_r *= sc;
                                acc_g *= sc;
                                acc_b *= sc;
                                acc_w *= sc;
                                m_log2 = x;
                            }
                            w = w_rel * ex2(x - m_log2);
                        }
                        acc_r = fmaf(w, er, acc_r);
                        acc_g = fmaf(w, eg, acc_g);
                        acc_b = fmaf(w, eb, acc_b);
                        acc_w += w;
                        if (pass == 0) ++n_acc;
                        if (DEBUG && pass == 0) {
                            ++mc;
                            mh += mix64((unsigned long long)qy * (unsigned long long)P.W + (unsigned long long)qx + 1ull);
                        }
                    }
                }
            }
            if (DEBUG && rec) {
                rec[1] = mc;
                rec[2] = (int32_t)(unsigned int)(mh & 0xffffffffull);
                rec[3] = (int32_t)(unsigned int)(mh >> 32);
            }
        }
    }
    sw_true = acc_w > 0.0f ? acc_w * exp2f(m_log2) : 0.0f;  // the true sum of weights of this pass
    if (INP && acc_w > 0.0f) {
        // this pass's weighted mean is the next pass's reference (and, after the last, the output)
        const float inv = 1.0f / acc_w;
        cref.x = fmaf(acc_r, inv, cref.x);
        cref.y = fmaf(acc_g, inv, cref.y);
        cref.z = fmaf(acc_b, inv, cref.z);
        acc_r = acc_g = acc_b = acc_w = 0.0f;
    }
    }  // passes

    if (active) {
        float o_r = cref.x, o_g = cref.y, o_b = cref.z;
        if (acc_w > 0.0f) {
            const float inv = 1.0f / acc_w;
            o_r = fmaf(acc_r, inv, o_r);
            o_g = fmaf(acc_g, inv, o_g);
            o_b = fmaf(acc_b, inv, o_b);
        }
        float *o = SR ? a.sr_out + (((long long)oi * Ho + v) * Wo + u) * 3 : P.out + (((long long)O * P.H + v) * P.W + u) * 3;
        o[0] = o_r;
        o[1] = o_g;
        o[2] = o_b;
        if (DEBUG && a.pixel_stats) {
            int32_t *ps = a.pixel_stats + crop_idx * 3;
            ps[0] = n_acc;
            ps[1] = (int32_t)min(n_exam, 0x7fffffffll);
            ps[2] = __float_as_int(sw_true);
        }
    }

    unsigned long long ce = (unsigned long long)n_exam, ca = (unsigned long long)n_acc;
    float sw = sw_true;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ce += __shfl_xor_sync(0xffffffffu, ce, o);
        ca += __shfl_xor_sync(0xffffffffu, ca, o);
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_cnt[0][warp] = ce; s_cnt[1][warp] = ca; s_w[warp] = sw; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long te = 0, ta = 0;
        double tw = 0.0;
        for (int i = 0; i < kFrThreads / 32; ++i) { te += s_cnt[0][i]; ta += s_cnt[1][i]; tw += s_w[i]; }
        atomicAdd(a.stat_counts, te);
        atomicAdd(a.stat_counts + 1, ta);
        atomicAdd(a.stat_sumw, tw);
    }
}

// Valid depth range of every frame: one block per (frame, row slice); positive floats order like
// their bit patterns, so the range is kept as atomicMax of the bits (max) and of their complement
// (min); zero words mean "no valid depth".
__global__ void __launch_bounds__(256) zrange_kernel(Planes P, unsigned int *zr) {
    const int f = blockIdx.y;
    unsigned int mx = 0u, mn = 0u;
    for (int y = blockIdx.x; y < P.H; y += gridDim.x) {
        const float *row = P.depth + (long long)f * P.fstride + (long long)(y + kPad) * P.pitch + kPad;
        for (int x = threadIdx.x; x < P.W; x += blockDim.x) {
            const unsigned int bits = __float_as_uint(__ldg(row + x));
            if (bits > 0u && bits < 0x7f800000u) {  // finite and > 0 (NaN pads fail)
                mx = max(mx, bits);
                mn = max(mn, ~bits);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = max(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if ((threadIdx.x & 31) == 0 && mx) {
        atomicMax(zr + 2 * f, mn);
        atomicMax(zr + 2 * f + 1, mx);
    }
}

template <bool SR, int INP>
void launch_frustum_t(const GatherArgs &a, const dim3 grid, cudaStream_t s) {
    const bool dbg = a.membership || a.pixel_stats;
    if (a.clip.colour_fmt == 0) {
        if (dbg) frustum_kernel<0, true, SR, INP><<<grid, kFrThreads, 0, s>>>(a);
        else frustum_kernel<0, false, SR, INP><<<grid, kFrThreads, 0, s>>>(a);
    } else {
        if (dbg) frustum_kernel<1, true, SR, INP><<<grid, kFrThreads, 0, s>>>(a);
        else frustum_kernel<1, false, SR, INP><<<grid, kFrThreads, 0, s>>>(a);
    }
}

// Eq. 8-9's mask from a scene-space box: per pixel of every frame, the world point of its depth
// (unprojected with K_J^-1 and the pose of J, in FP64 with every operation rounded on its own)
// inside the inclusive box -> 1.  cam: per frame K^-1 (9), R (9), t (3).  Pads stay 0.
__global__ void __launch_bounds__(256) mask_box_kernel(Planes P, const double *cam, double bx0, double by0, double bz0,
                                                       double bx1, double by1, double bz1) {
    const long long npx = (long long)P.W * P.H * P.F;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npx; i += (long long)gridDim.x * blockDim.x) {
        const long long f = i / ((long long)P.W * P.H);
        const int rem = (int)(i - f * (long long)P.W * P.H);
        const int y = rem / P.W, x = rem - y * P.W;
        const long long o = f * P.fstride + (long long)(y + kPad) * P.pitch + (x + kPad);
        const float d = P.depth[o];
        unsigned char m = 0;
        if (d > 0.0f && d < __int_as_float(0x7f800000)) {  // NaN (invalid) fails
            const double *Ki = cam + 21 * f, *R = Ki + 9, *t = Ki + 18;
            const double q[3] = {(double)x, (double)y, 1.0};
            double Xc[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double ray = __dadd_rn(__dadd_rn(__dmul_rn(Ki[3 * r], q[0]), __dmul_rn(Ki[3 * r + 1], q[1])),
                                             __dmul_rn(Ki[3 * r + 2], q[2]));
                Xc[r] = __dsub_rn(__dmul_rn((double)d, ray), t[r]);
            }
            double Xw[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Xw[c] = __dadd_rn(__dadd_rn(__dmul_rn(R[c], Xc[0]), __dmul_rn(R[3 + c], Xc[1])), __dmul_rn(R[6 + c], Xc[2]));
            m = Xw[0] >= bx0 && Xw[1] >= by0 && Xw[2] >= bz0 && Xw[0] <= bx1 && Xw[1] <= by1 && Xw[2] <= bz1;
        }
        P.mask[o] = m;
    }
}

}  // namespace

cudaError_t launch_frustum(const GatherArgs &a, cudaStream_t s) {
    const dim3 grid((a.cw + kFrTileX - 1) / kFrTileX, (a.ch + kFrTileY - 1) / kFrTileY, a.n_out);
    if (a.sr_out) launch_frustum_t<true, 0>(a, grid, s);
    else if (a.mode == SSVP_MODE_INPAINT) launch_frustum_t<false, 1>(a, grid, s);
    else if (a.mode == SSVP_MODE_SEMI) launch_frustum_t<false, 2>(a, grid, s);
    else launch_frustum_t<false, 0>(a, grid, s);
    return cudaGetLastError();
}

cudaError_t launch_mask_box(const Planes &p, const double *cam, const double *box, cudaStream_t s) {
    const long long n = (long long)p.W * p.H * p.F;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    mask_box_kernel<<<blocks, 256, 0, s>>>(p, cam, box[0], box[1], box[2], box[3], box[4], box[5]);
    return cudaGetLastError();
}

cudaError_t launch_zrange(const Planes &p, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(p.zrange, 0, 2 * sizeof(unsigned int) * (size_t)p.F, s);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)min(p.H, 64), (unsigned)p.F);
    zrange_kernel<<<grid, 256, 0, s>>>(p, p.zrange);
    return cudaGetLastError();
}

}  // namespace ssvp
