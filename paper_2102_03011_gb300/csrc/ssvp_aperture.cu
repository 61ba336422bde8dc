// ssvp_aperture.cu - fused virtual-aperture gather + filter (Sec. "Virtual aperture", Eq. 13-14).
//
// One thread per output pixel p of frame O.  The cone's axis is p's viewing ray; a sample X_q is
// accepted when its distance to the axis is below a(t) = a0 + (A / z0) |z0 - t|, t being the
// O-camera depth of its foot point on the axis (a thin lens of radius A focused on the plane at
// depth z0).  Per window frame J the scanned box is the bounding box of the projections of the
// lens seed points at the reference depth, grown by h and capped; the accepted samples are
// weighted by s_area / (pi a(t)^2) (Eq. 14, s_area of Eq. 6) and averaged (Eq. 3).
//
// Precision.  The cone is ~0.5 px wide at focus, so the axis distance is formed from small
// quantities only: in frame J, the offset of Y_q from the axis point at the same J-depth is
//     o_x = (dz (q_x - u_inf) + z' (q_x - u')) / f_x,  dz = d_q - z',
// with u' (projection of x_ref), z' (its J depth) and u_inf (vanishing point of the axis) carried
// as double-float numbers.  The FP32 evaluation of o carries a per-candidate error bound; the few
// candidates whose squared distance lies within that bound of a(t)^2 are re-evaluated in
// double-float, so membership is decided to ~1e-7 of the cone radius everywhere.
#include <cuda_fp16.h>

#include "ssvp_df.cuh"
#include "ssvp_internal.h"

namespace ssvp {
namespace {

constexpr float kInvPi = 0.3183098861837907f;
constexpr float kU = 5.9604645e-8f;  // 2^-24
constexpr int kApTileY = 8, kApThreads = 32 * kApTileY;

template <int CFMT, bool DEBUG>
__global__ void __launch_bounds__(kApThreads, 4) aperture_kernel(const GatherArgs a) {
    extern __shared__ float4 sgeom[];
    __shared__ float s_const[5];
    __shared__ unsigned long long s_cnt[2][kApThreads / 32];
    __shared__ float s_w[kApThreads / 32];

    const int oi = blockIdx.z;
    const int O = a.frame_begin + oi;
    const int u0 = a.x0 + blockIdx.x * 32, v0 = a.y0 + blockIdx.y * kApTileY;
    for (int j = threadIdx.x; j < a.n_slots; j += kApThreads)
        build_slot(a.geom[(long long)oi * a.n_slots + j], (float)u0, (float)v0, sgeom + kSlotVec * j);
    if (threadIdx.x == 0) {
        const float z0 = a.focal_depth > 0.0f ? a.focal_depth : *a.clip.median;
        // fx_O from the J = O slot (index T) of the table
        const float ifxO = a.geom[(long long)oi * a.n_slots + a.T].ifx;
        s_const[0] = z0;
        s_const[1] = a.a0 > 0.0f ? a.a0 : 0.5f * z0 * ifxO;
        s_const[2] = a.aperture / z0;
        s_const[3] = 1.0f / ifxO;
        s_const[4] = 1.0f / a.geom[(long long)oi * a.n_slots + a.T].ify;
    }
    __syncthreads();

    const Planes &P = a.clip;
    const int h = (a.k - 1) >> 1, hc = (a.cap - 1) >> 1;
    const float z0 = s_const[0], a0 = s_const[1], slope = s_const[2];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int u = u0 + tx, v = v0 + ty;
    const bool active = u < a.x0 + a.cw && v < a.y0 + a.ch;
    const long long crop_idx = (long long)(v - a.y0) * a.cw + (u - a.x0);
    const int rec_words = 5 + (a.cap * a.cap + 31) / 32;

    int n_acc = 0, n_exam = 0;
    float acc_w = 0.0f, acc_r = 0.0f, acc_g = 0.0f, acc_b = 0.0f;
    float3 cref = make_float3(0.f, 0.f, 0.f);
    float dref = 0.0f;
    if (active) {
        const long long pix = (long long)O * P.fstride + (long long)(v + kPad) * P.pitch + (u + kPad);
        dref = __ldg(P.depth + pix);
        cref = load_colour<CFMT>(P.colour, pix);
    }
    const bool gather = active && dref > 0.0f;
    if (DEBUG && active && !gather && a.membership)
        for (int j = 0; j < a.n_slots; ++j) a.membership[(crop_idx * a.n_slots + j) * rec_words] = -2;

    if (gather) {
        const float du = (float)(u - u0), dv = (float)(v - v0);
        const float s_seed = 1.0f - dref / z0;  // seed X_i = x_ref + s (L_i, 0)
        for (int j = 0; j < a.n_slots; ++j) {
            const float4 *g = sgeom + kSlotVec * j;
            const float4 q5 = g[5];
            const int J = __float_as_int(q5.w);
            int32_t *rec = DEBUG && a.membership ? a.membership + (crop_idx * a.n_slots + j) * rec_words : nullptr;
            if (J < 0) {
                if (DEBUG && rec) rec[0] = -1;
                continue;
            }
            const float4 q0 = g[0], q1 = g[1], q2 = g[2], q3 = g[3], q4 = g[4];
            const df m0 = df_add_f({q0.x, q0.w}, __fmaf_rn(q1.z, du, __fmul_rn(q1.w, dv)));
            const df m1 = df_add_f({q0.y, q1.x}, __fmaf_rn(q2.x, du, __fmul_rn(q2.y, dv)));
            const df m2 = df_add_f({q0.z, q1.y}, __fmaf_rn(q2.z, du, __fmul_rn(q2.w, dv)));
            const df w0 = df_add(df_mul_f(m0, dref), {q3.x, q3.w});
            const df w1 = df_add(df_mul_f(m1, dref), {q3.y, q4.x});
            const df w2 = df_add(df_mul_f(m2, dref), {q3.z, q4.y});
            if (!(w2.hi > 1e-6f * dref) || !(m2.hi > 0.0f)) {
                if (DEBUG && rec) rec[0] = 0;
                continue;
            }
            const float ifx = q4.z, ify = q4.w, fxO = s_const[3], fyO = s_const[4];
            // seeds: projections of x_ref + s (L_i, 0); K_J R_JO columns 0, 1 = fx_O M[:,0], fy_O M[:,1]
            float mnx = 3.0e38f, mny = 3.0e38f, mxx = -3.0e38f, mxy = -3.0e38f, sx = 0.0f, sy = 0.0f;
            bool behind = false;
            {
                const float c0x = fxO * q1.z, c0y = fxO * q2.x, c0z = fxO * q2.z;
                const float c1x = fyO * q1.w, c1y = fyO * q2.y, c1z = fyO * q2.w;
                for (int i = 0; i < a.lens_n; ++i) {
                    const float lx = a.aperture * a.lens_xy[2 * i] * s_seed, ly = a.aperture * a.lens_xy[2 * i + 1] * s_seed;
                    const float wx = fmaf(lx, c0x, fmaf(ly, c1x, w0.hi));
                    const float wy = fmaf(lx, c0y, fmaf(ly, c1y, w1.hi));
                    const float wz = fmaf(lx, c0z, fmaf(ly, c1z, w2.hi));
                    behind |= !(wz > 1e-6f * dref);
                    const float r = 1.0f / wz;
                    const float px = wx * r, py = wy * r;
                    mnx = fminf(mnx, px); mxx = fmaxf(mxx, px);
                    mny = fminf(mny, py); mxy = fmaxf(mxy, py);
                    sx += px; sy += py;
                }
            }
            if (behind) {
                if (DEBUG && rec) rec[0] = 0;
                continue;
            }
            const float lim = (float)(P.W + P.H + 4 * a.cap + 8);
            const float cmx = fminf(fmaxf(sx / (float)a.lens_n, -lim), lim), cmy = fminf(fmaxf(sy / (float)a.lens_n, -lim), lim);
            const float flim = 1.0e7f;
            const int ccx = (int)floorf(cmx + 0.5f), ccy = (int)floorf(cmy + 0.5f);
            const int bx0 = max((int)fmaxf(floorf(mnx + 0.5f), -flim) - h, ccx - hc);
            const int bx1 = min((int)fminf(floorf(mxx + 0.5f), flim) + h, ccx + hc);
            const int by0 = max((int)fmaxf(floorf(mny + 0.5f), -flim) - h, ccy - hc);
            const int by1 = min((int)fminf(floorf(mxy + 0.5f), flim) + h, ccy + hc);
            const int x0c = max(bx0, 0), x1c = min(bx1, P.W - 1), y0c = max(by0, 0), y1c = min(by1, P.H - 1);
            if (DEBUG && rec) {
                rec[1] = bx0; rec[2] = by0; rec[3] = bx1; rec[4] = by1;
                for (int wd = 5; wd < rec_words; ++wd) rec[wd] = 0;
            }
            if (x0c > x1c || y0c > y1c) {
                if (DEBUG && rec) rec[0] = 2;
                continue;
            }
            if (DEBUG && rec) rec[0] = 1;
            n_exam += (x1c - x0c + 1) * (y1c - y0c + 1);

            // reference point u', v', z' and the axis vanishing point u_inf, v_inf in J
            const float rz = rcp_approx(w2.hi);
            const df U = df_div(w0, w2, rz), V = df_div(w1, w2, rz);
            const float rm = rcp_approx(m2.hi);
            const df Ui = df_div(m0, m2, rm), Vi = df_div(m1, m2, rm);
            const float zh = w2.hi, zl = w2.lo;
            // axis direction b = K_J^-1 m (J coordinates), unit bn, and 1 / b_z
            const float bx = (Ui.hi - q5.x) * ifx, by = (Vi.hi - q5.y) * ify;  // b / b_z
            const float inv_bn = rsqrtf(fmaf(bx, bx, fmaf(by, by, 1.0f)));
            const float bnx = bx * inv_bn, bny = by * inv_bn;
            const float inv_bz = rm;                      // lambda - d_ref = dz / b_z
            const float foot = inv_bn * rm;              // (o . b) / |b|^2 = (o . bn) / |b|
            // offsets relative to the box origin (bx0, by0)
            const df gx = df_add_f({-Ui.hi, -Ui.lo}, (float)bx0), ex = df_add_f({-U.hi, -U.lo}, (float)bx0);
            const df gy = df_add_f({-Vi.hi, -Vi.lo}, (float)by0), ey = df_add_f({-V.hi, -V.lo}, (float)by0);
            const float zix = zh * ifx, ziy = zh * ify;
            const float gxf = gx.hi * ifx, exf = ex.hi * zix, gyf = gy.hi * ify, eyf = ey.hi * ziy;
            // error scale of the FP32 offsets: |o_fp32 - o| <= 8 u (|dz| Gm + Em)
            const float Gm = (fabsf(gx.hi) + (float)(x1c - bx0) + fabsf(gy.hi) + (float)(y1c - by0)) * fmaxf(ifx, ify);
            const float Em = zh * (fabsf(ex.hi) + (float)(x1c - bx0) + fabsf(ey.hi) + (float)(y1c - by0)) * fmaxf(ifx, ify);
            // error of the FP32 fast path on diff = q^2 - a(t)^2: |err| <= 4 (a + E) E with
            // E = 8 u (|dz| c1 + |o.b| c3 + c2) bounding both the offset error (8 u (|dz| Gm + Em))
            // and the cone-radius error from t (slope 8 u (d_ref + |dz / b_z| + |o.b| foot))
            const float c1 = Gm + slope * fabsf(inv_bz), c2 = Em + slope * dref, c3 = slope * foot;
            // one candidate: the FP32 fast path's diff and a(t) come in; refine near the cone
            // surface in double-float, then accumulate when inside
            auto finish = [&](float d, float iff, float jf, float diff, float ar, float E, long long idx, int qx, int qy) {
                if (fabsf(diff) <= 4.0f * (ar + E) * E) {
                    // near the cone surface: recompute the offsets in double-float
                    const df dzd = fast_two_sum(d - zh, -zl);
                    const df Gd = df_add_f(gx, iff), Ed = df_add_f(ex, iff);
                    const df Sx = df_add(df_mul(dzd, Gd), df_mul({zh, zl}, Ed));
                    const df Gyd = df_add_f(gy, jf), Eyd = df_add_f(ey, jf);
                    const df Sy = df_add(df_mul(dzd, Gyd), df_mul({zh, zl}, Eyd));
                    const float ox = (Sx.hi + Sx.lo) * ifx;
                    const float oy = (Sy.hi + Sy.lo) * ify;
                    const float ob = fmaf(ox, bnx, oy * bny);
                    const float p2 = fmaf(ox, ox, fmaf(oy, oy, -ob * ob));
                    const float t = fmaf(dzd.hi, inv_bz, dref) + ob * foot;
                    ar = fmaf(slope, fabsf(z0 - t), a0);
                    diff = p2 - ar * ar;
                }
                if (diff < 0.0f) {
                    const float3 c = load_colour<CFMT>(P.colour, idx);
                    const float e = d * ifx;
                    const float w = __fdividef(e * e * kInvPi, ar * ar);  // 2 ulp: far inside the tolerance
                    acc_r = fmaf(w, c.x - cref.x, acc_r);
                    acc_g = fmaf(w, c.y - cref.y, acc_g);
                    acc_b = fmaf(w, c.z - cref.z, acc_b);
                    acc_w += w;
                    ++n_acc;
                    if (DEBUG && rec) {
                        const int bit = (qy - by0) * a.cap + (qx - bx0);
                        rec[5 + (bit >> 5)] |= (int32_t)(1u << (bit & 31));
                    }
                }
            };
            // per-(pixel, J) constants, duplicated for the packed FP32x2 path
            const f32x2 zh2 = f2_pack(zh, zh), zl2 = f2_pack(zl, zl), ifx2 = f2_pack(ifx, ifx), zix2 = f2_pack(zix, zix);
            const f32x2 gxf2 = f2_pack(gxf, gxf), exf2 = f2_pack(exf, exf), bnx2 = f2_pack(bnx, bnx), bny2 = f2_pack(bny, bny);
            const f32x2 ibz2 = f2_pack(inv_bz, inv_bz), dref2 = f2_pack(dref, dref), foot2 = f2_pack(foot, foot);
            const f32x2 z02 = f2_pack(z0, z0), slope2 = f2_pack(slope, slope), a02 = f2_pack(a0, a0);
            const f32x2 c12 = f2_pack(c1, c1), c22 = f2_pack(c2, c2), c32 = f2_pack(c3, c3);
            const f32x2 k8u = f2_pack(8.0f * kU, 8.0f * kU), neg1 = f2_pack(-1.0f, -1.0f);
            const long long jbase = (long long)J * P.fstride;
            for (int qy = y0c; qy <= y1c; ++qy) {
                const float jf = (float)(qy - by0);
                const float Gy = fmaf(jf, ify, gyf), Ey = fmaf(jf, ziy, eyf);
                const f32x2 Gy2 = f2_pack(Gy, Gy), Ey2 = f2_pack(Ey, Ey);
                const long long rowb = jbase + (long long)(qy + kPad) * P.pitch + kPad;
                float iff = (float)(x0c - bx0);
                int qx = x0c;
                // two candidates per step in packed FP32x2 (invalid depth is NaN: it fails both
                // comparisons of finish)
                for (; qx + 1 <= x1c; qx += 2, iff += 2.0f) {
                    const float d0 = __ldg(P.depth + rowb + qx), d1 = __ldg(P.depth + rowb + qx + 1);
                    const f32x2 dz = f2_sub(f2_sub(f2_pack(d0, d1), zh2), zl2);
                    const f32x2 if2 = f2_pack(iff, iff + 1.0f);
                    const f32x2 ox = f2_fma(dz, f2_fma(if2, ifx2, gxf2), f2_fma(if2, zix2, exf2));
                    const f32x2 oy = f2_fma(dz, Gy2, Ey2);
                    const f32x2 ob = f2_fma(ox, bnx2, f2_mul(oy, bny2));
                    const f32x2 p2 = f2_fma(ox, ox, f2_fma(oy, oy, f2_mul(f2_mul(ob, neg1), ob)));
                    const f32x2 t = f2_fma(ob, foot2, f2_fma(dz, ibz2, dref2));
                    const f32x2 ar = f2_fma(slope2, f2_abs(f2_sub(z02, t)), a02);
                    const f32x2 diff = f2_fma(f2_mul(ar, neg1), ar, p2);
                    const f32x2 E = f2_mul(k8u, f2_fma(f2_abs(dz), c12, f2_fma(f2_abs(ob), c32, c22)));
                    float df0, df1, ar0, ar1, E0, E1;
                    f2_unpack(diff, df0, df1);
                    f2_unpack(ar, ar0, ar1);
                    f2_unpack(E, E0, E1);
                    finish(d0, iff, jf, df0, ar0, E0, rowb + qx, qx, qy);
                    finish(d1, iff + 1.0f, jf, df1, ar1, E1, rowb + qx + 1, qx + 1, qy);
                }
                if (qx <= x1c) {  // the odd last column
                    const float d = __ldg(P.depth + rowb + qx);
                    const float dz = (d - zh) - zl;
                    const float ox = fmaf(dz, fmaf(iff, ifx, gxf), fmaf(iff, zix, exf));
                    const float oy = fmaf(dz, Gy, Ey);
                    const float ob = fmaf(ox, bnx, oy * bny);
                    const float p2 = fmaf(ox, ox, fmaf(oy, oy, -ob * ob));
                    const float t = fmaf(ob, foot, fmaf(dz, inv_bz, dref));
                    const float ar = fmaf(slope, fabsf(z0 - t), a0);
                    const float diff = fmaf(-ar, ar, p2);
                    const float E = 8.0f * kU * fmaf(fabsf(dz), c1, fmaf(fabsf(ob), c3, c2));
                    finish(d, iff, jf, diff, ar, E, rowb + qx, qx, qy);
                }
            }
        }
    }

    if (active) {
        float o_r = cref.x, o_g = cref.y, o_b = cref.z;
        if (acc_w > 0.0f) {
            const float inv = 1.0f / acc_w;
            o_r = fmaf(acc_r, inv, o_r);
            o_g = fmaf(acc_g, inv, o_g);
            o_b = fmaf(acc_b, inv, o_b);
        }
        float *o = P.out + (((long long)O * P.H + v) * P.W + u) * 3;
        o[0] = o_r;
        o[1] = o_g;
        o[2] = o_b;
        if (DEBUG && a.pixel_stats) {
            int32_t *ps = a.pixel_stats + crop_idx * 3;
            ps[0] = n_acc;
            ps[1] = n_exam;
            ps[2] = __float_as_int(acc_w);
        }
    }
    unsigned long long ce = (unsigned long long)n_exam, ca = (unsigned long long)n_acc;
    float sw = acc_w;
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
        for (int i = 0; i < kApThreads / 32; ++i) { te += s_cnt[0][i]; ta += s_cnt[1][i]; tw += s_w[i]; }
        atomicAdd(a.stat_counts, te);
        atomicAdd(a.stat_counts + 1, ta);
        atomicAdd(a.stat_sumw, tw);
    }
}

}  // namespace

cudaError_t launch_aperture(const GatherArgs &a, cudaStream_t s) {
    if (a.n_out <= 0 || a.cw <= 0 || a.ch <= 0) return cudaSuccess;
    dim3 grid((a.cw + 31) / 32, (a.ch + kApTileY - 1) / kApTileY, a.n_out);
    size_t smem = sizeof(float4) * kSlotVec * (size_t)a.n_slots;
    const bool dbg = a.membership || a.pixel_stats;
    if (a.clip.colour_fmt == 0) {
        if (dbg) aperture_kernel<0, true><<<grid, kApThreads, smem, s>>>(a);
        else aperture_kernel<0, false><<<grid, kApThreads, smem, s>>>(a);
    } else {
        if (dbg) aperture_kernel<1, true><<<grid, kApThreads, smem, s>>>(a);
        else aperture_kernel<1, false><<<grid, kApThreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace ssvp
