// ssvp_gather.cu - the fused scene-space gather + filter kernel (steps A3-A7).
//
// One thread per output pixel p of frame O, CTAs of 32 x 8 pixels.  For every window slot j
// (frame J = O - T + j) the thread projects its reference point into J, tests the k x k
// candidates around the projection against the radius (the back-projection test of Eq. 2,
// seeded by the output depth) and accumulates the Eq. 4 weighted colour (Eq. 3).
//
// Precision.  The radius is ~0.5 % of the scene depth, so the distance test needs the reference
// point in J's pixel grid to ~1e-9 relative, beyond FP32.  The per-(pixel, J) reference
// quantities (u', v' = projected position, z' = depth in J) are therefore carried as unevaluated
// FP32 pairs ("double-float", error-free transformations with FMA), computed from the FP64 camera
// composition the host splits into hi/lo pairs.  The per-candidate test then only forms small
// differences, all in plain FP32:
//     Y_q - y_ref = ((d_q - z') (q_x - c_x) + z' (q_x - u')) / f_x, ... , d_q - z'
// so the FP32 error of the distance is ~1e-7 of the radius rather than ~1e-7 of the depth.
//
// Accepted candidates are recorded in a per-thread bit mask during the test loop and filtered
// afterwards by iterating the set bits, so a warp pays for the filter arithmetic only as often
// as its busiest lane accepts (warp-level compaction of the accepted samples).
#include <cuda.h>  // CUtensorMap (the type only; the host encodes maps through the runtime's driver entry point)
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/ssvp.h"
#include "ssvp_df.cuh"
#include "ssvp_internal.h"

namespace ssvp {
namespace {

#ifndef SSVP_MIN_CTAS
#define SSVP_MIN_CTAS 4  // resident CTAs per SM the register allocation must allow
#endif
// The extraction gather of the learned filter keeps four more values live than the plain one; at
// 64 registers (four CTAs per SM) it spills 80 bytes a thread, at 80 (three CTAs) 8.  Short windows,
// whose accepted samples are nearly all stored, run faster with three CTAs and no spill traffic;
// long ones, where the candidate loads dominate, with four CTAs and more warps to hide them.
constexpr int kLearnCtasShort = 3;
constexpr int kLearnShortSlots = 17;  // windows of up to +-8 frames



#ifndef SSVP_TILE_Y
#define SSVP_TILE_Y 8  // output rows per CTA (a warp covers 32 pixels of one row)
#endif
constexpr int kTileX = 32, kTileY = SSVP_TILE_Y, kThreads = kTileX * kTileY;
// ---------------------------------------------------------------- TMA staging of the window frames
// SSVP_GATHER_WINDOW_TMA.  Each warp (32 output pixels of one row) stages, for every window frame J,
// the depth of a kBoxW x kBoxH box of J's padded depth plane into shared memory with one 3-D tensor
// copy (cp.async.bulk.tensor, completion counted on an mbarrier), in two buffers: the copy of frame
// j + 1 is issued before frame j is tested.  The box is placed around the window of the warp's first
// gathering lane, whose projection into J is recomputed in FP32 for the purpose (a box needs no
// more); on a smooth surface the other lanes' windows lie beside it.  A lane whose window is not
// inside the box (at depth edges neighbouring pixels reproject far apart) tests from the global
// plane, so membership and results are those of the global-load path.  The waits are bounded: on a
// time-out the warp raises bit 1 of the error word, returns to global loads for its remaining
// frames, and its issuing lane waits once more (bounded) for the copies it has in flight.
constexpr int kBoxW = 48, kBoxH = 12;               // floats; a box row is 192 bytes (a multiple of 16)
constexpr unsigned kBoxBytes = kBoxW * kBoxH * 4;   // 2,304 bytes, a multiple of 128
constexpr int kNoBox = 0x40000000;                  // origin of a buffer holding no box: no window fits
constexpr int kStageMaxK = 7;
constexpr unsigned kStgWaitHintNs = 100000, kStgWaitLimit = 10000;  // about 1 s per wait

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// bounded wait for the completion of the phase with parity `parity`; false on time-out
__device__ __forceinline__ bool stg_wait(unsigned bar, unsigned parity) {
    for (unsigned it = 0; it < kStgWaitLimit; ++it) {
        unsigned done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity), "r"(kStgWaitHintNs)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Per warp of a staging CTA: two mbarriers (one per box) and the origin (x, y) in J's padded plane
// of each box, or kNoBox.  The boxes themselves follow the slot geometry in dynamic shared memory,
// 128-byte aligned, two per warp.
constexpr int kStgWarps = kThreads / 32;
__shared__ unsigned long long g_stg_bar[kStgWarps][2];
__shared__ int2 g_stg_org[kStgWarps][2];

// shared-space address of buffer b of this warp's boxes (the slot geometry has n_slots entries)
__device__ __forceinline__ unsigned stg_box(const float4 *sgeom, int n_slots, int b) {
    const unsigned end = smem_addr(sgeom + kSlotVec * n_slots);
    return ((end + 127u) & ~127u) + ((threadIdx.x >> 5) * 2 + b) * kBoxBytes;
}
__device__ __forceinline__ unsigned stg_bar(int b) { return smem_addr(&g_stg_bar[threadIdx.x >> 5][b]); }

// Issue the copy of window slot s (frame J) into buffer s & 1: called by the warp's first gathering
// lane, whose pixel offset in the tile is (du, dv), depth dref and lane index `lane`; tmap describes
// the clip's depth planes ({pitch, rows, F} floats, box {kBoxW, kBoxH, 1}).  skip (a test of the
// time-out path): the barrier is told to expect the box's bytes but no copy is issued, so the wait
// for it runs out.
template <int K>
__device__ __forceinline__ void stage_issue(const CUtensorMap *tmap, const float4 *sgeom, int n_slots, int s, float du,
                                            float dv, float dref, int lane, bool skip) {
    constexpr int h = (K - 1) / 2;
    const int b = s & 1;
    const float4 *g = sgeom + kSlotVec * s;
    const int J = __float_as_int(g[5].w);
    int x0 = kNoBox, y0 = kNoBox;
    if (J >= 0) {
        const float4 q0 = g[0], q1 = g[1], q2 = g[2], q3 = g[3];
        const float w0 = fmaf(dref, q0.x + fmaf(q1.z, du, q1.w * dv), q3.x);
        const float w1 = fmaf(dref, q0.y + fmaf(q2.x, du, q2.y * dv), q3.y);
        const float w2 = fmaf(dref, q0.z + fmaf(q2.z, du, q2.w * dv), q3.z);
        if (w2 > 1e-6f * dref) {
            const float rz = rcp_approx(w2), U = w0 * rz, V = w1 * rz;
            if (fabsf(U) < 1e6f && fabsf(V) < 1e6f) {
                const int ax = (int)floorf(U + 0.5f), ay = (int)floorf(V + 0.5f);
                // the warp's windows span columns [ax - lane - h, ax - lane + 31 + h]: centre them in
                // the box, x rounded down to a multiple of 4 floats (16 bytes, as tensor copies need)
                x0 = (ax - lane - h + kPad - (kBoxW - 34 - K) / 2) & ~3;
                y0 = ay - h + kPad - (kBoxH - K) / 2;
            }
        }
    }
    g_stg_org[threadIdx.x >> 5][b] = make_int2(x0, y0);
    const unsigned bar = stg_bar(b);
    if (x0 != kNoBox) {
        const unsigned dst = stg_box(sgeom, n_slots, b);
        // the warp's generic-proxy reads of this buffer (frame s - 2) precede the copy's writes
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(kBoxBytes) : "memory");
        if (!skip)
            asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];\n" ::"r"(dst),
            "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(x0), "r"(y0), "r"(J), "r"(bar)
            : "memory");
    } else {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
    }
}

// The gather and filter of one output pixel (u, v) of frame O (steps A3-A7).  sgeom holds the
// per-slot geometry built for the tile whose first pixel is (u0, v0).  n_acc, n_exam and acc_w
// return the pixel's accepted and examined counts and sum of weights (they start at 0).
// K > 0: compile-time window width (k*k <= 64, one 64-bit accept mask per frame).
// K == 0: runtime k up to 31, one 32-bit accept mask per window row.
constexpr int kMaxSamples = 64;  // learned filter: capped sample set
constexpr float kLn2 = 0.6931471805599453f;

// One accepted sample of the learned filter's capped set, compactly: its FP32 colour with the
// BF16 pair (dist / r, (J - O) / T) in one 16-byte record and the pair (depth residual / r,
// log w) in one word; the other features are rebuilt by the MLP kernels.
__device__ __forceinline__ unsigned bf16_pair(float lo, float hi) {
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&b2);
}
// i = crop pixel * 64 + slot: the host keeps the sets of a crop below 2^32 samples, so one 32-bit
// index (widened in the address arithmetic) addresses both arrays
__device__ __forceinline__ void store_sample(const GatherArgs &a, unsigned i, float3 c, float dist_r, float dj_t,
                                             float dz_r, float logw) {
    a.sets.col[i] = make_float4(c.x, c.y, c.z, __uint_as_float(bf16_pair(dist_r, dj_t)));
    a.sets.f89[i] = bf16_pair(dz_r, logw);
}
// the distance feature is rounded to BF16 (8 significant bits): the approximate square root
// (a few FP32 ulp, exact at 0) is enough
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// LEARN: visit the frames in canonical order (O, O-1, O+1, ...) and store the features of the
// first kMaxSamples accepted samples (learned filter); the Eq. 3/4 result goes to a.sets.plain.
// ACCB: accepted samples taken per iteration of the filter loop of a compile-time window (1, or
// 2 in packed FP32x2, which the kernels use; the runtime-k path takes them one at a time)
// STG: the candidate depths of the test loop come from the warp's staged boxes (K > 0, not LEARN);
// tmap describes the clip's depth planes
template <int K, int CFMT, bool DEBUG, bool LEARN = false, int ACCB = 1, bool STG = false>
__device__ __forceinline__ void gather_pixel(const GatherArgs &a, const Planes &P, const int O, const int u0,
                                             const int v0, const int u, const int v, const bool active,
                                             const long long crop_idx, const float4 *sgeom, const int n_slots,
                                             const float r2, const float a_rgb, const float a_xyz, const bool weighted,
                                             int &n_acc, int &n_exam, float &acc_w, const CUtensorMap *tmap = nullptr) {
    static_assert(!STG || (K > 0 && K <= kStageMaxK && !LEARN), "staging: compile-time k <= 7, plain gather");
    const int k = K > 0 ? K : a.k;
    const int h = (k - 1) >> 1;
    const int rec_words = 3 + (k * k + 31) / 32;
    float acc_r = 0.0f, acc_g = 0.0f, acc_b = 0.0f;
    int n_feat = 0;
    const int Tw = (n_slots - 1) >> 1;
    const float inv_r = LEARN ? rsqrtf(r2) : 0.0f, inv_T = LEARN ? 1.0f / (float)max(Tw, 1) : 0.0f;
    const unsigned set0 = LEARN ? (unsigned)crop_idx * (unsigned)kMaxSamples : 0u;
    float3 cref = make_float3(0.f, 0.f, 0.f);
    float dref = 0.0f;
    if (active) {
        const long long pix = (long long)O * P.fstride + (long long)(v + kPad) * P.pitch + (u + kPad);
        dref = __ldg(P.depth + pix);
        cref = load_colour<CFMT>(P.colour, pix);
    }
    const bool gather = active && dref > 0.0f;  // false for NaN (invalid) depth
    // staging: the warp's gathering lanes, the first of them issues the copies
    const unsigned G = STG ? __ballot_sync(0xffffffffu, gather) : 0u;
    int stg_fail = -1;  // staging: the slot whose wait gave up (-1: staging on)
    if (DEBUG && active && !gather && a.membership) {
        for (int j = 0; j < n_slots; ++j) a.membership[(crop_idx * n_slots + j) * rec_words] = -2;
    }

    if (gather) {
        const float du = (float)(u - u0), dv = (float)(v - v0);
        if (STG && (int)(threadIdx.x & 31) == __ffs(G) - 1)
            stage_issue<K>(tmap, sgeom, n_slots, 0, du, dv, dref, threadIdx.x & 31, a.stage == 2);
        for (int jj = 0; jj < n_slots; ++jj) {
            int2 org = make_int2(kNoBox, kNoBox);
            if (STG) {
                // every lane of G is done with buffer (jj + 1) & 1 (slot jj - 1): refill it with slot
                // jj + 1, then wait for slot jj
                __syncwarp(G);
                const bool leader = (int)(threadIdx.x & 31) == __ffs(G) - 1;
                if (stg_fail < 0 && leader && jj + 1 < n_slots)
                    stage_issue<K>(tmap, sgeom, n_slots, jj + 1, du, dv, dref, threadIdx.x & 31, a.stage == 2);
                const bool ok = stg_fail >= 0 || stg_wait(stg_bar(jj & 1), (unsigned)(jj >> 1) & 1u);
                if (__all_sync(G, ok)) {
                    if (stg_fail < 0) org = g_stg_org[threadIdx.x >> 5][jj & 1];
                } else if (stg_fail < 0) {
                    stg_fail = jj;  // the rest of this warp's frames test from the global plane
                    if (leader) atomicOr(a.err, 2);
                }
            }
            // canonical order for the learned filter: O, O-1, O+1, O-2, O+2, ...
            const int j = LEARN ? Tw + (jj == 0 ? 0 : ((jj & 1) ? -((jj + 1) >> 1) : (jj >> 1))) : jj;
            const float4 *g = sgeom + kSlotVec * j;
            const float4 q5 = g[5];
            const int J = __float_as_int(q5.w);
            int32_t *rec = DEBUG && a.membership ? a.membership + (crop_idx * n_slots + j) * rec_words : nullptr;
            if (J < 0) {
                if (DEBUG && rec) rec[0] = -1;
                continue;
            }
            const float4 q0 = g[0], q1 = g[1], q2 = g[2], q3 = g[3], q4 = g[4];
            // m = M (u, v, 1) = M (u0, v0, 1) + M (du, dv, 0): the base in double-float, the small
            // offset exactly enough in FP32
            df m0 = df_add_f({q0.x, q0.w}, __fmaf_rn(q1.z, du, __fmul_rn(q1.w, dv)));
            df m1 = df_add_f({q0.y, q1.x}, __fmaf_rn(q2.x, du, __fmul_rn(q2.y, dv)));
            df m2 = df_add_f({q0.z, q1.y}, __fmaf_rn(q2.z, du, __fmul_rn(q2.w, dv)));
            // w = d_ref m + e: homogeneous pixel coordinates of x_ref in J
            df w0 = df_add(df_mul_f(m0, dref), {q3.x, q3.w});
            df w1 = df_add(df_mul_f(m1, dref), {q3.y, q4.x});
            df w2 = df_add(df_mul_f(m2, dref), {q3.z, q4.y});
            if (!(w2.hi > 1e-6f * dref)) {  // behind (or at) camera J
                if (DEBUG && rec) rec[0] = 0;
                continue;
            }
            const float rz = rcp_approx(w2.hi);
            const df U = df_div(w0, w2, rz), V = df_div(w1, w2, rz);
            // window centre floor(u' + 0.5) and the exact offset u' - centre in [-0.5, 0.5)
            float cxf = floorf(U.hi + 0.5f), cyf = floorf(V.hi + 0.5f);
            float ou = __fadd_rn(__fsub_rn(U.hi, cxf), U.lo), ov = __fadd_rn(__fsub_rn(V.hi, cyf), V.lo);
            if (ou < -0.5f) { cxf -= 1.0f; ou += 1.0f; } else if (ou >= 0.5f) { cxf += 1.0f; ou -= 1.0f; }
            if (ov < -0.5f) { cyf -= 1.0f; ov += 1.0f; } else if (ov >= 0.5f) { cyf += 1.0f; ov -= 1.0f; }
            if (!(cxf >= (float)-h && cxf <= (float)(P.W - 1 + h) && cyf >= (float)-h && cyf <= (float)(P.H - 1 + h))) {
                if (DEBUG && rec) { rec[0] = 2; }
                continue;  // no window pixel inside the image
            }
            const int cx = (int)cxf, cy = (int)cyf;
            {
                int nx = min(cx + h, P.W - 1) - max(cx - h, 0) + 1;
                int ny = min(cy + h, P.H - 1) - max(cy - h, 0) + 1;
                n_exam += nx * ny;
            }
            const float ifx = q4.z, ify = q4.w;
            const float zh = w2.hi, zl = w2.lo;
            // ray_x(q) = (q_x - cx_J) / fx and z' (q_x - u') / fx as affine functions of dx
            const float Ax0 = (cxf - (float)h - q5.x) * ifx, zix = zh * ifx, Bx0 = (-(float)h - ou) * zix;
            const float Ay0 = (cyf - (float)h - q5.y) * ify, ziy = zh * ify, By0 = (-(float)h - ov) * ziy;
            const long long wbase = (long long)J * P.fstride + (long long)(cy - h + kPad) * P.pitch + (cx - h + kPad);
            const float *dwin = P.depth + wbase;
            const void *cwin = CFMT == 0 ? (const void *)(reinterpret_cast<const float4 *>(P.colour) + wbase)
                                         : (const void *)(reinterpret_cast<const uint2 *>(P.colour) + wbase);
            const float beta = q5.z;
            const float dj_t = LEARN ? (float)(j - Tw) * inv_T : 0.0f;  // the frame-offset feature
            if (DEBUG && rec) { rec[0] = 1; rec[1] = cx; rec[2] = cy; }

            if (K > 0) {
                // the test loop's depths: this lane's window in the staged box if it lies inside it
                const float *dtest = dwin;
                long long tpitch = P.pitch;
                if (STG) {
                    const int ox = cx - h + kPad - org.x, oy = cy - h + kPad - org.y;
                    if ((unsigned)ox <= (unsigned)(kBoxW - K) && (unsigned)oy <= (unsigned)(kBoxH - K)) {
                        dtest = reinterpret_cast<const float *>(reinterpret_cast<const char *>(sgeom) +
                                                                (stg_box(sgeom, n_slots, jj & 1) - smem_addr(sgeom))) +
                                oy * kBoxW + ox;
                        tpitch = kBoxW;
                    }
                }
                float Ax[K > 0 ? K : 1], Bx[K > 0 ? K : 1];
#pragma unroll
                for (int dx = 0; dx < K; ++dx) {
                    Ax[dx] = __fmaf_rn((float)dx, ifx, Ax0);
                    Bx[dx] = __fmaf_rn((float)dx, zix, Bx0);
                }
                // columns (dx, dx + 1) are tested as pairs with packed FP32x2 arithmetic: each half
                // runs the scalar sequence below, so the distances are the same to the bit
                constexpr int KP = K / 2;
                f32x2 AxP[KP > 0 ? KP : 1], BxP[KP > 0 ? KP : 1];
#pragma unroll
                for (int q = 0; q < KP; ++q) {
                    AxP[q] = f2_pack(Ax[2 * q], Ax[2 * q + 1]);
                    BxP[q] = f2_pack(Bx[2 * q], Bx[2 * q + 1]);
                }
                const f32x2 zh2 = f2_pack(zh, zh), zl2 = f2_pack(zl, zl);
                unsigned long long mask = 0ull;
#pragma unroll
                for (int dy = 0; dy < K; ++dy) {
                    const float Ay = __fmaf_rn((float)dy, ify, Ay0), By = __fmaf_rn((float)dy, ziy, By0);
                    const f32x2 Ay2 = f2_pack(Ay, Ay), By2 = f2_pack(By, By);
                    const float *drow = dtest + (long long)dy * tpitch;
#pragma unroll
                    for (int q = 0; q < KP; ++q) {
                        // staged: a generic load (shared memory, or the global plane outside the box)
                        const float da = STG ? drow[2 * q] : __ldg(drow + 2 * q);
                        const float db = STG ? drow[2 * q + 1] : __ldg(drow + 2 * q + 1);
                        const f32x2 dz = f2_sub(f2_sub(f2_pack(da, db), zh2), zl2);
                        const f32x2 X = f2_fma(dz, AxP[q], BxP[q]);
                        const f32x2 Y = f2_fma(dz, Ay2, By2);
                        const f32x2 d2 = f2_fma(X, X, f2_fma(Y, Y, f2_mul(dz, dz)));
                        float d2a, d2b;
                        f2_unpack(d2, d2a, d2b);
                        if (d2a < r2) mask |= 1ull << (dy * 8 + 2 * q);  // stride 8: cheap decode
                        if (d2b < r2) mask |= 1ull << (dy * 8 + 2 * q + 1);
                    }
                    if (K & 1) {
                        constexpr int dx = K - 1;
                        const float dz = ((STG ? drow[dx] : __ldg(drow + dx)) - zh) - zl;
                        const float X = fmaf(dz, Ax[dx], Bx[dx]);
                        const float Y = fmaf(dz, Ay, By);
                        const float d2 = fmaf(X, X, fmaf(Y, Y, dz * dz));
                        if (d2 < r2) mask |= 1ull << (dy * 8 + dx);
                    }
                }
                if (DEBUG && rec) {
                    unsigned long long packed = 0ull;  // record layout: bit dy*k+dx
                    for (int dy = 0; dy < K; ++dy)
                        packed |= ((mask >> (8 * dy)) & ((1ull << K) - 1ull)) << (dy * K);
                    rec[3] = (int32_t)(unsigned int)(packed & 0xffffffffull);
                    if (K * K > 32) rec[4] = (int32_t)(unsigned int)(packed >> 32);
                }
                // accepted samples, ACCB per iteration so that their loads overlap; with two,
                // the pair's sums are kept in packed partial sums and folded after the frame
                f32x2 pr = 0ull, pg = 0ull, pb = 0ull, pw = 0ull;  // +0.0f in both halves
#pragma unroll 1
                while (mask) {
                    int idx[ACCB];
                    bool ok[ACCB];
#pragma unroll
                    for (int t = 0; t < ACCB; ++t) {
                        ok[t] = mask != 0ull;
                        idx[t] = ok[t] ? __ffsll((long long)mask) - 1 : 0;  // slot 0 is always in bounds
                        mask &= mask - 1ull;
                    }
                    float dq[ACCB];
                    float3 cq[ACCB];
#pragma unroll
                    for (int t = 0; t < ACCB; ++t) {
                        const int off = (idx[t] >> 3) * P.pitch + (idx[t] & 7);
                        load_sample<CFMT>(dwin, cwin, off, dq[t], cq[t]);
                    }
                    if constexpr (ACCB == 2) {
                        // the two samples in packed FP32x2: per half the scalar sequence below
                        const f32x2 dxf = f2_pack(small_float(idx[0] & 7), small_float(idx[1] & 7));
                        const f32x2 dyf = f2_pack(small_float(idx[0] >> 3), small_float(idx[1] >> 3));
                        const f32x2 dz = f2_sub(f2_sub(f2_pack(dq[0], dq[1]), f2_pack(zh, zh)), f2_pack(zl, zl));
                        const f32x2 X = f2_fma(dz, f2_fma(dxf, f2_pack(ifx, ifx), f2_pack(Ax0, Ax0)),
                                               f2_fma(dxf, f2_pack(zix, zix), f2_pack(Bx0, Bx0)));
                        const f32x2 Y = f2_fma(dz, f2_fma(dyf, f2_pack(ify, ify), f2_pack(Ay0, Ay0)),
                                               f2_fma(dyf, f2_pack(ziy, ziy), f2_pack(By0, By0)));
                        const f32x2 d2 = f2_fma(X, X, f2_fma(Y, Y, f2_mul(dz, dz)));
                        const f32x2 er = f2_sub(f2_pack(cq[0].x, cq[1].x), f2_pack(cref.x, cref.x));
                        const f32x2 eg = f2_sub(f2_pack(cq[0].y, cq[1].y), f2_pack(cref.y, cref.y));
                        const f32x2 eb = f2_sub(f2_pack(cq[0].z, cq[1].z), f2_pack(cref.z, cref.z));
                        const f32x2 e = f2_fma(f2_pack(a_rgb, a_rgb), f2_fma(er, er, f2_fma(eg, eg, f2_mul(eb, eb))),
                                               f2_fma(f2_pack(a_xyz, a_xyz), d2, f2_pack(beta, beta)));
                        float e0, e1;
                        f2_unpack(e, e0, e1);
                        const float w0 = weighted ? ex2(-e0) : 1.0f;
                        const float w1 = ok[1] ? (weighted ? ex2(-e1) : 1.0f) : 0.0f;  // ok[0] holds in the loop
                        if (LEARN) {
                            float dd0, dd1, dz0, dz1;
                            f2_unpack(d2, dd0, dd1);
                            f2_unpack(dz, dz0, dz1);
                            if (n_feat < kMaxSamples) {
                                store_sample(a, set0 + n_feat, cq[0], sqrt_approx(dd0) * inv_r, dj_t, dz0 * inv_r,
                                             -e0 * kLn2);
                                ++n_feat;
                            }
                            if (ok[1] && n_feat < kMaxSamples) {
                                store_sample(a, set0 + n_feat, cq[1], sqrt_approx(dd1) * inv_r, dj_t, dz1 * inv_r,
                                             -e1 * kLn2);
                                ++n_feat;
                            }
                        }
                        const f32x2 w = f2_pack(w0, w1);
                        pr = f2_fma(w, er, pr);
                        pg = f2_fma(w, eg, pg);
                        pb = f2_fma(w, eb, pb);
                        pw = f2_add(pw, w);
                        n_acc += 1 + (ok[1] ? 1 : 0);
                    } else {
#pragma unroll
                    for (int t = 0; t < ACCB; ++t) {
                        const float dxf = small_float(idx[t] & 7), dyf = small_float(idx[t] >> 3);
                        const float dz = (dq[t] - zh) - zl;
                        const float X = fmaf(dz, __fmaf_rn(dxf, ifx, Ax0), __fmaf_rn(dxf, zix, Bx0));
                        const float Y = fmaf(dz, __fmaf_rn(dyf, ify, Ay0), __fmaf_rn(dyf, ziy, By0));
                        const float d2 = fmaf(X, X, fmaf(Y, Y, dz * dz));
                        const float er = cq[t].x - cref.x, eg = cq[t].y - cref.y, eb = cq[t].z - cref.z;
                        const float e = fmaf(a_rgb, fmaf(er, er, fmaf(eg, eg, eb * eb)), fmaf(a_xyz, d2, beta));
                        float w = 1.0f;
                        if (weighted) w = ex2(-e);
                        if (LEARN && ok[t] && n_feat < kMaxSamples) {
                            store_sample(a, set0 + n_feat, cq[t], sqrt_approx(d2) * inv_r, dj_t, dz * inv_r,
                                         -e * kLn2);
                            ++n_feat;
                        }
                        if (ok[t]) {
                            acc_r = fmaf(w, er, acc_r);
                            acc_g = fmaf(w, eg, acc_g);
                            acc_b = fmaf(w, eb, acc_b);
                            acc_w += w;
                            ++n_acc;
                        }
                    }
                    }
                }
                if (ACCB == 2) {
                    float lo, hi;
                    f2_unpack(pr, lo, hi);
                    acc_r += lo + hi;
                    f2_unpack(pg, lo, hi);
                    acc_g += lo + hi;
                    f2_unpack(pb, lo, hi);
                    acc_b += lo + hi;
                    f2_unpack(pw, lo, hi);
                    acc_w += lo + hi;
                }
            } else {
                if (DEBUG && rec)
                    for (int wd = 3; wd < rec_words; ++wd) rec[wd] = 0;
                for (int dy = 0; dy < k; ++dy) {
                    const float Ay = __fmaf_rn((float)dy, ify, Ay0), By = __fmaf_rn((float)dy, ziy, By0);
                    const float *drow = dwin + (long long)dy * P.pitch;
                    unsigned int mask = 0u;
                    for (int dx = 0; dx < k; ++dx) {
                        const float dz = (__ldg(drow + dx) - zh) - zl;
                        const float X = fmaf(dz, __fmaf_rn((float)dx, ifx, Ax0), __fmaf_rn((float)dx, zix, Bx0));
                        const float Y = fmaf(dz, Ay, By);
                        const float d2 = fmaf(X, X, fmaf(Y, Y, dz * dz));
                        if (d2 < r2) mask |= 1u << dx;
                    }
                    if (DEBUG && rec) {
                        for (int dx = 0; dx < k; ++dx)
                            if (mask >> dx & 1u) {
                                const int bit = dy * k + dx;
                                rec[3 + (bit >> 5)] |= (int32_t)(1u << (bit & 31));
                            }
                    }
                    while (mask) {
                        const int dx = __ffs((int)mask) - 1;
                        mask &= mask - 1u;
                        const long long off = (long long)dy * P.pitch + dx;
                        float dq;
                        float3 c;
                        load_sample<CFMT>(dwin, cwin, off, dq, c);
                        const float dz = (dq - zh) - zl;
                        const float X = fmaf(dz, __fmaf_rn((float)dx, ifx, Ax0), __fmaf_rn((float)dx, zix, Bx0));
                        const float Y = fmaf(dz, Ay, By);
                        const float d2 = fmaf(X, X, fmaf(Y, Y, dz * dz));
                        const float er = c.x - cref.x, eg = c.y - cref.y, eb = c.z - cref.z;
                        const float e = fmaf(a_rgb, fmaf(er, er, fmaf(eg, eg, eb * eb)), fmaf(a_xyz, d2, beta));
                        float w = 1.0f;
                        if (weighted) w = ex2(-e);
                        if (LEARN && n_feat < kMaxSamples) {
                            store_sample(a, set0 + n_feat, c, sqrt_approx(d2) * inv_r, dj_t, dz * inv_r, -e * kLn2);
                            ++n_feat;
                        }
                        acc_r = fmaf(w, er, acc_r);
                        acc_g = fmaf(w, eg, acc_g);
                        acc_b = fmaf(w, eb, acc_b);
                        acc_w += w;
                        ++n_acc;
                    }
                }
            }
        }
        if (STG && stg_fail >= 0 && (int)(threadIdx.x & 31) == __ffs(G) - 1) {
            // after a time-out: wait once more (bounded) for the copies that may still be in flight,
            // slot stg_fail and the slot issued before its wait
            stg_wait(stg_bar(stg_fail & 1), (unsigned)(stg_fail >> 1) & 1u);
            if (stg_fail + 1 < n_slots) stg_wait(stg_bar((stg_fail + 1) & 1), (unsigned)((stg_fail + 1) >> 1) & 1u);
        }
    }

    if (active) {
        // Eq. 3 written around the reference colour: c_ref + sum w (c - c_ref) / sum w
        float o_r = cref.x, o_g = cref.y, o_b = cref.z;
        if (acc_w > 0.0f) {
            const float inv = 1.0f / acc_w;
            o_r = fmaf(acc_r, inv, o_r);
            o_g = fmaf(acc_g, inv, o_g);
            o_b = fmaf(acc_b, inv, o_b);
        }
        float *o = LEARN ? a.sets.plain + crop_idx * 3 : P.out + (((long long)O * P.H + v) * P.W + u) * 3;
        o[0] = o_r;
        o[1] = o_g;
        o[2] = o_b;
        if (LEARN) {
            // per pixel: the count kept, c_ref and the size of the whole set / 64 (what the plain
            // fallback averages)
            a.sets.n[crop_idx] = n_feat;
            a.sets.info[crop_idx] = make_float4(cref.x, cref.y, cref.z, (float)n_acc * (1.0f / 64.0f));
        }
        if (DEBUG && a.pixel_stats) {
            int32_t *ps = a.pixel_stats + crop_idx * 3;
            ps[0] = n_acc;
            ps[1] = n_exam;
            ps[2] = __float_as_int(acc_w);
        }
    }

}

// One CTA per 32 x kTileY output tile of one output frame (grid: tiles x output frames).
// STG: the staged gather; dynamic shared memory then holds, after the slot geometry (aligned up to
// 128 bytes), two boxes per warp, and tmap describes the clip's depth planes.
template <int K, int CFMT, bool DEBUG, bool LEARN = false, int MINB = SSVP_MIN_CTAS, bool STG = false>
__global__ void __launch_bounds__(kThreads, MINB) gather_kernel(const GatherArgs a, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ float4 sgeom[];
    __shared__ float s_const[4];
    __shared__ unsigned long long s_cnt[2][kThreads / 32];
    __shared__ float s_w[kThreads / 32];
    if (STG && (threadIdx.x & 31) == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(stg_bar(0)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(stg_bar(1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }

    const int oi = blockIdx.z;
    const int O = a.frame_begin + oi;
    const int u0 = a.x0 + blockIdx.x * kTileX, v0 = a.y0 + blockIdx.y * kTileY;
    for (int j = threadIdx.x; j < a.n_slots; j += kThreads) {
        float4 *g = sgeom + kSlotVec * j;
        build_slot(a.geom[(long long)oi * a.n_slots + j], (float)u0, (float)v0, g);
        // per-frame weights (Eq. 5, Eq. 10) join the frame term of the exponent
        const int J = __float_as_int(g[5].w);
        if (J >= 0 && a.frame_log2w) g[5].z -= a.frame_log2w[J];
        if (J >= 0 && a.slot_log2w) g[5].z -= a.slot_log2w[j];
    }
    if (threadIdx.x == 0) {
        float r = a.radius > 0.0f ? a.radius : -a.radius * *a.clip.median;
        float sx = a.sigma_xyz > 0.0f ? a.sigma_xyz : r;
        // the shutter weight of Eq. 10 replaces Eq. 4: no colour and no position term
        const bool shutter = a.mode == SSVP_MODE_SHUTTER;
        s_const[0] = r * r;
        s_const[1] = shutter ? 0.0f : kLog2e / (2.0f * a.sigma_rgb * a.sigma_rgb);
        s_const[2] = shutter ? 0.0f : kLog2e / (2.0f * sx * sx);
        s_const[3] = a.mode == SSVP_MODE_MEAN ? 0.0f : 1.0f;
    }
    __syncthreads();

    const int tx = threadIdx.x % kTileX, ty = threadIdx.x / kTileX;
    const int u = u0 + tx, v = v0 + ty;
    const bool active = u < a.x0 + a.cw && v < a.y0 + a.ch;
    const long long crop_idx = (long long)(v - a.y0) * a.cw + (u - a.x0);
    int n_acc = 0, n_exam = 0;
    float acc_w = 0.0f;
    gather_pixel<K, CFMT, DEBUG, LEARN, 2, STG>(a, a.clip, O, u0, v0, u, v, active, crop_idx, sgeom, a.n_slots,
                                                s_const[0], s_const[1], s_const[2], s_const[3] != 0.0f, n_acc, n_exam,
                                                acc_w, &tmap);

    // launch statistics: warp, then block, then one atomic per CTA
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
        for (int i = 0; i < kThreads / 32; ++i) { te += s_cnt[0][i]; ta += s_cnt[1][i]; tw += s_w[i]; }
        atomicAdd(a.stat_counts, te);
        atomicAdd(a.stat_counts + 1, ta);
        atomicAdd(a.stat_sumw, tw);
    }
}


// Persistent batched gather (A10): CTAs of 32 x TY threads pull work items (clip, output-frame
// chunk, tile) from a device counter until the list is exhausted, so clips of uneven size share
// one launch without tail effects per clip.  The clip table is read from the kernel's parameter
// space (constant bank), so the per-clip plane pointers and strides need no registers.
template <int K, int CFMT, int TY>
__global__ void __launch_bounds__(32 * TY, 32 / TY) batch_kernel(const GatherArgs a, const BatchArgs b) {
    constexpr int NT = 32 * TY;
    extern __shared__ float4 sgeom[];
    __shared__ float s_const[4];
    // the work unit (one output frame of one item), kept in shared memory by thread 0 so that no
    // loop state stays live in registers across the gather
    __shared__ int s_c, s_u0, s_v0, s_oi, s_olast, s_done;
    __shared__ unsigned long long s_cnt[2][NT / 32];
    __shared__ double s_w[NT / 32];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_cnt[0][warp] = 0ull; s_cnt[1][warp] = 0ull; s_w[warp] = 0.0; }
    if (threadIdx.x == 0) { s_oi = 0; s_olast = 0; s_done = 0; }
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            // the next output frame of the current item, else the next item
            int c = -1;
            if (s_oi + 1 < s_olast) {
                ++s_oi;
                c = s_c;
            } else {
                const long long item = (long long)atomicAdd(b.counter, 1ull);
                if (item >= b.n_items) {
                    s_done = 1;
                } else {
                    c = 0;
                    while (c + 1 < b.n_clips && b.clip[c + 1].item_begin <= item) ++c;
                    s_c = c;
                    const BatchClip &bc = b.clip[c];
                    const long long local = item - bc.item_begin;
                    const int ntile = bc.tiles_x * bc.tiles_y;
                    const int tile = (int)(local % ntile), chunk = (int)(local / ntile);
                    s_u0 = (tile % bc.tiles_x) * 32;
                    s_v0 = (tile / bc.tiles_x) * TY;
                    s_oi = chunk * b.frame_chunk;
                    s_olast = min(s_oi + b.frame_chunk, bc.n_out);
                }
            }
            if (c >= 0) {
                const float r = a.radius > 0.0f ? a.radius : -a.radius * *b.clip[c].p.median;
                const float sx = a.sigma_xyz > 0.0f ? a.sigma_xyz : r;
                s_const[0] = r * r;
                s_const[1] = kLog2e / (2.0f * a.sigma_rgb * a.sigma_rgb);
                s_const[2] = kLog2e / (2.0f * sx * sx);
                s_const[3] = a.mode == 3 ? 0.0f : 1.0f;
            }
        }
        __syncthreads();
        if (s_done) break;
        const int c = s_c, oi = s_oi, u0 = s_u0, v0 = s_v0;
        const BatchClip &bc = b.clip[c];
        const PairGeom *geom = bc.geom + (long long)oi * a.n_slots;
        for (int j = threadIdx.x; j < a.n_slots; j += NT)
            build_slot(geom[j], (float)u0, (float)v0, sgeom + kSlotVec * j);
        __syncthreads();
        const int u = u0 + (threadIdx.x & 31), v = v0 + (threadIdx.x >> 5);
        const bool active = u < bc.p.W && v < bc.p.H;
        int n_acc = 0, n_exam = 0;
        float acc_w = 0.0f;
        gather_pixel<K, CFMT, false, false, 2>(a, bc.p, bc.frame_begin + oi, u0, v0, u, v, active, 0, sgeom, a.n_slots,
                                               s_const[0], s_const[1], s_const[2], s_const[3] != 0.0f, n_acc, n_exam,
                                               acc_w);
        // launch statistics go to per-warp shared slots after every tile
        unsigned ce = (unsigned)n_exam, ca = (unsigned)n_acc;
        float sw = acc_w;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ce += __shfl_xor_sync(0xffffffffu, ce, o);
            ca += __shfl_xor_sync(0xffffffffu, ca, o);
            sw += __shfl_xor_sync(0xffffffffu, sw, o);
        }
        if ((threadIdx.x & 31) == 0) { s_cnt[0][warp] += ce; s_cnt[1][warp] += ca; s_w[warp] += sw; }
        __syncthreads();  // the shared geometry and the work unit are rebuilt next
    }
    if (threadIdx.x == 0) {
        unsigned long long te = 0, ta = 0;
        double tw = 0.0;
        for (int i = 0; i < NT / 32; ++i) { te += s_cnt[0][i]; ta += s_cnt[1][i]; tw += s_w[i]; }
        atomicAdd(a.stat_counts, te);
        atomicAdd(a.stat_counts + 1, ta);
        atomicAdd(a.stat_sumw, tw);
    }
}

template <int K, int CFMT, int TY>
void *batch_fn() { return (void *)batch_kernel<K, CFMT, TY>; }

template <int CFMT, int TY>
void *batch_fn_k(int k) {
    switch (k) {
        case 1: return batch_fn<1, CFMT, TY>();
        case 3: return batch_fn<3, CFMT, TY>();
        case 5: return batch_fn<5, CFMT, TY>();
        case 7: return batch_fn<7, CFMT, TY>();
        default: return batch_fn<0, CFMT, TY>();
    }
}

void *batch_fn_any(int k, int tile_rows, int cfmt) {
    if (tile_rows == 4) return cfmt == 0 ? batch_fn_k<0, 4>(k) : batch_fn_k<1, 4>(k);
    if (tile_rows == 8) return cfmt == 0 ? batch_fn_k<0, 8>(k) : batch_fn_k<1, 8>(k);
    return nullptr;
}

// cuTensorMapEncodeTiled, from the driver through the runtime (no link against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// The clip's depth planes as a 3-D FP32 tensor {pitch, rows, F} (row and frame strides in bytes are
// multiples of 16: the pitch is a multiple of 32 floats), read in boxes of kBoxW x kBoxH x 1; reads
// outside the tensor return NaN, which fails the radius test as the padding does.
cudaError_t encode_depth_map(const Planes &P, CUtensorMap *m) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return cudaErrorSymbolNotFound;
    const cuuint64_t dims[3] = {(cuuint64_t)P.pitch, (cuuint64_t)P.rows, (cuuint64_t)P.F};
    const cuuint64_t strides[2] = {(cuuint64_t)P.pitch * sizeof(float), (cuuint64_t)P.fstride * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)kBoxH, 1u}, elem[3] = {1u, 1u, 1u};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, P.depth, dims, strides, box, elem,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int K, int CFMT>
cudaError_t launch_k(const GatherArgs &a, cudaStream_t s) {
    dim3 grid((a.cw + kTileX - 1) / kTileX, (a.ch + kTileY - 1) / kTileY, a.n_out);
    size_t smem = sizeof(float4) * kSlotVec * (size_t)a.n_slots;
    const bool dbg = a.membership || a.pixel_stats;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    if (a.stage) {
        if constexpr (K > 0 && K <= kStageMaxK) {
            if (a.sets.col) return cudaErrorInvalidValue;
            cudaError_t e = encode_depth_map(a.clip, &tmap);
            if (e != cudaSuccess) return e;
            smem += 128 + (size_t)(kThreads / 32) * 2 * kBoxBytes;
            void (*fn)(const GatherArgs, const CUtensorMap) =
                dbg ? gather_kernel<K, CFMT, true, false, SSVP_MIN_CTAS, true>
                    : gather_kernel<K, CFMT, false, false, SSVP_MIN_CTAS, true>;
            if (smem > 48 * 1024 &&
                (e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
                return e;
            fn<<<grid, kThreads, smem, s>>>(a, tmap);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (a.sets.col && a.n_slots <= kLearnShortSlots)
        gather_kernel<K, CFMT, false, true, kLearnCtasShort><<<grid, kThreads, smem, s>>>(a, tmap);
    else if (a.sets.col) gather_kernel<K, CFMT, false, true><<<grid, kThreads, smem, s>>>(a, tmap);
    else if (dbg) gather_kernel<K, CFMT, true><<<grid, kThreads, smem, s>>>(a, tmap);
    else gather_kernel<K, CFMT, false><<<grid, kThreads, smem, s>>>(a, tmap);
    return cudaGetLastError();
}

template <int CFMT>
cudaError_t launch_c(const GatherArgs &a, cudaStream_t s) {
    switch (a.k) {
        case 1: return launch_k<1, CFMT>(a, s);
        case 3: return launch_k<3, CFMT>(a, s);
        case 5: return launch_k<5, CFMT>(a, s);
        case 7: return launch_k<7, CFMT>(a, s);
        default: return launch_k<0, CFMT>(a, s);
    }
}

}  // namespace

cudaError_t launch_gather(const GatherArgs &a, cudaStream_t s) {
    if (a.n_out <= 0 || a.cw <= 0 || a.ch <= 0) return cudaSuccess;
    return a.clip.colour_fmt == 0 ? launch_c<0>(a, s) : launch_c<1>(a, s);
}

int batch_grid(int k, int tile_rows, int colour_fmt, int n_slots) {
    void *fn = batch_fn_any(k, tile_rows, colour_fmt);
    if (!fn) return 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    size_t smem = sizeof(float4) * kSlotVec * (size_t)n_slots;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * tile_rows, smem) != cudaSuccess) return 0;
    return sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_batch(const GatherArgs &a, const BatchArgs &b, int tile_rows, int colour_fmt, int grid,
                         cudaStream_t s) {
    void *fn = batch_fn_any(a.k, tile_rows, colour_fmt);
    if (!fn || grid <= 0) return cudaErrorInvalidValue;
    size_t smem = sizeof(float4) * kSlotVec * (size_t)a.n_slots;
    void *args[] = {(void *)&a, (void *)&b};
    return cudaLaunchKernel(fn, dim3(grid), dim3(32 * tile_rows), args, smem, s);
}

}  // namespace ssvp
