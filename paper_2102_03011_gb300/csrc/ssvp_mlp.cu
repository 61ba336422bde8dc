// ssvp_mlp.cu - training of the learned per-sample weighting: a 16 -> 64 -> 2 MLP over each
// pixel's capped sample set (up to 64 samples), on the BF16 tensor cores (warp-level mma.sync)
// with FP32 accumulation; inference runs on tcgen05 (ssvp_mlp_tc.cu) with the same arithmetic.
//
// One warp per pixel, 16 samples (one MMA row tile) at a time.  Layer 1 is H = F W1^T + b1 with
// F the tile's 16 x 16 feature block and W1^T held in B fragments for all eight 8-column tiles
// of the 64 hidden units (eight mma.sync.m16n8k16, bf16 x bf16 -> f32, b1 in the accumulator).
// ReLU and the rounding to BF16 happen in one conversion, and the accumulator fragments of two
// neighbouring hidden tiles are exactly the A fragment of the next product, so layer 2 (64 -> 2,
// padded to 8 output columns) is four more MMAs with b2 in the accumulator.  (z_w, z_c) per
// sample give w = softplus(z_w) and conf = mean sigmoid(z_c), the loss and dz; the backward pass
// recomputes H, forms dH in shared memory (BF16) and accumulates dW1 = dH^T F as a second MMA
// over the sample dimension.  The compact sample sets are also expanded here for callers that
// read them (ssvp_learned_samples).
#include <cuda_bf16.h>

#include "ssvp_internal.h"

namespace ssvp {
namespace {

constexpr int kS = 64, kF = 16, kH = 64;
constexpr int kWarps = 4;          // warps (pixels in flight) per CTA
constexpr int kLd = kH + 8;        // padded row of the shared dH tile (bf16 elements)

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1,
                                         const float (&c)[4]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]), "f"(c[2]), "f"(c[3]));
}

// the same with the accumulator's initial value as one quad (a 16-byte shared-memory load)
__device__ __forceinline__ void mma_bf16_q(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1, float4 c) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c.x), "f"(c.y), "f"(c.z), "f"(c.w));
}

// keep the kernels' copies of the master weights: W1 as BF16, W2 rounded to BF16 values
__device__ __forceinline__ void refresh_one(const MlpState &st, int i, float p) {
    if (i < kMlpB1) {
        __nv_bfloat16 b = __float2bfloat16_rn(p);
        st.W1_bf16[i] = *reinterpret_cast<unsigned short *>(&b);
    } else if (i >= kMlpW2 && i < kMlpB2) {
        st.W2_r[i - kMlpW2] = __bfloat162float(__float2bfloat16_rn(p));
    }
}

__device__ __forceinline__ float softplusf(float x) { return fmaxf(x, 0.0f) + log1pf(__expf(-fabsf(x))); }
// sigmoid with the fast reciprocal: it only enters the confidence mean and its derivative
__device__ __forceinline__ float sigmoidf(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }

__device__ __forceinline__ unsigned pack2(unsigned short lo, unsigned short hi) { return (unsigned)lo | ((unsigned)hi << 16); }

__device__ __forceinline__ unsigned short bf16_bits(float x) {
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<const unsigned short *>(&b);
}

// Feature word w (features 2w, 2w + 1 as a BF16 pair, the lower index in the low half) of one
// sample, rebuilt from its compact record (colour c, stored pairs c.w and f89) and the pixel's
// info (c_ref, |S(p)| / 64) and plain result:
//   w0 (c.x, c.y)  w1 (c.z, c.x - cref.x)  w2 (c.y - cref.y, c.z - cref.z)  w3 (dist / r, dJ / T)
//   w4 (dz / r, log w)  w5 (1, |S| / 64)  w6 (c.x - p.x, c.y - p.y)  w7 (c.z - p.z, 0)
// The differences are taken in FP32 before rounding, as the features are defined.
__device__ __forceinline__ unsigned feat_word(int w, float4 c, unsigned f89, float4 info, const float (&pl)[3]) {
    switch (w) {
    case 0: return pack2(bf16_bits(c.x), bf16_bits(c.y));
    case 1: return pack2(bf16_bits(c.z), bf16_bits(c.x - info.x));
    case 2: return pack2(bf16_bits(c.y - info.y), bf16_bits(c.z - info.z));
    case 3: return __float_as_uint(c.w);
    case 4: return f89;
    case 5: return pack2(0x3f80, bf16_bits(info.w));  // BF16 1.0
    case 6: return pack2(bf16_bits(c.x - pl[0]), bf16_bits(c.y - pl[1]));
    default: return pack2(bf16_bits(c.z - pl[2]), 0);
    }
}

// Feature i of sample s as BF16 bits (the B operand of the dW1 product)
__device__ __forceinline__ unsigned short feature_bits(const SampleSets &S, long long px, int s, int i, float4 info,
                                                       const float (&pl)[3]) {
    const long long k = px * kS + s;
    const unsigned w = feat_word(i >> 1, __ldg(S.col + k), i >> 1 == 4 ? __ldg(S.f89 + k) : 0u, info, pl);
    return (unsigned short)((i & 1) ? w >> 16 : w & 0xffffu);
}

// The A fragments hold the features in a different order from the logical one above, chosen so
// that lane t of a quad builds both of its words (t and 4 + t) with the same few operations:
//   word t < 3:   (c_t, c_t - cref_t)            word 3: (dist / r, dJ / T) as stored
//   word 4 + t:   (c_t - plain_t, x_t), x = (1, |S| / 64, 0)   word 7: (dz / r, log w) as stored
// slot_feature(word, half) is the logical feature in that half of that word; W1's B fragments
// are gathered in the same order, so F W1^T is unchanged.
__device__ __forceinline__ int slot_feature(int word, int half) {
    const int t = word & 3;
    if (word < 4) return t < 3 ? t + 3 * half : 6 + half;
    if (t == 3) return 8 + half;
    return half == 0 ? 12 + t : (t == 2 ? 15 : 10 + t);
}

__device__ __forceinline__ unsigned bf16x2(float lo, float hi) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&b);
}

__device__ __forceinline__ __nv_bfloat162 u32_as_bf162(unsigned u) { return *reinterpret_cast<const __nv_bfloat162 *>(&u); }

// ReLU, then round to BF16 (the A operand of layer 2): one conversion for a pair
__device__ __forceinline__ unsigned relu_bf16x2(float lo, float hi) {
    unsigned r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Per-lane constants of a pixel for the feature words: cref_t, plain_t, x_t
struct LaneFeat {
    float cr, pt, xt;
};
__device__ __forceinline__ LaneFeat lane_feat(int t, float4 info, const float (&pl)[3]) {
    LaneFeat f;
    f.cr = t == 0 ? info.x : (t == 1 ? info.y : info.z);
    f.pt = t == 0 ? pl[0] : (t == 1 ? pl[1] : pl[2]);
    f.xt = t == 0 ? 1.0f : (t == 1 ? info.w : 0.0f);
    return f;
}

// Words t (lo) and 4 + t (hi) of one sample (the differences in FP32, then rounded)
__device__ __forceinline__ void sample_words(int t, float4 c, unsigned f89, const LaneFeat &f, unsigned &lo,
                                             unsigned &hi) {
    const float ct = t == 0 ? c.x : (t == 1 ? c.y : c.z);
    lo = t == 3 ? __float_as_uint(c.w) : bf16x2(ct, ct - f.cr);
    hi = t == 3 ? f89 : bf16x2(ct - f.pt, f.xt);
}

// The two rows (g, g + 8) of 16-sample tile mt of pixel px; rows >= n read nothing
struct TileRows {
    float4 c[2];
    unsigned f89[2];
};
__device__ __forceinline__ void load_rows(const SampleSets &S, long long px, int mt, int n, int g, int t,
                                          TileRows &r) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = 16 * mt + g + 8 * h;
        const long long k = px * kS + s;
        r.c[h] = s < n ? __ldg(S.col + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        r.f89[h] = (t == 3 && s < n) ? __ldg(S.f89 + k) : 0u;
    }
}

// A fragment of a tile: words t (a0 row g, a1 row g + 8) and 4 + t (a2, a3); rows >= n are zero
__device__ __forceinline__ void tile_fragment(const TileRows &r, int mt, int n, int g, int t, const LaneFeat &f,
                                              unsigned (&a)[4]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        unsigned lo, hi;
        sample_words(t, r.c[h], r.f89[h], f, lo, hi);
        const bool in = 16 * mt + g + 8 * h < n;
        a[h] = in ? lo : 0u;
        a[2 + h] = in ? hi : 0u;
    }
}

// A fragments of all four tiles (the training kernel keeps them for the backward pass)
__device__ __forceinline__ void load_features(const SampleSets &S, long long px, int n, int g, int t, float4 info,
                                              const float (&pl)[3], unsigned (&a)[4][4]) {
    const LaneFeat f = lane_feat(t, info, pl);
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
        TileRows r;
        load_rows(S, px, mt, n, g, t, r);
        tile_fragment(r, mt, n, g, t, f, a[mt]);
    }
}

// Layer-2 B fragments: column n = g of W2^T (n = 0: z_w, 1: z_c, 2..7 zero), k = hidden units
__device__ __forceinline__ void load_w2(const MlpWeights &w, int g, int t, unsigned (&b)[4][2]) {
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        const int j = 16 * kt + 2 * t;
        b[kt][0] = g < 2 ? bf16x2(__ldg(w.W2 + g * kH + j), __ldg(w.W2 + g * kH + j + 1)) : 0u;
        b[kt][1] = g < 2 ? bf16x2(__ldg(w.W2 + g * kH + j + 8), __ldg(w.W2 + g * kH + j + 9)) : 0u;
    }
}

// Both layers of one 16-sample tile.  sb1[4 nt + t] = (b1[8 nt + 2 t], b1[8 nt + 2 t + 1]) twice:
// the layer-1 accumulator's initial quad for lane t of hidden tile nt.
// Returns the layer-2 accumulator: lane (g, 0) holds (z_w, z_c) of row g in e[0], e[1] and of
// row g + 8 in e[2], e[3] (b2 included); the other lanes hold the zero padding columns.
__device__ __forceinline__ void tile_forward(const unsigned (&a)[4], const unsigned (&bw)[8][2], const float4 *sb1,
                                             const unsigned (&bw2)[4][2], float b20, float b21, int t,
                                             float (&e)[4]) {
    e[0] = e[2] = t == 0 ? b20 : 0.0f;
    e[1] = e[3] = t == 0 ? b21 : 0.0f;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        float d0[4], d1[4];
        mma_bf16_q(d0, a, bw[2 * kt][0], bw[2 * kt][1], sb1[4 * (2 * kt) + t]);
        mma_bf16_q(d1, a, bw[2 * kt + 1][0], bw[2 * kt + 1][1], sb1[4 * (2 * kt + 1) + t]);
        // hidden columns 16 kt + 2 t (+1) and + 8: the A fragment of layer 2's k-tile kt
        const unsigned h[4] = {relu_bf16x2(d0[0], d0[1]), relu_bf16x2(d0[2], d0[3]), relu_bf16x2(d1[0], d1[1]),
                               relu_bf16x2(d1[2], d1[3])};
        mma_bf16(e, h, bw2[kt][0], bw2[kt][1], e);
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Layer-1 B fragments of the eight hidden tiles, in the A fragments' feature order
__device__ __forceinline__ void load_w1(const MlpWeights &w, int g, int t, unsigned (&bw)[8][2]) {
    const unsigned short *w1 = w.W1;
    const int f0 = slot_feature(t, 0), f1 = slot_feature(t, 1), f2 = slot_feature(4 + t, 0),
              f3 = slot_feature(4 + t, 1);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const unsigned short *row = w1 + (8 * nt + g) * kF;
        bw[nt][0] = pack2(__ldg(row + f0), __ldg(row + f1));
        bw[nt][1] = pack2(__ldg(row + f2), __ldg(row + f3));
    }
}

// b1 pairs, each twice, in shared memory (the layer-1 accumulator's initial quads); synchronises
// the block
__device__ __forceinline__ void load_b1(const MlpWeights &w, float4 *sb1) {
    for (int i = threadIdx.x; i < kH / 2; i += blockDim.x) {
        const float x = __ldg(w.b1 + 2 * i), y = __ldg(w.b1 + 2 * i + 1);
        sb1[i] = make_float4(x, y, x, y);
    }
    __syncthreads();
}

// ---------------------------------------------------------------- training: forward + backward
__global__ void __launch_bounds__(32 * kWarps) mlp_train_kernel(const MlpArgs m) {
    __shared__ unsigned short s_dh[kWarps][kS * kLd];
    __shared__ float s_g[kH + 2 * kH + 2 + 1];  // gb1, gW2, gb2, loss
    __shared__ float4 s_b1[kH / 2];
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kH + 2 * kH + 3; i += blockDim.x) s_g[i] = 0.0f;
    load_b1(m.w, s_b1);  // synchronises the block
    unsigned bw[8][2], bw2[4][2];
    load_w1(m.w, g, t, bw);
    load_w2(m.w, g, t, bw2);
    const float b20 = __ldg(m.w.b2), b21 = __ldg(m.w.b2 + 1);
    float dW1[4][2][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) dW1[i][j][0] = dW1[i][j][1] = dW1[i][j][2] = dW1[i][j][3] = 0.0f;
    unsigned short *dh = s_dh[wid];
    const float inv_np = 1.0f / (float)m.n_batch;
    const long long nwarps = (long long)gridDim.x * kWarps;
    for (long long bi = blockIdx.x * (long long)kWarps + wid; bi < m.n_batch; bi += nwarps) {
        const long long px = m.batch[bi];
        const int n = m.sets.n[px];
        if (n <= 0) continue;  // warp-uniform
        const float plv[3] = {m.sets.plain[3 * px], m.sets.plain[3 * px + 1], m.sets.plain[3 * px + 2]};
        const float4 info = __ldg(m.sets.info + px);
        unsigned a[4][4];
        load_features(m.sets, px, n, g, t, info, plv, a);
        // per-sample weights, outputs and the pixel's loss
        float zw[4], zc[4], w[4], cf[4], cr[4][3];
        bool valid[4];
        float sw = 0.f, sr = 0.f, sg = 0.f, sb = 0.f, sc = 0.f;
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            const int s = 16 * mt + g + 8 * t;
            float e[4];
            tile_forward(a[mt], bw, s_b1, bw2, b20, b21, t, e);
            const float zw8 = __shfl_sync(0xffffffffu, e[2], lane & ~3);
            const float zc8 = __shfl_sync(0xffffffffu, e[3], lane & ~3);
            zw[mt] = t == 0 ? e[0] : zw8;
            zc[mt] = t == 0 ? e[1] : zc8;
            valid[mt] = t < 2 && s < n;
            w[mt] = valid[mt] ? softplusf(zw[mt]) : 0.f;
            cf[mt] = valid[mt] ? sigmoidf(zc[mt]) : 0.f;
            const float4 c = __ldg(m.sets.col + px * kS + (valid[mt] ? s : 0));
            cr[mt][0] = valid[mt] ? c.x : 0.f;
            cr[mt][1] = valid[mt] ? c.y : 0.f;
            cr[mt][2] = valid[mt] ? c.z : 0.f;
            sw += w[mt];
            sr = fmaf(w[mt], cr[mt][0], sr);
            sg = fmaf(w[mt], cr[mt][1], sg);
            sb = fmaf(w[mt], cr[mt][2], sb);
            sc += cf[mt];
        }
        sw = warp_sum(sw);
        sr = warp_sum(sr);
        sg = warp_sum(sg);
        sb = warp_sum(sb);
        sc = warp_sum(sc);
        const float inv_w = 1.0f / sw;
        const float ol[3] = {sr * inv_w, sg * inv_w, sb * inv_w};
        const float conf = sc / (float)n;
        const long long u = px % m.cw + m.x0, v = px / m.cw + m.y0;
        const float *y = m.clean + (((long long)m.O * m.H + v) * m.W + u) * 3;
        const float *pl = plv;
        float el = 0.f, ep = 0.f, dO[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            el += (ol[c] - y[c]) * (ol[c] - y[c]) * (1.0f / 3.0f);
            ep += (pl[c] - y[c]) * (pl[c] - y[c]) * (1.0f / 3.0f);
            dO[c] = 2.0f * (ol[c] - y[c]) * (1.0f / 3.0f) * inv_np;
        }
        const float tgt = el <= ep ? 1.0f : 0.0f;
        const float cc = fminf(fmaxf(conf, 1e-6f), 1.0f - 1e-6f);
        const bool inside = conf > 1e-6f && conf < 1.0f - 1e-6f;
        const float dconf = inside ? m.bce_w * (cc - tgt) / (cc * (1.0f - cc)) * inv_np : 0.0f;
        if (lane == 0) atomicAdd(&s_g[kH + 2 * kH + 2], (el - m.bce_w * (tgt * logf(cc) + (1.0f - tgt) * logf(1.0f - cc))) * inv_np);
        // dz per sample (zero outside the set), broadcast to the lanes holding the same rows
        float dzw_own[4], dzc_own[4], gz0 = 0.f, gz1 = 0.f;
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            const float dw = (dO[0] * (cr[mt][0] - ol[0]) + dO[1] * (cr[mt][1] - ol[1]) + dO[2] * (cr[mt][2] - ol[2])) * inv_w;
            dzw_own[mt] = valid[mt] ? dw * sigmoidf(zw[mt]) : 0.f;
            dzc_own[mt] = valid[mt] ? dconf * cf[mt] * (1.0f - cf[mt]) / (float)n : 0.f;
            gz0 += dzw_own[mt];
            gz1 += dzc_own[mt];
        }
        gz0 = warp_sum(gz0);
        gz1 = warp_sum(gz1);
        if (lane == 0) {
            atomicAdd(&s_g[kH + 2 * kH], gz0);
            atomicAdd(&s_g[kH + 2 * kH + 1], gz1);
        }
        float dzw[4][2], dzc[4][2];
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            dzw[mt][0] = __shfl_sync(0xffffffffu, dzw_own[mt], g * 4 + 0);
            dzw[mt][1] = __shfl_sync(0xffffffffu, dzw_own[mt], g * 4 + 1);
            dzc[mt][0] = __shfl_sync(0xffffffffu, dzc_own[mt], g * 4 + 0);
            dzc[mt][1] = __shfl_sync(0xffffffffu, dzc_own[mt], g * 4 + 1);
        }
        // recompute H per 8-column tile: dW2, db1, dH (to shared memory as BF16)
#pragma unroll 1
        for (int nt = 0; nt < 8; ++nt) {
            const int c0 = 8 * nt + 2 * t;
            const float bias0 = __ldg(m.w.b1 + c0), bias1 = __ldg(m.w.b1 + c0 + 1);
            const float w00 = __ldg(m.w.W2 + c0), w01 = __ldg(m.w.W2 + c0 + 1);
            const float w10 = __ldg(m.w.W2 + kH + c0), w11 = __ldg(m.w.W2 + kH + c0 + 1);
            const float cinit[4] = {bias0, bias1, bias0, bias1};
            float g0a = 0.f, g0b = 0.f, g1a = 0.f, g1b = 0.f, gba = 0.f, gbb = 0.f;
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                float d[4];
                mma_bf16(d, a[mt], bw[nt][0], bw[nt][1], cinit);
                // the hidden values layer 2 saw: ReLU, rounded to BF16
                const __nv_bfloat162 r01 = u32_as_bf162(relu_bf16x2(d[0], d[1])), r23 = u32_as_bf162(relu_bf16x2(d[2], d[3]));
                const float h0 = __low2float(r01), h1 = __high2float(r01), h2 = __low2float(r23), h3 = __high2float(r23);
                g0a += dzw[mt][0] * h0 + dzw[mt][1] * h2;
                g0b += dzw[mt][0] * h1 + dzw[mt][1] * h3;
                g1a += dzc[mt][0] * h0 + dzc[mt][1] * h2;
                g1b += dzc[mt][0] * h1 + dzc[mt][1] * h3;
                const float dh0 = d[0] > 0.f ? dzw[mt][0] * w00 + dzc[mt][0] * w10 : 0.f;
                const float dh1 = d[1] > 0.f ? dzw[mt][0] * w01 + dzc[mt][0] * w11 : 0.f;
                const float dh2 = d[2] > 0.f ? dzw[mt][1] * w00 + dzc[mt][1] * w10 : 0.f;
                const float dh3 = d[3] > 0.f ? dzw[mt][1] * w01 + dzc[mt][1] * w11 : 0.f;
                gba += dh0 + dh2;
                gbb += dh1 + dh3;
                __nv_bfloat162 p01 = __floats2bfloat162_rn(dh0, dh1), p23 = __floats2bfloat162_rn(dh2, dh3);
                *reinterpret_cast<__nv_bfloat162 *>(dh + (16 * mt + g) * kLd + c0) = p01;
                *reinterpret_cast<__nv_bfloat162 *>(dh + (16 * mt + g + 8) * kLd + c0) = p23;
            }
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                g0a += __shfl_xor_sync(0xffffffffu, g0a, o);
                g0b += __shfl_xor_sync(0xffffffffu, g0b, o);
                g1a += __shfl_xor_sync(0xffffffffu, g1a, o);
                g1b += __shfl_xor_sync(0xffffffffu, g1b, o);
                gba += __shfl_xor_sync(0xffffffffu, gba, o);
                gbb += __shfl_xor_sync(0xffffffffu, gbb, o);
            }
            if (g == 0) {
                atomicAdd(&s_g[kH + c0], g0a);
                atomicAdd(&s_g[kH + c0 + 1], g0b);
                atomicAdd(&s_g[kH + kH + c0], g1a);
                atomicAdd(&s_g[kH + kH + c0 + 1], g1b);
                atomicAdd(&s_g[c0], gba);
                atomicAdd(&s_g[c0 + 1], gbb);
            }
        }
        __syncwarp();
        // dW1 (64 hidden x 16 features) += dH^T F over the 64 samples: M = hidden, N = feature, K = sample
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const int s0 = 16 * kt + 2 * t, s1 = s0 + 1, s8 = s0 + 8, s9 = s0 + 9;
            unsigned bf[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int i = 8 * nt + g;
                bf[nt][0] = pack2(s0 < n ? feature_bits(m.sets, px, s0, i, info, plv) : 0,
                                  s1 < n ? feature_bits(m.sets, px, s1, i, info, plv) : 0);
                bf[nt][1] = pack2(s8 < n ? feature_bits(m.sets, px, s8, i, info, plv) : 0,
                                  s9 < n ? feature_bits(m.sets, px, s9, i, info, plv) : 0);
            }
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                const int j0 = 16 * mt + g, j8 = j0 + 8;
                unsigned af[4];
                af[0] = pack2(dh[s0 * kLd + j0], dh[s1 * kLd + j0]);
                af[1] = pack2(dh[s0 * kLd + j8], dh[s1 * kLd + j8]);
                af[2] = pack2(dh[s8 * kLd + j0], dh[s9 * kLd + j0]);
                af[3] = pack2(dh[s8 * kLd + j8], dh[s9 * kLd + j8]);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    float d[4];
                    mma_bf16(d, af, bf[nt][0], bf[nt][1], dW1[mt][nt]);
                    dW1[mt][nt][0] = d[0];
                    dW1[mt][nt][1] = d[1];
                    dW1[mt][nt][2] = d[2];
                    dW1[mt][nt][3] = d[3];
                }
            }
        }
        __syncwarp();  // dH is rewritten by the next pixel
    }
    // flush: dW1 fragments (rows = hidden 16 mt + g (+8), cols = feature 8 nt + 2 t (+1))
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int j0 = 16 * mt + g, i0 = 8 * nt + 2 * t;
            atomicAdd(m.grad + j0 * kF + i0, dW1[mt][nt][0]);
            atomicAdd(m.grad + j0 * kF + i0 + 1, dW1[mt][nt][1]);
            atomicAdd(m.grad + (j0 + 8) * kF + i0, dW1[mt][nt][2]);
            atomicAdd(m.grad + (j0 + 8) * kF + i0 + 1, dW1[mt][nt][3]);
        }
    __syncthreads();
    for (int i = threadIdx.x; i < kH + 2 * kH + 3; i += blockDim.x) atomicAdd(m.grad + kH * kF + i, s_g[i]);
}

// ---------------------------------------------------------------- Adam on the FP32 master weights
// Compact sample sets expanded to the full layout (64 x 16 BF16 features, 64 x 3 colours per
// pixel), for callers that read the sets themselves.
__global__ void expand_sets_kernel(const SampleSets S, unsigned short *feat, float *col, int32_t *nsamp, float *plain,
                                   long long n_px) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n_px * kS) return;
    const long long px = i / kS;
    const int s = (int)(i - px * kS), n = S.n[px];
    const float pl[3] = {S.plain[3 * px], S.plain[3 * px + 1], S.plain[3 * px + 2]};
    if (s == 0) {
        nsamp[px] = n;
        for (int c = 0; c < 3; ++c) plain[3 * px + c] = pl[c];
    }
    unsigned *f = reinterpret_cast<unsigned *>(feat + i * kF);
    if (s >= n) {
        for (int w = 0; w < 8; ++w) f[w] = 0u;
        col[3 * i] = col[3 * i + 1] = col[3 * i + 2] = 0.0f;
        return;
    }
    const float4 c = S.col[i], info = S.info[px];
    const unsigned f89 = S.f89[i];
    for (int w = 0; w < 8; ++w) f[w] = feat_word(w, c, f89, info, pl);
    col[3 * i] = c.x;
    col[3 * i + 1] = c.y;
    col[3 * i + 2] = c.z;
}

__global__ void adam_kernel(MlpState st, float lr, float b1, float b2, float eps, int step) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float gr = st.grad[i];
    const float m = b1 * st.m[i] + (1.0f - b1) * gr;
    const float v = b2 * st.v[i] + (1.0f - b2) * gr * gr;
    st.m[i] = m;
    st.v[i] = v;
    const float mh = m / (1.0f - powf(b1, (float)step)), vh = v / (1.0f - powf(b2, (float)step));
    const float p = st.master[i] - lr * mh / (sqrtf(vh) + eps);
    st.master[i] = p;
    refresh_one(st, i, p);
}

__global__ void refresh_kernel(MlpState st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kMlpParams) refresh_one(st, i, st.master[i]);
}

}  // namespace

cudaError_t launch_mlp_train(const MlpArgs &m, cudaStream_t s) {
    if (m.n_batch <= 0) return cudaSuccess;
    long long blocks = (m.n_batch + kWarps - 1) / kWarps;
    if (blocks > 152 * 8) blocks = 152 * 8;
    mlp_train_kernel<<<(unsigned)blocks, 32 * kWarps, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_adam(const MlpState &st, float lr, int step, cudaStream_t s) {
    adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(st, lr, 0.9f, 0.999f, 1e-8f, step);
    return cudaGetLastError();
}

cudaError_t launch_mlp_refresh(const MlpState &st, cudaStream_t s) {
    refresh_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_expand_sets(const SampleSets &sets, unsigned short *feat, float *col, int32_t *nsamp, float *plain,
                               long long n_px, cudaStream_t s) {
    const long long n = n_px * kS;
    if (n == 0) return cudaSuccess;
    expand_sets_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sets, feat, col, nsamp, plain, n_px);
    return cudaGetLastError();
}

}  // namespace ssvp
