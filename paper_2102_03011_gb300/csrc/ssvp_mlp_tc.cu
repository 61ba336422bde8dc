// ssvp_mlp_tc.cu - learned-filter inference and training on the 5th-generation tensor cores
// (tcgen05).  Inference first; the training kernel, which reuses its forward pass, follows it.
//
// One CTA of 128 threads takes two pixels at a time: their 2 x 64 capped samples are the 128 rows
// of the layer-1 product.  While layer 2 of one pair runs, the threads build the next pair's
// features; while its layer 1 runs, they finish the previous pair and load the records of the
// next.  Eight CTAs share an SM (64 tensor-memory columns each), so that other CTAs' warps issue
// while one waits for its products.  Each thread owns one row (one sample):
//   1. it builds the sample's 16 BF16 features and stores them into shared memory in the
//      tensor cores' K-major core-matrix layout (8 rows x 16 bytes per core matrix);
//   2. one elected thread issues tcgen05.mma: D1 (128 x 64, FP32, in tensor memory) = F W1^T;
//      b1 enters the same accumulator: the logical feature 15 is the constant 0, so its slot
//      carries 1.0 and W1's column 15 b1's leading BF16 part, and a second MMA with a constant
//      operand adds b1's two lower BF16 parts (hi + mid + lo represent the FP32 b1 exactly);
//   3. each thread reads its row of D1 back (tcgen05.ld), applies the ReLU and rounds to BF16 in
//      one conversion, and writes the row back into tensor memory (tcgen05.st) as layer 2's A
//      operand: H's 64 BF16 values take D1's first 32 columns, two to a column;
//   4. four tcgen05.mma with A in tensor memory (K = 16 each): D2 (128 x 16 in the columns after
//      H, columns 0 and 1 used) = H W2^T;
//   5. each thread reads (z_w, z_c) of its row, adds b2, and forms softplus / sigmoid; the two
//      warps of each pixel reduce the weighted sums.
// BF16 operands, FP32 accumulation, h rounded to BF16 before layer 2 (the training kernel below
// runs the same forward pass).  Waits on the MMA-completion barrier are
// bounded: on a time-out the kernel raises the error word, leaves its loop, frees its tensor
// memory and returns.
#include <cuda_bf16.h>

#include "ssvp_internal.h"

namespace ssvp {
namespace {

constexpr int kS = 64, kF = 16, kH = 64;
constexpr int kTcThreads = 128;   // one sample row per thread, two pixels per CTA
constexpr unsigned kTmemCols = 64;  // D1; then H in its first 32 columns and D2 in the next 16
constexpr unsigned kColD2 = 32;
constexpr int kTcCtasPerSm = 8;
// shared operands, K-major core matrices; core (i, j) of an R x K operand holds rows 8i..8i+7 and
// K elements 8j..8j+7 at byte offset (i * K / 8 + j) * 128, row r of it at + 16 (r % 8).  One
// feature buffer: a pair's features are written after every thread has waited for the previous
// pair's layer 1.
constexpr int kSmA1 = 0;        // features, 128 x 16
constexpr int kSmB1 = 4096;     // W1, 64 x 16
constexpr int kSmB2 = 6144;     // W2 padded to 16 rows, 16 x 64
constexpr int kSmA0 = 8192;     // constant operand for the b1 residual: ones in K slots 0 and 1, 128 x 16
constexpr int kSmB0 = 12288;    // b1's two lower BF16 parts in K slots 0 and 1, 64 x 16
constexpr int kSmBytes = 14336;
// dynamic shared memory per CTA: the operands, 14 KB.  At most eight CTAs fit on an SM (registers:
// 128 threads x 8 at <= 64), all 1,216 in one wave on 152 SMs, and their 8 x 64 tensor-memory
// columns fit in the SM's 512
constexpr int kSmRequest = kSmBytes;
// a waiting thread suspends in try_wait for up to kWaitHintNs per poll; kWaitLimit polls (about
// 1 s) before a wait counts as timed out
constexpr unsigned kWaitHintNs = 100000, kWaitLimit = 10000;

__device__ __forceinline__ unsigned core_off(int r, int kc, int k_chunks) {
    return (unsigned)(((r >> 3) * k_chunks + kc) * 128 + (r & 7) * 16);
}

// shared-memory matrix descriptor: start, leading (K-direction) and stride (8-row direction) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ unsigned long long smem_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((saddr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, N x M
__host__ __device__ constexpr unsigned instr_desc(int n, int m) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mma_tc(unsigned d_tmem, unsigned long long adesc, unsigned long long bdesc,
                                       unsigned idesc, int accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// the same product with A (M x 16, BF16, two to a 32-bit column, row i in lane i) in tensor memory
__device__ __forceinline__ void mma_tc_ta(unsigned d_tmem, unsigned a_tmem, unsigned long long bdesc, unsigned idesc,
                                          int accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// 8 consecutive 32-bit columns of this thread's tensor-memory lane; the caller waits (tcgen05.wait::st)
__device__ __forceinline__ void tmem_st8(unsigned taddr, const unsigned (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void mma_commit(unsigned mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// bounded wait for the barrier phase with parity `parity`; false on time-out
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        unsigned done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "r"(kWaitHintNs)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane; the caller waits
// (tcgen05.wait::ld) before using them, so that several loads share one wait
__device__ __forceinline__ void tmem_ld32_nowait(unsigned taddr, unsigned (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16_nowait(unsigned taddr, unsigned (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld2(unsigned taddr, float &a, float &b) {
    unsigned r0, r1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    a = __uint_as_float(r0);
    b = __uint_as_float(r1);
}

__device__ __forceinline__ unsigned pack2(unsigned short lo, unsigned short hi) { return (unsigned)lo | ((unsigned)hi << 16); }
__device__ __forceinline__ unsigned short bf16_bits(float x) {
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<const unsigned short *>(&b);
}
// two floats rounded to BF16 in one conversion, the first in the low half
__device__ __forceinline__ unsigned bf16x2(float lo, float hi) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&b);
}
__device__ __forceinline__ unsigned relu_bf16x2(float lo, float hi) {
    unsigned r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
// softplus(x) = max(x, 0) + log(1 + y), y = e^-|x| in (0, 1]: log(1 + y) from the fast logarithm of
// 1 + y (absolute error ~1e-7), or y itself below 1e-4 (relative error < y / 2), so every weight
// keeps a relative error below ~1e-4 down to the smallest ones
__device__ __forceinline__ float softplusf(float x) {
    const float y = __expf(-fabsf(x));
    return fmaxf(x, 0.0f) + (y < 1e-4f ? y : __logf(1.0f + y));
}

// Sums of (a, b, c, d) over the warp's 32 lanes in 6 shuffles: each exchange hands half of the
// values still held to the partner lane, so that after the xor-16 and xor-8 steps every lane holds
// one value (a for lanes with bits (4, 3) = (0, 0), b for (0, 1), c for (1, 0), d for (1, 1)),
// which three more steps complete.  Returns the total of the lane's value.
__device__ __forceinline__ float warp_sum4(float a, float b, float c, float d, int lane) {
    const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0;
    const float ka = h4 ? c : a, kb = h4 ? d : b;
    const float sa = h4 ? a : c, sb = h4 ? b : d;
    const float x = ka + __shfl_xor_sync(0xffffffffu, sa, 16);
    const float y = kb + __shfl_xor_sync(0xffffffffu, sb, 16);
    float v = (h3 ? y : x) + __shfl_xor_sync(0xffffffffu, h3 ? x : y, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}
__device__ __forceinline__ float sigmoidf(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }

// Feature word w of one sample in the logical order (features 2w, 2w + 1, the lower in the low half)
__device__ __forceinline__ unsigned feat_word(int w, float4 c, unsigned f89, float4 info, const float (&pl)[3]) {
    switch (w) {
    case 0: return bf16x2(c.x, c.y);
    case 1: return bf16x2(c.z, c.x - info.x);
    case 2: return bf16x2(c.y - info.y, c.z - info.z);
    case 3: return __float_as_uint(c.w);
    case 4: return f89;
    case 5: return pack2(0x3f80, bf16_bits(info.w));  // BF16 1.0
    case 6: return bf16x2(c.x - pl[0], c.y - pl[1]);
    default: return bf16x2(c.z - pl[2], 0.0f);
    }
}

// The network's operands in shared memory, by the 128 threads of a CTA: W1 (64 x 16) with b1's
// leading BF16 part in column 15 (the logical feature 15 is the constant 0, so its A slot can
// carry 1.0), b1's two lower BF16 parts as the B operand of a residual product with the constant
// operand A0 (rows (1, 1, 0, ..., 0)), and W2 padded to 16 rows (16 x 64)
__device__ __forceinline__ void stage_weights(unsigned char *sm, int offB1, int offB0, int offA0, int offB2,
                                              const MlpWeights &mw, int tid) {
    {
        const int row = tid >> 1, kc = tid & 1;
        uint4 w = __ldg(reinterpret_cast<const uint4 *>(mw.W1 + row * kF + kc * 8));
        const float b = __ldg(mw.b1 + row);
        const unsigned short hi = bf16_bits(b);
        const float r1 = b - __uint_as_float((unsigned)hi << 16);
        const unsigned short mid = bf16_bits(r1);
        const unsigned short lo = bf16_bits(r1 - __uint_as_float((unsigned)mid << 16));
        if (kc == 1) w.w = (w.w & 0xffffu) | ((unsigned)hi << 16);
        *reinterpret_cast<uint4 *>(sm + offB1 + core_off(row, kc, 2)) = w;
        *reinterpret_cast<uint4 *>(sm + offB0 + core_off(row, kc, 2)) =
            kc == 0 ? make_uint4(pack2(mid, lo), 0u, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(sm + offA0 + core_off(tid, 0, 2)) = make_uint4(pack2(0x3f80, 0x3f80), 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(sm + offA0 + core_off(tid, 1, 2)) = make_uint4(0u, 0u, 0u, 0u);
    }
    {
        const int row = tid >> 3, kc = tid & 7;
        unsigned q[4] = {0u, 0u, 0u, 0u};
        if (row < 2) {
            const float *src = mw.W2 + row * kH + kc * 8;
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] = bf16x2(__ldg(src + 2 * i), __ldg(src + 2 * i + 1));
        }
        *reinterpret_cast<uint4 *>(sm + offB2 + core_off(row, kc, 8)) = make_uint4(q[0], q[1], q[2], q[3]);
    }
}

// One pixel pair's data as a thread needs it: its sample row (colour record, depth / weight
// pair), the pixel's info, plain result and set size
struct RowData {
    float4 c, info;
    unsigned f89;
    float pl[3];
    int n;
    int px;  // crop pixel (crops hold fewer than 2^26 pixels)
};

// what the epilogue of the previous pair keeps
struct PrevRow {
    float3 c;
    float pl[3];
    int n;
    int px;  // crop pixel (crops hold fewer than 2^26 pixels)
};

__device__ __forceinline__ void load_row(const MlpArgs &m, int pair, int tid, RowData &r) {
    r.px = 2 * pair + (tid >> 6);
    const int s = tid & 63;
    r.n = 0;
    r.c = r.info = make_float4(0.f, 0.f, 0.f, 0.f);
    r.f89 = 0u;
    r.pl[0] = r.pl[1] = r.pl[2] = 0.0f;
    if (r.px < m.n_px) {
        // the set's storage holds 64 rows per pixel: rows past n are read (in bounds) and ignored,
        // so that no load waits on the count
        const unsigned k = (unsigned)r.px * kS + s;  // below 2^32: crops hold fewer than 2^26 pixels
        r.n = m.sets.n[r.px];
        r.c = __ldg(m.sets.col + k);
        r.f89 = __ldg(m.sets.f89 + k);
        r.info = __ldg(m.sets.info + r.px);
        r.pl[0] = m.sets.plain[3 * r.px];
        r.pl[1] = m.sets.plain[3 * r.px + 1];
        r.pl[2] = m.sets.plain[3 * r.px + 2];
    }
}

// Iteration i of a CTA takes pixel pair blockIdx.x + i * gridDim.x.  The 64 tensor-memory
// columns hold D1 of pair i, then its H (columns 0-31) and D2 (columns 32-47): the threads read D2
// of pair i - 1 (after building the features of pair i) before layer 1 of pair i is issued.
__device__ __forceinline__ void pair_sums(float zw, float zc, const PrevRow &pr, float b20, float b21, int s_row,
                                          int warp, int lane, float (*s_red)[5]) {
    float sw = 0.f, sr = 0.f, sg = 0.f, sb = 0.f, sc = 0.f;
    if (s_row < pr.n) {
        const float w = softplusf(zw + b20);
        sw = w;
        sr = w * pr.c.x;
        sg = w * pr.c.y;
        sb = w * pr.c.z;
        sc = sigmoidf(zc + b21);
    }
    const float t4 = warp_sum4(sw, sr, sg, sb, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sc += __shfl_xor_sync(0xffffffffu, sc, o);
    if ((lane & 7) == 0) s_red[warp][lane >> 3] = t4;
    if (lane == 0) s_red[warp][4] = sc;
}

// the output of a pixel from the per-warp sums of its two warps (w0, w0 + 1)
__device__ __forceinline__ void pair_output(const MlpArgs &m, const PrevRow &pr, int w0, const float (*s_red)[5]) {
    float o0 = pr.pl[0], o1 = pr.pl[1], o2 = pr.pl[2], conf = 0.0f;
    if (pr.n > 0) {
        const float tw = s_red[w0][0] + s_red[w0 + 1][0];
        conf = __fdividef(s_red[w0][4] + s_red[w0 + 1][4], (float)pr.n);
        if (conf >= m.tau && tw > 0.0f) {
            const float inv = __frcp_rn(tw);
            o0 = (s_red[w0][1] + s_red[w0 + 1][1]) * inv;
            o1 = (s_red[w0][2] + s_red[w0 + 1][2]) * inv;
            o2 = (s_red[w0][3] + s_red[w0 + 1][3]) * inv;
        }
    }
    const long long u = m.x0 + pr.px % m.cw, v = m.y0 + pr.px / m.cw;
    float *o = m.out + (((long long)m.O * m.H + v) * m.W + u) * 3;
    o[0] = o0;
    o[1] = o1;
    o[2] = o2;
    if (m.conf_out) m.conf_out[pr.px] = conf;
}

__global__ void __launch_bounds__(kTcThreads, kTcCtasPerSm) mlp_infer_tc_kernel(const MlpArgs m, int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ float s_red[4][5];
    __shared__ unsigned long long s_mbar[2];  // layer-1 and layer-2 completion
    __shared__ unsigned s_tmem;
    __shared__ int s_bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, s_row = tid & 63;

    stage_weights(sm, kSmB1, kSmB0, kSmA0, kSmB2, m.w, tid);
    const float b20 = __ldg(m.w.b2), b21 = __ldg(m.w.b2 + 1);
    const unsigned bar1 = smem_u32(&s_mbar[0]), bar2 = smem_u32(&s_mbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar2) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_bad = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = s_tmem;
    const unsigned lane_base = (unsigned)(warp * 32) << 16;  // this warp's 32 lanes
    const unsigned sbase = smem_u32(sm);
    const unsigned long long dA1 = smem_desc(sbase + kSmA1, 128, 256), dB1 = smem_desc(sbase + kSmB1, 128, 256),
                             dA0 = smem_desc(sbase + kSmA0, 128, 256), dB0 = smem_desc(sbase + kSmB0, 128, 256);
    constexpr unsigned id1 = instr_desc(kH, 128), id2 = instr_desc(16, 128);
    unsigned ph1 = 0, ph2 = 0;
    bool bad = false;

    const int n_pairs = (int)((m.n_px + 1) / 2);
    RowData cur;
    PrevRow prev;
    prev.n = 0;
    prev.px = n_pairs * 2;
    if ((int)blockIdx.x < n_pairs) load_row(m, blockIdx.x, tid, cur);
    int it = 0;
    for (int pair = blockIdx.x; pair < n_pairs; pair += gridDim.x, ++it) {
        // 1. this pair's features (the single A1 buffer is free: every thread has waited for the
        // previous pair's layer 1)
        {
            unsigned wd[8];
#pragma unroll
            for (int w = 0; w < 8; ++w) wd[w] = s_row < cur.n ? feat_word(w, cur.c, cur.f89, cur.info, cur.pl) : 0u;
            if (s_row < cur.n) wd[7] |= 0x3f80u << 16;  // slot 15 (feature 15 = 0) carries 1.0 for b1
            unsigned char *A1 = sm + kSmA1;
            *reinterpret_cast<uint4 *>(A1 + core_off(tid, 0, 2)) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
            *reinterpret_cast<uint4 *>(A1 + core_off(tid, 1, 2)) = make_uint4(wd[4], wd[5], wd[6], wd[7]);
        }
        // 2. the previous pair's (z_w, z_c), read before this pair's layer 1 overwrites the columns
        if (it > 0) {
            bad |= !mbar_wait(bar2, ph2);
            ph2 ^= 1u;
            fence_after();
            float zw, zc;
            tmem_ld2(tmem + kColD2 + lane_base, zw, zc);
            pair_sums(zw, zc, prev, b20, b21, s_row, warp, lane, s_red);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (s_bad) break;  // uniform: written only between the second barrier and the next first one
        if (tid == 0 && !m.skip_mma) {
            fence_after();
            mma_tc(tmem, dA1, dB1, id1, 0);
            mma_tc(tmem, dA0, dB0, id1, 1);
            mma_commit(bar1);
        }
        // 3. the previous pair's outputs (threads 32 and 96: the second warp of each pixel, so that
        // warp 0, which issues the MMAs, goes on first)
        if (it > 0 && s_row == 32 && prev.px < m.n_px) pair_output(m, prev, warp - 1, s_red);
        prev.c = make_float3(cur.c.x, cur.c.y, cur.c.z);
        prev.n = cur.n;
        prev.px = cur.px;
        prev.pl[0] = cur.pl[0];
        prev.pl[1] = cur.pl[1];
        prev.pl[2] = cur.pl[2];
        // 4. the next pair's records, in flight during the waits below and the next features
        if (pair + (int)gridDim.x < n_pairs) load_row(m, pair + gridDim.x, tid, cur);
        // 5. H = ReLU(D1 + b1) in BF16, written over D1's first 32 columns as layer 2's A operand,
        // then layer 2 into the next 16 columns
        bad |= !mbar_wait(bar1, ph1);
        ph1 ^= 1u;
        fence_after();
        // a quarter of the row (16 columns) at a time: quarter q's 8 packed columns go to columns
        // 8q..8q+7, which this thread has read already (quarters 0 and 1)
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            unsigned v[16];
            tmem_ld16_nowait(tmem + lane_base + 16u * qq, v);
            tmem_wait_ld();
            unsigned h[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) h[i] = relu_bf16x2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
            tmem_st8(tmem + lane_base + 8u * qq, h);
        }
        tmem_wait_st();
        fence_before();
        __syncthreads();
        if (tid == 0 && !m.skip_mma) {
            fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_tc_ta(tmem + kColD2, tmem + 8u * kk, smem_desc(sbase + kSmB2 + kk * 256, 128, 1024), id2, kk);
            mma_commit(bar2);
        }
        if (bad) s_bad = 1;
    }
    __syncthreads();  // s_bad is settled for every thread
    // the last pair: its layer 2 is in flight
    if (it > 0 && !s_bad) {
        bad |= !mbar_wait(bar2, ph2);
        ph2 ^= 1u;
        fence_after();
        float zw, zc;
        tmem_ld2(tmem + kColD2 + lane_base, zw, zc);
        pair_sums(zw, zc, prev, b20, b21, s_row, warp, lane, s_red);
        __syncthreads();
        if (s_row == 32 && prev.px < m.n_px) pair_output(m, prev, warp - 1, s_red);
    }
    if (bad) atomicOr(err, 1);
    // after a time-out the tensor cores may still be busy: one more bounded wait on each barrier
    if (s_bad && tid == 0) {
        mbar_wait(bar1, ph1);
        mbar_wait(bar2, ph2);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------- training on the tensor cores
// One CTA of 128 threads takes two batch pixels at a time, one thread per sample row, and runs
// the forward pass exactly as the inference does (layer 1 with b1 folded in, ReLU and BF16
// rounding, layer 2).  Two threads then form their pixel's loss terms (the learned output, the
// MSE of it and of the plain result against the clean target, the BCE target and its confidence
// derivative), and every thread its sample's dz = (dL/dz_w, dL/dz_c) and
// dh_j = (dz_w W2[0][j] + dz_c W2[1][j]) [h_j > 0].  The weight gradients are one tcgen05 product
// per pair, accumulated over the whole kernel in tensor memory:
//   G (128 x 32) += A_G B_G^T, K = the pair's 128 sample rows, with
//   A_G rows 0..63 = h^T and rows 64..127 = dh^T (hidden unit x sample), and
//   B_G rows 0, 1 = dz_w, dz_c, rows 2..17 = the 16 features, row 18 = 1, rows 19..31 = 0,
// so G[j][0..1] holds dW2^T, G[64 + j][2..17] dW1 and G[64 + j][18] db1 (the other blocks go
// unused).  Each thread writes its sample's column of both operands (K-major, so a sample's
// values spread over the rows).  All operands are BF16 with FP32 accumulation: h, dh, dz and
// the features enter the gradient products rounded to BF16.  db2 and the loss are FP32 sums.
constexpr int kTrSmA1 = 0;          // features, 128 x 16
constexpr int kTrSmB1 = 4096;       // W1, 64 x 16
constexpr int kTrSmA0 = 6144;       // constant operand of the b1 residual, 128 x 16
constexpr int kTrSmB0 = 10240;      // b1's lower parts, 64 x 16
constexpr int kTrSmB2 = 12288;      // W2 padded, 16 x 64
constexpr int kTrSmA2 = 14336;      // H, 128 x 64
constexpr int kTrSmAG = 30720;      // A_G, 128 x 128
constexpr int kTrSmBG = 63488;      // B_G, 32 x 128
constexpr int kTrSmBytes = 71680;   // three CTAs per SM: 3 x 128 tensor-memory columns fit in 512
constexpr unsigned kTrTmemCols = 128;   // D1 [0, 64), D2 [64, 80), G [96, 128)
constexpr unsigned kTrColD2 = 64, kTrColG = 96;

// byte offset of element (row, k) of a K-major operand with K = 128 (16 core matrices per row group)
__device__ __forceinline__ unsigned kmajor128(int row, int k) { return core_off(row, k >> 3, 16) + (unsigned)(k & 7) * 2u; }

__global__ void __launch_bounds__(kTcThreads, 3) mlp_train_tc_kernel(const MlpArgs m, int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ float s_red[4][5];
    __shared__ float s_pix[2][8];  // per pixel: dL/d output (3), dL/d conf, 1 / sum w, learned output (3)
    __shared__ float s_w2[2][kH];  // W2 as rounded to BF16
    __shared__ float s_acc[3];     // db2 (2) and the loss of the CTA
    __shared__ unsigned long long s_mbar[3];  // layer 1, layer 2, gradient product
    __shared__ unsigned s_tmem;
    __shared__ int s_bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, srow = tid & 63, pix = tid >> 6;

    stage_weights(sm, kTrSmB1, kTrSmB0, kTrSmA0, kTrSmB2, m.w, tid);
    // the constant rows of B_G at this thread's sample column: row 18 = 1, rows 19..31 = 0
#pragma unroll
    for (int n = 18; n < 32; ++n)
        *reinterpret_cast<unsigned short *>(sm + kTrSmBG + kmajor128(n, tid)) = n == 18 ? (unsigned short)0x3f80 : 0;
    s_w2[tid >> 6][tid & 63] = __ldg(m.w.W2 + tid);
    const float b20 = __ldg(m.w.b2), b21 = __ldg(m.w.b2 + 1);
    const unsigned bar1 = smem_u32(&s_mbar[0]), bar2 = smem_u32(&s_mbar[1]), bar3 = smem_u32(&s_mbar[2]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar2) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar3) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_bad = 0;
        s_acc[0] = s_acc[1] = s_acc[2] = 0.0f;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTrTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = s_tmem;
    const unsigned lane_base = (unsigned)(warp * 32) << 16;
    const unsigned sbase = smem_u32(sm);
    const unsigned long long dA1 = smem_desc(sbase + kTrSmA1, 128, 256), dB1 = smem_desc(sbase + kTrSmB1, 128, 256),
                             dA0 = smem_desc(sbase + kTrSmA0, 128, 256), dB0 = smem_desc(sbase + kTrSmB0, 128, 256);
    constexpr unsigned id1 = instr_desc(kH, 128), id2 = instr_desc(16, 128), idg = instr_desc(32, 128);
    unsigned ph1 = 0, ph2 = 0, ph3 = 0;
    bool bad = false, g_started = false;
    float db2w = 0.0f, db2c = 0.0f, loss = 0.0f;
    const float inv_np = 1.0f / (float)m.n_batch;
    const long long n_pairs = (m.n_batch + 1) / 2;

    for (long long pair = blockIdx.x; pair < n_pairs; pair += gridDim.x) {
        // 1. the sample row of this thread
        const long long bi = 2 * pair + pix;
        long long px = 0;
        int n = 0;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f), info = make_float4(0.f, 0.f, 0.f, 0.f);
        unsigned f89 = 0u;
        float pl[3] = {0.f, 0.f, 0.f};
        if (bi < m.n_batch) {
            px = m.batch[bi];
            n = m.sets.n[px];
            const long long k = px * kS + srow;
            c = __ldg(m.sets.col + k);
            f89 = __ldg(m.sets.f89 + k);
            info = __ldg(m.sets.info + px);
            pl[0] = m.sets.plain[3 * px];
            pl[1] = m.sets.plain[3 * px + 1];
            pl[2] = m.sets.plain[3 * px + 2];
        }
        const bool valid = srow < n;
        // 2. features (logical order; slot 15 carries 1.0 for b1 in the layer-1 operand only)
        unsigned wd[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) wd[w] = valid ? feat_word(w, c, f89, info, pl) : 0u;
        *reinterpret_cast<uint4 *>(sm + kTrSmA1 + core_off(tid, 0, 2)) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        *reinterpret_cast<uint4 *>(sm + kTrSmA1 + core_off(tid, 1, 2)) =
            make_uint4(wd[4], wd[5], wd[6], valid ? wd[7] | (0x3f80u << 16) : 0u);
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (s_bad) break;  // uniform: written only before the barrier above
        if (tid == 0 && !m.skip_mma) {
            fence_after();
            mma_tc(tmem, dA1, dB1, id1, 0);
            mma_tc(tmem, dA0, dB0, id1, 1);
            mma_commit(bar1);
        }
        bad |= !mbar_wait(bar1, ph1);
        ph1 ^= 1u;
        fence_after();
        // 3. H = ReLU(D1) in BF16: layer 2's A operand, kept in registers for the gradients
        unsigned h[32];
        {
            unsigned v0[32], v1[32];
            tmem_ld32_nowait(tmem + lane_base, v0);
            tmem_ld32_nowait(tmem + lane_base + 32, v1);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                h[i] = relu_bf16x2(__uint_as_float(v0[2 * i]), __uint_as_float(v0[2 * i + 1]));
                h[16 + i] = relu_bf16x2(__uint_as_float(v1[2 * i]), __uint_as_float(v1[2 * i + 1]));
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            *reinterpret_cast<uint4 *>(sm + kTrSmA2 + core_off(tid, q, 8)) =
                make_uint4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (tid == 0 && !m.skip_mma) {
            fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_tc(tmem + kTrColD2, smem_desc(sbase + kTrSmA2 + kk * 256, 128, 1024),
                       smem_desc(sbase + kTrSmB2 + kk * 256, 128, 1024), id2, kk);
            mma_commit(bar2);
        }
        bad |= !mbar_wait(bar2, ph2);
        ph2 ^= 1u;
        fence_after();
        float zw, zc;
        tmem_ld2(tmem + kTrColD2 + lane_base, zw, zc);
        zw += b20;
        zc += b21;
        // 4. the pixel's sums: weights, weighted colours, confidences
        const float wgt = valid ? softplusf(zw) : 0.0f, sgm = valid ? sigmoidf(zc) : 0.0f;
        const float t4 = warp_sum4(wgt, wgt * c.x, wgt * c.y, wgt * c.z, lane);
        float sc = sgm;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sc += __shfl_xor_sync(0xffffffffu, sc, o);
        if ((lane & 7) == 0) s_red[warp][lane >> 3] = t4;
        if (lane == 0) s_red[warp][4] = sc;
        __syncthreads();
        // 5. the pixel's loss and the derivatives of its output and confidence
        if (srow == 32) {
            float P[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (n > 0) {
                const int w0 = warp - 1;
                const float sw = s_red[w0][0] + s_red[w0 + 1][0];
                const float inv_w = 1.0f / sw;
                const float ol[3] = {(s_red[w0][1] + s_red[w0 + 1][1]) * inv_w, (s_red[w0][2] + s_red[w0 + 1][2]) * inv_w,
                                     (s_red[w0][3] + s_red[w0 + 1][3]) * inv_w};
                const float conf = (s_red[w0][4] + s_red[w0 + 1][4]) / (float)n;
                const long long u = px % m.cw + m.x0, v = px / m.cw + m.y0;
                const float *y = m.clean + (((long long)m.O * m.H + v) * m.W + u) * 3;
                float el = 0.f, ep = 0.f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    el += (ol[ch] - y[ch]) * (ol[ch] - y[ch]) * (1.0f / 3.0f);
                    ep += (pl[ch] - y[ch]) * (pl[ch] - y[ch]) * (1.0f / 3.0f);
                    P[ch] = 2.0f * (ol[ch] - y[ch]) * (1.0f / 3.0f) * inv_np;
                    P[5 + ch] = ol[ch];
                }
                const float tgt = el <= ep ? 1.0f : 0.0f;
                const float cc = fminf(fmaxf(conf, 1e-6f), 1.0f - 1e-6f);
                const bool inside = conf > 1e-6f && conf < 1.0f - 1e-6f;
                P[3] = inside ? m.bce_w * (cc - tgt) / (cc * (1.0f - cc)) * inv_np : 0.0f;
                P[4] = inv_w;
                loss += (el - m.bce_w * (tgt * logf(cc) + (1.0f - tgt) * logf(1.0f - cc))) * inv_np;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) s_pix[pix][i] = P[i];
        }
        __syncthreads();
        // 6. this sample's dz
        float dzw = 0.0f, dzc = 0.0f;
        if (valid) {
            const float *P = s_pix[pix];
            const float dw = (P[0] * (c.x - P[5]) + P[1] * (c.y - P[6]) + P[2] * (c.z - P[7])) * P[4];
            dzw = dw * sigmoidf(zw);
            dzc = P[3] * sgm * (1.0f - sgm) / (float)n;
        }
        db2w += dzw;
        db2c += dzc;
        // 7. the previous gradient product has read A_G and B_G before they are rewritten
        if (g_started) {
            bad |= !mbar_wait(bar3, ph3);
            ph3 ^= 1u;
        }
        // 8. this sample's column of A_G (h, then dh) and of B_G (dz, features)
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const float h0 = __uint_as_float(h[q] << 16), h1 = __uint_as_float(h[q] & 0xffff0000u);
            const int j = 2 * q;
            const float dh0 = h0 > 0.0f ? fmaf(dzw, s_w2[0][j], dzc * s_w2[1][j]) : 0.0f;
            const float dh1 = h1 > 0.0f ? fmaf(dzw, s_w2[0][j + 1], dzc * s_w2[1][j + 1]) : 0.0f;
            const unsigned d2 = bf16x2(dh0, dh1);
            *reinterpret_cast<unsigned short *>(sm + kTrSmAG + kmajor128(j, tid)) = (unsigned short)(h[q] & 0xffffu);
            *reinterpret_cast<unsigned short *>(sm + kTrSmAG + kmajor128(j + 1, tid)) = (unsigned short)(h[q] >> 16);
            *reinterpret_cast<unsigned short *>(sm + kTrSmAG + kmajor128(64 + j, tid)) = (unsigned short)(d2 & 0xffffu);
            *reinterpret_cast<unsigned short *>(sm + kTrSmAG + kmajor128(65 + j, tid)) = (unsigned short)(d2 >> 16);
        }
        {
            const unsigned dz2 = bf16x2(dzw, dzc);
            *reinterpret_cast<unsigned short *>(sm + kTrSmBG + kmajor128(0, tid)) = (unsigned short)(dz2 & 0xffffu);
            *reinterpret_cast<unsigned short *>(sm + kTrSmBG + kmajor128(1, tid)) = (unsigned short)(dz2 >> 16);
#pragma unroll
            for (int i = 0; i < 16; ++i)
                *reinterpret_cast<unsigned short *>(sm + kTrSmBG + kmajor128(2 + i, tid)) =
                    (unsigned short)((i & 1) ? wd[i >> 1] >> 16 : wd[i >> 1] & 0xffffu);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (tid == 0 && !m.skip_mma) {
            fence_after();
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
                mma_tc(tmem + kTrColG, smem_desc(sbase + kTrSmAG + kk * 256, 128, 2048),
                       smem_desc(sbase + kTrSmBG + kk * 256, 128, 2048), idg, (g_started || kk > 0) ? 1 : 0);
            mma_commit(bar3);
        }
        g_started = true;
        if (bad) s_bad = 1;
    }
    __syncthreads();  // s_bad is settled for every thread
    // db2 and the loss: per-warp sums, then one atomic per warp into shared memory
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        db2w += __shfl_xor_sync(0xffffffffu, db2w, o);
        db2c += __shfl_xor_sync(0xffffffffu, db2c, o);
        loss += __shfl_xor_sync(0xffffffffu, loss, o);
    }
    if (lane == 0) {
        atomicAdd(&s_acc[0], db2w);
        atomicAdd(&s_acc[1], db2c);
        atomicAdd(&s_acc[2], loss);
    }
    // the accumulated weight gradients: row tid of G
    if (g_started && !s_bad) {
        bad |= !mbar_wait(bar3, ph3);
        ph3 ^= 1u;
        fence_after();
        unsigned gv[32];
        tmem_ld32_nowait(tmem + kTrColG + lane_base, gv);
        tmem_wait_ld();
        if (!bad) {
            if (tid < 64) {
                atomicAdd(m.grad + kMlpW2 + tid, __uint_as_float(gv[0]));
                atomicAdd(m.grad + kMlpW2 + kH + tid, __uint_as_float(gv[1]));
            } else {
                const int j = tid - 64;
#pragma unroll
                for (int i = 0; i < kF; ++i) atomicAdd(m.grad + j * kF + i, __uint_as_float(gv[2 + i]));
                atomicAdd(m.grad + kMlpB1 + j, __uint_as_float(gv[18]));
            }
        }
    }
    __syncthreads();
    if (tid == 0 && !s_bad && !bad) {
        atomicAdd(m.grad + kMlpB2, s_acc[0]);
        atomicAdd(m.grad + kMlpB2 + 1, s_acc[1]);
        atomicAdd(m.grad + kMlpParams, s_acc[2]);
    }
    if (bad) atomicOr(err, 1);
    // after a time-out the tensor cores may still be busy: one more bounded wait on each barrier
    if (s_bad && tid == 0) {
        mbar_wait(bar1, ph1);
        mbar_wait(bar2, ph2);
        if (g_started) mbar_wait(bar3, ph3);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTrTmemCols) : "memory");
    }
}

}  // namespace

cudaError_t launch_mlp_infer_tc(const MlpArgs &m, int *err, cudaStream_t s) {
    if (m.n_px <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    // more than the default 48 KB of dynamic shared memory (a per-device attribute; cheap to repeat)
    e = cudaFuncSetAttribute(mlp_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmRequest);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long pairs = (m.n_px + 1) / 2;
    long long blocks = (long long)sms * kTcCtasPerSm;
    if (blocks > pairs) blocks = pairs;
    static_assert(kSmBytes <= kSmRequest, "operands exceed the requested shared memory");
    mlp_infer_tc_kernel<<<(unsigned)blocks, kTcThreads, kSmRequest, s>>>(m, err);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train_tc(const MlpArgs &m, int *err, cudaStream_t s) {
    if (m.n_batch <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrSmBytes);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long pairs = (m.n_batch + 1) / 2;
    long long blocks = (long long)sms * 3;
    if (blocks > pairs) blocks = pairs;
    mlp_train_tc_kernel<<<(unsigned)blocks, kTcThreads, kTrSmBytes, s>>>(m, err);
    return cudaGetLastError();
}

}  // namespace ssvp
