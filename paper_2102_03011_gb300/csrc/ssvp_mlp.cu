// ssvp_mlp.cu - the learned per-sample weighting's support kernels: Adam on the FP32 master
// weights with their BF16 copies, and the expansion of compact capped sample sets into the full
// 64 x 16 BF16 feature layout for callers that read them (ssvp_learned_samples).  Inference and
// training run on the tcgen05 tensor cores (ssvp_mlp_tc.cu).
#include <cuda_bf16.h>

#include "ssvp_internal.h"

namespace ssvp {
namespace {

constexpr int kS = 64, kF = 16;

// keep the kernels' copies of the master weights: W1 as BF16, W2 rounded to BF16 values
__device__ __forceinline__ void refresh_one(const MlpState &st, int i, float p) {
    if (i < kMlpB1) {
        __nv_bfloat16 b = __float2bfloat16_rn(p);
        st.W1_bf16[i] = *reinterpret_cast<unsigned short *>(&b);
    } else if (i >= kMlpW2 && i < kMlpB2) {
        st.W2_r[i - kMlpW2] = __bfloat162float(__float2bfloat16_rn(p));
    }
}

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
