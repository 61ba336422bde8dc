// ssvp_pack.cu - load-time kernels: packing input frames into padded vector planes (A2) and the
// lower-median valid depth by a three-pass radix select (used for relative radii).
#include <cuda_fp16.h>

#include <mutex>

#include "../../include/ssvp.h"
#include "ssvp_df.cuh"
#include "ssvp_internal.h"

namespace ssvp {
namespace {

__device__ __forceinline__ bool valid_depth(float d) { return isfinite(d) && d > 0.0f; }

// One thread per input pixel of frames [0, nF): interleaved rgb (12 B) + depth -> padded planes
// (FP32: (r, g, b, depth) records; FP16: (r, g, b, 0) half records).
// Invalid depths become NaN so that a single comparison rejects them in the gather.
template <int CFMT>
__global__ void pack_kernel(const float *__restrict__ rgb, const float *__restrict__ depth, int W, int H,
                            long long npix, Planes P, int frame0) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix;
         i += (long long)gridDim.x * blockDim.x) {
        long long f = i / ((long long)W * H);
        int rem = (int)(i - f * (long long)W * H);
        int y = rem / W, x = rem - y * W;
        float d = depth[i];
        float r = rgb[3 * i], g = rgb[3 * i + 1], b = rgb[3 * i + 2];
        long long o = (f + frame0) * P.fstride + (long long)(y + kPad) * P.pitch + (x + kPad);
        const float dv = valid_depth(d) ? d : __int_as_float(0x7fffffff);
        P.depth[o] = dv;
        if (CFMT == 0) {
            // the fourth lane repeats the depth: the gather's filter loop reads both in one load
            reinterpret_cast<float4 *>(P.colour)[o] = make_float4(r, g, b, dv);
        } else {
            __half2 rg = __floats2half2_rn(r, g);
            __half2 b0 = __floats2half2_rn(b, 0.0f);
            uint2 raw;
            raw.x = *reinterpret_cast<unsigned int *>(&rg);
            raw.y = *reinterpret_cast<unsigned int *>(&b0);
            reinterpret_cast<uint2 *>(P.colour)[o] = raw;
        }
    }
}

// ---------------------------------------------------------------- radix select
// Positive finite floats order like their bit patterns.  Three passes over 11, 11 and 10 bits
// narrow the bit pattern of the element of rank floor((n - 1) / 2).
// scratch layout (32-bit words): [0, 2048) histogram, 2048 prefix, 2049 rank, 2050 n_valid.
constexpr int kHistWords = 2048;
__host__ __device__ constexpr int shift_of(int pass) { return pass == 0 ? 21 : (pass == 1 ? 10 : 0); }
__host__ __device__ constexpr int bins_of(int pass) { return pass == 2 ? 1024 : 2048; }

template <int PASS>
__global__ void hist_kernel(const float *__restrict__ depth, long long n, unsigned int *scratch) {
    __shared__ unsigned int h[kHistWords];
    for (int i = threadIdx.x; i < bins_of(PASS); i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned int prefix = PASS == 0 ? 0u : scratch[2048];
    const unsigned int *bits = reinterpret_cast<const unsigned int *>(depth);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned int b = __ldg(bits + i);
        bool ok = b > 0u && b < 0x7f800000u;
        if (PASS == 1) ok = ok && (b >> 21) == prefix;
        if (PASS == 2) ok = ok && (b >> 10) == prefix;
        if (ok) atomicAdd(&h[(b >> shift_of(PASS)) & (bins_of(PASS) - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < bins_of(PASS); i += blockDim.x)
        if (h[i]) atomicAdd(&scratch[i], h[i]);
}

// One block of 1024 threads: find the bin holding the wanted rank, fold it into the prefix,
// clear the histogram for the next pass; the last pass writes the median.
template <int PASS>
__global__ void select_kernel(unsigned int *scratch, float *median) {
    __shared__ unsigned int part[1024];
    const int t = threadIdx.x;
    const int per = bins_of(PASS) / 1024;  // 2 or 1 bins per thread
    unsigned int local = 0;
    for (int i = 0; i < per; ++i) local += scratch[t * per + i];
    part[t] = local;
    __syncthreads();
    // inclusive scan (Hillis-Steele)
    for (int off = 1; off < 1024; off <<= 1) {
        unsigned int v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    const unsigned int total = part[1023];
    unsigned int rank;
    if (PASS == 0) {
        rank = total ? (total - 1) / 2 : 0u;
    } else {
        rank = scratch[2049];
    }
    __syncthreads();
    unsigned int before = t ? part[t - 1] : 0u;
    if (total > 0 && rank >= before && rank < part[t]) {
        unsigned int r = rank - before;
        int bin = t * per;
        for (int i = 0; i < per; ++i) {
            unsigned int c = scratch[t * per + i];
            if (r < c) { bin = t * per + i; break; }
            r -= c;
        }
        unsigned int prefix = PASS == 0 ? (unsigned int)bin : ((scratch[2048] << (PASS == 1 ? 11 : 10)) | (unsigned int)bin);
        scratch[2048] = prefix;
        scratch[2049] = r;
        if (PASS == 2) *median = __uint_as_float(prefix);
    }
    if (PASS == 0) {
        if (t == 0) scratch[2050] = total;
        if (total == 0 && t == 0) *median = __int_as_float(0x7fffffff);
    }
    __syncthreads();
    for (int i = t; i < kHistWords; i += 1024) scratch[i] = 0;
}

// ---------------------------------------------------------------- Eq. 5 blurriness measure
// Per frame, the sum over pixels with a right and a lower neighbour of the forward-difference
// gradient magnitude (L2 over the colour channels and both axes).  Two deterministic passes:
// kGradSlices blocks per frame write FP64 partial sums, then one block adds them in order and
// derives log2(sum / max over frames), the per-frame term of the Eq. 5 weight in log2 units.
constexpr int kGradSlices = 64;

template <int CFMT>
__global__ void __launch_bounds__(256) grad_partial_kernel(Planes P, double *partial) {
    const int f = blockIdx.y;
    float sum = 0.0f;
    for (int y = blockIdx.x; y + 1 < P.H; y += kGradSlices) {
        const long long row = (long long)f * P.fstride + (long long)(y + kPad) * P.pitch + kPad;
        for (int x = threadIdx.x; x + 1 < P.W; x += blockDim.x) {
            const float3 a = load_colour<CFMT>(P.colour, row + x);
            const float3 r = load_colour<CFMT>(P.colour, row + x + 1);
            const float3 d = load_colour<CFMT>(P.colour, row + P.pitch + x);
            const float gx0 = r.x - a.x, gx1 = r.y - a.y, gx2 = r.z - a.z;
            const float gy0 = d.x - a.x, gy1 = d.y - a.y, gy2 = d.z - a.z;
            sum += sqrtf(gx0 * gx0 + gx1 * gx1 + gx2 * gx2 + gy0 * gy0 + gy1 * gy1 + gy2 * gy2);
        }
    }
    double v = sum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double s_part[8];
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += s_part[i];
        partial[(long long)f * kGradSlices + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256) grad_final_kernel(int F, const double *partial, double *sum, float *log2w) {
    __shared__ double s_max[256];
    double mx = 0.0;
    for (int f = threadIdx.x; f < F; f += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < kGradSlices; ++b) t += partial[(long long)f * kGradSlices + b];
        sum[f] = t;
        mx = fmax(mx, t);
    }
    s_max[threadIdx.x] = mx;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
        __syncthreads();
    }
    const double gmax = s_max[0];
    for (int f = threadIdx.x; f < F; f += blockDim.x) {
        // a frame without any gradient gets weight 0 (log2 = -inf); an all-flat clip weights all
        // frames equally
        log2w[f] = gmax > 0.0 ? (float)log2(sum[f] / gmax) : 0.0f;
    }
}

}  // namespace

cudaError_t launch_grad_sum(const Planes &p, cudaStream_t s) {
    const dim3 grid(kGradSlices, (unsigned)p.F);
    if (p.colour_fmt == 0) grad_partial_kernel<0><<<grid, 256, 0, s>>>(p, p.grad_partial);
    else grad_partial_kernel<1><<<grid, 256, 0, s>>>(p, p.grad_partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    grad_final_kernel<<<1, 256, 0, s>>>(p.F, p.grad_partial, p.grad_sum, p.grad_log2);
    return cudaGetLastError();
}

size_t grad_partial_words(int F) { return (size_t)F * kGradSlices; }

cudaError_t launch_pack(const float *rgb, const float *depth, int W, int H, int nF, const Planes &dst, int frame0,
                        cudaStream_t s) {
    long long n = (long long)W * H * nF;
    if (n == 0) return cudaSuccess;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (dst.colour_fmt == 0) pack_kernel<0><<<blocks, 256, 0, s>>>(rgb, depth, W, H, n, dst, frame0);
    else pack_kernel<1><<<blocks, 256, 0, s>>>(rgb, depth, W, H, n, dst, frame0);
    return cudaGetLastError();
}

size_t median_scratch_words() { return kHistWords + 4; }

cudaError_t launch_median(const Planes &p, unsigned int *scratch, cudaStream_t s) {
    long long n = (long long)p.F * p.fstride;
    int blocks = 152 * 4;
    cudaError_t e = cudaMemsetAsync(scratch, 0, median_scratch_words() * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    hist_kernel<0><<<blocks, 512, 0, s>>>(p.depth, n, scratch);
    select_kernel<0><<<1, 1024, 0, s>>>(scratch, p.median);
    hist_kernel<1><<<blocks, 512, 0, s>>>(p.depth, n, scratch);
    select_kernel<1><<<1, 1024, 0, s>>>(scratch, p.median);
    hist_kernel<2><<<blocks, 512, 0, s>>>(p.depth, n, scratch);
    select_kernel<2><<<1, 1024, 0, s>>>(scratch, p.median);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- median without allocation
// Scratch of ssvp_median_depth_noalloc: the radix-select histogram and its prefix/rank/count
// words live in this fixed device array instead of memory from cudaMalloc.  Every GPU that
// loads the library holds these 8,208 bytes until the process exits.
static __device__ __align__(256) unsigned int g_median_scratch[kHistWords + 4];

namespace {

// Device address of g_median_scratch, looked up once per device.  In host code the symbol's
// name is only a host-side stand-in; a kernel must be given this address instead.  The cached
// address belongs to the device's current context: the library must not be used across a
// cudaDeviceReset of that device (the module, and with it the array, is then loaded anew).
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned int *g_scratch_ptr[kMaxDevices] = {};

cudaError_t median_scratch_for_current_device(unsigned int **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_median_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned int *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace ssvp

extern "C" int ssvp_median_depth_noalloc(const float *depth_dev, unsigned long long n, float *median_dev,
                                         void *cuda_stream) {
    if (!depth_dev || !median_dev) {
        ssvp::set_global_error("ssvp_median_depth_noalloc: depth_dev and median_dev must not be NULL");
        return SSVP_EINVAL;
    }
    if (n == 0 || n > ssvp::kMedianNoallocMax) {
        ssvp::set_global_error("ssvp_median_depth_noalloc: n=%llu outside [1, %llu]: the fixed scratch counts "
                               "values in 32-bit words", n, (unsigned long long)ssvp::kMedianNoallocMax);
        return SSVP_EINVAL;
    }
    // both pointers must be memory the current device can read and write: a host address would
    // fault inside the kernels, so it is refused here
    for (int i = 0; i < 2; ++i) {
        const void *ptr = i == 0 ? (const void *)depth_dev : (const void *)median_dev;
        cudaPointerAttributes at{};
        const cudaError_t pe = cudaPointerGetAttributes(&at, ptr);
        if (pe != cudaSuccess || (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            ssvp::set_global_error("ssvp_median_depth_noalloc: %s is not device or managed memory",
                                   i == 0 ? "depth_dev" : "median_dev");
            return SSVP_EINVAL;
        }
    }
    unsigned int *scratch = nullptr;
    cudaError_t e = ssvp::median_scratch_for_current_device(&scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ssvp::set_global_error("ssvp_median_depth_noalloc: scratch address: %s", cudaGetErrorString(e));
        return SSVP_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long nn = (long long)n;
    const int blocks = 152 * 4;
    // the previous call's histogram stays in the array: clear it first
    e = cudaMemsetAsync(scratch, 0, ssvp::median_scratch_words() * sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        ssvp::hist_kernel<0><<<blocks, 512, 0, s>>>(depth_dev, nn, scratch);
        ssvp::select_kernel<0><<<1, 1024, 0, s>>>(scratch, median_dev);
        ssvp::hist_kernel<1><<<blocks, 512, 0, s>>>(depth_dev, nn, scratch);
        ssvp::select_kernel<1><<<1, 1024, 0, s>>>(scratch, median_dev);
        ssvp::hist_kernel<2><<<blocks, 512, 0, s>>>(depth_dev, nn, scratch);
        ssvp::select_kernel<2><<<1, 1024, 0, s>>>(scratch, median_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        ssvp::set_global_error("ssvp_median_depth_noalloc: %s", cudaGetErrorString(e));
        return SSVP_ECUDA;
    }
    return SSVP_OK;
}
