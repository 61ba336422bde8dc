// ssvp_df.cuh - device helpers shared by the gather kernels: double-float (unevaluated FP32 pair)
// arithmetic built from error-free transformations, fast reciprocal and exp2, colour loads.
#pragma once

#include <cuda_fp16.h>

#include "ssvp_internal.h"

namespace ssvp {
namespace {

// The _rn intrinsics are never contracted into FMAs, which keeps the error-free transforms exact.
struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}

// a / b given r ~ 1 / b.hi (relative error ~1e-7): the correction step makes the quotient
// accurate to ~1e-14 relative.
__device__ __forceinline__ df df_div(df a, df b, float r) {
    float q1 = __fmul_rn(a.hi, r);
    df p = two_prod(q1, b.hi);
    float rem = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), __fsub_rn(a.lo, __fmul_rn(q1, b.lo)));
    return fast_two_sum(q1, __fmul_rn(rem, r));
}

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// exact float of a small non-negative integer (< 2^23) without a conversion instruction
__device__ __forceinline__ float small_float(int v) { return __int_as_float(0x4b000000 | v) - 8388608.0f; }

template <int CFMT, typename I>
__device__ __forceinline__ float3 load_colour(const void *base, I idx) {
    if (CFMT == 0) {
        float4 c = __ldg(reinterpret_cast<const float4 *>(base) + idx);
        return make_float3(c.x, c.y, c.z);
    } else {
        uint2 raw = __ldg(reinterpret_cast<const uint2 *>(base) + idx);
        __half2 rg = *reinterpret_cast<__half2 *>(&raw.x);
        __half2 b0 = *reinterpret_cast<__half2 *>(&raw.y);
        float2 f = __half22float2(rg);
        return make_float3(f.x, f.y, __low2float(b0));
    }
}

// Depth and colour of one window sample.  The FP32 colour record carries the depth in its fourth
// lane (the same value as the depth plane), so one 16-byte load brings both; the FP16 record has
// no room for it and the depth comes from the depth plane.
template <int CFMT, typename I>
__device__ __forceinline__ void load_sample(const float *dwin, const void *cwin, I idx, float &d, float3 &c) {
    if (CFMT == 0) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(cwin) + idx);
        d = v.w;
        c = make_float3(v.x, v.y, v.z);
    } else {
        d = __ldg(dwin + idx);
        c = load_colour<1>(cwin, idx);
    }
}

// Packed FP32x2 arithmetic (sm_100 family): two IEEE single-precision operations, rounded to
// nearest each, in one instruction; the halves are exactly the scalar results.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 r, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 f2_abs(f32x2 a) { return a & 0x7fffffff7fffffffull; }

constexpr float kLog2e = 1.4426950408889634f;
constexpr int kSlotVec = 6;  // float4 words of per-slot geometry in shared memory

// Shared per-slot geometry (6 x float4):
//  q0 = mb_hi0 mb_hi1 mb_hi2 mb_lo0   (mb = M (u0, v0, 1) of the CTA's first pixel, double-float)
//  q1 = mb_lo1 mb_lo2 M00 M01
//  q2 = M10 M11 M20 M21
//  q3 = e_hi0 e_hi1 e_hi2 e_lo0
//  q4 = e_lo1 e_lo2 ifx ify
//  q5 = cx cy beta*log2e J(bits)
__device__ void build_slot(const PairGeom &g, float u0, float v0, float4 *dst) {
    df mb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        df t = df_mul_f({g.M_hi[3 * r], g.M_lo[3 * r]}, u0);
        t = df_add(t, df_mul_f({g.M_hi[3 * r + 1], g.M_lo[3 * r + 1]}, v0));
        mb[r] = df_add(t, {g.M_hi[3 * r + 2], g.M_lo[3 * r + 2]});
    }
    dst[0] = make_float4(mb[0].hi, mb[1].hi, mb[2].hi, mb[0].lo);
    dst[1] = make_float4(mb[1].lo, mb[2].lo, g.M_hi[0], g.M_hi[1]);
    dst[2] = make_float4(g.M_hi[3], g.M_hi[4], g.M_hi[6], g.M_hi[7]);
    dst[3] = make_float4(g.e_hi[0], g.e_hi[1], g.e_hi[2], g.e_lo[0]);
    dst[4] = make_float4(g.e_lo[1], g.e_lo[2], g.ifx, g.ify);
    dst[5] = make_float4(g.cx, g.cy, g.beta * kLog2e, __int_as_float(g.J));
}

}  // namespace
}  // namespace ssvp
