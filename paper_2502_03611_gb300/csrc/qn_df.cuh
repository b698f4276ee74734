// Exact fixed-point and float-pair (unevaluated hi + lo FP32 sums) helpers shared by the
// FP64-free kernels (the split solve's residual, the eigen solve's residual passes): GB300
// issues FP64 at about 2 operations per clock per SM, so these kernels keep FP64 off the
// per-node path.
#pragma once

#include <cuda_runtime.h>

#include "qn_numeric.cuh"

namespace qn {

constexpr int kFxG = 5;   // guard bits below the ulp of the fixed-point exponent E

static __device__ __noinline__ void flag_fbad(int *flag) {
    if (flag != nullptr) atomicOr(flag, 1);
}

static __device__ __noinline__ float2 f_pair_slow(double fv) {
    const float fh = __double2float_rn(fv);
    return make_float2(fh, __double2float_rn(fv - (double)fh));
}

// hi = f rounded to FP32, lo = (f - hi) rounded to FP32. The difference is
// taken exactly on the integer significands (|f| - |hi| has at most 29
// significant bits), so no FP64 operation is spent; tiny, huge and
// non-finite f take the FP64 route.
__device__ __forceinline__ float2 f_pair(double fv, int *flag) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fv);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex >= 1023 + 100) flag_fbad(flag);
    if (ex < 1075 - 126 || ex >= 1023 + 100) return f_pair_slow(fv);
    const float fh = d2f_rn(fv);
    const unsigned int fb = __float_as_uint(fh);
    const int ef = (int)((fb >> 23) & 0xFFu);
    const long long hu = (long long)((fb & 0x7FFFFFu) | 0x800000u) << (ef - ex + 925);   // 29, or 30 after a carry
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    float lo = __fmul_rn(__int2float_rn((int)(m - hu)), __int_as_float((ex - 1075 + 127) << 23));
    if (b >> 63) lo = -lo;
    return make_float2(fh, lo);
}

// Signed fixed-point value of the double with bit pattern b, in units of
// 2^(E - 1075 - kFxG); `bad` is set when its exponent exceeds E (the value
// returned is then 0 and must not be used). Every usable exponent E is >= 64,
// so zeros and subnormals (biased exponent 0) shift out entirely; the PTX
// shift clamps amounts of 64 or more to 64 (result 0), which needs no clamp here.
__device__ __forceinline__ long long fx_of(unsigned long long b, int E, unsigned &bad) {
    const unsigned int bh = (unsigned int)(b >> 32);
    const int ex = (int)((bh >> 20) & 0x7FFu);
    bad |= (unsigned)(ex > E);
    const unsigned int sh = (unsigned int)(E - ex);
    const unsigned long long m = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << kFxG;
    unsigned long long v;
    asm("shr.b64 %0, %1, %2;" : "=l"(v) : "l"(m), "r"(sh));
    const unsigned long long sg = (unsigned long long)((long long)b >> 63);   // 0 or all ones
    return (long long)((v ^ sg) - sg);
}

// Exact int -> float for |c| < 2^22 (the FP32 add of 1.5 * 2^23 trick, read backwards).
__device__ __forceinline__ float small_i2f(int c) {
    return __fsub_rn(__int_as_float(0x4B400000 + c), 12582912.0f);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Fixed-point value v (|v| < 2^62) times the power of two `scale`, as a float pair.
__device__ __forceinline__ void fx_to_pair(long long v, float scale, float &hi, float &lo) {
    const int c2 = (int)(v >> 42);                                   // signed, |c2| <= 2^20
    const int c1 = (int)((unsigned long long)v >> 21) & 0x1FFFFF;
    const int c0 = (int)v & 0x1FFFFF;
    const float f2 = __fmaf_rn(__int_as_float(0x4B400000 + c2), 0x1p42f, -0x1.8p65f);   // c2 * 2^42, exact
    const float f1 = __fmaf_rn(__int_as_float(0x4B400000 + c1), 0x1p21f, -0x1.8p44f);   // c1 * 2^21, exact
    const float f0 = small_i2f(c0);
    float s, e;
    two_sum(f2, f1, s, e);
    hi = __fmul_rn(s, scale);
    lo = __fmul_rn(__fadd_rn(e, f0), scale);
}

// Two-lane forms of the helpers above on the packed FP32x2 instructions of sm_100+
// (one FFMA2 / FADD2 / FMUL2 does the operation for two values, with the rounding
// of the scalar instruction, so the results equal the scalar ones bit for bit).
__device__ __forceinline__ float2 f2_splat(float v) { return make_float2(v, v); }

// a - b as one rounded FMA (b * -1 + a).
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2_splat(-1.0f), a); }

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = __fadd2_rn(a, b);
    const float2 bb = sub2(s, a);
    e = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// fx_to_pair for two fixed-point values.
__device__ __forceinline__ void fx_to_pair2(long long v0, long long v1, float scale, float2 &hi, float2 &lo) {
    const int a2 = (int)(v0 >> 42), b2 = (int)(v1 >> 42);
    const int a1 = (int)((unsigned long long)v0 >> 21) & 0x1FFFFF, b1 = (int)((unsigned long long)v1 >> 21) & 0x1FFFFF;
    const int a0 = (int)v0 & 0x1FFFFF, b0 = (int)v1 & 0x1FFFFF;
    const float2 f2 = __ffma2_rn(make_float2(__int_as_float(0x4B400000 + a2), __int_as_float(0x4B400000 + b2)),
                                 f2_splat(0x1p42f), f2_splat(-0x1.8p65f));
    const float2 f1 = __ffma2_rn(make_float2(__int_as_float(0x4B400000 + a1), __int_as_float(0x4B400000 + b1)),
                                 f2_splat(0x1p21f), f2_splat(-0x1.8p44f));
    const float2 f0 = __fadd2_rn(make_float2(__int_as_float(0x4B400000 + a0), __int_as_float(0x4B400000 + b0)),
                                 f2_splat(-12582912.0f));
    float2 s, e;
    two_sum2(f2, f1, s, e);
    hi = __fmul2_rn(s, f2_splat(scale));
    lo = __fmul2_rn(__fadd2_rn(e, f0), f2_splat(scale));
}

// (a + b) for two float pairs, renormalised.
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    const float hi = __fadd_rn(s, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

// a * b for float pairs, renormalised.
__device__ __forceinline__ float2 pair_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float hi = __fadd_rn(p, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, p)));
}

__device__ __forceinline__ float2 pair_neg(float2 a) { return make_float2(-a.x, -a.y); }

}  // namespace qn
