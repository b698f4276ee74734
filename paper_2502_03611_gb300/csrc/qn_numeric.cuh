// Precision conversions done with integer instructions.
//
// On GB300 the FP64 pipe issues about 2 operations per clock per SM (1/64 of
// FP32), so in the memory-bound kernels every FP64-pipe instruction counts.
// These helpers convert between FP64 and FP32 by rearranging the IEEE-754 bit
// fields with integer operations, which run on the (64x wider) integer pipe.
// Both round exactly as the hardware conversions do (round to nearest even for
// the narrowing one; the widening one is exact); the rare special inputs
// (float-subnormal results, inf, nan) take the hardware conversion instead.
#pragma once

#include <stdint.h>

namespace qn {

// Rare-path helpers are kept out of line: inlined, the compiler turns them
// into predicated instructions that issue (on the FP64 pipe) at every call
// site even when the predicate is false.
static __device__ __noinline__ float d2f_slow(double d) { return __double2float_rn(d); }
static __device__ __noinline__ double f2d_slow(float f) { return (double)f; }

// double -> float, round to nearest even.
__device__ __forceinline__ float d2f_rn(double d) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    const unsigned int sign = (unsigned int)(bits >> 63) << 31;
    const int e = (int)((bits >> 52) & 0x7FF);
    const int ef = e - 1023 + 127;                    // float biased exponent
    if (e == 0) return __int_as_float((int)sign);     // zero (and double subnormals) -> signed zero
    if (ef <= 0 || ef >= 255) return d2f_slow(d);   // float subnormal, overflow, inf, nan
    const unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    const unsigned int mhi = (unsigned int)(m >> 29);             // top 23 mantissa bits
    const unsigned int mlo = (unsigned int)(m & 0x1FFFFFFFu);     // 29 dropped bits
    unsigned int fb = ((unsigned int)ef << 23) | mhi;
    const unsigned int half = 0x10000000u;
    if (mlo > half || (mlo == half && (mhi & 1u))) fb += 1u;      // carry may reach the exponent: correct
    return __int_as_float((int)(fb | sign));
}

// float -> double (exact).
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned int fb = (unsigned int)__float_as_int(f);
    const unsigned int ef = (fb >> 23) & 0xFFu;
    if (ef == 0u || ef == 255u) {
        if ((fb & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)((unsigned long long)(fb >> 31) << 63));
        return f2d_slow(f);                            // subnormal, inf, nan
    }
    const unsigned long long db = ((unsigned long long)(fb >> 31) << 63) |
                                  ((unsigned long long)(ef + 896u) << 52) |
                                  ((unsigned long long)(fb & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)db);
}

// |d| as an unsigned integer that orders like |d| (for min/max of |U| without FP64 ops).
__device__ __forceinline__ unsigned long long abs_bits(double d) {
    return (unsigned long long)__double_as_longlong(d) & 0x7FFFFFFFFFFFFFFFull;
}

}  // namespace qn

namespace qn {

// ---------------------------------------------------------------------------
// Exact fixed-point sum of a 5/7-point difference stencil on the integer pipe.
//
// lap = c0 * v0 - (v1 + ... + vK) for FP64 inputs: every value is aligned to
// the largest exponent E among them and held as an integer multiple of
// 2^(E - 1075 - G) (G = 5 guard bits; magnitudes < 2^58, so 12 of them
// cannot overflow int64); the weighted sum is then exact, and one rounding
// (to nearest even) turns it back into a double. The only error is the
// truncation of each aligned input below 2^(E - 1075 - G), i.e. at most
// 2^-57 of the largest input - below the rounding error of summing the
// stencil in FP64, and without spending FP64-pipe instructions.
// Non-finite inputs return NaN-propagating FP64 arithmetic instead.
// ---------------------------------------------------------------------------
struct Unpacked {
    unsigned long long m;   // 53-bit significand (hidden bit included for normal numbers)
    int e;                  // biased exponent, subnormals and zero as 1
    int neg;
};

__device__ __forceinline__ Unpacked unpack_d(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    Unpacked u;
    u.neg = (int)(b >> 63);
    const int ex = (int)((b >> 52) & 0x7FF);
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    u.m = ex ? (mant | (1ull << 52)) : mant;
    u.e = ex ? ex : 1;
    return u;
}

constexpr int kGuard = 5;

static __device__ __noinline__ double fixed_to_double_slow(long long acc, int E) {
    return ldexp((double)acc, E - 1075 - kGuard);
}

static __device__ __noinline__ double stencil_fp64(double c0, double u, double a, double b, double c,
                                                    double d, double e, double f) {
    return c0 * u - (((a + b) + (c + d)) + (e + f));
}

__device__ __forceinline__ long long aligned(const Unpacked &u, int E) {
    const int s = E - u.e;
    const long long v = (s >= 58) ? 0ll : (long long)((u.m << kGuard) >> s);
    return u.neg ? -v : v;
}

// Round an int64 multiple of 2^(E - 1075 - kGuard) to the nearest double.
__device__ __forceinline__ double fixed_to_double(long long acc, int E) {
    if (acc == 0) return 0.0;
    const unsigned long long sign = acc < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = acc < 0 ? (unsigned long long)(-acc) : (unsigned long long)acc;
    const int lz = __clzll((long long)a);
    const unsigned long long norm = a << lz;           // leading one at bit 63
    unsigned long long mant = norm >> 11;              // 53 bits
    const unsigned long long rem = norm & 0x7FFull;
    int be = E + 11 - kGuard - lz;                     // biased exponent of the result
    if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
        mant += 1ull;
        if (mant >> 53) {
            mant >>= 1;
            be += 1;
        }
    }
    if (be <= 0 || be >= 2047) return fixed_to_double_slow(acc, E);   // outside the normal range
    return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// 2*DIM*u - sum(nb[0..2*DIM-1]), exactly summed, one final rounding.
template <int DIM>
__device__ __forceinline__ double stencil_fixed(double u, const double (&nb)[2 * DIM]) {
    const Unpacked c = unpack_d(u);
    Unpacked q[2 * DIM];
    int E = c.e;
#pragma unroll
    for (int i = 0; i < 2 * DIM; ++i) {
        q[i] = unpack_d(nb[i]);
        E = q[i].e > E ? q[i].e : E;
    }
    if (E == 0x7FF)   // inf / nan: let FP64 arithmetic propagate it
        return stencil_fp64(2.0 * DIM, u, nb[0], nb[1], nb[2], nb[3], DIM == 3 ? nb[2 * DIM - 2] : 0.0,
                            DIM == 3 ? nb[2 * DIM - 1] : 0.0);
    const long long vc = aligned(c, E);
    long long acc = (DIM == 3) ? (vc << 2) + (vc << 1) : (vc << 2);
#pragma unroll
    for (int i = 0; i < 2 * DIM; ++i) acc -= aligned(q[i], E);
    return fixed_to_double(acc, E);
}

}  // namespace qn
