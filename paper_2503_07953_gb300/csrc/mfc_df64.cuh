// Double-float arithmetic: a real number carried as the unevaluated sum of
// two float32 values, hi + lo with |lo| <= ulp(hi)/2 (a 48-bit significand
// with float32's exponent range).  Every operation runs on the float32
// pipes, which on GB300 execute 64 times more operations per clock than the
// float64 pipe.
//
// The building blocks are the error-free transformations of Dekker (1971)
// and Knuth (TAOCP vol. 2): the rounding error of a float32 sum is
// recovered exactly by TwoSum, that of a product by one fused multiply-add.
// Addition is the "sloppy" double-float sum (error bounded by a small
// multiple of 2^-48 (|a| + |b|), as for a rounded float64 sum of inputs
// that carry their own rounding); multiplication, division and square root
// are accurate to a few units of 2^-48 relative.  All steps use the
// explicitly rounded intrinsics so the compiler neither contracts nor
// reassociates them, whatever the translation unit's FMA setting.
#pragma once

#include <cuda_runtime.h>

namespace mfc {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // nearest double-float to a float64 value: hi is x rounded to float32,
    // lo the rounded remainder (x - hi is exact in float64)
    __host__ __device__ explicit constexpr df64(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e as a normalised pair when |s| >= |e| (Dekker's Fast2Sum)
__device__ __forceinline__ df64 df_fast2sum(float s, float e) {
    const float h = __fadd_rn(s, e);
    return df64(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    // TwoSum of the leading parts, then the trailing parts folded into the error
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_fast2sum(s, e);
}

__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // exact rounding error of a.hi b.hi
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast2sum(p, e);
}

// a times a float32 value b
__device__ __forceinline__ df64 df_mulf(df64 a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return df_fast2sum(p, e);
}

// a times a power of two (exact barring overflow and underflow)
__device__ __forceinline__ df64 df_scale(df64 a, float two_pow) {
    return df64(__fmul_rn(a.hi, two_pow), __fmul_rn(a.lo, two_pow));
}

// float32 reciprocal: the hardware approximation (1 ulp) refined by one
// Newton step, r <- r + r (1 - b r)
__device__ __forceinline__ float rcp_f32(float b) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(b));
    const float e = __fmaf_rn(-b, r, 1.0f);
    return __fmaf_rn(r, e, r);
}

// a / b: a float32 quotient q1 = a.hi / b.hi, the remainder a - q1 b in
// double-float (its leading part is exact by Sterbenz's lemma), and the
// correction q2 = remainder / b.hi.
__device__ __forceinline__ df64 df_div(df64 a, df64 b) {
    const float r = rcp_f32(b.hi);
    const float q1 = __fmul_rn(a.hi, r);
    const float p = __fmul_rn(q1, b.hi);
    const float pe = __fmaf_rn(q1, b.hi, -p);
    float rem = __fsub_rn(a.hi, p);
    rem = __fsub_rn(rem, pe);
    rem = __fadd_rn(rem, a.lo);
    rem = __fmaf_rn(-q1, b.lo, rem);
    return df_fast2sum(q1, __fmul_rn(rem, r));
}

__device__ __forceinline__ df64 operator/(df64 a, df64 b) { return df_div(a, b); }

// sqrt(a): y = a.hi x with x a refined 1/sqrt(a.hi), then one Newton
// correction y + (a - y^2) / (2 y) with the residual in double-float.
__device__ __forceinline__ df64 df_sqrt(df64 a) {
    if (!(a.hi > 0.0f)) return df64(sqrtf(a.hi), 0.0f);  // 0 -> 0, negative or NaN -> NaN
    float x;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(x) : "f"(a.hi));
    // x <- x (3 - a x^2) / 2
    x = __fmul_rn(x, __fmaf_rn(__fmul_rn(-0.5f, a.hi), __fmul_rn(x, x), 1.5f));
    const float y = __fmul_rn(a.hi, x);
    const float p = __fmul_rn(y, y);
    const float pe = __fmaf_rn(y, y, -p);
    float rem = __fsub_rn(a.hi, p);
    rem = __fsub_rn(rem, pe);
    rem = __fadd_rn(rem, a.lo);
    return df_fast2sum(y, __fmul_rn(rem, __fmul_rn(0.5f, x)));
}

__device__ __forceinline__ df64 df_abs(df64 a) { return a.hi < 0.0f ? -a : a; }

// Conversions between float64 and double-float by integer operations on
// the bit patterns.  On GB300 the float32 <-> float64 conversion
// instructions run on the float64 pipe, the scarcest unit here; these run
// on the integer pipe (and one int -> float32 conversion).

// Nearest double-float of x: the leading part is x rounded to 24
// significant bits (a carry out of the mantissa moves into the exponent),
// the trailing part the signed remainder, at most half an ulp of the
// leading part, rounded to float32.  Exact to 2^-48 relative for
// 2^-74 <= |x| < 2^128; smaller magnitudes keep only their leading part
// (zero below 2^-126), larger ones become infinite, NaN stays NaN.
__device__ __forceinline__ df64 df_from_f64_bits(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned s = hi & 0x80000000u;
    const unsigned e = (hi >> 20) & 0x7ffu;  // biased float64 exponent
    const unsigned up = (lo >> 28) & 1u;     // the first dropped bit rounds the leading part
    unsigned h = (((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29)) + up;
    const int rem = (int)(lo & 0x1fffffffu) - (int)(up << 29);  // remainder in units of 2^(e - 1075)
    float t = (float)rem * __uint_as_float((e - 948u) << 23);
    if (e < 949u || e > 1150u) t = 0.0f;
    if (e < 897u) h = 0u;
    if (e > 1150u) h = (e == 2047u && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u;
    return df64(__uint_as_float(s | h), __uint_as_float(__float_as_uint(t) ^ s));
}

// A float32 value as float64 (exact for normal numbers; subnormals become
// zero, infinities and NaN keep their class).
__device__ __forceinline__ double f64_from_f32_bits(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned m = (e == 0u) ? 0u : (b & 0x7fffffu);
    const unsigned de = (e == 0u) ? 0u : ((e == 0xffu) ? 0x7ffu : e + 896u);
    return __hiloint2double((int)((b & 0x80000000u) | (de << 20) | (m >> 3)), (int)(m << 29));
}

// Two double-float numbers side by side, in the x and y lanes of float2
// leading and trailing parts.  Every step of the operations below is one
// paired float32 instruction for both numbers (FADD2, FMUL2, FFMA2 on
// sm_100 and later), with the same rounding as the scalar operations above
// lane by lane: for two computations that perform the same operations on
// different values, such as the right- and left-edge weights of WENO5.
struct df64x2 {
    float2 hi, lo;
};

__device__ __forceinline__ df64x2 dfx2(df64 x, df64 y) {
    return {make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)};
}
__device__ __forceinline__ df64x2 dfx2(double x, double y) { return dfx2(df64(x), df64(y)); }
__device__ __forceinline__ df64 lane_x(df64x2 a) { return df64(a.hi.x, a.lo.x); }
__device__ __forceinline__ df64 lane_y(df64x2 a) { return df64(a.hi.y, a.lo.y); }

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }

__device__ __forceinline__ df64x2 df_fast2sum(float2 s, float2 e) {
    const float2 h = __fadd2_rn(s, e);
    return {h, sub2(e, sub2(h, s))};
}

__device__ __forceinline__ df64x2 operator+(df64x2 a, df64x2 b) {
    const float2 s = __fadd2_rn(a.hi, b.hi);
    const float2 v = sub2(s, a.hi);
    float2 e = __fadd2_rn(sub2(a.hi, sub2(s, v)), sub2(b.hi, v));
    e = __fadd2_rn(e, __fadd2_rn(a.lo, b.lo));
    return df_fast2sum(s, e);
}

__device__ __forceinline__ df64x2 operator-(df64x2 a) { return {neg2(a.hi), neg2(a.lo)}; }
__device__ __forceinline__ df64x2 operator-(df64x2 a, df64x2 b) { return a + (-b); }

__device__ __forceinline__ df64x2 operator*(df64x2 a, df64x2 b) {
    const float2 p = __fmul2_rn(a.hi, b.hi);
    float2 e = __ffma2_rn(a.hi, b.hi, neg2(p));
    e = __ffma2_rn(a.hi, b.lo, e);
    e = __ffma2_rn(a.lo, b.hi, e);
    return df_fast2sum(p, e);
}

// 1 / b lane by lane, as df_div(1, b)
__device__ __forceinline__ df64x2 df_rcp(df64x2 b) {
    float2 r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r.x) : "f"(b.hi.x));
    asm("rcp.approx.f32 %0, %1;" : "=f"(r.y) : "f"(b.hi.y));
    r = __ffma2_rn(r, __ffma2_rn(neg2(b.hi), r, make_float2(1.0f, 1.0f)), r);
    const float2 q1 = r;
    const float2 p = __fmul2_rn(q1, b.hi);
    const float2 pe = __ffma2_rn(q1, b.hi, neg2(p));
    float2 rem = sub2(make_float2(1.0f, 1.0f), p);
    rem = sub2(rem, pe);
    rem = __ffma2_rn(neg2(q1), b.lo, rem);
    return df_fast2sum(q1, __fmul2_rn(rem, r));
}

// Comparisons of normalised pairs: by the leading part, then the trailing part.
__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }

}  // namespace mfc
