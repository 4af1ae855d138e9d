// Arithmetic policies of the FP64 operator kernels.
//
// F64    native double precision (the FP64 pipe: 2 FMA/clk/SM on GB300).
// TF64   triple-float, at least FP64-wide (below).
// DF64   "double-float": a value is an unevaluated sum hi + lo of two floats
//        (48-bit significand), evaluated on the FP32 pipe, which is 61x
//        faster than the FP64 pipe on GB300.  Products use the FMA-based
//        exact product (Dekker / Karp-Markstein), sums Knuth's two-sum;
//        dot products accumulate lazily: the running sum of the leading
//        products is kept error-free with two-sum, all rounding errors and
//        low-order cross terms collect in a float that is folded in once at
//        the end (in the spirit of Ogita, Rump & Oishi's Dot2).  Relative
//        accuracy about 2^-47 of the sum of |terms|, against 2^-53 for FP64.
//        All float operations use the _rn intrinsics, which the compiler never
//        contracts into FMAs, so the error-free transformations stay exact.
#pragma once
#include <cuda_runtime.h>

namespace dgns {

struct df64 {
  float hi, lo;
};

struct F32 {
  typedef float G;     // type in global memory
  typedef float V;
  typedef float Acc;
  static constexpr bool emulated = false;
  __device__ __forceinline__ static V from_double(double x) { return (float)x; }
  __device__ __forceinline__ static V load(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static double to_double(V x) { return x; }
  __host__ static V make(double x) { return (float)x; }
  __device__ __forceinline__ static void acc_zero(Acc& a) { a = 0.0f; }
  __device__ __forceinline__ static void acc_set(Acc& a, V x) { a = x; }
  __device__ __forceinline__ static void acc_fma(Acc& a, V c, V x) { a = fmaf(c, x, a); }
  __device__ __forceinline__ static void acc_first(Acc& a, V c, V x) { a = c * x; }
  __device__ __forceinline__ static V acc_get(const Acc& a) { return a; }
  __device__ __forceinline__ static V acc_get_norm(const Acc& a) { return a; }
  __device__ __forceinline__ static G store(V x) { return x; }
};

struct F64 {
  typedef double G;    // type in global memory
  typedef double V;    // value
  typedef double Acc;  // dot-product accumulator
  static constexpr bool emulated = false;
  __device__ __forceinline__ static V from_double(double x) { return x; }
  __device__ __forceinline__ static V load(const double* p) { return __ldg(p); }
  __device__ __forceinline__ static V split(double x) { return x; }
  __device__ __forceinline__ static double to_double(V x) { return x; }
  __host__ static V make(double x) { return x; }
  __device__ __forceinline__ static V zero() { return 0.0; }
  __device__ __forceinline__ static void acc_zero(Acc& a) { a = 0.0; }
  __device__ __forceinline__ static void acc_set(Acc& a, V x) { a = x; }
  __device__ __forceinline__ static void acc_fma(Acc& a, V c, V x) { a = fma(c, x, a); }
  __device__ __forceinline__ static void acc_first(Acc& a, V c, V x) { a = c * x; }
  __device__ __forceinline__ static V acc_get(const Acc& a) { return a; }
  __device__ __forceinline__ static V acc_get_norm(const Acc& a) { return a; }
  __device__ __forceinline__ static V add(V a, V b) { return a + b; }
  __device__ __forceinline__ static V sub(V a, V b) { return a - b; }
  __device__ __forceinline__ static V mul(V a, V b) { return a * b; }
  __device__ __forceinline__ static V mul_nr(V a, V b) { return a * b; }
  __device__ __forceinline__ static V add_nr(V a, V b) { return a + b; }
  __device__ __forceinline__ static V sub_nr(V a, V b) { return a - b; }
  __device__ __forceinline__ static V neg(V a) { return -a; }
  __device__ __forceinline__ static V fmadd(V a, V b, V c) { return fma(a, b, c); }
  __device__ __forceinline__ static V half(V a) { return 0.5 * a; }
  // a * f for f a power of two, its negative or zero (exact)
  __device__ __forceinline__ static V scale_pow2(V a, float f) { return (double)f * a; }
  __device__ __forceinline__ static V absval(V a) { return fabs(a); }
  __device__ __forceinline__ static V sqrt_(V a) { return sqrt(a); }
  __device__ __forceinline__ static bool greater(V a, V b) { return a > b; }
  __device__ __forceinline__ static bool equal(V a, V b) { return a == b; }
  __device__ __forceinline__ static int sign(V a) { return a > 0.0 ? 1 : (a < 0.0 ? -1 : 0); }
  __device__ __forceinline__ static G store(V x) { return x; }
};

struct DF64 {
  typedef double G;
  typedef df64 V;
  struct Acc {
    float s, e;
  };
  static constexpr bool emulated = true;

  __device__ __forceinline__ static void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  }
  __device__ __forceinline__ static V renorm(float s, float e) {
    V r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
    return r;
  }
  __device__ __forceinline__ static V from_double(double x) {
    V r;
    r.hi = __double2float_rn(x);
    r.lo = __double2float_rn(x - (double)r.hi);
    return r;
  }
  // Split of a double held in global memory, by integer operations only (no
  // FP64 instruction): hi = sign, exponent and the leading 23 fraction bits
  // (truncated), lo = the remaining 29 fraction bits rounded to a float, same
  // sign.  |hi + lo - x| <= 2^-47 |x| for 2^-74 <= |x| < 2^127; below 2^-74
  // lo is dropped (absolute error < 2^-97), below 2^-126 the value is zero.
  __device__ __forceinline__ static V load(const double* p) { return split(__ldg(p)); }
  __device__ __forceinline__ static V split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
    const unsigned sgn = h & 0x80000000u;
    const int e = (int)((h >> 20) & 0x7FFu);
    const unsigned m23 = ((h & 0xFFFFFu) << 3) | (l >> 29);
    V r;
    r.hi = e >= 897 ? __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | m23) : 0.0f;
    const float rest = __uint2float_rn(l & 0x1FFFFFFFu);
    const float scale = __uint_as_float((unsigned)(e >= 949 ? e - 948 : 1) << 23);
    r.lo = e >= 949 ? __uint_as_float(__float_as_uint(__fmul_rn(rest, scale)) | sgn) : 0.0f;
    return r;
  }
  __device__ __forceinline__ static double to_double(V x) { return (double)x.hi + (double)x.lo; }
  __device__ __forceinline__ static G store(V x) { return to_double(x); }
  __host__ static V make(double x) {
    V r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
  }
  __device__ __forceinline__ static V zero() {
    V r;
    r.hi = 0.0f;
    r.lo = 0.0f;
    return r;
  }
  __device__ __forceinline__ static void acc_zero(Acc& a) {
    a.s = 0.0f;
    a.e = 0.0f;
  }
  __device__ __forceinline__ static void acc_set(Acc& a, V x) {
    a.s = x.hi;
    a.e = x.lo;
  }
  // a += c * x
  __device__ __forceinline__ static void acc_fma(Acc& a, V c, V x) {
    const float p = __fmul_rn(c.hi, x.hi);
    float pe = __fmaf_rn(c.hi, x.hi, -p);
    pe = __fmaf_rn(c.hi, x.lo, pe);
    pe = __fmaf_rn(c.lo, x.hi, pe);
    float s, e;
    two_sum(a.s, p, s, e);
    a.s = s;
    a.e = __fadd_rn(a.e, __fadd_rn(e, pe));
  }
  // a = c * x (the first term of a dot product: no two-sum with zero)
  __device__ __forceinline__ static void acc_first(Acc& a, V c, V x) {
    a.s = __fmul_rn(c.hi, x.hi);
    float pe = __fmaf_rn(c.hi, x.hi, -a.s);
    pe = __fmaf_rn(c.hi, x.lo, pe);
    a.e = __fmaf_rn(c.lo, x.hi, pe);
  }
  // The value of an accumulator as hi + lo without renormalisation: lo holds
  // the collected rounding errors, small against the terms but not
  // necessarily below half an ulp of hi.  Products and sums take such values
  // as they are; acc_get_norm renormalises (for values that are compared,
  // and in the convective kernels, whose cancelling sums need the accuracy).
  __device__ __forceinline__ static V acc_get(const Acc& a) {
    V r;
    r.hi = a.s;
    r.lo = a.e;
    return r;
  }
  // Renormalisation by Dekker's Fast2Sum, exact when |e| <= |s| up to the
  // exponent (the error sum is far smaller than the running sum unless the
  // sum cancels to its own rounding level); measured identical to the
  // branch-free two-sum on the full-size convective parity cases.
  __device__ __forceinline__ static V acc_get_norm(const Acc& a) {
    V r;
    r.hi = __fadd_rn(a.s, a.e);
    r.lo = __fsub_rn(a.e, __fsub_rn(r.hi, a.s));
    return r;
  }
  __device__ __forceinline__ static V add(V a, V b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return renorm(s, e);
  }
  __device__ __forceinline__ static V neg(V a) {
    a.hi = -a.hi;
    a.lo = -a.lo;
    return a;
  }
  __device__ __forceinline__ static V sub(V a, V b) { return add(a, neg(b)); }
  __device__ __forceinline__ static V mul(V a, V b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return renorm(p, e);
  }
  // Product and sums without the final renormalisation (hi + lo is exact up
  // to the product's or sum's own rounding, lo not necessarily below half an
  // ulp of hi): for intermediates that only feed further products and sums.
  __device__ __forceinline__ static V mul_nr(V a, V b) {
    V r;
    r.hi = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -r.hi);
    e = __fmaf_rn(a.hi, b.lo, e);
    r.lo = __fmaf_rn(a.lo, b.hi, e);
    return r;
  }
  __device__ __forceinline__ static V add_nr(V a, V b) {
    V r;
    float e;
    two_sum(a.hi, b.hi, r.hi, e);
    r.lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return r;
  }
  __device__ __forceinline__ static V sub_nr(V a, V b) { return add_nr(a, neg(b)); }
  // a * b + c
  __device__ __forceinline__ static V fmadd(V a, V b, V c) {
    Acc t;
    acc_set(t, c);
    acc_fma(t, a, b);
    return acc_get(t);
  }
  __device__ __forceinline__ static V half(V a) {
    a.hi *= 0.5f;
    a.lo *= 0.5f;
    return a;
  }
  // a * f for f a power of two, its negative or zero (exact)
  __device__ __forceinline__ static V scale_pow2(V a, float f) {
    a.hi *= f;
    a.lo *= f;
    return a;
  }
  __device__ __forceinline__ static V absval(V a) { return a.hi < 0.0f ? neg(a) : a; }
  // Square root: the float root r of hi and one Newton correction
  // (a - r^2) / (2 r), with r^2 formed exactly by the FMA (a - r^2 is then
  // exact up to the rounding of the small remainder); ~2^-47 relative.
  __device__ __forceinline__ static V sqrt_(V a) {
    if (!(a.hi > 0.0f)) return zero();
    const float r = __fsqrt_rn(a.hi);
    const float p = __fmul_rn(r, r);
    const float pe = __fmaf_rn(r, r, -p);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
    return renorm(r, __fdiv_rn(d, __fmul_rn(2.0f, r)));
  }
  __device__ __forceinline__ static bool greater(V a, V b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
  __device__ __forceinline__ static bool equal(V a, V b) { return a.hi == b.hi && a.lo == b.lo; }
  __device__ __forceinline__ static int sign(V a) { return a.hi > 0.0f ? 1 : (a.hi < 0.0f ? -1 : 0); }
};

// TF64   "triple-float": a value is an unevaluated sum x + y + z of three
//        floats (up to 72 significant bits: at least as wide as FP64), on the
//        FP32 pipe.  A double splits into three floats exactly (the leading
//        24 bits, the next 24, the last 5).  Dot products run in three levels:
//        the leading products c.x v.x are exact (FMA), their running sum is
//        kept error-free with two-sum; the second-order terms (the product
//        errors, the two-sum errors and the exact cross products c.x v.y,
//        c.y v.x) are summed error-free in a second float, whose errors and
//        the third-order terms (c.x v.z, c.y v.y, c.z v.x and the cross
//        products' errors) collect in a third.  The error of a dot product of
//        n terms is about n^2 2^-72 of the sum of |terms|, against n 2^-53
//        for FP64 arithmetic.  Values handed on to further products are
//        renormalised (two two-sums), so that y and z stay below the
//        rounding level of x and y.  Range: a loaded double keeps its 29 low
//        bits above 2^-74 (|x| >= 2^-74 keeps all 53 bits, below 2^-126 it is
//        zero); the float exponent bounds |x| < 2^128.
struct tf64 {
  float x, y, z;
};

struct TF64 {
  typedef double G;
  typedef tf64 V;
  struct Acc {
    float s, t, u;
  };
  static constexpr bool emulated = true;

  __device__ __forceinline__ static void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  }
  __device__ __forceinline__ static void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
  }
  // s + t + u (s leading) as a triple with two two-sums: x + e = s + t
  // exactly, then y + z = e + u exactly.
  __device__ __forceinline__ static V norm3(float s, float t, float u) {
    V r;
    float e;
    two_sum(s, t, r.x, e);
    two_sum(e, u, r.y, r.z);
    return r;
  }
  // Exact split of a double by integer operations (no FP64 instruction):
  // x = sign, exponent and the leading 23 fraction bits, y = the next 24
  // fraction bits, z = the last 5, all with the sign of d.  Exact for
  // 2^-74 <= |d| < 2^128; below 2^-74 z, below 2^-79 y and below 2^-126 x
  // are dropped.
  __device__ __forceinline__ static V split(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
    const unsigned sgn = h & 0x80000000u;
    const int e = (int)((h >> 20) & 0x7FFu);
    const unsigned m23 = ((h & 0xFFFFFu) << 3) | (l >> 29);
    const unsigned rest = l & 0x1FFFFFFFu;
    V r;
    r.x = e >= 897 ? __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | m23) : 0.0f;
    const float fy = __uint2float_rn(rest >> 5), fz = __uint2float_rn(rest & 31u);   // exact
    const float sy = __uint_as_float((unsigned)(e >= 944 ? e - 943 : 1) << 23);     // 2^(e-1070)
    const float sz = __uint_as_float((unsigned)(e >= 949 ? e - 948 : 1) << 23);     // 2^(e-1075)
    r.y = e >= 944 ? __uint_as_float(__float_as_uint(__fmul_rn(fy, sy)) | sgn) : 0.0f;
    r.z = e >= 949 ? __uint_as_float(__float_as_uint(__fmul_rn(fz, sz)) | sgn) : 0.0f;
    return r;
  }
  __device__ __forceinline__ static V load(const double* p) { return split(__ldg(p)); }
  __device__ __forceinline__ static V from_double(double d) { return split(d); }
  // y + z is exact in FP64 for a renormalised triple; one rounding to FP64
  __device__ __forceinline__ static double to_double(V v) {
    return (double)v.x + ((double)v.y + (double)v.z);
  }
  __device__ __forceinline__ static G store(V v) { return to_double(v); }
  __host__ static V make(double d) {
    V r;
    r.x = (float)d;
    const double a = d - (double)r.x;
    r.y = (float)a;
    r.z = (float)(a - (double)r.y);
    return r;
  }
  __device__ __forceinline__ static V zero() {
    V r;
    r.x = r.y = r.z = 0.0f;
    return r;
  }
  __device__ __forceinline__ static void acc_zero(Acc& a) { a.s = a.t = a.u = 0.0f; }
  __device__ __forceinline__ static void acc_set(Acc& a, V v) {
    a.s = v.x;
    a.t = v.y;
    a.u = v.z;
  }
  // a = c * v
  __device__ __forceinline__ static void acc_first(Acc& a, V c, V v) {
    float e0, m1, e1, m2, e2, f1, f2;
    two_prod(c.x, v.x, a.s, e0);
    two_prod(c.x, v.y, m1, e1);
    two_prod(c.y, v.x, m2, e2);
    two_sum(m1, m2, a.t, f1);
    two_sum(a.t, e0, a.t, f2);
    float u = __fadd_rn(__fadd_rn(f1, f2), __fadd_rn(e1, e2));
    u = __fmaf_rn(c.x, v.z, u);
    u = __fmaf_rn(c.y, v.y, u);
    a.u = __fmaf_rn(c.z, v.x, u);
  }
  // a += c * v
  __device__ __forceinline__ static void acc_fma(Acc& a, V c, V v) {
    float p, e0, g, m1, e1, m2, e2, q, f1, r, f2, f3, f4;
    two_prod(c.x, v.x, p, e0);
    two_sum(a.s, p, a.s, g);
    two_prod(c.x, v.y, m1, e1);
    two_prod(c.y, v.x, m2, e2);
    two_sum(m1, m2, q, f1);
    two_sum(g, e0, r, f2);
    two_sum(q, r, q, f3);
    two_sum(a.t, q, a.t, f4);
    float u = __fadd_rn(a.u, __fadd_rn(__fadd_rn(f1, f2), __fadd_rn(f3, f4)));
    u = __fadd_rn(u, __fadd_rn(e1, e2));
    u = __fmaf_rn(c.x, v.z, u);
    u = __fmaf_rn(c.y, v.y, u);
    a.u = __fmaf_rn(c.z, v.x, u);
  }
  __device__ __forceinline__ static V acc_get(const Acc& a) { return norm3(a.s, a.t, a.u); }
  __device__ __forceinline__ static V acc_get_norm(const Acc& a) { return norm3(a.s, a.t, a.u); }
  // a + b without the final renormalisation: the leading parts and the
  // second parts summed error-free, the errors and third parts in z
  __device__ __forceinline__ static V add_nr(V a, V b) {
    float s, e1, t, e2, e3;
    two_sum(a.x, b.x, s, e1);
    two_sum(a.y, b.y, t, e2);
    two_sum(t, e1, t, e3);
    V r;
    r.x = s;
    r.y = t;
    r.z = __fadd_rn(__fadd_rn(a.z, b.z), __fadd_rn(e2, e3));
    return r;
  }
  __device__ __forceinline__ static V add(V a, V b) {
    const V r = add_nr(a, b);
    return norm3(r.x, r.y, r.z);
  }
  __device__ __forceinline__ static V neg(V a) {
    a.x = -a.x;
    a.y = -a.y;
    a.z = -a.z;
    return a;
  }
  __device__ __forceinline__ static V sub(V a, V b) { return add(a, neg(b)); }
  __device__ __forceinline__ static V sub_nr(V a, V b) { return add_nr(a, neg(b)); }
  __device__ __forceinline__ static V mul(V a, V b) {
    Acc t;
    acc_first(t, a, b);
    return acc_get(t);
  }
  __device__ __forceinline__ static V mul_nr(V a, V b) { return mul(a, b); }
  // a * b + c
  __device__ __forceinline__ static V fmadd(V a, V b, V c) {
    Acc t;
    acc_set(t, c);
    acc_fma(t, a, b);
    return acc_get(t);
  }
  __device__ __forceinline__ static V half(V a) {
    a.x *= 0.5f;
    a.y *= 0.5f;
    a.z *= 0.5f;
    return a;
  }
  // a * f for f a power of two, its negative or zero (exact)
  __device__ __forceinline__ static V scale_pow2(V a, float f) {
    a.x *= f;
    a.y *= f;
    a.z *= f;
    return a;
  }
  __device__ __forceinline__ static int sign(V a) {
    return a.x > 0.0f ? 1 : a.x < 0.0f ? -1 : a.y > 0.0f ? 1 : a.y < 0.0f ? -1 : a.z > 0.0f ? 1 : (a.z < 0.0f ? -1 : 0);
  }
  __device__ __forceinline__ static V absval(V a) { return sign(a) < 0 ? neg(a) : a; }
  // Square root by two Newton corrections of the float root r0 of a.x:
  // r1 = r0 + (a - r0^2) / (2 r0) with a - r0^2 formed exactly to float
  // accuracy (~2^-48), then r2 = r1 + (a - r1^2) / (2 r0) with the residual
  // in triple-float (~2^-72).
  __device__ __forceinline__ static V sqrt_(V a) {
    if (!(a.x > 0.0f)) return zero();
    const float r0 = __fsqrt_rn(a.x);
    float p, pe;
    two_prod(r0, r0, p, pe);
    const float d1 = __fadd_rn(__fsub_rn(__fsub_rn(a.x, p), pe), __fadd_rn(a.y, a.z));
    const float inv2r = __fdiv_rn(1.0f, __fmul_rn(2.0f, r0));
    V r1 = norm3(r0, __fmul_rn(d1, inv2r), 0.0f);
    const V res = sub(a, mul(r1, r1));
    return norm3(r1.x, r1.y, __fmul_rn(res.x, inv2r));
  }
  __device__ __forceinline__ static bool greater(V a, V b) { return sign(sub(a, b)) > 0; }
  __device__ __forceinline__ static bool equal(V a, V b) { return a.x == b.x && a.y == b.y && a.z == b.z; }
};

}  // namespace dgns
