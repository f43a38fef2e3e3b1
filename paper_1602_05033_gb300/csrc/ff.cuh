// Float-pair ("double-float") arithmetic on the fp32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2 after
// normalisation: about 48 significant bits, an exponent range of fp32.  GB300 issues fp32
// FMAs at 64 times its fp64 rate, so a float pair costs far less than an fp64 operation here
// while carrying close to fp64 precision.  The building blocks are the error-free
// transformations of Knuth (TwoSum: the exact rounding error of an addition) and of Dekker with
// a fused multiply-add (TwoProd: the exact rounding error of a product).  Sums of many terms
// are accumulated lazily: the exact error of every addition to hi goes into lo, which is
// folded back by one renormalisation at the end.
#pragma once
#include <cuda_runtime.h>

struct ff {
  float hi, lo;
};

__host__ __device__ __forceinline__ ff ff_make(float h, float l) {
  ff r;
  r.hi = h;
  r.lo = l;
  return r;
}

// s + e = a + b exactly (Knuth)
__host__ __device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float v = s - a;
  e = (a - (s - v)) + (b - v);
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__host__ __device__ __forceinline__ void ff_fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__host__ __device__ __forceinline__ ff ff_norm(ff a) {
  ff r;
  ff_fast_two_sum(a.hi, a.lo, r.hi, r.lo);
  return r;
}

// a + b (both pairs), normalised
__host__ __device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  ff_two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  ff r;
  ff_fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// acc += a * x with a float and x a pair (lazy: acc is left unnormalised)
__host__ __device__ __forceinline__ void ff_acc(ff& acc, float a, ff x) {
  const float p = a * x.hi;
  float e = fmaf(a, x.hi, -p);
  e = fmaf(a, x.lo, e);
  float s, t;
  ff_two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo += t + e;
}

// acc += x * y with both pairs (lazy); the lo * lo term is below the pair's precision
__host__ __device__ __forceinline__ void ff_acc(ff& acc, ff x, ff y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  float s, t;
  ff_two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo += t + e;
}

// acc -= x * y (lazy)
__host__ __device__ __forceinline__ void ff_sub_acc(ff& acc, ff x, ff y) {
  ff nx = ff_make(-x.hi, -x.lo);
  ff_acc(acc, nx, y);
}

// x * y, normalised
__host__ __device__ __forceinline__ ff ff_mul(ff x, ff y) {
  ff r = ff_make(0.f, 0.f);
  ff_acc(r, x, y);
  return ff_norm(r);
}

// the pair nearest a double: hi = fl32(d), lo = fl32(d - hi) (the subtraction is exact)
__host__ __device__ __forceinline__ ff ff_from_double(double d) {
  ff r;
  r.hi = (float)d;
  r.lo = (float)(d - (double)r.hi);
  return r;
}

__host__ __device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// a - b, normalised
__host__ __device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_make(-b.hi, -b.lo)); }

// a / b, normalised: the quotient of the leading parts, corrected once by the remainder
// a - q1 b (formed as a pair), about 2^-47 relative
__host__ __device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q1 = a.hi / b.hi;
  ff p = ff_make(0.f, 0.f);
  ff_acc(p, q1, b);
  const ff r = ff_sub(a, ff_norm(p));
  const float q2 = r.hi / b.hi;
  ff q;
  ff_fast_two_sum(q1, q2, q.hi, q.lo);
  return q;
}

// The pair as an arithmetic type for code templated on its number type (a banded solver run in
// fp32, pairs or fp64): conversions from and to double, the four operations, fma, fabs and
// comparisons.  Comparisons order by the leading part, then the trailing one.
struct fd {
  ff v;
  fd() = default;
  __host__ __device__ __forceinline__ fd(double d) : v(ff_from_double(d)) {}
  __host__ __device__ __forceinline__ explicit fd(ff x) : v(x) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return ff_to_double(v); }
};
__host__ __device__ __forceinline__ fd operator-(fd a) { return fd(ff_make(-a.v.hi, -a.v.lo)); }
__host__ __device__ __forceinline__ fd operator+(fd a, fd b) { return fd(ff_add(a.v, b.v)); }
__host__ __device__ __forceinline__ fd operator-(fd a, fd b) { return fd(ff_sub(a.v, b.v)); }
__host__ __device__ __forceinline__ fd operator*(fd a, fd b) { return fd(ff_mul(a.v, b.v)); }
__host__ __device__ __forceinline__ fd operator/(fd a, fd b) { return fd(ff_div(a.v, b.v)); }
__host__ __device__ __forceinline__ fd fma(fd a, fd b, fd c) {
  ff r = c.v;
  ff_acc(r, a.v, b.v);
  return fd(ff_norm(r));
}
__host__ __device__ __forceinline__ fd fabs(fd a) { return a.v.hi < 0.f ? -a : a; }
__host__ __device__ __forceinline__ bool operator<(fd a, fd b) {
  return a.v.hi < b.v.hi || (a.v.hi == b.v.hi && a.v.lo < b.v.lo);
}
__host__ __device__ __forceinline__ bool operator>(fd a, fd b) { return b < a; }
