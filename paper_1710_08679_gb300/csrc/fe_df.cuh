// Float-float ("double-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits. GB300 executes FP64 at 1/61 of its FP32 rate, so the
// FP64-accurate element products run in this arithmetic instead: the same
// element code (templated on the scalar type) is instantiated with `df`.
//
// Building blocks are the classical error-free transformations: Knuth's TwoSum,
// Dekker's Fast2Sum and the FMA-based TwoProd (see Muller et al., Handbook of
// Floating-Point Arithmetic, ch. 4, and Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic",
// ACM TOMS 2017). Addition is the "sloppy" double-word sum (TwoSum of the high
// parts plus the low parts, then Fast2Sum): its error is bounded by a small
// multiple of 2^-48 (|a| + |b|) rather than of |a + b|, which is the normwise
// accuracy a sum of element contributions needs. Multiplication uses TwoProd on
// the high parts plus the two cross terms.
#pragma once

namespace fe {

struct df {
  float hi, lo;
  __host__ __device__ df() : hi(0.f), lo(0.f) {}
  __host__ __device__ explicit df(float h, float l) : hi(h), lo(l) {}
  // small constants of the element code (exact in float)
  __host__ __device__ df(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  const float s = a + b;
  return df(s, b - (s - a));
}

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ df operator+(const df& a, const df& b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ df operator-(const df& a) { return df(-a.hi, -a.lo); }

__device__ __forceinline__ df operator-(const df& a, const df& b) { return a + (-b); }

__device__ __forceinline__ df operator*(const df& a, const df& b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  return df_fast_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}

__device__ __forceinline__ df& operator+=(df& a, const df& b) {
  a = a + b;
  return a;
}

// exact split of a double into float-float (hi = RN(x), lo = RN(x - hi))
__device__ __forceinline__ df df_from_double(double x) {
  const float h = __double2float_rn(x);
  return df(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double df_to_double(const df& a) { return (double)a.hi + (double)a.lo; }

}  // namespace fe
