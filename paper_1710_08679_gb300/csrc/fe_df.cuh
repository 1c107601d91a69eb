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
  // small constants of the element code (0, 2, 3, 4, 0.25: exact in float)
  __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ constexpr df(double v) : hi((float)v), lo(0.f) {}
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

// The rare cases of the two conversions below (values outside the float range,
// sums crossing a binade) take the FP64 conversion or addition. They live in
// functions that are never inlined: inlined, the compiler evaluates such a
// one-instruction branch for every value and selects the result, which puts an
// FP64-rate instruction on every conversion.
__device__ __noinline__ df df_split_rare(double x) { return df(__double2float_rn(x), 0.f); }

__device__ __noinline__ double df_add_rare(float hi, float lo) { return (double)hi + (double)lo; }

// Double -> float-float with integer operations only. (On GB300 the double to
// float conversion and double additions run at the FP64 rate, 1/61 of FP32.)
// hi: the double rounded to 24 significant bits (round half away from zero, by
// adding half a unit of the 24th bit to the bit pattern and truncating; a carry
// into the exponent is the correct rounding); lo: the remaining x - hi, counted
// in units of the double's last place and scaled back. |x| below 2^-74 keeps lo = 0
// (an error below 2^-98 absolute); zero, infinities and NaN map to hi = (float)x.
__device__ __forceinline__ df df_split(double x) {
  const long long b = __double_as_longlong(x);
  const long long mag = b & 0x7FFFFFFFFFFFFFFFLL;
  const int e = (int)(mag >> 52);                                  // biased double exponent
  if (e < 1023 - 126 || e > 1023 + 127) return df_split_rare(x);   // rare: out of float range
  const long long rmag = (mag + (1LL << 28)) & ~((1LL << 29) - 1);  // magnitude rounded to 24 bits
  const int re = (int)(rmag >> 52);
  if (re > 1023 + 127) return df_split_rare(x);
  const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
  const float hi = __int_as_float((int)(sign | (unsigned)((re - 1023 + 127) << 23) |
                                        (unsigned)((rmag >> 29) & 0x7FFFFF)));
  float lo = 0.f;
  if (e >= 1023 - 74) {
    const int d = (int)(mag - rmag);                                 // ulps of x's binade, |d| <= 2^28
    const float ulp = __int_as_float((e - 1023 - 52 + 127) << 23);   // 2^(e - 1075), a normal float
    lo = (float)d * ulp;
    if (sign) lo = -lo;
  }
  return df(hi, lo);
}

// Float-float -> double: hi widened to double by rebuilding its bit pattern
// (exact for normal floats), plus lo counted in units of that double's last
// place and added to the pattern. Zero, subnormal, infinite and NaN hi, and sums
// that cross into another binade, take the exact double addition (rare).
__device__ __forceinline__ double df_to_double(const df& a) {
  const unsigned hb = __float_as_uint(a.hi);
  const int eh = (int)((hb >> 23) & 0xFF);                          // biased float exponent of hi
  // the ulp of the double is 2^(eh - 127 - 52); its inverse 2^(179 - eh) is a normal float for eh >= 52
  if (eh < 52 || eh == 255) return df_add_rare(a.hi, a.lo);
  const long long db = (long long)((unsigned long long)(hb >> 31) << 63 |
                                   (unsigned long long)(eh - 127 + 1023) << 52 |
                                   (unsigned long long)(hb & 0x7FFFFFu) << 29);
  if (a.lo == 0.f) return __longlong_as_double(db);
  const float scale = __int_as_float((306 - eh) << 23);
  const int k = __float2int_rn(a.lo * scale);
  const long long rb = db + ((hb >> 31) ? -(long long)k : (long long)k);
  if ((rb >> 52) != (db >> 52)) return df_add_rare(a.hi, a.lo);
  return __longlong_as_double(rb);
}

}  // namespace fe
