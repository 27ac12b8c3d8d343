// Double-float numbers: a value hi + lo held in two floats with |lo| <= ulp(hi)/2, about 48
// significant bits, computed on the FP32 pipes (GB300 runs FP64 at 1/73 of its FP32 rate).
// Built from the error-free transformations of Dekker (1971) and Knuth (TwoSum) and the
// double-word algorithms analysed by Joldes, Muller & Popescu (ACM TOMS 2017), u = 2^-24:
//   add  the "sloppy" double-word sum (TwoSum of the high words, the low words added in float,
//        Fast2Sum): 11 operations, absolute error below about 3u^2 (|x| + |y|) -- as accurate as
//        the "accurate" 20-operation sum except under cancellation, where its error is relative to
//        the operands rather than to the result: the same backward-stable behaviour as a double
//        add at 2^-48 in place of 2^-53.  add_acc is the accurate sum (relative error < 3u^2 +
//        13u^3), kept for the pressure recovery E - |m|^2/(2 rho), where cancellation in cold,
//        fast gas is the reason for extra precision;
//   mul  double-word x double-word with FMA, the low-by-low product dropped: 8 operations,
//        relative error below about 6u^2; mulf_ (double-word x float) 6 operations;
//   rcp, div, sqrt: one Newton correction of an SFU approximation, relative error ~2^-45.
// Comparisons are exact (lexicographic on (hi, lo) of normalised values).  The exponent range is
// that of float: the hydro state here stays far inside it.
#pragma once
#include <cuda_runtime.h>

namespace hydro {

struct df {
  float h, l;
  df() = default;
  __host__ __device__ constexpr df(float hi, float lo) : h(hi), l(lo) {}
  __host__ __device__ df(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
  __host__ __device__ df(float x) : h(x), l(0.f) {}
  __host__ __device__ df(int x) : h((float)x), l(0.f) {}
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  return df(s, (a - (s - bp)) + (b - bp));
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = a + b;
  return df(s, b - (s - a));
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = a * b;
  return df(p, fmaf(a, b, -p));
}

__device__ __forceinline__ df operator-(const df& x) { return df(-x.h, -x.l); }

__device__ __forceinline__ df operator+(const df& x, const df& y) {
  const df s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, s.l + (x.l + y.l));
}
__device__ __forceinline__ df operator-(const df& x, const df& y) { return x + (-y); }
__device__ __forceinline__ df add_acc(const df& x, const df& y) {
  const df s = two_sum(x.h, y.h);
  const df t = two_sum(x.l, y.l);
  const df v = fast_two_sum(s.h, s.l + t.h);
  return fast_two_sum(v.h, v.l + t.l);
}

__device__ __forceinline__ df operator*(const df& x, const df& y) {
  const df c = two_prod(x.h, y.h);
  const float t = fmaf(x.l, y.h, x.h * y.l);
  return fast_two_sum(c.h, c.l + t);
}

// Exact scaling by a power of two, and double-word x float (TwoProd + one FMA + Fast2Sum).
__device__ __forceinline__ df half_(const df& x) { return df(0.5f * x.h, 0.5f * x.l); }
__device__ __forceinline__ df twice_(const df& x) { return df(2.f * x.h, 2.f * x.l); }
__device__ __forceinline__ df mulf_(const df& x, float f) {
  const df c = two_prod(x.h, f);
  return fast_two_sum(c.h, fmaf(x.l, f, c.l));
}
__device__ __forceinline__ df rabs(const df& x) { return x.h < 0.f ? -x : x; }

// Reciprocal: r0 from the SFU, then r = r0 + r0 (1 - y r0) with the residual formed exactly.
__device__ __forceinline__ df rcp_(const df& y) {
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(y.h));
  const df p = two_prod(y.h, r0);          // y.h r0 exactly
  const float e = (1.f - p.h) - p.l;        // 1 - y.h r0 (1 - p.h is exact near 1)
  const float res = fmaf(-y.l, r0, e);      // 1 - y r0
  return fast_two_sum(r0, r0 * res);
}
__device__ __forceinline__ df div_(const df& x, const df& y) {
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(y.h));
  const float q1 = x.h * r0;
  const df r = x - mulf_(y, q1);  // remainder x - y q1
  const float q2 = r.h * r0;
  return fast_two_sum(q1, q2);
}
__device__ __forceinline__ df rsqrt_(const df& x) {  // the square root (named like the float one)
  if (!(x.h > 0.f)) return df(0.f, 0.f);
  float s0;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s0) : "f"(x.h));
  const df p = two_prod(s0, s0);
  const float r = ((x.h - p.h) - p.l) + x.l;  // x - s0^2
  float i0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(i0) : "f"(s0));
  return fast_two_sum(s0, 0.5f * r * i0);
}

// Comparisons of normalised values.
__device__ __forceinline__ bool operator<(const df& a, const df& b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ bool operator>(const df& a, const df& b) { return b < a; }
__device__ __forceinline__ bool operator<=(const df& a, const df& b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(const df& a, const df& b) { return !(a < b); }
__device__ __forceinline__ df dabs(const df& x) { return x.h < 0.f ? -x : x; }

__device__ __forceinline__ bool cmp_lt_floor(const df& x, const df& f) { return x < f; }
__device__ __forceinline__ bool cmp_neg(const df& x) { return x.h < 0.f; }
__device__ __forceinline__ bool cmp_pos(const df& x) { return x.h > 0.f; }
__device__ __forceinline__ bool abs_le(const df& a, const df& b) { return dabs(a) <= dabs(b); }
__device__ __forceinline__ bool abs_lt(const df& a, const df& b) { return dabs(a) < dabs(b); }
__device__ __forceinline__ bool prod_nonpos(const df& a, const df& b) {
  return a.h == 0.f || b.h == 0.f || ((a.h > 0.f) != (b.h > 0.f));
}
__device__ __forceinline__ bool isfinite_(const df& x) { return isfinite(x.h); }

__device__ __forceinline__ df shfl_xor_(const df& v, int o) {
  return df(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
}

}  // namespace hydro
