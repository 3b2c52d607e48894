// Double-float arithmetic for the setup kernels (sm_103a).
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 44 significant bits.  The setup path (PSF and measurement spectra,
// the per-frequency Gram matrix, its Cholesky inverse and the data term) needs
// far more than FP32 precision -- the factor is ill-conditioned where the PSFs
// vanish -- but this part issues FP64 at a small fraction of its FP32 rate,
// so for complex64 plans those kernels compute in double-float on the FP32
// pipes instead.  The building blocks are the classical error-free
// transformations: Knuth's two-sum, the fast two-sum for ordered operands,
// and the product error a*b - fl(a*b) obtained exactly with one fused
// multiply-add.  Addition is the "sloppy" double-float sum (error about 2^-44
// of the operands' magnitude), the normwise error model an FFT or a Cholesky
// factorisation needs.  Nothing here may be compiled with reassociation or
// fast-math.
#pragma once
#include "common.cuh"

namespace cip {

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df64(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ constexpr df64(int i) : hi((float)i), lo(0.0f) {}
  // hi = round(d), lo = round(d - hi)
  __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

__host__ __device__ __forceinline__ double to_double(df64 a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ float to_float(df64 a) { return a.hi + a.lo; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df64(s, e);
}
// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return df64(s, e);
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  df64 s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);  // exact rounding error of the leading product
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
// a * b + c with one renormalisation less than a product followed by a sum (named
// apart from fma so that it never hides the float and double overloads here)
__device__ __forceinline__ df64 dfma(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  df64 s = two_sum(p, c.hi);
  s.lo += e + c.lo;
  return fast_two_sum(s.hi, s.lo);
}

// complex double-float (16 bytes, the size of a double2)
struct __align__(16) cdf {
  df64 x, y;
};
template <> struct CT<df64> { using type = cdf; };

template <> __host__ __device__ __forceinline__ cdf mk<cdf>(double re, double im) {
  cdf c;
  c.x = df64(re);
  c.y = df64(im);
  return c;
}
__device__ __forceinline__ cdf cmk(df64 re, df64 im) {
  cdf c;
  c.x = re;
  c.y = im;
  return c;
}
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return cmk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return cmk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
  return cmk(dfma(a.x, b.x, -(a.y * b.y)), dfma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ cdf cmulc(cdf a, cdf b) {
  return cmk(dfma(a.x, b.x, a.y * b.y), dfma(a.x, b.y, -(a.y * b.x)));
}
// acc += a * b
__device__ __forceinline__ void cfma(cdf& acc, cdf a, cdf b) {
  acc.x = dfma(a.x, b.x, dfma(-a.y, b.y, acc.x));
  acc.y = dfma(a.x, b.y, dfma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(cdf& acc, cdf a, cdf b) {
  acc.x = dfma(a.x, b.x, dfma(a.y, b.y, acc.x));
  acc.y = dfma(a.x, b.y, dfma(-a.y, b.x, acc.y));
}
// read-only cached load of a complex double-float table entry (one 16-byte access)
__device__ __forceinline__ cdf ldg_tw(const cdf* p) {
  const float4 v = ::__ldg(reinterpret_cast<const float4*>(p));
  cdf c;
  c.x = df64(v.x, v.y);
  c.y = df64(v.z, v.w);
  return c;
}

// The same operations on FP64 values, so that a setup kernel is written once
// for double-float (complex64 plans) and FP64 (complex128 plans).
__device__ __forceinline__ double dfma(double a, double b, double c) { return ::fma(a, b, c); }
__host__ __device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double2 cmk(double re, double im) { return make_double2(re, im); }

// conversions between the complex types: cconv<Cout>(v)
template <typename Cout> __device__ __forceinline__ Cout cconv(cdf v);
template <> __device__ __forceinline__ float2 cconv<float2>(cdf v) { return make_float2(to_float(v.x), to_float(v.y)); }
template <> __device__ __forceinline__ double2 cconv<double2>(cdf v) {
  return make_double2(to_double(v.x), to_double(v.y));
}
template <> __device__ __forceinline__ cdf cconv<cdf>(cdf v) { return v; }
template <typename Cout> __device__ __forceinline__ Cout cconv(double2 v);
template <> __device__ __forceinline__ float2 cconv<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 cconv<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ cdf cconv<cdf>(double2 v) {
  cdf c;
  c.x = df64(v.x);
  c.y = df64(v.y);
  return c;
}
// exact scaling by a power of two (the 1/N^2 of the inverse DFT)
__device__ __forceinline__ cdf cscale_pow2(cdf v, float s) {
  v.x.hi *= s;
  v.x.lo *= s;
  v.y.hi *= s;
  v.y.lo *= s;
  return v;
}
__device__ __forceinline__ double2 cscale_pow2(double2 v, float s) { return make_double2(v.x * s, v.y * s); }

// arithmetic of the setup path: double-float for complex64 plans, FP64 for complex128 plans
template <typename T> struct SetupReal { using type = df64; };
template <> struct SetupReal<double> { using type = double; };
template <typename T> using SetupC = typename CT<typename SetupReal<T>::type>::type;

// host: split an FP64 value into a double-float
inline df64 df64_from_host(double d) {
  const float h = (float)d;
  return df64(h, (float)(d - (double)h));
}

}  // namespace cip
