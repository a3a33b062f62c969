// Double-float ("double-word") arithmetic on the FP32 units.
//
// A dfloat is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2: about 48 significant bits, at FP32 exponent range.  It
// carries the frequency domain of the adjoint's demag transpose, where FP32
// rounding (a relative error of a Fourier coefficient is a global error in
// space) would swamp the small adjoint field far from its sources.  FP64 on
// this GPU runs at 1/64 of the FP32 rate; a double-float add costs 11 FP32
// operations and a product 8.
//
// The building blocks are the error-free transformations
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, any a, b;
//   Fast2Sum (Dekker 1971): s + e = a + b exactly when exp(a) >= exp(b);
//   TwoProd with a fused multiply-add: p + e = a * b exactly;
// and the double-word algorithms analysed by Joldes, Muller and Popescu
// (ACM TOMS 44(2), 2017): the "sloppy" sum (their Algorithm 4), whose error
// is bounded in absolute terms by a small multiple of 2^-48 (|a| + |b|) but
// not relative to the result under cancellation -- which is what an FFT
// needs, its own error bound being normwise -- and the product with one FMA
// per cross term (their Algorithm 11), relative error below 5 * 2^-48.
//
// Device code uses the _rn intrinsics, which the compiler never contracts
// into FMAs or reassociates; host code (the host build of the FFT tests)
// uses plain operations and std::fma with contraction off.
#pragma once

#include <cmath>

#include <cuda_runtime.h>

namespace llg {

namespace dw {

__host__ __device__ __forceinline__ float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
__host__ __device__ __forceinline__ float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// s + e == a + b exactly.
__host__ __device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = add(a, b);
  const float bb = sub(s, a);
  e = add(sub(a, sub(s, bb)), sub(b, bb));
  return s;
}
// s + e == a + b exactly when the exponent of a is at least that of b.
__host__ __device__ __forceinline__ float fast_two_sum(float a, float b, float& e) {
  const float s = add(a, b);
  e = sub(b, sub(s, a));
  return s;
}
// p + e == a * b exactly (barring underflow).
__host__ __device__ __forceinline__ float two_prod(float a, float b, float& e) {
  const float p = mul(a, b);
  e = fma(a, b, -p);
  return p;
}

}  // namespace dw

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit dfloat(float h) : hi(h), lo(0.f) {}
  __host__ __device__ constexpr explicit dfloat(int i) : hi((float)i), lo(0.f) {}
  // rounds d to the nearest pair (compile-time constants, host-side tables;
  // on the device only in set-up kernels, since it takes FP64 operations)
  __host__ __device__ constexpr explicit dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  // nearest FP32 value of hi + lo
  __host__ __device__ __forceinline__ float to_float() const { return dw::add(hi, lo); }
};

__host__ __device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }

// Sloppy double-word sum (Joldes, Muller, Popescu, Algorithm 4).
__host__ __device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float e;
  const float s = dw::two_sum(a.hi, b.hi, e);
  const float t = dw::add(e, dw::add(a.lo, b.lo));
  float l;
  const float h = dw::fast_two_sum(s, t, l);
  return dfloat(h, l);
}
__host__ __device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

// Double-word product with FMA cross terms (Joldes, Muller, Popescu,
// Algorithm 11; the lo * lo term is below the error bound and dropped).
__host__ __device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  float e;
  const float p = dw::two_prod(a.hi, b.hi, e);
  const float t = dw::fma(a.lo, b.hi, dw::mul(a.hi, b.lo));
  float l;
  const float h = dw::fast_two_sum(p, dw::add(e, t), l);
  return dfloat(h, l);
}

// Complex double-float.  16 bytes, loaded and stored as one float4.
struct __align__(16) dcplx {
  dfloat x, y;
};

// Complex product fused per component: re = a.x b.x - a.y b.y as TwoProd of
// the high parts, one TwoSum of the two products, the four cross terms and
// the two product errors added to its error, and one renormalisation -- 19
// operations per component instead of two products and a sum (27); the
// error stays below a few 2^-48 (|a.x b.x| + |a.y b.y|), normwise as above.
__host__ __device__ __forceinline__ dfloat dot2_sub(dfloat a, dfloat b, dfloat c, dfloat d) {
  // a b - c d
  float e1, e2, es;
  const float p1 = dw::two_prod(a.hi, b.hi, e1);
  const float p2 = dw::two_prod(c.hi, d.hi, e2);
  const float s = dw::two_sum(p1, -p2, es);
  float t = dw::sub(e1, e2);
  t = dw::fma(a.hi, b.lo, t);
  t = dw::fma(a.lo, b.hi, t);
  t = dw::fma(-c.hi, d.lo, t);
  t = dw::fma(-c.lo, d.hi, t);
  float l;
  const float h = dw::fast_two_sum(s, dw::add(es, t), l);
  return dfloat(h, l);
}
__host__ __device__ __forceinline__ dfloat dot2_add(dfloat a, dfloat b, dfloat c, dfloat d) {
  // a b + c d
  return dot2_sub(a, b, -c, d);
}

__host__ __device__ __forceinline__ dcplx cmul(dcplx a, dcplx b) {
  dcplx r;
  r.x = dot2_sub(a.x, b.x, a.y, b.y);
  r.y = dot2_add(a.x, b.y, a.y, b.x);
  return r;
}

}  // namespace llg
