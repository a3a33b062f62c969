// Double-float ("double-word") arithmetic on the FP32 units.
//
// A dfloat is the unevaluated sum hi + lo of two FP32 numbers: about 48
// significant bits, at FP32 exponent range.  It carries the frequency domain
// of the adjoint's demag transpose, where FP32 rounding (a relative error of
// a Fourier coefficient is a global error in space) would swamp the small
// adjoint field far from its sources.  FP64 on this GPU runs at 1/64 of the
// FP32 rate.
//
// The arithmetic is compensated rather than renormalised: hi evolves exactly
// as the plain FP32 computation would, and lo carries the exact rounding
// error of every operation on the hi parts forward, in FP32 (the scheme of
// compensated summation and dot products, Ogita, Rump and Oishi, SIAM J. Sci.
// Comput. 26(6), 2005, applied to every operation of the transform).  The
// errors committed on the lo parts are of order 2^-24 |lo|, so hi + lo agrees
// with the exact result to a small multiple of 2^-48 times the magnitudes
// involved: a normwise bound, which is what an FFT needs (its own error
// bound is normwise).  |lo| is not kept below ulp(hi)/2 -- under
// cancellation hi may even be 0 -- which costs nothing here: the products
// take lo times the other factor's hi in FP32 too.  A sum costs 8 FP32
// operations, a product 5, a complex product 32.
//
// Error-free transformations used:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, any a, b;
//   TwoProd with a fused multiply-add: p + e = a * b exactly.
//
// Device code uses the _rn intrinsics, which the compiler never contracts
// into FMAs or reassociates; host code (the host build of the FFT tests)
// uses plain operations and std::fma with contraction off.
#pragma once

#include <cmath>

#include <cuda_runtime.h>

// A host build that defines LLG_HOST_COUNT_OPS (and the counter) counts
// every FP32 operation of the double-float arithmetic; a test compares the
// count of whole transforms with the benchmark's operation model.  Device
// code and the library's host code are unaffected.
#if defined(LLG_HOST_COUNT_OPS) && !defined(__CUDA_ARCH__)
extern unsigned long long llg_host_fp32_ops;
#define LLG_HOST_OP() (++llg_host_fp32_ops)
#else
#define LLG_HOST_OP() ((void)0)
#endif

namespace llg {

namespace dw {

__host__ __device__ __forceinline__ float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  LLG_HOST_OP();
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  LLG_HOST_OP();
  return a - b;
#endif
}
__host__ __device__ __forceinline__ float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  LLG_HOST_OP();
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  LLG_HOST_OP();
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
  // FP32 value of hi + lo
  __host__ __device__ __forceinline__ float to_float() const { return dw::add(hi, lo); }
};

__host__ __device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }

// Compensated sum: hi = fl(a.hi + b.hi), lo = its error + a.lo + b.lo.
__host__ __device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float e;
  const float s = dw::two_sum(a.hi, b.hi, e);
  return dfloat(s, dw::add(e, dw::add(a.lo, b.lo)));
}
__host__ __device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

// Compensated product: hi = fl(a.hi b.hi), lo = its error + the cross
// terms (the lo * lo term is of second order in the errors and dropped).
__host__ __device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  float e;
  const float p = dw::two_prod(a.hi, b.hi, e);
  const float t = dw::fma(a.lo, b.hi, dw::mul(a.hi, b.lo));
  return dfloat(p, dw::add(e, t));
}

// Complex double-float.  16 bytes, loaded and stored as one float4.
struct __align__(16) dcplx {
  dfloat x, y;
};

// Complex product fused per component: re = a.x b.x - a.y b.y as TwoProd of
// the high parts, one TwoSum of the two products, and the product errors
// and the four cross terms added to its error -- 16 operations per
// component instead of two products and a sum (18).
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
  return dfloat(s, dw::add(es, t));
}
__host__ __device__ __forceinline__ dfloat dot2_add(dfloat a, dfloat b, dfloat c, dfloat d) {
  // a b + c d
  return dot2_sub(a, b, -c, d);
}

// Complex sums with the real and imaginary parts' identical operation
// sequences paired into FP32x2 instructions (sm_100 and later; the same
// round-to-nearest result per part): a TwoSum of the hi pairs and two sums
// of lo pairs, 8 packed operations instead of 16.
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ dcplx cadd_packed(float2 ah, float2 al, float2 bh, float2 bl) {
  const float2 s = __fadd2_rn(ah, bh);
  const float2 bb = __fadd2_rn(s, neg2(ah));
  const float2 e = __fadd2_rn(__fadd2_rn(ah, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(bh, neg2(bb)));
  const float2 l = __fadd2_rn(e, __fadd2_rn(al, bl));
  dcplx r;
  r.x = dfloat(s.x, l.x);
  r.y = dfloat(s.y, l.y);
  return r;
}
__device__ __forceinline__ dcplx cadd(dcplx a, dcplx b) {
  return cadd_packed(f2(a.x.hi, a.y.hi), f2(a.x.lo, a.y.lo), f2(b.x.hi, b.y.hi), f2(b.x.lo, b.y.lo));
}
__device__ __forceinline__ dcplx csub(dcplx a, dcplx b) {
  return cadd_packed(f2(a.x.hi, a.y.hi), f2(a.x.lo, a.y.lo), f2(-b.x.hi, -b.y.hi), f2(-b.x.lo, -b.y.lo));
}
#endif

__host__ __device__ __forceinline__ dcplx cmul(dcplx a, dcplx b) {
  dcplx r;
  r.x = dot2_sub(a.x, b.x, a.y, b.y);
  r.y = dot2_add(a.x, b.y, a.y, b.x);
  return r;
}

}  // namespace llg
