// Double-float arithmetic: a real number held as the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significand bits (relative
// rounding ~2^-47 per operation).  On GB300 an FP64 instruction has 1/61 of the FP32
// throughput (measured: 1.25 vs 76.7 TFLOP/s), so the FP64 path's refinement of the
// large blocks runs its arithmetic in this form at several times the rate, with
// accuracy far inside the path's 1e-10 parity bar.
//
// The operations are built from the error-free transformations of Knuth (TwoSum),
// Dekker (FastTwoSum) and the FMA-based TwoProd: for FP32 a, b,
//   TwoSum(a, b)  = (s, e) with s = fl(a + b) and s + e = a + b exactly;
//   TwoProd(a, b) = (p, e) with p = fl(a b), e = fma(a, b, -p), p + e = a b exactly.
// dd_add is the accurate double-float sum (both parts combined through TwoSum, then
// renormalised), with relative error ~2^-47 even under cancellation; dd_mul uses
// TwoProd on the high parts and adds the cross terms.  Every step that must round
// exactly as written uses the _rn intrinsics, which the compiler never contracts
// into FMAs (a contracted product would break the error-free transformations).
//
// Dot products (the Jacobi pair inner products) use the compensated scheme of Ogita,
// Rump and Oishi (2005, "Dot2"): the high parts are summed with TwoSum, the rounding
// errors and the cross terms in an FP32 correction, which each lane carries over a
// short chain (the h rows are split over 32 lanes) before the lanes' partial sums are
// combined with dd_add.
#pragma once
#include <math.h>

#if !defined(__CUDACC__) && !defined(__host__)
// host-only compilation (the CPU accuracy test): plain inline functions
#define __host__
#define __device__
#define __forceinline__ inline
#endif

#if defined(__CUDA_ARCH__)
#define DD_ADD(a, b) __fadd_rn((a), (b))
#define DD_SUB(a, b) __fsub_rn((a), (b))
#define DD_MUL(a, b) __fmul_rn((a), (b))
#define DD_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#define DD_RSQRT(a) rsqrtf(a)
#else
#define DD_ADD(a, b) ((a) + (b))
#define DD_SUB(a, b) ((a) - (b))
#define DD_MUL(a, b) ((a) * (b))
#define DD_FMA(a, b, c) fmaf((a), (b), (c))
#define DD_RSQRT(a) (1.0f / sqrtf(a))
#endif

struct dd {
  float hi, lo;
};
// a complex double-float: 16 bytes, the size of a complex128 element
struct ddc {
  dd re, im;
};

__host__ __device__ __forceinline__ dd dd_make(float hi, float lo) { dd r; r.hi = hi; r.lo = lo; return r; }
__host__ __device__ __forceinline__ dd dd_zero() { return dd_make(0.f, 0.f); }

__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = DD_ADD(a, b);
  const float bb = DD_SUB(s, a);
  e = DD_ADD(DD_SUB(a, DD_SUB(s, bb)), DD_SUB(b, bb));
}
// requires |a| >= |b| (or a = 0)
__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = DD_ADD(a, b);
  e = DD_SUB(b, DD_SUB(s, a));
}

__host__ __device__ __forceinline__ dd dd_from(double x) {
  const float h = (float)x;
  return dd_make(h, (float)(x - (double)h));
}
__host__ __device__ __forceinline__ double dd_to(dd a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ dd dd_neg(dd a) { return dd_make(-a.hi, -a.lo); }

__host__ __device__ __forceinline__ dd dd_add(dd a, dd b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = DD_ADD(e, t);
  fast_two_sum(s, e, s, e);
  e = DD_ADD(e, f);
  fast_two_sum(s, e, s, e);
  return dd_make(s, e);
}
__host__ __device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
// a + f for a double-float a and an FP32 f (one TwoSum on the high parts, the low part
// folded into the error, one renormalisation)
__host__ __device__ __forceinline__ dd dd_add_f(dd a, float f) {
  float s, e;
  two_sum(a.hi, f, s, e);
  e = DD_ADD(e, a.lo);
  fast_two_sum(s, e, s, e);
  return dd_make(s, e);
}

__host__ __device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = DD_MUL(a.hi, b.hi);
  float e = DD_FMA(a.hi, b.hi, -p);
  e = DD_FMA(a.hi, b.lo, e);
  e = DD_FMA(a.lo, b.hi, e);
  float s, r;
  fast_two_sum(p, e, s, r);
  return dd_make(s, r);
}

// 1 / sqrt(x) for a double-float x > 0 (x.hi a normal FP32 number): the FP32 estimate
// y0 and two Newton steps y <- y + y (1 - x y^2) / 2, with 1 - x y^2 formed in
// double-float.  Each step squares the relative error (the estimate's 2^-22 at most,
// then ~2^-43, then the double-float rounding of the last step): rotation cosines and
// unit phases built on it stay unitary to a few u^2.
__host__ __device__ __forceinline__ dd dd_rsqrt(dd x) {
  dd y = dd_make(DD_RSQRT(x.hi), 0.f);
  for (int it = 0; it < 2; ++it) {
    const dd r = dd_sub(dd_make(1.f, 0.f), dd_mul(x, dd_mul(y, y)));
    y = dd_add_f(y, DD_MUL(DD_MUL(0.5f, y.hi), r.hi));
  }
  return y;
}

// c x + s y for real double-floats
__host__ __device__ __forceinline__ dd dd_lin(dd c, dd x, dd s, dd y) { return dd_add(dd_mul(c, x), dd_mul(s, y)); }

// ---- compensated accumulation (Dot2): sum = hi + (lo + corr)
struct dd_acc {
  float hi, lo;  // running TwoSum of the leading parts; lo collects every error term
};
__host__ __device__ __forceinline__ dd_acc dd_acc_zero() { dd_acc a; a.hi = 0.f; a.lo = 0.f; return a; }
// acc += a b for double-floats a, b (the lo x lo product is below the target accuracy)
__host__ __device__ __forceinline__ void dd_acc_mac(dd_acc& acc, dd a, dd b) {
  const float p = DD_MUL(a.hi, b.hi);
  float e = DD_FMA(a.hi, b.hi, -p);
  e = DD_FMA(a.hi, b.lo, e);
  e = DD_FMA(a.lo, b.hi, e);
  float s, q;
  two_sum(acc.hi, p, s, q);
  acc.hi = s;
  acc.lo = DD_ADD(acc.lo, DD_ADD(q, e));
}
__host__ __device__ __forceinline__ dd dd_acc_value(dd_acc a) {
  float s, e;
  two_sum(a.hi, a.lo, s, e);
  return dd_make(s, e);
}

// ---- complex.  Products and linear combinations of two terms go through the
// compensated accumulator: both products exactly (TwoProd of the high parts plus
// the cross terms), one TwoSum, the rounding errors summed in FP32, then one
// renormalisation -- an error of a few u^2 relative to the terms' magnitudes, which is
// what the Jacobi rotations need, at about 28 FP32 operations per result.
__host__ __device__ __forceinline__ ddc ddc_make(dd re, dd im) { ddc r; r.re = re; r.im = im; return r; }
__host__ __device__ __forceinline__ ddc ddc_zero() { return ddc_make(dd_zero(), dd_zero()); }
__host__ __device__ __forceinline__ ddc ddc_from(double re, double im) { return ddc_make(dd_from(re), dd_from(im)); }
__host__ __device__ __forceinline__ ddc ddc_conj(ddc a) { return ddc_make(a.re, dd_neg(a.im)); }
// a b + c d for real double-floats
__host__ __device__ __forceinline__ dd dd_dot2(dd a, dd b, dd c, dd d) {
  dd_acc s = dd_acc_zero();
  dd_acc_mac(s, a, b);
  dd_acc_mac(s, c, d);
  return dd_acc_value(s);
}
__host__ __device__ __forceinline__ ddc ddc_mul(ddc a, ddc b) {
  return ddc_make(dd_dot2(a.re, b.re, dd_neg(a.im), b.im), dd_dot2(a.re, b.im, a.im, b.re));
}
__host__ __device__ __forceinline__ ddc ddc_add(ddc a, ddc b) { return ddc_make(dd_add(a.re, b.re), dd_add(a.im, b.im)); }
// c x + s y with real c, s
__host__ __device__ __forceinline__ ddc ddc_lin(dd c, ddc x, dd s, ddc y) {
  return ddc_make(dd_dot2(c, x.re, s, y.re), dd_dot2(c, x.im, s, y.im));
}

