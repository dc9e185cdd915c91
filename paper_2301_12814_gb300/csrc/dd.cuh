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
#define DD_F2I(a) __float_as_int(a)
#define DD_I2F(a) __int_as_float(a)
#else
#define DD_ADD(a, b) ((a) + (b))
#define DD_SUB(a, b) ((a) - (b))
#define DD_MUL(a, b) ((a) * (b))
#define DD_FMA(a, b, c) fmaf((a), (b), (c))
#define DD_RSQRT(a) (1.0f / sqrtf(a))
#include <string.h>
static inline int dd_f2i_host(float a) { int i; memcpy(&i, &a, sizeof i); return i; }
static inline float dd_i2f_host(int i) { float a; memcpy(&a, &i, sizeof a); return a; }
#define DD_F2I(a) dd_f2i_host(a)
#define DD_I2F(a) dd_i2f_host(a)
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

// ---- Jacobi rotations of complex double-float column pairs (the FP64 path's one-sided
// refinement).  A pair (a, b) with squared norms al, be and inner product g = a^dag b
// is rotated so that a'^dag b' = 0: t = tan(angle) from tau = (be - al) / 2|g|, the
// cosine c and sine s = t c, and the unit phase e = g / |g|.

// Rotation parameters of a double-float column pair on the FP32 pipe (GB300 runs FP64
// at 1/61 of the FP32 rate, and the cluster sweeps form them in every lane of the
// pair's warp).  The decision and angle of the FP64 sweeps: rotate when both columns
// are above the floor and |g| exceeds tol_abs and os_rel sqrt(al be); tau =
// (be - al) / 2|g| with be - al in double-float, t = tan(angle) rounded to FP32.  Then
// c = 1 / sqrt(1 + t^2) and s = t c in double-float (1 + t^2 exact, dd_rsqrt), and the
// unit phase e = g / |g| in double-float from g scaled by a power of two (exact) so
// that |g|^2 neither underflows nor overflows.  r2 = |g|^2 / (al be) for the sweep stop.
__host__ __device__ __forceinline__ float pow2_recip(float m) {  // 2^-E with m in [2^E, 2^(E+1)), m > 0 finite
  const int ex = (DD_F2I(m) >> 23) & 0xff;
  return DD_I2F((254 - (ex > 0 ? ex : 1)) << 23);
}
__host__ __device__ __forceinline__ bool dd_os_params(dd al, dd be, dd gr, dd gi, bool selfm, float tol_abs,
                                                      float col_floor, float os_rel, dd& c, dd& s, ddc& e, dd& gabs,
                                                      float& r2) {
  if (selfm) gi = dd_zero();
  const float a = al.hi, b = be.hi;
  const float gf = selfm ? fabsf(gr.hi) : hypotf(gr.hi, gi.hi);
  const bool above = a > col_floor && b > col_floor;
  const float rel = above ? gf * DD_RSQRT(a) * DD_RSQRT(b) : 0.f;
  r2 = rel * rel;
  if (!(above && gf > tol_abs && rel > os_rel)) return false;
  const float tau = 0.5f * dd_sub(be, al).hi / gf;
  if (!(fabsf(tau) < 1e30f)) return false;  // angle below any representable rotation
  const float af = fabsf(tau);
  const float t = (tau >= 0.f ? 1.f : -1.f) * (af > 1e4f ? 0.5f / af : 1.f / (af + sqrtf(1.f + tau * tau)));
  const float p = DD_MUL(t, t), pe = DD_FMA(t, t, -p);
  c = dd_rsqrt(dd_add_f(dd_add_f(dd_make(1.f, 0.f), p), pe));
  s = dd_mul(dd_make(t, 0.f), c);
  if (selfm) {
    const bool neg = gr.hi < 0.f;
    e = ddc_make(dd_make(neg ? -1.f : 1.f, 0.f), dd_zero());
    gabs = neg ? dd_neg(gr) : gr;
  } else {
    const float sc = pow2_recip(fmaxf(fabsf(gr.hi), fabsf(gi.hi))), isc = 1.f / sc;
    const dd xr = dd_make(gr.hi * sc, gr.lo * sc), xi = dd_make(gi.hi * sc, gi.lo * sc);
    const dd g2 = dd_add(dd_mul(xr, xr), dd_mul(xi, xi));  // in [1, 8)
    const dd inv = dd_rsqrt(g2);
    e = ddc_make(dd_mul(xr, inv), dd_mul(xi, inv));
    const dd gs = dd_mul(g2, inv);
    gabs = dd_make(gs.hi * isc, gs.lo * isc);
  }
  return true;
}
// Squared column norms after the rotation (c, s, e) of a pair with norms al, be and
// inner product g: with b~ = conj(e) b, a^dag b~ = |g|, so
//   |a'|^2 = c^2 al + s^2 be - 2 c s |g|,  |b'|^2 = s^2 al + c^2 be + 2 c s |g|
// (both rotation forms of ddc_rotate_dd give these).  The double-float sweeps carry the
// norms this way from pair to pair and recompute them at the start of every sweep,
// so a sweep forms one inner product per pair instead of three.
__host__ __device__ __forceinline__ void rotated_norms_dd(dd& al, dd& be, dd gabs, dd c, dd s) {
  const dd cc = dd_mul(c, c), ss = dd_mul(s, s);
  dd x = dd_mul(dd_mul(c, s), gabs);
  x = dd_add(x, x);
  const dd a2 = dd_sub(dd_add(dd_mul(cc, al), dd_mul(ss, be)), x);
  const dd b2 = dd_add(dd_add(dd_mul(ss, al), dd_mul(cc, be)), x);
  al = a2;
  be = b2;
}

// Rotation angles below this apply through FP32 corrections (ddc_rotate_dd).
constexpr double DD_SMALL_ROT = 1e-7;

// Apply the rotation (c, s, e) to the column pair (x, y) in double-float, elements
// lane, lane + 32, ... < len.  Large angles: x' = c x - s conj(e) y, y' = s x + c conj(e) y
// (the column-q phase form of the FP64 path).  Angles |s| < DD_SMALL_ROT: the
// phase-free rotation x' = c x - s conj(e) y, y' = c y + s e x -- the same unitary up
// to the phase conj(e) on column q, a gauge that W and V share (the product W V^dag,
// and with it X and Y of the re-split, is unchanged) -- written as x + dx, y + dy with
// dx = (c - 1) x - s conj(e) y and dy = (c - 1) y + s e x formed in FP32 from the high
// parts: |dx|, |dy| <= ~1e-7 |x, y|, so the FP32 rounding and the neglected low parts
// stay near 1e-14 relative, and an element costs a TwoSum per component instead of two
// double-float products.
__host__ __device__ __forceinline__ void ddc_rotate_dd(ddc* x, ddc* y, int len, int lane, dd c, dd s, ddc e) {
  if (fabsf(s.hi) < (float)DD_SMALL_ROT) {
    const float cm1 = (c.hi - 1.f) + c.lo, sf = s.hi;  // c.hi - 1 is exact (Sterbenz)
    const float er = e.re.hi, ei = e.im.hi;
    for (int k = lane; k < len; k += 32) {
      const ddc a = x[k], b = y[k];
      const float ceb_r = er * b.re.hi + ei * b.im.hi, ceb_i = er * b.im.hi - ei * b.re.hi;  // conj(e) b
      const float ea_r = er * a.re.hi - ei * a.im.hi, ea_i = er * a.im.hi + ei * a.re.hi;    // e a
      const float dxr = cm1 * a.re.hi - sf * ceb_r, dxi = cm1 * a.im.hi - sf * ceb_i;
      const float dyr = cm1 * b.re.hi + sf * ea_r, dyi = cm1 * b.im.hi + sf * ea_i;
      x[k] = ddc_make(dd_add_f(a.re, dxr), dd_add_f(a.im, dxi));
      y[k] = ddc_make(dd_add_f(b.re, dyr), dd_add_f(b.im, dyi));
    }
    return;
  }
  const dd msd = dd_neg(s);
  const ddc ec = ddc_conj(e);
  for (int k = lane; k < len; k += 32) {
    const ddc a = x[k], bs = ddc_mul(y[k], ec);
    x[k] = ddc_lin(c, a, msd, bs);
    y[k] = ddc_lin(s, a, c, bs);
  }
}

// ---- products of the Newton-Schulz orthonormalisation and of W = Theta V

// sum_{i < len} conj(a[i sa]) b[i sb] (conj_a) or a[i sa] b[i sb], in double-float
__host__ __device__ __forceinline__ ddc ddc_dot(const ddc* a, long long sa, const ddc* b, long long sb, int len,
                                                bool conj_a) {
  dd tr = dd_zero(), ti = dd_zero();
  for (int i0 = 0; i0 < len; i0 += 16) {
    dd_acc ar = dd_acc_zero(), ai = dd_acc_zero();
    const int i1 = len < i0 + 16 ? len : i0 + 16;
    for (int i = i0; i < i1; ++i) {
      const ddc x = a[(long long)i * sa], y = b[(long long)i * sb];
      const dd xi = conj_a ? dd_neg(x.im) : x.im;
      dd_acc_mac(ar, x.re, y.re);
      dd_acc_mac(ar, dd_neg(xi), y.im);
      dd_acc_mac(ai, x.re, y.im);
      dd_acc_mac(ai, xi, y.re);
    }
    tr = dd_add(tr, dd_acc_value(ar));
    ti = dd_add(ti, dd_acc_value(ai));
  }
  return ddc_make(tr, ti);
}

// One element of a Newton-Schulz step V <- V (3 I - S) / 2 = V - V E / 2 with
// S = V^dag V (double-float, column-major n x n) and E = S - I: element (i, b) of the
// new V.  |E| is the non-orthogonality of V (~1e-6 after the FP32 seed, ~1e-11 after
// one step), so V E is formed in FP32 from the high parts: its rounding is below
// 1e-7 |E| sqrt(n), which the next step (or, after the second, the double-float
// precision itself) absorbs, and the correction is added to v_ib by one TwoSum per
// component.  The product costs n complex FP32 FMAs instead of n complex
// double-float ones.
__host__ __device__ __forceinline__ ddc ns_update(const ddc* V, const ddc* S, int n, int b, int i) {
  float cr = 0.f, ci = 0.f;
  const ddc* sb = S + (long long)b * n;
  for (int a = 0; a < n; ++a) {
    const ddc sv = sb[a];
    const float er = a == b ? (sv.re.hi - 1.f) + sv.re.lo : sv.re.hi;  // hi - 1 is exact near 1
    const float ei = sv.im.hi;
    const ddc v = V[(long long)a * n + i];
    cr = fmaf(v.re.hi, er, fmaf(-v.im.hi, ei, cr));
    ci = fmaf(v.re.hi, ei, fmaf(v.im.hi, er, ci));
  }
  const ddc v = V[(long long)b * n + i];
  return ddc_make(dd_add_f(v.re, -0.5f * cr), dd_add_f(v.im, -0.5f * ci));
}
