// Accuracy of the double-float arithmetic of csrc/dd.cuh (CPU test; built by
// tests/test_dd_cpu.py with the host compiler, FMA contraction off).
//
// Reference values come from long double (64-bit significand on x86-64, 113-bit on
// AArch64), exact for the products and sums checked here to well below the ~2^-47
// accuracy of a double-float.  Checked over random inputs spanning 2^-40..2^40, with
// cancellation: dd_add, dd_add_f (a double-float plus an FP32 correction), dd_mul,
// dd_rsqrt, the complex product, c x + s y, and the compensated dot product
// over 16-term chains combined pairwise with dd_add (the Jacobi inner products: h rows
// split over 32 lanes, then a butterfly).  Prints the worst relative errors (to the
// magnitude sum for dot products) and exits 1 if one exceeds its bound.
#include <cmath>
#include <cstdio>
#include <random>
#include "dd.cuh"

typedef long double LD;
static LD val(dd a) { return (LD)a.hi + (LD)a.lo; }
static dd rnd_dd(std::mt19937_64& g) {
  std::uniform_real_distribution<double> u(-1.0, 1.0), ex(-40.0, 40.0);
  const double x = u(g) * std::ldexp(1.0, (int)ex(g));
  return dd_from(x);
}

int main() {
  std::mt19937_64 g(7);
  double w_add = 0, w_mul = 0, w_cmul = 0, w_dot = 0;
  for (int t = 0; t < 200000; ++t) {
    dd a = rnd_dd(g), b = rnd_dd(g);
    if (t % 4 == 0) b = dd_neg(dd_add(a, dd_make(b.hi * 1e-7f, 0.f)));  // near-cancellation
    const LD ra = val(a), rb = val(b);
    const LD s = ra + rb, p = ra * rb;
    const dd ds = dd_add(a, b), dp = dd_mul(a, b);
    const LD scale_s = fabsl(ra) + fabsl(rb);
    if (scale_s > 0) w_add = std::fmax(w_add, (double)(fabsl(val(ds) - s) / scale_s));
    if (p != 0) w_mul = std::fmax(w_mul, (double)(fabsl(val(dp) - p) / fabsl(p)));
  }
  for (int t = 0; t < 100000; ++t) {
    ddc x = ddc_make(rnd_dd(g), rnd_dd(g)), y = ddc_make(rnd_dd(g), rnd_dd(g));
    const ddc z = ddc_mul(x, y);
    const LD re = val(x.re) * val(y.re) - val(x.im) * val(y.im), im = val(x.re) * val(y.im) + val(x.im) * val(y.re);
    const LD sc = fabsl(val(x.re) * val(y.re)) + fabsl(val(x.im) * val(y.im)) + fabsl(val(x.re) * val(y.im)) +
                  fabsl(val(x.im) * val(y.re));
    if (sc > 0) w_cmul = std::fmax(w_cmul, (double)((fabsl(val(z.re) - re) + fabsl(val(z.im) - im)) / sc));
  }
  double w_lin = 0;
  for (int t = 0; t < 100000; ++t) {  // c x + s y: a Jacobi rotation's update
    const dd c = rnd_dd(g), sn = rnd_dd(g);
    const ddc x = ddc_make(rnd_dd(g), rnd_dd(g)), y = ddc_make(rnd_dd(g), rnd_dd(g));
    const ddc z = ddc_lin(c, x, sn, y);
    const LD re = val(c) * val(x.re) + val(sn) * val(y.re), im = val(c) * val(x.im) + val(sn) * val(y.im);
    const LD sc = fabsl(val(c) * val(x.re)) + fabsl(val(sn) * val(y.re)) + fabsl(val(c) * val(x.im)) +
                  fabsl(val(sn) * val(y.im));
    if (sc > 0) w_lin = std::fmax(w_lin, (double)((fabsl(val(z.re) - re) + fabsl(val(z.im) - im)) / sc));
  }
  double w_addf = 0;
  for (int t = 0; t < 200000; ++t) {  // a + f: the small-angle rotation's update
    const dd a = rnd_dd(g);
    std::uniform_real_distribution<double> u1(-1.0, 1.0);
    const float f = (float)(u1(g) * std::fabs((double)a.hi) * (t % 2 ? 1e-7 : 1.0));
    const LD ex = val(a) + (LD)f, sc = fabsl(val(a)) + fabsl((LD)f);
    if (sc > 0) w_addf = std::fmax(w_addf, (double)(fabsl(val(dd_add_f(a, f)) - ex) / sc));
  }
  double w_rsq = 0;
  for (int t = 0; t < 200000; ++t) {  // 1 / sqrt(x): rotation cosines and unit phases
    std::uniform_real_distribution<double> u1(0.0, 1.0), ex(-60.0, 60.0);
    const dd x = dd_from(std::ldexp(0.5 + u1(g), (int)ex(g)));
    const LD ex_v = 1.0L / sqrtl(val(x));
    w_rsq = std::fmax(w_rsq, (double)(fabsl(val(dd_rsqrt(x)) - ex_v) / ex_v));
  }
  std::normal_distribution<double> nd(0.0, 1.0);
  for (int t = 0; t < 2000; ++t) {
    // 32 lanes x 16 terms of a unit-scale dot product, lane sums combined pairwise
    dd part[32];
    LD exact = 0, mag = 0;
    for (int l = 0; l < 32; ++l) {
      dd_acc acc = dd_acc_zero();
      for (int k = 0; k < 16; ++k) {
        const dd a = dd_from(nd(g)), b = dd_from(nd(g) * (t % 2 ? 1e-6 : 1.0));
        dd_acc_mac(acc, a, b);
        exact += val(a) * val(b);
        mag += fabsl(val(a) * val(b));
      }
      part[l] = dd_acc_value(acc);
    }
    for (int o = 16; o > 0; o >>= 1)
      for (int l = 0; l < o; ++l) part[l] = dd_add(part[l], part[l + o]);
    w_dot = std::fmax(w_dot, (double)(fabsl(val(part[0]) - exact) / mag));
  }
  const double u = std::ldexp(1.0, -24);
  std::printf("add %.3e add_f %.3e mul %.3e rsqrt %.3e cmul %.3e lin %.3e dot %.3e "
              "(units of u^2: %.1f %.1f %.1f %.1f %.1f %.1f %.1f)\n",
              w_add, w_addf, w_mul, w_rsq, w_cmul, w_lin, w_dot, w_add / (u * u), w_addf / (u * u), w_mul / (u * u),
              w_rsq / (u * u), w_cmul / (u * u), w_lin / (u * u), w_dot / (u * u));
  const bool ok = w_add <= 4 * u * u && w_addf <= 4 * u * u && w_mul <= 8 * u * u && w_rsq <= 4 * u * u &&
                  w_cmul <= 16 * u * u && w_lin <= 16 * u * u && w_dot <= 64 * u * u;
  return ok ? 0 : 1;
}
