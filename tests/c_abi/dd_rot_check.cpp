// One-sided Jacobi rotations of complex double-float column pairs (csrc/dd.cuh:
// dd_os_params, ddc_rotate_dd, rotated_norms_dd), checked on the host against long
// double (CPU test; built by tests/test_dd_cpu.py with the host compiler, FMA
// contraction off).
//
// For random column pairs (length 48, entries spanning two decades, in both rotation
// regimes: large angles and angles below DD_SMALL_ROT, complex and real pairs):
//   * c^2 + s^2 = 1 and |e| = 1 to a few u^2 (u = 2^-24): the rotation is unitary to
//     the double-float precision, so repeated rotations keep V unitary;
//   * after the rotation the pair's inner product is below 1e-6 of sqrt(al be) (the
//     angle is rounded to FP32), or below the double-float rounding of the columns;
//   * |a'|^2 + |b'|^2 = |a|^2 + |b|^2 to a few u^2 (relative);
//   * rotated_norms_dd gives the rotated columns' squared norms to a few u^2 of the
//     pair's total.
// Prints the worst values and exits 1 if one exceeds its bound.
#include <cmath>
#include <cstdio>
#include <random>
#include "dd.cuh"

typedef long double LD;
static LD val(dd a) { return (LD)a.hi + (LD)a.lo; }

struct Col {
  ddc v[48];
};
static const int H = 48;

static void inner(const Col& a, const Col& b, LD& re, LD& im) {  // a^dag b
  re = 0;
  im = 0;
  for (int k = 0; k < H; ++k) {
    const LD ar = val(a.v[k].re), ai = val(a.v[k].im), br = val(b.v[k].re), bi = val(b.v[k].im);
    re += ar * br + ai * bi;
    im += ar * bi - ai * br;
  }
}
static LD norm2(const Col& a) {
  LD s = 0;
  for (int k = 0; k < H; ++k) s += val(a.v[k].re) * val(a.v[k].re) + val(a.v[k].im) * val(a.v[k].im);
  return s;
}
static dd to_dd(LD x) {
  const float h = (float)x;
  return dd_make(h, (float)(x - (LD)h));
}

int main() {
  std::mt19937_64 g(11);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::uniform_real_distribution<double> u01(0.0, 1.0);
  const double u = std::ldexp(1.0, -24), u2 = u * u;
  double w_unit = 0, w_phase = 0, w_resid = 0, w_total = 0, w_carry = 0;
  int n_small = 0, n_large = 0, n_rot = 0;
  for (int t = 0; t < 20000; ++t) {
    const bool selfm = t % 5 == 0;  // real pairs
    const int regime = t % 2;       // 0: independent columns (large angles), 1: nearly orthogonal
    Col a, b;
    const double sa = std::pow(10.0, 2.0 * u01(g) - 1.0), sb = std::pow(10.0, 2.0 * u01(g) - 1.0);
    for (int k = 0; k < H; ++k) {
      a.v[k] = ddc_make(dd_from(sa * nd(g)), selfm ? dd_zero() : dd_from(sa * nd(g)));
      b.v[k] = ddc_make(dd_from(sb * nd(g)), selfm ? dd_zero() : dd_from(sb * nd(g)));
    }
    if (regime == 1) {  // b <- b - (a^dag b / |a|^2) a + tiny a: inner product ~1e-9 relative
      LD re, im;
      inner(a, b, re, im);
      const LD na = norm2(a), eps = 1e-9L * std::sqrt((double)(norm2(b) / na)) * nd(g);
      const LD cr = re / na - eps, ci = selfm ? 0.0L : im / na;
      for (int k = 0; k < H; ++k) {
        const LD ar = val(a.v[k].re), ai = val(a.v[k].im);
        const LD br = val(b.v[k].re) - (cr * ar - ci * ai), bi = val(b.v[k].im) - (cr * ai + ci * ar);
        b.v[k] = ddc_make(to_dd(br), selfm ? dd_zero() : to_dd(bi));
      }
    }
    LD gr, gi;
    inner(a, b, gr, gi);
    const LD al = norm2(a), be = norm2(b);
    dd c, s, gabs;
    ddc e;
    float r2;
    const bool rot = dd_os_params(to_dd(al), to_dd(be), to_dd(gr), to_dd(gi), selfm, 1e-30f, 1e-28f, 4e-15f, c, s,
                                  e, gabs, r2);
    if (!rot) continue;
    ++n_rot;
    if (std::fabs(s.hi) < (float)DD_SMALL_ROT) ++n_small; else ++n_large;
    const LD cl = val(c), sl = val(s), er = val(e.re), ei = val(e.im);
    w_unit = std::fmax(w_unit, (double)std::fabs(cl * cl + sl * sl - 1.0L));
    w_phase = std::fmax(w_phase, (double)std::fabs(er * er + ei * ei - 1.0L));
    dd a2 = to_dd(al), b2 = to_dd(be);
    rotated_norms_dd(a2, b2, gabs, c, s);
    for (int lane = 0; lane < 32; ++lane) ddc_rotate_dd(a.v, b.v, H, lane, c, s, e);
    LD pr, pi;
    inner(a, b, pr, pi);
    const LD na = norm2(a), nb = norm2(b), tot = al + be;
    // residual relative to the pair, floored at the double-float rounding of the columns
    const LD resid = std::sqrt((double)(pr * pr + pi * pi)) / std::sqrt((double)(al * be));
    const LD floor_r = 64.0L * u2 * std::sqrt((double)(tot * tot / (al * be)));
    w_resid = std::fmax(w_resid, (double)(resid > floor_r ? resid : 0.0L));
    w_total = std::fmax(w_total, (double)(std::fabs(na + nb - tot) / tot));
    w_carry = std::fmax(w_carry, (double)((std::fabs(val(a2) - na) + std::fabs(val(b2) - nb)) / tot));
  }
  std::printf("rotations %d (large %d, small %d): |c^2+s^2-1| %.2e (%.1f u^2), ||e|^2-1| %.2e (%.1f u^2), "
              "residual %.2e, norm sum %.2e (%.1f u^2), carried norms %.2e (%.1f u^2)\n",
              n_rot, n_large, n_small, w_unit, w_unit / u2, w_phase, w_phase / u2, w_resid, w_total, w_total / u2,
              w_carry, w_carry / u2);
  const bool ok = n_large > 1000 && n_small > 1000 && w_unit <= 16 * u2 && w_phase <= 16 * u2 && w_resid <= 1e-6 &&
                  w_total <= 16 * u2 && w_carry <= 16 * u2;
  return ok ? 0 : 1;
}
