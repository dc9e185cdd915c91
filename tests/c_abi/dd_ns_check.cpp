// Newton-Schulz orthonormalisation of the FP64 path's refinement (csrc/dd.cuh:
// ddc_dot for S = V^dag V, ns_update for V <- V - V (S - I) / 2), checked on the host
// against long double (CPU test; built by tests/test_dd_cpu.py with the host compiler,
// FMA contraction off).
//
// V starts as an exactly unitary matrix (Gram-Schmidt in long double, then rounded to
// FP32 as the FP32 seed would be) perturbed by 1e-6: the seed's non-orthogonality.  Two
// steps, each with S formed in double-float and the correction product in FP32, must
// leave |V^dag V - I| at the double-float level (a few 1e-14).  V must also stay close
// to the same two steps done in long double: the first step's FP32 product moves V by
// about 1e-7 |S - I| sqrt(n) (~1e-12), which the second step makes unitary again
// without undoing (any unitary V serves as the refinement's starting basis), so the
// bound there is 1e-11.  Complex and real matrices, sizes 40 and 120.  Prints the worst
// values and exits 1 if one exceeds its bound.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
#include "dd.cuh"

typedef long double LD;
static LD val(dd a) { return (LD)a.hi + (LD)a.lo; }

struct CL {
  LD re, im;
};

// one Newton-Schulz step in long double on a column-major n x n matrix
static void ns_exact(std::vector<CL>& V, int n) {
  std::vector<CL> S((size_t)n * n), T((size_t)n * n);
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < n; ++a) {
      LD sr = 0, si = 0;
      for (int i = 0; i < n; ++i) {
        const CL x = V[(size_t)a * n + i], y = V[(size_t)b * n + i];
        sr += x.re * y.re + x.im * y.im;
        si += x.re * y.im - x.im * y.re;
      }
      S[(size_t)b * n + a] = {sr, si};
    }
  for (int b = 0; b < n; ++b)
    for (int i = 0; i < n; ++i) {
      LD tr = 0, ti = 0;
      for (int a = 0; a < n; ++a) {
        const CL v = V[(size_t)a * n + i];
        CL w = S[(size_t)b * n + a];
        w.re = (a == b ? 1.5L : 0.0L) - 0.5L * w.re;
        w.im = -0.5L * w.im;
        tr += v.re * w.re - v.im * w.im;
        ti += v.re * w.im + v.im * w.re;
      }
      T[(size_t)b * n + i] = {tr, ti};
    }
  V = T;
}

int main() {
  std::mt19937_64 g(5);
  std::normal_distribution<double> nd(0.0, 1.0);
  double w_orth = 0, w_diff = 0, w_start = 0;
  for (int trial = 0; trial < 8; ++trial) {
    const int n = trial < 4 ? 40 : 120;
    const bool real = trial % 2 == 1;
    // random unitary by Gram-Schmidt in long double
    std::vector<CL> U((size_t)n * n);
    for (auto& z : U) z = {(LD)nd(g), real ? 0.0L : (LD)nd(g)};
    for (int k = 0; k < n; ++k) {
      for (int j = 0; j < k; ++j) {
        LD pr = 0, pi = 0;  // <u_j, u_k>
        for (int i = 0; i < n; ++i) {
          const CL x = U[(size_t)j * n + i], y = U[(size_t)k * n + i];
          pr += x.re * y.re + x.im * y.im;
          pi += x.re * y.im - x.im * y.re;
        }
        for (int i = 0; i < n; ++i) {
          const CL x = U[(size_t)j * n + i];
          U[(size_t)k * n + i].re -= pr * x.re - pi * x.im;
          U[(size_t)k * n + i].im -= pr * x.im + pi * x.re;
        }
      }
      LD nn = 0;
      for (int i = 0; i < n; ++i) nn += U[(size_t)k * n + i].re * U[(size_t)k * n + i].re +
                                        U[(size_t)k * n + i].im * U[(size_t)k * n + i].im;
      const LD inv = 1.0L / std::sqrt((double)nn);
      for (int i = 0; i < n; ++i) { U[(size_t)k * n + i].re *= inv; U[(size_t)k * n + i].im *= inv; }
    }
    // the FP32 seed: perturbed by 1e-6 and rounded to FP32
    std::vector<ddc> V((size_t)n * n), S((size_t)n * n), T((size_t)n * n);
    std::vector<CL> Ve((size_t)n * n);
    for (size_t e = 0; e < V.size(); ++e) {
      const float re = (float)(U[e].re + 1e-6L * nd(g) / std::sqrt((double)n));
      const float im = real ? 0.f : (float)(U[e].im + 1e-6L * nd(g) / std::sqrt((double)n));
      V[e] = ddc_make(dd_make(re, 0.f), dd_make(im, 0.f));
      Ve[e] = {(LD)re, (LD)im};
    }
    auto orth = [&](const std::vector<ddc>& X) {
      LD w = 0;
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          LD sr = 0, si = 0;
          for (int i = 0; i < n; ++i) {
            const ddc x = X[(size_t)a * n + i], y = X[(size_t)b * n + i];
            sr += val(x.re) * val(y.re) + val(x.im) * val(y.im);
            si += val(x.re) * val(y.im) - val(x.im) * val(y.re);
          }
          w = std::fmax((double)w, (double)(std::fabs((double)(sr - (a == b ? 1.0L : 0.0L))) + std::fabs((double)si)));
        }
      return (double)w;
    };
    w_start = std::fmax(w_start, orth(V));
    for (int it = 0; it < 2; ++it) {
      for (int b = 0; b < n; ++b)
        for (int a = 0; a <= b; ++a) {
          const ddc v = ddc_dot(&V[(size_t)a * n], 1, &V[(size_t)b * n], 1, n, true);
          S[(size_t)b * n + a] = v;
          S[(size_t)a * n + b] = ddc_conj(v);
        }
      for (int b = 0; b < n; ++b)
        for (int i = 0; i < n; ++i) T[(size_t)b * n + i] = ns_update(V.data(), S.data(), n, b, i);
      V = T;
      ns_exact(Ve, n);
    }
    w_orth = std::fmax(w_orth, orth(V));
    for (size_t e = 0; e < V.size(); ++e)
      w_diff = std::fmax(w_diff, (double)(std::fabs((double)(val(V[e].re) - Ve[e].re)) +
                                           std::fabs((double)(val(V[e].im) - Ve[e].im))));
  }
  std::printf("non-orthogonality: seed %.2e, after two steps %.2e; largest difference from the long-double "
              "steps %.2e\n", w_start, w_orth, w_diff);
  const bool ok = w_start > 1e-7 && w_orth <= 5e-14 && w_diff <= 1e-11;
  return ok ? 0 : 1;
}
