// Bounds walk of the observables kernel's index arithmetic on corrupted bond tables
// (CPU test; built by tests/test_obs_clamp_cpu.py with the host compiler).
//
// k_obs (csrc/obs.cu) reads chi, charge and segoff from device buffers that the
// allocation-free entry point takes from the caller.  It clamps what it reads with
// clamp_chi, pair_ok and clamp_seg (csrc/mpo_internal.cuh).  This program includes
// those same helpers, walks the kernel's three passes (left environments, right
// environments, moments) and the purity loop over random tables with out-of-range
// chi, pair indices and segment offsets, and checks that every index into gam, lam,
// charge, the environments and the output stays inside its buffer.  Exit status 0 =
// every access in bounds.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>
using std::fma;
using std::fmaf;
static int atomicCAS(int* a, int c, int v) { int o = *a; if (o == c) *a = v; return o; }
#include "mpo_internal.cuh"

static long long g_bad = 0;
static void chk(long long idx, long long size, const char* what) {
  if (idx < 0 || idx >= size) {
    if (g_bad < 10) std::printf("out of bounds: %s index %lld size %lld\n", what, idx, size);
    ++g_bad;
  }
}

int main() {
  std::mt19937 rng(12345);
  long long accesses = 0;
  for (int trial = 0; trial < 400; ++trial) {
    const int M = 2 + (int)(rng() % 6), ncap = 1 + (int)(rng() % 7), q = ncap + 1, P = q * q;
    const int D = 1 + (int)(rng() % 40);
    std::uniform_int_distribution<int> wild(-3 * D - 5, 3 * D + 5), wildp(-2 * P, 2 * P);
    std::vector<int> chi(M + 1), charge((size_t)(M + 1) * D), segoff((size_t)(M + 1) * (P + 1));
    for (auto& x : chi) x = (rng() % 3 == 0) ? wild(rng) : (int)(rng() % (D + 1));
    for (auto& x : charge) x = (rng() % 4 == 0) ? wildp(rng) : (int)(rng() % P);
    for (auto& x : segoff) x = (rng() % 3 == 0) ? wild(rng) : (int)(rng() % (D + 1));
    const long long nG = (long long)M * D * D, nL = (long long)(M + 1) * D, nEF = (long long)(M + 1) * D;
    const long long nCh = (long long)(M + 1) * D, nSeg = (long long)(M + 1) * (P + 1), nOut = 1 + 2 * M + (M + 1);
    auto chi_at = [&](int b) { chk(b, M + 1, "chi"); return clamp_chi(chi[b], D); };
    // left environments
    for (int a = 0; a < chi_at(0); ++a) { chk(a, nEF, "E"); chk(a, nL, "lam"); ++accesses; }
    for (int j = 0; j < M; ++j) {
      const int chiA = chi_at(j), chiB = chi_at(j + 1);
      const int* segA = segoff.data() + (long long)j * (P + 1);
      for (int b = 0; b < chiB; ++b) {
        chk((long long)(j + 1) * D + b, nCh, "charge");
        const int pb = charge[(long long)(j + 1) * D + b];
        if (pair_ok(pb, P)) {
          const int x = pair_c(pb, ncap), y = pair_cb(pb, ncap);
          for (int i = 0; x + i <= ncap && y + i <= ncap; ++i) {
            const int pa = (x + i) * q + (y + i);
            chk((long long)j * (P + 1) + pa + 1, nSeg, "segoff");
            int a0, a1;
            clamp_seg(segA, pa, chiA, a0, a1);
            for (int a = a0; a < a1; ++a) {
              chk((long long)j * D + a, nEF, "E");
              chk((long long)j * D * D + (long long)a * D + b, nG, "gam");
              ++accesses;
            }
          }
        }
        chk((long long)(j + 1) * D + b, nEF, "E");
        chk((long long)(j + 1) * D + b, nL, "lam");
      }
    }
    // right environments and moments share the traversal from bond j to bond j+1
    for (int pass = 0; pass < 2; ++pass)
      for (int j = M - 1; j >= 0; --j) {
        const int chiA = chi_at(j), chiB = chi_at(j + 1);
        const int* segB = segoff.data() + (long long)(j + 1) * (P + 1);
        for (int a = 0; a < chiA; ++a) {
          chk((long long)j * D + a, nCh, "charge");
          const int pa = charge[(long long)j * D + a];
          if (!pair_ok(pa, P)) continue;
          const int x = pair_c(pa, ncap), y = pair_cb(pa, ncap);
          for (int i = pass; i <= x && i <= y; ++i) {
            const int pb = (x - i) * q + (y - i);
            chk((long long)(j + 1) * (P + 1) + pb + 1, nSeg, "segoff");
            int b0, b1;
            clamp_seg(segB, pb, chiB, b0, b1);
            for (int b = b0; b < b1; ++b) {
              chk((long long)j * D * D + (long long)a * D + b, nG, "gam");
              chk((long long)(j + 1) * D + b, nEF, "F");
              chk((long long)(j + 1) * D + b, nL, "lam");
              ++accesses;
            }
          }
          chk((long long)j * D + a, nEF, pass ? "E" : "F");
        }
        if (pass) { chk(1 + j, nOut, "out"); chk(1 + M + j, nOut, "out"); }
      }
    for (int b = 0; b <= M; ++b) {
      for (int i = 0; i < chi_at(b); ++i) chk((long long)b * D + i, nL, "lam");
      chk(1 + 2 * M + b, nOut, "out");
    }
    chk((long long)M * D, nEF, "E (trace)");
  }
  std::printf("%lld in-range checks, %lld out of bounds\n", accesses, g_bad);
  return g_bad == 0 ? 0 : 1;
}
