// Two-site U(1) MPO update for every gate of one mesh layer (all instances at once).
//
// Paper (arXiv:2301.12814, App. D): for the gate on modes (j, j+1) with bonds
// A = j, C = j+1, B = j+2, compute for every new centre charge m
//   Theta(m)[alpha, beta] = lambda_A lambda_B sum_gamma u(a, b, c, m)
//                           Gamma_j[alpha, gamma] lambda_C[gamma] Gamma_{j+1}[gamma, beta]
// (Eq. `theta`), factorise every Theta(m) (block-diagonal SVD), keep the chi largest
// singular values over all blocks, and re-split Gamma_j = X / lambda_A,
// Gamma_{j+1} = Y / lambda_B.
//
// GB300 design (differs from the paper's A100 kernels, a SIMT GEMM with unitary
// lookups over the whole Theta plus a library SVD):
// * Hermiticity of rho makes Theta(mbar) the ket/bra mirror of Theta(m)
//   (Theta(mbar)[pi a, pi b] = conj Theta(m)[a, b]).  Only the canonical blocks
//   m = (c, cbar) with c <= cbar are contracted and factorised; the mirror block's
//   singular values are bitwise copies and its vectors are conjugated copies.  This
//   halves the work and makes the mirror spectra exactly degenerate, so the
//   keep-chi rule never splits a mirror pair.  Self-mirror blocks (c = cbar) are
//   diagonalised in the basis where the mirror acts as complex conjugation: their
//   Gram matrix is real there (real arithmetic, mirror-symmetric vectors).
// * The contraction runs per (row segment a, column segment b): the partial product
//   P_c = Gamma_j[a, c] lambda_c Gamma_{j+1}[c, b] of every old centre segment c is
//   formed once and mixed into every canonical new centre m between a and b with the
//   weight u(a, b, c, m).  Eq. `theta` evaluates the same sum per m; factoring P_c out
//   removes the repeated inner products and all padding of small segments.
// * The SVD: a Gram matrix (smaller side) and a parallel-order cyclic Jacobi
//   eigensolver, both in FP32 on every path, give a starting basis; a one-sided
//   Jacobi refinement in the path's precision (FP64 on the FP64 path) then iterates
//   to convergence on W = Theta V.  Both run in k_svd: one persistent CTA per SM
//   takes the layer's blocks longest first and keeps each block in 200 KB of shared
//   memory when it fits.
// * The beam-splitter Fock blocks are built on the device by the creation-operator
//   recurrence U|j, n-j> = (S11 a1^dag + S21 a2^dag) U|j-1, n-j> / sqrt(j).
// * Precision: R = double (FP64 path) or float (mixed path: contraction and
//   refinement in FP32); selection, lambda, discarded weight, entropy and the stored
//   state are FP64 on both.
// * The Gram eigenvectors seed a one-sided Jacobi refinement on W = Theta V, which
//   makes the singular values and vectors accurate relative to s_max (not s_max^2)
//   and yields both factors, so the re-split is a scaled copy.
// Stages: k_setup -> k_theta -> k_gram -> k_order -> k_svd -> k_select -> k_resplit.
#include <cooperative_groups.h>
#include <cstdlib>

#include <type_traits>
#include "dd.cuh"
#include "mpo_internal.cuh"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int TILE = 16;
constexpr double TIE_REL = 1e-9;
constexpr int JACOBI_MAX_SWEEPS = 60;
// Which blocks are factorised on a whole thread-block cluster (see the large-block
// section) instead of one CTA: those that would otherwise be the layer's critical
// path, and the large ones.  A block goes to a cluster when its Gram side is at least
// min_n and either its Jacobi work estimate n^2 (n + h) exceeds the layer's total over
// the CTAs of k_svd (it alone would hold one SM longer than the average SM is busy),
// or its Gram side is at least always_n and its work at least 1/16 of that average
// (on one CTA such a block costs more SM-time than on a cluster, unless the layer has
// work enough to keep every SM busy without it: the 64-instance batched mesh lost
// 2.4 % with its blocks from 48 up on clusters).  A throughput-bound layer of small
// blocks (many instances) therefore keeps every block on one CTA.  Measured on GB300,
// s per mesh with every block from a Gram side n0 up on a cluster and no other (the
// load rule alone sent blocks there from about 110 at 48 modes and about 60 at 32
// modes):
//   n0                       48     64     80     96     112    128    load rule
//   48 modes chi 512 FP64   4.23   4.24   4.46   4.51   5.31   5.72   4.51
//   48 modes chi 512 TF32   1.33   1.26   1.31   1.35   1.46   1.57   1.35
//   32 modes chi 256 FP64   0.426  0.472                             0.462
//   32 modes chi 256 TF32   0.210  0.185                             0.197
// The FP64 path (min_n 16: its refinement is the expensive part, and small critical
// blocks gain from a cluster, 16 modes chi 64: +26 %) sends every block from 48 up;
// the FP32 path (CTAs of 1024 threads) keeps blocks below 64 on one CTA.
// ws.big_min > 0 replaces the rule by "Gram side >= big_min" (used by the tests).
template <typename R> struct SvdRoute;
template <> struct SvdRoute<double> { static constexpr int min_n = 16, always_n = 48; };
template <> struct SvdRoute<float> { static constexpr int min_n = 64, always_n = 64; };
__device__ __forceinline__ unsigned long long svd_work(int n, int h) {
  return (unsigned long long)n * n * (unsigned long long)(n + h);
}

template <typename R> struct Prec;
// tol_* (FP32 only: the Gram seed is FP32 on both paths): two-sided Jacobi on the
// Gram matrix; os_*: one-sided refinement on W = Theta V; floor: singular values with
// s^2 <= floor * s_max^2 are dropped (the refined values are accurate to a few ulps of
// s_max, not of s_max^2).
// stop2: once the largest relative off-diagonal |w_p^dag w_q|^2 / (|w_p|^2 |w_q|^2) of a
// one-sided sweep is below stop2, the iteration stops after this sweep: it leaves
// off-diagonals of order stop2 (quadratic convergence), which perturb the singular
// values at second order and the vectors at first order.  FP64: 1e-12 (vectors to
// ~1e-12, two orders inside the 1e-10 parity bar; the whole 32-mode chi = 256 mesh
// meets the oracle to 1.2e-12 with it); FP32: 1e-10.  The criterion covers every
// pair above the column floor: a small kept column still matters, because the
// re-split divides by the neighbouring bonds' lambda.
template <> struct Prec<double> {
  typedef double2 C;
  typedef double T;  // type of the thresholds
  static constexpr double stop2 = 1e-12;
  static constexpr double os_rel = 4e-15, os_abs = 1e-30;
  static constexpr double floor = 1e-28;
};
template <> struct Prec<float> {
  typedef float2 C;
  typedef float T;
  static constexpr double stop2 = 1e-10;
  // off-diagonals below ~3 FP32 ulps of the largest diagonal are rounding noise
  static constexpr float tol_rel = 2e-7f, tol_abs = 2e-7f;
  static constexpr float os_rel = 2e-6f, os_abs = 1e-13f;
  static constexpr double floor = 1e-12;
};
// The FP64 path's refinement of cluster blocks in double-float arithmetic (dd.cuh):
// the same thresholds as FP64, vectors stored as complex double-floats.
template <> struct Prec<dd> {
  typedef ddc C;
  typedef double T;
  static constexpr double stop2 = Prec<double>::stop2;
  static constexpr double os_abs = Prec<double>::os_abs;
  static constexpr double floor = Prec<double>::floor;
};

// ---- element helpers for real (self-mirror) and complex Jacobi ----
__device__ __forceinline__ float re(float x) { return x; }
__device__ __forceinline__ float re(float2 x) { return x.x; }
__device__ __forceinline__ float absv(float x) { return fabsf(x); }
__device__ __forceinline__ float absv(float2 x) { return hypotf(x.x, x.y); }
__device__ __forceinline__ float cj(float x) { return x; }
__device__ __forceinline__ double2 cj(double2 x) { return make_double2(x.x, -x.y); }
__device__ __forceinline__ float2 cj(float2 x) { return make_float2(x.x, -x.y); }
__device__ __forceinline__ float mulv(float a, float b) { return a * b; }
__device__ __forceinline__ double2 mulv(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ float2 mulv(float2 a, float2 b) { return cmul(a, b); }
__device__ __forceinline__ float lin(float c, float x, float s, float y) { return c * x + s * y; }
__device__ __forceinline__ double2 lin(double c, double2 x, double s, double2 y) {
  return make_double2(c * x.x + s * y.x, c * x.y + s * y.y);
}
__device__ __forceinline__ float2 lin(float c, float2 x, float s, float2 y) {
  return make_float2(c * x.x + s * y.x, c * x.y + s * y.y);
}
template <typename E, typename R> __device__ __forceinline__ E divr(E g, R h);
template <> __device__ __forceinline__ float divr<float, float>(float g, float h) { return g / h; }
template <> __device__ __forceinline__ float2 divr<float2, float>(float2 g, float h) {
  return make_float2(g.x / h, g.y / h);
}
template <typename E> __device__ __forceinline__ E unit_e();
template <> __device__ __forceinline__ float unit_e<float>() { return 1.0f; }
template <> __device__ __forceinline__ double2 unit_e<double2>() { return make_double2(1.0, 0.0); }
template <> __device__ __forceinline__ float2 unit_e<float2>() { return make_float2(1.0f, 0.0f); }
template <typename E> __device__ __forceinline__ E zero_e();
template <> __device__ __forceinline__ float zero_e<float>() { return 0.0f; }
template <> __device__ __forceinline__ double2 zero_e<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 zero_e<float2>() { return make_float2(0.0f, 0.0f); }
template <typename C> __device__ __forceinline__ C cvt(double2 a);
template <> __device__ __forceinline__ double2 cvt<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 cvt<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

struct Slot {
  int* blk; int* scal; int* rowoff; int* coloff; int* rowmap; int* colmap;
  double2* fock; void* theta; void* G; void* V; double* sval; int* perm;
  double* dscal; int* order; int* items; void* W; void* NS; void* VC;
  int Pc;
  __device__ __forceinline__ int& f(int field, int t) const { return blk[field * (Pc + 1) + t]; }
};

__device__ __forceinline__ Slot get_slot(const SlotWS& ws, int s) {
  Slot sl;
  sl.Pc = ws.Pc;
  sl.blk = ws.blk + (long long)s * BF_NFIELDS * (ws.Pc + 1);
  sl.scal = ws.scal + (long long)s * SS_NFIELDS;
  sl.rowoff = ws.rowoff + (long long)s * ws.Pc * ws.P;
  sl.coloff = ws.coloff + (long long)s * ws.Pc * ws.P;
  sl.rowmap = ws.rowmap + (long long)s * ws.capRC;
  sl.colmap = ws.colmap + (long long)s * ws.capRC;
  sl.fock = ws.fock + (long long)s * MPO_FOCK_MAX;
  const long long pt = ws.poff[2 * s], pg = ws.poff[2 * s + 1];
  sl.theta = ws.theta + pt;
  sl.G = ws.G + pg;
  sl.V = ws.V + pg;
  sl.sval = ws.sval + (long long)s * ws.capCand;
  sl.perm = ws.perm + (long long)s * ws.capCand;
  sl.dscal = ws.dscal + (long long)s * 4;
  sl.order = ws.order + (long long)s * ws.capCand * 2;
  sl.items = ws.items + (long long)s * ws.P * ws.P;
  sl.W = ws.W + pt;
  sl.NS = ws.NS + pg;
  sl.VC = ws.VC + pg;
  return sl;
}

// largest t in [0, n) with pre[t] <= z  (pre non-decreasing, pre[0] = 0)
__device__ __forceinline__ int find_block(const int* pre, int n, int z) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pre[mid] <= z) lo = mid; else hi = mid;
  }
  return lo;
}

// 2-D inclusive prefix count over a (q x q) occupancy table; S has (q+1)^2 entries
__device__ __forceinline__ int box_count(const int* S, int q, int x0, int x1, int y0, int y1) {
  const int w = q + 1;
  return S[(x1 + 1) * w + (y1 + 1)] - S[x0 * w + (y1 + 1)] - S[(x1 + 1) * w + y0] + S[x0 * w + y0];
}

// ---------------------------------------------------------------- k_setup
__device__ void setup_gate(const MpoDev& st, const SlotWS& ws, const GateDesc* __restrict__ gates) {
  const int s = blockIdx.x;
  const GateDesc g = gates[s];
  Slot sl = get_slot(ws, s);
  const int ncap = st.ncap, q = ncap + 1, P = st.P, M = st.M, Pc = ws.Pc;
  const int tid = threadIdx.x, nth = blockDim.x;
  __shared__ int segA[MPO_P_MAX + 1], segC[MPO_P_MAX + 1], segB[MPO_P_MAX + 1];
  __shared__ double2 fk[MPO_FOCK_MAX];
  __shared__ int preC[(MPO_NCAP_MAX + 2) * (MPO_NCAP_MAX + 2)], preM[(MPO_NCAP_MAX + 2) * (MPO_NCAP_MAX + 2)];
  __shared__ int preA[(MPO_NCAP_MAX + 2) * (MPO_NCAP_MAX + 2)], preB[(MPO_NCAP_MAX + 2) * (MPO_NCAP_MAX + 2)];
  __shared__ int cntA[MPO_P_MAX + 1];
  __shared__ int bad;
  if (tid == 0) bad = (g.j < 0 || g.j > M - 2 || g.inst < 0 || g.inst >= st.B);
  __syncthreads();
  if (bad) {
    if (tid == 0) { sl.scal[SS_STATUS] = 1; dev_set_error(st.err, DEV_ERR_INTERNAL, 1); }
    return;
  }
  const long long bA = (long long)g.inst * (M + 1) + g.j;
  for (int p = tid; p <= P; p += nth) {
    segA[p] = st.segoff[bA * (P + 1) + p];
    segC[p] = st.segoff[(bA + 1) * (P + 1) + p];
    segB[p] = st.segoff[(bA + 2) * (P + 1) + p];
  }
  // Fock blocks U_n[i][jj] = <i, n-i| U(S) |jj, n-jj>, n = 0..ncap, by the recurrence
  const double ct = cos(g.theta), sn = sin(g.theta), cp = cos(g.phi), spp = sin(g.phi);
  const double2 S11 = make_double2(cp * ct, spp * ct), S21 = make_double2(cp * sn, spp * sn);
  const double2 S12 = make_double2(-sn, 0.0), S22 = make_double2(ct, 0.0);
  // sqrt(k) and 1/sqrt(k) for k <= ncap, once per CTA (FP64 square roots and divisions
  // are long instruction sequences on this part; the recurrence below only looks them up)
  __shared__ double sqt[MPO_NCAP_MAX + 2], isqt[MPO_NCAP_MAX + 2];
  if (tid <= ncap + 1) {
    sqt[tid] = sqrt((double)tid);
    isqt[tid] = tid > 0 ? 1.0 / sqt[tid] : 0.0;
  }
  if (tid == 0) fk[0] = make_double2(1.0, 0.0);
  __syncthreads();
  for (int n = 1; n <= ncap; ++n) {
    const int o1 = fock_off(n - 1), o = fock_off(n);
    for (int e = tid; e < (n + 1) * (n + 1); e += nth) {
      const int jj = e % (n + 1), i = e / (n + 1);
      const int src = (jj >= 1) ? jj - 1 : 0;
      const double2 al = (jj >= 1) ? S11 : S12, be = (jj >= 1) ? S21 : S22;
      double2 acc = make_double2(0.0, 0.0);
      if (i >= 1) cfma(acc, cscale(al, sqt[i]), fk[o1 + (i - 1) * n + src]);
      if (i <= n - 1) cfma(acc, cscale(be, sqt[n - i]), fk[o1 + i * n + src]);
      fk[o + i * (n + 1) + jj] = cscale(acc, isqt[(jj >= 1) ? jj : n]);
    }
    __syncthreads();
  }
  for (int e = tid; e < fock_off(ncap + 1); e += nth) sl.fock[e] = fk[e];
  // 2-D prefix counts of the pairs present at A, B and C
  if (tid == 0) {
    const int w = q + 1;
    for (int x = 0; x <= q; ++x)
      for (int y = 0; y <= q; ++y) {
        int va = 0, vb = 0, vc = 0;
        if (x > 0 && y > 0) {
          const int p = (x - 1) * q + (y - 1);
          va = segA[p + 1] > segA[p]; vb = segB[p + 1] > segB[p]; vc = segC[p + 1] > segC[p];
          va += preA[(x - 1) * w + y] + preA[x * w + y - 1] - preA[(x - 1) * w + y - 1];
          vb += preB[(x - 1) * w + y] + preB[x * w + y - 1] - preB[(x - 1) * w + y - 1];
          vc += preC[(x - 1) * w + y] + preC[x * w + y - 1] - preC[(x - 1) * w + y - 1];
        }
        preA[x * w + y] = va; preB[x * w + y] = vb; preC[x * w + y] = vc;
      }
  }
  __syncthreads();
  // per canonical block (one warp each): rows, cols, non-empty test, segment offsets.
  // The row (column) offset of pair a is the running sum of the sizes of the earlier
  // pairs a' >= m (<= m): an inclusive warp scan per group of 32 pairs plus a carry.
  {
    const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    for (int t = warp; t < Pc; t += nwarp) {
      const int m = canon_pair(t, ncap), cm = pair_c(m, ncap), cbm = pair_cb(m, ncap);
      int r = 0, c = 0;
      for (int a0 = 0; a0 < P; a0 += 32) {
        const int a = a0 + lane;
        int na = 0, nb = 0;
        if (a < P) {
          const int ca = pair_c(a, ncap), cba = pair_cb(a, ncap);
          if (ca >= cm && cba >= cbm) na = segA[a + 1] - segA[a];
          if (ca <= cm && cba <= cbm) nb = segB[a + 1] - segB[a];
        }
        int sa = na, sb = nb;  // inclusive scans
        for (int o = 1; o < 32; o <<= 1) {
          const int ua = __shfl_up_sync(0xffffffffu, sa, o), ub = __shfl_up_sync(0xffffffffu, sb, o);
          if (lane >= o) { sa += ua; sb += ub; }
        }
        if (a < P) {
          sl.rowoff[t * P + a] = na > 0 ? r + sa - na : -1;
          sl.coloff[t * P + a] = nb > 0 ? c + sb - nb : -1;
        }
        r += __shfl_sync(0xffffffffu, sa, 31);
        c += __shfl_sync(0xffffffffu, sb, 31);
      }
      // non-empty: some present c, a >= max(c, m), b <= min(c, m)
      bool path = false;
      for (int c0 = 0; c0 < P && !path; c0 += 32) {
        const int cc = c0 + lane;
        bool ok = false;
        if (cc < P && segC[cc + 1] > segC[cc]) {
          const int x = pair_c(cc, ncap), y = pair_cb(cc, ncap);
          const int hx = x > cm ? x : cm, hy = y > cbm ? y : cbm;
          const int lx = x < cm ? x : cm, ly = y < cbm ? y : cbm;
          ok = box_count(preA, q, hx, ncap, hy, ncap) > 0 && box_count(preB, q, 0, lx, 0, ly) > 0;
        }
        path = __any_sync(0xffffffffu, ok);
      }
      if (lane == 0) {
        const int gg = (r > 0 && c > 0 && path) ? (r < c ? r : c) : 0;
        sl.f(BF_M, t) = m;
        sl.f(BF_R, t) = gg ? r : 0;
        sl.f(BF_C, t) = gg ? c : 0;
        sl.f(BF_G, t) = gg;
        sl.f(BF_SIDE, t) = (r <= c) ? 0 : 1;
      }
    }
  }
  __syncthreads();
  // occupancy of non-empty canonical blocks for the item test; offsets and capacities
  if (tid == 0) {
    const int w = q + 1;
    for (int x = 0; x <= q; ++x)
      for (int y = 0; y <= q; ++y) {
        int v = 0;
        if (x > 0 && y > 0) {
          const int cx = x - 1, cy = y - 1;
          v = (cx <= cy) ? (sl.f(BF_G, canon_index(cx * q + cy, ncap)) > 0) : 0;
          v += preM[(x - 1) * w + y] + preM[x * w + y - 1] - preM[(x - 1) * w + y - 1];
        }
        preM[x * w + y] = v;
      }
    long long toff = 0, goff = 0, coff = 0, rm = 0, cm2 = 0;
    int gt = 0;
    for (int t = 0; t < Pc; ++t) {
      const int r = sl.f(BF_R, t), c = sl.f(BF_C, t), gg = sl.f(BF_G, t);
      sl.f(BF_TOFF, t) = (int)toff; sl.f(BF_GOFF, t) = (int)goff; sl.f(BF_COFF, t) = (int)coff;
      sl.f(BF_RMOFF, t) = (int)rm; sl.f(BF_CMOFF, t) = (int)cm2;
      sl.f(BF_GT, t) = gt;
      toff += (long long)r * c; goff += (long long)gg * gg; coff += gg; rm += r; cm2 += c;
      const int ntg = (gg + TILE - 1) / TILE;
      gt += ntg * (ntg + 1) / 2;
    }
    sl.f(BF_GT, Pc) = gt;
    sl.f(BF_TOFF, Pc) = (int)toff; sl.f(BF_COFF, Pc) = (int)coff; sl.f(BF_GOFF, Pc) = (int)goff;
    int status = 0;
    // Theta and Gram sizes go to the layer's pools (checked once all slots are known);
    // here only what one slot's fixed-size arrays and 32-bit offsets can hold
    if (toff > 0x7fffffffll || goff > 0x7fffffffll || coff > ws.capCand || rm > ws.capRC || cm2 > ws.capRC) {
      status = 1;
      dev_set_error(st.err, DEV_ERR_CAPACITY, 2000);
    }
    sl.scal[SS_NBLK] = Pc;
    sl.scal[SS_GTILES] = status ? 0 : gt;
    sl.scal[SS_TTILES] = 0;
    sl.scal[SS_STATUS] = status;
  }
  __syncthreads();
  if (sl.scal[SS_STATUS]) return;
  // contraction items (a, b): a >= b both present and some non-empty canonical new
  // centre m with a >= m >= b.  Items without an old centre c between a and b write
  // the zero sub-block, so every element of every Theta(m) is written each gate.
  for (int a = tid; a < P; a += nth) {
    int cnt = 0;
    if (segA[a + 1] > segA[a]) {
      const int ca = pair_c(a, ncap), cba = pair_cb(a, ncap);
      for (int b = 0; b < P; ++b) {
        if (segB[b + 1] == segB[b]) continue;
        const int cb = pair_c(b, ncap), cbb = pair_cb(b, ncap);
        if (cb > ca || cbb > cba) continue;
        if (box_count(preM, q, cb, ca, cbb, cba) > 0) ++cnt;
      }
    }
    cntA[a] = cnt;
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int a = 0; a < P; ++a) { int c = cntA[a]; cntA[a] = acc; acc += c; }
    cntA[P] = acc;
    sl.scal[SS_TTILES] = acc;
  }
  __syncthreads();
  for (int a = tid; a < P; a += nth) {
    if (segA[a + 1] == segA[a]) continue;
    int o = cntA[a];
    const int ca = pair_c(a, ncap), cba = pair_cb(a, ncap);
    for (int b = 0; b < P; ++b) {
      if (segB[b + 1] == segB[b]) continue;
      const int cb = pair_c(b, ncap), cbb = pair_cb(b, ncap);
      if (cb > ca || cbb > cba) continue;
      if (box_count(preM, q, cb, ca, cbb, cba) > 0) sl.items[o++] = a * P + b;
    }
  }
  // row / column maps: Theta(m) row i -> bond A index, column -> bond B index (one warp
  // per block, lanes over pairs)
  {
    const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    for (int t = warp; t < Pc; t += nwarp) {
      if (sl.f(BF_G, t) == 0) continue;
      int* rmap = sl.rowmap + sl.f(BF_RMOFF, t);
      int* cmap = sl.colmap + sl.f(BF_CMOFF, t);
      for (int a = lane; a < P; a += 32) {
        const int o = sl.rowoff[t * P + a];
        if (o >= 0) for (int i = segA[a]; i < segA[a + 1]; ++i) rmap[o + i - segA[a]] = i;
        const int oc = sl.coloff[t * P + a];
        if (oc >= 0) for (int i = segB[a]; i < segB[a + 1]; ++i) cmap[oc + i - segB[a]] = i;
      }
    }
  }
}

// The last CTA of k_setup to finish lays out the layer's pools: slot s's Theta-sized
// and Gram-sized regions start at the exclusive prefix sums of the slots' sizes (zero for
// a slot whose setup failed).  If the layer does not fit the pools, every slot of the
// layer is marked failed (MPO_ERR_CAPACITY), so no later kernel touches the pools.
// Then the arrival counter is reset for the next layer.
__device__ void pool_offsets(const MpoDev& st, const SlotWS& ws) {
  __shared__ int last;
  __shared__ long long part[2][256 / 32];
  __syncthreads();
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(ws.sctr, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // each thread sums a contiguous chunk of slots, then a block-wide exclusive scan
  const int S = gridDim.x, Pc = ws.Pc;
  const int chunk = (S + nth - 1) / nth, s0 = min(S, tid * chunk), s1 = min(S, s0 + chunk);
  long long nt = 0, ng = 0;
  for (int s = s0; s < s1; ++s) {
    volatile const int* scal = ws.scal + (long long)s * SS_NFIELDS;
    volatile const int* blk = ws.blk + (long long)s * BF_NFIELDS * (Pc + 1);
    if (scal[SS_STATUS] == 0) {
      nt += blk[BF_TOFF * (Pc + 1) + Pc];
      ng += blk[BF_GOFF * (Pc + 1) + Pc];
    }
  }
  long long it = nt, ig = ng;  // inclusive warp scans
  for (int o = 1; o < 32; o <<= 1) {
    const long long ut = __shfl_up_sync(0xffffffffu, it, o), ug = __shfl_up_sync(0xffffffffu, ig, o);
    if (lane >= o) { it += ut; ig += ug; }
  }
  if (lane == 31) { part[0][warp] = it; part[1][warp] = ig; }
  __syncthreads();
  long long bt = 0, bg = 0, tt = 0, tg = 0;
  for (int w = 0; w < nth / 32; ++w) {
    if (w < warp) { bt += part[0][w]; bg += part[1][w]; }
    tt += part[0][w]; tg += part[1][w];
  }
  long long t = bt + it - nt, g = bg + ig - ng;  // exclusive prefix of this chunk
  for (int s = s0; s < s1; ++s) {
    volatile const int* scal = ws.scal + (long long)s * SS_NFIELDS;
    volatile const int* blk = ws.blk + (long long)s * BF_NFIELDS * (Pc + 1);
    ws.poff[2 * s] = t;
    ws.poff[2 * s + 1] = g;
    if (scal[SS_STATUS] == 0) {
      t += blk[BF_TOFF * (Pc + 1) + Pc];
      g += blk[BF_GOFF * (Pc + 1) + Pc];
    }
  }
  __syncthreads();  // every slot's status has been read before any is overwritten
  if (tt > ws.poolTheta || tg > ws.poolGram) {
    if (tid == 0) dev_set_error(st.err, DEV_ERR_CAPACITY, 2001);
    for (int s = tid; s < S; s += nth) {
      int* scal = ws.scal + (long long)s * SS_NFIELDS;
      scal[SS_STATUS] = 1;
      scal[SS_GTILES] = 0;
      scal[SS_TTILES] = 0;
    }
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    *ws.sctr = 0;
  }
}

__global__ void __launch_bounds__(256) k_setup(MpoDev st, SlotWS ws, const GateDesc* __restrict__ gates) {
  setup_gate(st, ws, gates);
  pool_offsets(st, ws);
}

// ---------------------------------------------------------------- k_theta
// One warp per (row segment a, column segment b) item of a gate.  The warp lists
// the old centre segments c between a and b (non-empty) and the canonical new
// centres m between them whose block is non-empty (ballot compaction), then works
// through the item's na x nb entries in chunks that fit its P buffer:
//   phase 1, lanes over (c, entry):  P_c[i][j] = sum_gamma Gamma_j[a_i, gamma] lambda_C[gamma] Gamma_{j+1}[gamma, b_j]
//   phase 2, lanes over (m, entry):  Theta(m)[a_i, b_j] = lambda_A lambda_B sum_c u(a, b, c, m) P_c[i][j]
// Every P_c and every Theta entry is formed once; segments of a few indices keep
// all lanes busy because the lanes span c and m as well as the entries.
constexpr int THETA_WARPS = 8;
constexpr int THETA_PBUF = 512;  // complex P entries per warp
constexpr int THETA_EG = 4;      // entries per lane in the mixing phase

// Dynamic shared memory of k_theta (byte offsets, every section 16-byte aligned):
// Fock table | segment offsets of bonds A, C, B | 4 ints | per-warp c/m lists |
// per-warp P buffers (a large item uses all of them together).
struct ThetaSmem {
  size_t seg, misc, lists, pbuf, total;
};
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline ThetaSmem theta_smem(int ncap, size_t celem) {
  ThetaSmem L;
  L.seg = align16((size_t)fock_off(ncap + 1) * celem);
  L.misc = align16(L.seg + 3 * (size_t)(MPO_P_MAX + 1) * sizeof(int));  // 4 ints
  L.lists = L.misc + 16;
  L.pbuf = align16(L.lists + (size_t)THETA_WARPS * (2 * MPO_P_MAX + 3 * MPO_PC_MAX) * sizeof(int));
  L.total = L.pbuf + (size_t)THETA_WARPS * THETA_PBUF * celem;
  return L;
}
__host__ __device__ inline size_t theta_smem_bytes(int ncap, size_t celem) { return theta_smem(ncap, celem).total; }

constexpr int THETA_BIG = 64;  // items with at least this many entries are done by the whole CTA

// One warp lists, for the item (a, b), the old centre segments c with a >= c >= b that
// are non-empty (and their Fock columns c_a - c_c, cbar_a - cbar_c packed in cfk) and
// the canonical new centres m with a >= m >= b whose block is non-empty (with the
// item's row and column offsets inside Theta(m)); ballot compaction, warp-synchronous.
__device__ __forceinline__ void theta_lists(const Slot& sl, const int* segC, int a, int b, int ncap, int P,
                                            int lane, int* clist, int* cfk, int* mlist, int* mro, int* mco,
                                            int& nc, int& nm) {
  const int q = ncap + 1;
  const int ca = pair_c(a, ncap), cba = pair_cb(a, ncap), cb = pair_c(b, ncap), cbb = pair_cb(b, ncap);
  const int dk = ca - cb, db = cba - cbb, span = db + 1, ncand = (dk + 1) * span;
  const unsigned lt = (1u << lane) - 1u;
  nc = 0;
  nm = 0;
  for (int c0 = 0; c0 < ncand; c0 += 32) {
    const int u = c0 + lane;
    int cc = 0;
    bool ok = false;
    if (u < ncand) {
      cc = (cb + u / span) * q + (cbb + u % span);
      ok = segC[cc + 1] > segC[cc];
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const int o = nc + __popc(bal & lt);
      clist[o] = cc;
      cfk[o] = (dk - u / span) | ((db - u % span) << 16);
    }
    nc += __popc(bal);
  }
  for (int c0 = 0; c0 < ncand; c0 += 32) {
    const int u = c0 + lane;
    int t = 0;
    bool ok = false;
    if (u < ncand) {
      const int cm = cb + u / span, cbm = cbb + u % span;
      if (cm <= cbm) {
        t = canon_index(cm * q + cbm, ncap);
        ok = sl.f(BF_G, t) != 0;
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const int o = nm + __popc(bal & lt);
      mlist[o] = t;
      mro[o] = sl.rowoff[t * P + a];
      mco[o] = sl.coloff[t * P + b];
    }
    nm += __popc(bal);
  }
  __syncwarp();
}

template <typename R>
__global__ void __launch_bounds__(THETA_WARPS * 32, 2) k_theta(MpoDev st, SlotWS ws, const GateDesc* __restrict__ gates) {
  typedef typename Prec<R>::C C;
  extern __shared__ __align__(16) unsigned char tsm[];
  const int s = blockIdx.y;
  Slot sl = get_slot(ws, s);
  if (sl.scal[SS_STATUS]) return;
  const GateDesc g = gates[s];
  const int ncap = st.ncap, P = st.P, M = st.M, D = st.D;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nfk = fock_off(ncap + 1);
  const ThetaSmem TL = theta_smem(ncap, sizeof(C));
  C* fk = reinterpret_cast<C*>(tsm);
  int* segA = reinterpret_cast<int*>(tsm + TL.seg);
  int* segC = segA + (MPO_P_MAX + 1);
  int* segB = segC + (MPO_P_MAX + 1);
  int* clist = reinterpret_cast<int*>(tsm + TL.lists) + warp * (2 * MPO_P_MAX + 3 * MPO_PC_MAX);
  int* cfk = clist + MPO_P_MAX;   // per c: (c_a - c_c) | (cbar_a - cbar_c) << 16, the Fock columns
  int* mlist = cfk + MPO_P_MAX;
  int* mro = mlist + MPO_PC_MAX;
  int* mco = mro + MPO_PC_MAX;
  C* pbuf = reinterpret_cast<C*>(tsm + TL.pbuf) + warp * THETA_PBUF;
  for (int e = tid; e < nfk; e += blockDim.x) fk[e] = cvt<C>(sl.fock[e]);
  const long long bA = (long long)g.inst * (M + 1) + g.j, bC = bA + 1, bB = bA + 2;
  for (int p = tid; p <= P; p += blockDim.x) {
    segA[p] = st.segoff[bA * (P + 1) + p];
    segC[p] = st.segoff[bC * (P + 1) + p];
    segB[p] = st.segoff[bB * (P + 1) + p];
  }
  __syncthreads();
  const double* lA = st.lam + bA * D;
  const double* lC = st.lam + bC * D;
  const double* lB = st.lam + bB * D;
  const double2* G1 = st.gam + ((long long)g.inst * M + g.j) * D * D;
  const double2* G2 = G1 + (long long)D * D;
  C* Th = reinterpret_cast<C*>(sl.theta);
  const int nitems = sl.scal[SS_TTILES];
  unsigned long long flops = 0, fth = 0;  // executed two-stage form; one-stage F_Theta
  // large items: the whole CTA per item (lists in warp 0's area, the Gamma tiles in
  // the CTA's P buffers)
  int* shn = reinterpret_cast<int*>(tsm + TL.misc);  // [0] nc, [1] nm of the current large item
  C* accs = reinterpret_cast<C*>(tsm + TL.pbuf);
  // FP64 path: the large items contract in double-float arithmetic on the FP32 pipe
  // (GB300's FP64 rate is 1/61 of its FP32 rate), with the Fock table as double-floats
  // behind the two staged tiles (the P buffers are free until the small items)
  ddc* fkd = reinterpret_cast<ddc*>(accs + 2 * TILE * (TILE + 1));
  if constexpr (sizeof(R) == 8) {
    for (int e = tid; e < nfk; e += blockDim.x) fkd[e] = ddc_from(sl.fock[e].x, sl.fock[e].y);
    __syncthreads();
  }
  for (int z = blockIdx.x; z < nitems; z += gridDim.x) {
    const int item = sl.items[z];
    const int a = item / P, b = item % P;
    const int na = segA[a + 1] - segA[a], nb = segB[b + 1] - segB[b];
    if (na * nb < THETA_BIG) continue;  // CTA-uniform
    int* cl0 = reinterpret_cast<int*>(tsm + TL.lists);
    if (warp == 0) {
      int nc, nm;
      theta_lists(sl, segC, a, b, ncap, P, lane, cl0, cl0 + MPO_P_MAX, cl0 + 2 * MPO_P_MAX,
                  cl0 + 2 * MPO_P_MAX + MPO_PC_MAX, cl0 + 2 * MPO_P_MAX + 2 * MPO_PC_MAX, nc, nm);
      if (lane == 0) { shn[0] = nc; shn[1] = nm; }
    }
    __syncthreads();
    const int nc = shn[0], nm = shn[1];
    const int* ccl = cl0;
    const int* cf = cl0 + MPO_P_MAX;
    const int* ml = cl0 + 2 * MPO_P_MAX;
    const int* mr = ml + MPO_PC_MAX;
    const int* mc = mr + MPO_PC_MAX;
    const int ca = pair_c(a, ncap), cba = pair_cb(a, ncap), cb = pair_c(b, ncap), cbb = pair_cb(b, ncap);
    const int dk = ca - cb, db = cba - cbb;
    const int a0 = segA[a], b0 = segB[b], nent = na * nb;
    // 16 x 16 entry tiles, one thread per entry; for each c the Gamma tiles are staged
    // in shared memory (each element loaded once per tile) and P_c is mixed into the
    // accumulators of up to TMCH canonical m held in registers (P_c is recomputed for
    // every further group of TMCH m)
    constexpr int TMCH = sizeof(R) == 8 ? 8 : 16;
    C (*As)[TILE + 1] = reinterpret_cast<C (*)[TILE + 1]>(accs);
    C (*Bs)[TILE + 1] = reinterpret_cast<C (*)[TILE + 1]>(accs + TILE * (TILE + 1));
    const int tx = tid & 15, ty = tid >> 4;
    if constexpr (sizeof(R) == 8) {
      // the same tiles in double-float: Gamma converted once per staged element, each
      // k-tile's products summed by four compensated accumulators of at most 16 terms
      // (Dot2), the weights u(a, b, c, m) and the mixing in double-float
      ddc (*Ad)[TILE + 1] = reinterpret_cast<ddc (*)[TILE + 1]>(accs);
      ddc (*Bd)[TILE + 1] = reinterpret_cast<ddc (*)[TILE + 1]>(accs + TILE * (TILE + 1));
      for (int mc0 = 0; mc0 < nm; mc0 += TMCH) {
        const int nq = (nm - mc0) < TMCH ? (nm - mc0) : TMCH;
        for (int i0 = 0; i0 < na; i0 += TILE)
          for (int j0 = 0; j0 < nb; j0 += TILE) {
            const int i = i0 + ty, jc = j0 + tx;
            const bool valid = (i < na) && (jc < nb);
            ddc acc[TMCH];
#pragma unroll
            for (int k = 0; k < TMCH; ++k) acc[k] = ddc_zero();
            for (int ci = 0; ci < nc; ++ci) {
              const int cc = ccl[ci], f = cf[ci];
              const int k0 = segC[cc], k1 = segC[cc + 1];
              ddc part = ddc_zero();
              for (int kb = k0; kb < k1; kb += TILE) {
                const int kn = (k1 - kb) < TILE ? (k1 - kb) : TILE;
                if (i0 + ty < na && tx < kn) {
                  const double2 v = G1[(long long)(a0 + i0 + ty) * D + kb + tx];
                  Ad[ty][tx] = ddc_from(v.x, v.y);
                } else {
                  Ad[ty][tx] = ddc_zero();
                }
                if (ty < kn && j0 + tx < nb) {
                  const double2 v = cscale(G2[(long long)(kb + ty) * D + b0 + j0 + tx], lC[kb + ty]);
                  Bd[ty][tx] = ddc_from(v.x, v.y);
                } else {
                  Bd[ty][tx] = ddc_zero();
                }
                __syncthreads();
                if (valid) {
                  dd_acc rr = dd_acc_zero(), ii = dd_acc_zero(), ri = dd_acc_zero(), ir = dd_acc_zero();
                  for (int kk = 0; kk < kn; ++kk) {
                    const ddc x = Ad[ty][kk], y = Bd[kk][tx];
                    dd_acc_mac(rr, x.re, y.re);
                    dd_acc_mac(ii, x.im, y.im);
                    dd_acc_mac(ri, x.re, y.im);
                    dd_acc_mac(ir, x.im, y.re);
                  }
                  part = ddc_add(part, ddc_make(dd_sub(dd_acc_value(rr), dd_acc_value(ii)),
                                                dd_add(dd_acc_value(ri), dd_acc_value(ir))));
                }
                __syncthreads();
              }
              if (valid) {
#pragma unroll
                for (int k = 0; k < TMCH; ++k) {
                  if (k < nq) {
                    const int m = sl.f(BF_M, ml[mc0 + k]);
                    const ddc w = ddc_mul(fkd[fock_off(dk) + (ca - pair_c(m, ncap)) * (dk + 1) + (f & 0xffff)],
                                          ddc_conj(fkd[fock_off(db) + (cba - pair_cb(m, ncap)) * (db + 1) + (f >> 16)]));
                    acc[k] = ddc_add(acc[k], ddc_mul(w, part));
                  }
                }
              }
            }
            if (valid) {
              const double sc = lA[a0 + i] * lB[b0 + jc];
#pragma unroll
              for (int k = 0; k < TMCH; ++k) {
                if (k < nq) {
                  const int t = ml[mc0 + k];
                  const double2 v = make_double2(dd_to(acc[k].re), dd_to(acc[k].im));
                  Th[sl.f(BF_TOFF, t) + (long long)(mr[mc0 + k] + i) * sl.f(BF_C, t) + (mc[mc0 + k] + jc)] =
                      cvt<C>(cscale(v, sc));
                }
              }
            }
          }
      }
    } else
    for (int mc0 = 0; mc0 < nm; mc0 += TMCH) {
      const int nq = (nm - mc0) < TMCH ? (nm - mc0) : TMCH;
      for (int i0 = 0; i0 < na; i0 += TILE)
        for (int j0 = 0; j0 < nb; j0 += TILE) {
          const int i = i0 + ty, jc = j0 + tx;
          const bool valid = (i < na) && (jc < nb);
          C acc[TMCH];
#pragma unroll
          for (int k = 0; k < TMCH; ++k) acc[k] = zero_e<C>();
          for (int ci = 0; ci < nc; ++ci) {
            const int cc = ccl[ci], f = cf[ci];
            const int k0 = segC[cc], k1 = segC[cc + 1];
            C part = zero_e<C>();
            for (int kb = k0; kb < k1; kb += TILE) {
              const int kn = (k1 - kb) < TILE ? (k1 - kb) : TILE;
              As[ty][tx] = (i0 + ty < na && tx < kn) ? cvt<C>(G1[(long long)(a0 + i0 + ty) * D + kb + tx]) : zero_e<C>();
              Bs[ty][tx] = (ty < kn && j0 + tx < nb)
                               ? cvt<C>(cscale(G2[(long long)(kb + ty) * D + b0 + j0 + tx], lC[kb + ty]))
                               : zero_e<C>();
              __syncthreads();
              if (valid)
                for (int kk = 0; kk < kn; ++kk) cfma(part, As[ty][kk], Bs[kk][tx]);
              __syncthreads();
            }
            if (valid) {
#pragma unroll
              for (int k = 0; k < TMCH; ++k) {
                if (k < nq) {
                  const int m = sl.f(BF_M, ml[mc0 + k]);
                  const C w = cmul(fk[fock_off(dk) + (ca - pair_c(m, ncap)) * (dk + 1) + (f & 0xffff)],
                                   cj(fk[fock_off(db) + (cba - pair_cb(m, ncap)) * (db + 1) + (f >> 16)]));
                  cfma(acc[k], w, part);
                }
              }
            }
          }
          if (valid) {
            const R sc = (R)(lA[a0 + i] * lB[b0 + jc]);
#pragma unroll
            for (int k = 0; k < TMCH; ++k) {
              if (k < nq) {
                const int t = ml[mc0 + k];
                Th[sl.f(BF_TOFF, t) + (long long)(mr[mc0 + k] + i) * sl.f(BF_C, t) + (mc[mc0 + k] + jc)] =
                    cscale(acc[k], sc);
              }
            }
          }
        }
    }
    if (st.ctr && tid == 0) {
      unsigned long long kc = 0;
      for (int ci = 0; ci < nc; ++ci) kc += (unsigned long long)(segC[ccl[ci] + 1] - segC[ccl[ci]]);
      flops += 8ull * (unsigned long long)nent * (kc + (unsigned long long)nc * nm);
      fth += 8ull * (unsigned long long)nent * kc * (unsigned long long)nm;
    }
    __syncthreads();  // lists and accumulators are reused by the next item
  }
  // small items: one warp per item
  for (int z = blockIdx.x * THETA_WARPS + warp; z < nitems; z += gridDim.x * THETA_WARPS) {
    const int item = sl.items[z];
    const int a = item / P, b = item % P;
    const int na = segA[a + 1] - segA[a], nb = segB[b + 1] - segB[b];
    if (na * nb >= THETA_BIG) continue;  // warp-uniform
    const int ca = pair_c(a, ncap), cba = pair_cb(a, ncap), cb = pair_c(b, ncap), cbb = pair_cb(b, ncap);
    const int dk = ca - cb, db = cba - cbb;
    int nc, nm;
    theta_lists(sl, segC, a, b, ncap, P, lane, clist, cfk, mlist, mro, mco, nc, nm);
    if (nm == 0) continue;  // (with no c between, the entries are written as zeros below)
    const int a0 = segA[a], b0 = segB[b];
    const int nent = na * nb;
    const int E = nc > 0 ? THETA_PBUF / nc : THETA_PBUF;  // entries per chunk (nc <= P_MAX = THETA_PBUF)
    for (int e0 = 0; e0 < nent; e0 += E) {
      const int En = (nent - e0) < E ? (nent - e0) : E;
      for (int u = lane; u < nc * En; u += 32) {
        const int ci = u / En, el = u % En, e = e0 + el, i = e / nb, j = e % nb;
        const int cc = clist[ci];
        const double2* g1 = G1 + (long long)(a0 + i) * D;
        const double2* g2 = G2 + b0 + j;
        C acc = zero_e<C>();
        for (int k = segC[cc]; k < segC[cc + 1]; ++k)
          cfma(acc, cvt<C>(g1[k]), cvt<C>(cscale(g2[(long long)k * D], lC[k])));
        pbuf[ci * En + el] = acc;
      }
      __syncwarp();
      // lanes over (m, group of THETA_EG entries): the weight u(a, b, c, m) is formed
      // once per c and applied to the group's entries
      const int ng = (En + THETA_EG - 1) / THETA_EG;
      for (int u = lane; u < nm * ng; u += 32) {
        const int mi = u / ng, el0 = (u % ng) * THETA_EG;
        const int t = mlist[mi];
        const int m = sl.f(BF_M, t);
        const C* fu = fk + fock_off(dk) + (ca - pair_c(m, ncap)) * (dk + 1);
        const C* fb = fk + fock_off(db) + (cba - pair_cb(m, ncap)) * (db + 1);
        C acc[THETA_EG];
#pragma unroll
        for (int x = 0; x < THETA_EG; ++x) acc[x] = zero_e<C>();
        const int ne = (En - el0) < THETA_EG ? (En - el0) : THETA_EG;
        for (int ci = 0; ci < nc; ++ci) {
          const int f = cfk[ci];
          const C w = cmul(fu[f & 0xffff], cj(fb[f >> 16]));
          const C* pc = pbuf + ci * En + el0;
#pragma unroll
          for (int x = 0; x < THETA_EG; ++x)
            if (x < ne) cfma(acc[x], w, pc[x]);
        }
        const long long tb = sl.f(BF_TOFF, t), ccols = sl.f(BF_C, t);
#pragma unroll
        for (int x = 0; x < THETA_EG; ++x) {
          if (x < ne) {
            const int e = e0 + el0 + x, i = e / nb, j = e % nb;
            const R sc = (R)(lA[a0 + i] * lB[b0 + j]);
            Th[tb + (long long)(mro[mi] + i) * ccols + (mco[mi] + j)] = cscale(acc[x], sc);
          }
        }
      }
      __syncwarp();
    }
    if (st.ctr && lane == 0) {
      unsigned long long kc = 0;
      for (int ci = 0; ci < nc; ++ci) kc += (unsigned long long)(segC[clist[ci] + 1] - segC[clist[ci]]);
      flops += 8ull * (unsigned long long)nent * (kc + (unsigned long long)nc * nm);
      fth += 8ull * (unsigned long long)nent * kc * (unsigned long long)nm;
    }
  }
  if (st.ctr && lane == 0 && flops) atomicAdd(st.ctr + CTR_THETA, flops);
  if (st.ctr && lane == 0 && fth) atomicAdd(st.ctr + CTR_FTHETA, fth);
}

// ---------------------------------------------------------------- k_theta_tc
// Eq. `theta` on the tensor cores (tcgen05, see tc.cuh), for the TF32 and BF16 paths.
// A work item is (canonical block m, a tile of 128 rows of Theta(m), one column
// segment b of Theta(m), up to 64 of its columns).  For fixed m and b the weight
// u(a, b, c, m) of a row alpha (charge a) and a centre index gamma (charge c) is a
// function of (a, c) alone, so it is folded into the A operand while staging:
//   A[alpha, gamma] = u(a, b, c, m) Gamma_j[alpha, gamma]      (0 unless a >= c >= b)
//   B[beta, gamma]  = lambda_C[gamma] Gamma_{j+1}[gamma, beta]
//   Theta(m)[alpha, beta] = lambda_A[alpha] lambda_B[beta] sum_gamma A B  (epilogue)
// K runs over the centre indices whose charge dominates b (a gathered list of
// segments; per stage, a table of the 32 indices' bond positions and charges).  Each
// item writes every entry of its region of Theta(m), zeros included.  This is the
// one-stage form of Eq. `theta` (flops F_Theta, counted per row over the c between
// a and b); the FP64 path keeps the SIMT two-stage kernel.
constexpr int THETA_TN = 64;
// Dynamic shared memory of k_theta_tc (byte offsets; the Fock table is sized for the
// handle's n_cap).  At least 80 KB, so that at most two CTAs share an SM (two TMEM
// allocations of 256 columns); up to n_cap = 12 it stays within 113 KB, so that two do.
struct ThetaTcSmem {
  size_t fk, seg, bpre, clist, cpre, rinfo, kinfo, misc, rlam, clam, total;
};
template <int MODE>
__host__ __device__ inline ThetaTcSmem theta_tc_smem(int ncap) {
  ThetaTcSmem L;
  const size_t stage = tc::CTile<MODE>::stage_bytes(THETA_TN);
  L.fk = (stage + 1023) & ~(size_t)1023;
  L.seg = align16(L.fk + (size_t)fock_off(ncap + 1) * sizeof(float2));
  L.bpre = L.seg + 3 * (size_t)(MPO_P_MAX + 1) * sizeof(int);
  L.clist = L.bpre + (size_t)(MPO_PC_MAX + 1) * sizeof(int);
  L.cpre = L.clist + (size_t)MPO_P_MAX * sizeof(int);
  L.rinfo = align16(L.cpre + (size_t)(MPO_P_MAX + 1) * sizeof(int));
  L.kinfo = L.rinfo + 128 * sizeof(int4);
  L.misc = L.kinfo + 32 * sizeof(int4);
  L.rlam = L.misc + 64;                   // lambda_A of the tile's rows (FP32)
  L.clam = L.rlam + 128 * sizeof(float);  // lambda_B of the item's columns (FP32)
  const size_t used = L.clam + THETA_TN * sizeof(float);
  L.total = used > 80 * 1024 ? used : 80 * 1024;
  return L;
}

// Number of column tiles of segment width nb (tiles of up to THETA_TN columns).
__device__ __forceinline__ int theta_ntiles(int nb) { return (nb + THETA_TN - 1) / THETA_TN; }

template <int MODE>
__global__ void __launch_bounds__(256) k_theta_tc(MpoDev st, SlotWS ws, const GateDesc* __restrict__ gates) {
  extern __shared__ __align__(1024) unsigned char ttsm[];
  const ThetaTcSmem L = theta_tc_smem<MODE>(st.ncap);
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int s = blockIdx.y;
  Slot sl = get_slot(ws, s);
  if (sl.scal[SS_STATUS]) return;
  const GateDesc g = gates[s];
  const int ncap = st.ncap, P = st.P, M = st.M, D = st.D, Pc = ws.Pc;
  const int tid = threadIdx.x;
  float2* fk = reinterpret_cast<float2*>(ttsm + L.fk);
  int* segA = reinterpret_cast<int*>(ttsm + L.seg);
  int* segC = segA + (MPO_P_MAX + 1);
  int* segB = segC + (MPO_P_MAX + 1);
  int* bpre = reinterpret_cast<int*>(ttsm + L.bpre);
  int* clist = reinterpret_cast<int*>(ttsm + L.clist);
  int* cpre = reinterpret_cast<int*>(ttsm + L.cpre);
  int4* rinfo = reinterpret_cast<int4*>(ttsm + L.rinfo);
  int4* kinfo = reinterpret_cast<int4*>(ttsm + L.kinfo);
  int* misc = reinterpret_cast<int*>(ttsm + L.misc);
  // lambda factors in FP32, formed once per row, column and centre index: an FP64
  // multiply or conversion per staged element would keep the FP64 pipe busy
  float* rlam = reinterpret_cast<float*>(ttsm + L.rlam);
  float* clam = reinterpret_cast<float*>(ttsm + L.clam);
  const long long bA = (long long)g.inst * (M + 1) + g.j, bC = bA + 1, bB = bA + 2;
  for (int p = tid; p <= P; p += blockDim.x) {
    segA[p] = st.segoff[bA * (P + 1) + p];
    segC[p] = st.segoff[bC * (P + 1) + p];
    segB[p] = st.segoff[bB * (P + 1) + p];
  }
  for (int e = tid; e < fock_off(ncap + 1); e += blockDim.x) fk[e] = cvt<float2>(sl.fock[e]);
  __syncthreads();
  // items per block: row tiles x (column tiles over the block's column segments)
  for (int t = tid; t < Pc; t += blockDim.x) {
    int n = 0;
    if (sl.f(BF_G, t) > 0) {
      int ct = 0;
      for (int b = 0; b < P; ++b)
        if (sl.coloff[t * P + b] >= 0) ct += theta_ntiles(segB[b + 1] - segB[b]);
      n = ((sl.f(BF_R, t) + 127) / 128) * ct;
    }
    bpre[t + 1] = n;
  }
  if (tid == 0) bpre[0] = 0;
  __syncthreads();
  if (tid == 0)
    for (int t = 0; t < Pc; ++t) bpre[t + 1] += bpre[t];
  __syncthreads();
  const int nitems = bpre[Pc];
  if ((int)blockIdx.x >= nitems) return;  // CTA-uniform, before any TMEM is held
  constexpr uint32_t NCOL = tc::CTile<MODE>::tmem_cols(THETA_TN);
  if (tid < 32) tc::tmem_alloc(&tslot, NCOL);
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  tc::Engine E{tslot, &bar, 0u, st.err};
  const double* lA = st.lam + bA * D;
  const double* lC = st.lam + bC * D;
  const double* lB = st.lam + bB * D;
  const int* chA = st.charge + bA * D;
  const double2* G1 = st.gam + ((long long)g.inst * M + g.j) * D * D;
  const double2* G2 = G1 + (long long)D * D;
  float2* Th = reinterpret_cast<float2*>(sl.theta);
  unsigned long long flops = 0;
  for (int z = blockIdx.x; z < nitems; z += gridDim.x) {
    const int t = find_block(bpre, Pc + 1, z);
    int rem = z - bpre[t];
    const int m = sl.f(BF_M, t), cm = pair_c(m, ncap), cbm = pair_cb(m, ncap);
    const int R = sl.f(BF_R, t), Ccols = sl.f(BF_C, t);
    int ct = 0;
    for (int b = 0; b < P; ++b)
      if (sl.coloff[t * P + b] >= 0) ct += theta_ntiles(segB[b + 1] - segB[b]);
    const int ti = rem / ct;
    rem -= ti * ct;
    int b = 0;
    for (; b < P; ++b) {
      if (sl.coloff[t * P + b] < 0) continue;
      const int nt = theta_ntiles(segB[b + 1] - segB[b]);
      if (rem < nt) break;
      rem -= nt;
    }
    const int cb = pair_c(b, ncap), cbb = pair_cb(b, ncap);
    const int n0 = rem * THETA_TN, nbt = min(THETA_TN, segB[b + 1] - segB[b] - n0);
    const int beta0 = segB[b] + n0, col0 = sl.coloff[t * P + b] + n0, r0 = ti * 128;
    // centre segments c >= b (the K list) and their prefix
    if (tid == 0) {
      int nc = 0, kk = 0;
      for (int cc = 0; cc < P; ++cc) {
        if (segC[cc + 1] == segC[cc]) continue;
        if (pair_c(cc, ncap) < cb || pair_cb(cc, ncap) < cbb) continue;
        clist[nc] = cc;
        cpre[nc] = kk;
        kk += segC[cc + 1] - segC[cc];
        ++nc;
      }
      cpre[nc] = kk;
      misc[0] = nc;
    }
    // rows: bond-A index, charges of a and the Fock row offsets of the weight
    if (tid < 128) {
      const int r = r0 + tid;
      int4 ri = make_int4(-1, 0, 0, 0);
      if (r < R) {
        const int alpha = sl.rowmap[sl.f(BF_RMOFF, t) + r];
        const int pa = chA[alpha], ca = pair_c(pa, ncap), cba = pair_cb(pa, ncap);
        const int dk = ca - cb, db = cba - cbb;
        ri.x = alpha;
        ri.y = ca | (cba << 8);
        ri.z = fock_off(dk) + (ca - cm) * (dk + 1) + ca;    // + (-c_c): U_dk[ca - cm, ca - c_c]
        ri.w = fock_off(db) + (cba - cbm) * (db + 1) + cba;  // + (-cbar_c)
      }
      rinfo[tid] = ri;
      rlam[tid] = ri.x >= 0 ? (float)lA[ri.x] : 0.f;
    }
    if (tid < THETA_TN) clam[tid] = tid < nbt ? (float)lB[beta0 + tid] : 0.f;
    __syncthreads();
    const int nc = misc[0], K = cpre[nc];
    if (st.ctr && tid < 128 && rinfo[tid].x >= 0) {  // F_Theta of this row: c between a and b
      const int ca = rinfo[tid].y & 0xff, cba = rinfo[tid].y >> 8;
      unsigned long long kk = 0;
      for (int ci = 0; ci < nc; ++ci)
        if (pair_c(clist[ci], ncap) <= ca && pair_cb(clist[ci], ncap) <= cba) kk += cpre[ci + 1] - cpre[ci];
      flops += 8ull * kk * (unsigned long long)nbt;
    }
    auto prep = [&](int k0) -> bool {
      if (tid < 32) {
        const int k = k0 + tid;
        int4 ki = make_int4(-1, 0, 0, 0);
        if (k < K) {
          const int ci = find_block(cpre, nc + 1, k);
          const int cc = clist[ci];
          ki.x = segC[cc] + (k - cpre[ci]);
          ki.y = pair_c(cc, ncap);
          ki.z = pair_cb(cc, ncap);
          ki.w = __float_as_int((float)lC[ki.x]);
        }
        kinfo[tid] = ki;
      }
      return true;
    };
    auto lda = [&](int i, int k) -> float2 {
      const int4 ri = rinfo[i];
      const int4 ki = kinfo[k & 31];
      if (ri.x < 0 || ki.x < 0) return make_float2(0.f, 0.f);
      const int ca = ri.y & 0xff, cba = ri.y >> 8;
      if (ki.y > ca || ki.z > cba) return make_float2(0.f, 0.f);
      const float2 w = cmul(fk[ri.z - ki.y], cj(fk[ri.w - ki.z]));
      const double2 gv = G1[(long long)ri.x * D + ki.x];
      return cmul(w, make_float2((float)gv.x, (float)gv.y));
    };
    auto ldb = [&](int j, int k) -> float2 {
      const int4 ki = kinfo[k & 31];
      if (j >= nbt || ki.x < 0) return make_float2(0.f, 0.f);
      const double2 gv = G2[(long long)ki.x * D + beta0 + j];
      const float l = __int_as_float(ki.w);
      return make_float2((float)gv.x * l, (float)gv.y * l);
    };
    auto sto = [&](int i, int j, float re, float im) {
      if (r0 + i >= R || j >= nbt) return;
      const float sc = rlam[i] * clam[j];
      Th[sl.f(BF_TOFF, t) + (long long)(r0 + i) * Ccols + col0 + j] = make_float2(re * sc, im * sc);
    };
    bool ok;
    if (nbt <= 32) ok = tc::tile_gemm<MODE, 32>(E, ttsm, K, lda, ldb, sto, prep);
    else ok = tc::tile_gemm<MODE, THETA_TN>(E, ttsm, K, lda, ldb, sto, prep);
    if (!ok) break;
  }
  tc::fence_before();
  __syncthreads();
  if (tid < 32) tc::tmem_dealloc(tslot, NCOL);
  if (st.ctr && flops) {
    atomicAdd(st.ctr + CTR_THETA, flops);
    atomicAdd(st.ctr + CTR_FTHETA, flops);
  }
}

// ---------------------------------------------------------------- k_gram
// Upper-triangular 16 x 16 tiles of G = Theta Theta^dag (side 0) or Theta^dag Theta,
// in FP32: the Gram eigenvectors only seed the one-sided refinement (k_refine),
// which iterates to the accuracy of the path's own precision from any complete basis.
template <typename RT>
__global__ void __launch_bounds__(256) k_gram(SlotWS ws, unsigned long long* ctr, int tc_min) {
  typedef typename Prec<RT>::C CT;
  typedef float2 C;
  const int s = blockIdx.y;
  Slot sl = get_slot(ws, s);
  if (sl.scal[SS_STATUS]) return;
  const int Pc = ws.Pc;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  __shared__ C As[TILE][TILE + 1], Bs[TILE][TILE + 1];
  __shared__ int gpre[MPO_PC_MAX + 1];
  for (int t = threadIdx.x; t <= Pc; t += blockDim.x) gpre[t] = sl.f(BF_GT, t);
  __syncthreads();
  const CT* ThAll = reinterpret_cast<const CT*>(sl.theta);
  C* GAll = reinterpret_cast<C*>(sl.G);
  const int total = sl.scal[SS_GTILES];
  unsigned long long flops = 0;
  for (int z = blockIdx.x; z < total; z += gridDim.x) {
    const int t = find_block(gpre, Pc + 1, z);
    const int r = sl.f(BF_R, t), c = sl.f(BF_C, t), gg = sl.f(BF_G, t), side = sl.f(BF_SIDE, t);
    if (gg >= tc_min) continue;  // on the tensor cores (k_gram_tc); CTA-uniform
    const CT* Th = ThAll + sl.f(BF_TOFF, t);
    C* Gm = GAll + sl.f(BF_GOFF, t);
    const int nt = (gg + TILE - 1) / TILE;
    int rem = z - gpre[t], ti = 0;
    while (rem >= nt - ti) { rem -= nt - ti; ++ti; }
    const int tj = ti + rem;
    const int K = side == 0 ? c : r;
    C acc = zero_e<C>();
    for (int k0 = 0; k0 < K; k0 += TILE) {
      __syncthreads();
      if (side == 0) {
        int ia = ti * TILE + ty, ib = tj * TILE + ty, kk = k0 + tx;
        As[ty][tx] = (ia < gg && kk < K) ? cvt<C>(to_d2(Th[(long long)ia * c + kk])) : zero_e<C>();
        Bs[ty][tx] = (ib < gg && kk < K) ? cvt<C>(to_d2(Th[(long long)ib * c + kk])) : zero_e<C>();
      } else {
        int kr = k0 + ty, ja = ti * TILE + tx, jb = tj * TILE + tx;
        As[ty][tx] = (kr < K && ja < gg) ? cvt<C>(to_d2(Th[(long long)kr * c + ja])) : zero_e<C>();
        Bs[ty][tx] = (kr < K && jb < gg) ? cvt<C>(to_d2(Th[(long long)kr * c + jb])) : zero_e<C>();
      }
      __syncthreads();
      const int kn = (K - k0) < TILE ? (K - k0) : TILE;
      if (side == 0) {
        for (int kk = 0; kk < kn; ++kk) cfma_cj(acc, Bs[tx][kk], As[ty][kk]);
      } else {
        for (int kk = 0; kk < kn; ++kk) cfma_cj(acc, As[kk][ty], Bs[kk][tx]);
      }
    }
    const int gi = ti * TILE + ty, gj = tj * TILE + tx;
    if (gi < gg && gj < gg && (ti < tj || ty <= tx)) flops += 8ull * (unsigned long long)K;
    if (gi < gg && gj < gg) {
      if (ti < tj || ty < tx) {
        Gm[(long long)gi * gg + gj] = acc;
        Gm[(long long)gj * gg + gi] = cj(acc);
      } else if (ty == tx) {
        C d = acc;
        d.y = 0;
        Gm[(long long)gi * gg + gi] = d;
      }
    }
  }
  if (ctr) {
    flops = __reduce_add_sync(0xffffffffu, (unsigned)flops);
    if ((threadIdx.x & 31) == 0 && flops) atomicAdd(ctr + CTR_GRAM, flops);
  }
}

// ---------------------------------------------------------------- k_gram_tc
// The Gram matrices of the larger blocks on the tensor cores (tcgen05, see tc.cuh):
// G = Theta Theta^dag (side 0) or Theta^dag Theta (side 1) in output tiles of 128 x 64
// complex entries; only tiles holding entries with i <= j are computed, and every
// such entry is written to G[i][j] and, conjugated, to G[j][i] (the diagonal real).
// Products in 3xTF32 (FP32-level accuracy), FP32 accumulation.  Blocks with a Gram side below tc_min stay on
// k_gram.  One TMEM allocation of 256 columns per CTA (at most two CTAs per SM).
constexpr int GRAM_TN = 64;
constexpr int GRAM_TC_MIN = 48;
template <int MODE>
__host__ __device__ constexpr size_t gram_tc_smem() {
  return tc::CTile<MODE>::stage_bytes(GRAM_TN) > 80 * 1024 ? tc::CTile<MODE>::stage_bytes(GRAM_TN) : 80 * 1024;
}

// Output tiles of a block of Gram side gg: 128-row tiles ti, 64-column tiles tj with
// a column at or right of the tile's first row.
__device__ __forceinline__ int gram_tc_tiles(int gg) {
  const int ntr = (gg + 127) / 128, ntc = (gg + GRAM_TN - 1) / GRAM_TN;
  int n = 0;
  for (int ti = 0; ti < ntr; ++ti) n += ntc - (128 * ti) / GRAM_TN;
  return n;
}

template <typename RT, int MODE>
__global__ void __launch_bounds__(256) k_gram_tc(SlotWS ws, unsigned long long* ctr, int* err, int tc_min) {
  typedef typename Prec<RT>::C CT;
  extern __shared__ __align__(1024) unsigned char gsm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int s = blockIdx.y;
  Slot sl = get_slot(ws, s);
  if (sl.scal[SS_STATUS]) return;
  const int Pc = ws.Pc;
  int nitems = 0;
  for (int t = 0; t < Pc; ++t) {
    const int gg = sl.f(BF_G, t);
    if (gg >= tc_min) nitems += gram_tc_tiles(gg);
  }
  if ((int)blockIdx.x >= nitems) return;  // CTA-uniform, before any TMEM is held
  const int tid = threadIdx.x;
  constexpr uint32_t NCOL = tc::CTile<MODE>::tmem_cols(GRAM_TN);
  if (tid < 32) tc::tmem_alloc(&tslot, NCOL);
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  tc::Engine E{tslot, &bar, 0u, err};
  const CT* ThAll = reinterpret_cast<const CT*>(sl.theta);
  float2* GAll = reinterpret_cast<float2*>(sl.G);
  unsigned long long flops = 0;
  for (int z = blockIdx.x; z < nitems; z += gridDim.x) {
    int rem = z, t = 0, ti = 0, tj = 0;
    for (t = 0; t < Pc; ++t) {
      const int gg = sl.f(BF_G, t);
      if (gg < tc_min) continue;
      const int n = gram_tc_tiles(gg);
      if (rem < n) break;
      rem -= n;
    }
    const int gg = sl.f(BF_G, t), c = sl.f(BF_C, t), r = sl.f(BF_R, t), side = sl.f(BF_SIDE, t);
    {
      const int ntc = (gg + GRAM_TN - 1) / GRAM_TN;
      while (rem >= ntc - (128 * ti) / GRAM_TN) { rem -= ntc - (128 * ti) / GRAM_TN; ++ti; }
      tj = (128 * ti) / GRAM_TN + rem;
    }
    const int i0 = 128 * ti, j0 = GRAM_TN * tj, K = side == 0 ? c : r;
    const CT* Th = ThAll + sl.f(BF_TOFF, t);
    float2* Gm = GAll + sl.f(BF_GOFF, t);
    auto lda = [&](int i, int k) -> float2 {
      const int gi = i0 + i;
      if (gi >= gg || k >= K) return make_float2(0.f, 0.f);
      const float2 v = cvt<float2>(to_d2(side == 0 ? Th[(long long)gi * c + k] : Th[(long long)k * c + gi]));
      return side == 0 ? v : make_float2(v.x, -v.y);
    };
    auto ldb = [&](int j, int k) -> float2 {
      const int gj = j0 + j;
      if (gj >= gg || k >= K) return make_float2(0.f, 0.f);
      const float2 v = cvt<float2>(to_d2(side == 0 ? Th[(long long)gj * c + k] : Th[(long long)k * c + gj]));
      return side == 0 ? make_float2(v.x, -v.y) : v;
    };
    auto st = [&](int i, int j, float re, float im) {
      const int gi = i0 + i, gj = j0 + j;
      if (gi >= gg || gj >= gg || gi > gj) return;
      if (gi == gj) {
        Gm[(long long)gi * gg + gi] = make_float2(re, 0.f);
      } else {
        Gm[(long long)gi * gg + gj] = make_float2(re, im);
        Gm[(long long)gj * gg + gi] = make_float2(re, -im);
      }
    };
    if (!tc::tile_gemm<MODE, GRAM_TN>(E, gsm, K, lda, ldb, st)) break;
    if (ctr && tid == 0) {
      for (int i = i0; i < i0 + 128 && i < gg; ++i) {
        const int jlo = i > j0 ? i : j0, jhi = (j0 + GRAM_TN < gg ? j0 + GRAM_TN : gg);
        if (jhi > jlo) flops += 8ull * (unsigned long long)K * (unsigned long long)(jhi - jlo);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (tid < 32) tc::tmem_dealloc(tslot, NCOL);
  if (ctr && tid == 0 && flops) atomicAdd(ctr + CTR_GRAM, flops);
}

// ---------------------------------------------------------------- Jacobi core
// Cyclic Jacobi with the round-robin (circle) pairing: n/2 disjoint rotations per
// round, n-1 rounds per sweep.  For the pair (p, q) with g = G_pq = |g| e:
// D = diag(1, conj(e)) makes the 2x2 block real, the real rotation
// R = [[c, s], [-s, c]] with t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// tau = (G_qq - G_pp) / (2|g|) annihilates it, and J = D R is applied as
// G <- J^dag G J, V <- V J.  E = R for real symmetric, E = complex for Hermitian.
// The pairs of a round are disjoint, so a round is processed in chunks of at most
// PAIR_CHUNK pairs: a chunk's 2x2 sub-blocks are untouched by the other chunks.
template <typename R, typename E> struct Rot { int p, q; R c, s; E e; };
constexpr int PAIR_CHUNK = 256;

__device__ __forceinline__ void circle_pair(int rnd, int k, int np, int& p, int& q) {
  if (k == 0) { p = rnd; q = np - 1; }
  else { p = (rnd + k) % (np - 1); q = (rnd - k + np - 1) % (np - 1); }
  if (p > q) { const int t = p; p = q; q = t; }
}

template <typename R, typename E>
__device__ int jacobi(E* A, E* V, int n, Rot<R, E>* rot, int* flags, R tol_rel, R tol_abs_rel) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int np = n + (n & 1), half = np / 2;
  for (int e = tid; e < n * n; e += nth) V[e] = ((e / n) == (e % n)) ? unit_e<E>() : zero_e<E>();
  __syncthreads();
  R dm = 0;
  for (int i = 0; i < n; ++i) dm = fmax(dm, absv(re(A[(long long)i * n + i])));  // every thread
  const R tol_abs = tol_abs_rel * dm;
  int sweep = 0;
  for (; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
    __syncthreads();  // every thread has read flags[0] of the previous sweep
    if (tid == 0) flags[0] = 0;
    __syncthreads();
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int c0 = 0; c0 < half; c0 += PAIR_CHUNK) {
        const int cn = (half - c0) < PAIR_CHUNK ? (half - c0) : PAIR_CHUNK;
        for (int k = tid; k < cn; k += nth) {
          int p, qq;
          circle_pair(rnd, c0 + k, np, p, qq);
          Rot<R, E> rp;
          rp.p = p; rp.q = -1; rp.c = 1; rp.s = 0; rp.e = unit_e<E>();
          if (qq < n) {
            const R a = re(A[(long long)p * n + p]), b = re(A[(long long)qq * n + qq]);
            const E gpq = A[(long long)p * n + qq];
            const R hh = absv(gpq);
            if (hh > tol_rel * sqrt(fabs(a * b)) && hh > tol_abs) {
              const R tau = (b - a) / (2 * hh);
              const R tt = (tau >= 0 ? (R)1 : (R)-1) / (fabs(tau) + sqrt((R)1 + tau * tau));
              rp.q = qq;
              rp.c = (R)1 / sqrt((R)1 + tt * tt);
              rp.s = tt * rp.c;
              rp.e = divr<E, R>(gpq, hh);
              flags[0] = 1;
              atomicAdd(&flags[1], 1);
            }
          }
          rot[k] = rp;
        }
        __syncthreads();
        // columns: [x, y] <- [c x - s y conj(e), s x + c y conj(e)]
        for (int w2 = tid; w2 < n * cn; w2 += nth) {
          const int i = w2 / cn, k = w2 % cn;
          const Rot<R, E> rp = rot[k];
          if (rp.q < 0) continue;
          const E ec = cj(rp.e);
          E* Ai = A + (long long)i * n;
          const E x = Ai[rp.p], ys = mulv(Ai[rp.q], ec);
          Ai[rp.p] = lin(rp.c, x, -rp.s, ys);
          Ai[rp.q] = lin(rp.s, x, rp.c, ys);
          E* Vi = V + (long long)i * n;
          const E vx = Vi[rp.p], vys = mulv(Vi[rp.q], ec);
          Vi[rp.p] = lin(rp.c, vx, -rp.s, vys);
          Vi[rp.q] = lin(rp.s, vx, rp.c, vys);
        }
        __syncthreads();
        // rows: [x; y] <- [c x - s e y; s x + c e y]
        for (int w2 = tid; w2 < n * cn; w2 += nth) {
          const int k = w2 / n, i = w2 % n;
          const Rot<R, E> rp = rot[k];
          if (rp.q < 0) continue;
          const E x = A[(long long)rp.p * n + i], ye = mulv(rp.e, A[(long long)rp.q * n + i]);
          A[(long long)rp.p * n + i] = lin(rp.c, x, -rp.s, ye);
          A[(long long)rp.q * n + i] = lin(rp.s, x, rp.c, ye);
        }
        __syncthreads();
      }
    }
    if (!flags[0]) break;
  }
  __syncthreads();
  return sweep;
}

// One-sided rotation parameters from the column 2x2 Gram [[al, ga], [conj ga, be]].
// Returns false when the pair is already orthogonal to the path's tolerance or one
// column is at or below the selection floor.  The FP64 path takes the angle from
// FP32 arithmetic (its accuracy only sets the convergence rate) and makes c, s and
// e exactly unitary in FP64 by Newton steps on FP32 reciprocal square roots, which
// avoids FP64 division and square root (slow on this part).
__device__ __forceinline__ double rsqrt_newton(double x) {
  double r = rsqrt(x);               // FP64 approximation, no division
  return r * (1.5 - 0.5 * x * r * r);  // one Newton step to full precision
}
__device__ __forceinline__ bool os_params(double al, double be, double2 ga, bool selfm, double tol_abs,
                                          double col_floor, double& c, double& s, double2& e) {
  if (selfm) ga.y = 0;
  const double g2 = ga.x * ga.x + ga.y * ga.y;
  const double rel = Prec<double>::os_rel;
  if (!(g2 > rel * rel * al * be && g2 > tol_abs * tol_abs && al > col_floor && be > col_floor)) return false;
  const double inv = rsqrt_newton(g2);
  const double tau = (be - al) * 0.5 * inv;
  if (fabs(tau) > 1e30) return false;  // angle below any representable rotation
  const float tf = (float)tau, af = fabsf(tf);
  // t = sign / (|tau| + sqrt(1 + tau^2)); for |tau| > 1e4 this is 1 / (2 |tau|) to
  // FP32 accuracy, and tau^2 would overflow FP32 beyond ~1.8e19
  const float t32 = (tf >= 0.f ? 1.f : -1.f) * (af > 1e4f ? 0.5f / af : 1.f / (af + sqrtf(1.f + tf * tf)));
  const double t = (double)t32;
  c = rsqrt_newton(1.0 + t * t);
  s = t * c;
  e = make_double2(ga.x * inv, ga.y * inv);
  return true;
}
__device__ __forceinline__ bool os_params(float al, float be, float2 ga, bool selfm, float tol_abs,
                                          float col_floor, float& c, float& s, float2& e) {
  if (selfm) ga.y = 0;
  const float hh = hypotf(ga.x, ga.y);
  if (!(hh > Prec<float>::os_rel * sqrtf(al * be) && hh > tol_abs && al > col_floor && be > col_floor)) return false;
  const float tau = (be - al) / (2.f * hh);
  const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
  c = rsqrtf(1.f + t * t);
  s = t * c;
  e = make_float2(ga.x / hh, ga.y / hh);
  return true;
}

// Relative off-diagonal |g|^2 / (a b) of a column pair, in FP32 (it only steers the
// sweep stop).  The FP64 version rescales all three by the same power of two taken
// from a's exponent bits, so the FP32 quotient neither divides in FP64 nor underflows
// (b >= the column floor, a fraction >= 1e-28 of the largest column).
__device__ __forceinline__ float rel_off2(float a, float b, float g2) { return g2 / (a * b); }
__device__ __forceinline__ float rel_off2(double a, double b, double g2) {
  const int e = ((__double2hiint(a) >> 20) & 0x7ff) - 1023;
  const double sc = __hiloint2double((1023 - e) << 20, 0);  // 2^-e
  const float fa = (float)(a * sc), fb = (float)(b * sc), fg = (float)(g2 * sc * sc);
  return fg / (fa * fb);
}

template <typename R> struct PairWork {
  R al, be, c, s;
  typename Prec<R>::C ga, e;
  int act;
};

// One-sided Jacobi sweeps on the n columns (length h) of W, the same rotations on the
// columns (length n) of Vc.  Each round: inner products (one warp per pair), rotation
// parameters (one thread per pair), updates (one warp per pair).
// FP32: one phase per round -- each warp computes its pair's inner products, the
// rotation (redundantly in every lane, cheap in FP32) and the update.
__device__ int refine_sweeps_fp32(float2* W, float2* Vc, int n, int h, bool selfm, float tol_abs, float col_floor,
                                  int* flags) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int np = n + (n & 1), half = np / 2;
  int sweep = 0;
  for (; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
    __syncthreads();
    if (tid == 0) { flags[0] = 0; flags[2] = 0; }
    __syncthreads();
    float wr2 = 0.f;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int k = warp; k < half; k += nwarp) {
        int p, qq;
        circle_pair(rnd, k, np, p, qq);
        if (qq >= n) continue;
        float2* wp = W + (long long)p * h;
        float2* wq = W + (long long)qq * h;
        float al = 0.f, be = 0.f;
        float2 ga = make_float2(0.f, 0.f);
        for (int x = lane; x < h; x += 32) {
          const float2 a = wp[x], b = wq[x];
          al += a.x * a.x + a.y * a.y;
          be += b.x * b.x + b.y * b.y;
          cfma_cj(ga, a, b);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
          ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
        }
        if (al > col_floor && be > col_floor)
          wr2 = fmaxf(wr2, rel_off2(al, be, selfm ? ga.x * ga.x : ga.x * ga.x + ga.y * ga.y));
        float c, sn;
        float2 e;
        if (!os_params(al, be, ga, selfm, tol_abs, col_floor, c, sn, e)) continue;  // warp-uniform
        const float2 ec = cj(e);
        for (int x = lane; x < h; x += 32) {
          const float2 a = wp[x], bs = mulv(wq[x], ec);
          wp[x] = lin(c, a, -sn, bs);
          wq[x] = lin(sn, a, c, bs);
        }
        float2* vp = Vc + (long long)p * n;
        float2* vq = Vc + (long long)qq * n;
        for (int x = lane; x < n; x += 32) {
          const float2 a = vp[x], bs = mulv(vq[x], ec);
          vp[x] = lin(c, a, -sn, bs);
          vq[x] = lin(sn, a, c, bs);
        }
        if (lane == 0) { flags[0] = 1; atomicAdd(&flags[1], 1); }
      }
      __syncthreads();
    }
    if (lane == 0) atomicMax(reinterpret_cast<unsigned*>(&flags[2]), __float_as_uint(wr2));
    __syncthreads();
    if (!flags[0]) break;
    if ((double)__uint_as_float((unsigned)flags[2]) < Prec<float>::stop2) { ++sweep; break; }
  }
  __syncthreads();
  return sweep;
}

template <typename R>
__device__ int refine_sweeps(typename Prec<R>::C* W, typename Prec<R>::C* Vc, int n, int h, bool selfm,
                             R tol_abs, R col_floor, PairWork<R>* pw, int* flags) {
  typedef typename Prec<R>::C C;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  const int np = n + (n & 1), half = np / 2;
  int sweep = 0;
  for (; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
    __syncthreads();
    if (tid == 0) { flags[0] = 0; flags[2] = 0; }
    __syncthreads();
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int c0 = 0; c0 < half; c0 += PAIR_CHUNK) {
        const int cn = (half - c0) < PAIR_CHUNK ? (half - c0) : PAIR_CHUNK;
        for (int k = warp; k < cn; k += nwarp) {
          int p, qq;
          circle_pair(rnd, c0 + k, np, p, qq);
          if (qq >= n) { if (lane == 0) pw[k].act = 0; continue; }
          const C* wp = W + (long long)p * h;
          const C* wq = W + (long long)qq * h;
          R al = 0, be = 0;
          C ga = zero_e<C>();
          for (int x = lane; x < h; x += 32) {
            const C a = wp[x], b = wq[x];
            al += a.x * a.x + a.y * a.y;
            be += b.x * b.x + b.y * b.y;
            cfma_cj(ga, a, b);
          }
          for (int o = 16; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
            ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
          }
          if (lane == 0) { pw[k].al = al; pw[k].be = be; pw[k].ga = ga; pw[k].act = 1; }
        }
        __syncthreads();
        for (int k = tid; k < cn; k += nth) {
          if (!pw[k].act) continue;
          const R al = pw[k].al, be = pw[k].be;
          if (al > col_floor && be > col_floor) {
            const C ga = pw[k].ga;
            const float r2 = rel_off2(al, be, selfm ? ga.x * ga.x : ga.x * ga.x + ga.y * ga.y);
            atomicMax(reinterpret_cast<unsigned*>(&flags[2]), __float_as_uint(r2));
          }
          R c, s;
          C e;
          if (os_params(pw[k].al, pw[k].be, pw[k].ga, selfm, tol_abs, col_floor, c, s, e)) {
            pw[k].c = c; pw[k].s = s; pw[k].e = e;
            flags[0] = 1;
            atomicAdd(&flags[1], 1);
          } else {
            pw[k].act = 0;
          }
        }
        __syncthreads();
        for (int k = warp; k < cn; k += nwarp) {
          if (!pw[k].act) continue;
          int p, qq;
          circle_pair(rnd, c0 + k, np, p, qq);
          const R cs = pw[k].c, sn = pw[k].s;
          const C ec = cj(pw[k].e);
          C* wp = W + (long long)p * h;
          C* wq = W + (long long)qq * h;
          for (int x = lane; x < h; x += 32) {
            const C a = wp[x], bs = mulv(wq[x], ec);
            wp[x] = lin(cs, a, -sn, bs);
            wq[x] = lin(sn, a, cs, bs);
          }
          C* vp = Vc + (long long)p * n;
          C* vq = Vc + (long long)qq * n;
          for (int x = lane; x < n; x += 32) {
            const C a = vp[x], bs = mulv(vq[x], ec);
            vp[x] = lin(cs, a, -sn, bs);
            vq[x] = lin(sn, a, cs, bs);
          }
        }
        __syncthreads();
      }
    }
    if (!flags[0]) break;
    if ((double)__uint_as_float((unsigned)flags[2]) < Prec<R>::stop2) { ++sweep; break; }
  }
  __syncthreads();
  return sweep;
}

__device__ __forceinline__ int mirror_coord(const Slot& sl, const MpoDev& st, const GateDesc& g, int t,
                                            int side, int i, const int* segX) {
  const int ncap = st.ncap, P = st.P, D = st.D, M = st.M;
  const long long bX = (long long)g.inst * (M + 1) + g.j + (side == 0 ? 0 : 2);
  const int idx = side == 0 ? sl.rowmap[sl.f(BF_RMOFF, t) + i] : sl.colmap[sl.f(BF_CMOFF, t) + i];
  const int pa = st.charge[bX * D + idx];
  const int pm = pair_mirror(pa, ncap);
  const int off = side == 0 ? sl.rowoff[t * P + pm] : sl.coloff[t * P + pm];
  const int pos = idx - segX[pa];
  if (off < 0 || pos >= segX[pm + 1] - segX[pm]) {  // mirror structure broken: never index with it
    dev_set_error(st.err, DEV_ERR_INTERNAL, 8000 + t);
    return i;
  }
  return off + pos;
}

// Shared-memory layout of k_svd (host and device agree through this function).
struct SvdLayout {
  size_t hdr, pw, mpos, seg, nrm, data, total;
};
template <typename R>
__host__ __device__ inline SvdLayout svd_layout(int D, size_t total) {
  SvdLayout L;
  size_t o = 0;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  L.hdr = o; o = al(o + 128);  // 32 ints (Jacobi flags, work item, cluster sweep totals)
  const size_t pwb = (size_t)PAIR_CHUNK * sizeof(PairWork<R>);
  const size_t rtb = (size_t)PAIR_CHUNK * sizeof(Rot<float, float2>);
  L.pw = o; o = al(o + (pwb > rtb ? pwb : rtb));
  L.mpos = o; o = al(o + (size_t)D * sizeof(int));
  L.seg = o; o = al(o + (size_t)(MPO_P_MAX + 2) * sizeof(int));
  L.nrm = o; o = al(o + (size_t)(D > 32 ? D : 32) * sizeof(R));
  L.data = o;
  L.total = total;
  return L;
}

// FP32 seed for one canonical block: Gram eigenvectors by two-sided Jacobi (real
// arithmetic in the mirror-conjugation basis for self-mirror blocks), written
// row-major to the slot's V buffer as complex FP32.
__device__ void seed_block(const MpoDev& st, const Slot& sl, const GateDesc& g, int t, unsigned char* smem,
                           const SvdLayout& L) {
  typedef float R;
  typedef float2 C;
  const int n = sl.f(BF_G, t), side = sl.f(BF_SIDE, t), m = sl.f(BF_M, t);
  const int ncap = st.ncap, P = st.P, M = st.M;
  const bool selfm = pair_mirror(m, ncap) == m;
  const int tid = threadIdx.x, nth = blockDim.x;
  int* flags = reinterpret_cast<int*>(smem + L.hdr);
  int* mpos = reinterpret_cast<int*>(smem + L.mpos);
  int* segX = reinterpret_cast<int*>(smem + L.seg);
  const size_t room = L.total - L.data;
  C* gG = reinterpret_cast<C*>(sl.G) + sl.f(BF_GOFF, t);
  C* gV = reinterpret_cast<C*>(sl.V) + sl.f(BF_GOFF, t);
  if (tid == 0) { flags[0] = 0; flags[1] = 0; }  // published by the barriers below
  if (selfm) {
    const bool in_smem = 2ull * n * n * sizeof(R) <= room;
    const long long bX = (long long)g.inst * (M + 1) + g.j + (side == 0 ? 0 : 2);
    for (int p = tid; p <= P; p += nth) segX[p] = st.segoff[bX * (P + 1) + p];
    __syncthreads();
    for (int i = tid; i < n; i += nth) mpos[i] = mirror_coord(sl, st, g, t, side, i, segX);
    __syncthreads();
    // real Gram in the basis e_i (fixed), (e_p + e_q)/sqrt2 at p, i(e_p - e_q)/sqrt2 at q (p < q)
    R* A = in_smem ? reinterpret_cast<R*>(smem + L.data) : reinterpret_cast<R*>(gV);
    R* V = in_smem ? A + (long long)n * n : reinterpret_cast<R*>(gG);
    const R h = (R)0.70710678118654752440;
    for (int e = tid; e < n * n; e += nth) {
      const int i = e / n, j = e % n;
      int ai[2], bj[2]; C wa[2], wb[2]; int na = 0, nb = 0;
      const int pi = mpos[i], pj = mpos[j];
      if (pi == i) { ai[0] = i; wa[0] = mk((R)1, (R)0); na = 1; }
      else if (i < pi) { ai[0] = i; wa[0] = mk(h, (R)0); ai[1] = pi; wa[1] = mk(h, (R)0); na = 2; }
      else { ai[0] = pi; wa[0] = mk((R)0, h); ai[1] = i; wa[1] = mk((R)0, -h); na = 2; }
      if (pj == j) { bj[0] = j; wb[0] = mk((R)1, (R)0); nb = 1; }
      else if (j < pj) { bj[0] = j; wb[0] = mk(h, (R)0); bj[1] = pj; wb[1] = mk(h, (R)0); nb = 2; }
      else { bj[0] = pj; wb[0] = mk((R)0, h); bj[1] = j; wb[1] = mk((R)0, -h); nb = 2; }
      R acc = 0;
      for (int x = 0; x < na; ++x)
        for (int y = 0; y < nb; ++y) acc += cmul(cmul(cj(wa[x]), gG[(long long)ai[x] * n + bj[y]]), wb[y]).x;
      A[(long long)i * n + j] = acc;
    }
    __syncthreads();  // gG fully read before V (global mode) overwrites it
    const int sweeps = jacobi<R, R>(A, V, n, reinterpret_cast<Rot<R, R>*>(smem + L.pw), flags,
                                    Prec<R>::tol_rel, Prec<R>::tol_abs);
    // eigenvectors back to the original basis: x = W x~ (x~ real).  In global mode A
    // (dead now) shares gV's storage and V lives in gG, so writing gV is safe.
    for (int e = tid; e < n * n; e += nth) {
      const int i = e / n, k = e % n;
      const int pi = mpos[i];
      C out;
      if (pi == i) out = mk(V[(long long)i * n + k], (R)0);
      else if (i < pi) out = mk(h * V[(long long)i * n + k], h * V[(long long)pi * n + k]);
      else out = mk(h * V[(long long)pi * n + k], -h * V[(long long)i * n + k]);
      gV[e] = out;
    }
    if (st.ctr && tid == 0) {
      // real rotation: 6 flops per index for A columns, A rows and V columns each
      atomicAdd(st.ctr + CTR_EIG, 18ull * (unsigned long long)n * (unsigned long long)flags[1]);
      atomicAdd(st.ctr + CTR_SWEEPS, (unsigned long long)(sweeps + 1));
      atomicAdd(st.ctr + CTR_EIGBLK, 1ull);
    }
  } else {
    const bool in_smem = 2ull * n * n * sizeof(C) <= room;
    C* A = in_smem ? reinterpret_cast<C*>(smem + L.data) : gG;
    C* V = in_smem ? A + (long long)n * n : gV;
    if (in_smem) {
      for (int e = tid; e < n * n; e += nth) A[e] = gG[e];
    }
    __syncthreads();
    const int sweeps = jacobi<R, C>(A, V, n, reinterpret_cast<Rot<R, C>*>(smem + L.pw), flags,
                                    Prec<R>::tol_rel, Prec<R>::tol_abs);
    if (in_smem) {
      for (int e = tid; e < n * n; e += nth) gV[e] = V[e];
    }
    if (st.ctr && tid == 0) {
      // per active rotation and per index: A columns, A rows and V columns, 18 flops each
      atomicAdd(st.ctr + CTR_EIG, 54ull * (unsigned long long)n * (unsigned long long)flags[1]);
      atomicAdd(st.ctr + CTR_SWEEPS, (unsigned long long)(sweeps + 1));
      atomicAdd(st.ctr + CTR_EIGBLK, 1ull);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- large blocks
// A block whose Jacobi work would hold one SM long after the rest of the layer has
// finished runs on a whole thread-block cluster (K CTAs, one per SM): a parallel
// one-sided block Jacobi.  The n columns of W (length h) and of V (length n) are cut
// into 2K w column blocks of width b = ceil(n / 2K w), w the smallest power of two
// (<= 8) for which a CTA's two blocks fit in shared memory; a round-robin tournament
// over the blocks gives every CTA w block pairs per round (2K w - 1 rounds per sweep).  A CTA
// stages its two blocks in shared memory, orthogonalises every column of one block
// against every column of the other (b rounds of b disjoint pairs, one warp per
// pair; in the first round of a sweep also the pairs inside each block), writes them
// back to the slot scratch (L2-resident) and meets the others at a cluster barrier.
// Every pair of columns is visited once per sweep, as in a cyclic sweep.  Sweeps stop
// when no CTA of the cluster rotated (a sum over distributed shared memory).
//
// Precision: the FP32 phase starts from the basis B (identity, or the mirror-real
// basis of a self-mirror block) and converges in FP32.  A polish in the path's
// precision follows: two Newton-Schulz steps make V unitary again (distributed by
// columns), W = Theta V is formed afresh and the sweeps repeat.  The result layout is the single-CTA refinement's (W, V column-major in
// the slot's W and VC buffers), so the selection and re-split do not change.

// shared-memory header words of k_svd (ints): [0..1] Jacobi flags, [8] work item,
// [10] rotations of this CTA in the current sweep, [11] cluster total (leader),
// [12] broadcast copy of the total, [14..15] a double (partial maximum)
constexpr int HDR_ITEM = 8, HDR_ROT = 10, HDR_TOT = 11, HDR_BC = 12, HDR_MAX = 14;
constexpr int HDR_RMAX = 16, HDR_RTOT = 17, HDR_RBC = 18;  // largest relative off-diagonal^2 of a sweep

// Global-memory hand-over between the CTAs of a cluster: every write before the
// barrier is visible to every read after it (fences at device scope on both sides,
// so no CTA reads a line it cached before another CTA rewrote it).
__device__ __forceinline__ void cluster_exchange(cg::cluster_group& cl) {
  __threadfence();
  cl.sync();
  __threadfence();
}

// Mirror partner (position in the block) of every index on the small side of block
// t, in shared memory.
__device__ void block_mirror_map(const MpoDev& st, const Slot& sl, const GateDesc& g, int t, int* mpos,
                                 int* segX) {
  const int n = sl.f(BF_G, t), side = sl.f(BF_SIDE, t), P = st.P, M = st.M;
  const long long bX = (long long)g.inst * (M + 1) + g.j + (side == 0 ? 0 : 2);
  for (int p = threadIdx.x; p <= P; p += blockDim.x) segX[p] = st.segoff[bX * (P + 1) + p];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) mpos[i] = mirror_coord(sl, st, g, t, side, i, segX);
  __syncthreads();
}

// Column k of the starting basis of a one-sided Jacobi without a seed: e_k, or for a
// self-mirror block the basis in which the mirror acts as complex conjugation, so that
// the columns of Theta B are mirror-real and their inner products real:
// e_k (k is its own mirror), (e_k + e_p)/sqrt2 (k < p = mirror of k),
// i (e_p - e_k)/sqrt2 (k > p).  Returns the number of entries (1 or 2).
template <typename C, typename R>
__device__ __forceinline__ int basis_col(int k, const int* mpos, bool selfm, int* idx, C* wt) {
  const R h = (R)0.70710678118654752440;
  const int p = selfm ? mpos[k] : k;
  if (p == k) { idx[0] = k; wt[0] = unit_e<C>(); return 1; }
  if (k < p) { idx[0] = k; wt[0] = mk(h, (R)0); idx[1] = p; wt[1] = mk(h, (R)0); return 2; }
  idx[0] = p; wt[0] = mk((R)0, h); idx[1] = k; wt[1] = mk((R)0, -h); return 2;
}

// One warp: one one-sided Jacobi rotation of the column pair (p, q) of W (length h)
// and the same rotation of the columns of V (length n).  Returns whether it rotated
// (warp-uniform: the butterfly sums are identical in every lane).
template <typename R>
__device__ __forceinline__ bool warp_rotate(typename Prec<R>::C* wp, typename Prec<R>::C* wq,
                                            typename Prec<R>::C* vp, typename Prec<R>::C* vq, int h, int n,
                                            bool selfm, typename Prec<R>::T tol_abs,
                                            typename Prec<R>::T col_floor, int lane, float& r2,
                                            typename Prec<R>::T*, typename Prec<R>::T*) {
  // (the FP32 sweeps recompute both column norms for every pair: carrying them as the
  // double-float sweeps do was measured slower, 4.2 against 3.8 ms of FP32 phase per
  // 48-mode cluster block, with a recompute of norms that a rotation shrinks)
  typedef typename Prec<R>::C C;
  R al = 0, be = 0;
  C ga = zero_e<C>();
  for (int x = lane; x < h; x += 32) {
    const C a = wp[x], b = wq[x];
    al += a.x * a.x + a.y * a.y;
    be += b.x * b.x + b.y * b.y;
    cfma_cj(ga, a, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
    ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
  }
  r2 = (al > col_floor && be > col_floor) ? rel_off2(al, be, selfm ? ga.x * ga.x : ga.x * ga.x + ga.y * ga.y)
                                          : 0.f;
  R c, s;
  C e;
  if (!os_params(al, be, ga, selfm, tol_abs, col_floor, c, s, e)) return false;
  const C ec = cj(e);
  for (int x = lane; x < h; x += 32) {
    const C a = wp[x], bs = mulv(wq[x], ec);
    wp[x] = lin(c, a, -s, bs);
    wq[x] = lin(s, a, c, bs);
  }
  for (int x = lane; x < n; x += 32) {
    const C a = vp[x], bs = mulv(vq[x], ec);
    vp[x] = lin(c, a, -s, bs);
    vq[x] = lin(s, a, c, bs);
  }
  return true;
}

// ---- double-float helpers of the FP64 refinement (dd.cuh)
__device__ __forceinline__ dd dd_shfl_xor(dd v, int o) {
  return dd_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
// sum over the warp, bitwise the same in every lane (dd_add is commutative bit for bit:
// both TwoSums are exact)
__device__ __forceinline__ dd dd_warp_sum(dd v) {
  for (int o = 16; o > 0; o >>= 1) v = dd_add(v, dd_shfl_xor(v, o));
  return v;
}
__device__ __forceinline__ ddc ddc_conv(double2 a) { return ddc_from(a.x, a.y); }
__device__ __forceinline__ double2 ddc_back(ddc a) { return make_double2(dd_to(a.re), dd_to(a.im)); }




// One-sided rotation of a column pair in double-float: the inner product by
// compensated accumulation in every lane and a double-float butterfly (the squared
// column norms are carried by the caller), the rotation parameters in FP64 from their
// FP64 roundings (as on the FP64 path: per pair, not per element), the update of W
// and V in double-float.
template <>
__device__ __forceinline__ bool warp_rotate<dd>(ddc* wp, ddc* wq, ddc* vp, ddc* vq, int h, int n, bool selfm,
                                                double tol_abs, double col_floor, int lane, float& r2, double* np_,
                                                double* nq_) {
  // np_, nq_: the pair's squared column norms as double-floats (8 bytes, like the
  // double they are stored as), carried from rotation to rotation; read before the
  // inner product, written by lane 0 after it
  dd* pn = reinterpret_cast<dd*>(np_);
  dd* qn = reinterpret_cast<dd*>(nq_);
  const dd al = *pn, be = *qn;
  dd_acc gr = dd_acc_zero(), gi = dd_acc_zero();
  for (int x = lane; x < h; x += 32) {
    const ddc a = wp[x], b = wq[x];
    dd_acc_mac(gr, a.re, b.re);  // conj(a) b
    dd_acc_mac(gr, a.im, b.im);
    dd_acc_mac(gi, a.re, b.im);
    dd_acc_mac(gi, dd_neg(a.im), b.re);
  }
  const dd g_re = dd_warp_sum(dd_acc_value(gr)), g_im = dd_warp_sum(dd_acc_value(gi));
  dd c, s, gabs;
  ddc e;
  if (!dd_os_params(al, be, g_re, g_im, selfm, (float)tol_abs, (float)col_floor, (float)Prec<double>::os_rel,
                    c, s, e, gabs, r2))
    return false;
  if (lane == 0) {
    dd a2 = al, b2 = be;
    rotated_norms_dd(a2, b2, gabs, c, s);
    *pn = a2;
    *qn = b2;
  }
  ddc_rotate_dd(wp, wq, h, lane, c, s, e);
  ddc_rotate_dd(vp, vq, n, lane, c, s, e);
  return true;
}

// Squared norm of a column of length len, in double-float by one warp (every lane
// gets the same value).
__device__ __forceinline__ dd ddc_col_norm2_dd(const ddc* w, int len, int lane) {
  dd_acc a = dd_acc_zero();
  for (int x = lane; x < len; x += 32) {
    const ddc v = w[x];
    dd_acc_mac(a, v.re, v.re);
    dd_acc_mac(a, v.im, v.im);
  }
  return dd_warp_sum(dd_acc_value(a));
}
// The same, rounded to FP64.
__device__ __forceinline__ double ddc_col_norm2(const ddc* w, int len, int lane) {
  dd_acc a = dd_acc_zero();
  for (int x = lane; x < len; x += 32) {
    const ddc v = w[x];
    dd_acc_mac(a, v.re, v.re);
    dd_acc_mac(a, v.im, v.im);
  }
  return dd_to(dd_warp_sum(dd_acc_value(a)));
}

// Largest column norm^2 of the columns [k0, k1) of W over the whole cluster.
template <typename R>
__device__ R cluster_max_norm2(cg::cluster_group& cl, const typename Prec<R>::C* W, int h, int k0, int k1,
                               int* hdr, R* red) {
  typedef typename Prec<R>::C C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  R mx = 0;
  for (int k = k0 + warp; k < k1; k += nwarp) {
    R a = 0;
    for (int x = lane; x < h; x += 32) { const C w = W[(long long)k * h + x]; a += w.x * w.x + w.y * w.y; }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    mx = fmax(mx, a);
  }
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    R m = 0;
    for (int w2 = 0; w2 < nwarp; ++w2) m = fmax(m, red[w2]);
    *reinterpret_cast<double*>(hdr + HDR_MAX) = (double)m;
  }
  cl.sync();
  double g = 0;
  for (unsigned r = 0; r < cl.num_blocks(); ++r)
    g = fmax(g, *cl.map_shared_rank(reinterpret_cast<double*>(hdr + HDR_MAX), r));
  cl.sync();  // every CTA has read every partial before any is overwritten
  return (R)g;
}

// Sweeps of the parallel one-sided block Jacobi over the cluster on W (h x n) and
// V (n x n), column-major in global memory.  Returns the number of sweeps that
// rotated; *rotations accumulates this CTA's applied rotations.
template <typename R>
// gN (double-float sweeps, where it is required; null otherwise): n squared column
// norms in global memory, recomputed at the start of every sweep and carried through
// it (staged with the block pair in the CTA's norm area of shared memory).
__device__ int cluster_sweeps(cg::cluster_group& cl, typename Prec<R>::C* gW, typename Prec<R>::C* gV, int n,
                              int h, bool selfm, typename Prec<R>::T tol_abs, typename Prec<R>::T col_floor,
                              unsigned char* smem, const SvdLayout& L, int* hdr, unsigned long long* rotations,
                              typename Prec<R>::T* gN = nullptr) {
  typedef typename Prec<R>::C C;
  typedef typename Prec<R>::T T;
  const int K = (int)cl.num_blocks(), kr = (int)cl.block_rank();
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  const size_t room = L.total - L.data;
  // 2 K wb column blocks: wb (1..8) grows until a CTA's two blocks of W and V fit in
  // shared memory; each CTA then takes wb block pairs of a round one after another
  int wb = 1;
  while (wb < 8 && (size_t)2 * ((n + 2 * K * wb - 1) / (2 * K * wb)) * ((size_t)h + n) * sizeof(C) > room) wb *= 2;
  const int nb = 2 * K * wb, b = (n + nb - 1) / nb;
  const bool w_st = (size_t)2 * b * h * sizeof(C) <= room;
  const bool v_st = w_st && (size_t)2 * b * ((size_t)h + n) * sizeof(C) <= room;
  C* sW = reinterpret_cast<C*>(smem + L.data);
  C* sV = sW + (size_t)2 * b * h;
  T* sN = gN ? reinterpret_cast<T*>(smem + L.nrm) : nullptr;  // 2 b <= n <= D entries
  int sweep = 0;
  float wr2 = 0.f;  // this warp's largest relative off-diagonal^2 in the sweep
  for (; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
    if (tid == 0) { hdr[HDR_ROT] = 0; hdr[HDR_RMAX] = 0; }
    wr2 = 0.f;
    if constexpr (std::is_same<R, dd>::value) {
      if (gN) {  // this CTA's share of the columns, read by every CTA after the barrier
        const int c0 = (int)((long long)kr * n / K), c1 = (int)((long long)(kr + 1) * n / K);
        for (int k = c0 + warp; k < c1; k += nwarp) {  // stored as double-floats (see warp_rotate<dd>)
          const dd v = ddc_col_norm2_dd(gW + (long long)k * h, h, lane);
          if (lane == 0) reinterpret_cast<dd*>(gN)[k] = v;
        }
        cluster_exchange(cl);
      }
    }
    __syncthreads();
    for (int rho = 0; rho < nb - 1; ++rho) {
     for (int pi = kr; pi < nb / 2; pi += K) {
      int I, J;
      circle_pair(rho, pi, nb, I, J);
      const int i0 = I * b, j0 = J * b;
      const int nI = max(0, min(n, i0 + b) - i0), nJ = max(0, min(n, j0 + b) - j0);
      const int nl = nI + nJ;
      auto gcol = [&](int l) { return l < nI ? i0 + l : j0 + (l - nI); };
      auto wcol = [&](int l) { return w_st ? sW + (size_t)l * h : gW + (long long)gcol(l) * h; };
      auto vcol = [&](int l) { return v_st ? sV + (size_t)l * n : gV + (long long)gcol(l) * n; };
      auto rotate = [&](int p, int q) {
        float r2 = 0.f;
        const bool rot = warp_rotate<R>(wcol(p), wcol(q), vcol(p), vcol(q), h, n, selfm, tol_abs, col_floor, lane,
                                        r2, sN ? sN + p : nullptr, sN ? sN + q : nullptr);
        wr2 = fmaxf(wr2, r2);
        if (rot && lane == 0) atomicAdd(&hdr[HDR_ROT], 1);
      };
      if (w_st) {
        for (long long e = tid; e < (long long)nl * h; e += nth) sW[e] = gW[(long long)gcol((int)(e / h)) * h + e % h];
        if (v_st)
          for (long long e = tid; e < (long long)nl * n; e += nth) sV[e] = gV[(long long)gcol((int)(e / n)) * n + e % n];
      }
      if (sN)
        for (int l = tid; l < nl; l += nth) sN[l] = gN[gcol(l)];
      __syncthreads();
      if (rho == 0) {
        // pairs inside each of the two blocks (every block is in exactly one pair of round 0)
        const int pI = nI + (nI & 1), pJ = nJ + (nJ & 1);
        const int rounds = max(pI, pJ) - 1;
        for (int r = 0; r < rounds; ++r) {
          const int hI = r < pI - 1 ? pI / 2 : 0, hJ = r < pJ - 1 ? pJ / 2 : 0;
          for (int k = warp; k < hI + hJ; k += nwarp) {
            int p, q;
            if (k < hI) {
              circle_pair(r, k, pI, p, q);
              if (q >= nI) continue;
            } else {
              circle_pair(r, k - hI, pJ, p, q);
              if (q >= nJ) continue;
              p += nI; q += nI;
            }
            rotate(p, q);
          }
          __syncthreads();
        }
      }
      // pairs across the two blocks: round r pairs column i of I with column (i + r) mod b of J
      for (int r = 0; r < b; ++r) {
        for (int i = warp; i < nI; i += nwarp) {
          const int j = (i + r) % b;
          if (j >= nJ) continue;
          rotate(i, nI + j);
        }
        __syncthreads();
      }
      if (w_st) {
        for (long long e = tid; e < (long long)nl * h; e += nth) gW[(long long)gcol((int)(e / h)) * h + e % h] = sW[e];
        if (v_st)
          for (long long e = tid; e < (long long)nl * n; e += nth) gV[(long long)gcol((int)(e / n)) * n + e % n] = sV[e];
      }
      if (sN)
        for (int l = tid; l < nl; l += nth) gN[gcol(l)] = sN[l];
      __syncthreads();  // the staging buffers are refilled for the next block pair
     }
      cluster_exchange(cl);
    }
    // cluster-wide count of this sweep's rotations and its largest relative off-diagonal
    if (lane == 0) atomicMax(reinterpret_cast<unsigned*>(&hdr[HDR_RMAX]), __float_as_uint(wr2));
    __syncthreads();
    if (tid == 0) {
      *rotations += (unsigned long long)hdr[HDR_ROT];
      atomicAdd(cl.map_shared_rank(&hdr[HDR_TOT], 0), hdr[HDR_ROT]);
      atomicMax(cl.map_shared_rank(reinterpret_cast<unsigned*>(&hdr[HDR_RTOT]), 0), (unsigned)hdr[HDR_RMAX]);
    }
    cl.sync();
    if (tid == 0) {
      hdr[HDR_BC] = *cl.map_shared_rank(&hdr[HDR_TOT], 0);
      hdr[HDR_RBC] = *cl.map_shared_rank(&hdr[HDR_RTOT], 0);
    }
    cl.sync();  // every CTA has read the totals before the leader clears them
    if (kr == 0 && tid == 0) { hdr[HDR_TOT] = 0; hdr[HDR_RTOT] = 0; }
    __syncthreads();
    if (hdr[HDR_BC] == 0) break;
    if ((double)__uint_as_float((unsigned)hdr[HDR_RBC]) < Prec<R>::stop2) { ++sweep; break; }
  }
  return sweep;
}

// W = Theta V for the columns [k0, k1) (side 1: W = Theta V, h = rows; side 0:
// W = Theta^dag V, h = cols), V column-major n x n, in the path precision C.
template <typename C, typename CT>
__device__ void form_w_cols(const CT* Th, const C* V, C* W, int r, int c, int side, int n, int h, int k0, int k1) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (long long e = tid; e < (long long)(k1 - k0) * h; e += nth) {
    const int k = k0 + (int)(e / h), x = (int)(e % h);
    C acc = zero_e<C>();
    if (side == 1) {
      for (int q = 0; q < n; ++q) cfma(acc, cvt<C>(to_d2(Th[(long long)x * c + q])), V[(long long)k * n + q]);
    } else {
      for (int i = 0; i < n; ++i) cfma_cj(acc, cvt<C>(to_d2(Th[(long long)i * c + x])), V[(long long)k * n + i]);
    }
    W[(long long)k * h + x] = acc;
  }
}

// The singular values of block t: column norms of the converged W, ranked descending
// (ties by index), written to the candidate list; norms go through global scratch.
template <typename R>
__device__ void cluster_rank(cg::cluster_group& cl, const MpoDev& st, const Slot& sl, int t,
                             const typename Prec<R>::C* W, R* nrm, int n, int h, int k0, int k1) {
  typedef typename Prec<R>::C C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int K = (int)cl.num_blocks(), kr = (int)cl.block_rank();
  for (int k = k0 + warp; k < k1; k += nwarp) {
    R a = 0;
    for (int x = lane; x < h; x += 32) { const C w = W[(long long)k * h + x]; a += w.x * w.x + w.y * w.y; }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) nrm[k] = a;
  }
  cluster_exchange(cl);
  const int coff = sl.f(BF_COFF, t);
  const int r0 = (int)((long long)kr * n / K), r1 = (int)((long long)(kr + 1) * n / K);
  for (int i = r0 + tid; i < r1; i += blockDim.x) {
    const R wi = nrm[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (nrm[j] > wi) || (nrm[j] == wi && j < i);
    if (!isfinite((double)wi)) dev_set_error(st.err, DEV_ERR_NUMERIC, 4600 + t);
    sl.sval[coff + rank] = sqrt((double)wi);
    sl.perm[coff + rank] = i;
  }
}

// ---------------------------------------------------------------- double-float polish
// The FP64 path's polish of a cluster block, in double-float arithmetic (dd.cuh):
// the same steps as the polish in the path precision -- two Newton-Schulz steps on V,
// W = Theta V afresh, one-sided sweeps to the FP64 thresholds, singular values as
// column norms -- with every vector operation on pairs of FP32 numbers.  Long inner
// products are summed in chunks of 16 by compensated accumulation and the chunks
// combined by dd_add, which bounds their error by ~20 u^2 times the magnitude sum.


// Largest column norm^2 of the columns [k0, k1) of W over the cluster (FP64 rounding).
__device__ double cluster_max_norm2_dd(cg::cluster_group& cl, const ddc* W, int h, int k0, int k1, int* hdr,
                                       double* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  double mx = 0;
  for (int k = k0 + warp; k < k1; k += nwarp) mx = fmax(mx, ddc_col_norm2(W + (long long)k * h, h, lane));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    double m = 0;
    for (int w2 = 0; w2 < nwarp; ++w2) m = fmax(m, red[w2]);
    *reinterpret_cast<double*>(hdr + HDR_MAX) = m;
  }
  cl.sync();
  double g = 0;
  for (unsigned r = 0; r < cl.num_blocks(); ++r)
    g = fmax(g, *cl.map_shared_rank(reinterpret_cast<double*>(hdr + HDR_MAX), r));
  cl.sync();  // every CTA has read every partial before any is overwritten
  return g;
}

// Polish of block t on the cluster.  On entry V (FP32) is the seed: row-major in Vs
// (Gram seed) or column-major in V32; Theta is FP64.  On exit gW and gV hold W and V
// as complex128 (the layout the re-split reads) and the singular values are ranked.
// Returns the sweeps; *rot counts this CTA's rotations.
__device__ int polish_dd(cg::cluster_group& cl, const MpoDev& st, const Slot& sl, int t, double2* Th,
                         double2* gW, double2* gV, const float2* Vs, const float2* V32, bool gram_seed, int n,
                         int h, int r, int c, int side, bool selfm, int k0, int k1, unsigned char* smem,
                         const SvdLayout& L, int* hdr, unsigned long long* rot, long long* tc, bool timed) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int K = (int)cl.num_blocks(), kr = (int)cl.block_rank();
  ddc* Vd = reinterpret_cast<ddc*>(gV);
  ddc* Wd = reinterpret_cast<ddc*>(gW);
  ddc* Sd = reinterpret_cast<ddc*>(sl.NS) + sl.f(BF_GOFF, t);
  ddc* Td = Wd;  // W is formed only after Newton-Schulz
  ddc* Thd = reinterpret_cast<ddc*>(Th);
  auto lap = [&](int ctr) {
    if (timed) {
      const long long now = clock64();
      atomicAdd(st.ctr + ctr, (unsigned long long)(now - *tc));
      *tc = now;
    }
  };
  for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {  // V, column-major, exact in double-float
    const int k = k0 + (int)(e / n), i = (int)(e % n);
    const float2 v = gram_seed ? Vs[(long long)i * n + k] : V32[(long long)k * n + i];
    Vd[(long long)k * n + i] = ddc_make(dd_make(v.x, 0.f), dd_make(v.y, 0.f));
  }
  cluster_exchange(cl);
  for (int it = 0; it < 2; ++it) {
    // S[:, k] = V^dag v_k: S is Hermitian, so the entries a <= k are formed and mirrored
    for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {
      const int k = k0 + (int)(e / n), a = (int)(e % n);
      if (a > k) continue;
      const ddc v = ddc_dot(Vd + (long long)a * n, 1, Vd + (long long)k * n, 1, n, true);
      Sd[(long long)k * n + a] = v;
      Sd[(long long)a * n + k] = ddc_conj(v);
    }
    cluster_exchange(cl);
    for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {
      const int k = k0 + (int)(e / n), i = (int)(e % n);
      Td[(long long)k * n + i] = ns_update(Vd, Sd, n, k, i);
    }
    cluster_exchange(cl);
    for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {
      const long long o = (long long)k0 * n + e;
      Vd[o] = Td[o];
    }
    cluster_exchange(cl);
  }
  lap(CTR_CYC_NS);
  {  // Theta to double-float in place (nothing reads it as FP64 afterwards)
    const long long tot = (long long)r * c, a0 = tot * kr / K, a1 = tot * (kr + 1) / K;
    for (long long e = a0 + tid; e < a1; e += nth) Thd[e] = ddc_conv(Th[e]);
  }
  cluster_exchange(cl);
  for (long long e = tid; e < (long long)(k1 - k0) * h; e += nth) {  // W = Theta V or Theta^dag V
    const int k = k0 + (int)(e / h), x = (int)(e % h);
    Wd[(long long)k * h + x] = side == 1 ? ddc_dot(Thd + (long long)x * c, 1, Vd + (long long)k * n, 1, n, false)
                                         : ddc_dot(Thd + x, c, Vd + (long long)k * n, 1, n, true);
  }
  cluster_exchange(cl);
  const double mx = cluster_max_norm2_dd(cl, Wd, h, k0, k1, hdr, reinterpret_cast<double*>(smem + L.nrm));
  const int sw = cluster_sweeps<dd>(cl, Wd, Vd, n, h, selfm, Prec<dd>::os_abs * mx, Prec<dd>::floor * mx, smem, L,
                                    hdr, rot, reinterpret_cast<double*>(Sd));
  if (sw >= JACOBI_MAX_SWEEPS && tid == 0) dev_set_error(st.err, DEV_ERR_NUMERIC, 3600 + t);
  lap(CTR_CYC_POLISH);
  // singular values: column norms of W, ranked descending (ties by index)
  double* nrm = reinterpret_cast<double*>(Sd);
  {
    const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    for (int k = k0 + warp; k < k1; k += nwarp) {
      const double a = ddc_col_norm2(Wd + (long long)k * h, h, lane);
      if (lane == 0) nrm[k] = a;
    }
  }
  cluster_exchange(cl);
  const int coff = sl.f(BF_COFF, t);
  const int r0 = (int)((long long)kr * n / K), r1 = (int)((long long)(kr + 1) * n / K);
  for (int i = r0 + tid; i < r1; i += nth) {
    const double wi = nrm[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (nrm[j] > wi) || (nrm[j] == wi && j < i);
    if (!isfinite(wi)) dev_set_error(st.err, DEV_ERR_NUMERIC, 4600 + t);
    sl.sval[coff + rank] = sqrt(wi);
    sl.perm[coff + rank] = i;
  }
  // back to complex128 for the re-split (each CTA its own columns)
  for (long long e = tid; e < (long long)(k1 - k0) * h; e += nth) {
    const long long o = (long long)k0 * h + e;
    gW[o] = ddc_back(Wd[o]);
  }
  for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {
    const long long o = (long long)k0 * n + e;
    gV[o] = ddc_back(Vd[o]);
  }
  return sw;
}

// One large block on the whole cluster (see the section comment).
template <typename R>
__device__ void big_block(cg::cluster_group& cl, const MpoDev& st, const Slot& sl, const GateDesc& g, int t,
                          unsigned char* smem, const SvdLayout& L, int ws_cl_seed_max) {
  typedef typename Prec<R>::C C;
  const int n = sl.f(BF_G, t);
  const int r = sl.f(BF_R, t), c = sl.f(BF_C, t), side = sl.f(BF_SIDE, t);
  const int h = side == 0 ? c : r;
  const bool selfm = pair_mirror(sl.f(BF_M, t), st.ncap) == sl.f(BF_M, t);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int K = (int)cl.num_blocks(), kr = (int)cl.block_rank();
  const int k0 = (int)((long long)kr * n / K), k1 = (int)((long long)(kr + 1) * n / K);
  int* hdr = reinterpret_cast<int*>(smem + L.hdr);
  int* mpos = reinterpret_cast<int*>(smem + L.mpos);
  int* segX = reinterpret_cast<int*>(smem + L.seg);
  if (selfm) block_mirror_map(st, sl, g, t, mpos, segX);
  const C* Th = reinterpret_cast<const C*>(sl.theta) + sl.f(BF_TOFF, t);
  C* gW = reinterpret_cast<C*>(sl.W) + sl.f(BF_TOFF, t);      // this block's region of the W buffer
  C* gV = reinterpret_cast<C*>(sl.VC) + sl.f(BF_GOFF, t);     // this block's region of the VC buffer
  // FP32 phase buffers: the mixed path works in place; the FP64 path keeps W32 in the
  // low half of its own (complex128) W region and V32 in its float2 region of the
  // seed buffer, which every block addresses with float2 offsets
  float2* W32 = reinterpret_cast<float2*>(gW);
  float2* V32 = sizeof(R) == 8 ? reinterpret_cast<float2*>(sl.V) + sl.f(BF_GOFF, t) : reinterpret_cast<float2*>(gV);
  unsigned long long rot32 = 0, rot64 = 0;
  // A block small enough takes the FP32 Gram seed (two-sided Jacobi in the shared
  // memory of the cluster's first CTA, written row-major to the seed buffer) instead
  // of the FP32 one-sided phase: a few hundred CTA-local rounds in place of ~8
  // sweeps of cluster rounds.
  const bool gram_seed =
      n <= ws_cl_seed_max && 2ull * n * n * (selfm ? sizeof(float) : sizeof(float2)) <= L.total - L.data;
  const float2* Vs = reinterpret_cast<const float2*>(sl.V) + sl.f(BF_GOFF, t);
  int sw32 = 0;
  const bool timed = st.ctr && kr == 0 && tid == 0;
  long long tc = timed ? clock64() : 0;
  auto lap = [&](int ctr) {
    if (timed) {
      const long long now = clock64();
      atomicAdd(st.ctr + ctr, (unsigned long long)(now - tc));
      tc = now;
    }
  };
  if (gram_seed) {
    if (kr == 0) seed_block(st, sl, g, t, smem, L);
    cluster_exchange(cl);
  } else {
  // W32 = Theta B, V32 = B on this CTA's columns
  for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {
    const int k = k0 + (int)(e / n), i = (int)(e % n);
    int idx[2]; float2 wt[2];
    const int ne = basis_col<float2, float>(k, mpos, selfm, idx, wt);
    float2 v = zero_e<float2>();
    for (int u = 0; u < ne; ++u) if (idx[u] == i) v = wt[u];
    V32[(long long)k * n + i] = v;
  }
  for (long long e = tid; e < (long long)(k1 - k0) * h; e += nth) {
    const int k = k0 + (int)(e / h), x = (int)(e % h);
    int idx[2]; float2 wt[2];
    const int ne = basis_col<float2, float>(k, mpos, selfm, idx, wt);
    float2 acc = zero_e<float2>();
    for (int u = 0; u < ne; ++u) {
      if (side == 1) cfma(acc, cvt<float2>(to_d2(Th[(long long)x * c + idx[u]])), wt[u]);
      else cfma_cj(acc, cvt<float2>(to_d2(Th[(long long)idx[u] * c + x])), wt[u]);
    }
    W32[(long long)k * h + x] = acc;
  }
  cluster_exchange(cl);
  float* red32 = reinterpret_cast<float*>(smem + L.nrm);
  const float mx32 = cluster_max_norm2<float>(cl, W32, h, k0, k1, hdr, red32);
  sw32 = cluster_sweeps<float>(cl, W32, V32, n, h, selfm, Prec<float>::os_abs * mx32,
                               (float)(Prec<float>::floor * mx32), smem, L, hdr, &rot32);
  }
  lap(CTR_CYC_SEED);
  int sw64 = 0;
  if constexpr (sizeof(R) == 8) {
    // the FP64 path polishes in double-float arithmetic (see polish_dd)
    sw64 = polish_dd(cl, st, sl, t, reinterpret_cast<double2*>(const_cast<C*>(Th)), reinterpret_cast<double2*>(gW),
                     reinterpret_cast<double2*>(gV), Vs, V32, gram_seed, n, h, r, c, side, selfm, k0, k1, smem, L,
                     hdr, &rot64, &tc, timed);
  } else {
  R* nrm = reinterpret_cast<R*>(reinterpret_cast<C*>(sl.NS) + sl.f(BF_GOFF, t));
  {
    // Polish in the path precision: two Newton-Schulz steps V <- V (3 I - V^dag V) / 2
    // remove the non-unitarity that the FP32 rotations accumulated in V (S in the NS
    // buffer, the product in this block's W region, W32 being dead now); then
    // W = Theta V is formed afresh and the sweeps repeat (one or two, typically).
    C* S = reinterpret_cast<C*>(sl.NS) + sl.f(BF_GOFF, t);
    C* T = gW;
    if (gram_seed) {
      for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {  // column-major from row-major
        const int k = k0 + (int)(e / n), i = (int)(e % n);
        gV[(long long)k * n + i] = cvt<C>(to_d2(Vs[(long long)i * n + k]));
      }
    } else if ((const void*)gV != (const void*)V32) {
      for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {
        const long long o = (long long)k0 * n + e;
        gV[o] = cvt<C>(to_d2(V32[o]));
      }
    }
    cluster_exchange(cl);
    for (int it = 0; it < 2; ++it) {
      for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {  // S[:, k] = V^dag v_k
        const int k = k0 + (int)(e / n), a = (int)(e % n);
        C acc = zero_e<C>();
        for (int i = 0; i < n; ++i) cfma_cj(acc, gV[(long long)a * n + i], gV[(long long)k * n + i]);
        S[(long long)k * n + a] = acc;
      }
      cluster_exchange(cl);
      for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {  // T[:, k] = V (3 e_k - S[:, k]) / 2
        const int k = k0 + (int)(e / n), i = (int)(e % n);
        C acc = zero_e<C>();
        for (int a = 0; a < n; ++a) {
          C w = S[(long long)k * n + a];
          w.x = (a == k ? (R)1.5 : (R)0) - (R)0.5 * w.x;
          w.y = -(R)0.5 * w.y;
          cfma(acc, gV[(long long)a * n + i], w);
        }
        T[(long long)k * n + i] = acc;
      }
      cluster_exchange(cl);
      for (long long e = tid; e < (long long)(k1 - k0) * n; e += nth) {
        const long long o = (long long)k0 * n + e;
        gV[o] = T[o];
      }
      cluster_exchange(cl);
    }
    lap(CTR_CYC_NS);
    form_w_cols<C, C>(Th, gV, gW, r, c, side, n, h, k0, k1);
    cluster_exchange(cl);
    R* red = reinterpret_cast<R*>(smem + L.nrm);
    const R mx = cluster_max_norm2<R>(cl, gW, h, k0, k1, hdr, red);
    sw64 = cluster_sweeps<R>(cl, gW, gV, n, h, selfm, Prec<R>::os_abs * mx, (R)Prec<R>::floor * mx, smem, L, hdr,
                             &rot64);
    if (sw64 >= JACOBI_MAX_SWEEPS && tid == 0) dev_set_error(st.err, DEV_ERR_NUMERIC, 3600 + t);
  }
  lap(CTR_CYC_POLISH);
  cluster_rank<R>(cl, st, sl, t, gW, nrm, n, h, k0, k1);
  }
  if (st.ctr && tid == 0) {
    // the FP32 phase counts as the seed, the polish (Newton-Schulz, W = Theta V and
    // the final sweeps, in the path's precision) as the refinement
    const unsigned long long per = 48ull * h + 24ull * n;
    atomicAdd(st.ctr + CTR_EIG, rot32 * per);
    atomicAdd(st.ctr + CTR_REFINE, rot64 * per + 8ull * (unsigned long long)h * n * (k1 - k0) +
                                       32ull * (unsigned long long)n * n * (k1 - k0));
    if (kr == 0) {
      if (!gram_seed) {  // (seed_block counts its own sweeps and block)
        atomicAdd(st.ctr + CTR_SWEEPS, (unsigned long long)(sw32 + 1));
        atomicAdd(st.ctr + CTR_EIGBLK, 1ull);
      }
      atomicAdd(st.ctr + CTR_RSWEEPS, (unsigned long long)(sw64 + 1));
    }
  }
  cluster_exchange(cl);
}

// ---------------------------------------------------------------- double-float refinement (FP64 path, one CTA)
// refine_sweeps in double-float arithmetic: per round, one warp per pair forms the
// inner product (compensated, dd.cuh; the squared column norms are carried through
// the sweep and recomputed at its start), one thread per pair the rotation parameters
// and the new norms on the FP32 pipe (dd_os_params), one warp per pair applies the
// rotation in double-float.  Same thresholds and stopping rule as the FP64 sweeps.
struct PairWorkDD {
  dd gr, gi, c, s;
  ddc e;
  int act;
};
static_assert(sizeof(PairWorkDD) <= sizeof(PairWork<double>), "pair work area");
__device__ int refine_sweeps_dd(ddc* W, ddc* Vc, int n, int h, bool selfm, double tol_abs, double col_floor,
                                PairWorkDD* pw, int* flags, dd* cnrm) {
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  const int np = n + (n & 1), half = np / 2;
  const float tol_f = (float)tol_abs, floor_f = (float)col_floor;
  int sweep = 0;
  for (; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
    __syncthreads();
    if (tid == 0) { flags[0] = 0; flags[2] = 0; }
    for (int k = warp; k < n; k += nwarp) {  // squared column norms, carried through the sweep
      const dd v = ddc_col_norm2_dd(W + (long long)k * h, h, lane);
      if (lane == 0) cnrm[k] = v;
    }
    __syncthreads();
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int c0 = 0; c0 < half; c0 += PAIR_CHUNK) {
        const int cn = (half - c0) < PAIR_CHUNK ? (half - c0) : PAIR_CHUNK;
        for (int k = warp; k < cn; k += nwarp) {
          int p, qq;
          circle_pair(rnd, c0 + k, np, p, qq);
          if (qq >= n) { if (lane == 0) pw[k].act = 0; continue; }
          const ddc* wp = W + (long long)p * h;
          const ddc* wq = W + (long long)qq * h;
          dd_acc gr = dd_acc_zero(), gi = dd_acc_zero();
          for (int x = lane; x < h; x += 32) {
            const ddc a = wp[x], b = wq[x];
            dd_acc_mac(gr, a.re, b.re);
            dd_acc_mac(gr, a.im, b.im);
            dd_acc_mac(gi, a.re, b.im);
            dd_acc_mac(gi, dd_neg(a.im), b.re);
          }
          const dd g_re = dd_warp_sum(dd_acc_value(gr)), g_im = dd_warp_sum(dd_acc_value(gi));
          if (lane == 0) { pw[k].gr = g_re; pw[k].gi = g_im; pw[k].act = 1; }
        }
        __syncthreads();
        for (int k = tid; k < cn; k += nth) {
          if (!pw[k].act) continue;
          int p, qq;  // each column is in one pair of the round: no other thread touches its norm
          circle_pair(rnd, c0 + k, np, p, qq);
          dd al = cnrm[p], be = cnrm[qq], c, s, gabs;
          ddc e;
          float r2 = 0.f;
          const bool rot = dd_os_params(al, be, pw[k].gr, pw[k].gi, selfm, tol_f, floor_f,
                                        (float)Prec<double>::os_rel, c, s, e, gabs, r2);
          atomicMax(reinterpret_cast<unsigned*>(&flags[2]), __float_as_uint(r2));
          if (rot) {
            pw[k].c = c; pw[k].s = s; pw[k].e = e;
            flags[0] = 1;
            atomicAdd(&flags[1], 1);
            rotated_norms_dd(al, be, gabs, c, s);
            cnrm[p] = al;
            cnrm[qq] = be;
          } else {
            pw[k].act = 0;
          }
        }
        __syncthreads();
        for (int k = warp; k < cn; k += nwarp) {
          if (!pw[k].act) continue;
          int p, qq;
          circle_pair(rnd, c0 + k, np, p, qq);
          ddc_rotate_dd(W + (long long)p * h, W + (long long)qq * h, h, lane, pw[k].c, pw[k].s, pw[k].e);
          ddc_rotate_dd(Vc + (long long)p * n, Vc + (long long)qq * n, n, lane, pw[k].c, pw[k].s, pw[k].e);
        }
        __syncthreads();
      }
    }
    if (!flags[0]) break;
    if ((double)__uint_as_float((unsigned)flags[2]) < Prec<dd>::stop2) { ++sweep; break; }
  }
  __syncthreads();
  return sweep;
}

// The FP64 path's refinement of one block on one CTA, in double-float: the steps of
// refine_block (Newton-Schulz on the FP32 seed, W = Theta V, one-sided sweeps, column
// norms) with the vectors as complex double-floats; Theta is converted in place, W
// and V go back to complex128 for the re-split.
__device__ void refine_block_dd(const MpoDev& st, const Slot& sl, const GateDesc& g, int t, unsigned char* smem,
                                const SvdLayout& L, bool seeded) {
  const int n = sl.f(BF_G, t);
  const int r = sl.f(BF_R, t), c = sl.f(BF_C, t), side = sl.f(BF_SIDE, t);
  const int h = side == 0 ? c : r;
  const bool selfm = pair_mirror(sl.f(BF_M, t), st.ncap) == sl.f(BF_M, t);
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  int* flags = reinterpret_cast<int*>(smem + L.hdr);
  double* nrm = reinterpret_cast<double*>(smem + L.nrm);
  PairWorkDD* pw = reinterpret_cast<PairWorkDD*>(smem + L.pw);  // smaller than PairWork<double>
  const size_t room = L.total - L.data;
  const bool w_smem = (size_t)h * n * sizeof(ddc) <= room;
  const bool in_smem = ((size_t)h * n + (size_t)n * n) * sizeof(ddc) <= room;
  double2* Th = reinterpret_cast<double2*>(sl.theta) + sl.f(BF_TOFF, t);
  ddc* Thd = reinterpret_cast<ddc*>(Th);
  const float2* V0 = reinterpret_cast<const float2*>(sl.V) + sl.f(BF_GOFF, t);  // row-major FP32 seed
  ddc* gW = reinterpret_cast<ddc*>(sl.W) + sl.f(BF_TOFF, t);
  ddc* gVc = reinterpret_cast<ddc*>(sl.VC) + sl.f(BF_GOFF, t);
  ddc* W = w_smem ? reinterpret_cast<ddc*>(smem + L.data) : gW;
  ddc* Vc = in_smem ? W + (size_t)h * n : gVc;
  if (tid == 0) { flags[0] = 0; flags[1] = 0; }
  if (!seeded) {
    int* mpos = reinterpret_cast<int*>(smem + L.mpos);
    if (selfm) block_mirror_map(st, sl, g, t, mpos, reinterpret_cast<int*>(smem + L.seg));
    for (int e = tid; e < n * n; e += nth) {
      const int k = e / n, i = e % n;
      int idx[2];
      double2 wt[2];
      const int ne = basis_col<double2, double>(k, mpos, selfm, idx, wt);
      double2 v = make_double2(0.0, 0.0);
      for (int u = 0; u < ne; ++u)
        if (idx[u] == i) v = wt[u];
      Vc[e] = ddc_conv(v);
    }
  } else {
    // two Newton-Schulz steps V <- V (3 I - V^dag V) / 2 in global scratch (S in the
    // NS buffer, the product in the W buffer, free until W is formed)
    ddc* S = reinterpret_cast<ddc*>(sl.NS) + sl.f(BF_GOFF, t);
    ddc* T = gW;
    for (int e = tid; e < n * n; e += nth) {
      const float2 v = V0[(long long)(e % n) * n + e / n];
      gVc[e] = ddc_make(dd_make(v.x, 0.f), dd_make(v.y, 0.f));
    }
    __syncthreads();
    for (int it = 0; it < 2; ++it) {
      for (int e = tid; e < n * n; e += nth) {  // S[:, b] = V^dag v_b, Hermitian: a <= b formed, mirrored
        const int b = e / n, a = e % n;
        if (a > b) continue;
        const ddc v = ddc_dot(gVc + (long long)a * n, 1, gVc + (long long)b * n, 1, n, true);
        S[e] = v;
        S[(long long)a * n + b] = ddc_conj(v);
      }
      __syncthreads();
      for (int e = tid; e < n * n; e += nth) T[e] = ns_update(gVc, S, n, e / n, e % n);
      __syncthreads();
      for (int e = tid; e < n * n; e += nth) gVc[e] = T[e];
      __syncthreads();
    }
    if (in_smem)
      for (int e = tid; e < n * n; e += nth) Vc[e] = gVc[e];
  }
  for (long long e = tid; e < (long long)r * c; e += nth) Thd[e] = ddc_conv(Th[e]);  // Theta to double-float
  __syncthreads();
  for (int e = tid; e < h * n; e += nth) {  // W = Theta V or Theta^dag V
    const int k = e / h, x = e % h;
    W[e] = side == 1 ? ddc_dot(Thd + (long long)x * c, 1, Vc + (long long)k * n, 1, n, false)
                     : ddc_dot(Thd + x, c, Vc + (long long)k * n, 1, n, true);
  }
  __syncthreads();
  double mx = 0;
  for (int k = warp; k < n; k += nwarp) mx = fmax(mx, ddc_col_norm2(W + (long long)k * h, h, lane));
  if (lane == 0) nrm[warp] = mx;
  __syncthreads();
  mx = 0;
  for (int w2 = 0; w2 < nwarp; ++w2) mx = fmax(mx, nrm[w2]);
  __syncthreads();
  const int sweeps =
      refine_sweeps_dd(W, Vc, n, h, selfm, Prec<dd>::os_abs * mx, Prec<dd>::floor * mx, pw, flags,
                       reinterpret_cast<dd*>(nrm));
  if (sweeps >= JACOBI_MAX_SWEEPS && tid == 0) dev_set_error(st.err, DEV_ERR_NUMERIC, 3500 + t);
  for (int k = warp; k < n; k += nwarp) {
    const double a = ddc_col_norm2(W + (long long)k * h, h, lane);
    if (lane == 0) nrm[k] = a;
  }
  __syncthreads();
  const int coff = sl.f(BF_COFF, t);
  for (int i = tid; i < n; i += nth) {
    const double wi = nrm[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (nrm[j] > wi) || (nrm[j] == wi && j < i);
    if (!isfinite(wi)) dev_set_error(st.err, DEV_ERR_NUMERIC, 4500 + t);
    sl.sval[coff + rank] = sqrt(wi);
    sl.perm[coff + rank] = i;
  }
  // back to complex128 for the re-split (each element read and rewritten by one thread)
  double2* gWd = reinterpret_cast<double2*>(gW);
  double2* gVd = reinterpret_cast<double2*>(gVc);
  for (int e = tid; e < h * n; e += nth) gWd[e] = ddc_back(W[e]);
  for (int e = tid; e < n * n; e += nth) gVd[e] = ddc_back(Vc[e]);
  if (st.ctr && tid == 0) {
    atomicAdd(st.ctr + CTR_REFINE, (unsigned long long)flags[1] * (48ull * h + 24ull * n) +
                                       8ull * (unsigned long long)h * n * n);
    atomicAdd(st.ctr + CTR_RSWEEPS, (unsigned long long)(sweeps + 1));
  }
  __syncthreads();
}

// ---------------------------------------------------------------- refinement
// One-sided Jacobi (Hestenes) refinement of each canonical block's SVD.  The Gram
// eigenvectors V (n x n, FP32 seed) give W = Theta V (side 1, n = cols) or
// W = Theta^dag V (side 0, n = rows), whose n columns are orthogonal up to the seed's
// error.  Sweeps of pairwise rotations that orthogonalise the columns of W (the 2x2
// Gram [[|w_p|^2, w_p^dag w_q], [., |w_q|^2]] recomputed from W at each step, the same
// rotation applied to V) converge quadratically to the SVD of Theta without squaring
// its condition number: s_k = |w_k|.  Both factors come out: side 1:
// X[:, k] = w_k / s_k, Y[k, :] = conj(v_k);  side 0: X[:, k] = v_k,
// Y[k, :] = conj(w_k) / s_k.  W (h x n) and V (n x n) are column-major, in shared
// memory when they fit, else in the slot scratch (W buffer, VC buffer).  For
// self-mirror blocks the columns are mirror-symmetric, so w_p^dag w_q is real in exact
// arithmetic; its imaginary part (rounding) is dropped to keep the rotations real.
template <typename R>
__device__ void refine_block(const MpoDev& st, const Slot& sl, const GateDesc& g, int t, unsigned char* smem,
                             const SvdLayout& L, bool seeded) {
  if constexpr (sizeof(R) == 8) {  // the FP64 path refines in double-float (refine_block_dd)
    refine_block_dd(st, sl, g, t, smem, L, seeded);
    return;
  }
  typedef typename Prec<R>::C C;
  const int n = sl.f(BF_G, t);
  const int r = sl.f(BF_R, t), c = sl.f(BF_C, t), side = sl.f(BF_SIDE, t);
  const int h = side == 0 ? c : r;
  const bool selfm = pair_mirror(sl.f(BF_M, t), st.ncap) == sl.f(BF_M, t);
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  int* flags = reinterpret_cast<int*>(smem + L.hdr);
  R* nrm = reinterpret_cast<R*>(smem + L.nrm);
  PairWork<R>* pw = reinterpret_cast<PairWork<R>*>(smem + L.pw);
  const size_t room = L.total - L.data;
  const bool w_smem = (size_t)h * n * sizeof(C) <= room;
  const bool in_smem = ((size_t)h * n + (size_t)n * n) * sizeof(C) <= room;  // V too
  const C* Th = reinterpret_cast<const C*>(sl.theta) + sl.f(BF_TOFF, t);
  const float2* V0 = reinterpret_cast<const float2*>(sl.V) + sl.f(BF_GOFF, t);  // row-major FP32 seed
  C* gW = reinterpret_cast<C*>(sl.W) + sl.f(BF_TOFF, t);
  C* gVc = reinterpret_cast<C*>(sl.VC) + sl.f(BF_GOFF, t);
  C* W = w_smem ? reinterpret_cast<C*>(smem + L.data) : gW;
  C* Vc = in_smem ? W + (size_t)h * n : gVc;
  if (tid == 0) { flags[0] = 0; flags[1] = 0; }
  if (!seeded) {
    // no seed (the Gram eigensolver did not fit): one-sided Jacobi from the basis B
    // (identity, or the mirror-real basis of a self-mirror block, which the real
    // rotations below require)
    int* mpos = reinterpret_cast<int*>(smem + L.mpos);
    if (selfm) block_mirror_map(st, sl, g, t, mpos, reinterpret_cast<int*>(smem + L.seg));
    for (int e = tid; e < n * n; e += nth) {
      const int k = e / n, i = e % n;
      int idx[2];
      C wt[2];
      const int ne = basis_col<C, R>(k, mpos, selfm, idx, wt);
      C v = zero_e<C>();
      for (int u = 0; u < ne; ++u)
        if (idx[u] == i) v = wt[u];
      Vc[e] = v;
    }
  } else if (sizeof(R) == 8) {
    // The FP32 seed is unitary only to ~1e-7 and the rotations below keep any
    // non-unitarity, so it is first orthonormalised in FP64 by two Newton-Schulz
    // steps V <- V (3 I - V^dag V) / 2 (error delta -> ~delta^2 per step), in global
    // scratch: S = V^dag V in the slot's NS buffer, V S in the W buffer (free until W
    // is formed below).
    C* S = reinterpret_cast<C*>(sl.NS) + sl.f(BF_GOFF, t);
    C* T = gW;
    for (int e = tid; e < n * n; e += nth) T[e] = cvt<C>(to_d2(V0[(long long)(e % n) * n + e / n]));
    __syncthreads();
    for (int e = tid; e < n * n; e += nth) gVc[e] = T[e];
    __syncthreads();
    for (int it = 0; it < 2; ++it) {
      for (int e = tid; e < n * n; e += nth) {  // S[a][b] = v_a^dag v_b (column-major)
        const int b = e / n, a = e % n;
        C acc = zero_e<C>();
        for (int i = 0; i < n; ++i) cfma_cj(acc, gVc[(long long)a * n + i], gVc[(long long)b * n + i]);
        S[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < n * n; e += nth) {  // T[:, b] = sum_a V[:, a] (3 delta_ab - S_ab) / 2
        const int b = e / n, i = e % n;
        C acc = zero_e<C>();
        for (int a = 0; a < n; ++a) {
          C w = S[(long long)b * n + a];
          w.x = (a == b ? (R)1.5 : (R)0) - (R)0.5 * w.x;
          w.y = -(R)0.5 * w.y;
          cfma(acc, gVc[(long long)a * n + i], w);
        }
        T[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < n * n; e += nth) gVc[e] = T[e];
      __syncthreads();
    }
    if (in_smem) {
      for (int e = tid; e < n * n; e += nth) Vc[e] = gVc[e];
    }
  } else {
    for (int e = tid; e < n * n; e += nth) {  // column-major copy of V
      const int k = e / n, i = e % n;
      Vc[e] = cvt<C>(to_d2(V0[(long long)i * n + k]));
    }
  }
  __syncthreads();
  for (int e = tid; e < h * n; e += nth) {
    const int k = e / h, x = e % h;
    C acc = zero_e<C>();
    if (side == 1) {
      for (int q = 0; q < n; ++q) cfma(acc, Th[(long long)x * c + q], Vc[(long long)k * n + q]);
    } else {
      for (int i = 0; i < n; ++i) cfma_cj(acc, Th[(long long)i * c + x], Vc[(long long)k * n + i]);
    }
    W[e] = acc;
  }
  __syncthreads();
  // largest column norm^2 (scale of the absolute thresholds)
  R mx = 0;
  for (int k = warp; k < n; k += nwarp) {
    R a = 0;
    for (int x = lane; x < h; x += 32) { const C w = W[(long long)k * h + x]; a += w.x * w.x + w.y * w.y; }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    mx = fmax(mx, a);
  }
  if (lane == 0) nrm[warp] = mx;
  __syncthreads();
  mx = 0;
  for (int w2 = 0; w2 < nwarp; ++w2) mx = fmax(mx, nrm[w2]);
  __syncthreads();
  // columns at or below the selection floor are dropped anyway: rotating them only
  // churns rounding noise, so pairs involving one are skipped
  int sweeps;
  if (sizeof(R) == 8)
    sweeps = refine_sweeps<R>(W, Vc, n, h, selfm, Prec<R>::os_abs * mx, (R)Prec<R>::floor * mx, pw, flags);
  else
    sweeps = refine_sweeps_fp32(reinterpret_cast<float2*>(W), reinterpret_cast<float2*>(Vc), n, h, selfm,
                                (float)(Prec<R>::os_abs * mx), (float)(Prec<R>::floor * mx), flags);
  if (sweeps >= JACOBI_MAX_SWEEPS && sizeof(R) == 8 && tid == 0) dev_set_error(st.err, DEV_ERR_NUMERIC, 3500 + t);
  // singular values = column norms, ranked descending (ties by index)
  for (int k = warp; k < n; k += nwarp) {
    R a = 0;
    for (int x = lane; x < h; x += 32) { const C w = W[(long long)k * h + x]; a += w.x * w.x + w.y * w.y; }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) nrm[k] = a;
  }
  __syncthreads();
  const int coff = sl.f(BF_COFF, t);
  for (int i = tid; i < n; i += nth) {
    const R wi = nrm[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (nrm[j] > wi) || (nrm[j] == wi && j < i);
    if (!isfinite((double)wi)) dev_set_error(st.err, DEV_ERR_NUMERIC, 4500 + t);
    sl.sval[coff + rank] = sqrt((double)wi);
    sl.perm[coff + rank] = i;
  }
  if (w_smem) {
    for (int e = tid; e < h * n; e += nth) gW[e] = W[e];
  }
  if (in_smem) {
    for (int e = tid; e < n * n; e += nth) gVc[e] = Vc[e];
  }
  if (st.ctr && tid == 0) {
    // per applied rotation: 3 inner products (24 h) and 2 x 12 (h + n) for the updates
    atomicAdd(st.ctr + CTR_REFINE, (unsigned long long)flags[1] * (48ull * h + 24ull * n) +
                                       8ull * (unsigned long long)h * n * n);
    atomicAdd(st.ctr + CTR_RSWEEPS, (unsigned long long)(sweeps + 1));
  }
  __syncthreads();
}

// ---------------------------------------------------------------- small blocks on one warp
// On the FP32 path a block of Gram side n <= 64 whose matrices fit in a slice of the
// CTA's shared memory is factorised by a single warp, several blocks per CTA at a time,
// with warp synchronisation only:
//  * the FP32 Gram seed: two-sided parallel-order Jacobi on G (n x n, rows padded to
//    n + 1), in the mirror-real basis for self-mirror blocks (real arithmetic): one
//    lane per pair for the rotation parameters, lanes over rows / columns for the
//    updates of each round;
//  * W = Theta V (or Theta^dag V) and one-sided FP32 sweeps with one lane per column
//    pair of a round, stopped as in the CTA refinement.
// Slices: eight of 1/8 of the CTA's space for the smaller blocks, four of 1/4 for the
// rest (a separate phase).  The results go where the CTA path puts them (sval, perm,
// W, VC).
constexpr int WARP_SVD_N = 64;
constexpr int SVD_WARPS = 8;  // shared-memory slices of the warp-block phase
// Threads of a k_svd CTA.  One CTA holds an SM (its ~200 KB shared-memory block), so
// the CTA's warps are the SM's parallelism: the Jacobi rounds give each warp a pair at
// a time, and with 16 warps a round of b pairs takes half the turns it takes with 8.
// Measured on GB300 (48 modes, chi = 512, updates/s):
//   threads        256   512   768   1024
//   FP64 path      196   234   222   223    (128 registers at 512, no spills)
//   TF32 path      514   692   771   784
// The FP64 path's double-float polish needs the registers of 512 threads; the FP32
// path's Jacobi gains from more warps despite a few spilled registers at 1024.
template <typename R> struct SvdThreads;
template <> struct SvdThreads<double> { static constexpr int value = 512; };
template <> struct SvdThreads<float> { static constexpr int value = 1024; };
static_assert(SvdThreads<double>::value >= 32 * SVD_WARPS && SvdThreads<float>::value <= 1024, "k_svd CTA size");
// Threads of a k_svd launch (every code path of the kernel works for any multiple of
// 32 from 32 * SVD_WARPS up to the bound above).  The FP64 path with bonds of at most
// 64 has blocks of Gram side <= ~30, whose rounds keep few warps busy while every
// barrier waits for all of them: 256 threads there (16 modes, chi = 64: 8449 against
// 7670 updates/s with 512; the FP32 path is faster with 1024 there too).
template <typename R>
__host__ inline int svd_threads(int D) {
  return (sizeof(R) == 8 && D <= 64) ? 256 : SvdThreads<R>::value;
}

// A warp's slice: [header: rotation parameters of up to 32 pairs, the mirror map and
// the column norms, 1280 B | seed A and V (padded rows), later W (n columns of stride
// h | 1) | V (n columns of stride n | 1)].  The V offset clears both the seed and W;
// the odd strides keep the lanes of the refinement, one per column pair, on distinct
// shared-memory banks.
constexpr size_t WARP_HDR_BYTES = 1280;
__host__ __device__ __forceinline__ size_t warp_vc_offset(int n, int h) {
  const size_t seed = 2ull * n * (n + 1) * sizeof(float2);
  const size_t w = (size_t)(h + 1) * n * sizeof(float2);
  return (seed > w ? seed : w);
}
__host__ __device__ __forceinline__ size_t warp_svd_bytes(int n, int h) {
  return WARP_HDR_BYTES + warp_vc_offset(n, h) + (size_t)n * (n + 1) * sizeof(float2);
}

// header layout (byte offsets)
constexpr int WH_CS = 0;      // 32 float2 (c, s)
constexpr int WH_E = 256;     // 32 complex (or real) phases
constexpr int WH_PQ = 512;    // 64 ints (p, q; q < 0: no rotation)
constexpr int WH_MP = 768;    // 64 ints: mirror partner of each small-side index
constexpr int WH_NRM = 1024;  // 64 floats: column norms^2

template <typename E>
__device__ int warp_jacobi(E* A, E* V, int n, int ld, unsigned char* hdr, int lane) {
  const int np = n + (n & 1), half = np / 2;
  float2* cs = reinterpret_cast<float2*>(hdr + WH_CS);
  E* ph = reinterpret_cast<E*>(hdr + WH_E);
  int* pq = reinterpret_cast<int*>(hdr + WH_PQ);
  for (int i = lane; i < n; i += 32)
    for (int j = 0; j < n; ++j) V[i * ld + j] = (i == j) ? unit_e<E>() : zero_e<E>();
  float dm = 0.f;
  for (int i = 0; i < n; ++i) dm = fmaxf(dm, absv(re(A[i * ld + i])));
  const float tol_abs = Prec<float>::tol_abs * dm, tol_rel = Prec<float>::tol_rel;
  int sweep = 0;
  __syncwarp();
  for (; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
    bool any = false;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      if (lane < half) {
        int p, q;
        circle_pair(rnd, lane, np, p, q);
        int qq = -1;
        float c = 1.f, s = 0.f;
        E e = unit_e<E>();
        if (q < n) {
          const float a = re(A[p * ld + p]), b = re(A[q * ld + q]);
          const E gpq = A[p * ld + q];
          const float hh = absv(gpq);
          if (hh > tol_rel * sqrtf(fabsf(a * b)) && hh > tol_abs) {
            const float tau = (b - a) / (2.f * hh);
            const float tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + tt * tt);
            s = tt * c;
            e = divr<E, float>(gpq, hh);
            qq = q;
          }
        }
        pq[2 * lane] = p;
        pq[2 * lane + 1] = qq;
        cs[lane] = make_float2(c, s);
        ph[lane] = e;
        any = any || (qq >= 0);
      }
      __syncwarp();
      for (int k = 0; k < half; ++k) {
        const int q = pq[2 * k + 1];
        if (q < 0) continue;
        const int p = pq[2 * k];
        const float c = cs[k].x, s = cs[k].y;
        const E ec = cj(ph[k]);
        for (int i = lane; i < n; i += 32) {  // columns p, q of A and V
          const E x = A[i * ld + p], ys = mulv(A[i * ld + q], ec);
          A[i * ld + p] = lin(c, x, -s, ys);
          A[i * ld + q] = lin(s, x, c, ys);
          const E vx = V[i * ld + p], vys = mulv(V[i * ld + q], ec);
          V[i * ld + p] = lin(c, vx, -s, vys);
          V[i * ld + q] = lin(s, vx, c, vys);
        }
      }
      __syncwarp();
      for (int k = 0; k < half; ++k) {
        const int q = pq[2 * k + 1];
        if (q < 0) continue;
        const int p = pq[2 * k];
        const float c = cs[k].x, s = cs[k].y;
        const E e = ph[k];
        for (int i = lane; i < n; i += 32) {  // rows p, q of A
          const E x = A[p * ld + i], ye = mulv(e, A[q * ld + i]);
          A[p * ld + i] = lin(c, x, -s, ye);
          A[q * ld + i] = lin(s, x, c, ye);
        }
      }
      __syncwarp();
    }
    if (!__any_sync(0xffffffffu, any)) break;
  }
  return sweep;
}

// One block on one warp (FP32 path).  slice: this warp's shared-memory slice.
__device__ void warp_block(const MpoDev& st, const Slot& sl, const GateDesc& g, int t, unsigned char* slice,
                           int lane) {
  typedef float2 C;
  const int n = sl.f(BF_G, t), r = sl.f(BF_R, t), c = sl.f(BF_C, t), side = sl.f(BF_SIDE, t);
  const int h = side == 0 ? c : r;
  const int ncap = st.ncap, P = st.P, M = st.M;
  const bool selfm = pair_mirror(sl.f(BF_M, t), ncap) == sl.f(BF_M, t);
  const int ld = n + 1;
  unsigned char* hdr = slice;
  int* mp = reinterpret_cast<int*>(hdr + WH_MP);
  float* nrm = reinterpret_cast<float*>(hdr + WH_NRM);
  unsigned char* data = slice + WARP_HDR_BYTES;
  const C* gG = reinterpret_cast<const C*>(sl.G) + sl.f(BF_GOFF, t);
  const C* Th = reinterpret_cast<const C*>(sl.theta) + sl.f(BF_TOFF, t);
  C* Vc = reinterpret_cast<C*>(data + warp_vc_offset(n, h));  // V for the refinement
  const int ldv = n | 1, ldw = h | 1;  // odd strides (<= n + 1, h + 1: within the slice layout)
  const float hs = 0.70710678118654752440f;
  for (int i = lane; i < n; i += 32) mp[i] = i;
  if (selfm) {
    const long long bX = (long long)g.inst * (M + 1) + g.j + (side == 0 ? 0 : 2);
    for (int i = lane; i < n; i += 32) mp[i] = mirror_coord(sl, st, g, t, side, i, st.segoff + bX * (P + 1));
  }
  __syncwarp();
  // column k of the mirror-real basis B: e_k (k its own mirror), (e_k + e_p)/sqrt2 (k < p),
  // i (e_p - e_k)/sqrt2 (k > p), p the mirror of k
  auto basis = [&](int k, int* idx, C* wt) {
    const int p = mp[k];
    if (p == k) { idx[0] = k; wt[0] = make_float2(1.f, 0.f); return 1; }
    if (k < p) { idx[0] = k; wt[0] = make_float2(hs, 0.f); idx[1] = p; wt[1] = make_float2(hs, 0.f); return 2; }
    idx[0] = p; wt[0] = make_float2(0.f, hs); idx[1] = k; wt[1] = make_float2(0.f, -hs); return 2;
  };
  int sweeps;
  if (selfm) {
    float* A = reinterpret_cast<float*>(data);
    float* V = A + n * ld;
    for (int e = lane; e < n * n; e += 32) {  // A[i][j] = Re(b_i^dag G b_j)
      const int i = e / n, j = e % n;
      int ia[2], jb[2];
      C wa[2], wb[2];
      const int na = basis(i, ia, wa), nb = basis(j, jb, wb);
      float acc = 0.f;
      for (int x = 0; x < na; ++x)
        for (int y = 0; y < nb; ++y) acc += cmul(cmul(cj(wa[x]), gG[(long long)ia[x] * n + jb[y]]), wb[y]).x;
      A[i * ld + j] = acc;
    }
    __syncwarp();
    sweeps = warp_jacobi<float>(A, V, n, ld, hdr, lane);
    for (int e = lane; e < n * n; e += 32) {  // V = B V~, column-major
      const int k = e / n, i = e % n, pi = mp[i];
      C out;
      if (pi == i) out = make_float2(V[i * ld + k], 0.f);
      else if (i < pi) out = make_float2(hs * V[i * ld + k], hs * V[pi * ld + k]);
      else out = make_float2(hs * V[pi * ld + k], -hs * V[i * ld + k]);
      Vc[(size_t)k * ldv + i] = out;
    }
  } else {
    C* A = reinterpret_cast<C*>(data);
    C* V = A + n * ld;
    for (int e = lane; e < n * n; e += 32) A[(e / n) * ld + e % n] = gG[e];
    __syncwarp();
    sweeps = warp_jacobi<C>(A, V, n, ld, hdr, lane);
    for (int e = lane; e < n * n; e += 32) Vc[(size_t)(e / n) * ldv + e % n] = V[(e % n) * ld + e / n];
  }
  __syncwarp();
  if (st.ctr && lane == 0) {
    atomicAdd(st.ctr + CTR_SWEEPS, (unsigned long long)(sweeps + 1));
    atomicAdd(st.ctr + CTR_EIGBLK, 1ull);
  }
  // W = Theta V (side 1) or Theta^dag V (side 0), at the slice data start
  C* W = reinterpret_cast<C*>(data);
  for (long long e = lane; e < (long long)h * n; e += 32) {
    const int k = (int)(e / h), x = (int)(e % h);
    C acc = zero_e<C>();
    if (side == 1) {
      for (int q = 0; q < n; ++q) cfma(acc, Th[(long long)x * c + q], Vc[(size_t)k * ldv + q]);
    } else {
      for (int i = 0; i < n; ++i) cfma_cj(acc, Th[(long long)i * c + x], Vc[(size_t)k * ldv + i]);
    }
    W[(size_t)k * ldw + x] = acc;
  }
  __syncwarp();
  auto col_norms = [&]() {
    for (int k = lane; k < n; k += 32) {
      float a = 0.f;
      for (int x = 0; x < h; ++x) { const C w = W[(size_t)k * ldw + x]; a += w.x * w.x + w.y * w.y; }
      nrm[k] = a;
    }
    __syncwarp();
  };
  col_norms();
  float mx = 0.f;
  for (int k = 0; k < n; ++k) mx = fmaxf(mx, nrm[k]);
  const float tol_abs = (float)Prec<float>::os_abs * mx, col_floor = (float)(Prec<float>::floor * mx);
  // one-sided sweeps, one lane per column pair of the round
  const int np = n + (n & 1), half = np / 2;
  int rs = 0;
  unsigned long long nrot = 0;
  for (; rs < JACOBI_MAX_SWEEPS; ++rs) {
    bool any = false;
    float wr2 = 0.f;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      if (lane < half) {
        int p, q;
        circle_pair(rnd, lane, np, p, q);
        if (q < n) {
          C* wp = W + (size_t)p * ldw;
          C* wq = W + (size_t)q * ldw;
          float al = 0.f, be = 0.f;
          C ga = zero_e<C>();
          for (int x = 0; x < h; ++x) {
            const C a = wp[x], b = wq[x];
            al += a.x * a.x + a.y * a.y;
            be += b.x * b.x + b.y * b.y;
            cfma_cj(ga, a, b);
          }
          if (al > col_floor && be > col_floor)
            wr2 = fmaxf(wr2, rel_off2(al, be, selfm ? ga.x * ga.x : ga.x * ga.x + ga.y * ga.y));
          float cs_, sn;
          C e;
          if (os_params(al, be, ga, selfm, tol_abs, col_floor, cs_, sn, e)) {
            const C ec = cj(e);
            for (int x = 0; x < h; ++x) {
              const C a = wp[x], bs = mulv(wq[x], ec);
              wp[x] = lin(cs_, a, -sn, bs);
              wq[x] = lin(sn, a, cs_, bs);
            }
            C* vp = Vc + (size_t)p * ldv;
            C* vq = Vc + (size_t)q * ldv;
            for (int x = 0; x < n; ++x) {
              const C a = vp[x], bs = mulv(vq[x], ec);
              vp[x] = lin(cs_, a, -sn, bs);
              vq[x] = lin(sn, a, cs_, bs);
            }
            any = true;
            ++nrot;
          }
        }
      }
      __syncwarp();
    }
    any = __any_sync(0xffffffffu, any);
    for (int o = 16; o > 0; o >>= 1) wr2 = fmaxf(wr2, __shfl_xor_sync(0xffffffffu, wr2, o));
    if (!any) break;
    if ((double)wr2 < Prec<float>::stop2) { ++rs; break; }
  }
  for (int o = 16; o > 0; o >>= 1) nrot += __shfl_xor_sync(0xffffffffu, nrot, o);
  // singular values = column norms, ranked descending (ties by index)
  col_norms();
  const int coff = sl.f(BF_COFF, t);
  for (int i = lane; i < n; i += 32) {
    const float wi = nrm[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (nrm[j] > wi) || (nrm[j] == wi && j < i);
    if (!isfinite(wi)) dev_set_error(st.err, DEV_ERR_NUMERIC, 4700 + t);
    sl.sval[coff + rank] = sqrt((double)wi);
    sl.perm[coff + rank] = i;
  }
  C* gW = reinterpret_cast<C*>(sl.W) + sl.f(BF_TOFF, t);
  C* gVc = reinterpret_cast<C*>(sl.VC) + sl.f(BF_GOFF, t);
  for (long long e = lane; e < (long long)h * n; e += 32) gW[e] = W[(size_t)(e / h) * ldw + e % h];
  for (int e = lane; e < n * n; e += 32) gVc[e] = Vc[(size_t)(e / n) * ldv + e % n];
  if (st.ctr && lane == 0) {
    atomicAdd(st.ctr + CTR_REFINE, nrot * (48ull * h + 24ull * n) + 8ull * (unsigned long long)h * n * n);
    atomicAdd(st.ctr + CTR_RSWEEPS, (unsigned long long)(rs + 1));
  }
  __syncwarp();
}

// ---------------------------------------------------------------- k_order, k_svd
// The blocks of all gates of a layer go into one list: the large ones first, then the
// rest, each part longest first (bucketed by log2 of an n^2 (n + h) work estimate),
// for k_svd to take in that order (longest-processing-time scheduling).  counter:
// [0] next large item, [1] large items, [2] next small item (starts at [1]),
// [3] all items.  The order inside a bucket does not matter: every block's
// factorisation depends on its own data only.
// seed_max: the largest Gram side whose FP32 seed fits in one CTA's shared memory;
// a larger block would run its whole Jacobi unseeded on one SM, so it always goes
// to a cluster.
__device__ __forceinline__ bool route_big(const SlotWS& ws, int n, int h, int min_n, int always_n, int seed_max,
                                          unsigned long long total, int ncta) {
  if (ws.big_min > 0) return n >= ws.big_min;
  const unsigned long long w = svd_work(n, h) * (unsigned long long)ncta;
  return n >= min_n && (n > seed_max || w > total || (n >= always_n && 16ull * w > total));
}

// category: 0 cluster, 1 one CTA, 2 one warp in a quarter slice, 3 one warp in an
// eighth slice
__device__ __forceinline__ int order_key(int cat, int n, int h) {
  return cat * 64 + 63 - min(63, (int)log2((double)svd_work(n, h) + 1.0));
}

// ncta: CTAs of the k_svd launch; min_n: the path's smallest cluster block; always_n:
// the Gram side from which every block goes to a cluster; room: the shared memory a
// CTA has for block data on the FP32 path (0: the FP64 path, no warp blocks).
// counter: cursor and end of the cluster ([0], [1]), CTA ([2], [3]), quarter-slice
// warp ([4], [5]) and eighth-slice warp ([6], [7]) parts of list.
__global__ void __launch_bounds__(1024) k_order(SlotWS ws, int ngates, int* list, int* counter, int ncta,
                                                int min_n, int always_n, int seed_max, int room) {
  __shared__ int hist[256], start[256];
  __shared__ unsigned long long total;
  const int tid = threadIdx.x, lane = tid & 31, Pc = ws.Pc, E = ngates * Pc;
  if (tid < 256) hist[tid] = 0;
  if (tid == 0) total = 0;
  __syncthreads();
  // every warp walks whole rounds of 32 entries so that the warp-level reductions and
  // key matching below always run with all lanes (entries past E are invalid)
  const int Er = (E + 31) & ~31;
  auto entry = [&](int e, int& n, int& h) {
    n = 0; h = 0;
    if (e >= E) return;
    Slot sl = get_slot(ws, e / Pc);
    const int t = e % Pc;
    if (sl.scal[SS_STATUS]) return;
    n = sl.f(BF_G, t);
    h = sl.f(BF_SIDE, t) == 0 ? sl.f(BF_C, t) : sl.f(BF_R, t);
  };
  for (int e = tid; e < Er; e += blockDim.x) {
    int n, h;
    entry(e, n, h);
    unsigned long long w = n > 0 ? svd_work(n, h) : 0ull;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0 && w) atomicAdd(&total, w);
  }
  __syncthreads();
  const unsigned long long tot = total;
  const size_t eighth = (((size_t)room / SVD_WARPS) & ~(size_t)15), quarter = (((size_t)room / 4) & ~(size_t)15);
  auto category = [&](int n, int h) {
    if (route_big(ws, n, h, min_n, always_n, seed_max, tot, ncta)) return 0;
    // a block on the layer's critical path keeps a whole CTA (lower latency than one warp)
    const bool critical = svd_work(n, h) * (unsigned long long)ncta > tot;
    if (room > 0 && n <= WARP_SVD_N && !critical) {
      const size_t b = warp_svd_bytes(n, h);
      if (b <= eighth) return 3;
      if (b <= quarter) return 2;
    }
    return 1;
  };
  // warp-aggregated atomics: one per distinct key in the warp (keys cluster heavily)
  auto key_of = [&](int e) {
    int n, h;
    entry(e, n, h);
    return n > 0 ? order_key(category(n, h), n, h) : -1;
  };
  for (int e = tid; e < Er; e += blockDim.x) {
    const int key = key_of(e);
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && lane == __ffs(grp) - 1) atomicAdd(&hist[key], __popc(grp));
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int k = 0; k < 256; ++k) {
      if (k % 64 == 0 && k > 0) { counter[2 * (k / 64) - 1] = acc; counter[2 * (k / 64)] = acc; }
      start[k] = acc;
      acc += hist[k];
    }
    counter[0] = 0;
    counter[7] = acc;
  }
  __syncthreads();
  for (int e = tid; e < Er; e += blockDim.x) {
    const int key = key_of(e);
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (key >= 0 && lane == leader) base = atomicAdd(&start[key], __popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (key >= 0) list[base + __popc(grp & ((1u << lane) - 1u))] = e;
  }
}

// Persistent: launched as clusters of K CTAs (one CTA per SM).  Each cluster first
// takes large blocks one at a time and factorises each on all its CTAs (big_block);
// when none is left, every CTA takes small blocks on its own (FP32 Gram seed when
// it fits in shared memory, then the one-sided refinement).  Every cluster barrier
// is reached by all CTAs of the cluster: the work item is broadcast from the
// cluster's first CTA and every loop bound inside big_block is cluster-uniform.
template <typename R>
__global__ void __launch_bounds__(SvdThreads<R>::value, 1) k_svd(MpoDev st, SlotWS ws, const GateDesc* __restrict__ gates,
                                             const int* __restrict__ list, int* counter, int smem_bytes) {
  extern __shared__ __align__(256) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const SvdLayout L = svd_layout<R>(ws.D, (size_t)smem_bytes);
  int* hdr = reinterpret_cast<int*>(smem + L.hdr);
  if (threadIdx.x == 0) { hdr[HDR_TOT] = 0; hdr[HDR_RTOT] = 0; }
  const int nbig = counter[1], ncta_end = counter[3], nwide_end = counter[5], total = counter[7];
  for (;;) {
    if (cl.block_rank() == 0 && threadIdx.x == 0) hdr[HDR_ITEM] = atomicAdd(&counter[0], 1);
    cl.sync();
    if (threadIdx.x == 0) hdr[HDR_ITEM + 1] = *cl.map_shared_rank(&hdr[HDR_ITEM], 0);
    cl.sync();  // the leader's item has been read everywhere before it changes
    const int idx = hdr[HDR_ITEM + 1];
    if (idx >= nbig) break;
    const int e = list[idx];
    const int s = e / ws.Pc, t = e % ws.Pc;
    Slot sl = get_slot(ws, s);
    const GateDesc g = gates[s];
    const long long c0 = clock64();
    big_block<R>(cl, st, sl, g, t, smem, L, ws.cl_seed_max);
    if (st.ctr && threadIdx.x == 0 && cl.block_rank() == 0) {
      atomicAdd(st.ctr + CTR_CYC_BIG, (unsigned long long)(clock64() - c0));
      atomicAdd(st.ctr + CTR_NBIG, 1ull);
    }
  }
  for (;;) {
    if (threadIdx.x == 0) hdr[HDR_ITEM] = atomicAdd(&counter[2], 1);
    __syncthreads();
    const int idx = hdr[HDR_ITEM];
    __syncthreads();
    if (idx >= ncta_end) break;
    const int e = list[idx];
    const int s = e / ws.Pc, t = e % ws.Pc;
    Slot sl = get_slot(ws, s);
    const GateDesc g = gates[s];
    // the FP32 Gram seed runs only when its matrices fit in shared memory; a seed in
    // global memory costs more than the extra one-sided sweeps it would save
    const int n = sl.f(BF_G, t);
    const bool selfm = pair_mirror(sl.f(BF_M, t), st.ncap) == sl.f(BF_M, t);
    const bool seeded = 2ull * n * n * (selfm ? sizeof(float) : sizeof(float2)) <= L.total - L.data;
    const long long c0 = clock64();
    if (seeded) seed_block(st, sl, g, t, smem, L);
    refine_block<R>(st, sl, g, t, smem, L, seeded);
    if (st.ctr && threadIdx.x == 0) atomicAdd(st.ctr + CTR_CYC_SMALL, (unsigned long long)(clock64() - c0));
  }
  // small blocks on the FP32 path: one warp each, in a quarter (warps 0-3) and then
  // an eighth (all warps) of the shared memory
  if (sizeof(R) == 4 && total > ncta_end) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto warp_phase = [&](int* cursor, int end, int nslices) {
      const size_t slice_bytes = ((L.total - L.data) / nslices) & ~(size_t)15;
      if (warp >= nslices) return;
      unsigned char* slice = smem + L.data + warp * slice_bytes;
      for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(cursor, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= end) break;
        const int e = list[idx];
        const int s = e / ws.Pc, t = e % ws.Pc;
        Slot sl = get_slot(ws, s);
        const GateDesc g = gates[s];
        const long long c0 = clock64();
        warp_block(st, sl, g, t, slice, lane);
        if (st.ctr && lane == 0) {
          atomicAdd(st.ctr + CTR_CYC_WARP, (unsigned long long)(clock64() - c0));
          atomicAdd(st.ctr + CTR_NWARP, 1ull);
        }
      }
    };
    warp_phase(&counter[4], nwide_end, 4);
    __syncthreads();  // the quarter slices overlap the eighth slices
    warp_phase(&counter[6], total, SVD_WARPS);
  }
}

// ---------------------------------------------------------------- k_select
__device__ double block_sum(double v, double* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

// count of entries of a descending list that precede key (s, m, k) in the order
// (s desc, m asc, k asc); the list has pair index ml and alive length len.
constexpr int SELECT_STAGE = 3072;  // alive singular values k_select stages in shared memory

__device__ __forceinline__ int count_before(const double* lst, int len, int ml, double sv, int m, int k) {
  if (ml == m) return k;
  int lo = 0, hi = len;
  while (lo < hi) { int mid = (lo + hi) >> 1; if (lst[mid] > sv) lo = mid + 1; else hi = mid; }
  if (ml > m) return lo;
  hi = len;
  while (lo < hi) { int mid = (lo + hi) >> 1; if (lst[mid] >= sv) lo = mid + 1; else hi = mid; }
  return lo;
}

__global__ void __launch_bounds__(1024) k_select(MpoDev st, SlotWS ws, const GateDesc* __restrict__ gates,
                                                 double* __restrict__ disc, double floor_rel) {
  const int s = blockIdx.x;
  Slot sl = get_slot(ws, s);
  if (sl.scal[SS_STATUS]) return;
  const GateDesc g = gates[s];
  const int ncap = st.ncap, P = st.P, M = st.M, D = st.D, Pc = ws.Pc;
  const int tid = threadIdx.x, nth = blockDim.x;
  __shared__ double red[1024];
  __shared__ int lstart[2 * MPO_PC_MAX + 1];
  __shared__ int lalive[2 * MPO_PC_MAX], lkept[2 * MPO_PC_MAX], lpair[2 * MPO_PC_MAX];
  __shared__ int newseg[MPO_P_MAX + 1];
  __shared__ int keep_sh, nalive_sh;
  const int NL = 2 * Pc;
  // 1. s_max and total weight: one thread per candidate value (the blocks' value lists
  // are contiguous in candidate order; a non-self-mirror block's values count twice)
  __shared__ int coffs[MPO_PC_MAX + 1];
  __shared__ unsigned char cmult[MPO_PC_MAX];
  for (int t = tid; t <= Pc; t += nth) {
    coffs[t] = sl.f(BF_COFF, t);
    if (t < Pc) cmult[t] = pair_mirror(sl.f(BF_M, t), ncap) == sl.f(BF_M, t) ? 1 : 2;
  }
  __syncthreads();
  double smax = 0.0, tot = 0.0;
  for (int e = tid; e < coffs[Pc]; e += nth) {
    const double v = sl.sval[e];
    smax = fmax(smax, v);
    tot += cmult[find_block(coffs, Pc + 1, e)] * (v * v);
  }
  red[tid] = smax;
  __syncthreads();
  for (int w = nth / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] = fmax(red[tid], red[tid + w]);
    __syncthreads();
  }
  smax = red[0];
  __syncthreads();
  tot = block_sum(tot, red);
  const double floor2 = floor_rel * smax * smax;
  // 2. alive prefix per list (list 2t = block t, list 2t+1 = its mirror)
  for (int l = tid; l < NL; l += nth) {
    const int t = l >> 1, n = sl.f(BF_G, t), mt = sl.f(BF_M, t);
    const bool self = pair_mirror(mt, ncap) == mt;
    int alive = 0;
    if (n > 0 && !((l & 1) && self)) {
      const double* lst = sl.sval + sl.f(BF_COFF, t);
      int lo = 0, hi = n;
      while (lo < hi) { int mid = (lo + hi) >> 1; if (lst[mid] * lst[mid] > floor2) lo = mid + 1; else hi = mid; }
      alive = lo;
    }
    lalive[l] = alive;
    lpair[l] = (l & 1) ? pair_mirror(mt, ncap) : mt;
    lkept[l] = 0;
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int l = 0; l < NL; ++l) { lstart[l] = acc; acc += lalive[l]; }
    lstart[NL] = acc;
    nalive_sh = acc;
    const int cap = st.chi_cap[g.inst];
    int keep = acc;
    if (cap > 0 && acc > cap) keep = -1;  // needs ranks
    if (cap <= 0 && acc > D) keep = -2;
    keep_sh = keep;
  }
  __syncthreads();
  const int nalive = nalive_sh;
  int keep = keep_sh;
  if (keep == -2) {
    if (tid == 0) { dev_set_error(st.err, DEV_ERR_CAPACITY, 5000); sl.scal[SS_STATUS] = 1; }
    return;
  }
  const int cap = st.chi_cap[g.inst];
  if (keep == -1) {
    // 3. ranks of every alive candidate; order[rank] for rank <= cap.  The alive values
    // of every list (a mirror list repeats its block's values) are staged in shared
    // memory when they fit, so the binary searches below do not go to L2.
    __shared__ double svs[SELECT_STAGE];
    const bool staged = nalive <= SELECT_STAGE;
    if (staged)
      for (int e = tid; e < nalive; e += nth) {
        const int l = find_block(lstart, NL + 1, e);
        svs[e] = sl.sval[sl.f(BF_COFF, l >> 1) + (e - lstart[l])];
      }
    __syncthreads();
    auto list_of = [&](int l) {
      return staged ? svs + lstart[l] : sl.sval + sl.f(BF_COFF, l >> 1);
    };
    for (int e = tid; e < nalive; e += nth) {
      const int l = find_block(lstart, NL + 1, e);
      const int k = e - lstart[l];
      const double sv = list_of(l)[k];
      const int mpair = lpair[l];
      int rank = 0;
      for (int l2 = 0; l2 < NL; ++l2) {
        if (lalive[l2] == 0) continue;
        rank += count_before(list_of(l2), lalive[l2], lpair[l2], sv, mpair, k);
      }
      if (rank <= cap) sl.order[rank] = e;
    }
    __syncthreads();
    if (tid == 0) {
      auto sval_of = [&](int e) {
        const int l = find_block(lstart, NL + 1, e);
        return list_of(l)[e - lstart[l]];
      };
      int jc = cap;
      while (jc > 0 && sval_of(sl.order[jc]) >= sval_of(sl.order[jc - 1]) * (1.0 - TIE_REL)) --jc;
      keep_sh = jc > 0 ? jc : cap;
    }
    __syncthreads();
    keep = keep_sh;
    for (int r2 = tid; r2 < keep; r2 += nth) {
      const int l = find_block(lstart, NL + 1, sl.order[r2]);
      atomicAdd(&lkept[l], 1);
    }
  } else {
    for (int l = tid; l < NL; l += nth) lkept[l] = lalive[l];
  }
  __syncthreads();
  // 4. new bond C: segments in pair order
  if (tid == 0) {
    for (int p = 0; p <= P; ++p) newseg[p] = 0;
    for (int l = 0; l < NL; ++l) if (lkept[l] > 0) newseg[lpair[l]] += lkept[l];
    int acc = 0;
    for (int p = 0; p < P; ++p) { int cnt = newseg[p]; newseg[p] = acc; acc += cnt; }
    newseg[P] = acc;
    int koff = 0;
    for (int t = 0; t < Pc; ++t) {
      const int mt = sl.f(BF_M, t);
      const bool self = pair_mirror(mt, ncap) == mt;
      const int kt = lkept[2 * t];
      if (!self && lkept[2 * t + 1] != kt) dev_set_error(st.err, DEV_ERR_INTERNAL, 6000 + t);
      sl.f(BF_KEPT, t) = kt;
      sl.f(BF_NEWPOS, t) = newseg[mt];
      sl.f(BF_NEWPOS_MIR, t) = newseg[pair_mirror(mt, ncap)];
      sl.f(BF_KOFF, t) = koff;
      koff += kt;
    }
    sl.f(BF_KOFF, Pc) = koff;
    sl.scal[SS_NITEMS] = koff;
  }
  __syncthreads();
  const long long bC = (long long)g.inst * (M + 1) + g.j + 1;
  int* chC = st.charge + bC * D;
  double* lC = st.lam + bC * D;
  double keptw = 0.0;
  for (int l = tid; l < NL; l += nth) {
    const int kl = lkept[l];
    if (kl == 0) continue;
    const double* lst = sl.sval + sl.f(BF_COFF, l >> 1);
    const int base = newseg[lpair[l]];
    for (int k = 0; k < kl; ++k) {
      chC[base + k] = lpair[l];
      lC[base + k] = lst[k];
      keptw += lst[k] * lst[k];
    }
  }
  for (int p = tid; p <= P; p += nth) st.segoff[bC * (P + 1) + p] = newseg[p];
  keptw = block_sum(keptw, red);  // its barriers also publish the lC writes above
  const int chinew = newseg[P];
  double ent = 0.0;
  for (int i = tid; i < chinew; i += nth) {
    const double pr = lC[i] * lC[i] / keptw;
    if (pr > 0.0) ent -= pr * log2(pr);
  }
  ent = block_sum(ent, red);
  if (tid == 0) {
    st.chi[bC] = chinew;
    st.entropy[bC] = ent;
    const double eps = tot > 0.0 ? fmax(0.0, (tot - keptw) / tot) : 0.0;  // rounding can go below 0
    sl.dscal[0] = eps;
    if (disc != nullptr && g.out >= 0) disc[g.out] = eps;
    if (chinew == 0) dev_set_error(st.err, DEV_ERR_NUMERIC, 7000);
  }
}


// mirror of bond index a (segment of pair pa at position a - seg[pa]); -1 if the
// mirror segment is too short (broken symmetry: reported, never dereferenced)
__device__ __forceinline__ int mirror_index(const int* seg, const int* ch, int a, int ncap, int* err) {
  const int pa = ch[a], pm = pair_mirror(pa, ncap);
  const int pos = a - seg[pa];
  if (pos >= seg[pm + 1] - seg[pm]) { dev_set_error(err, DEV_ERR_INTERNAL, 9000); return -1; }
  return seg[pm] + pos;
}

// ---------------------------------------------------------------- k_resplit
// For every kept singular triple of a canonical block (refined by k_refine):
// Gamma_j[:, beta] = X / lambda_A and Gamma_{j+1}[beta, :] = Y / lambda_B, plus the
// conjugated, mirror-permuted copies for the mirror block.
template <typename R>
__global__ void __launch_bounds__(256) k_resplit(MpoDev st, SlotWS ws, const GateDesc* __restrict__ gates) {
  typedef typename Prec<R>::C C;
  const int s = blockIdx.y;
  Slot sl = get_slot(ws, s);
  if (sl.scal[SS_STATUS]) return;
  const GateDesc g = gates[s];
  const int ncap = st.ncap, P = st.P, M = st.M, D = st.D, Pc = ws.Pc;
  const int tid = threadIdx.x, nth = blockDim.x;
  __shared__ int kpre[MPO_PC_MAX + 1];
  __shared__ int segA[MPO_P_MAX + 1], segB[MPO_P_MAX + 1];
  extern __shared__ double rinv[];  // 1 / lambda of bonds A (first D) and B (next D)
  const long long bA = (long long)g.inst * (M + 1) + g.j, bB = bA + 2;
  for (int t = tid; t <= Pc; t += nth) kpre[t] = sl.f(BF_KOFF, t);
  for (int p = tid; p <= P; p += nth) {
    segA[p] = st.segoff[bA * (P + 1) + p];
    segB[p] = st.segoff[bB * (P + 1) + p];
  }
  const int* chA = st.charge + bA * D;
  const int* chB = st.charge + bB * D;
  const double* lA = st.lam + bA * D;
  const double* lB = st.lam + bB * D;
  // the reciprocals once per CTA (an FP64 division is a long instruction sequence here)
  {
    const int nA = st.chi[bA], nB = st.chi[bB];
    for (int i = tid; i < nA; i += nth) rinv[i] = 1.0 / lA[i];
    for (int i = tid; i < nB; i += nth) rinv[D + i] = 1.0 / lB[i];
  }
  __syncthreads();
  const double* rA = rinv;
  const double* rB = rinv + D;
  double2* G1 = st.gam + ((long long)g.inst * M + g.j) * D * D;
  double2* G2 = G1 + (long long)D * D;
  const int items = sl.scal[SS_NITEMS];
  for (int z = blockIdx.x; z < items; z += gridDim.x) {
    const int t = find_block(kpre, Pc + 1, z);
    const int k = z - kpre[t];
    const int r = sl.f(BF_R, t), c = sl.f(BF_C, t), n = sl.f(BF_G, t), side = sl.f(BF_SIDE, t);
    const int h = side == 0 ? c : r;
    const int mt = sl.f(BF_M, t);
    const bool mir = pair_mirror(mt, ncap) != mt;
    const int coff = sl.f(BF_COFF, t);
    const double isig = 1.0 / sl.sval[coff + k];
    const int vc = sl.perm[coff + k];
    const C* wk = reinterpret_cast<const C*>(sl.W) + sl.f(BF_TOFF, t) + (long long)vc * h;
    const C* vk = reinterpret_cast<const C*>(sl.VC) + sl.f(BF_GOFF, t) + (long long)vc * n;
    const int* rmap = sl.rowmap + sl.f(BF_RMOFF, t);
    const int* cmap = sl.colmap + sl.f(BF_CMOFF, t);
    const int beta = sl.f(BF_NEWPOS, t) + k, betam = sl.f(BF_NEWPOS_MIR, t) + k;
    if (st.ctr && tid == 0) atomicAdd(st.ctr + CTR_RESPLIT, 2ull * (unsigned long long)(r + c));
    // X column (length r) and Y row (length c)
    for (int i = tid; i < r; i += nth) {
      const double2 x = side == 1 ? cscale(to_d2(wk[i]), isig) : to_d2(vk[i]);
      const int a = rmap[i];
      G1[(long long)a * D + beta] = cscale(x, rA[a]);
      if (mir) {
        const int am = mirror_index(segA, chA, a, ncap, st.err);
        if (am >= 0) G1[(long long)am * D + betam] = cscale(cconj(x), rA[am]);
      }
    }
    for (int qq = tid; qq < c; qq += nth) {
      const double2 y = side == 1 ? cconj(to_d2(vk[qq])) : cscale(cconj(to_d2(wk[qq])), isig);
      const int b = cmap[qq];
      G2[(long long)beta * D + b] = cscale(y, rB[b]);
      if (mir) {
        const int bm = mirror_index(segB, chB, b, ncap, st.err);
        if (bm >= 0) G2[(long long)betam * D + bm] = cscale(cconj(y), rB[bm]);
      }
    }
  }
}

// ---------------------------------------------------------------- phases
__global__ void k_phases(MpoDev st, const double* __restrict__ phase) {
  const int j = blockIdx.x, inst = blockIdx.y;
  const int M = st.M, D = st.D, ncap = st.ncap;
  const long long bA = (long long)inst * (M + 1) + j, bB = bA + 1;
  const int chiA = st.chi[bA], chiB = st.chi[bB];
  const int* chA = st.charge + bA * D;
  const int* chB = st.charge + bB * D;
  double2* G = st.gam + ((long long)inst * M + j) * D * D;
  const double ph = phase[(long long)inst * M + j];
  for (int e = threadIdx.x + blockIdx.z * blockDim.x; e < chiA * chiB; e += blockDim.x * gridDim.z) {
    const int ia = e / chiB, ib = e % chiB;
    const int pa = chA[ia], pb = chB[ib];
    const int i = pair_c(pa, ncap) - pair_c(pb, ncap), ibar = pair_cb(pa, ncap) - pair_cb(pb, ncap);
    if (i < 0 || ibar < 0) continue;
    double sn, cs;
    sincos(ph * (double)(i - ibar), &sn, &cs);
    G[(long long)ia * D + ib] = cmul(G[(long long)ia * D + ib], make_double2(cs, sn));
  }
}

int g_sm_count = 0;
int sm_count() {
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (g_sm_count <= 0) g_sm_count = 148;
  }
  return g_sm_count;
}

constexpr size_t SVD_SMEM = 200 * 1024;
// k_svd cluster shape: K CTAs per cluster and the number of such clusters that fit on
// the GPU at once (per precision and K = 1, 2, 4, 8), from
// cudaOccupancyMaxActiveClusters at start-up; 0 clusters = launch without clusters
// (every large block then runs on one CTA).  The process default is 4 CTAs per
// cluster, or GBS_MPO_SVD_CLUSTER_SIZE (1, 2, 4 or 8) from the environment; a handle
// may choose another (mpo_set_tuning).
// Measured on GB300 (updates/s, K = 2 / 4 / 8): 16 modes FP64 5182 / 6131 / 5701, 32
// modes chi 256 mixed 1187 / 1730 / 1434, 48 modes chi 512 mixed 291 / 476 / 350,
// 64 instances mixed 71822 / 69018 / 60310.  36 clusters of 4 fit (144 CTAs).
int svd_cluster_size() {
  static int v = -1;
  if (v < 0) {
    v = 4;
    const char* e = getenv("GBS_MPO_SVD_CLUSTER_SIZE");
    if (e) {
      const int k = atoi(e);
      if (k == 1 || k == 2 || k == 4 || k == 8) v = k;
    }
  }
  return v;
}
int g_svd_clusters[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};  // [precision][log2 K]
__host__ inline int log2_k(int K) { return K >= 8 ? 3 : K >= 4 ? 2 : K >= 2 ? 1 : 0; }
// clusters of K that fit for precision R (0: launch without clusters)
template <typename R>
int svd_clusters(int K) {
  return K > 1 ? g_svd_clusters[sizeof(R) == 8 ? 0 : 1][log2_k(K)] : 0;
}

// CTAs of the k_svd launch for a layer of nblk blocks (a multiple of the cluster size
// when clusters are available).
template <typename R>
int svd_grid(int nblk, int K) {
  const int ncl = svd_clusters<R>(K);
  if (ncl > 0) {
    int want = (nblk + K - 1) / K;
    if (want < 1) want = 1;
    return (want < ncl ? want : ncl) * K;
  }
  const int sms = sm_count();
  return nblk < sms ? (nblk > 0 ? nblk : 1) : sms;
}

template <typename R>
cudaError_t launch_svd(const MpoDev& s, const SlotWS& ws, const GateDesc* d_gates, int grid, int K,
                       cudaStream_t st) {
  const int ncl = svd_clusters<R>(K);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  cfg.blockDim = dim3(svd_threads<R>(ws.D));
  cfg.dynamicSmemBytes = SVD_SMEM;
  cfg.stream = st;
  cfg.gridDim = dim3(grid);
  if (ncl > 0) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = K;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, k_svd<R>, s, ws, d_gates, (const int*)ws.list, ws.counter, (int)SVD_SMEM);
}

template <typename R>
int max_svd_clusters(int K) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  cfg.gridDim = dim3(K * 64);
  cfg.blockDim = dim3(SvdThreads<R>::value);
  cfg.dynamicSmemBytes = SVD_SMEM;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = K;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)k_svd<R>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Contraction form by default (mpo_set_tuning overrides it): the BF16 path contracts
// Theta on the tensor cores in BF16 (k_theta_tc), the FP64 and TF32 paths with the
// SIMT two-stage kernel (k_theta).  Measured on GB300: the one-stage tensor-core form
// on the TF32 path took 205 ms per 48-mode chi = 512 mesh against 85 ms for the FP32
// two-stage kernel, and made the 64-instance batched mesh 2.7x slower (190 vs 71 ms):
// its 3.4x larger flop count (F_Theta) and the staging of weighted operands cost more
// than the tensor pipe saves on blocks of these sizes.  The autotuner picks the form
// per workload.

// The tensor-core Gram kernel runs FP32-level (3xTF32) products on every path: the
// Gram eigenvectors seed the one-sided refinement, whose sweep count grows with the
// seed's error.
template <typename R>
void launch_gram_tc(const MpoDev& s, const SlotWS& ws, int ngates, int gmin, cudaStream_t st) {
  int per = (2 * sm_count() + ngates - 1) / ngates;
  if (per < 1) per = 1;
  k_gram_tc<R, tc::TC_3XTF32><<<dim3(per, ngates), 256, gram_tc_smem<tc::TC_3XTF32>(), st>>>(ws, s.ctr, s.err,
                                                                                                gmin);
}

template <typename R>
void launch_layer_t(const MpoDev& s, const SlotWS& ws, const GateDesc* d_gates, int ngates, double* d_disc,
                    cudaStream_t st, cudaEvent_t* ev, int mode) {
  const int sms = sm_count();
  int per = (4 * sms + ngates - 1) / ngates;
  if (per < 1) per = 1;
  if (per > 4096) per = 4096;
  const int nblk = ngates * ws.Pc;
  NvtxRange layer("gbs_mpo/layer");
  if (ev) record_stage_event(ev[0], st);
  { NvtxRange r("gbs_mpo/k_setup"); k_setup<<<ngates, 256, 0, st>>>(s, ws, d_gates); }
  if (ev) record_stage_event(ev[1], st);
  {
    NvtxRange r("gbs_mpo/k_theta");
    const bool tc_theta = sizeof(R) == 4 && (ws.theta_form == 2 || (ws.theta_form == 0 && mode == 2));
    if (tc_theta) {
      int per_tc = (2 * sms + ngates - 1) / ngates;
      if (per_tc < 1) per_tc = 1;
      if (mode == 2)
        k_theta_tc<tc::TC_BF16><<<dim3(per_tc, ngates), 256, theta_tc_smem<tc::TC_BF16>(s.ncap).total, st>>>(
            s, ws, d_gates);
      else
        k_theta_tc<tc::TC_3XTF32><<<dim3(per_tc, ngates), 256, theta_tc_smem<tc::TC_3XTF32>(s.ncap).total, st>>>(
            s, ws, d_gates);
    } else {
      k_theta<R><<<dim3(per, ngates), THETA_WARPS * 32, theta_smem_bytes(s.ncap, sizeof(typename Prec<R>::C)),
                   st>>>(s, ws, d_gates);
    }
  }
  if (ev) record_stage_event(ev[2], st);
  {
    NvtxRange r("gbs_mpo/k_gram");
    const int gmin = ws.gram_tc_min > 0 ? ws.gram_tc_min : GRAM_TC_MIN;
    k_gram<R><<<dim3(per, ngates), 256, 0, st>>>(ws, s.ctr, gmin);
    launch_gram_tc<R>(s, ws, ngates, gmin, st);
  }
  if (ev) record_stage_event(ev[3], st);
  const int K = ws.cl_size > 0 ? ws.cl_size : svd_cluster_size();
  const int svd_ctas = svd_grid<R>(nblk, K);
  const SvdLayout SL = svd_layout<R>(ws.D, SVD_SMEM);
  const int seed_max = (int)sqrt((double)(SL.total - SL.data) / (2.0 * sizeof(float2)));
  const int room = sizeof(R) == 4 ? (int)(SL.total - SL.data) : 0;
  {
    NvtxRange r("gbs_mpo/k_order");
    k_order<<<1, 1024, 0, st>>>(ws, ngates, ws.list, ws.counter, svd_ctas, SvdRoute<R>::min_n, SvdRoute<R>::always_n,
                                seed_max, room);
  }
  if (ev) record_stage_event(ev[4], st);
  { NvtxRange r("gbs_mpo/k_svd"); launch_svd<R>(s, ws, d_gates, svd_ctas, K, st); }
  if (ev) record_stage_event(ev[5], st);
  { NvtxRange r("gbs_mpo/k_select"); k_select<<<ngates, 1024, 0, st>>>(s, ws, d_gates, d_disc, Prec<R>::floor); }
  if (ev) record_stage_event(ev[6], st);
  {
    NvtxRange r("gbs_mpo/k_resplit");
    k_resplit<R><<<dim3(per, ngates), 256, 2 * (size_t)s.D * sizeof(double), st>>>(s, ws, d_gates);
  }
  if (ev) record_stage_event(ev[7], st);
}

}  // namespace

// One-time per-process setup (called outside any stream capture).
cudaError_t gate_module_init() {
  sm_count();
  cudaError_t e = cudaFuncSetAttribute(k_svd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SVD_SMEM);
  // k_resplit: 1 / lambda of two bonds, D <= 4096 (the capacity limit of mpo_init_*)
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_resplit<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4096 * 8);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_resplit<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4096 * 8);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_theta<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)theta_smem_bytes(MPO_NCAP_MAX, sizeof(double2)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_theta<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)theta_smem_bytes(MPO_NCAP_MAX, sizeof(float2)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_svd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SVD_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_theta_tc<tc::TC_3XTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)theta_tc_smem<tc::TC_3XTF32>(MPO_NCAP_MAX).total);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_theta_tc<tc::TC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)theta_tc_smem<tc::TC_BF16>(MPO_NCAP_MAX).total);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gram_tc<double, tc::TC_3XTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gram_tc_smem<tc::TC_3XTF32>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gram_tc<float, tc::TC_3XTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gram_tc_smem<tc::TC_3XTF32>());

  if (e != cudaSuccess) return e;
  for (int l = 1; l < 4; ++l) {
    g_svd_clusters[0][l] = max_svd_clusters<double>(1 << l);
    g_svd_clusters[1][l] = max_svd_clusters<float>(1 << l);
  }
  return cudaSuccess;
}

// 0: blocks go to a cluster by the load rule (see SvdRoute); GBS_MPO_SVD_CLUSTER_MIN_N
// (>= 1) in the environment replaces the rule by "Gram side >= that value" (the
// tests route every block through the cluster path with it).
int svd_big_min() {
  static int v = -1;
  if (v < 0) {
    v = 0;
    const char* e = getenv("GBS_MPO_SVD_CLUSTER_MIN_N");
    if (e && atoi(e) >= 1) v = atoi(e);
  }
  return v;
}

// Largest Gram side of a cluster block that takes the single-CTA Gram seed, from
// GBS_MPO_SVD_CLUSTER_SEED_MAX (>= 0) in the environment; -1 when it is not set (the
// handle then chooses by precision: 0 on the FP64 path, 64 on the FP32 path).
int svd_cluster_seed_max() {
  static int v = -2;
  if (v == -2) {
    v = -1;
    const char* e = getenv("GBS_MPO_SVD_CLUSTER_SEED_MAX");
    if (e && atoi(e) >= 0) v = atoi(e);
  }
  return v;
}

int svd_cluster_info(int* cluster_size, int* clusters_fp64, int* clusters_fp32) {
  if (cluster_size) *cluster_size = svd_cluster_size();
  if (clusters_fp64) *clusters_fp64 = svd_clusters<double>(svd_cluster_size());
  if (clusters_fp32) *clusters_fp32 = svd_clusters<float>(svd_cluster_size());
  return 0;
}

// stage_events (optional, 8 events): recorded before each stage launch and after the
// last one, for per-stage timing (setup, theta, gram, order, svd, select, resplit).
// They are recorded as external events, so under stream capture they become event
// record nodes of the graph and time every replay.
void launch_layer(const MpoDev& s, const SlotWS& ws, const GateDesc* d_gates, int ngates, double* d_disc,
                  int prec, cudaStream_t st, int* nlaunch, cudaEvent_t* ev) {
  if (prec == 0) launch_layer_t<double>(s, ws, d_gates, ngates, d_disc, st, ev, 0);
  else launch_layer_t<float>(s, ws, d_gates, ngates, d_disc, st, ev, prec == 2 ? 2 : 1);
  if (nlaunch) *nlaunch += 8;
}

void launch_phases(const MpoDev& s, const double* d_phase, cudaStream_t st) {
  k_phases<<<dim3(s.M, s.B, 4), 256, 0, st>>>(s, d_phase);
}
