// asym.cu -- the asymptotic operator-entanglement estimator of arXiv:2301.12814, App. C,
// for batches of parameter points (r, mu, theta) on sm_103a.
//
// One squeezed input mode, truncated at n_max photons, goes through the pure-loss
// channel (App. C, Eq. `lossy`) and is split over the two halves of the bipartition by
// the basis transform of Eq. `transform` / `kun`.  The vectorised output operator
// X[(k_u, k_u'), (k_d, k_d')] = rho_out[k_u, k_d; k_u', k_d'] has the reduced operator
// tr_u |rho_out>><<rho_out| with eigenvalues = the squared singular values of X; they
// are normalised and give S_1 and the Renyi entropy S_alpha (App. C).
//
// X is real and, because rho_out is real symmetric, invariant under the joint swap
// (k_u <-> k_u', k_d <-> k_d'); and rho_lossy[m, m'] vanishes for odd m - m' (the input
// has even photon numbers only), so X only couples (k_u + k_u') and (k_d + k_d') of equal
// parity.  In the basis e_(k,k), (e_(k,k') +- e_(k',k)) / sqrt 2 (k < k') on both sides
// X is therefore block diagonal with four blocks: symmetric/antisymmetric x even/odd
// parity, of about (n_max+1)^2 / 4 columns each.  Every block is factorised by a
// one-sided (Hestenes) Jacobi SVD in FP64 by one CTA, with its columns resident in
// shared memory; a second kernel normalises the pooled values, sorts them and takes the
// entropies.  No value is dropped or approximated by the block split: the four spectra
// together are the spectrum of X.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

#include "../../include/gbs_mpo.h"

namespace {

constexpr int ASYM_THREADS = 256;
constexpr int ASYM_WARPS = ASYM_THREADS / 32;
constexpr int ASYM_MAX_SWEEPS = 40;
constexpr double ASYM_TOL = 1e-15;  // rotate while |a_p . a_q| > tol |a_p| |a_q| ...
// ... and |a_p . a_q| > floor ||A||_F^2.  The blocks are strongly graded (entries carry
// powers of mu and tanh r down to ~1e-30), and without the floor cyclic Jacobi keeps
// rotating pairs of negligible columns for tens of sweeps (43 at n_max = 23; 20 with
// the floor).  A skipped rotation moves a squared singular value by at most
// |a_p . a_q|, i.e. a normalised eigenvalue by at most 1e-30 and its square root by at
// most 1e-15: the rounding level of what S_1 and Renyi orders >= 1/2 are built from.
constexpr double ASYM_FLOOR = 1e-30;

// Size and offset (in the pooled spectrum) of block sec for photon numbers 0..n:
// 0 symmetric/even, 1 symmetric/odd, 2 antisymmetric/even, 3 antisymmetric/odd.
// The four sizes add up to (n+1)^2; block 0 is the largest.
__host__ __device__ inline void asym_block_of(int n, int sec, int& nb, int& off) {
  const int L = n + 1, E = n / 2 + 1, O = L - E;  // E even, O odd photon numbers
  const int s0 = E * (E + 1) / 2 + O * (O + 1) / 2, s1 = E * O, s2 = E * (E - 1) / 2 + O * (O - 1) / 2;
  nb = sec == 0 ? s0 : sec == 1 ? s1 : sec == 2 ? s2 : s1;
  off = sec == 0 ? 0 : sec == 1 ? s0 : sec == 2 ? s0 + s1 : s0 + s1 + s2;
}

// shared-memory layout of k_asym_block (byte offsets; every section 16-byte aligned)
struct AsymSmem {
  size_t a, rho, v, tab, pairs, total;
};

__host__ __device__ inline size_t asym_align(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline AsymSmem asym_smem(int n) {
  int nb0, off0;
  asym_block_of(n, 0, nb0, off0);  // block 0 is the largest
  const size_t L = (size_t)n + 1;
  AsymSmem s;
  s.a = 0;
  s.rho = asym_align(s.a + (size_t)nb0 * (nb0 | 1) * sizeof(double));  // odd column stride
  s.v = asym_align(s.rho + L * L * sizeof(double));
  s.tab = asym_align(s.v + L * L * sizeof(double));  // binomials, then Kraus factors
  s.pairs = asym_align(s.tab + 2 * L * L * sizeof(double) + 5 * L * sizeof(double));
  s.total = asym_align(s.pairs + (size_t)nb0 * sizeof(int) + 64);
  return s;
}

__device__ inline double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Tournament pairing (circle method) for nbe (even) players: round k in [0, nbe-1),
// slot i in [0, nbe/2).  Every pair meets once per nbe - 1 rounds, slots are disjoint.
__device__ inline void asym_pair(int nbe, int k, int i, int& p, int& q) {
  const int m = nbe - 1;
  if (i == 0) {
    p = m;
    q = k;
  } else {
    p = (k + i) % m;
    q = (k - i + m) % m;
  }
}

// CTA width for photon cutoff n: one warp per 32 column pairs of the largest block
// (one warp up to n = 12, three at n = 23).
__host__ __device__ inline int asym_threads(int n) {
  int nb0, off0;
  asym_block_of(n, 0, nb0, off0);
  const int pairs = (nb0 + 1) / 2;
  int w = (pairs + 31) / 32;
  return 32 * (w < 1 ? 1 : (w > ASYM_WARPS ? ASYM_WARPS : w));
}

// One work item: block sec of point pt (the whole CTA).
__device__ void asym_item(int sec, int pt, int n, const double* __restrict__ r_all,
                          const double* __restrict__ mu_all, const double* __restrict__ th_all,
                          double* __restrict__ spec, int ld, int* __restrict__ sweeps, unsigned char* smem) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int L = n + 1;
  int nb, boff;
  asym_block_of(n, sec, nb, boff);
  const int lda = nb | 1;  // odd column stride: lanes on different columns hit different banks
  const AsymSmem lay = asym_smem(n);
  double* A = (double*)(smem + lay.a);      // column b at A + b * lda, rows 0..nb-1
  double* rho = (double*)(smem + lay.rho);  // [L][L] rho_lossy
  double* V = (double*)(smem + lay.v);      // [L][L] <k_u, k_d|U|k_u + k_d>
  double* bin = (double*)(smem + lay.tab);  // [L][L] C(a, b)
  double* kr = bin + L * L;                 // [L][L] Kraus factor K^(l)[o, o + l] at [o][l]
  double* psi = kr + L * L;                 // [L] squeezed amplitudes
  double* pw = psi + L;                     // [4][L] mu^o, (1-mu)^l, cos^k, sin^k
  int* pairs = (int*)(smem + lay.pairs);    // [nb] packed (k | k' << 8)
  __shared__ double s_red[ASYM_WARPS];

  const double r = r_all[pt], mu = mu_all[pt], th = th_all[pt];
  const int item = 4 * pt + sec;
  if (nb == 0) {
    if (tid == 0 && sweeps) sweeps[item] = 0;
    return;
  }

  // 1. tables: squeezed amplitudes (App. C), powers for the Kraus factors (Eq. `lossy`)
  //    and the split (Eq. `kun`), exact binomials, pair list of this block
  if (tid == 0) {
    const double t = -tanh(r);
    psi[0] = 1.0 / sqrt(cosh(r));
    for (int k = 1; k < L; ++k) psi[k] = (k & 1) ? 0.0 : psi[k - 2] * t * sqrt((double)(k - 1) / (double)k);
  } else if (tid == 1 % nth) {
    const double cth = cos(th), sth = sin(th);
    double a = 1.0, b = 1.0, c = 1.0, d = 1.0;
    for (int k = 0; k < L; ++k) {
      pw[k] = a; pw[L + k] = b; pw[2 * L + k] = c; pw[3 * L + k] = d;
      a *= mu; b *= (1.0 - mu); c *= cth; d *= sth;
    }
  }
  if (tid == (2 % nth)) {
    int cnt = 0;
    const bool sym = sec < 2;
    const int par = sec & 1;
    for (int u = 0; u < L; ++u)
      for (int u2 = sym ? u : u + 1; u2 < L; ++u2)
        if (((u + u2) & 1) == par) pairs[cnt++] = u | (u2 << 8);
  }
  for (int idx = tid; idx < L * L; idx += nth) {
    const int a = idx / L, b = idx % L;
    long long c = 0;
    if (b <= a) {
      c = 1;
      for (int i = 1; i <= b; ++i) c = c * (a - b + i) / i;  // exact: C(a-b+i, i) at every step
    }
    bin[idx] = (double)c;
  }
  __syncthreads();
  for (int idx = tid; idx < L * L; idx += nth) {
    const int o = idx / L, l = idx % L;
    kr[idx] = (o + l < L) ? sqrt(bin[(o + l) * L + o] * pw[o] * pw[L + l]) : 0.0;
    V[idx] = (o + l < L) ? sqrt(bin[(o + l) * L + o]) * pw[2 * L + o] * pw[3 * L + l] : 0.0;  // V[k_u][k_d]
  }
  __syncthreads();
  for (int idx = tid; idx < L * L; idx += nth) {
    const int m = idx / L, m2 = idx % L;
    double acc = 0.0;
    if (((m + m2) & 1) == 0) {
      const int lmax = n - (m > m2 ? m : m2);
      for (int l = 0; l <= lmax; ++l) acc += kr[m * L + l] * psi[m + l] * psi[m2 + l] * kr[m2 * L + l];
    }
    rho[idx] = acc;
  }
  __syncthreads();

  // 2. the block of X in the (anti)symmetric pair basis, column-major
  const bool sym = sec < 2;
#define ASYM_F(u, u2, d, d2) \
  (((u) + (d) > n || (u2) + (d2) > n) ? 0.0 : V[(u) * L + (d)] * V[(u2) * L + (d2)] * rho[((u) + (d)) * L + ((u2) + (d2))])
  double f2 = 0.0;
  for (int idx = tid; idx < nb * nb; idx += nth) {
    const int b = idx / nb, a = idx % nb;
    const int pa = pairs[a], pb = pairs[b];
    const int u = pa & 255, u2 = pa >> 8, d = pb & 255, d2 = pb >> 8;
    double x;
    if (sym) {
      if (u < u2 && d < d2) x = ASYM_F(u, u2, d, d2) + ASYM_F(u, u2, d2, d);
      else if (u < u2) x = 1.4142135623730951 * ASYM_F(u, u2, d, d);
      else if (d < d2) x = 1.4142135623730951 * ASYM_F(u, u, d, d2);
      else x = ASYM_F(u, u, d, d);
    } else {
      x = ASYM_F(u, u2, d, d2) - ASYM_F(u, u2, d2, d);
    }
    A[b * lda + a] = x;
    f2 = fma(x, x, f2);
  }
#undef ASYM_F
  f2 = warp_sum(f2);
  if ((tid & 31) == 0) s_red[tid >> 5] = f2;
  __syncthreads();
  double frob2 = 0.0;
  for (int w = 0; w < nth / 32; ++w) frob2 += s_red[w];
  const double gfloor = ASYM_FLOOR * frob2;

  // 3. one-sided Jacobi over the columns.  Each column pair of a round goes to a group
  //    of g lanes (g a power of two, as large as the CTA allows) that split the rows;
  //    the xor butterfly leaves bitwise identical sums in every lane of a group, so the
  //    group agrees on the rotation.  Every lane runs the same number of slots, so the
  //    full-mask shuffles always see the whole warp.
  const int nbe = nb + (nb & 1), P = nbe / 2;
  int g = 1;
  while (g < 32 && 2 * g * P <= nth) g *= 2;
  int gsh = 0;
  while ((1 << gsh) < g) ++gsh;
  const int slot = tid >> gsh, sub = tid & (g - 1), nslots = nth >> gsh;
  int sw = 0;
  for (; sw < ASYM_MAX_SWEEPS; ++sw) {
    int rotated = 0;
    for (int k = 0; k < nbe - 1; ++k) {
      for (int base = 0; base < P; base += nslots) {
        const int i = base + slot;
        int p = 0, q = 0;
        if (i < P) asym_pair(nbe, k, i, p, q);
        const bool act = i < P && p < nb && q < nb;
        double* ap = A + p * lda;
        double* aq = A + q * lda;
        double al = 0.0, be = 0.0, ga = 0.0;
        if (act) {
          for (int e = sub; e < nb; e += g) {
            const double x = ap[e], y = aq[e];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
        }
        for (int o = g >> 1; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (act && fabs(ga) > gfloor && ga * ga > ASYM_TOL * ASYM_TOL * (al * be)) {
          // the tangent t of the rotation angle in FP32 (from the FP64 ratio zeta); c and
          // s = c t in FP64 keep the rotation orthogonal to FP64 rounding whatever t is,
          // so only the angle, not the accuracy of the singular values, is FP32
          const double zeta = (be - al) / (2.0 * ga);
          double t;
          if (fabs(zeta) < 1e18) {
            const float zf = (float)zeta;
            t = (double)(copysignf(1.0f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f))));
          } else {
            t = 0.5 / zeta;
          }
          const double c = rsqrt(fma(t, t, 1.0)), s = c * t;
          for (int e = sub; e < nb; e += g) {
            const double x = ap[e], y = aq[e];
            ap[e] = fma(c, x, -s * y);
            aq[e] = fma(s, x, c * y);
          }
          rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) break;
  }

  // 4. squared column norms = squared singular values of the block
  for (int b = tid; b < nb; b += nth) {
    const double* ab = A + b * lda;
    double s2 = 0.0;
    for (int e = 0; e < nb; ++e) s2 = fma(ab[e], ab[e], s2);
    spec[(size_t)pt * ld + boff + b] = s2;
  }
  if (tid == 0 && sweeps) sweeps[item] = sw + 1;
}


// grid: as many CTAs of asym_threads(n) threads as fit on the SMs, each looping over work items
// f = blockIdx.x, blockIdx.x + gridDim.x, ...  Items are block-major (f = block * npts +
// point), so the items a CTA takes -- and those of the CTAs sharing an SM -- mix the
// four block sizes: with point-major items and a grid-wide stride divisible by 4 every
// SM would see one block size only (3.8x more work on the SMs of the largest block at
// n_max = 8).  Writes the block's squared singular values to
// spec[point * ld + off[block] + j] and its sweep count to sweeps[4 * point + block].
__global__ void __launch_bounds__(ASYM_THREADS)
k_asym_block(int npts, int n, const double* __restrict__ r_all, const double* __restrict__ mu_all,
             const double* __restrict__ th_all, double* __restrict__ spec, int ld, int* __restrict__ sweeps) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (int f = blockIdx.x; f < 4 * npts; f += gridDim.x) {
    asym_item(f / npts, f % npts, n, r_all, mu_all, th_all, spec, ld, sweeps, smem);
    __syncthreads();  // shared memory is rebuilt by the next item
  }
}

// grid: npts CTAs.  Normalises the pooled squared singular values of a point, writes
// them back sorted in descending order, and the entropies (App. C, in bits).
__global__ void __launch_bounds__(ASYM_THREADS)
k_asym_finalize(int npts, int n, double alpha, int want_alpha, double* __restrict__ spec, int ld,
                double* __restrict__ S1, double* __restrict__ Sa) {
  __shared__ double v[(MPO_ASYM_NMAX + 1) * (MPO_ASYM_NMAX + 1)];
  __shared__ double red[3][ASYM_WARPS];
  const int pt = blockIdx.x;
  if (pt >= npts) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = (n + 1) * (n + 1);
  double* row = spec + (size_t)pt * ld;
  double tot = 0.0;
  for (int i = tid; i < K; i += ASYM_THREADS) {
    v[i] = row[i];
    tot += v[i];
  }
  tot = warp_sum(tot);
  if (lane == 0) red[0][warp] = tot;
  __syncthreads();
  tot = 0.0;
  for (int w = 0; w < ASYM_WARPS; ++w) tot += red[0][w];
  const double inv = tot > 0.0 ? 1.0 / tot : 0.0;
  double h = 0.0, ha = 0.0;
  for (int i = tid; i < K; i += ASYM_THREADS) {
    const double p = v[i] * inv;
    if (p > 0.0) {
      h -= p * log2(p);
      if (want_alpha) ha += pow(p, alpha);
    }
  }
  h = warp_sum(h);
  ha = warp_sum(ha);
  __syncthreads();
  if (lane == 0) {
    red[1][warp] = h;
    red[2][warp] = ha;
  }
  __syncthreads();
  if (tid == 0) {
    double hs = 0.0, has = 0.0;
    for (int w = 0; w < ASYM_WARPS; ++w) {
      hs += red[1][w];
      has += red[2][w];
    }
    S1[pt] = hs;
    if (want_alpha) Sa[pt] = (alpha == 1.0) ? hs : (has > 0.0 ? log2(has) / (1.0 - alpha) : 0.0);
  }
  // rank sort, descending; ties keep index order
  for (int i = tid; i < K; i += ASYM_THREADS) {
    const double x = v[i];
    int rank = 0;
    for (int j = 0; j < K; ++j) {
      const double y = v[j];
      rank += (y > x) || (y == x && j < i);
    }
    row[rank] = x * inv;
  }
}

// Cap on resident CTAs per SM of k_asym_block; 0 (the default) = the occupancy limit.
// GBS_MPO_ASYM_CTAS_PER_SM sets a cap.  At n_max = 8 (Fig. 1 grid, 768 points) the
// occupancy limit (24) gave 3.67 ms, caps of 4 / 8 / 12 / 16 gave 5.91 / 4.08 / 3.91 /
// 4.06 ms.
int asym_ctas_per_sm() {
  static int v = [] {
    const char* e = getenv("GBS_MPO_ASYM_CTAS_PER_SM");
    const int x = e ? atoi(e) : 0;
    return x > 0 ? x : 0;
  }();
  return v;
}

mpo_status asym_cuda(cudaError_t e) {
  if (e == cudaSuccess) return MPO_OK;
  if (e == cudaErrorMemoryAllocation) return MPO_ERR_OOM;
  return MPO_ERR_CUDA;
}

}  // namespace

extern "C" mpo_status mpo_asymptotic_ee_device(int npts, int n_max, const double* r, const double* mu,
                                               const double* theta, double alpha, double* S1, double* S_alpha,
                                               double* spectrum, int ld, int* sweeps, void* cuda_stream) {
  if (npts < 0 || n_max < 1 || n_max > MPO_ASYM_NMAX) return MPO_ERR_ARG;
  if (npts == 0) return MPO_OK;
  if (!r || !mu || !theta || !S1 || !spectrum || ld < (n_max + 1) * (n_max + 1)) return MPO_ERR_ARG;
  if (S_alpha && !(alpha > 0.0)) return MPO_ERR_ARG;
  if ((long long)npts * 4 > 0x7fffffffll) return MPO_ERR_ARG;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return asym_cuda(e);
  const size_t smem = asym_smem(n_max).total;
  if (smem > (size_t)optin) return MPO_ERR_ARG;
  e = cudaFuncSetAttribute(k_asym_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return asym_cuda(e);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int threads = asym_threads(n_max);
  int nsm = 0, per_sm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_asym_block, threads, smem);
  if (e != cudaSuccess) return asym_cuda(e);
  if (per_sm < 1) return MPO_ERR_ARG;
  const long long items = 4ll * npts;
  const int cap = asym_ctas_per_sm();
  const int grid = (int)std::min<long long>(items, (long long)nsm * (cap > 0 ? std::min(per_sm, cap) : per_sm));
  k_asym_block<<<grid, threads, smem, st>>>(npts, n_max, r, mu, theta, spectrum, ld, sweeps);
  k_asym_finalize<<<npts, ASYM_THREADS, 0, st>>>(npts, n_max, alpha, S_alpha ? 1 : 0, spectrum, ld, S1,
                                                 S_alpha);
  return asym_cuda(cudaGetLastError());
}

extern "C" mpo_status mpo_asymptotic_ee(int npts, int n_max, const double* r, const double* mu,
                                        const double* theta, double alpha, double* S1, double* S_alpha,
                                        double* spectrum, int ld) {
  if (npts < 0 || n_max < 1 || n_max > MPO_ASYM_NMAX) return MPO_ERR_ARG;
  if (npts == 0) return MPO_OK;
  if (!r || !mu || !theta || !S1) return MPO_ERR_ARG;
  const int K = (n_max + 1) * (n_max + 1);
  if (spectrum && ld < K) return MPO_ERR_ARG;
  if (S_alpha && !(alpha > 0.0)) return MPO_ERR_ARG;
  for (int i = 0; i < npts; ++i)
    if (!(r[i] >= 0.0 && r[i] <= 3.0) || !(mu[i] >= 0.0 && mu[i] <= 1.0) || !isfinite(theta[i]))
      return MPO_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return MPO_ERR_NOT_BUILT;
  const size_t n_in = 3 * (size_t)npts, n_out = 2 * (size_t)npts, n_spec = (size_t)npts * K;
  const size_t bytes = (n_in + n_out + n_spec) * sizeof(double) + 4 * (size_t)npts * sizeof(int);
  char* buf = nullptr;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return asym_cuda(e);
  e = cudaMalloc(&buf, bytes);
  if (e != cudaSuccess) {
    cudaStreamDestroy(st);
    return asym_cuda(e);
  }
  double* d_in = (double*)buf;
  double* d_out = d_in + n_in;
  double* d_spec = d_out + n_out;
  int* d_sw = (int*)(d_spec + n_spec);
  std::vector<int> hsw;
  mpo_status rs = MPO_OK;
  e = cudaMemcpyAsync(d_in, r, npts * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_in + npts, mu, npts * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_in + 2 * npts, theta, npts * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    rs = mpo_asymptotic_ee_device(npts, n_max, d_in, d_in + npts, d_in + 2 * npts, alpha, d_out,
                                  S_alpha ? d_out + npts : nullptr, d_spec, K, d_sw, st);
    if (rs == MPO_OK) {
      e = cudaMemcpyAsync(S1, d_out, npts * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && S_alpha)
        e = cudaMemcpyAsync(S_alpha, d_out + npts, npts * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && spectrum)
        e = cudaMemcpy2DAsync(spectrum, ld * sizeof(double), d_spec, K * sizeof(double), K * sizeof(double), npts,
                              cudaMemcpyDeviceToHost, st);
      hsw.resize(4 * (size_t)npts);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hsw.data(), d_sw, hsw.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  cudaStreamDestroy(st);
  if (e != cudaSuccess) return asym_cuda(e);
  if (rs != MPO_OK) return rs;
  for (int s : hsw)
    if (s > ASYM_MAX_SWEEPS) return MPO_ERR_NUMERIC;
  return MPO_OK;
}
