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
// GB300 design (differs from the paper's A100 kernels, which were a SIMT GEMM with
// unitary lookups and a library SVD):
// * Hermiticity of rho makes Theta(mbar) the ket/bra mirror of Theta(m)
//   (Theta(mbar)[pi a, pi b] = conj Theta(m)[a, b]).  Only the canonical blocks
//   m = (c, cbar) with c <= cbar are contracted and factorised; the mirror block's
//   singular values are bitwise copies and its vectors are conjugated copies.  This
//   halves the work and makes the mirror spectra exactly degenerate, so the
//   keep-chi rule never splits a mirror pair.  Self-mirror blocks (c = cbar) are
//   diagonalised in the basis where the mirror acts as complex conjugation; their
//   Gram matrix is real there, so the vectors come out mirror-symmetric.
// * The SVD is a Gram matrix (smaller side) plus a parallel-order cyclic Jacobi
//   eigensolver, one CTA per block; singular values below the Gram accuracy floor
//   are dropped.
// * The beam-splitter Fock blocks are built on the device by the creation-operator
//   recurrence U|j, n-j> = (S11 a1^dag + S21 a2^dag) U|j-1, n-j> / sqrt(j).
// Stages: k_setup (Fock tables, charge bookkeeping) -> k_theta -> k_gram -> k_eig ->
// k_select (global keep-chi, new bond, lambda, discarded weight, entropy) ->
// k_resplit (back-multiply, Gamma_j and Gamma_{j+1} including mirror copies).
#include "mpo_internal.cuh"

namespace {

constexpr int TILE = 16;
constexpr double GRAM_FLOOR_FP64 = 1e-13;  // drop s^2 <= floor * s_max^2
constexpr double TIE_REL = 1e-9;           // keep-chi: never split a run closer than this
constexpr int JACOBI_MAX_SWEEPS = 60;

struct Slot {
  int* blk; int* scal; int* rowoff; int* coloff; int* rowmap; int* colmap;
  double2* fock; double2* theta; double2* G; double2* V; double* sval; int* perm;
  double* dscal; int* order;
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
  sl.theta = ws.theta + (long long)s * ws.capTheta;
  sl.G = ws.G + (long long)s * ws.capGram;
  sl.V = ws.V + (long long)s * ws.capGram;
  sl.sval = ws.sval + (long long)s * ws.capCand;
  sl.perm = ws.perm + (long long)s * ws.capCand;
  sl.dscal = ws.dscal + (long long)s * 4;
  sl.order = ws.order + (long long)s * ws.capCand * 2;
  return sl;
}

// largest t in [0, n) with pre[t] <= z  (pre non-decreasing, pre[0] = 0)
__device__ __forceinline__ int find_block(const int* pre, int n, int z) {
  int lo = 0, hi = n;  // invariant: pre[lo] <= z, answer in [lo, hi)
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pre[mid] <= z) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- k_setup
__global__ void k_setup(MpoDev st, SlotWS ws, const GateDesc* __restrict__ gates) {
  const int s = blockIdx.x;
  const GateDesc g = gates[s];
  Slot sl = get_slot(ws, s);
  const int ncap = st.ncap, q = ncap + 1, P = st.P, M = st.M, Pc = ws.Pc;
  const int tid = threadIdx.x, nth = blockDim.x;
  __shared__ int segA[MPO_P_MAX + 1], segC[MPO_P_MAX + 1], segB[MPO_P_MAX + 1];
  __shared__ double2 fk[MPO_FOCK_MAX];
  __shared__ unsigned char supA[MPO_P_MAX], infB[MPO_P_MAX];
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
  if (tid == 0) fk[0] = make_double2(1.0, 0.0);
  __syncthreads();
  for (int n = 1; n <= ncap; ++n) {
    const int o1 = fock_off(n - 1), o = fock_off(n);
    for (int jj = tid; jj <= n; jj += nth) {
      const int src = (jj >= 1) ? jj - 1 : 0;
      const double2 al = (jj >= 1) ? S11 : S12, be = (jj >= 1) ? S21 : S22;
      const double sc = 1.0 / sqrt((double)((jj >= 1) ? jj : n));
      for (int i = 0; i <= n; ++i) {
        double2 acc = make_double2(0.0, 0.0);
        if (i >= 1) cfma(acc, cscale(al, sqrt((double)i)), fk[o1 + (i - 1) * n + src]);
        if (i <= n - 1) cfma(acc, cscale(be, sqrt((double)(n - i))), fk[o1 + i * n + src]);
        fk[o + i * (n + 1) + jj] = cscale(acc, sc);
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < fock_off(ncap + 1); e += nth) sl.fock[e] = fk[e];
  // dominance tables: supA[x, y] = some A pair (c, cb) present with c >= x, cb >= y
  //                   infB[x, y] = some B pair present with c <= x, cb <= y
  for (int p = tid; p < P; p += nth) {
    int x = pair_c(p, ncap), y = pair_cb(p, ncap);
    unsigned char sa = 0, ib = 0;
    for (int a = 0; a < P; ++a) {
      int ca = pair_c(a, ncap), cba = pair_cb(a, ncap);
      if (segA[a + 1] > segA[a] && ca >= x && cba >= y) sa = 1;
      if (segB[a + 1] > segB[a] && ca <= x && cba <= y) ib = 1;
    }
    supA[p] = sa; infB[p] = ib;
  }
  __syncthreads();
  // per canonical block: rows, cols, non-empty test, segment offsets
  for (int t = tid; t < Pc; t += nth) {
    const int m = canon_pair(t, ncap), cm = pair_c(m, ncap), cbm = pair_cb(m, ncap);
    int r = 0, c = 0;
    for (int a = 0; a < P; ++a) {
      int na = segA[a + 1] - segA[a];
      if (na > 0 && pair_c(a, ncap) >= cm && pair_cb(a, ncap) >= cbm) {
        sl.rowoff[t * P + a] = r; r += na;
      } else sl.rowoff[t * P + a] = -1;
      int nb = segB[a + 1] - segB[a];
      if (nb > 0 && pair_c(a, ncap) <= cm && pair_cb(a, ncap) <= cbm) {
        sl.coloff[t * P + a] = c; c += nb;
      } else sl.coloff[t * P + a] = -1;
    }
    bool path = false;
    for (int cc = 0; cc < P && !path; ++cc) {
      if (segC[cc + 1] == segC[cc]) continue;
      int x = pair_c(cc, ncap), y = pair_cb(cc, ncap);
      int hx = x > cm ? x : cm, hy = y > cbm ? y : cbm;
      int lx = x < cm ? x : cm, ly = y < cbm ? y : cbm;
      if (supA[hx * q + hy] && infB[lx * q + ly]) path = true;
    }
    const int gg = (r > 0 && c > 0 && path) ? (r < c ? r : c) : 0;
    sl.f(BF_M, t) = m;
    sl.f(BF_R, t) = gg ? r : 0;
    sl.f(BF_C, t) = gg ? c : 0;
    sl.f(BF_G, t) = gg;
    sl.f(BF_SIDE, t) = (r <= c) ? 0 : 1;
  }
  __syncthreads();
  if (tid == 0) {
    long long toff = 0, goff = 0, coff = 0, rm = 0, cm2 = 0;
    int tt = 0, gt = 0;
    for (int t = 0; t < Pc; ++t) {
      const int r = sl.f(BF_R, t), c = sl.f(BF_C, t), gg = sl.f(BF_G, t);
      sl.f(BF_TOFF, t) = (int)toff; sl.f(BF_GOFF, t) = (int)goff; sl.f(BF_COFF, t) = (int)coff;
      sl.f(BF_RMOFF, t) = (int)rm; sl.f(BF_CMOFF, t) = (int)cm2;
      sl.f(BF_TT, t) = tt; sl.f(BF_GT, t) = gt;
      toff += (long long)r * c; goff += (long long)gg * gg; coff += gg; rm += r; cm2 += c;
      const int ntr = (r + TILE - 1) / TILE, ntc = (c + TILE - 1) / TILE, ntg = (gg + TILE - 1) / TILE;
      tt += ntr * ntc; gt += ntg * (ntg + 1) / 2;
    }
    sl.f(BF_TT, Pc) = tt; sl.f(BF_GT, Pc) = gt;
    sl.f(BF_TOFF, Pc) = (int)toff; sl.f(BF_COFF, Pc) = (int)coff;
    int status = 0;
    if (toff > ws.capTheta || goff > ws.capGram || coff > ws.capCand || rm > ws.capRC || cm2 > ws.capRC) {
      status = 1;
      dev_set_error(st.err, DEV_ERR_CAPACITY, 2000);
    }
    sl.scal[SS_NBLK] = Pc;
    sl.scal[SS_TTILES] = status ? 0 : tt;
    sl.scal[SS_GTILES] = status ? 0 : gt;
    sl.scal[SS_STATUS] = status;
  }
  __syncthreads();
  if (sl.scal[SS_STATUS]) return;
  // row / column maps: Theta(m) row i -> bond A index, column -> bond B index
  for (int t = tid; t < Pc; t += nth) {
    if (sl.f(BF_G, t) == 0) continue;
    int* rmap = sl.rowmap + sl.f(BF_RMOFF, t);
    int* cmap = sl.colmap + sl.f(BF_CMOFF, t);
    for (int a = 0; a < P; ++a) {
      int o = sl.rowoff[t * P + a];
      if (o >= 0) for (int i = segA[a]; i < segA[a + 1]; ++i) rmap[o + i - segA[a]] = i;
      int oc = sl.coloff[t * P + a];
      if (oc >= 0) for (int i = segB[a]; i < segB[a + 1]; ++i) cmap[oc + i - segB[a]] = i;
    }
  }
}

// ---------------------------------------------------------------- k_theta
// One 16 x 16 output tile of Theta(m) per iteration; K runs over the segments of the
// old centre bond C, each weighted by the unitary element u(a, b, c, m).
template <typename CT>
__global__ void __launch_bounds__(256) k_theta(MpoDev st, SlotWS ws, const GateDesc* __restrict__ gates) {
  const int s = blockIdx.y;
  Slot sl = get_slot(ws, s);
  if (sl.scal[SS_STATUS]) return;
  const GateDesc g = gates[s];
  const int ncap = st.ncap, q = ncap + 1, P = st.P, M = st.M, D = st.D, Pc = ws.Pc;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  __shared__ double2 fk[MPO_FOCK_MAX];
  __shared__ int segC[MPO_P_MAX + 1];
  __shared__ CT As[TILE][TILE + 1], Bs[TILE][TILE + 1];
  __shared__ int rA[TILE], pA[TILE], cB[TILE], pB[TILE];
  __shared__ int tpre[MPO_PC_MAX + 1];
  for (int e = threadIdx.x; e < fock_off(ncap + 1); e += blockDim.x) fk[e] = sl.fock[e];
  const long long bA = (long long)g.inst * (M + 1) + g.j, bC = bA + 1, bB = bA + 2;
  for (int p = threadIdx.x; p <= P; p += blockDim.x) segC[p] = st.segoff[bC * (P + 1) + p];
  for (int t = threadIdx.x; t <= Pc; t += blockDim.x) tpre[t] = sl.f(BF_TT, t);
  __syncthreads();
  const int* chA = st.charge + bA * D;
  const int* chB = st.charge + bB * D;
  const double* lA = st.lam + bA * D;
  const double* lC = st.lam + bC * D;
  const double* lB = st.lam + bB * D;
  const double2* G1 = st.gam + ((long long)g.inst * M + g.j) * D * D;
  const double2* G2 = G1 + (long long)D * D;
  const int total = sl.scal[SS_TTILES];
  unsigned long long flops = 0;
  for (int z = blockIdx.x; z < total; z += gridDim.x) {
    const int t = find_block(tpre, Pc + 1, z);
    const int r = sl.f(BF_R, t), c = sl.f(BF_C, t);
    const int m = sl.f(BF_M, t), cm = pair_c(m, ncap), cbm = pair_cb(m, ncap);
    const int ntc = (c + TILE - 1) / TILE;
    const int local = z - tpre[t];
    const int i0 = (local / ntc) * TILE, q0 = (local % ntc) * TILE;
    __syncthreads();
    if (threadIdx.x < TILE) {
      int i = i0 + threadIdx.x;
      int a = (i < r) ? sl.rowmap[sl.f(BF_RMOFF, t) + i] : -1;
      rA[threadIdx.x] = a; pA[threadIdx.x] = (a >= 0) ? chA[a] : -1;
    } else if (threadIdx.x < 2 * TILE) {
      int qq = q0 + threadIdx.x - TILE;
      int b = (qq < c) ? sl.colmap[sl.f(BF_CMOFF, t) + qq] : -1;
      cB[threadIdx.x - TILE] = b; pB[threadIdx.x - TILE] = (b >= 0) ? chB[b] : -1;
    }
    __syncthreads();
    const int myA = pA[ty], myB = pB[tx];
    const int ca = myA >= 0 ? pair_c(myA, ncap) : -1, cba = myA >= 0 ? pair_cb(myA, ncap) : -1;
    const int cb = myB >= 0 ? pair_c(myB, ncap) : 1 << 20, cbb = myB >= 0 ? pair_cb(myB, ncap) : 1 << 20;
    // loader roles: row loader uses (ty) row, column loader uses (tx) column
    const int la = pA[ty];
    const int lca = la >= 0 ? pair_c(la, ncap) : -1, lcba = la >= 0 ? pair_cb(la, ncap) : -1;
    const int lb = pB[tx];
    const int lcb = lb >= 0 ? pair_c(lb, ncap) : 1 << 20, lcbb = lb >= 0 ? pair_cb(lb, ncap) : 1 << 20;
    double2 acc = make_double2(0.0, 0.0);
    const bool mine = (i0 + ty < r) && (q0 + tx < c);
    for (int cc = 0; cc < P; ++cc) {
      const int k0 = segC[cc], k1 = segC[cc + 1];
      if (k1 == k0) continue;
      const int xc = pair_c(cc, ncap), yc = pair_cb(cc, ncap);
      const bool ok = (ca >= xc && cba >= yc && xc >= cb && yc >= cbb);
      if (!__syncthreads_or(ok)) continue;
      const bool rowok = (lca >= xc && lcba >= yc);
      const bool colok = (xc >= lcb && yc >= lcbb);
      CT part;
      part.x = 0; part.y = 0;
      for (int kb = k0; kb < k1; kb += TILE) {
        {
          int kk = kb + tx;
          double2 v = make_double2(0.0, 0.0);
          if (rowok && kk < k1) v = G1[(long long)rA[ty] * D + kk];
          As[ty][tx] = from_d2<CT>(v);
          int kr = kb + ty;
          double2 w = make_double2(0.0, 0.0);
          if (colok && kr < k1) w = cscale(G2[(long long)kr * D + cB[tx]], lC[kr]);
          Bs[ty][tx] = from_d2<CT>(w);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TILE; ++kk) cfma(part, As[ty][kk], Bs[kk][tx]);
        __syncthreads();
      }
      if (ok) {
        if (mine) flops += 8ull * (unsigned long long)(k1 - k0) + 8ull;
        const int dk = ca - cb, db = cba - cbb;
        const double2 uk = fk[fock_off(dk) + (ca - cm) * (dk + 1) + (ca - xc)];
        const double2 ub = fk[fock_off(db) + (cba - cbm) * (db + 1) + (cba - yc)];
        const double2 u = cmul(uk, cconj(ub));
        cfma(acc, u, to_d2(part));
      }
    }
    const int i = i0 + ty, qq = q0 + tx;
    if (i < r && qq < c) {
      double sc = lA[rA[ty]] * lB[cB[tx]];
      sl.theta[sl.f(BF_TOFF, t) + (long long)i * c + qq] = cscale(acc, sc);
    }
  }
  if (st.ctr) {
    flops = __reduce_add_sync(0xffffffffu, (unsigned)flops);
    if ((threadIdx.x & 31) == 0 && flops) atomicAdd(st.ctr + CTR_THETA, flops);
  }
}

// ---------------------------------------------------------------- k_gram
// Upper-triangular 16 x 16 tiles of G = Theta Theta^dag (side 0) or Theta^dag Theta.
__global__ void __launch_bounds__(256) k_gram(SlotWS ws, unsigned long long* ctr) {
  const int s = blockIdx.y;
  Slot sl = get_slot(ws, s);
  if (sl.scal[SS_STATUS]) return;
  const int Pc = ws.Pc;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  __shared__ double2 As[TILE][TILE + 1], Bs[TILE][TILE + 1];
  __shared__ int gpre[MPO_PC_MAX + 1];
  for (int t = threadIdx.x; t <= Pc; t += blockDim.x) gpre[t] = sl.f(BF_GT, t);
  __syncthreads();
  const int total = sl.scal[SS_GTILES];
  unsigned long long flops = 0;
  for (int z = blockIdx.x; z < total; z += gridDim.x) {
    const int t = find_block(gpre, Pc + 1, z);
    const int r = sl.f(BF_R, t), c = sl.f(BF_C, t), gg = sl.f(BF_G, t), side = sl.f(BF_SIDE, t);
    const double2* Th = sl.theta + sl.f(BF_TOFF, t);
    double2* Gm = sl.G + sl.f(BF_GOFF, t);
    const int nt = (gg + TILE - 1) / TILE;
    int rem = z - gpre[t], ti = 0;
    while (rem >= nt - ti) { rem -= nt - ti; ++ti; }
    const int tj = ti + rem;
    const int K = side == 0 ? c : r;
    double2 acc = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < K; k0 += TILE) {
      __syncthreads();
      if (side == 0) {
        int ia = ti * TILE + ty, ib = tj * TILE + ty, kk = k0 + tx;
        As[ty][tx] = (ia < gg && kk < K) ? Th[(long long)ia * c + kk] : make_double2(0, 0);
        Bs[ty][tx] = (ib < gg && kk < K) ? Th[(long long)ib * c + kk] : make_double2(0, 0);
      } else {
        int kr = k0 + ty, ja = ti * TILE + tx, jb = tj * TILE + tx;
        As[ty][tx] = (kr < K && ja < gg) ? Th[(long long)kr * c + ja] : make_double2(0, 0);
        Bs[ty][tx] = (kr < K && jb < gg) ? Th[(long long)kr * c + jb] : make_double2(0, 0);
      }
      __syncthreads();
      if (side == 0) {
#pragma unroll
        for (int kk = 0; kk < TILE; ++kk) cfma_cj(acc, Bs[tx][kk], As[ty][kk]);
      } else {
#pragma unroll
        for (int kk = 0; kk < TILE; ++kk) cfma_cj(acc, As[kk][ty], Bs[kk][tx]);
      }
    }
    const int gi = ti * TILE + ty, gj = tj * TILE + tx;
    if (gi < gg && gj < gg && (ti < tj || ty <= tx)) flops += 8ull * (unsigned long long)K;
    if (gi < gg && gj < gg) {
      if (ti < tj || ty < tx) {
        Gm[(long long)gi * gg + gj] = acc;
        Gm[(long long)gj * gg + gi] = cconj(acc);
      } else if (ty == tx) {
        Gm[(long long)gi * gg + gi] = make_double2(acc.x, 0.0);
      }
    }
  }
  if (ctr) {
    flops = __reduce_add_sync(0xffffffffu, (unsigned)flops);
    if ((threadIdx.x & 31) == 0 && flops) atomicAdd(ctr + CTR_GRAM, flops);
  }
}

// ---------------------------------------------------------------- k_eig
// Cyclic Jacobi with the round-robin (circle) pairing: n/2 disjoint rotations per
// round, n-1 rounds per sweep.  For the pair (p, q) with g = G_pq = |g| e^{i psi}:
// D = diag(1, e^{-i psi}) makes the 2x2 block real, the real rotation
// R = [[c, s], [-s, c]] with t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// tau = (G_qq - G_pp) / (2|g|) annihilates it, and J = D R is applied as
// G <- J^dag G J, V <- V J.
struct RotPair { int p, q; double c, s; double2 e; };

__device__ __forceinline__ void mirror_coord(const Slot& sl, const MpoDev& st, const GateDesc& g,
                                             int t, int side, int i, const int* segX, int& mi) {
  const int ncap = st.ncap, P = st.P, D = st.D, M = st.M;
  const long long bX = (long long)g.inst * (M + 1) + g.j + (side == 0 ? 0 : 2);
  const int idx = side == 0 ? sl.rowmap[sl.f(BF_RMOFF, t) + i] : sl.colmap[sl.f(BF_CMOFF, t) + i];
  const int pa = st.charge[bX * D + idx];
  const int pm = pair_mirror(pa, ncap);
  const int off = side == 0 ? sl.rowoff[t * P + pm] : sl.coloff[t * P + pm];
  const int pos = idx - segX[pa];
  if (off < 0 || pos >= segX[pm + 1] - segX[pm]) {  // mirror structure broken: never index with it
    dev_set_error(st.err, DEV_ERR_INTERNAL, 8000 + t);
    mi = i;
    return;
  }
  mi = off + pos;
}

__global__ void __launch_bounds__(256) k_eig(MpoDev st, SlotWS ws, const GateDesc* __restrict__ gates,
                                             int smem_bytes) {
  const int t = blockIdx.x, s = blockIdx.y;
  Slot sl = get_slot(ws, s);
  if (sl.scal[SS_STATUS] || t >= ws.Pc) return;
  const int n = sl.f(BF_G, t);
  if (n == 0) return;
  const GateDesc g = gates[s];
  const int side = sl.f(BF_SIDE, t), m = sl.f(BF_M, t);
  const int ncap = st.ncap, P = st.P, M = st.M;
  const bool selfm = pair_mirror(m, ncap) == m;
  const int np = n + (n & 1), half = np / 2;
  const int tid = threadIdx.x, nth = blockDim.x;
  extern __shared__ __align__(16) unsigned char smem[];
  RotPair* rot = reinterpret_cast<RotPair*>(smem);
  int* mpos = reinterpret_cast<int*>(rot + (ws.D / 2 + 1));
  int* segX = mpos + ws.D;
  double* red = reinterpret_cast<double*>(segX + MPO_P_MAX + 2);
  int* flags = reinterpret_cast<int*>(red + 2);
  size_t fixed = (size_t)(ws.D / 2 + 1) * sizeof(RotPair) + ws.D * sizeof(int) +
                 (MPO_P_MAX + 2) * sizeof(int) + 2 * sizeof(double) + 4 * sizeof(int);
  fixed = (fixed + 15) & ~(size_t)15;
  const bool in_smem = fixed + 2ull * n * n * sizeof(double2) <= (size_t)smem_bytes;
  double2* gG = sl.G + sl.f(BF_GOFF, t);
  double2* gV = sl.V + sl.f(BF_GOFF, t);
  double2* A = in_smem ? reinterpret_cast<double2*>(smem + fixed) : gG;
  double2* V = in_smem ? A + (long long)n * n : gV;

  if (selfm) {
    const long long bX = (long long)g.inst * (M + 1) + g.j + (side == 0 ? 0 : 2);
    for (int p = tid; p <= P; p += nth) segX[p] = st.segoff[bX * (P + 1) + p];
    __syncthreads();
    for (int i = tid; i < n; i += nth) { int mi; mirror_coord(sl, st, g, t, side, i, segX, mi); mpos[i] = mi; }
    __syncthreads();
    // realified Gram in the basis e_i (fixed), (e_p + e_q)/sqrt2 at p, i(e_p - e_q)/sqrt2 at q (p < q)
    double2* dst = in_smem ? A : gV;  // global mode: stage in V, copy back below
    const double h = 0.70710678118654752440;
    for (int e = tid; e < n * n; e += nth) {
      const int i = e / n, j = e % n;
      int ai[2], bj[2]; double2 wa[2], wb[2]; int na = 0, nb = 0;
      const int pi = mpos[i], pj = mpos[j];
      if (pi == i) { ai[0] = i; wa[0] = make_double2(1, 0); na = 1; }
      else if (i < pi) { ai[0] = i; wa[0] = make_double2(h, 0); ai[1] = pi; wa[1] = make_double2(h, 0); na = 2; }
      else { ai[0] = pi; wa[0] = make_double2(0, h); ai[1] = i; wa[1] = make_double2(0, -h); na = 2; }
      if (pj == j) { bj[0] = j; wb[0] = make_double2(1, 0); nb = 1; }
      else if (j < pj) { bj[0] = j; wb[0] = make_double2(h, 0); bj[1] = pj; wb[1] = make_double2(h, 0); nb = 2; }
      else { bj[0] = pj; wb[0] = make_double2(0, h); bj[1] = j; wb[1] = make_double2(0, -h); nb = 2; }
      double acc = 0.0;
      for (int x = 0; x < na; ++x)
        for (int y = 0; y < nb; ++y) {
          double2 v = cmul(cmul(cconj(wa[x]), gG[(long long)ai[x] * n + bj[y]]), wb[y]);
          acc += v.x;
        }
      dst[(long long)i * n + j] = make_double2(acc, 0.0);
    }
    __syncthreads();
    if (!in_smem) {
      for (int e = tid; e < n * n; e += nth) A[e] = gV[e];
      __syncthreads();
    }
  } else if (in_smem) {
    for (int e = tid; e < n * n; e += nth) A[e] = gG[e];
  }
  for (int e = tid; e < n * n; e += nth) V[e] = make_double2((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
  if (tid == 0) {
    double dm = 0.0;
    for (int i = 0; i < n; ++i) dm = fmax(dm, fabs(A[(long long)i * n + i].x));
    red[0] = dm;
  }
  __syncthreads();
  const double tol_rel = 1e-15, tol_abs = 1e-18 * red[0];
  if (tid == 0) flags[1] = 0;
  int sweep = 0;
  for (; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
    if (tid == 0) flags[0] = 0;
    __syncthreads();
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int k = tid; k < half; k += nth) {
        int p, qq;
        if (k == 0) { p = rnd; qq = np - 1; }
        else { p = (rnd + k) % (np - 1); qq = (rnd - k + np - 1) % (np - 1); }
        if (p > qq) { int tmp = p; p = qq; qq = tmp; }
        RotPair rp; rp.p = p; rp.q = qq; rp.c = 1.0; rp.s = 0.0; rp.e = make_double2(1.0, 0.0);
        if (qq < n) {
          const double a = A[(long long)p * n + p].x, b = A[(long long)qq * n + qq].x;
          const double2 gpq = A[(long long)p * n + qq];
          const double hh = hypot(gpq.x, gpq.y);
          if (hh > tol_rel * sqrt(fabs(a * b)) && hh > tol_abs) {
            const double tau = (b - a) / (2.0 * hh);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            rp.c = 1.0 / sqrt(1.0 + tt * tt);
            rp.s = tt * rp.c;
            rp.e = make_double2(gpq.x / hh, gpq.y / hh);
            flags[0] = 1;
            if (st.ctr) atomicAdd(&flags[1], 1);
          } else rp.q = -1;
        } else rp.q = -1;
        rot[k] = rp;
      }
      __syncthreads();
      // columns: [x, y] <- [x, y] [[c, s], [-s conj(e), c conj(e)]]
      for (int w2 = tid; w2 < n * half; w2 += nth) {
        const int i = w2 / half, k = w2 % half;
        const RotPair rp = rot[k];
        if (rp.q < 0) continue;
        const double2 ec = cconj(rp.e);
        double2* Ai = A + (long long)i * n;
        const double2 x = Ai[rp.p], y = Ai[rp.q];
        const double2 ys = cmul(y, ec);
        Ai[rp.p] = make_double2(rp.c * x.x - rp.s * ys.x, rp.c * x.y - rp.s * ys.y);
        Ai[rp.q] = make_double2(rp.s * x.x + rp.c * ys.x, rp.s * x.y + rp.c * ys.y);
        double2* Vi = V + (long long)i * n;
        const double2 vx = Vi[rp.p], vy = Vi[rp.q];
        const double2 vys = cmul(vy, ec);
        Vi[rp.p] = make_double2(rp.c * vx.x - rp.s * vys.x, rp.c * vx.y - rp.s * vys.y);
        Vi[rp.q] = make_double2(rp.s * vx.x + rp.c * vys.x, rp.s * vx.y + rp.c * vys.y);
      }
      __syncthreads();
      // rows: [x; y] <- J^dag [x; y] = [[c, -s e], [s, c e]] [x; y]
      for (int w2 = tid; w2 < n * half; w2 += nth) {
        const int k = w2 / n, i = w2 % n;
        const RotPair rp = rot[k];
        if (rp.q < 0) continue;
        const double2 x = A[(long long)rp.p * n + i], y = A[(long long)rp.q * n + i];
        const double2 ye = cmul(y, rp.e);
        A[(long long)rp.p * n + i] = make_double2(rp.c * x.x - rp.s * ye.x, rp.c * x.y - rp.s * ye.y);
        A[(long long)rp.q * n + i] = make_double2(rp.s * x.x + rp.c * ye.x, rp.s * x.y + rp.c * ye.y);
      }
      __syncthreads();
    }
    const int any = flags[0];
    __syncthreads();
    if (!any) break;
  }
  if (sweep >= JACOBI_MAX_SWEEPS && tid == 0) dev_set_error(st.err, DEV_ERR_NUMERIC, 3000 + t);
  if (st.ctr && tid == 0) {
    // per active rotation and per index: A columns, A rows and V columns, 18 flops each
    atomicAdd(st.ctr + CTR_EIG, 54ull * (unsigned long long)n * (unsigned long long)flags[1]);
    atomicAdd(st.ctr + CTR_SWEEPS, (unsigned long long)(sweep + 1));
    atomicAdd(st.ctr + CTR_EIGBLK, 1ull);
  }
  // eigenvalues, descending ranks (ties by index)
  const int coff = sl.f(BF_COFF, t);
  for (int i = tid; i < n; i += nth) {
    const double wi = A[(long long)i * n + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double wj = A[(long long)j * n + j].x;
      rank += (wj > wi) || (wj == wi && j < i);
    }
    if (!isfinite(wi)) dev_set_error(st.err, DEV_ERR_NUMERIC, 4000 + t);
    sl.sval[coff + rank] = sqrt(fmax(wi, 0.0));
    sl.perm[coff + rank] = i;
  }
  __syncthreads();  // every diagonal read above happens before A is reused below
  // eigenvectors out to gV (back to the original basis for self-mirror blocks)
  if (selfm) {
    const double h = 0.70710678118654752440;
    for (int e = tid; e < n * n; e += nth) {
      const int i = e / n, k = e % n;
      const int pi = mpos[i];
      double2 out;
      if (pi == i) out = make_double2(V[(long long)i * n + k].x, 0.0);
      else if (i < pi) out = make_double2(h * V[(long long)i * n + k].x, h * V[(long long)pi * n + k].x);
      else out = make_double2(h * V[(long long)pi * n + k].x, -h * V[(long long)i * n + k].x);
      if (in_smem) gV[e] = out;
      else A[e] = out;  // V lives in gV: stage through A (no longer needed)
    }
    if (!in_smem) {
      __syncthreads();
      for (int e = tid; e < n * n; e += nth) gV[e] = A[e];
    }
  } else if (in_smem) {
    for (int e = tid; e < n * n; e += nth) gV[e] = V[e];
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
__device__ __forceinline__ int count_before(const double* lst, int len, int ml, double sv, int m, int k) {
  if (ml == m) return k;
  // first index with lst[i] < sv (strictly smaller), and first with lst[i] <= sv
  int lo = 0, hi = len;
  while (lo < hi) { int mid = (lo + hi) >> 1; if (lst[mid] > sv) lo = mid + 1; else hi = mid; }
  int gt = lo;
  if (ml > m) return gt;
  hi = len;
  while (lo < hi) { int mid = (lo + hi) >> 1; if (lst[mid] >= sv) lo = mid + 1; else hi = mid; }
  return lo;  // includes equal values
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
  __shared__ int lstart[2 * MPO_PC_MAX + 1];   // prefix of alive counts over lists
  __shared__ int lalive[2 * MPO_PC_MAX], lkept[2 * MPO_PC_MAX], lpair[2 * MPO_PC_MAX];
  __shared__ int newseg[MPO_P_MAX + 1];
  __shared__ int keep_sh, nalive_sh;
  const int NL = 2 * Pc;
  // 1. s_max and total weight
  double smax = 0.0, tot = 0.0;
  for (int t = tid; t < Pc; t += nth) {
    const int n = sl.f(BF_G, t);
    if (n == 0) continue;
    const double* lst = sl.sval + sl.f(BF_COFF, t);
    smax = fmax(smax, lst[0]);
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += lst[k] * lst[k];
    const int mult = pair_mirror(sl.f(BF_M, t), ncap) == sl.f(BF_M, t) ? 1 : 2;
    tot += mult * acc;
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
    // 3. ranks of every alive candidate; order[rank] for rank <= cap
    for (int e = tid; e < nalive; e += nth) {
      const int l = find_block(lstart, NL + 1, e);
      const int k = e - lstart[l];
      const int t = l >> 1;
      const double sv = sl.sval[sl.f(BF_COFF, t) + k];
      const int mpair = lpair[l];
      int rank = 0;
      for (int l2 = 0; l2 < NL; ++l2) {
        if (lalive[l2] == 0) continue;
        rank += count_before(sl.sval + sl.f(BF_COFF, l2 >> 1), lalive[l2], lpair[l2], sv, mpair, k);
      }
      if (rank <= cap) sl.order[rank] = e;
    }
    __syncthreads();
    if (tid == 0) {
      auto sval_of = [&](int e) {
        const int l = find_block(lstart, NL + 1, e);
        return sl.sval[sl.f(BF_COFF, l >> 1) + (e - lstart[l])];
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
  keptw = block_sum(keptw, red);
  const int chinew = newseg[P];
  double ent = 0.0;
  for (int i = tid; i < chinew; i += nth) {
    const double pr = lC[i] * lC[i] / keptw;
    if (pr > 0.0) ent -= pr * log2(pr);
  }
  __syncthreads();  // lC writes above are visible to every thread
  ent = block_sum(ent, red);
  if (tid == 0) {
    st.chi[bC] = chinew;
    st.entropy[bC] = ent;
    const double eps = tot > 0.0 ? (tot - keptw) / tot : 0.0;
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
// For every kept singular triple of a canonical block: X column and Y row (one of
// them is an eigenvector, the other Theta times it over sigma), written as
// Gamma_j[:, beta] = X / lambda_A and Gamma_{j+1}[beta, :] = Y / lambda_B, plus the
// conjugated, mirror-permuted copies for the mirror block.
__global__ void __launch_bounds__(256) k_resplit(MpoDev st, SlotWS ws, const GateDesc* __restrict__ gates) {
  const int s = blockIdx.y;
  Slot sl = get_slot(ws, s);
  if (sl.scal[SS_STATUS]) return;
  const GateDesc g = gates[s];
  const int ncap = st.ncap, P = st.P, M = st.M, D = st.D, Pc = ws.Pc;
  const int tid = threadIdx.x, nth = blockDim.x;
  __shared__ int kpre[MPO_PC_MAX + 1];
  __shared__ int segA[MPO_P_MAX + 1], segB[MPO_P_MAX + 1];
  extern __shared__ __align__(16) unsigned char smem[];
  double2* vec = reinterpret_cast<double2*>(smem);  // [D]
  const long long bA = (long long)g.inst * (M + 1) + g.j, bB = bA + 2;
  for (int t = tid; t <= Pc; t += nth) kpre[t] = sl.f(BF_KOFF, t);
  for (int p = tid; p <= P; p += nth) {
    segA[p] = st.segoff[bA * (P + 1) + p];
    segB[p] = st.segoff[bB * (P + 1) + p];
  }
  __syncthreads();
  const int* chA = st.charge + bA * D;
  const int* chB = st.charge + bB * D;
  const double* lA = st.lam + bA * D;
  const double* lB = st.lam + bB * D;
  double2* G1 = st.gam + ((long long)g.inst * M + g.j) * D * D;
  double2* G2 = G1 + (long long)D * D;
  const int items = sl.scal[SS_NITEMS];
  const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  for (int z = blockIdx.x; z < items; z += gridDim.x) {
    const int t = find_block(kpre, Pc + 1, z);
    const int k = z - kpre[t];
    const int r = sl.f(BF_R, t), c = sl.f(BF_C, t), n = sl.f(BF_G, t), side = sl.f(BF_SIDE, t);
    const int mt = sl.f(BF_M, t);
    const bool mir = pair_mirror(mt, ncap) != mt;
    const int coff = sl.f(BF_COFF, t);
    const double sig = sl.sval[coff + k];
    const int vc = sl.perm[coff + k];
    const double2* Vm = sl.V + sl.f(BF_GOFF, t);
    const double2* Th = sl.theta + sl.f(BF_TOFF, t);
    const int* rmap = sl.rowmap + sl.f(BF_RMOFF, t);
    const int* cmap = sl.colmap + sl.f(BF_CMOFF, t);
    const int beta = sl.f(BF_NEWPOS, t) + k, betam = sl.f(BF_NEWPOS_MIR, t) + k;
    if (st.ctr && tid == 0) atomicAdd(st.ctr + CTR_RESPLIT, 8ull * (unsigned long long)r * c);
    __syncthreads();
    for (int i = tid; i < n; i += nth) vec[i] = Vm[(long long)i * n + vc];
    __syncthreads();
    if (side == 0) {
      // X = eigenvector (rows); Y = X^dag Theta / sigma
      for (int i = tid; i < r; i += nth) {
        const int a = rmap[i];
        G1[(long long)a * D + beta] = cscale(vec[i], 1.0 / lA[a]);
        if (mir) {
          const int am = mirror_index(segA, chA, a, ncap, st.err);
          if (am >= 0) G1[(long long)am * D + betam] = cscale(cconj(vec[i]), 1.0 / lA[am]);
        }
      }
      for (int qq = tid; qq < c; qq += nth) {
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < r; ++i) cfma_cj(acc, vec[i], Th[(long long)i * c + qq]);
        const int b = cmap[qq];
        G2[(long long)beta * D + b] = cscale(acc, 1.0 / (sig * lB[b]));
        if (mir) {
          const int bm = mirror_index(segB, chB, b, ncap, st.err);
          if (bm >= 0) G2[(long long)betam * D + bm] = cscale(cconj(acc), 1.0 / (sig * lB[bm]));
        }
      }
    } else {
      // Y = eigenvector^dag (cols); X = Theta v / sigma
      for (int qq = tid; qq < c; qq += nth) {
        const int b = cmap[qq];
        G2[(long long)beta * D + b] = cscale(cconj(vec[qq]), 1.0 / lB[b]);
        if (mir) {
          const int bm = mirror_index(segB, chB, b, ncap, st.err);
          if (bm >= 0) G2[(long long)betam * D + bm] = cscale(vec[qq], 1.0 / lB[bm]);
        }
      }
      for (int i = warp; i < r; i += nwarp) {
        double2 acc = make_double2(0.0, 0.0);
        for (int qq = lane; qq < c; qq += 32) cfma(acc, Th[(long long)i * c + qq], vec[qq]);
        for (int o = 16; o > 0; o >>= 1) {
          acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
          acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) {
          const int a = rmap[i];
          G1[(long long)a * D + beta] = cscale(acc, 1.0 / (sig * lA[a]));
          if (mir) {
            const int am = mirror_index(segA, chA, a, ncap, st.err);
            if (am >= 0) G1[(long long)am * D + betam] = cscale(cconj(acc), 1.0 / (sig * lA[am]));
          }
        }
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

}  // namespace

size_t eig_smem_bytes(int D) {
  size_t fixed = (size_t)(D / 2 + 1) * sizeof(RotPair) + D * sizeof(int) + (MPO_P_MAX + 2) * sizeof(int) +
                 2 * sizeof(double) + 4 * sizeof(int);
  fixed = (fixed + 15) & ~(size_t)15;
  size_t full = fixed + 2ull * D * D * sizeof(double2);
  const size_t cap = 200 * 1024;
  return full < cap ? full : cap;
}

// One-time per-process setup (called outside any stream capture).
cudaError_t gate_module_init() {
  sm_count();
  return cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// stage_events (optional, 7 events): recorded before each of the 6 stage launches
// and after the last one, for per-stage timing.
void launch_layer(const MpoDev& s, const SlotWS& ws, const GateDesc* d_gates, int ngates,
                  double* d_disc, int prec, cudaStream_t st, int* nlaunch, cudaEvent_t* ev) {
  (void)prec;
  const size_t esm = eig_smem_bytes(ws.D);
  const int sms = sm_count();
  int per = (4 * sms + ngates - 1) / ngates;
  if (per < 1) per = 1;
  if (per > 4096) per = 4096;
  if (ev) cudaEventRecord(ev[0], st);
  k_setup<<<ngates, 256, 0, st>>>(s, ws, d_gates);
  if (ev) cudaEventRecord(ev[1], st);
  k_theta<double2><<<dim3(per, ngates), 256, 0, st>>>(s, ws, d_gates);
  if (ev) cudaEventRecord(ev[2], st);
  k_gram<<<dim3(per, ngates), 256, 0, st>>>(ws, s.ctr);
  if (ev) cudaEventRecord(ev[3], st);
  k_eig<<<dim3(ws.Pc, ngates), 256, esm, st>>>(s, ws, d_gates, (int)esm);
  if (ev) cudaEventRecord(ev[4], st);
  k_select<<<ngates, 1024, 0, st>>>(s, ws, d_gates, d_disc, GRAM_FLOOR_FP64);
  if (ev) cudaEventRecord(ev[5], st);
  k_resplit<<<dim3(per, ngates), 256, ws.D * sizeof(double2), st>>>(s, ws, d_gates);
  if (ev) cudaEventRecord(ev[6], st);
  if (nlaunch) *nlaunch += 6;
}

void launch_phases(const MpoDev& s, const double* d_phase, cudaStream_t st) {
  k_phases<<<dim3(s.M, s.B, 4), 256, 0, st>>>(s, d_phase);
}
