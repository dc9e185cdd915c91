// Initial state: rho_0 = P_cap (x)_j rho_j P_cap / Tr in exactly canonical U(1) Vidal form.
//
// Paper (arXiv:2301.12814): squeezed vacuum amplitudes of one mode (App. C), the
// pure-loss Kraus channel applied to the input because uniform loss commutes with
// the interferometer (Method; App. B), U(1) charges = photons to the right of a
// bond (App. D), the left-most charge = total photon number (App. A).
//
// One CTA per instance.  Thread p owns charge pair p = (c, cbar).  The lossy mode
// state is evaluated element by element as
//   rho[n, nb] = sum_l sqrt(C(n+l, n) C(nb+l, nb)) eta^{(n+nb)/2} (1-eta)^l c_{n+l} c_{nb+l}
// (the Kraus sum written out), with c_{2j} from the ratio recurrence
//   c_0 = 1/sqrt(cosh r),  c_{2j} = -tanh(r) sqrt((2j-1)/(2j)) c_{2j-2}.
// Per-mode normalisation is skipped: the global trace normalisation absorbs it.
// R_b^2 (weights of configurations right of bond b at each total) and W_b (left
// of bond b) are convolution recursions over modes; L_b^2 sums W_b over the
// totals the cap still allows.  lambda_b = L_b R_b / T and
// Gamma_j[a, b] = T rho_j[c_a - c_b, cbar_a - cbar_b] / (R_j(a) L_{j+1}(b)).
#include "mpo_internal.cuh"

namespace {

__device__ double binom_d(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

__global__ void k_init(MpoDev s, const double* __restrict__ r_all, const double* __restrict__ eta_all,
                       int dloc, double* __restrict__ scratch) {
  const int inst = blockIdx.x;
  const int M = s.M, ncap = s.ncap, q = ncap + 1, P = s.P, D = s.D;
  const int tid = threadIdx.x, nth = blockDim.x;
  const long long per = (long long)(M + 1) * P * 3 + (long long)M * P * 2 + 64;
  double* R2 = scratch + per * inst;           // [M+1][P]
  double* W2 = R2 + (long long)(M + 1) * P;    // [M+1][P]
  double* L2 = W2 + (long long)(M + 1) * P;    // [M+1][P]
  double* rho = L2 + (long long)(M + 1) * P;   // [M][P] real part of rho_j[n, nb]
  double* wgt = rho + (long long)M * P;        // [M][P] |rho_j|^2
  double* misc = wgt + (long long)M * P;       // [64]
  const double* r = r_all + (long long)inst * M;
  const double* eta = eta_all + (long long)inst * M;

  // Every (c, cbar) quantity below is computed for c <= cbar and copied to the
  // mirror pair (cbar, c), so the initial state is exactly ket/bra mirror-symmetric.
  // 1. per-mode lossy states and weights
  for (int idx = tid; idx < M * P; idx += nth) {
    int j = idx / P, p = idx % P;
    int n = pair_c(p, ncap), nb = pair_cb(p, ncap);
    if (n > nb) continue;
    double val = 0.0;
    if (((n + nb) & 1) == 0) {
      double rr = r[j], et = eta[j];
      double amp[MPO_D_LOCAL_MAX];
      double th = -tanh(rr);
      amp[0] = 1.0 / sqrt(cosh(rr));
      for (int k = 1; k < dloc; ++k) {
        if (k & 1) amp[k] = 0.0;
        else amp[k] = amp[k - 2] * th * sqrt((double)(k - 1) / (double)k);
      }
      double se = sqrt(et);
      double pw = 1.0;
      for (int i = 0; i < n + nb; ++i) pw *= se;
      double lossf = 1.0;
      int lmax = dloc - 1 - (n > nb ? n : nb);
      for (int l = 0; l <= lmax; ++l) {
        double term = sqrt(binom_d(n + l, n) * binom_d(nb + l, nb)) * pw * lossf * amp[n + l] * amp[nb + l];
        val += term;
        lossf *= (1.0 - et);
      }
    }
    rho[idx] = val;
    wgt[idx] = val * val;
    const long long mi = (long long)j * P + pair_mirror(p, ncap);
    rho[mi] = val;
    wgt[mi] = val * val;
  }
  __syncthreads();

  // 2. right weights R2[b] (b = M .. 0) and left weights W2[b] (b = 0 .. M)
  for (int p = tid; p < P; p += nth) {
    R2[(long long)M * P + p] = (p == 0) ? 1.0 : 0.0;
    W2[p] = (p == 0) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int b = M - 1; b >= 0; --b) {
    for (int p = tid; p < P; p += nth) {
      int c = pair_c(p, ncap), cb = pair_cb(p, ncap);
      if (c > cb) continue;
      double acc = 0.0;
      for (int n = 0; n <= c; ++n)
        for (int nb = 0; nb <= cb; ++nb)
          acc += wgt[(long long)b * P + n * q + nb] * R2[(long long)(b + 1) * P + (c - n) * q + (cb - nb)];
      R2[(long long)b * P + p] = acc;
      R2[(long long)b * P + pair_mirror(p, ncap)] = acc;
    }
    __syncthreads();
  }
  for (int b = 0; b < M; ++b) {
    for (int p = tid; p < P; p += nth) {
      int c = pair_c(p, ncap), cb = pair_cb(p, ncap);
      if (c > cb) continue;
      double acc = 0.0;
      for (int n = 0; n <= c; ++n)
        for (int nb = 0; nb <= cb; ++nb)
          acc += wgt[(long long)b * P + n * q + nb] * W2[(long long)b * P + (c - n) * q + (cb - nb)];
      W2[(long long)(b + 1) * P + p] = acc;
      W2[(long long)(b + 1) * P + pair_mirror(p, ncap)] = acc;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < (M + 1) * P; idx += nth) {
    int b = idx / P, p = idx % P;
    int c = pair_c(p, ncap), cb = pair_cb(p, ncap);
    if (c > cb) continue;
    double acc = 0.0;
    for (int x = 0; x <= ncap - c; ++x)
      for (int xb = 0; xb <= ncap - cb; ++xb) acc += W2[(long long)b * P + x * q + xb];
    L2[idx] = acc;
    L2[(long long)b * P + pair_mirror(p, ncap)] = acc;
  }
  // 3. trace normalisation T = Tr(P_cap (x) rho_j P_cap): diagonal convolution
  if (tid == 0) {
    double t[MPO_NCAP_MAX + 1], nt[MPO_NCAP_MAX + 1];
    for (int x = 0; x < q; ++x) t[x] = (x == 0) ? 1.0 : 0.0;
    for (int j = 0; j < M; ++j) {
      for (int x = 0; x < q; ++x) {
        double acc = 0.0;
        for (int n = 0; n <= x; ++n) acc += rho[(long long)j * P + n * q + n] * t[x - n];
        nt[x] = acc;
      }
      for (int x = 0; x < q; ++x) t[x] = nt[x];
    }
    double T = 0.0;
    for (int x = 0; x < q; ++x) T += t[x];
    misc[0] = T;
  }
  __syncthreads();
  const double T = misc[0];

  // 4. bonds: one index per pair with non-zero weight on both sides
  for (int b = tid; b <= M; b += nth) {
    long long bi = (long long)inst * (M + 1) + b;
    int* seg = s.segoff + bi * (P + 1);
    int* ch = s.charge + bi * D;
    double* lam = s.lam + bi * D;
    int cnt = 0;
    double tot = 0.0;
    for (int p = 0; p < P; ++p) {
      seg[p] = cnt;
      double rv = R2[(long long)b * P + p], lv = L2[(long long)b * P + p];
      if (rv > 0.0 && lv > 0.0) {
        if (cnt < D) {
          ch[cnt] = p;
          lam[cnt] = sqrt(lv * rv) / T;
          tot += lam[cnt] * lam[cnt];
        }
        ++cnt;
      }
    }
    seg[P] = cnt;
    if (cnt > D) { dev_set_error(s.err, DEV_ERR_CAPACITY, 1000 + b); cnt = D; }
    s.chi[bi] = cnt;
    double S = 0.0;
    for (int i = 0; i < cnt; ++i) {
      double pr = lam[i] * lam[i] / tot;
      if (pr > 0.0) S -= pr * log2(pr);
    }
    s.entropy[bi] = S;
  }
  __syncthreads();

  // 5. Gamma_j entries a >= b (componentwise); other entries stay zero
  for (int j = 0; j < M; ++j) {
    long long bA = (long long)inst * (M + 1) + j, bB = bA + 1;
    int chiA = s.chi[bA], chiB = s.chi[bB];
    const int* chA = s.charge + bA * D;
    const int* chB = s.charge + bB * D;
    double2* G = s.gam + ((long long)inst * M + j) * D * D;
    for (int e = tid; e < chiA * chiB; e += nth) {
      int ia = e / chiB, ib = e % chiB;
      int pa = chA[ia], pb = chB[ib];
      int i = pair_c(pa, ncap) - pair_c(pb, ncap);
      int ibar = pair_cb(pa, ncap) - pair_cb(pb, ncap);
      if (i < 0 || ibar < 0) continue;
      double v = T * rho[(long long)j * P + i * q + ibar] /
                 (sqrt(R2[(long long)j * P + pa]) * sqrt(L2[(long long)(j + 1) * P + pb]));
      G[(long long)ia * D + ib] = make_double2(v, 0.0);
    }
  }
}

}  // namespace

void launch_init(const MpoDev& s, const double* d_r, const double* d_eta, int d_local,
                 double* scratch, cudaStream_t st) {
  k_init<<<s.B, 256, 0, st>>>(s, d_r, d_eta, d_local, scratch);
}
