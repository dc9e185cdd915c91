// Observables of the U(1) MPO by trace environments (one CTA per instance).
//
// Tr rho sums the vectorised state over configurations whose ket and bra photon
// numbers agree at every mode.  With the charge-implied physical indices of App. D,
// an entry Gamma_j[a, b] contributes to the trace only when the ket and bra local
// photon numbers coincide: c_a - c_b = cbar_a - cbar_b (>= 0).
//   E_0 = lambda_0,  E_{j+1}(b) = lambda_{j+1}(b) sum_a E_j(a) Gamma_j[a, b]
//   F_M = 1,         F_j(a)     = sum_b Gamma_j[a, b] lambda_{j+1}(b) F_{j+1}(b)
//   Tr rho = E_M,    <n_j^p> Tr rho = sum_{a,b} E_j(a) Gamma_j[a, b] i^p lambda_{j+1}(b) F_{j+1}(b)
// Sums run over segments: the partners of b are the pairs (c_b + i, cbar_b + i).
#include "mpo_internal.cuh"

namespace {

__device__ double2 block_sum2(double2 v, double2* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] = cadd(red[tid], red[tid + w]);
    __syncthreads();
  }
  double2 r = red[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) k_obs(MpoDev s, double2* __restrict__ scratch, double* __restrict__ out) {
  const int inst = blockIdx.x;
  const int M = s.M, D = s.D, P = s.P, ncap = s.ncap, q = ncap + 1;
  const int tid = threadIdx.x, nth = blockDim.x;
  __shared__ double2 red[256];
  double2* E = scratch + (long long)inst * 2 * (M + 1) * D;
  double2* F = E + (long long)(M + 1) * D;
  double* o = out + (long long)inst * (1 + 2 * M + (M + 1));
  auto bi = [&](int b) { return (long long)inst * (M + 1) + b; };
  {
    const int chi0 = s.chi[bi(0)];
    for (int a = tid; a < chi0; a += nth) E[a] = make_double2(s.lam[bi(0) * D + a], 0.0);
  }
  __syncthreads();
  for (int j = 0; j < M; ++j) {
    const int chiB = s.chi[bi(j + 1)];
    const int* chB = s.charge + bi(j + 1) * D;
    const int* segA = s.segoff + bi(j) * (P + 1);
    const double2* G = s.gam + ((long long)inst * M + j) * D * D;
    const double* lB = s.lam + bi(j + 1) * D;
    const double2* Ej = E + (long long)j * D;
    double2* En = E + (long long)(j + 1) * D;
    for (int b = tid; b < chiB; b += nth) {
      const int pb = chB[b], x = pair_c(pb, ncap), y = pair_cb(pb, ncap);
      double2 acc = make_double2(0.0, 0.0);
      for (int i = 0; x + i <= ncap && y + i <= ncap; ++i) {
        const int pa = (x + i) * q + (y + i);
        for (int a = segA[pa]; a < segA[pa + 1]; ++a) cfma(acc, Ej[a], G[(long long)a * D + b]);
      }
      En[b] = cscale(acc, lB[b]);
    }
    __syncthreads();
  }
  if (tid == 0) F[(long long)M * D] = make_double2(1.0, 0.0);
  __syncthreads();
  for (int j = M - 1; j >= 0; --j) {
    const int chiA = s.chi[bi(j)];
    const int* chA = s.charge + bi(j) * D;
    const int* segB = s.segoff + bi(j + 1) * (P + 1);
    const double2* G = s.gam + ((long long)inst * M + j) * D * D;
    const double* lB = s.lam + bi(j + 1) * D;
    const double2* Fn = F + (long long)(j + 1) * D;
    double2* Fj = F + (long long)j * D;
    for (int a = tid; a < chiA; a += nth) {
      const int pa = chA[a], x = pair_c(pa, ncap), y = pair_cb(pa, ncap);
      double2 acc = make_double2(0.0, 0.0);
      for (int i = 0; i <= x && i <= y; ++i) {
        const int pb = (x - i) * q + (y - i);
        for (int b = segB[pb]; b < segB[pb + 1]; ++b)
          cfma(acc, G[(long long)a * D + b], cscale(Fn[b], lB[b]));
      }
      Fj[a] = acc;
    }
    __syncthreads();
  }
  const double tr = E[(long long)M * D].x;
  if (tid == 0) o[0] = tr;
  for (int j = 0; j < M; ++j) {
    const int chiA = s.chi[bi(j)];
    const int* chA = s.charge + bi(j) * D;
    const int* segB = s.segoff + bi(j + 1) * (P + 1);
    const double2* G = s.gam + ((long long)inst * M + j) * D * D;
    const double* lB = s.lam + bi(j + 1) * D;
    const double2* Ej = E + (long long)j * D;
    const double2* Fn = F + (long long)(j + 1) * D;
    double2 s1 = make_double2(0.0, 0.0), s2 = make_double2(0.0, 0.0);
    for (int a = tid; a < chiA; a += nth) {
      const int pa = chA[a], x = pair_c(pa, ncap), y = pair_cb(pa, ncap);
      double2 acc1 = make_double2(0.0, 0.0), acc2 = make_double2(0.0, 0.0);
      for (int i = 1; i <= x && i <= y; ++i) {
        const int pb = (x - i) * q + (y - i);
        for (int b = segB[pb]; b < segB[pb + 1]; ++b) {
          const double2 v = cmul(G[(long long)a * D + b], cscale(Fn[b], lB[b]));
          acc1 = cadd(acc1, cscale(v, (double)i));
          acc2 = cadd(acc2, cscale(v, (double)(i * i)));
        }
      }
      cfma(s1, Ej[a], acc1);
      cfma(s2, Ej[a], acc2);
    }
    s1 = block_sum2(s1, red);
    s2 = block_sum2(s2, red);
    if (tid == 0) { o[1 + j] = s1.x; o[1 + M + j] = s2.x; }
  }
  // purity sum lambda^2 per bond
  for (int b = tid; b <= M; b += nth) {
    const int chi = s.chi[bi(b)];
    double acc = 0.0;
    for (int i = 0; i < chi; ++i) { const double l = s.lam[bi(b) * D + i]; acc += l * l; }
    o[1 + 2 * M + b] = acc;
  }
}

}  // namespace

void launch_observables(const MpoDev& s, double2* scratch, double* out, cudaStream_t st) {
  k_obs<<<s.B, 256, 0, st>>>(s, scratch, out);
}
