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
//
// The bond tables may come from caller-owned device buffers (mpo_observables_static),
// so every device-read size and index is clamped before use: chi to [0, D], pair
// indices to [0, P), segment offsets to [0, chi of their bond].  For valid tables the
// clamps change nothing; for invalid ones the numbers are meaningless but every access
// stays inside gam, lam, charge and the scratch.
#include <cuda.h>
#include <mutex>

#include "../../include/gbs_mpo.h"
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

__device__ __forceinline__ int chi_at(const MpoDev& s, long long b) { return clamp_chi(s.chi[b], s.D); }
__device__ __forceinline__ void seg_at(const int* seg, int p, int chi, int& lo, int& hi) {
  clamp_seg(seg, p, chi, lo, hi);
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
    const int chi0 = chi_at(s, bi(0));
    for (int a = tid; a < chi0; a += nth) E[a] = make_double2(s.lam[bi(0) * D + a], 0.0);
  }
  __syncthreads();
  for (int j = 0; j < M; ++j) {
    const int chiA = chi_at(s, bi(j)), chiB = chi_at(s, bi(j + 1));
    const int* chB = s.charge + bi(j + 1) * D;
    const int* segA = s.segoff + bi(j) * (P + 1);
    const double2* G = s.gam + ((long long)inst * M + j) * D * D;
    const double* lB = s.lam + bi(j + 1) * D;
    const double2* Ej = E + (long long)j * D;
    double2* En = E + (long long)(j + 1) * D;
    for (int b = tid; b < chiB; b += nth) {
      const int pb = chB[b];
      double2 acc = make_double2(0.0, 0.0);
      if (pair_ok(pb, P)) {
        const int x = pair_c(pb, ncap), y = pair_cb(pb, ncap);
        for (int i = 0; x + i <= ncap && y + i <= ncap; ++i) {
          int a0, a1;
          seg_at(segA, (x + i) * q + (y + i), chiA, a0, a1);
          for (int a = a0; a < a1; ++a) cfma(acc, Ej[a], G[(long long)a * D + b]);
        }
      }
      En[b] = cscale(acc, lB[b]);
    }
    __syncthreads();
  }
  if (tid == 0) F[(long long)M * D] = make_double2(1.0, 0.0);
  __syncthreads();
  for (int j = M - 1; j >= 0; --j) {
    const int chiA = chi_at(s, bi(j)), chiB = chi_at(s, bi(j + 1));
    const int* chA = s.charge + bi(j) * D;
    const int* segB = s.segoff + bi(j + 1) * (P + 1);
    const double2* G = s.gam + ((long long)inst * M + j) * D * D;
    const double* lB = s.lam + bi(j + 1) * D;
    const double2* Fn = F + (long long)(j + 1) * D;
    double2* Fj = F + (long long)j * D;
    for (int a = tid; a < chiA; a += nth) {
      const int pa = chA[a];
      double2 acc = make_double2(0.0, 0.0);
      if (pair_ok(pa, P)) {
        const int x = pair_c(pa, ncap), y = pair_cb(pa, ncap);
        for (int i = 0; i <= x && i <= y; ++i) {
          int b0, b1;
          seg_at(segB, (x - i) * q + (y - i), chiB, b0, b1);
          for (int b = b0; b < b1; ++b) cfma(acc, G[(long long)a * D + b], cscale(Fn[b], lB[b]));
        }
      }
      Fj[a] = acc;
    }
    __syncthreads();
  }
  const double tr = E[(long long)M * D].x;
  if (tid == 0) o[0] = tr;
  for (int j = 0; j < M; ++j) {
    const int chiA = chi_at(s, bi(j)), chiB = chi_at(s, bi(j + 1));
    const int* chA = s.charge + bi(j) * D;
    const int* segB = s.segoff + bi(j + 1) * (P + 1);
    const double2* G = s.gam + ((long long)inst * M + j) * D * D;
    const double* lB = s.lam + bi(j + 1) * D;
    const double2* Ej = E + (long long)j * D;
    const double2* Fn = F + (long long)(j + 1) * D;
    double2 s1 = make_double2(0.0, 0.0), s2 = make_double2(0.0, 0.0);
    for (int a = tid; a < chiA; a += nth) {
      const int pa = chA[a];
      if (!pair_ok(pa, P)) continue;
      const int x = pair_c(pa, ncap), y = pair_cb(pa, ncap);
      double2 acc1 = make_double2(0.0, 0.0), acc2 = make_double2(0.0, 0.0);
      for (int i = 1; i <= x && i <= y; ++i) {
        int b0, b1;
        seg_at(segB, (x - i) * q + (y - i), chiB, b0, b1);
        for (int b = b0; b < b1; ++b) {
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
    const int chi = chi_at(s, bi(b));
    double acc = 0.0;
    for (int i = 0; i < chi; ++i) { const double l = s.lam[bi(b) * D + i]; acc += l * l; }
    o[1 + 2 * M + b] = acc;
  }
}

}  // namespace

void launch_observables(const MpoDev& s, double2* scratch, double* out, cudaStream_t st) {
  k_obs<<<s.B, 256, 0, st>>>(s, scratch, out);
}

// ---------------------------------------------------------------------------
// Observables without any allocation (mpo_observables_static in gbs_mpo.h).
//
// Some callers cannot allocate device memory at the point where they need the
// observables: a host application or framework that owns all device memory
// (its own pool allocator or a fixed, pre-partitioned budget) and forbids direct
// cudaMalloc/cudaFree, for instance because those calls synchronise the device
// and would stall its other work.  This variant runs the same k_obs kernel on a
// single MPO held in buffers the caller already owns; the only scratch it needs,
// the left and right trace environments (2 (M+1) D complex values), lives in the
// file-scope array below.  Every GPU that loads the library keeps this array
// (MPO_STATIC_SCRATCH_ELEMS complex doubles, 1 MiB) until the process exits.
#define MPO_STATIC_SCRATCH_ELEMS (1 << 16)
static __device__ __align__(256) double2 g_obs_scratch[MPO_STATIC_SCRATCH_ELEMS];

namespace {
// Device address of g_obs_scratch per device, looked up by cudaGetSymbolAddress with
// that device current: in host code the symbol's name is only a host-side stand-in,
// never a device address.  The address belongs to the device's current CUDA context,
// so it is cached together with that context's unique ID and looked up again when the
// ID changes (after cudaDeviceReset the runtime creates a new primary context and
// loads the module anew).  The driver calls are reached through the runtime's
// entry-point query, so the library keeps no link-time dependency on libcuda; if the
// query fails, the address is looked up on every call.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double2* g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// ID of the calling thread's current context; false if none is current or the driver
// calls are unavailable.
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_cur = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    cudaGetLastError();  // a failed query leaves no sticky error behind
  }
  if (!get_cur || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_cur(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

cudaError_t static_scratch(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  if (g_scratch_ptr[dev] == nullptr || !have_id || id != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_obs_scratch);  // also makes the primary context current
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double2*>(p);
    g_scratch_ctx[dev] = current_context_id(&id) ? id : 0;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" mpo_status mpo_observables_static(int M, int n_cap, int D, const int* chi, const int* charge,
                                             const int* segoff, const double* lam, const void* gam,
                                             double* out, void* cuda_stream) {
  if (M < 2 || M > 256 || n_cap < 1 || n_cap > MPO_NCAP_MAX || D < 1) return MPO_ERR_ARG;
  if (!chi || !charge || !segoff || !lam || !gam || !out) return MPO_ERR_ARG;
  if (2ll * (M + 1) * D > MPO_STATIC_SCRATCH_ELEMS) return MPO_ERR_CAPACITY;
  double2* scratch = nullptr;
  cudaError_t e = static_scratch(&scratch);
  if (e != cudaSuccess) return MPO_ERR_CUDA;
  MpoDev s{};
  s.B = 1; s.M = M; s.ncap = n_cap; s.P = (n_cap + 1) * (n_cap + 1); s.D = D;
  s.chi = const_cast<int*>(chi);
  s.charge = const_cast<int*>(charge);
  s.segoff = const_cast<int*>(segoff);
  s.lam = const_cast<double*>(lam);
  s.gam = static_cast<double2*>(const_cast<void*>(gam));
  // nothing in the scratch has to start at zero: k_obs writes every environment
  // entry before it reads it
  launch_observables(s, scratch, out, static_cast<cudaStream_t>(cuda_stream));
  return cudaGetLastError() == cudaSuccess ? MPO_OK : MPO_ERR_CUDA;
}
