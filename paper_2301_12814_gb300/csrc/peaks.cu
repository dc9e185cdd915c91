// Measured arithmetic peaks of the current GPU, for the roofline denominators of the
// benchmark (a measurement utility; the paper has no counterpart).
//
// * FP64 and FP32 FMA: every thread runs 8 independent fused multiply-add chains
//   x <- x * a + b (a just below 1, so nothing overflows) on a grid of 8 CTAs of 256
//   threads per SM; flops = 2 per FMA.
// * TF32 and BF16 tensor cores: one CTA of 128 threads per SM issues tcgen05.mma of
//   M = 128, N = 256 (K = 8 TF32 / 16 BF16 per instruction) on operands resident in
//   shared memory, accumulating in TMEM; flops = 2 M N K per instruction.  This is the
//   rate of the tensor pipe with no operand traffic, the ceiling a kernel reaches.
// Each measurement is one warm-up launch and one launch timed with CUDA events.
#include "../../include/gbs_mpo.h"
#include "mpo_internal.cuh"
#include "tc.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = x[i] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == (T)-1.2345) out[blockIdx.x] = s;  // keeps the chains live; never true in practice
}

constexpr int PK_N = 256;
template <int BF16>
__global__ void __launch_bounds__(128) k_mma_loop(int reps, int* err) {
  constexpr int KBYTES = 128;  // 32 TF32 / 64 BF16 elements of K resident
  constexpr uint32_t SBO = (KBYTES / 16) * 128;
  extern __shared__ __align__(1024) unsigned char pk[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x;
  // operands: 128 x K (A) and 256 x K (B), any finite values
  uint32_t* w = reinterpret_cast<uint32_t*>(pk);
  const uint32_t bf_one = 0x3f803f80u;  // two BF16 ones
  for (int i = tid; i < (128 + PK_N) * KBYTES / 4; i += 128) w[i] = BF16 ? bf_one : 0x3f800000u;
  if (tid < 32) tc::tmem_alloc(&tslot, 256);
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (tid == 0) {
    const uint32_t a = tc::smem_u32(pk), b = a + 128 * KBYTES;
    constexpr uint32_t id = tc::idesc(128, PK_N, BF16 != 0);
    for (int r = 0; r < reps; ++r)
      for (int s = 0; s < KBYTES / 32; ++s) {
        const uint64_t da = tc::desc(a + 256 * s, 128, SBO), db = tc::desc(b + 256 * s, 128, SBO);
        if (BF16) tc::mma_bf16(tslot, da, db, id, (r | s) ? 1u : 0u);
        else tc::mma_tf32(tslot, da, db, id, (r | s) ? 1u : 0u);
      }
    tc::commit(&bar);
  }
  __syncwarp();
  if (!tc::mbar_wait(&bar, 0) && (tid & 31) == 0) atomicAdd(err, 1);
  tc::fence_before();
  __syncthreads();
  if (tid < 32) tc::tmem_dealloc(tslot, 256);
}

int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <typename L>
cudaError_t time_ms(L launch, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  launch();  // warm-up
  cudaEventRecord(e0);
  launch();
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" mpo_status mpo_measure_peaks(double* tflops, double* ms_out) {
  if (!tflops) return MPO_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return MPO_ERR_NOT_BUILT;
  }
  const int n = sms();
  void* out = nullptr;
  int* err = nullptr;
  if (cudaMalloc(&out, 8 * 4096) != cudaSuccess) return MPO_ERR_OOM;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) { cudaFree(out); return MPO_ERR_OOM; }
  cudaMemset(err, 0, sizeof(int));
  float ms[4] = {0, 0, 0, 0};
  const int grid = 8 * n, threads = 256;
  const int it64 = 2000, it32 = 100000, reps = 4000;
  const size_t pk_smem = (size_t)(128 + PK_N) * 128 + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_mma_loop<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pk_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mma_loop<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pk_smem);
  if (e == cudaSuccess)
    e = time_ms([&] { k_fma_chain<double><<<grid, threads>>>((double*)out, it64, 0.999999, 1e-7); }, &ms[0]);
  if (e == cudaSuccess)
    e = time_ms([&] { k_fma_chain<float><<<grid, threads>>>((float*)out, it32, 0.999999f, 1e-7f); }, &ms[1]);
  if (e == cudaSuccess) e = time_ms([&] { k_mma_loop<0><<<n, 128, pk_smem>>>(reps, err); }, &ms[2]);
  if (e == cudaSuccess) e = time_ms([&] { k_mma_loop<1><<<n, 128, pk_smem>>>(reps, err); }, &ms[3]);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(out);
  cudaFree(err);
  if (e != cudaSuccess) return MPO_ERR_CUDA;
  if (herr) return MPO_ERR_TIMEOUT;
  const double thr = (double)grid * threads * 8.0 * 2.0;
  const double fl[4] = {thr * it64, thr * it32, 2.0 * 128 * PK_N * 32 * (double)reps * n,
                        2.0 * 128 * PK_N * 64 * (double)reps * n};
  for (int i = 0; i < 4; ++i) {
    tflops[i] = ms[i] > 0 ? fl[i] / (ms[i] * 1e-3) / 1e12 : 0.0;
    if (ms_out) ms_out[i] = ms[i];
  }
  return MPO_OK;
}
