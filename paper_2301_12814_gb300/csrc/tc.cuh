// Fifth-generation tensor cores (tcgen05) on sm_103a: the primitives and a CTA-level
// complex tile GEMM used by the contraction, the Gram products and the SVD polish.
//
// Primitives (inline PTX): tensor-memory (TMEM) allocation, shared-memory matrix
// descriptors for the canonical K-major layout without swizzle, tcgen05.mma of
// kind::tf32 and kind::f16 (bf16 operands) with FP32 accumulation in TMEM, commit to
// an mbarrier, a bounded wait on it, and tcgen05.ld of the accumulators.
//
// Operand layout in shared memory (no swizzle, K-major): a "core matrix" is 8 rows x
// 16 bytes stored as 128 contiguous bytes; core matrices adjacent along K are 128
// bytes apart (leading byte offset, LBO) and 8-row groups are SBO = (K bytes / 16) *
// 128 bytes apart.  With this choice the 4-byte word f of a plane sits at byte 4 f,
// where f enumerates (word in chunk, row in group, chunk along K, row group) from the
// fastest to the slowest: a warp writing 32 consecutive words stores 128 contiguous
// bytes, free of bank conflicts.  One MMA consumes 32 bytes of K (8 TF32 or 16 BF16
// elements), i.e. two core matrices along K.
//
// Complex products on real tensor cores: every complex operand is staged as separate
// real and imaginary planes (and, for 3xTF32, high and low parts of each), and three
// FP32 accumulators are kept in TMEM:  acc_rr = sum Ar Br,  acc_ii = sum Ai Bi,
// acc_ri = sum (Ar Bi + Ai Br).  The epilogue forms Re = acc_rr - acc_ii and
// Im = acc_ri, so no operand has to be negated.
//
// Precision modes:
//   TC_TF32  one TF32 product per real product (operands rounded to TF32, ~1e-3 rel)
//   TC_3XTF32  a = a_hi + a_lo with a_hi = tf32(a), a_lo = tf32(a - a_hi); the products
//            a_hi b_hi + a_hi b_lo + a_lo b_hi give FP32-level accuracy (the a_lo b_lo
//            term is below FP32 rounding)
//   TC_BF16  one BF16 product per real product (operands rounded to BF16, ~1e-2 rel)
// Accumulation is FP32 in TMEM in every mode.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace tc {

enum Mode { TC_TF32 = 0, TC_3XTF32 = 1, TC_BF16 = 2 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (SM100 format): start address, LBO and SBO in
// 16-byte units, version 1 at bits 46-47, no swizzle (layout type 0 at bits 61-63).
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32 / kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B formats (bits 7-9, 10-12: TF32 = 2, BF16 = 1), both K-major, N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc(int M, int N, bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 2u) << 7) | ((bf16 ? 1u : 2u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

// Arrive on the mbarrier once every MMA this thread issued so far has completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the phase with the given parity to complete; gives up after `limit` polls
// (each poll may suspend the thread for a while), returning false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long limit = (1L << 24)) {
  const uint32_t a = smem_u32(bar);
  for (long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Generic-proxy stores to shared memory become visible to the tensor cores' async proxy.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation by one whole warp; the base address is written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 16 consecutive FP32 columns of the calling thread's TMEM lane (warp w reads lanes
// 32 (w % 4) .. +31; the lane offset is in bits 16-31 of the address).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t t;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
  return t;
}

// ---------------------------------------------------------------- complex tile GEMM
// C[i][j] = sum_k a(i, k) b(j, k) for one output tile of TM = 128 rows and TN columns
// (TN a multiple of 16, <= 128), with K streamed through shared memory in stages of
// KS elements.  The operand loaders return complex float2 values (zero outside the
// problem); they carry any conjugation, transposition or scaling.  The CTA has
// NT = 256 threads; every thread takes part in staging and in the epilogue.
template <int MODE>
struct CTile {
  static constexpr int TM = 128;
  static constexpr int KS = 32;                              // K elements per stage
  static constexpr int ESZ = MODE == TC_BF16 ? 2 : 4;        // bytes per element
  static constexpr int WPR = KS * ESZ / 4;                   // 4-byte words per row of a plane
  static constexpr int KSTEP = MODE == TC_BF16 ? 16 : 8;     // K elements per MMA
  static constexpr uint32_t LBO = 128, SBO = (WPR / 4) * 128;
  static constexpr int NPL = MODE == TC_3XTF32 ? 4 : 2;      // planes per operand
  static constexpr int NT = 256;
  // bytes of one operand's planes for R rows
  static __host__ __device__ constexpr uint32_t plane_bytes(int R) { return (uint32_t)R * WPR * 4; }
  static __host__ __device__ constexpr uint32_t stage_bytes(int TN) {
    return NPL * (plane_bytes(TM) + plane_bytes(TN));
  }
  // TMEM columns for the three accumulators (power of two >= 32)
  static __host__ __device__ constexpr uint32_t tmem_cols(int TN) {
    return 3 * TN <= 32 ? 32 : 3 * TN <= 64 ? 64 : 3 * TN <= 128 ? 128 : 3 * TN <= 256 ? 256 : 512;
  }
};

// Write one stage of an operand (R rows, K range [k0, k0 + KS)) into its planes.
// Plane order: re, im (, re_lo, im_lo for 3xTF32).  Each thread first gathers U words'
// worth of operand values (U independent loads in flight, which hides the L2 latency
// of the loaders' global reads), then converts and stores them.
template <int MODE, typename Ld>
__device__ __forceinline__ void stage_operand(unsigned char* base, int R, int k0, Ld ld) {
  typedef CTile<MODE> T;
  constexpr int U = 8;
  constexpr int EPW = MODE == TC_BF16 ? 2 : 1;  // elements per 4-byte word
  const uint32_t pb = T::plane_bytes(R);
  uint32_t* p0 = reinterpret_cast<uint32_t*>(base);
  uint32_t* p1 = reinterpret_cast<uint32_t*>(base + pb);
  uint32_t* p2 = reinterpret_cast<uint32_t*>(base + 2 * pb);
  uint32_t* p3 = reinterpret_cast<uint32_t*>(base + 3 * pb);
  const int nw = R * T::WPR;
  for (int f0 = threadIdx.x; f0 < nw; f0 += T::NT * U) {
    float2 v[U][EPW];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int f = f0 + u * T::NT;
      const int w = f & 3, rr = (f >> 2) & 7, rest = f >> 5;
      const int chunk = rest % (T::WPR / 4), rg = rest / (T::WPR / 4);
      const int r = rg * 8 + rr;
      const int k = k0 + chunk * 4 * EPW + EPW * w;
#pragma unroll
      for (int e = 0; e < EPW; ++e) v[u][e] = f < nw ? ld(r, k + e) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int f = f0 + u * T::NT;
      if (f >= nw) break;
      if (MODE == TC_BF16) {
        __nv_bfloat162 re = __floats2bfloat162_rn(v[u][0].x, v[u][EPW - 1].x);
        __nv_bfloat162 im = __floats2bfloat162_rn(v[u][0].y, v[u][EPW - 1].y);
        p0[f] = *reinterpret_cast<uint32_t*>(&re);
        p1[f] = *reinterpret_cast<uint32_t*>(&im);
      } else {
        const float2 x = v[u][0];
        const uint32_t hr = to_tf32(x.x), hi = to_tf32(x.y);
        p0[f] = hr;
        p1[f] = hi;
        if (MODE == TC_3XTF32) {
          p2[f] = to_tf32(x.x - __uint_as_float(hr));
          p3[f] = to_tf32(x.y - __uint_as_float(hi));
        }
      }
    }
  }
}

// Issue the MMAs of one stage (single thread).  first: the stage opens the tile's
// accumulation (the first MMA into each accumulator overwrites it).
template <int MODE, int TN>
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint32_t a_base, uint32_t b_base, bool first) {
  typedef CTile<MODE> T;
  constexpr uint32_t id = idesc(T::TM, TN, MODE == TC_BF16);
  const uint32_t pa = T::plane_bytes(T::TM), pbb = T::plane_bytes(TN);
  const uint32_t acc_rr = tmem, acc_ii = tmem + TN, acc_ri = tmem + 2 * TN;
#pragma unroll
  for (int s = 0; s < T::KS / T::KSTEP; ++s) {
    const uint32_t ko = s * 2 * T::LBO;
    const uint32_t first_k = (first && s == 0) ? 0u : 1u;
    auto A = [&](int pl) { return desc(a_base + pl * pa + ko, T::LBO, T::SBO); };
    auto B = [&](int pl) { return desc(b_base + pl * pbb + ko, T::LBO, T::SBO); };
    if (MODE == TC_BF16) {
      mma_bf16(acc_rr, A(0), B(0), id, first_k);
      mma_bf16(acc_ii, A(1), B(1), id, first_k);
      mma_bf16(acc_ri, A(0), B(1), id, first_k);
      mma_bf16(acc_ri, A(1), B(0), id, 1u);
    } else {
      mma_tf32(acc_rr, A(0), B(0), id, first_k);
      mma_tf32(acc_ii, A(1), B(1), id, first_k);
      mma_tf32(acc_ri, A(0), B(1), id, first_k);
      mma_tf32(acc_ri, A(1), B(0), id, 1u);
      if (MODE == TC_3XTF32) {  // + hi*lo + lo*hi of every real product
        mma_tf32(acc_rr, A(0), B(2), id, 1u);
        mma_tf32(acc_rr, A(2), B(0), id, 1u);
        mma_tf32(acc_ii, A(1), B(3), id, 1u);
        mma_tf32(acc_ii, A(3), B(1), id, 1u);
        mma_tf32(acc_ri, A(0), B(3), id, 1u);
        mma_tf32(acc_ri, A(2), B(1), id, 1u);
        mma_tf32(acc_ri, A(1), B(2), id, 1u);
        mma_tf32(acc_ri, A(3), B(0), id, 1u);
      }
    }
  }
}

// State of one CTA's tensor-core engine: the TMEM base, the mbarrier and its phase.
struct Engine {
  uint32_t tmem;
  uint64_t* bar;
  uint32_t phase;
  int* err;  // device error word (first code wins); a timed-out wait records a code
};

struct NoPrep {
  __device__ __forceinline__ bool operator()(int) const { return false; }
};

// One output tile: K in [0, K) streamed in stages through smem (one buffer; the MMAs
// of a stage run while nothing else uses the buffer).  store(i, j, re, im) receives
// every element of the TM x TN tile (rows i in [0, 128), columns j in [0, TN)).
// prep(k0), called by every thread before stage k0 is loaded, may fill per-stage
// tables in shared memory; it returns true if it wrote any (a barrier then follows).
// Returns false if a wait timed out (the error word is then set).
template <int MODE, int TN, typename LdA, typename LdB, typename St, typename Pr = NoPrep>
__device__ bool tile_gemm(Engine& E, unsigned char* smem, int K, LdA lda, LdB ldb, St store, Pr prep = Pr()) {
  typedef CTile<MODE> T;
  static_assert(TN % 32 == 0 && TN >= 32 && TN <= 128, "TN: 32, 64, 96 or 128 columns");
  unsigned char* sa = smem;
  unsigned char* sb = smem + T::NPL * T::plane_bytes(T::TM);
  const uint32_t a_base = smem_u32(sa), b_base = smem_u32(sb);
  bool ok = true;
  const int nst = K > 0 ? (K + T::KS - 1) / T::KS : 0;
  for (int st = 0; st < nst; ++st) {
    const int k0 = st * T::KS;
    if (prep(k0)) __syncthreads();
    stage_operand<MODE>(sa, T::TM, k0, lda);
    stage_operand<MODE>(sb, TN, k0, ldb);
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_after();
      issue_stage<MODE, TN>(E.tmem, a_base, b_base, st == 0);
      commit(E.bar);
    }
    // the buffer is rewritten by the next stage: wait until these MMAs have read it
    // (the decision is made CTA-wide, so every thread leaves the loop together)
    const bool w = mbar_wait(E.bar, E.phase);
    E.phase ^= 1u;
    if (!__syncthreads_and(w)) {
      ok = false;
      if (threadIdx.x == 0) atomicCAS(E.err, 0, 5 /* MPO_ERR_TIMEOUT */);
      break;
    }
  }
  fence_after();
  // epilogue: warp w reads TMEM lanes 32 (w % 4).. and the column half w / 4
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (warp & 3) + lane;
  const uint32_t lane_addr = E.tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  constexpr int HALF = TN / 2;
  for (int c0 = (warp >> 2) * HALF; c0 < (warp >> 2) * HALF + HALF; c0 += 16) {
    float rr[16], ii[16], ri[16];
    if (ok && nst > 0) {
      tmem_ld16(lane_addr + c0, rr);
      tmem_ld16(lane_addr + TN + c0, ii);
      tmem_ld16(lane_addr + 2 * TN + c0, ri);
    } else {
#pragma unroll
      for (int x = 0; x < 16; ++x) { rr[x] = 0.f; ii[x] = 0.f; ri[x] = 0.f; }
    }
#pragma unroll
    for (int x = 0; x < 16; ++x) store(row, c0 + x, rr[x] - ii[x], ri[x]);
  }
  // every thread has read its accumulators before the next tile's MMAs overwrite them
  fence_before();
  __syncthreads();
  return ok;
}

}  // namespace tc
