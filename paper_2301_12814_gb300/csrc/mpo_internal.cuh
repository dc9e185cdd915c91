// Internal layout of the GB300 U(1) MPO library.
//
// Device state of one handle (B instances, M modes, capacity D per bond):
//   chi     [B][M+1]            bond dimensions
//   charge  [B][M+1][D]         pair index p = c*(n_cap+1) + cbar of every bond index,
//                               ascending (indices of one pair form a segment)
//   segoff  [B][M+1][P+1]       segment offsets per pair (P = (n_cap+1)^2)
//   lam     [B][M+1][D]         Vidal weights lambda (float64)
//   gam     [B][M][D][D]        Gamma_j as a dense D x D frame (complex128), row =
//                               bond j index, column = bond j+1 index.  Only entries
//                               whose row charge dominates the column charge
//                               componentwise are meaningful; every reader masks the
//                               rest, so they are never cleared.
//   entropy [B][M+1]
// A gate slot is the scratch of one gate in flight (all gates of a layer run at
// once, one slot each).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

// Host-side NVTX range for the enclosing scope (named gbs_mpo/<what>): marks each
// stage launch and each entry point for Nsight tools; free when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

#define MPO_NCAP_MAX 15
#define MPO_P_MAX ((MPO_NCAP_MAX + 1) * (MPO_NCAP_MAX + 1))
#define MPO_PC_MAX ((MPO_NCAP_MAX + 1) * (MPO_NCAP_MAX + 2) / 2)
#define MPO_FOCK_MAX ((MPO_NCAP_MAX + 1) * (MPO_NCAP_MAX + 2) * (2 * MPO_NCAP_MAX + 3) / 6)
#define MPO_D_LOCAL_MAX 32

// Record a timing event on st.  Under stream capture it becomes an event record node
// of the graph (external event), so it times every replay; outside capture it is an
// ordinary record (the external flag is only valid while capturing).
static inline cudaError_t record_stage_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, st);
}

// device error codes (mirror mpo_status)
#define DEV_ERR_NUMERIC 4
#define DEV_ERR_CAPACITY 6
#define DEV_ERR_INTERNAL 7

struct MpoDev {
  int B, M, ncap, P, D;
  int* chi;
  int* charge;
  int* segoff;
  double* lam;
  double2* gam;
  double* entropy;
  int* chi_cap;   // [B], <= 0 = no cap
  int* err;       // [4]: first error code, info...
  unsigned long long* ctr;  // nullable work counters (profiling replay only), CTR_*
};

// algorithmic work counters (real flops of the executed form)
enum { CTR_THETA = 0, CTR_GRAM, CTR_EIG, CTR_RESPLIT, CTR_SWEEPS, CTR_EIGBLK, CTR_REFINE, CTR_RSWEEPS,
       CTR_NBIG, CTR_CYC_BIG, CTR_CYC_SMALL, CTR_CYC_SEED, CTR_CYC_NS, CTR_CYC_POLISH, CTR_NWARP,
       CTR_CYC_WARP,
       CTR_FTHETA,  // F_Theta: real flops of the one-stage Eq. `theta` over the canonical blocks
       CTR_N };

struct GateDesc {
  int inst, j, out, pad;
  double theta, phi;
};

// Per-canonical-block integer fields (stride Pc in the slot table)
enum BlockField {
  BF_M = 0,      // pair index of the canonical centre charge (c <= cbar)
  BF_R,          // rows of Theta(m)
  BF_C,          // cols of Theta(m)
  BF_G,          // Gram side size min(R, C) (0 = empty block)
  BF_SIDE,       // 0: G = Theta Theta^dag (rows), 1: G = Theta^dag Theta (cols)
  BF_TOFF,       // Theta offset
  BF_GOFF,       // Gram / eigenvector offset
  BF_COFF,       // candidate offset
  BF_RMOFF,      // rowmap offset
  BF_CMOFF,      // colmap offset
  BF_TT,         // theta tile prefix (tiles before this block)
  BF_GT,         // gram tile prefix
  BF_NALIVE,     // eigenvalues above the floor (sorted prefix)
  BF_KEPT,       // kept singular values of this block (and of its mirror)
  BF_NEWPOS,     // first new bond index of this block's kept values
  BF_NEWPOS_MIR, // first new bond index of the mirror block's kept values
  BF_KOFF,       // prefix of kept (resplit work items)
  BF_NFIELDS
};

enum SlotScalar {
  SS_NBLK = 0,  // canonical blocks (Pc, fixed)
  SS_TTILES,    // contraction work items: (row pair a, column pair b) segment pairs
  SS_GTILES,    // total gram tiles
  SS_NITEMS,    // resplit work items
  SS_STATUS,
  SS_NFIELDS
};

struct SlotWS {
  int Pc, D, P;
  long long capTheta, capGram, capRC, capCand;
  int* blk;        // [S][BF_NFIELDS][Pc+1]
  int* scal;       // [S][SS_NFIELDS]
  int* rowoff;     // [S][Pc][P]  offset of segment a within rows of block t (-1 = absent)
  int* coloff;     // [S][Pc][P]
  int* rowmap;     // [S][capRC]
  int* colmap;     // [S][capRC]
  double2* fock;   // [S][MPO_FOCK_MAX]
  double2* theta;  // [S][capTheta]
  double2* G;      // [S][capGram]
  double2* V;      // [S][capGram]
  double* sval;    // [S][capCand]  sorted singular values per block
  int* perm;       // [S][capCand]  eigenvector column of the k-th largest
  double* dscal;   // [S][4]
  int* order;      // [S][capCand*2] candidate ids by rank (select)
  int* items;      // [S][P*P] contraction items a*P + b
  double2* W;      // [S][capTheta] one-sided Jacobi vectors (Theta V or Theta^dag V), column-major
  int big_min;     // > 0: blocks with a Gram side >= big_min go to a CTA cluster (else the load rule)
  int cl_seed_max; // cluster blocks with a Gram side <= this take the single-CTA Gram seed
  // launch choices of the handle (mpo_set_tuning), read on the host when a layer is issued
  int theta_form;  // 0: path default, 1: SIMT two-stage, 2: tensor-core one-stage (FP32 paths)
  int gram_tc_min; // Gram side from which the Gram runs on the tensor cores (0: default)
  int cl_size;     // CTAs per k_svd cluster (0: process default)
  double2* NS;     // [S][capGram] Newton-Schulz scratch V^dag V of the FP64 refinement
  double2* VC;     // [S][capGram] refined right/left factors, column-major, path precision
                   // (never aliases the FP32 Gram or seed buffers of other blocks)
  int* list;       // [S * Pc] layer's blocks, longest first (k_order)
  int* counter;    // [8]: cursors and ends of the cluster, CTA and warp parts of list (k_order)
  // Theta, W (poolTheta entries each) and G, V, NS, VC (poolGram entries each) are pools
  // shared by the slots of a layer: slot s's region starts at poff[2s] (Theta-sized)
  // and poff[2s + 1] (Gram-sized), laid out by the last CTA of k_setup from the slots'
  // actual sizes.  capTheta / capGram are one slot's worst case.
  long long poolTheta, poolGram;
  long long* poff;       // [S][2]
  unsigned int* sctr;    // k_setup arrival counter (the last CTA lays out the pools, resets it)
};

__host__ __device__ inline int pair_c(int p, int ncap) { return p / (ncap + 1); }
__host__ __device__ inline int pair_cb(int p, int ncap) { return p % (ncap + 1); }
__host__ __device__ inline int pair_mirror(int p, int ncap) {
  return (p % (ncap + 1)) * (ncap + 1) + p / (ncap + 1);
}
// Clamped reads of bond tables that may come from caller-owned device buffers
// (k_obs): chi to [0, D], a pair index is usable only inside [0, P), and the segment
// [lo, hi) of pair p to [0, chi] with lo <= hi.  No-ops on valid tables.
__host__ __device__ inline int clamp_chi(int chi, int D) { return chi < 0 ? 0 : (chi > D ? D : chi); }
__host__ __device__ inline bool pair_ok(int p, int P) { return p >= 0 && p < P; }
__host__ __device__ inline void clamp_seg(const int* seg, int p, int chi, int& lo, int& hi) {
  lo = seg[p] < 0 ? 0 : (seg[p] > chi ? chi : seg[p]);
  hi = seg[p + 1] < lo ? lo : (seg[p + 1] > chi ? chi : seg[p + 1]);
}
__host__ __device__ inline int fock_off(int n) { return n * (n + 1) * (2 * n + 1) / 6; }
// inverse of canon_pair for a pair with c <= cbar
__host__ __device__ inline int canon_index(int m, int ncap) {
  const int q = ncap + 1, c = m / q, cb = m % q;
  return c * q - c * (c - 1) / 2 + (cb - c);
}
// canonical block t -> pair index m (pairs with c <= cbar, ascending pair index)
__host__ __device__ inline int canon_pair(int t, int ncap) {
  int q = ncap + 1;
  for (int c = 0; c < q; ++c) {
    int n = q - c;  // pairs (c, cb) with cb >= c
    if (t < n) return c * q + c + t;
    t -= n;
  }
  return -1;
}

// complex helpers (double2 / float2)
template <typename T> struct cplx;
template <> struct cplx<double> { typedef double2 t; };
template <> struct cplx<float> { typedef float2 t; };

__host__ __device__ inline double2 mk(double x, double y) { return make_double2(x, y); }
__host__ __device__ inline float2 mk(float x, float y) { return make_float2(x, y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a += b * c
__host__ __device__ inline void cfma(double2& a, double2 b, double2 c) {
  a.x = fma(b.x, c.x, a.x); a.x = fma(-b.y, c.y, a.x);
  a.y = fma(b.x, c.y, a.y); a.y = fma(b.y, c.x, a.y);
}
__host__ __device__ inline void cfma(float2& a, float2 b, float2 c) {
  a.x = fmaf(b.x, c.x, a.x); a.x = fmaf(-b.y, c.y, a.x);
  a.y = fmaf(b.x, c.y, a.y); a.y = fmaf(b.y, c.x, a.y);
}
// a += conj(b) * c
__host__ __device__ inline void cfma_cj(double2& a, double2 b, double2 c) {
  a.x = fma(b.x, c.x, a.x); a.x = fma(b.y, c.y, a.x);
  a.y = fma(b.x, c.y, a.y); a.y = fma(-b.y, c.x, a.y);
}
__host__ __device__ inline void cfma_cj(float2& a, float2 b, float2 c) {
  a.x = fmaf(b.x, c.x, a.x); a.x = fmaf(b.y, c.y, a.x);
  a.y = fmaf(b.x, c.y, a.y); a.y = fmaf(-b.y, c.x, a.y);
}
__host__ __device__ inline double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ inline double2 to_d2(double2 a) { return a; }
template <typename C> __host__ __device__ inline C from_d2(double2 a);
template <> __host__ __device__ inline double2 from_d2<double2>(double2 a) { return a; }
template <> __host__ __device__ inline float2 from_d2<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

__device__ inline void dev_set_error(int* err, int code, int info) {
  if (atomicCAS(err, 0, code) == 0) err[1] = info;
}

// ---- host-side launchers (defined in the .cu files) ----
void launch_init(const MpoDev& s, const double* d_r, const double* d_eta, int d_local,
                 double* scratch, cudaStream_t st);
void launch_layer(const MpoDev& s, const SlotWS& ws, const GateDesc* d_gates, int ngates,
                  double* d_disc, int prec, cudaStream_t st, int* nlaunch,
                  cudaEvent_t* stage_events = nullptr);
void launch_phases(const MpoDev& s, const double* d_phase, cudaStream_t st);
void launch_observables(const MpoDev& s, double2* scratch, double* out, cudaStream_t st);
