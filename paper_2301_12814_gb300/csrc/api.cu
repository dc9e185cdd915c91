// C ABI of the GB300 U(1) MPO beam-splitter mesh (declared in include/gbs_mpo.h).
//
// Host responsibilities only: argument checks, device memory ownership, the layer
// schedule of a mesh (gates on disjoint mode pairs commute and run in one batched
// pass, the single-GPU form of the paper's gate-level parallelism, App. D.4),
// CUDA-graph capture of a planned mesh, and polling of the device error flag.
// Every arithmetic step of the method runs in the kernels of init.cu, gate.cu and
// obs.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/gbs_mpo.h"
#include "mpo_internal.cuh"

size_t eig_smem_bytes(int D);
cudaError_t gate_module_init();
int svd_big_min();
int svd_cluster_seed_max();
int svd_cluster_info(int* cluster_size, int* clusters_fp64, int* clusters_fp32);

// Device allocator of handles and plans: the CUDA runtime, or a caller's pair
// installed by mpo_set_allocator (copied into each handle when it is created, so a
// handle always frees with the functions that allocated its memory).
struct DevAllocator {
  mpo_alloc_fn alloc = nullptr;
  mpo_free_fn free = nullptr;
  void* ctx = nullptr;
};
DevAllocator g_allocator;
std::mutex g_allocator_mu;

struct mpo_ctx {
  DevAllocator al;
  int M = 0, d = 0, ncap = 0, B = 0, P = 0, Pc = 0, D = 0;
  int prec = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* state = nullptr;   // chi | charge | segoff | lam | entropy | gam
  void* snap = nullptr;
  size_t state_bytes = 0;
  MpoDev dev{};
  int* d_err = nullptr;
  int* d_chicap = nullptr;
  std::vector<int> chicap;
  std::vector<double> kept;   // [B] probability kept by the Fock and photon-number cut
  // gate workspace
  void* ws_buf = nullptr;
  SlotWS ws{};
  int nslots = 0;
  // single-gate helpers
  GateDesc* d_gate1 = nullptr;
  double* d_disc1 = nullptr;
  // observables
  double2* d_obs_scratch = nullptr;
  double* d_obs_out = nullptr;
  // pinned host staging for mpo_sweep_mesh (gate descriptors in, discarded weights out)
  void* pin = nullptr;
  size_t pin_bytes = 0;
  std::vector<mpo_plan> plans;  // live plans; mpo_destroy destroys them first
  int poisoned = 0;
  mpo_tuning tun{0, 0, 0, 0, -1};  // launch choices (mpo_set_tuning); defaults
};

struct mpo_plan_s {
  mpo_handle h = nullptr;
  std::vector<int> layer_off, layer_cnt;
  GateDesc* d_gates = nullptr;
  double* d_disc = nullptr;
  double* d_phase = nullptr;
  int ngates = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
  // stage events captured in the graph: per layer MPO_NSTAGES, then two around the
  // phase screen
  std::vector<cudaEvent_t> ev;
  int runs = 0;
};

namespace {

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Long-lived buffers: cudaMalloc, or the caller's allocator on the handle's stream.
cudaError_t dev_alloc(const mpo_ctx* h, void** p, size_t bytes) {
  *p = nullptr;
  if (h->al.alloc) {
    *p = h->al.alloc(bytes, (void*)h->stream, h->al.ctx);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}
void dev_free(const mpo_ctx* h, void* p) {
  if (!p) return;
  if (h && h->al.free) h->al.free(p, (void*)h->stream, h->al.ctx);
  else cudaFree(p);
}
// Per-call temporaries: stream-ordered (cudaMallocAsync on the handle's stream), or the
// caller's allocator.
cudaError_t tmp_alloc(const mpo_ctx* h, void** p, size_t bytes) {
  *p = nullptr;
  if (h->al.alloc) return dev_alloc(h, p, bytes);
  return cudaMallocAsync(p, bytes, h->stream);
}
void tmp_free(const mpo_ctx* h, void* p) {
  if (!p) return;
  if (h->al.free) h->al.free(p, (void*)h->stream, h->al.ctx);
  else cudaFreeAsync(p, h->stream);
}

// Runs a cleanup when the scope ends, on error returns too.
template <typename F>
struct ScopeExit {
  F f;
  ~ScopeExit() { f(); }
};
template <typename F>
ScopeExit<F> on_scope_exit(F f) {
  return ScopeExit<F>{f};
}

mpo_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MPO_OK;
  if (e == cudaErrorMemoryAllocation) return MPO_ERR_OOM;
  return MPO_ERR_CUDA;
}

#define CK(call)                                       \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      return cuda_status(e_);                          \
    }                                                  \
  } while (0)

// number of configurations of k modes (photons 0..d-1 each) with total exactly x
double n_configs(int k, int x, int d) {
  std::vector<double> cur(x + 1, 0.0), nxt(x + 1);
  cur[0] = 1.0;
  for (int m = 0; m < k; ++m) {
    std::fill(nxt.begin(), nxt.end(), 0.0);
    for (int t = 0; t <= x; ++t)
      for (int n = 0; n < d && n <= t; ++n) nxt[t] += cur[t - n];
    cur.swap(nxt);
  }
  return cur[x];
}

// largest exact Schmidt rank over the bonds of the capped augmented state
long long exact_rank_bound(int M, int d, int ncap) {
  double best = 0.0;
  for (int b = 0; b <= M; ++b) {
    double tot = 0.0;
    for (int c = 0; c <= ncap; ++c)
      for (int cb = 0; cb <= ncap; ++cb) {
        double R = n_configs(M - b, c, d) * n_configs(M - b, cb, d);
        double L1 = 0.0, L2 = 0.0;
        for (int x = 0; x <= ncap - c; ++x) L1 += n_configs(b, x, d);
        for (int x = 0; x <= ncap - cb; ++x) L2 += n_configs(b, x, d);
        tot += std::min(R, L1 * L2);
      }
    best = std::max(best, tot);
  }
  return best > 1e9 ? (long long)1e9 : (long long)best;
}

mpo_status poll_error(mpo_handle h) {
  int err[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(err, h->d_err, sizeof(err), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (err[0] != 0) {
    h->poisoned = 1;
    fprintf(stderr, "gbs_mpo: device error %d (info %d)\n", err[0], err[1]);
    return (mpo_status)err[0];
  }
  return MPO_OK;
}

// The handle's launch choices in the workspace descriptor.  Cluster routing: the load
// rule, GBS_MPO_SVD_CLUSTER_MIN_N, or the handle's threshold (negative: no block goes
// to a cluster).  Cluster blocks on the FP64 path all run the FP32 one-sided cluster
// phase: its seed keeps the small singular values (a Gram seed squares their
// conditioning), so the critical blocks' FP64 polish needs 2 sweeps instead of 3 to 4
// (16 modes, chi = 64: 6543 -> 8218 updates/s).  On the FP32 path the single-CTA Gram
// seed stays for Gram sides up to 64.  GBS_MPO_SVD_CLUSTER_SEED_MAX or the handle's
// value overrides both.
void apply_tuning(const mpo_ctx* h, SlotWS& w) {
  const mpo_tuning& t = h->tun;
  w.big_min = t.svd_cluster_min_n > 0 ? t.svd_cluster_min_n : t.svd_cluster_min_n < 0 ? 0x3fffffff : svd_big_min();
  const int sm = t.svd_cluster_seed_max >= 0 ? t.svd_cluster_seed_max : svd_cluster_seed_max();
  w.cl_seed_max = sm >= 0 ? sm : (h->prec == MPO_FP64 ? 0 : 64);
  w.theta_form = t.theta_form;
  w.gram_tc_min = t.gram_tc_min;
  w.cl_size = t.svd_cluster_size;
}

mpo_status ensure_slots(mpo_handle h, int need) {
  if (need <= h->nslots) return MPO_OK;
  if (h->ws_buf) {
    CK(cudaStreamSynchronize(h->stream));
    dev_free(h, h->ws_buf);
    h->ws_buf = nullptr;
    h->nslots = 0;  // no workspace until the new one is in place
  }
  SlotWS w{};
  w.Pc = h->Pc; w.D = h->D; w.P = h->P;
  apply_tuning(h, w);
  const long long D = h->D;
  w.capRC = (long long)h->Pc * D;
  w.capCand = (long long)h->Pc * D;
  w.capTheta = (long long)h->Pc * D * D;  // one slot's worst case
  w.capGram = w.capTheta;
  const int S = need;
  // Theta, W, G, V, NS and VC are pools shared by a layer's slots (k_setup lays them
  // out from the actual block sizes, which are far below the worst case S x Pc D^2 at
  // large chi).  Each pool holds the worst case if that fits a budget for the six
  // pools -- GBS_MPO_WORKSPACE_GB, else a quarter of the free device memory -- and the
  // budget otherwise; a layer whose blocks do not fit fails with MPO_ERR_CAPACITY.
  {
    const long long worst = (long long)S * w.capTheta;
    size_t freeb = 0, totalb = 0;
    CK(cudaMemGetInfo(&freeb, &totalb));
    const char* env = getenv("GBS_MPO_WORKSPACE_GB");
    const double gb = env ? atof(env) : 0.0;
    const double bytes = gb > 0.0 ? gb * (double)(1ll << 30) : 0.25 * (double)freeb;
    const long long budget = std::max(1ll, (long long)(bytes / (6.0 * sizeof(double2))));
    w.poolTheta = std::min(worst, budget);
    w.poolGram = w.poolTheta;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  size_t o_blk = take((size_t)S * BF_NFIELDS * (w.Pc + 1) * sizeof(int));
  size_t o_scal = take((size_t)S * SS_NFIELDS * sizeof(int));
  size_t o_ro = take((size_t)S * w.Pc * w.P * sizeof(int));
  size_t o_co = take((size_t)S * w.Pc * w.P * sizeof(int));
  size_t o_rm = take((size_t)S * w.capRC * sizeof(int));
  size_t o_cm = take((size_t)S * w.capRC * sizeof(int));
  size_t o_fk = take((size_t)S * MPO_FOCK_MAX * sizeof(double2));
  size_t o_th = take((size_t)w.poolTheta * sizeof(double2));
  size_t o_g = take((size_t)w.poolGram * sizeof(double2));
  size_t o_v = take((size_t)w.poolGram * sizeof(double2));
  size_t o_sv = take((size_t)S * w.capCand * sizeof(double));
  size_t o_pm = take((size_t)S * w.capCand * sizeof(int));
  size_t o_ds = take((size_t)S * 4 * sizeof(double));
  size_t o_or = take((size_t)S * w.capCand * 2 * sizeof(int));
  size_t o_it = take((size_t)S * w.P * w.P * sizeof(int));
  size_t o_w = take((size_t)w.poolTheta * sizeof(double2));
  size_t o_ns = take((size_t)w.poolGram * sizeof(double2));
  size_t o_vc = take((size_t)w.poolGram * sizeof(double2));
  size_t o_ls = take((size_t)S * w.Pc * sizeof(int));
  size_t o_ct = take(8 * sizeof(int));
  size_t o_po = take((size_t)S * 2 * sizeof(long long));
  size_t o_sc = take(sizeof(unsigned int));
  void* buf = nullptr;
  CK(dev_alloc(h, &buf, off));
  const cudaError_t me = cudaMemsetAsync(buf, 0, off, h->stream);
  if (me != cudaSuccess) {
    dev_free(h, buf);
    return cuda_status(me);
  }
  char* b = (char*)buf;
  w.blk = (int*)(b + o_blk); w.scal = (int*)(b + o_scal); w.rowoff = (int*)(b + o_ro);
  w.coloff = (int*)(b + o_co); w.rowmap = (int*)(b + o_rm); w.colmap = (int*)(b + o_cm);
  w.fock = (double2*)(b + o_fk); w.theta = (double2*)(b + o_th); w.G = (double2*)(b + o_g);
  w.V = (double2*)(b + o_v); w.sval = (double*)(b + o_sv); w.perm = (int*)(b + o_pm);
  w.dscal = (double*)(b + o_ds); w.order = (int*)(b + o_or); w.items = (int*)(b + o_it); w.W = (double2*)(b + o_w); w.NS = (double2*)(b + o_ns); w.VC = (double2*)(b + o_vc);
  w.list = (int*)(b + o_ls); w.counter = (int*)(b + o_ct);
  w.poff = (long long*)(b + o_po); w.sctr = (unsigned int*)(b + o_sc);
  h->ws_buf = buf;
  h->ws = w;
  h->nslots = S;
  return MPO_OK;
}

// Greedy layering per instance; layer l of the plan holds every instance's layer l.
mpo_status build_schedule(mpo_handle h, const int* n_gates, const int* k, const double* theta,
                          const double* phi, std::vector<GateDesc>& out, std::vector<int>& loff,
                          std::vector<int>& lcnt, int& total) {
  total = 0;
  for (int i = 0; i < h->B; ++i) {
    if (n_gates[i] < 0) return MPO_ERR_ARG;
    total += n_gates[i];
  }
  std::vector<std::vector<GateDesc>> layers;
  int g0 = 0;
  for (int i = 0; i < h->B; ++i) {
    std::vector<int> last(h->M, -1);
    for (int t = 0; t < n_gates[i]; ++t) {
      const int gi = g0 + t;
      const int kk = k[gi];
      if (kk < 0 || kk > h->M - 2 || !std::isfinite(theta[gi]) || !std::isfinite(phi[gi])) return MPO_ERR_ARG;
      const int l = std::max(last[kk], last[kk + 1]) + 1;
      last[kk] = last[kk + 1] = l;
      if ((int)layers.size() <= l) layers.resize(l + 1);
      GateDesc gd{};
      gd.inst = i; gd.j = kk; gd.out = gi; gd.theta = theta[gi]; gd.phi = phi[gi];
      layers[l].push_back(gd);
    }
    g0 += n_gates[i];
  }
  out.clear(); loff.clear(); lcnt.clear();
  for (auto& L : layers) {
    loff.push_back((int)out.size());
    lcnt.push_back((int)L.size());
    out.insert(out.end(), L.begin(), L.end());
  }
  return MPO_OK;
}

// ev (nullable): MPO_NSTAGES events per layer, then two around the phase screen.
mpo_status run_layers(mpo_handle h, const GateDesc* d_gates, const std::vector<int>& loff,
                      const std::vector<int>& lcnt, double* d_disc, const double* d_phase, int* launches,
                      cudaEvent_t* ev = nullptr) {
  const size_t L = loff.size();
  for (size_t l = 0; l < L; ++l) {
    launch_layer(h->dev, h->ws, d_gates + loff[l], lcnt[l], d_disc, h->prec, h->stream, launches,
                 ev ? ev + l * MPO_NSTAGES : nullptr);
    CK(cudaGetLastError());
  }
  if (ev) CK(record_stage_event(ev[L * MPO_NSTAGES], h->stream));
  if (d_phase) {
    launch_phases(h->dev, d_phase, h->stream);
    if (launches) *launches += 1;
    CK(cudaGetLastError());
  }
  if (ev) CK(record_stage_event(ev[L * MPO_NSTAGES + 1], h->stream));
  return MPO_OK;
}

}  // namespace

extern "C" {

const char* mpo_status_string(mpo_status s) {
  switch (s) {
    case MPO_OK: return "ok";
    case MPO_ERR_ARG: return "invalid argument";
    case MPO_ERR_OOM: return "device out of memory";
    case MPO_ERR_CUDA: return "CUDA runtime error";
    case MPO_ERR_NUMERIC: return "numerical failure (eigensolver sweep cap or non-finite value)";
    case MPO_ERR_TIMEOUT: return "bounded device wait ran out";
    case MPO_ERR_CAPACITY: return "workspace capacity exceeded (layer pools or a per-gate table)";
    case MPO_ERR_INTERNAL: return "device consistency check failed";
    case MPO_ERR_POISONED: return "handle poisoned by an earlier device error";
    case MPO_ERR_NOT_BUILT: return "CUDA library unavailable";
  }
  return "unknown status";
}

mpo_status mpo_init_lossy_squeezed(mpo_handle* out, const mpo_params* p, const double* r,
                                   const double* eta) {
  NvtxRange nv("gbs_mpo/init");
  if (!out || !p || !r || !eta) return MPO_ERR_ARG;
  *out = nullptr;
  const int M = p->M, d = p->d, B = p->batch;
  const int ncap = p->n_cap <= 0 ? d - 1 : p->n_cap;
  if (M < 2 || M > 256 || d < 2 || d > MPO_D_LOCAL_MAX || B < 1 || ncap > d - 1 || ncap > MPO_NCAP_MAX)
    return MPO_ERR_ARG;
  if (p->prec != MPO_FP64 && p->prec != MPO_MIXED_TF32 && p->prec != MPO_MIXED_BF16) return MPO_ERR_ARG;
  for (long long i = 0; i < (long long)B * M; ++i) {
    if (!(r[i] >= 0.0 && r[i] <= 3.0) || !(eta[i] >= 0.0 && eta[i] <= 1.0)) return MPO_ERR_ARG;
  }
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) return MPO_ERR_NOT_BUILT;
  mpo_ctx* h = new (std::nothrow) mpo_ctx();
  if (!h) return MPO_ERR_OOM;
  {
    std::lock_guard<std::mutex> lk(g_allocator_mu);
    h->al = g_allocator;
  }
  h->M = M; h->d = d; h->ncap = ncap; h->B = B;
  h->P = (ncap + 1) * (ncap + 1);
  h->Pc = (ncap + 1) * (ncap + 2) / 2;
  h->prec = p->prec;
  h->chicap.resize(B);
  long long D = h->P;
  bool any_nocap = false;
  for (int i = 0; i < B; ++i) {
    int c = p->chi_max ? p->chi_max[i] : 0;
    h->chicap[i] = c;
    if (c <= 0) any_nocap = true;
    else D = std::max<long long>(D, c);
  }
  if (any_nocap) D = std::max<long long>(D, exact_rank_bound(M, d, ncap));
  D = (D + 7) / 8 * 8;
  if (D > 4096) { delete h; return MPO_ERR_ARG; }
  h->D = (int)D;
  if (p->cuda_stream) h->stream = (cudaStream_t)p->cuda_stream;
  else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) { delete h; return MPO_ERR_CUDA; }
    h->own_stream = true;
  }
  // state layout
  const long long nb = (long long)B * (M + 1);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  size_t o_chi = take(nb * sizeof(int));
  size_t o_ch = take(nb * D * sizeof(int));
  size_t o_seg = take(nb * (h->P + 1) * sizeof(int));
  size_t o_lam = take(nb * D * sizeof(double));
  size_t o_ent = take(nb * sizeof(double));
  size_t o_gam = take((size_t)B * M * D * D * sizeof(double2));
  h->state_bytes = off;
  mpo_status st = MPO_OK;
  auto fail = [&](mpo_status s) { mpo_destroy(h); return s; };
  if (dev_alloc(h, &h->state, off) != cudaSuccess) return fail(MPO_ERR_OOM);
  if (dev_alloc(h, &h->snap, off) != cudaSuccess) return fail(MPO_ERR_OOM);
  if (cudaMemsetAsync(h->state, 0, off, h->stream) != cudaSuccess) return fail(MPO_ERR_CUDA);
  char* sb = (char*)h->state;
  MpoDev& dv = h->dev;
  dv.B = B; dv.M = M; dv.ncap = ncap; dv.P = h->P; dv.D = (int)D;
  dv.chi = (int*)(sb + o_chi); dv.charge = (int*)(sb + o_ch); dv.segoff = (int*)(sb + o_seg);
  dv.lam = (double*)(sb + o_lam); dv.entropy = (double*)(sb + o_ent); dv.gam = (double2*)(sb + o_gam);
  if (dev_alloc(h, (void**)&h->d_err, 4 * sizeof(int)) != cudaSuccess) return fail(MPO_ERR_OOM);
  if (dev_alloc(h, (void**)&h->d_chicap, B * sizeof(int)) != cudaSuccess) return fail(MPO_ERR_OOM);
  dv.err = h->d_err; dv.chi_cap = h->d_chicap;
  if (cudaMemsetAsync(h->d_err, 0, 4 * sizeof(int), h->stream) != cudaSuccess) return fail(MPO_ERR_CUDA);
  if (cudaMemcpyAsync(h->d_chicap, h->chicap.data(), B * sizeof(int), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return fail(MPO_ERR_CUDA);
  // init scratch
  const long long per = (long long)(M + 1) * h->P * 3 + (long long)M * h->P * 2 + 64;
  double* d_scr = nullptr; double* d_re = nullptr;
  if (dev_alloc(h, (void**)&d_scr, per * B * sizeof(double)) != cudaSuccess) return fail(MPO_ERR_OOM);
  if (dev_alloc(h, (void**)&d_re, 2ll * B * M * sizeof(double)) != cudaSuccess) { dev_free(h, d_scr); return fail(MPO_ERR_OOM); }
  cudaMemcpyAsync(d_re, r, (size_t)B * M * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(d_re + (size_t)B * M, eta, (size_t)B * M * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  launch_init(h->dev, d_re, d_re + (size_t)B * M, d, d_scr, h->stream);
  cudaError_t e = cudaGetLastError();
  // k_init leaves each instance's kept probability T in the first slot after its
  // per-mode tables; one strided copy gathers them before the scratch is freed.
  h->kept.assign(B, 0.0);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(h->kept.data(), sizeof(double), d_scr + (per - 64), per * sizeof(double),
                          sizeof(double), B, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, d_scr); dev_free(h, d_re);
  if (e != cudaSuccess) return fail(cuda_status(e));
  if (gate_module_init() != cudaSuccess) return fail(MPO_ERR_CUDA);
  st = poll_error(h);
  if (st != MPO_OK) return fail(st);
  if (cudaMemcpyAsync(h->snap, h->state, off, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
    return fail(MPO_ERR_CUDA);
  // helpers
  if (dev_alloc(h, (void**)&h->d_gate1, sizeof(GateDesc)) != cudaSuccess) return fail(MPO_ERR_OOM);
  if (dev_alloc(h, (void**)&h->d_disc1, sizeof(double)) != cudaSuccess) return fail(MPO_ERR_OOM);
  if (dev_alloc(h, (void**)&h->d_obs_scratch, 2ll * B * (M + 1) * D * sizeof(double2)) != cudaSuccess) return fail(MPO_ERR_OOM);
  if (dev_alloc(h, (void**)&h->d_obs_out, (size_t)B * (1 + 2 * M + M + 1) * sizeof(double)) != cudaSuccess)
    return fail(MPO_ERR_OOM);
  st = ensure_slots(h, 1);
  if (st != MPO_OK) return fail(st);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(MPO_ERR_CUDA);
  *out = h;
  return MPO_OK;
}

mpo_status mpo_reset(mpo_handle h) {
  if (!h) return MPO_ERR_ARG;
  if (h->poisoned) return MPO_ERR_POISONED;
  CK(cudaMemcpyAsync(h->state, h->snap, h->state_bytes, cudaMemcpyDeviceToDevice, h->stream));
  return MPO_OK;
}

mpo_status mpo_apply_bs(mpo_handle h, int inst, int k, double theta, double phi, double* discarded_weight) {
  NvtxRange nv("gbs_mpo/apply_bs");
  if (!h) return MPO_ERR_ARG;
  if (h->poisoned) return MPO_ERR_POISONED;
  if (inst < 0 || inst >= h->B || k < 0 || k > h->M - 2 || !std::isfinite(theta) || !std::isfinite(phi))
    return MPO_ERR_ARG;
  GateDesc gd{};
  gd.inst = inst; gd.j = k; gd.out = 0; gd.theta = theta; gd.phi = phi;
  CK(cudaMemcpyAsync(h->d_gate1, &gd, sizeof(gd), cudaMemcpyHostToDevice, h->stream));
  launch_layer(h->dev, h->ws, h->d_gate1, 1, h->d_disc1, h->prec, h->stream, nullptr);
  CK(cudaGetLastError());
  if (discarded_weight) {
    CK(cudaMemcpyAsync(discarded_weight, h->d_disc1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return poll_error(h);
  }
  CK(cudaStreamSynchronize(h->stream));  // the host GateDesc must outlive the copy
  return MPO_OK;
}

mpo_status mpo_sweep_mesh(mpo_handle h, const int* n_gates, const int* k, const double* theta,
                          const double* phi, const double* final_phase, double* discarded) {
  NvtxRange nv("gbs_mpo/sweep_mesh");
  if (!h || !n_gates || !k || !theta || !phi) return MPO_ERR_ARG;
  if (h->poisoned) return MPO_ERR_POISONED;
  std::vector<GateDesc> gates;
  std::vector<int> loff, lcnt;
  int total = 0;
  mpo_status st = build_schedule(h, n_gates, k, theta, phi, gates, loff, lcnt, total);
  if (st != MPO_OK) return st;
  int maxl = 1;
  for (int c : lcnt) maxl = std::max(maxl, c);
  st = ensure_slots(h, maxl);
  if (st != MPO_OK) return st;
  GateDesc* d_g = nullptr; double* d_disc = nullptr; double* d_ph = nullptr;
  auto release = on_scope_exit([&] {
    tmp_free(h, d_g);
    tmp_free(h, d_disc);
    tmp_free(h, d_ph);
  });
  const size_t ng = std::max<size_t>(1, gates.size());
  const size_t nph = final_phase ? (size_t)h->B * h->M : 0;
  // pinned staging: [gates | phases | discarded]
  const size_t need = align_up(ng * sizeof(GateDesc)) + align_up(nph * sizeof(double) + 8) +
                      align_up(std::max(1, total) * sizeof(double));
  if (need > h->pin_bytes) {
    CK(cudaStreamSynchronize(h->stream));
    if (h->pin) cudaFreeHost(h->pin);
    h->pin = nullptr; h->pin_bytes = 0;
    CK(cudaHostAlloc(&h->pin, need, cudaHostAllocDefault));
    h->pin_bytes = need;
  }
  char* pb = (char*)h->pin;
  GateDesc* hg = (GateDesc*)pb;
  double* hph = (double*)(pb + align_up(ng * sizeof(GateDesc)));
  double* hdisc = (double*)(pb + align_up(ng * sizeof(GateDesc)) + align_up(nph * sizeof(double) + 8));
  if (!gates.empty()) std::memcpy(hg, gates.data(), gates.size() * sizeof(GateDesc));
  if (nph) std::memcpy(hph, final_phase, nph * sizeof(double));
  CK(tmp_alloc(h, (void**)&d_g, ng * sizeof(GateDesc)));
  CK(tmp_alloc(h, (void**)&d_disc, std::max(1, total) * sizeof(double)));
  if (nph) CK(tmp_alloc(h, (void**)&d_ph, nph * sizeof(double)));
  if (!gates.empty())
    CK(cudaMemcpyAsync(d_g, hg, gates.size() * sizeof(GateDesc), cudaMemcpyHostToDevice, h->stream));
  if (nph) CK(cudaMemcpyAsync(d_ph, hph, nph * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  st = run_layers(h, d_g, loff, lcnt, d_disc, d_ph, nullptr);
  if (st == MPO_OK && discarded && total > 0)
    st = cuda_status(cudaMemcpyAsync(hdisc, d_disc, total * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (st != MPO_OK) return st;
  st = poll_error(h);
  if (st == MPO_OK && discarded && total > 0) std::memcpy(discarded, hdisc, total * sizeof(double));
  return st;
}

mpo_status mpo_plan_mesh(mpo_handle h, const int* n_gates, const int* k, const double* theta,
                         const double* phi, const double* final_phase, mpo_plan* out) {
  if (!h || !n_gates || !k || !theta || !phi || !out) return MPO_ERR_ARG;
  if (h->poisoned) return MPO_ERR_POISONED;
  *out = nullptr;
  mpo_plan_s* pl = new (std::nothrow) mpo_plan_s();
  if (!pl) return MPO_ERR_OOM;
  pl->h = h;
  std::vector<GateDesc> gates;
  int total = 0;
  mpo_status st = build_schedule(h, n_gates, k, theta, phi, gates, pl->layer_off, pl->layer_cnt, total);
  if (st != MPO_OK) { delete pl; return st; }
  pl->ngates = total;
  int maxl = 1;
  for (int c : pl->layer_cnt) maxl = std::max(maxl, c);
  st = ensure_slots(h, maxl);
  if (st != MPO_OK) { delete pl; return st; }
  auto fail = [&](mpo_status s) { mpo_plan_destroy(pl); return s; };
  if (dev_alloc(h, (void**)&pl->d_gates, std::max<size_t>(1, gates.size()) * sizeof(GateDesc)) != cudaSuccess) return fail(MPO_ERR_OOM);
  if (dev_alloc(h, (void**)&pl->d_disc, std::max(1, total) * sizeof(double)) != cudaSuccess) return fail(MPO_ERR_OOM);
  if (!gates.empty() && cudaMemcpy(pl->d_gates, gates.data(), gates.size() * sizeof(GateDesc),
                                   cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(MPO_ERR_CUDA);
  if (final_phase) {
    if (dev_alloc(h, (void**)&pl->d_phase, (size_t)h->B * h->M * sizeof(double)) != cudaSuccess) return fail(MPO_ERR_OOM);
    if (cudaMemcpy(pl->d_phase, final_phase, (size_t)h->B * h->M * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(MPO_ERR_CUDA);
  }
  pl->ev.assign(pl->layer_off.size() * MPO_NSTAGES + 2, nullptr);
  for (auto& e : pl->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(MPO_ERR_CUDA);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(MPO_ERR_CUDA);
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(MPO_ERR_CUDA);
  int launches = 0;
  st = run_layers(h, pl->d_gates, pl->layer_off, pl->layer_cnt, pl->d_disc, pl->d_phase, &launches,
                  pl->ev.data());
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (st != MPO_OK) { if (graph) cudaGraphDestroy(graph); return fail(st); }
  if (e != cudaSuccess) return fail(MPO_ERR_CUDA);
  pl->graph = graph;
  if (cudaGraphInstantiate(&pl->exec, graph, 0) != cudaSuccess) return fail(MPO_ERR_CUDA);
  pl->launches = launches;
  h->plans.push_back(pl);
  *out = pl;
  return MPO_OK;
}

mpo_status mpo_plan_run(mpo_plan p) {
  NvtxRange nv("gbs_mpo/plan_run");
  if (!p || !p->h) return MPO_ERR_ARG;
  if (p->h->poisoned) return MPO_ERR_POISONED;
  CK(cudaGraphLaunch(p->exec, p->h->stream));
  ++p->runs;
  return MPO_OK;
}

mpo_status mpo_set_tuning(mpo_handle h, const mpo_tuning* t) {
  if (!h || !t) return MPO_ERR_ARG;
  if (t->theta_form < 0 || t->theta_form > 2 || t->gram_tc_min < 0 || t->svd_cluster_seed_max < -1) return MPO_ERR_ARG;
  if (t->svd_cluster_size != 0 && t->svd_cluster_size != 1 && t->svd_cluster_size != 2 &&
      t->svd_cluster_size != 4 && t->svd_cluster_size != 8)
    return MPO_ERR_ARG;
  h->tun = *t;
  apply_tuning(h, h->ws);  // the pools and tables stay; only the launch choices change
  return MPO_OK;
}

mpo_status mpo_get_tuning(mpo_handle h, mpo_tuning* t) {
  if (!h || !t) return MPO_ERR_ARG;
  *t = h->tun;
  return MPO_OK;
}

mpo_status mpo_svd_cluster_shape(int* cluster_size, int* clusters_fp64, int* clusters_fp32, int* min_n) {
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) return MPO_ERR_NOT_BUILT;
  if (gate_module_init() != cudaSuccess) return MPO_ERR_CUDA;
  svd_cluster_info(cluster_size, clusters_fp64, clusters_fp32);
  if (min_n) *min_n = svd_big_min();
  return MPO_OK;
}

mpo_status mpo_plan_stage_times(mpo_plan p, double* stage_ms) {
  if (!p || !p->h || !stage_ms || p->runs == 0) return MPO_ERR_ARG;
  mpo_handle h = p->h;
  if (h->poisoned) return MPO_ERR_POISONED;
  CK(cudaStreamSynchronize(h->stream));
  const size_t L = p->layer_off.size();
  constexpr int NS = MPO_NSTAGES - 1;
  for (int st = 0; st < MPO_NSTAGES; ++st) stage_ms[st] = 0.0;
  for (size_t l = 0; l < L; ++l)
    for (int st = 0; st < NS; ++st) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, p->ev[l * MPO_NSTAGES + st], p->ev[l * MPO_NSTAGES + st + 1]));
      stage_ms[st] += t;
    }
  float tp = 0.f;
  CK(cudaEventElapsedTime(&tp, p->ev[L * MPO_NSTAGES], p->ev[L * MPO_NSTAGES + 1]));
  stage_ms[NS] = tp;
  return poll_error(h);
}

mpo_status mpo_plan_discarded(mpo_plan p, double* discarded) {
  if (!p || !discarded) return MPO_ERR_ARG;
  if (p->ngates > 0)
    CK(cudaMemcpyAsync(discarded, p->d_disc, p->ngates * sizeof(double), cudaMemcpyDeviceToHost, p->h->stream));
  return poll_error(p->h);
}

int mpo_plan_launches(mpo_plan p) { return p ? p->launches : 0; }

mpo_status mpo_plan_profile(mpo_plan p, double* stage_ms, int* stage_launches, double* stage_flops,
                            double* jacobi) {
  if (!p || !p->h) return MPO_ERR_ARG;
  mpo_handle h = p->h;
  if (h->poisoned) return MPO_ERR_POISONED;
  const int L = (int)p->layer_off.size();
  constexpr int NS = MPO_NSTAGES - 1;  // per-layer stages; the last stage is the phase screen
  std::vector<cudaEvent_t> ev((size_t)L * (NS + 1) + 2, nullptr);
  unsigned long long* d_ctr = nullptr;
  auto release = on_scope_exit([&] {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    tmp_free(h, d_ctr);
  });
  for (auto& e : ev) CK(cudaEventCreate(&e));
  CK(tmp_alloc(h, (void**)&d_ctr, CTR_N * sizeof(unsigned long long)));
  CK(cudaMemsetAsync(d_ctr, 0, CTR_N * sizeof(unsigned long long), h->stream));
  MpoDev dv = h->dev;
  dv.ctr = d_ctr;
  for (int l = 0; l < L; ++l)
    launch_layer(dv, h->ws, p->d_gates + p->layer_off[l], p->layer_cnt[l], p->d_disc, h->prec,
                 h->stream, nullptr, ev.data() + (size_t)l * (NS + 1));
  CK(cudaEventRecord(ev[(size_t)L * (NS + 1)], h->stream));
  if (p->d_phase) launch_phases(h->dev, p->d_phase, h->stream);
  CK(cudaEventRecord(ev[(size_t)L * (NS + 1) + 1], h->stream));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  double ms[MPO_NSTAGES] = {0};
  for (int l = 0; l < L; ++l)
    for (int st = 0; st < NS; ++st) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, ev[(size_t)l * (NS + 1) + st], ev[(size_t)l * (NS + 1) + st + 1]));
      ms[st] += t;
    }
  float tp = 0.f;
  CK(cudaEventElapsedTime(&tp, ev[(size_t)L * (NS + 1)], ev[(size_t)L * (NS + 1) + 1]));
  ms[NS] = tp;
  unsigned long long ctr[CTR_N];
  CK(cudaMemcpyAsync(ctr, d_ctr, sizeof(ctr), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  // stage order: setup, theta, gram, order, svd, select, resplit, phases
  const double fl[MPO_NSTAGES] = {0.0, (double)ctr[CTR_THETA], (double)ctr[CTR_GRAM], 0.0,
                                  (double)(ctr[CTR_EIG] + ctr[CTR_REFINE]), 0.0, (double)ctr[CTR_RESPLIT], 0.0};
  for (int st = 0; st < MPO_NSTAGES; ++st) {
    if (stage_ms) stage_ms[st] = ms[st];
    // the Gram stage is two launches per layer (SIMT blocks, tensor-core blocks)
    if (stage_launches) stage_launches[st] = st < NS ? (st == 2 ? 2 * L : L) : (p->d_phase ? 1 : 0);
    if (stage_flops) stage_flops[st] = fl[st];
  }
  if (jacobi) {
    jacobi[0] = (double)ctr[CTR_EIGBLK];
    jacobi[1] = (double)ctr[CTR_SWEEPS];
    jacobi[2] = (double)ctr[CTR_RSWEEPS];
    jacobi[3] = (double)ctr[CTR_EIG];
    jacobi[4] = (double)ctr[CTR_REFINE];
    jacobi[5] = (double)ctr[CTR_NBIG];
    jacobi[6] = (double)ctr[CTR_CYC_BIG];
    jacobi[7] = (double)ctr[CTR_CYC_SMALL];
    jacobi[8] = (double)ctr[CTR_CYC_SEED];
    jacobi[9] = (double)ctr[CTR_CYC_NS];
    jacobi[10] = (double)ctr[CTR_CYC_POLISH];
    jacobi[11] = (double)ctr[CTR_NWARP];
    jacobi[12] = (double)ctr[CTR_CYC_WARP];
    jacobi[13] = (double)ctr[CTR_FTHETA];
  }
  return poll_error(h);
}

void mpo_plan_destroy(mpo_plan p) {
  if (!p) return;
  if (p->h) {
    auto& v = p->h->plans;
    v.erase(std::remove(v.begin(), v.end(), p), v.end());
    if (p->h->stream) cudaStreamSynchronize(p->h->stream);
  }
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  dev_free(p->h, p->d_gates);
  dev_free(p->h, p->d_disc);
  dev_free(p->h, p->d_phase);
  for (auto e : p->ev)
    if (e) cudaEventDestroy(e);
  delete p;
}

mpo_status mpo_observables(mpo_handle h, double* trace, double* n_mean, double* n2_mean, int normalize_by_trace) {
  if (!h) return MPO_ERR_ARG;
  if (h->poisoned) return MPO_ERR_POISONED;
  launch_observables(h->dev, h->d_obs_scratch, h->d_obs_out, h->stream);
  CK(cudaGetLastError());
  const int M = h->M, per = 1 + 2 * M + M + 1;
  std::vector<double> buf((size_t)h->B * per);
  CK(cudaMemcpyAsync(buf.data(), h->d_obs_out, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  mpo_status st = poll_error(h);
  if (st != MPO_OK) return st;
  for (int i = 0; i < h->B; ++i) {
    const double* o = buf.data() + (size_t)i * per;
    const double tr = o[0];
    const double sc = normalize_by_trace ? 1.0 / tr : 1.0;
    if (trace) trace[i] = tr;
    for (int j = 0; j < M; ++j) {
      if (n_mean) n_mean[(size_t)i * M + j] = o[1 + j] * sc;
      if (n2_mean) n2_mean[(size_t)i * M + j] = o[1 + M + j] * sc;
    }
  }
  return MPO_OK;
}

mpo_status mpo_truncated_probability(mpo_handle h, double* tail) {
  if (!h || !tail) return MPO_ERR_ARG;
  for (int i = 0; i < h->B; ++i) tail[i] = 1.0 - h->kept[i];
  return MPO_OK;
}

mpo_status mpo_operator_entropy(mpo_handle h, double* S, double* purity, double* S_max_running) {
  if (!h) return MPO_ERR_ARG;
  if (h->poisoned) return MPO_ERR_POISONED;
  const int M = h->M;
  std::vector<double> ent((size_t)h->B * (M + 1));
  CK(cudaMemcpyAsync(ent.data(), h->dev.entropy, ent.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  std::vector<double> buf;
  if (purity) {
    launch_observables(h->dev, h->d_obs_scratch, h->d_obs_out, h->stream);
    CK(cudaGetLastError());
    const int per = 1 + 2 * M + M + 1;
    buf.resize((size_t)h->B * per);
    CK(cudaMemcpyAsync(buf.data(), h->d_obs_out, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  mpo_status st = poll_error(h);
  if (st != MPO_OK) return st;
  for (int i = 0; i < h->B; ++i) {
    double mx = 0.0;
    for (int b = 0; b <= M; ++b) {
      const double v = ent[(size_t)i * (M + 1) + b];
      if (S) S[(size_t)i * (M + 1) + b] = v;
      mx = std::max(mx, v);
      if (purity) purity[(size_t)i * (M + 1) + b] = buf[(size_t)i * (1 + 3 * M + 1) + 1 + 2 * M + b];
    }
    if (S_max_running) S_max_running[i] = mx;
  }
  return MPO_OK;
}

mpo_status mpo_get_bonds(mpo_handle h, int inst, int ld, int* chi, double* lam, int* charge) {
  if (!h || inst < 0 || inst >= h->B) return MPO_ERR_ARG;
  if (h->poisoned) return MPO_ERR_POISONED;
  const int M = h->M, D = h->D;
  std::vector<int> c(M + 1);
  CK(cudaMemcpyAsync(c.data(), h->dev.chi + (size_t)inst * (M + 1), (M + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  int mx = 0;
  for (int v : c) mx = std::max(mx, v);
  if ((lam || charge) && ld < mx) return MPO_ERR_ARG;
  if (chi) std::memcpy(chi, c.data(), (M + 1) * sizeof(int));
  std::vector<double> l((size_t)(M + 1) * D);
  std::vector<int> ch((size_t)(M + 1) * D);
  CK(cudaMemcpyAsync(l.data(), h->dev.lam + (size_t)inst * (M + 1) * D, l.size() * sizeof(double),
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(ch.data(), h->dev.charge + (size_t)inst * (M + 1) * D, ch.size() * sizeof(int),
                     cudaMemcpyDeviceToHost, h->stream));
  mpo_status st = poll_error(h);
  if (st != MPO_OK) return st;
  for (int b = 0; b <= M; ++b)
    for (int i = 0; i < c[b]; ++i) {
      if (lam) lam[(size_t)b * ld + i] = l[(size_t)b * D + i];
      if (charge) {
        const int p = ch[(size_t)b * D + i];
        charge[((size_t)b * ld + i) * 2] = pair_c(p, h->ncap);
        charge[((size_t)b * ld + i) * 2 + 1] = pair_cb(p, h->ncap);
      }
    }
  return MPO_OK;
}

int mpo_bond_capacity(mpo_handle h) { return h ? h->D : 0; }

// ---------------------------------------------------------------- checkpoints
// Layout: CkptHeader (128 bytes) | device state image (state_bytes) | kept [B] doubles.
// The state image is the handle's own device layout, so a checkpoint is only valid for
// a handle of the same shape (M, d, n_cap, batch, D, precision) built by this library.
namespace {
constexpr char kCkptMagic[8] = {'G', 'B', 'S', 'M', 'P', 'O', 'C', 'K'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int32_t M, d, ncap, B, P, D, prec, reserved0;
  uint64_t state_bytes, cursor, checksum;
  uint8_t reserved[128 - 8 - 8 - 32 - 24];
};
static_assert(sizeof(CkptHeader) == 128, "checkpoint header is 128 bytes");

// FNV-1a, 64 bit (Fowler, Noll, Vo): detects torn or corrupted buffers, not tampering
uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t hsh = 1469598103934665603ull) {
  for (size_t i = 0; i < n; ++i) {
    hsh ^= p[i];
    hsh *= 1099511628211ull;
  }
  return hsh;
}

size_t ckpt_bytes(const mpo_ctx* h) { return sizeof(CkptHeader) + h->state_bytes + (size_t)h->B * sizeof(double); }
}  // namespace

mpo_status mpo_checkpoint_bytes(mpo_handle h, size_t* bytes) {
  if (!h || !bytes) return MPO_ERR_ARG;
  *bytes = ckpt_bytes(h);
  return MPO_OK;
}

mpo_status mpo_save(mpo_handle h, void* buf, size_t bytes, long long cursor) {
  if (!h || !buf) return MPO_ERR_ARG;
  if (h->poisoned) return MPO_ERR_POISONED;
  if (bytes < ckpt_bytes(h)) return MPO_ERR_ARG;
  unsigned char* out = (unsigned char*)buf;
  unsigned char* img = out + sizeof(CkptHeader);
  CK(cudaMemcpyAsync(img, h->state, h->state_bytes, cudaMemcpyDeviceToHost, h->stream));
  mpo_status st = poll_error(h);
  if (st != MPO_OK) return st;
  std::memcpy(img + h->state_bytes, h->kept.data(), (size_t)h->B * sizeof(double));
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = kCkptVersion;
  hd.header_bytes = sizeof(CkptHeader);
  hd.M = h->M; hd.d = h->d; hd.ncap = h->ncap; hd.B = h->B; hd.P = h->P; hd.D = h->D; hd.prec = h->prec;
  hd.state_bytes = h->state_bytes;
  hd.cursor = (uint64_t)cursor;
  hd.checksum = fnv1a(img, h->state_bytes + (size_t)h->B * sizeof(double));
  std::memcpy(out, &hd, sizeof(hd));
  return MPO_OK;
}

mpo_status mpo_load(mpo_handle h, const void* buf, size_t bytes, long long* cursor) {
  if (!h || !buf) return MPO_ERR_ARG;
  if (h->poisoned) return MPO_ERR_POISONED;
  if (bytes < sizeof(CkptHeader)) return MPO_ERR_ARG;
  CkptHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != kCkptVersion || hd.header_bytes != sizeof(CkptHeader))
    return MPO_ERR_ARG;
  if (hd.M != h->M || hd.d != h->d || hd.ncap != h->ncap || hd.B != h->B || hd.P != h->P || hd.D != h->D ||
      hd.prec != h->prec || hd.state_bytes != h->state_bytes || bytes < ckpt_bytes(h))
    return MPO_ERR_ARG;
  const unsigned char* img = (const unsigned char*)buf + sizeof(CkptHeader);
  if (fnv1a(img, h->state_bytes + (size_t)h->B * sizeof(double)) != hd.checksum) return MPO_ERR_ARG;
  CK(cudaMemcpyAsync(h->state, img, h->state_bytes, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::memcpy(h->kept.data(), img + h->state_bytes, (size_t)h->B * sizeof(double));
  if (cursor) *cursor = (long long)hd.cursor;
  return MPO_OK;
}

mpo_status mpo_sync(mpo_handle h) {
  if (!h) return MPO_ERR_ARG;
  if (h->poisoned) return MPO_ERR_POISONED;
  return poll_error(h);
}

mpo_status mpo_set_allocator(mpo_alloc_fn alloc, mpo_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return MPO_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_allocator_mu);
  g_allocator.alloc = alloc;
  g_allocator.free = free_fn;
  g_allocator.ctx = alloc ? ctx : nullptr;
  return MPO_OK;
}

void mpo_destroy(mpo_handle h) {
  if (!h) return;
  while (!h->plans.empty()) mpo_plan_destroy(h->plans.back());
  if (h->stream) cudaStreamSynchronize(h->stream);
  dev_free(h, h->state);
  dev_free(h, h->snap);
  dev_free(h, h->d_err);
  dev_free(h, h->d_chicap);
  dev_free(h, h->ws_buf);
  dev_free(h, h->d_gate1);
  dev_free(h, h->d_disc1);
  dev_free(h, h->d_obs_scratch);
  dev_free(h, h->d_obs_out);
  if (h->pin) cudaFreeHost(h->pin);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
