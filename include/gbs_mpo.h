/*
 * gbs_mpo.h -- C ABI of the GB300 (sm_103a) U(1)-symmetric MPO beam-splitter mesh.
 *
 * The library simulates lossy Gaussian boson sampling as in Liu et al.,
 * "Simulating lossy Gaussian boson sampling with matrix product operators"
 * (arXiv:2301.12814): the lossy squeezed input state is held as a vectorised
 * density operator in U(1)-symmetric Vidal MPO form (App. D), and every
 * nearest-neighbour beam splitter of a mesh is applied by the two-site update
 * of App. D (Eq. `theta` contraction per new centre charge, SVD of every charge
 * block, global keep-chi truncation, re-split Gamma = V / lambda).
 *
 * Conventions shared by every call
 *   modes     j = 0..M-1; bond b = 0..M sits left of mode b (bond 0 = left edge).
 *   charge    every bond index carries the pair (c, cbar) = (ket, bra) photons to
 *             the RIGHT of the bond (App. D), 0 <= c, cbar <= n_cap.
 *   gate k    acts on modes (k, k+1) with the 2x2 mode matrix
 *             [[e^{i phi} cos theta, -sin theta], [e^{i phi} sin theta, cos theta]],
 *             i.e. a_k^dag -> S00 a_k^dag + S10 a_{k+1}^dag (Clements' T block).
 *   memory    every pointer argument is a HOST pointer unless stated otherwise.
 *             Inputs are copied before the call returns; outputs are written by
 *             the time the call returns.  The handle owns all device memory.
 *   streams   all device work of a handle is issued on params.cuda_stream.
 *             Calls that return host results synchronise that stream; the
 *             plan/reset calls are asynchronous.
 *   threads   one host thread at a time per handle.
 *   errors    return codes only.  After MPO_ERR_NUMERIC, MPO_ERR_CAPACITY,
 *             MPO_ERR_INTERNAL or MPO_ERR_CUDA the handle is poisoned: every call
 *             but mpo_destroy returns MPO_ERR_POISONED.
 */
#ifndef GBS_MPO_H
#define GBS_MPO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpo_ctx* mpo_handle;
typedef struct mpo_plan_s* mpo_plan;

typedef enum {
  MPO_OK = 0,
  MPO_ERR_ARG = 1,       /* invalid argument: sizes, ranges, null pointers        */
  MPO_ERR_OOM = 2,       /* device allocation failed                             */
  MPO_ERR_CUDA = 3,      /* a CUDA runtime call failed                           */
  MPO_ERR_NUMERIC = 4,   /* eigensolver sweep cap reached or a non-finite value  */
  MPO_ERR_TIMEOUT = 5,   /* a bounded device wait ran out (a tensor-core kernel's
                            wait for its own MMAs, or the peak probe's)             */
  MPO_ERR_CAPACITY = 6,  /* a workspace bound was exceeded on device: the layer's
                            pools of Theta- and Gram-sized arrays (sized at most to
                            GBS_MPO_WORKSPACE_GB, else a quarter of the free device
                            memory) or a per-gate table                            */
  MPO_ERR_INTERNAL = 7,  /* a device-side consistency check failed               */
  MPO_ERR_POISONED = 8,  /* handle unusable after an earlier device-side error   */
  MPO_ERR_NOT_BUILT = 9  /* the CUDA library could not be loaded or has no GPU   */
} mpo_status;

typedef enum {
  MPO_FP64 = 0,        /* FP64-accurate: Theta contraction in FP64 (its large items in
                          double-float arithmetic on the FP32 pipe), the Jacobi
                          refinement (Newton-Schulz, W = Theta V, one-sided sweeps) in
                          double-float (about 48 significand bits), re-split, lambda and
                          observables in float64 / complex128; the Gram matrix (3xTF32
                          tensor cores from a Gram side of 48, FP32 below) and the Jacobi
                          seed that only starts the refinement are FP32                   */
  MPO_MIXED_TF32 = 1,  /* mixed: Theta contraction (FP32 SIMT two-stage; 3xTF32 tensor
                          cores by launch choice), Gram, Jacobi seed and one-sided
                          refinement in FP32 (FP32 accumulation); keep-chi selection,
                          discarded weight, lambda, entropy, observables and the stored
                          Gamma in FP64                                                   */
  MPO_MIXED_BF16 = 2   /* as MPO_MIXED_TF32, with the Theta contraction on the tensor
                          cores in BF16 (one BF16 pass per operand, FP32 accumulation)   */
} mpo_precision;

typedef struct {
  int M;              /* modes, 2 <= M <= 256                                        */
  int d;              /* local Fock cutoff: photon numbers 0..d-1 per mode, 2..32    */
  int n_cap;          /* cap on total ket (and bra) photons; <= 0 means d - 1;
                         must satisfy n_cap <= d - 1 and n_cap <= 15                 */
  int batch;          /* independent instances held by the handle, >= 1             */
  mpo_precision prec; /* arithmetic of the gate pipeline                             */
  const int* chi_max; /* [batch] host: bond-dimension cap per instance; a value <= 0
                         means "no cap" (exact, only values below the numerical
                         floor are dropped); NULL means no cap for every instance   */
  void* cuda_stream;  /* cudaStream_t for all work of the handle; NULL = default    */
} mpo_params;

/* Device memory of handles and plans.  By default a handle's long-lived buffers come
 * from cudaMalloc and per-call temporaries are stream-ordered (cudaMallocAsync on the
 * handle's stream).  mpo_set_allocator installs a caller's pair instead -- for
 * example one backed by a framework's caching allocator -- for every handle created
 * afterwards; each handle keeps the pair it was created with and frees its memory
 * through it.  alloc returns device memory of at least `bytes` bytes usable in
 * stream order on `stream` (the handle's cudaStream_t), or NULL (the call then
 * fails with MPO_ERR_OOM); free releases a pointer alloc returned, after the work the
 * library queued on `stream`.  ctx is passed back unchanged.  NULL, NULL restores the
 * CUDA runtime.  MPO_ERR_ARG if exactly one of the two is NULL.  The App. C entry
 * points allocate through the CUDA runtime. */
typedef void* (*mpo_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*mpo_free_fn)(void* ptr, void* stream, void* ctx);
mpo_status mpo_set_allocator(mpo_alloc_fn alloc, mpo_free_fn free, void* ctx);

/* Create a handle and build the initial state of every instance (App. B/C: each
 * mode starts as single-mode squeezed vacuum c_{2j} ~ (-tanh r)^j, truncated at d,
 * sent through a pure-loss channel of transmission eta; uniform loss commutes with
 * the mesh and is applied to the input, Method section).  The state is
 * rho_0 = P_cap (x)_j rho_j P_cap / Tr, written in exactly canonical U(1) Vidal form
 * with the bond-0 index ranging over the total-charge pairs.
 *   r   [batch*M] squeezing per instance and mode (r = 0: vacuum), 0 <= r <= 3
 *   eta [batch*M] transmission per instance and mode, 0 <= eta <= 1
 * On success *out owns the device state and a snapshot used by mpo_reset.
 * Synchronises the stream. */
mpo_status mpo_init_lossy_squeezed(mpo_handle* out, const mpo_params* p,
                                   const double* r, const double* eta);

/* Restore every instance to the state built by mpo_init_lossy_squeezed
 * (device-to-device copy on the stream; asynchronous). */
mpo_status mpo_reset(mpo_handle h);

/* Apply one beam splitter (k, theta, phi) to instance inst: the two-site U(1)
 * update of App. D (Eq. `theta`, block SVD, keep chi, Gamma = V / lambda).
 *   discarded_weight  nullable host pointer: sum of dropped s^2 / sum of all s^2.
 * Synchronises the stream when discarded_weight is non-NULL. */
mpo_status mpo_apply_bs(mpo_handle h, int inst, int k, double theta, double phi,
                        double* discarded_weight);

/* Apply a whole mesh to every instance.  Instance i's gates are the n_gates[i]
 * consecutive entries of k/theta/phi after those of instances 0..i-1, in
 * application order (U = D T_L ... T_1).  Gates on disjoint mode pairs are
 * grouped into layers and every layer of every instance runs in one batched pass.
 *   final_phase  [batch*M] or NULL: phase screen D applied after the last gate.
 *   discarded    [sum n_gates] or NULL: per-gate discarded weight, same order.
 * Copies the gate list to the device through a pinned staging buffer owned by the
 * handle, runs, copies the results back the same way; synchronises. */
mpo_status mpo_sweep_mesh(mpo_handle h, const int* n_gates, const int* k,
                          const double* theta, const double* phi,
                          const double* final_phase, double* discarded);

/* Plans: the same mesh as mpo_sweep_mesh, uploaded once and captured in a CUDA
 * graph; mpo_plan_run replays it asynchronously on the handle's stream with the
 * gate list already resident in device memory.  A plan belongs to its handle:
 * mpo_destroy(h) destroys every plan of h that is still alive, after which those
 * plan pointers must not be used. */
mpo_status mpo_plan_mesh(mpo_handle h, const int* n_gates, const int* k,
                         const double* theta, const double* phi,
                         const double* final_phase, mpo_plan* out);
mpo_status mpo_plan_run(mpo_plan p);
/* Per-gate discarded weights of the last run ([sum n_gates], host); synchronises. */
mpo_status mpo_plan_discarded(mpo_plan p, double* discarded);
/* Number of kernel launches one mpo_plan_run performs. */
int mpo_plan_launches(mpo_plan p);
/* Stages of one gate layer, in launch order (plus the final phase screen). */
#define MPO_NSTAGES 8
/* Replay the plan once without the graph, with a CUDA event between consecutive
 * stage launches on the handle's stream, and report per stage (setup, theta, gram,
 * order, svd, select, resplit, phases) the summed device time in ms, the launch
 * count and the real flops of the executed form (theta, FP64 path: the two-stage SIMT
 * form, 8 n_a n_b (sum_c n_c + n_c n_m) per row/column segment pair; TF32 and BF16
 * paths: the one-stage Eq. `theta` on the tensor cores, F_Theta below; gram: upper
 * triangle x 8 x inner size; svd: FP32
 * seed Jacobi, per applied rotation 54 n (complex) or 18 n (real), plus the
 * refinement, W = Theta V and 48 h + 24 n per applied one-sided rotation, in the
 * path's precision; resplit: element copies).  Each array
 * is [MPO_NSTAGES] host memory and nullable.  jacobi (nullable, [14]): blocks
 * factorised, seed sweeps (two-sided, or the FP32 phase of a cluster block),
 * refinement sweeps, seed flops (FP32), refinement flops (path precision), blocks
 * factorised on a CTA cluster, SM clock cycles spent on cluster blocks (first CTA
 * of the cluster) and on single-CTA blocks, the cluster blocks' cycles in their
 * seed (or FP32 phase), Newton-Schulz and final sweeps, and the blocks factorised
 * by one warp and their cycles, summed over the replay; then F_Theta, the real flops
 * of Eq. `theta` in one stage over the canonical blocks, sum over m, a >= m >= b and
 * a >= c >= b of 8 n_a n_c n_b (whatever form ran).
 * Same results as mpo_plan_run.  Synchronises. */
mpo_status mpo_plan_profile(mpo_plan p, double* stage_ms, int* stage_launches,
                            double* stage_flops, double* jacobi);
/* Device time of each stage (same order as mpo_plan_profile) summed over the layers
 * of the most recent mpo_plan_run of p, in ms.  The plan's graph holds a CUDA event
 * record node before and after every stage launch on the handle's stream, so these
 * are the times of the replay itself, not of a separate instrumented run.
 * stage_ms: [MPO_NSTAGES] host memory.  MPO_ERR_ARG if p has never been run.
 * Synchronises. */
mpo_status mpo_plan_stage_times(mpo_plan p, double* stage_ms);

/* Launch shape of the block SVD (no counterpart in the paper; for benchmarks and
 * diagnostics).  Blocks whose Gram side is at least *min_n are factorised on a
 * thread-block cluster of *cluster_size CTAs; *clusters_fp64 / *clusters_fp32 such
 * clusters fit on the current device at once (0 = launched without clusters).  All
 * pointers are host memory and nullable.  Initialises the CUDA library if needed;
 * MPO_ERR_NOT_BUILT without a GPU. */
mpo_status mpo_svd_cluster_shape(int* cluster_size, int* clusters_fp64, int* clusters_fp32, int* min_n);
void mpo_plan_destroy(mpo_plan p);

/* Observables of every instance (once per mesh; trace environments):
 *   trace   [batch]    Tr rho (its deficit 1 - Tr rho is the truncation error proxy)
 *   n_mean  [batch*M]  <n_j>
 *   n2_mean [batch*M]  <n_j^2>
 * normalize_by_trace != 0 divides the moments by Tr rho.  Synchronises. */
mpo_status mpo_observables(mpo_handle h, double* trace, double* n_mean, double* n2_mean,
                           int normalize_by_trace);

/* Probability removed by the truncation of the initial state (App. A: d is the
 * smallest local dimension for which less than 1% of the probability is cut).
 *   tail [batch]  1 - Tr(P_cap (x)_j rho_j P_cap), where rho_j is mode j's lossy
 *                 squeezed vacuum from amplitudes normalised in the infinite Fock
 *                 space and truncated at d levels before loss (App. C, App. B), and
 *                 P_cap keeps total photon numbers <= n_cap (App. A: the left-most
 *                 charge is the total photon number).
 * Fixed when the handle is made (the mesh is unitary on the kept space); host
 * memory; MPO_ERR_ARG for a NULL argument.  Does not synchronise. */
mpo_status mpo_truncated_probability(mpo_handle h, double* tail);

/* Operator entanglement of the U(1) MPO at every bond (Method, Eq. `schmidt`;
 * App. B: p = lambda^2 / sum lambda^2, S = -sum p log2 p):
 *   S             [batch*(M+1)]  bonds 0..M
 *   purity        [batch*(M+1)]  sum lambda^2 per bond, nullable
 *   S_max_running [batch]        max over bonds of S, nullable
 * Synchronises. */
mpo_status mpo_operator_entropy(mpo_handle h, double* S, double* purity,
                                double* S_max_running);

/* Bond data of one instance (tests and inspection): chi [M+1] dimensions;
 * lam [(M+1)*ld] and charge [(M+1)*ld*2] (c, cbar per index), row b holding bond
 * b's chi[b] entries; either may be NULL.  ld >= largest chi.  Synchronises. */
mpo_status mpo_get_bonds(mpo_handle h, int inst, int ld, int* chi, double* lam, int* charge);

/* Checkpoints (no counterpart in the paper: restart support for long meshes).
 * A checkpoint is a host byte buffer: a 128-byte header (magic "GBSMPOCK", format
 * version, M, d, n_cap, batch, charge-pair count, bond capacity D, precision, the
 * caller's gate cursor, an FNV-1a checksum of the payload), then the handle's device
 * state image (bond dimensions, charges, segment offsets, lambda, entropies, Gamma)
 * and the per-instance kept probability.  The image is the library's own layout: a
 * checkpoint loads only into a handle of the same M, d, n_cap, batch, D and precision
 * (chi caps may differ) from the same library version.
 *   mpo_checkpoint_bytes  *bytes = the buffer size a checkpoint of h needs.
 *   mpo_save   copies the current state into buf (host, >= that size) with the
 *              caller's gate cursor (for example the number of gates applied);
 *              synchronises; device errors first poison the handle as usual.
 *   mpo_load   replaces the state of h by the checkpoint; *cursor (nullable)
 *              receives the saved cursor.  MPO_ERR_ARG for a short buffer, a wrong
 *              magic or version, a shape mismatch or a checksum mismatch (the state
 *              is then unchanged).  mpo_reset still returns to the initial state.
 *              Synchronises. */
mpo_status mpo_checkpoint_bytes(mpo_handle h, size_t* bytes);
mpo_status mpo_save(mpo_handle h, void* buf, size_t bytes, long long cursor);
mpo_status mpo_load(mpo_handle h, const void* buf, size_t bytes, long long* cursor);

/* Device pointers/sizes for callers that manage their own buffers: the bond
 * capacity D (Gamma matrices are D x D) and the number of instances. */
int mpo_bond_capacity(mpo_handle h);

/* Synchronise the handle's stream and report any device-side error. */
mpo_status mpo_sync(mpo_handle h);

void mpo_destroy(mpo_handle h);
const char* mpo_status_string(mpo_status s);

/* Asymptotic operator entanglement of one squeezed input mode (App. C): the estimate
 * the paper uses for system sizes beyond direct MPO simulation (Results, Fig. 1).
 * For each point i: the squeezed vacuum of r[i] truncated at n_max photons (App. C),
 * pure loss of transmission mu[i] with the state and Kraus operators truncated at
 * n_max (Eq. `lossy`), the split <k_u, k_d|U|n> = sqrt(C(n, k_u)) cos^k_u sin^k_d of
 * theta[i] (Eq. `transform` / `kun`; pi/4 in the asymptotic limit), vectorisation
 * X[(k_u, k_u'), (k_d, k_d')] = rho_out[k_u, k_d; k_u', k_d'], and the eigenvalues of
 * tr_u |rho_out>><<rho_out| (the squared singular values of X) normalised to sum 1.
 * The system estimate is N times S1 at mu = beta N^gamma / N; the caller forms it.
 *   npts      number of points (0 is a no-op)
 *   n_max     photon cutoff, 1 <= n_max <= MPO_ASYM_NMAX
 *   r, mu, theta [npts]  squeezing (0..3), transmission (0..1), split angle (finite)
 *   alpha     Renyi order (> 0) for S_alpha; ignored when S_alpha is NULL
 *   S1        [npts]     von Neumann entropy of the normalised spectrum, bits
 *   S_alpha   [npts]     log2(sum p^alpha) / (1 - alpha) (S1 at alpha = 1), nullable
 *   spectrum  [npts*ld]  normalised eigenvalues, descending, (n_max+1)^2 per point;
 *                        nullable; ld >= (n_max+1)^2
 * Host pointers; allocates and frees its own device memory; synchronises.  Errors:
 * MPO_ERR_ARG (sizes, ranges, NULL), MPO_ERR_NUMERIC (a Jacobi sweep cap reached),
 * MPO_ERR_NOT_BUILT (no GPU), MPO_ERR_OOM / MPO_ERR_CUDA. */
#define MPO_ASYM_NMAX 23
mpo_status mpo_asymptotic_ee(int npts, int n_max, const double* r, const double* mu,
                             const double* theta, double alpha, double* S1, double* S_alpha,
                             double* spectrum, int ld);

/* The same on DEVICE pointers with no allocation and no synchronisation: the two
 * kernels are issued on cuda_stream (NULL = legacy default) and the outputs are ready
 * when the stream reaches that point.  spectrum [npts*ld] is required (it is also the
 * workspace); sweeps [4*npts] (nullable) receives the Jacobi sweeps of each point's
 * four blocks (symmetric/even, symmetric/odd, antisymmetric/even, antisymmetric/odd
 * under the swap (k_u, k_d) <-> (k_u', k_d') and by photon-number parity); a value
 * above 40 means the sweep cap was reached.  Inputs are not range-checked on the
 * device: values outside the ranges above give meaningless numbers, never a fault.
 * MPO_ERR_ARG for sizes and NULLs, MPO_ERR_CUDA if a launch fails. */
mpo_status mpo_asymptotic_ee_device(int npts, int n_max, const double* r, const double* mu,
                                    const double* theta, double alpha, double* S1, double* S_alpha,
                                    double* spectrum, int ld, int* sweeps, void* cuda_stream);

/* Observables of one MPO held in buffers the caller owns, with no allocation.
 * The paper has no counterpart: this is a library-interface addition for callers
 * that cannot allocate device memory when they need the observables -- code inside
 * a host application or framework that owns all device memory (its own pool
 * allocator or a fixed budget) and forbids direct cudaMalloc/cudaFree, which also
 * synchronise the device.  It runs the same trace-environment kernel as
 * mpo_observables; its scratch (2 (M+1) D complex doubles) is a file-scope device
 * array of 65536 complex doubles (1 MiB) that every GPU loading the library holds
 * until the process exits.  Larger M or D return MPO_ERR_CAPACITY.
 *   M, n_cap, D  modes, charge cap (<= 15), bond capacity (row stride of Gamma)
 *   chi     [M+1]            device: bond dimensions
 *   charge  [(M+1)*D]        device: pair index c*(n_cap+1)+cbar of each bond index,
 *                            ascending within a bond
 *   segoff  [(M+1)*P1]       device: per bond P1 = (n_cap+1)^2 + 1 segment offsets
 *                            (indices of pair p occupy [segoff[p], segoff[p+1]))
 *   lam     [(M+1)*D]        device: Vidal weights
 *   gam     [M*D*D]          device: complex128 (re, im) Gamma_j, row-major D x D,
 *                            rows = bond j, columns = bond j+1 (the handle's layout)
 *   out     [3M+2]           device: Tr rho, <n_j> Tr rho (M), <n_j^2> Tr rho (M),
 *                            sum lambda^2 per bond (M+1) -- moments not divided by Tr
 *   cuda_stream              stream to run on (NULL = legacy default)
 * Asynchronous: out is ready when the stream reaches this point.  The first call on
 * a device looks up the scratch array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The address
 * is cached with the ID of the device's current CUDA context and looked up again when
 * that ID changes (for example after cudaDeviceReset); the first call after such a
 * change must likewise come before any capture.  Every call shares the one scratch
 * array, which keeps the last call's contents (nothing in it needs to start at zero):
 * calls that overlap on the GPU race with each other.  The device tables are not
 * validated on the host: the kernel clamps every size and index it reads from them
 * (chi to [0, D], pair indices to [0, (n_cap+1)^2), segment offsets to [0, chi]), so
 * out-of-range values give meaningless numbers, never an out-of-bounds access. */
mpo_status mpo_observables_static(int M, int n_cap, int D, const int* chi, const int* charge,
                                  const int* segoff, const double* lam, const void* gam,
                                  double* out, void* cuda_stream);

/* Launch choices of one handle (no counterpart in the paper: tuning knobs of this
 * implementation, for the autotuner in paper_2301_12814_gb300/autotune.py).  They
 * change how the work is split over the GPU, never what is computed: every choice
 * gives the same method; the FP64 path stays within its parity bar and the mixed paths
 * within their stated bounds (rounding differs between routes).
 *   theta_form         0 = the path's default (FP64 and TF32: SIMT two-stage; BF16:
 *                      the tensor-core one-stage contraction in BF16), 1 = SIMT
 *                      two-stage, 2 = tensor-core one-stage (3xTF32 on the TF32 path,
 *                      BF16 on the BF16 path; ignored on the FP64 path)
 *   gram_tc_min        Gram side from which Gram matrices run on the tensor cores
 *                      (0 = 48); smaller blocks use the SIMT kernel
 *   svd_cluster_size   CTAs per thread-block cluster of the SVD kernel: 0 = the process
 *                      default (4, or GBS_MPO_SVD_CLUSTER_SIZE), 1 = no clusters, 2, 4, 8
 *   svd_cluster_min_n  > 0: every block with a Gram side >= this goes to a cluster;
 *                      0 = the load rule (a block goes to a cluster when it would hold
 *                      one SM longer than the layer's average SM, or when its Gram side
 *                      is at least 48 on the FP64 path, 64 on the others); < 0 = no
 *                      block does
 *   svd_cluster_seed_max  cluster blocks with a Gram side <= this take the single-CTA
 *                      Gram seed; -1 = the path's default (FP64 0, FP32 64)
 * mpo_set_tuning applies to layers issued afterwards: mpo_apply_bs, mpo_sweep_mesh,
 * mpo_plan_mesh (a plan keeps the choices it was captured with).  MPO_ERR_ARG for
 * values outside these ranges.  mpo_get_tuning returns the handle's current values. */
typedef struct {
  int theta_form;
  int gram_tc_min;
  int svd_cluster_size;
  int svd_cluster_min_n;
  int svd_cluster_seed_max;
} mpo_tuning;
mpo_status mpo_set_tuning(mpo_handle h, const mpo_tuning* t);
mpo_status mpo_get_tuning(mpo_handle h, mpo_tuning* t);

/* Measured arithmetic peaks of the current GPU, for roofline denominators (a
 * measurement utility; the paper has no counterpart).  tflops[4] (host) receives, in
 * TFLOP/s: FP64 FMA, FP32 FMA (8 independent FMA chains per thread, 8 CTAs of 256
 * threads per SM), TF32 and BF16 tensor-core MMA (tcgen05.mma M = 128, N = 256 on
 * operands resident in shared memory, FP32 accumulation in TMEM, one CTA per SM);
 * ms[4] (host, nullable) the timed launch durations.  One warm-up and one timed
 * launch each, with CUDA events, on the legacy default stream (synchronous; about
 * 0.1 s in all).  Allocates and frees a few KB of device memory.  MPO_ERR_NOT_BUILT
 * without a GPU, MPO_ERR_TIMEOUT if a tensor-core wait ran out, MPO_ERR_CUDA /
 * MPO_ERR_OOM otherwise. */
mpo_status mpo_measure_peaks(double* tflops, double* ms);

#ifdef __cplusplus
}
#endif
#endif /* GBS_MPO_H */
