/*
 * libhfx -- Gamma-point Hartree-Fock exact exchange (E_x and V_x phi) on one GB300 GPU.
 *
 * What one call computes (paper Sec. 2.1, Eqs. "vx", "vij" and "HFX"), for real occupied
 * orbitals phi_i sampled on an n1 x n2 x n3 grid of a periodic cell (volume Omega, N points):
 *
 *   rho_ij(r)   = phi_i(r) phi_j(r)                                   (pair density)
 *   F_ij(G)     = sum_r rho_ij(r) exp(-i G.r)                          (forward 3D FFT)
 *   v(G)        = 4 pi / |G|^2, v(0) = 0                               (Coulomb kernel)
 *   v_ij(r)     = (1/N) sum_G v(G) F_ij(G) exp(i G.r)                  (Eq. vij, Poisson solve)
 *   E_x         = -(alpha/2) (Omega/N^2) sum_{(i,j) ordered} sum_G v(G) |F_ij(G)|^2   (Eq. HFX)
 *   (V_x phi)_i = -alpha sum_j v_ij(r) phi_j(r)                          (Eq. vx)
 *
 * over a list of unordered pairs i <= j: an off-diagonal entry stands for (i,j) and (j,i)
 * (energy weight 2, and it adds to both V_i and V_j because v_ij = v_ji), a diagonal entry
 * for itself (weight 1).  The cost is N_orb^2 N log N per call (Sec. 1), which is why
 * the paper's multiple-time-step scheme evaluates it only on its slow (outer) steps.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grid data is row-major [n_orb][n1][n2][n3], the last index (n3) contiguous; point
 *   (p1,p2,p3) sits at r = a1 p1/n1 + a2 p2/n2 + a3 p3/n3 for lattice rows a_k.
 * - Device pointers must be 16-byte aligned.  The library never frees caller memory.
 * - Every call that takes a cuda_stream (a cudaStream_t passed as void*, NULL = legacy
 *   default stream) only enqueues work on it: no host synchronisation, no allocation
 *   (except the first hfx_apply for a new n_orb, which uploads a small schedule table
 *   and must therefore come before any stream capture).
 * - Errors are returned before anything is enqueued when they can be seen on the host;
 *   the library never aborts.  hfx_last_error() gives the calling thread's last message.
 */
#ifndef HFX_H_
#define HFX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hfx_ctx hfx_ctx;

typedef enum {
  HFX_OK = 0,
  HFX_ERR_INVALID_ARG = -1,      /* null pointer, bad size, misaligned pointer, bad flag   */
  HFX_ERR_UNSUPPORTED_GRID = -2, /* an edge is not {2,3,5}-smooth, or a plane exceeds the
                                    on-chip capacity of the chosen precision              */
  HFX_ERR_OOM = -3,              /* a table allocation failed, or the workspace is short  */
  HFX_ERR_CUDA = -4,             /* a CUDA runtime call or a kernel launch failed         */
  HFX_ERR_BAD_PAIR_LIST = -5,    /* (device-detected) an entry outside 0 <= i <= j < n_orb
                                    or more copies of a pair than fit; those entries were
                                    skipped                                               */
  HFX_ERR_TIMEOUT = -6,          /* (device-detected) a bounded device-side wait gave up  */
  HFX_ERR_NOT_POSITIVE_DEFINITE = -7, /* (device-detected) ACE construction: -M had a pivot
                                    <= 0 in its Cholesky factorisation (include/hfx_ace.h) */
  HFX_ERR_RANK_DEFICIENT = -8,   /* (device-detected) SCDM: no grid point with a positive
                                    residual norm was left to pick (include/hfx_ace.h)     */
  HFX_ERR_CORRUPTION = -9        /* (device-detected, HFX_DEBUG builds) a guard band of the
                                    workspace was overwritten, or a placed couple broke the
                                    canonical layout of its block pair                     */
} hfx_status;

/* Frequencies m_d in (-n_d/2, n_d/2], G = m1 b1 + m2 b2 + m3 b3.  On a Nyquist plane (m_d = n_d/2,
 * even n_d) of a non-orthogonal cell the grid point and its mirror (-m mod n) have different |G|;
 * the kernel used there is the mean of the two (its inversion-symmetric part), which keeps every
 * pair potential real and equals the energy of v itself for real pair densities. */
typedef enum {
  HFX_KERNEL_COULOMB = 0,        /* v = 4 pi/|G|^2 on the whole grid, v(0) = 0 (default)   */
  HFX_KERNEL_COULOMB_SPHERE = 1  /* also v = 0 where |G|^2/2 >= 4 ecut (pair-density sphere) */
} hfx_kernel;

typedef enum {
  HFX_PREC_FP64 = 0,     /* all arithmetic in FP64                                       */
  HFX_PREC_FP32 = 1,     /* pair products and FFTs in FP32; energy sums in FP64; V_x phi
                            summed per call in an FP32 workspace accumulator (a few dozen
                            additions per element) and widened exactly into the FP64 output */
  HFX_PREC_MIXED_TC = 2  /* as HFX_PREC_FP32, but the forward DFTs of the plane pass (along
                            z and y) run on the tensor cores: each axis one complex DFT as a
                            dense GEMM with split TF32 operands (hi + lo, three products)
                            and FP32 accumulation; cubic grids of edge 32, 48, 64 or 96
                            (HFX_ERR_UNSUPPORTED_GRID otherwise)                          */
} hfx_precision;

/* flags for hfx_apply */
#define HFX_ENERGY_ONLY   0x1u  /* compute E_x only; vxphi is not touched (may be NULL)    */
#define HFX_ACCUMULATE    0x2u  /* add to *ex_dev and vxphi instead of overwriting them      */
#define HFX_ORBITALS_F32  0x4u  /* orbitals are FP32 (HFX_PREC_FP32 only); default FP64     */

typedef struct {
  double lattice[3][3]; /* rows are the cell vectors a1, a2, a3 in bohr; cubic = diag(L,L,L) */
} hfx_box;

/* hfx_create -- build a context for one cell and grid (Sec. 2.1; the grid holds the
 * Gamma-point orbitals whose pair potentials are solved by FFT, Sec. 2.2).
 *   box    : cell vectors (bohr); must have a non-zero volume.
 *   grid   : n1, n2, n3; each {2,3,5}-smooth, 2 <= n <= 256; a plane of n2*n3 (and n1*n3)
 *            complex values must fit in shared memory (FP32: n2*n3 <= 24576; FP64: <= 12288).
 *   ecut   : wavefunction cutoff in Ha, used only by HFX_KERNEL_COULOMB_SPHERE (> 0 then).
 *   kernel : hfx_kernel.
 *   alpha  : fraction of exact exchange (0.25 for PBE0).
 *   prec   : hfx_precision.
 *   out    : receives the new context (owned by the caller; free with hfx_destroy).
 * Allocates the context's small device tables (twiddles, the Coulomb table v(G) of N values)
 * on the current device.  Returns HFX_ERR_INVALID_ARG, HFX_ERR_UNSUPPORTED_GRID, HFX_ERR_OOM
 * or HFX_ERR_CUDA on failure (and *out = NULL).
 * Environment variables read here (schedule and kernel-form choices; results do not depend on
 * them beyond rounding order): HFX_BLOCK (orbitals per block), HFX_BATCH_MB (transform budget),
 * HFX_PIPELINE=0 (one stream), HFX_NO_CT=1 (runtime-geometry kernels on every grid),
 * HFX_PENCIL=1 (pencil form of the plane passes), HFX_NO_TC=1 (ACE contractions off the
 * tensor cores), HFX_DENSE_TMA=0 (dense accumulate pass with per-thread copies instead of TMA),
 * HFX_PREFETCH=0 (no L2 prefetch of the next work item), HFX_GRID_WAVES (blocks per resident
 * slot of the compile-time plane passes, default 16). */
hfx_status hfx_create(const hfx_box* box, const int32_t grid[3], double ecut, hfx_kernel kernel,
                      double alpha, hfx_precision prec, hfx_ctx** out);

/* hfx_workspace_bytes -- device scratch that hfx_apply needs for n_orb orbitals and a list
 * of n_pairs pairs (pair staging, the per-batch transforms and the per-couple energy sums;
 * plus, on the FP32 paths, an FP32 copy of the orbitals and the FP32 accumulator of V_x phi that
 * is widened into the caller's FP64 array at the end of the call).  Returns 0 on bad arguments.
 * (Library plumbing; the paper has no counterpart.) */
size_t hfx_workspace_bytes(const hfx_ctx* c, int32_t n_orb, int64_t n_pairs);

/* hfx_set_workspace -- hand the context a caller-owned device buffer (e.g. a torch tensor)
 * of `bytes` bytes, 256-byte aligned.  The context keeps the pointer until it is replaced
 * or the context is destroyed; it never frees it.  Calls that use the same context must
 * not overlap on the GPU.
 * (Library plumbing; the paper has no counterpart.) */
hfx_status hfx_set_workspace(hfx_ctx* c, void* dev_ptr, size_t bytes);

/* hfx_apply -- one exact-exchange evaluation (Eqs. vx, vij, HFX).
 *   orbitals : device, [n_orb][n1][n2][n3], FP64 (FP32 with HFX_ORBITALS_F32); read only.
 *   n_orb    : number of occupied orbitals (> 0).
 *   pairs    : device int32 [n_pairs][2], entries 0 <= i <= j < n_orb, any order (Sec. 2.1
 *              screening: any subset of pairs may be listed).  Invalid entries are skipped
 *              and reported by hfx_sync_status as HFX_ERR_BAD_PAIR_LIST.
 *   n_pairs  : >= 0; 0 gives E_x = 0 and V_x phi = 0 (or leaves them with HFX_ACCUMULATE).
 *   flags    : HFX_ENERGY_ONLY | HFX_ACCUMULATE | HFX_ORBITALS_F32.
 *   ex_dev   : device FP64 scalar receiving E_x (Hartree).
 *   vxphi    : device FP64 [n_orb][n1][n2][n3] receiving V_x phi; NULL only with
 *              HFX_ENERGY_ONLY.
 *   cuda_stream : stream to enqueue on.
 * Needs a workspace of at least hfx_workspace_bytes(c, n_orb, n_pairs).  Asynchronous:
 * results are valid once the stream reaches them.  Deterministic: the same inputs give
 * bit-identical results. */
hfx_status hfx_apply(hfx_ctx* c, const void* orbitals, int32_t n_orb, const int32_t* pairs,
                     int64_t n_pairs, uint32_t flags, double* ex_dev, double* vxphi,
                     void* cuda_stream);

/* One problem of a batched call: the arguments of hfx_apply for one context. */
typedef struct {
  const void* orbitals;
  int32_t n_orb;
  const int32_t* pairs;
  int64_t n_pairs;
  uint32_t flags;
  double* ex_dev;
  double* vxphi;
} hfx_apply_args;

/* hfx_apply_batched -- several independent problems (each with its own context, so its own
 * cell, grid, orbital count and workspace), all their passes in ONE persistent launch: the
 * uneven batch of independent configurations, distributed as independent work the way Sec. 2.2
 * spreads independent work over processor groups.
 *   Per problem the call first enqueues its staging (V_x phi cleared, pairs placed, the FP32
 *   orbital copy), then one launch runs every pass of every problem from a device work queue:
 *   items (planes, tiles) are taken in a fixed task order by all blocks; the tasks of one problem
 *   run as a chain (forward, x/Coulomb and accumulate pass of each batch of couples, then the
 *   energy sum) and the chains of different problems are interleaved, so the problems share the
 *   GPU.  A block whose item depends on an unfinished task waits for it at most the context's
 *   wait budget (hfx_set_wait_budget); a wait that runs out sets HFX_ERR_TIMEOUT in the error
 *   word of that problem's context, every block then stops, and the call's results are undefined.
 *   Results equal hfx_apply's up to rounding order (the batched passes are the runtime-geometry
 *   forms for every grid).
 *   Rules: same argument rules per problem as hfx_apply; one distinct context per problem; every
 *   context needs the same precision and device and planes that fit in shared memory
 *   (HFX_ERR_UNSUPPORTED_GRID otherwise); each context's workspace must hold hfx_workspace_bytes
 *   for its problem; batched calls led by one context must not overlap on the GPU.  The queue tables live in a
 *   device buffer owned by the first context (ctxs[0]); the first call that needs a larger one
 *   allocates it (and synchronises the stream), so make that call before any stream capture --
 *   during capture such a call is rejected with HFX_ERR_INVALID_ARG.  Stops at the first problem
 *   whose arguments are rejected and returns that error. */
hfx_status hfx_apply_batched(hfx_ctx* const* ctxs, const hfx_apply_args* args, int32_t n,
                             void* cuda_stream);

/* flag for failure-detection tests (no GPU fault is involved; the call's result is void):
 *   in hfx_apply_args of hfx_apply_batched: the problem's first dependent wait expects one more
 *   finished item than its predecessor task has, so it can only end by running out of the wait
 *   budget (HFX_ERR_TIMEOUT);
 *   with hfx_apply on an FP32 context whose dense accumulate pass moves its tiles by TMA (cubic
 *   compile-time edges that are multiples of 4): the first tile barrier of every dense block
 *   expects 16 bytes more than its tensor copy brings, so its wait runs out (about 1 s per block
 *   resident at the time; later blocks of the launch skip their work) and hfx_sync_status
 *   reports HFX_ERR_TIMEOUT; on other contexts the flag has no effect.
 * hfx_apply_sequential rejects it. */
#define HFX_TEST_STALL    0x100u

/* hfx_apply_sequential -- (Sec. 2.2, independent work, as for hfx_apply_batched) the same
 * problems as separate hfx_apply calls, one after another on the stream, each with the fastest
 * passes its own context has (compile-time geometry where the edge has it).  Same argument
 * rules; HFX_TEST_STALL is rejected. */
hfx_status hfx_apply_sequential(hfx_ctx* const* ctxs, const hfx_apply_args* args, int32_t n,
                                void* cuda_stream);

/* hfx_set_wait_budget -- clock cycles one device-side wait of hfx_apply_batched may last when
 * this context leads the batch (0: the default, 2^34 cycles, about 8 s at 2 GHz).
 * (Library plumbing; the paper has no counterpart.) */
hfx_status hfx_set_wait_budget(hfx_ctx* c, int64_t cycles);

/* hfx_apply_noalloc -- hfx_apply for callers that cannot allocate device memory.
 * The paper has no counterpart: this exists for callers that must not call cudaMalloc when
 * they evaluate the exchange -- code running inside a device allocator or memory-pool callback
 * (allocating there would recurse), hosts whose CUDA memory is owned by another framework that
 * forbids side allocations, and latency-critical loops that cannot afford cudaMalloc's implicit
 * synchronisation.  It computes exactly what hfx_apply computes, with the same arguments and
 * argument errors, but takes no workspace: its scratch (pair staging, transforms, energy sums,
 * the FP32 orbital copy and the schedule tables) is one static device array of
 * HFX_NOALLOC_SCRATCH_BYTES bytes inside the library, which every GPU that loads the library
 * holds until the process exits.  It allocates nothing (no cudaMalloc, cudaFree or allocating
 * library call) and never touches the context's own workspace.
 *   - The batches of one call run one after another on cuda_stream (no second stream), each sized
 *     to the scratch left after the tables: problems whose default batches would not fit run in
 *     more, smaller batches.  Problems in which one orbital-block pair's transforms, plus the
 *     per-call tables, exceed HFX_NOALLOC_SCRATCH_BYTES are rejected with HFX_ERR_OOM before
 *     anything is enqueued (e.g. 32 orbitals on a 32^3 grid fit in both precisions, 32 orbitals
 *     on 72^3 do not; use hfx_apply with a workspace beyond that).
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture.
 *   - The schedule tables reach the array as the arguments of small kernels launched on
 *     cuda_stream (no host-to-device copy, so no host buffer has to outlive the call).
 *   - The context itself is only read: its workspace, streams and profiling settings are neither
 *     used nor changed, so the caller's workspace keeps its contents.
 *   - Every call shares the one array, which keeps the previous call's contents (each call
 *     re-initialises what it needs).  Calls that overlap on the GPU -- on any stream, any
 *     context -- race on the array: serialise them. */
#define HFX_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
hfx_status hfx_apply_noalloc(hfx_ctx* c, const void* orbitals, int32_t n_orb, const int32_t* pairs,
                             int64_t n_pairs, uint32_t flags, double* ex_dev, double* vxphi,
                             void* cuda_stream);

/* hfx_sync_status -- wait for `cuda_stream` and return (then clear) the device-side error
 * word of the context: HFX_OK, HFX_ERR_BAD_PAIR_LIST, HFX_ERR_TIMEOUT,
 * HFX_ERR_NOT_POSITIVE_DEFINITE or HFX_ERR_RANK_DEFICIENT.
 * (Library plumbing; the paper has no counterpart.) */
hfx_status hfx_sync_status(hfx_ctx* c, void* cuda_stream);

/* hfx_set_tuning -- schedule parameters of the context (what an autotuner varies; results do
 * not depend on them beyond rounding order):
 *   block       : orbitals per block (1..32, default 8; 4 and 8 have register-accumulating
 *                 kernels for full off-diagonal block pairs);
 *   batch_bytes : device memory for one batch of packed transforms (default 1 GiB);
 *   pipeline    : nonzero = the forward/x passes of the next batch run on a second stream beside
 *                 the accumulate pass of the current one (two transform buffers), 0 = one stream.
 * Synchronises the device when cached schedules have to be dropped; not during stream capture.
 * The workspace size (hfx_workspace_bytes) changes with these settings.
 * (Library plumbing; the paper has no counterpart.) */
hfx_status hfx_set_tuning(hfx_ctx* c, int32_t block, size_t batch_bytes, int32_t pipeline);

/* hfx_plan_stats -- what hfx_apply(c, ..., n_orb, ..., n_pairs, flags, ...) will launch, from the
 * host schedule alone (no device work):
 *   out[0] = kernel launches per call, out[1] = batches, out[2] = orbital block size,
 *   out[3] = largest number of packed pair couples (two pairs per complex 3D transform) held
 *   by one batch, out[4] = couples of the whole call when every block pair is full (the
 *   exact count for the complete pair list), out[5] = the part of out[4] in full off-diagonal
 *   block pairs (handled by the register-accumulating inverse-y pass).
 * (Measurement support; the paper has no counterpart.) */
hfx_status hfx_plan_stats(const hfx_ctx* c, int32_t n_orb, int64_t n_pairs, uint32_t flags, int64_t out[6]);

/* hfx_profile_enable / hfx_profile_read -- per-pass device time.  While enabled, every
 * hfx_apply on the context records CUDA events around each pass on its own stream.
 * hfx_profile_read waits for the recorded events and returns, per pass, the summed
 * milliseconds and the number of launches since the last read, then resets them; index
 * 0 pair staging (and the FP32 orbital copy), 1 forward yz-plane pass, 2 x/Coulomb pass,
 * 3 inverse-y/accumulate pass for full off-diagonal block pairs, 4 energy sum,
 * 5 inverse-y/accumulate pass for the other block pairs.  Not for use inside stream capture.
 * (Measurement support; the paper has no counterpart.) */
hfx_status hfx_profile_enable(hfx_ctx* c, int on);
hfx_status hfx_profile_read(hfx_ctx* c, double ms[6], int64_t launches[6]);

/* hfx_debug_check_guards -- HFX_DEBUG builds (libhfx_debug.so): enqueue on cuda_stream a check of
 * the guard bands that separate the slices of the context's workspace as the last hfx_apply laid
 * them out (every call fills them before its first pass and checks them after its last one); a
 * band that lost its pattern sets the corruption bit of the error word (hfx_sync_status:
 * HFX_ERR_CORRUPTION).  Debug builds also check, after the pair placement of every call, that each
 * placed couple sits at its canonical place in its block pair.  Release builds return
 * HFX_ERR_INVALID_ARG.
 * (A debugging aid; the paper has no counterpart.) */
hfx_status hfx_debug_check_guards(hfx_ctx* c, void* cuda_stream);

/* hfx_test_fail_allocation / hfx_test_live_allocations -- failure injection on the host, for
 * tests of the error paths (the paper has no counterpart).  Every device allocation the library
 * makes for itself (the context's tables in hfx_create, an n_orb's schedule tables on its first
 * hfx_apply, the batch tables of hfx_apply_batched) goes through one allocator.  After
 * hfx_test_fail_allocation(k), k >= 0, that allocator lets k allocations through and fails the
 * next one as cudaMalloc does when the device is out of memory (cudaMalloc is not called for it);
 * the call that needed it returns HFX_ERR_OOM and frees what it had allocated; later allocations
 * succeed again.  k < 0 cancels a pending failure.  Process-wide, all devices and contexts.
 * hfx_test_live_allocations returns the number of device allocations the library holds (all
 * contexts): a failed call leaves it where it was before the call.  Neither touches the GPU. */
void hfx_test_fail_allocation(int64_t k);
int64_t hfx_test_live_allocations(void);

/* hfx_last_error -- the calling thread's last error message ("" if none); valid until the
 * thread's next libhfx call.
 * (Library plumbing; the paper has no counterpart.) */
const char* hfx_last_error(void);

/* hfx_destroy -- free the context and its tables (not the workspace).  NULL is a no-op.
 * (Library plumbing; the paper has no counterpart.) */
void hfx_destroy(hfx_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* HFX_H_ */
