// libhfx host side: contexts, tables, the pair-block schedule, workspace layout, the
// device-side pair-list staging kernels and the per-call launch sequence.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hfx.h"
#include "../../include/hfx_ace.h"
#include "../../include/hfx_sinr.h"
#include "hfx_ace_internal.h"
#include "hfx_internal.h"
#include "hfx_schedule.h"
#include "tc_sm100.cuh"

using namespace hfx;

// an NVTX range around the enqueueing of one pass (host side; near free without a tool attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// ------------------------------------------------------------------------------------
// error reporting
// ------------------------------------------------------------------------------------
static thread_local std::string g_last_error;

static hfx_status fail(hfx_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define HFX_CUDA_TRY(expr)                                                                     \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(HFX_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                   \
  } while (0)

// ------------------------------------------------------------------------------------
// FFT plans: each edge is split by best_factors (fft_plan.h)
// ------------------------------------------------------------------------------------
static bool make_dim_plan(int n, DimPlan& d) {
  if (n < 2 || n > 256) return false;
  const Factors f = best_factors(n);
  if (f.ns < 1) return false;
  d.n = n;
  d.ns = f.ns;
  int m = n;
  for (int s = 0; s < d.ns; ++s) {
    d.r[s] = f.r[s];
    m /= f.r[s];
    d.m[s] = m;
  }
  for (int s = d.ns; s < kMaxStages; ++s) { d.r[s] = 1; d.m[s] = 1; }
  for (int s = 0; s < kMaxStages; ++s) d.mdiv[s] = FastDiv::make((uint32_t)d.m[s]);
  d.ndiv = FastDiv::make((uint32_t)n);
  return true;
}

// frequency index stored at position `pos` after the forward (DIF) stages of plan d
static int freq_of_pos(const DimPlan& d, int pos) {
  int freq = 0, mult = 1, n = d.n;
  for (int s = 0; s < d.ns; ++s) {
    const int m = n / d.r[s];
    const int k2 = pos / m;
    pos %= m;
    freq += mult * k2;
    mult *= d.r[s];
    n = m;
  }
  return freq;
}

// workspace slices of one call (offsets from the workspace base)
struct Layout {
  size_t orb32, v32, W, W2, epart, eblk, couples, total;
  // HFX_DEBUG builds: guard bands after the slices (offsets), filled before and checked after a call
  int nguard = 0;
  size_t guard[8] = {};
};
constexpr size_t kGuardBytes = 256;
constexpr uint32_t kGuardWord = 0xA5C3F00Du;

// ------------------------------------------------------------------------------------
// tensor maps (TMA)
// ------------------------------------------------------------------------------------
// cuTensorMapEncodeTiled, reached through the runtime's driver entry point (the library does not
// link the driver library itself); NULL when the driver does not offer it
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// a 4-D FP32 tensor map over `base`: extents dims (dims[0] contiguous), byte strides of dimensions
// 1..3 (any order), box sizes; elements outside the tensor read as zero.  False when the driver
// refuses the description (alignment, sizes) or offers no encoder.
static bool encode_f32_4d(CUtensorMap* m, const void* base, const cuuint64_t dims[4], const cuuint64_t strides[3],
                          const cuuint32_t box[4]) {
  const EncodeTiledFn f = encode_tiled();
  if (!f) return false;
  const cuuint32_t unit[4] = {1, 1, 1, 1};
  return f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides, box, unit,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the maps of the TMA dense accumulate pass (tiles it reads; V also the tensor its reduce-adds
// write) for a cubic grid of edge n: a transform buffer of
// `cap` couples, W[couple][x][y][z] complex FP32, as (z reals, couple, y, x) with boxes of 8
// complex x `cpi` couples x n rows; the FP32 orbitals orb[orbital][x][y][z] and the FP32
// accumulator V (same layout) as (z, y, orbital, x) with boxes of 8 x n x 8
static bool encode_dense_maps(CUtensorMap* tmW, const void* W, long long cap, int cpi, CUtensorMap* tmOrb,
                              const void* orb, CUtensorMap* tmV, const void* V, int n_orb, int n) {
  const cuuint64_t nn = (cuuint64_t)n, N3 = nn * nn * nn;
  const cuuint64_t dw[4] = {2 * nn, (cuuint64_t)cap, nn, nn};
  const cuuint64_t sw[3] = {N3 * 8, nn * 8, nn * nn * 8};
  const cuuint32_t bw[4] = {16, (cuuint32_t)cpi, (cuuint32_t)n, 1};
  const cuuint64_t dorb[4] = {nn, nn, (cuuint64_t)n_orb, nn};
  const cuuint64_t sorb[3] = {nn * 4, N3 * 4, nn * nn * 4};
  const cuuint32_t borb[4] = {8, (cuuint32_t)n, 8, 1};
  return cap > 0 && encode_f32_4d(tmW, W, dw, sw, bw) && encode_f32_4d(tmOrb, orb, dorb, sorb, borb) &&
         encode_f32_4d(tmV, V, dorb, sorb, borb);
}

// ------------------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------------------
struct hfx_ctx {
  int grid[3];
  long long N;
  double lat[3][3];
  double omega;
  double ecut;
  int kernel;
  double alpha;
  int prec;
  int device;
  int sm_count;
  int max_smem;
  Geo geo;
  void* d_tw[3] = {nullptr, nullptr, nullptr};
  void* d_vtab = nullptr;
  int* d_err = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int bsize = 8;
  size_t transform_budget = size_t(1) << 30;
  int blocks_fwd = 1, blocks_x = 1;
  int gen_grp = 1, gen_phi = 0;  // generic accumulate pass: couples per group, orbital tiles on chip
  // second stream and events: the forward and x passes of batch b+1 run beside the accumulate
  // pass of batch b (double-buffered transforms)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_p2 = nullptr, ev_p3[2] = {nullptr, nullptr};
  bool pipeline = true;
  // pencil form of the forward/x passes (a plane does not fit in shared memory): row-block size
  bool pencil = false;
  int rb = 0;
  // compile-time-geometry passes (FP32, cubic grid with an instantiated edge), else NULL
  const CtFns* ct = nullptr;
  void* d_twct = nullptr;        // per-stage twiddle tables of the edge
  int blocks_fwd_ct = 1, blocks_x_ct = 1;
  // the compile-time dense accumulate pass moves its tiles by TMA (HFX_DENSE_TMA=0: per-thread
  // asynchronous copies)
  bool dense_tma = true;
  // the compile-time forward and x passes prefetch their next work item into L2 (HFX_PREFETCH=0: no)
  bool prefetch = true;
  // blocks of the compile-time forward and x passes per resident block slot (each block loops over
  // items; HFX_GRID_WAVES)
  int ct_waves = 16;
  // HFX_PREC_MIXED_TC: the forward plane pass's DFTs on the tensor cores (pre-split DFT matrix)
  bool tc_dft = false;
  void* d_dftb = nullptr;
  int blocks_fwd_tc = 1;
  std::map<int, std::unique_ptr<Schedule>> sched;  // by n_orb
  // queue tables of hfx_apply_batched when this context comes first in a batch
  void* d_batch = nullptr;
  size_t batch_bytes = 0;
  long long wait_budget = 1LL << 34;  // clock cycles a device-side wait may take (~8 s)
  // HFX_DEBUG builds: the guard bands of the last call's workspace layout
  Layout dbg_layout;
  char* dbg_ws = nullptr;
  // FP32 contexts: the ACE contractions on the tensor cores (tcgen05, TF32 x 3); HFX_NO_TC=1
  // keeps them on the FP32 SIMT kernels
  bool ace_tc = true;
  // optional per-pass device timing (hfx_profile_enable)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double prof_ms[9] = {};
  long long prof_n[9] = {};
};

// slots 0..5: exchange passes (hfx_profile_read); 6..8: ACE / screen kernels (hfx_ace_profile_read)
enum { kProfStage = 0, kProfFwd = 1, kProfX = 2, kProfAcc = 3, kProfEnergy = 4, kProfAccGeneric = 5, kProfSlots = 6,
       kProfAceGram = 6, kProfAceLmul = 7, kProfAceSmall = 8, kProfAllSlots = 9 };

static cudaEvent_t prof_event(hfx_ctx* c) {
  if (c->ev_pool.empty()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = c->ev_pool.back();
  c->ev_pool.pop_back();
  return e;
}

// records an event on `st` when profiling is on; returns it (or NULL)
static cudaEvent_t prof_mark(hfx_ctx* c, cudaStream_t st) {
  if (!c->prof_on) return nullptr;
  cudaEvent_t e = prof_event(c);
  if (e) cudaEventRecord(e, st);
  return e;
}
static void prof_close(hfx_ctx* c, int slot, cudaEvent_t begin, cudaStream_t st) {
  if (!c->prof_on || !begin) return;
  cudaEvent_t e = prof_event(c);
  if (!e) return;
  cudaEventRecord(e, st);
  c->ev_pending.push_back({slot, {begin, e}});
}

static size_t real_size(const hfx_ctx* c) { return c->prec == HFX_PREC_FP64 ? 8 : 4; }
static size_t cplx_size(const hfx_ctx* c) { return 2 * real_size(c); }
static int zchunk(const hfx_ctx* c) { return c->prec == HFX_PREC_FP64 ? 4 : 8; }

static size_t smem_fwd(const hfx_ctx* c) {
  return (size_t)(c->grid[1] * (c->grid[2] + 1) + c->grid[1] + c->grid[2]) * cplx_size(c);
}
static size_t smem_x(const hfx_ctx* c) {
  return (size_t)(c->grid[0] * (c->grid[2] + 1) + c->grid[0] + c->grid[2]) * cplx_size(c);
}
static int gen_cap_max(const hfx_ctx* c) { return (c->bsize * c->bsize + 1) / 2; }
static size_t smem_acc_cfg(const hfx_ctx* c, int grp, int phi) {
  const int zc = zchunk(c);
  const size_t pts = (size_t)c->grid[1] * zc;
  return (size_t)(kGenRing * c->grid[1] * grp * zc + c->grid[1]) * cplx_size(c) +
         (size_t)(2 * c->bsize) * pts * real_size(c) * (1 + phi) + (size_t)gen_cap_max(c) * sizeof(int4);
}
static size_t smem_acc(const hfx_ctx* c) { return smem_acc_cfg(c, c->gen_grp, c->gen_phi); }
// largest couple group (4, 2, 1), orbital tiles on chip when they fit, for the generic pass
static bool choose_generic(hfx_ctx* c) {
  for (int grp : {4, 2, 1})
    for (int phi : {1, 0})
      if (smem_acc_cfg(c, grp, phi) + 512 <= (size_t)c->max_smem) {
        c->gen_grp = grp;
        c->gen_phi = phi;
        return true;
      }
  return false;
}
static size_t smem_dense(const hfx_ctx* c) {
  const int zc = zchunk(c);
  return (size_t)(kDenseRing * c->grid[1] * (c->bsize / 2) * zc + c->grid[1]) * cplx_size(c) +
         (size_t)2 * c->bsize * c->grid[1] * zc * real_size(c);
}
static size_t smem_plane_ct(int n) { return (size_t)(n * (n + 1) + stage_plan(n).twtotal) * sizeof(float2); }
static size_t smem_dense_ct(int n, int b) {
  const int zc = 8, ln = dense_rows_ct(n) * (b / 2) * zc, pts = n * zc;
  return (size_t)(kDenseRingCt * n * ln + stage_plan(n).twtotal) * sizeof(float2) + (size_t)2 * b * pts * sizeof(float);
}
// the TMA form: 128 more bytes, so that its tensor-copy destinations can start on 128-byte boundaries
static size_t smem_dense_tma_ct(int n) { return smem_dense_ct(n, 8) + 128; }
static size_t smem_diag_ct(int n, int b) {
  const int zc = 8, ln = kDiagCouplesPerItCt * zc, pts = n * zc;
  return (size_t)(kDenseRingCt * n * ln + stage_plan(n).twtotal) * sizeof(float2) + (size_t)b * pts * sizeof(float);
}

// per-stage twiddle tables of one edge: stage s with m > 1 holds w_L^{j1 k}, j1 < m, k < r, L = r m
static std::vector<double> stage_twiddles(int n) {
  const StagePlan p = stage_plan(n);
  std::vector<double> tw(2 * (size_t)std::max(p.twtotal, 1), 0.0);
  for (int s = 0; s < p.ns; ++s) {
    if (p.m[s] <= 1) continue;
    const int r = p.r[s], m = p.m[s], L = r * m;
    for (int j1 = 0; j1 < m; ++j1)
      for (int k = 0; k < r; ++k) {
        const cs_pair w = cossin_2pi_frac((long long)j1 * k, L);
        const size_t idx = (size_t)p.twoff[s] + (size_t)j1 * r + k;
        tw[2 * idx] = w.c;
        tw[2 * idx + 1] = -w.s;
      }
  }
  return tw;
}

// pencil kernels: rows blocks of rb rows (padded stride n3 + 1) and single z-chunk columns
static size_t smem_rows(const hfx_ctx* c, int rb) {
  return (size_t)(rb * (c->grid[2] + 1) + c->grid[2]) * cplx_size(c);
}
static size_t smem_cols(const hfx_ctx* c, int n) { return (size_t)(n * zchunk(c) + n) * cplx_size(c); }
// energy partial sums per couple: one per y-plane, or per (y-plane, z-chunk) in the pencil form
static int eparts(const hfx_ctx* c) { return c->pencil ? c->grid[1] * (c->grid[2] / zchunk(c)) : c->grid[1]; }

static bool dense_available(const hfx_ctx* c) {
  return c->prec == HFX_PREC_FP64 ? Passes<double>::has_dense(c->bsize) : Passes<float>::has_dense(c->bsize);
}
// the register-accumulating pass for full diagonal block pairs exists for the compile-time FP32
// geometry with blocks of 8
static bool diag_available(const hfx_ctx* c) {
  return c->ct != nullptr && c->prec == HFX_PREC_FP32 && c->bsize == 8;
}

// Every device allocation the library makes for itself (context tables, schedules, batch tables)
// goes through dev_alloc / dev_free: one place that counts what is held and that a test can make
// fail (hfx_test_fail_allocation), so the error paths are exercised without exhausting a GPU.
static std::mutex g_alloc_mu;
static long long g_alloc_fail_in = -1;  // allocations to let through before one fails; -1: none fails
static long long g_alloc_live = 0;      // device allocations held by the library, all contexts

static cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_alloc_fail_in >= 0 && g_alloc_fail_in-- == 0) return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    ++g_alloc_live;
  } else {
    *p = nullptr;
  }
  return e;
}

static void dev_free(void* p) {
  if (!p) return;
  cudaFree(p);
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  --g_alloc_live;
}

extern "C" void hfx_test_fail_allocation(int64_t k) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc_fail_in = k >= 0 ? (long long)k : -1;
}

extern "C" int64_t hfx_test_live_allocations(void) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return (int64_t)g_alloc_live;
}

static void free_ctx_tables(hfx_ctx* c) {
  for (cudaEvent_t* e : {&c->ev_fork, &c->ev_p2, &c->ev_p3[0], &c->ev_p3[1]}) {
    if (*e) cudaEventDestroy(*e);
    *e = nullptr;
  }
  if (c->side) cudaStreamDestroy(c->side);
  c->side = nullptr;
  dev_free(c->d_twct);
  c->d_twct = nullptr;
  dev_free(c->d_batch);
  c->d_batch = nullptr;
  dev_free(c->d_dftb);
  c->d_dftb = nullptr;
  c->batch_bytes = 0;
  for (auto& pe : c->ev_pending) { cudaEventDestroy(pe.second.first); cudaEventDestroy(pe.second.second); }
  c->ev_pending.clear();
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
  for (auto& p : c->d_tw) { dev_free(p); p = nullptr; }
  dev_free(c->d_vtab);
  dev_free(c->d_err);
  c->d_vtab = nullptr;
  c->d_err = nullptr;
  for (auto& kv : c->sched) {
    Schedule& S = *kv.second;
    for (void* p : {(void*)S.d_slot_blocks, (void*)S.d_slot_of_bp, (void*)S.d_slot_couple_base,
                    (void*)S.d_dense_slots, (void*)S.d_generic_slots, (void*)S.d_diag_slots})
      dev_free(p);
  }
  c->sched.clear();
}

template <typename T>
static std::vector<T> to_real_vec(const std::vector<double>& v) {
  std::vector<T> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
  return o;
}

static hfx_status upload(void** dst, const void* src, size_t bytes) {
  cudaError_t e = dev_alloc(dst, bytes);
  if (e != cudaSuccess) return fail(HFX_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(HFX_ERR_CUDA, "cudaMemcpy failed: %s", cudaGetErrorString(e));
  return HFX_OK;
}

static hfx_status build_tables(hfx_ctx* c) {
  // twiddles w_n^t = exp(-2 pi i t / n), t < n, from the rational angle t/n
  for (int d = 0; d < 3; ++d) {
    const int n = c->grid[d];
    std::vector<double> tw(2 * n);
    for (int t = 0; t < n; ++t) {
      const cs_pair w = cossin_2pi_frac(t, n);
      tw[2 * t] = w.c;
      tw[2 * t + 1] = -w.s;
    }
    hfx_status st;
    if (c->prec == HFX_PREC_FP64) st = upload(&c->d_tw[d], tw.data(), tw.size() * sizeof(double));
    else { auto f = to_real_vec<float>(tw); st = upload(&c->d_tw[d], f.data(), f.size() * sizeof(float)); }
    if (st != HFX_OK) return st;
  }
  // Coulomb table in storage order: v[x_pos][y_pos][z_pos] = 4 pi / |G|^2 (0 at G = 0)
  double B[3][3];  // reciprocal rows b_k with a_i . b_k = 2 pi delta_ik
  {
    const double (*A)[3] = c->lat;
    const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                       A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                       A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    // inverse transpose: b_k = 2 pi (a_{k+1} x a_{k+2}) / det
    for (int k = 0; k < 3; ++k) {
      const double* p = A[(k + 1) % 3];
      const double* q = A[(k + 2) % 3];
      B[k][0] = 2.0 * kPi * (p[1] * q[2] - p[2] * q[1]) / det;
      B[k][1] = 2.0 * kPi * (p[2] * q[0] - p[0] * q[2]) / det;
      B[k][2] = 2.0 * kPi * (p[0] * q[1] - p[1] * q[0]) / det;
    }
  }
  const int n1 = c->grid[0], n2 = c->grid[1], n3 = c->grid[2];
  std::vector<int> mf[3];
  for (int d = 0; d < 3; ++d) {
    const int n = c->grid[d];
    mf[d].resize(n);
    for (int pos = 0; pos < n; ++pos) {
      const int f = freq_of_pos(c->geo.d[d], pos);
      mf[d][pos] = (f <= n / 2) ? f : f - n;
    }
  }
  // v at the integer frequency m (each component in (-n/2, n/2])
  auto kernel_at = [&](const int m[3]) {
    double G[3];
    for (int k = 0; k < 3; ++k) G[k] = m[0] * B[0][k] + m[1] * B[1][k] + m[2] * B[2][k];
    const double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    double val = (g2 > 0.0) ? 4.0 * kPi / g2 : 0.0;
    if (c->kernel == HFX_KERNEL_COULOMB_SPHERE && 0.5 * g2 >= 4.0 * c->ecut) val = 0.0;
    return val;
  };
  // The table holds the inversion-symmetric part of the kernel, (v(m) + v(m'))/2 with m' the
  // frequency of grid index -k: m' = -m except on a Nyquist plane (m_d = n_d/2, its own mirror).
  // In an orthogonal cell v(m') = v(m) bit for bit and nothing changes; in a non-orthogonal one
  // the two differ on the Nyquist planes, and only the symmetric part keeps every v_ij real and
  // the two-pairs-per-transform packing exact (for real pair densities it gives the same E_x as
  // v itself, and V_x phi = the real part of the inverse transform of v F).
  std::vector<double> v((size_t)c->N);
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n2; ++b)
      for (int e = 0; e < n3; ++e) {
        const int m[3] = {mf[0][a], mf[1][b], mf[2][e]};
        int mm[3];
        for (int d = 0; d < 3; ++d) mm[d] = (2 * m[d] == c->grid[d]) ? m[d] : -m[d];
        v[((size_t)a * n2 + b) * n3 + e] = 0.5 * (kernel_at(m) + kernel_at(mm));
      }
  hfx_status st;
  if (c->prec == HFX_PREC_FP64) st = upload(&c->d_vtab, v.data(), v.size() * sizeof(double));
  else { auto f = to_real_vec<float>(v); st = upload(&c->d_vtab, f.data(), f.size() * sizeof(float)); }
  if (st != HFX_OK) return st;
  {
    const cudaError_t e = dev_alloc((void**)&c->d_err, sizeof(int));
    if (e != cudaSuccess) return fail(HFX_ERR_OOM, "cudaMalloc(%zu) failed: %s", sizeof(int), cudaGetErrorString(e));
  }
  HFX_CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
  return HFX_OK;
}

// The DFT matrix of edge n for the tensor-core forward pass: B[j][k] over outputs j (Re of the
// frequency at position j for j < n, Im of the one at position j - n beyond) and inputs k (Re of
// point k for k < n, Im of point k - n beyond), forward sign; per k-block of 32 inputs a TF32 hi
// tile and a lo tile (x = hi + lo, hi rounded to the nearest TF32) in the SWIZZLE_128B K-major
// layout of 2n rows.
static std::vector<uint32_t> dft_tc_table(const DimPlan& d) {
  const int n = d.n, nb = 2 * n, kb_count = 2 * n / 32;
  const size_t tile_words = (size_t)nb * 32;
  std::vector<uint32_t> t((size_t)kb_count * 2 * tile_words, 0u);
  for (int j = 0; j < nb; ++j) {
    const int f = freq_of_pos(d, j % n);
    const bool im_out = j >= n;
    for (int k = 0; k < 2 * n; ++k) {
      const int tin = k % n;
      const bool im_in = k >= n;
      const cs_pair w = cossin_2pi_frac((long long)tin * f, n);
      const double v = im_out ? (im_in ? w.c : -w.s) : (im_in ? w.s : w.c);
      const float x = (float)v;
      uint32_t u;
      std::memcpy(&u, &x, 4);
      const uint32_t hu = (u + 0x1000u) & 0xFFFFE000u;
      float hi;
      std::memcpy(&hi, &hu, 4);
      const float lo = x - hi;
      uint32_t lu;
      std::memcpy(&lu, &lo, 4);
      const int kb = k / 32;
      const size_t w0 = (size_t)kb * 2 * tile_words + tc::swz128(j, k % 32) / 4;
      t[w0] = hu;
      t[w0 + tile_words] = lu;
    }
  }
  return t;
}

extern "C" hfx_status hfx_create(const hfx_box* box, const int32_t grid[3], double ecut, hfx_kernel kernel,
                                 double alpha, hfx_precision prec, hfx_ctx** out) {
  g_last_error.clear();
  if (!out) return fail(HFX_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!box || !grid) return fail(HFX_ERR_INVALID_ARG, "box or grid is NULL");
  if (kernel != HFX_KERNEL_COULOMB && kernel != HFX_KERNEL_COULOMB_SPHERE)
    return fail(HFX_ERR_INVALID_ARG, "unknown kernel %d", (int)kernel);
  if (prec != HFX_PREC_FP64 && prec != HFX_PREC_FP32 && prec != HFX_PREC_MIXED_TC)
    return fail(HFX_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
  const bool mixed_tc = prec == HFX_PREC_MIXED_TC;
  if (mixed_tc) prec = HFX_PREC_FP32;  // FP32 data and SIMT stages elsewhere; the forward DFTs on tensor cores
  if (kernel == HFX_KERNEL_COULOMB_SPHERE && !(ecut > 0.0)) return fail(HFX_ERR_INVALID_ARG, "ecut must be > 0");
  if (!std::isfinite(alpha)) return fail(HFX_ERR_INVALID_ARG, "alpha is not finite");
  std::unique_ptr<hfx_ctx> c(new hfx_ctx());
  for (int d = 0; d < 3; ++d) {
    c->grid[d] = grid[d];
    if (grid[d] % 2 != 0 || !make_dim_plan(grid[d], c->geo.d[d]))
      return fail(HFX_ERR_UNSUPPORTED_GRID, "grid edge %d = %d: need an even {2,3,5}-smooth size in [2, 256]", d,
                  (int)grid[d]);
  }
  c->N = (long long)grid[0] * grid[1] * grid[2];
  c->geo.n1 = grid[0]; c->geo.n2 = grid[1]; c->geo.n3 = grid[2]; c->geo.N = c->N;
  c->geo.S = grid[2] + 1;  // odd row stride: column accesses of consecutive lines hit distinct banks
  std::memcpy(c->lat, box->lattice, sizeof(c->lat));
  const double (*A)[3] = c->lat;
  const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return fail(HFX_ERR_INVALID_ARG, "cell volume is zero");
  c->omega = std::fabs(det);
  c->ecut = ecut;
  c->kernel = kernel;
  c->alpha = alpha;
  c->prec = prec;
  if (const char* s = std::getenv("HFX_BLOCK")) c->bsize = std::max(1, std::min(32, atoi(s)));
  if (const char* s = std::getenv("HFX_BATCH_MB")) c->transform_budget = (size_t)std::max(1, atoi(s)) << 20;
  if (const char* s = std::getenv("HFX_PIPELINE")) c->pipeline = atoi(s) != 0;
  if (const char* s = std::getenv("HFX_NO_TC")) c->ace_tc = atoi(s) == 0;
  if (const char* s = std::getenv("HFX_DENSE_TMA")) c->dense_tma = atoi(s) != 0;
  if (const char* s = std::getenv("HFX_PREFETCH")) c->prefetch = atoi(s) != 0;
  if (const char* s = std::getenv("HFX_GRID_WAVES")) c->ct_waves = std::max(1, std::min(64, atoi(s)));

  HFX_CUDA_TRY(cudaGetDevice(&c->device));
  HFX_CUDA_TRY(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
  HFX_CUDA_TRY(cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  if (!choose_generic(c.get()))
    return fail(HFX_ERR_UNSUPPORTED_GRID, "the accumulation tile of this grid does not fit in shared memory");
  const char* force_pencil = std::getenv("HFX_PENCIL");  // the pencil form on any grid (testing)
  if (std::max(smem_fwd(c.get()), smem_x(c.get())) + 512 > (size_t)c->max_smem ||
      (force_pencil && atoi(force_pencil) != 0)) {
    // planes too large for one SM: the forward and x passes run as row blocks and z-chunk pencils
    if (grid[2] % zchunk(c.get()) != 0)
      return fail(HFX_ERR_UNSUPPORTED_GRID, "grid planes exceed shared memory and n3 = %d is not a multiple of %d",
                  (int)grid[2], zchunk(c.get()));
    c->pencil = true;
    c->rb = std::max(1, std::min(grid[1], (int)((48 * 1024) / ((grid[2] + 1) * cplx_size(c.get())))));
  }
  const size_t plane_need = c->pencil ? std::max(smem_rows(c.get(), c->rb),
                                                 std::max(smem_cols(c.get(), grid[0]), smem_cols(c.get(), grid[1])))
                                      : std::max(smem_fwd(c.get()), smem_x(c.get()));
  const size_t need = std::max(plane_need, std::max(smem_acc(c.get()), smem_dense(c.get()))) + 512;
  if (need > (size_t)c->max_smem)
    return fail(HFX_ERR_UNSUPPORTED_GRID, "a grid tile needs %zu bytes of shared memory (limit %d) at this precision",
                need, c->max_smem);
  cudaError_t e = (prec == HFX_PREC_FP64) ? Passes<double>::set_smem_limit(c->max_smem - 512)
                                          : Passes<float>::set_smem_limit(c->max_smem - 512);
  if (e != cudaSuccess) return fail(HFX_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  if (!c->pencil) {
    e = (prec == HFX_PREC_FP64)
            ? Passes<double>::occupancy(smem_fwd(c.get()), smem_x(c.get()), &c->blocks_fwd, &c->blocks_x)
            : Passes<float>::occupancy(smem_fwd(c.get()), smem_x(c.get()), &c->blocks_fwd, &c->blocks_x);
    if (e != cudaSuccess) return fail(HFX_ERR_CUDA, "occupancy query: %s", cudaGetErrorString(e));
  }
  c->blocks_fwd = std::max(1, c->blocks_fwd);
  c->blocks_x = std::max(1, c->blocks_x);
  hfx_status st = build_tables(c.get());
  if (st != HFX_OK) { free_ctx_tables(c.get()); return st; }
  {
    cudaError_t es = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&c->ev_fork, &c->ev_p2, &c->ev_p3[0], &c->ev_p3[1]})
      if (es == cudaSuccess) es = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (es != cudaSuccess) {
      free_ctx_tables(c.get());
      return fail(HFX_ERR_CUDA, "stream/event creation failed: %s", cudaGetErrorString(es));
    }
  }
  // compile-time-geometry passes for FP32 cubic grids with an instantiated edge
  const char* no_ct = std::getenv("HFX_NO_CT");
  if (prec == HFX_PREC_FP32 && !c->pencil && grid[0] == grid[1] && grid[1] == grid[2] && !(no_ct && atoi(no_ct) != 0)) {
    const CtFns* f = ct_fns(grid[0]);
    const int n = grid[0];
    if (f && std::max({smem_plane_ct(n), smem_dense_tma_ct(n), smem_diag_ct(n, 8) + 128}) + 512 <= (size_t)c->max_smem) {
      e = f->prepare(c->max_smem - 512, smem_plane_ct(n), &c->blocks_fwd_ct, &c->blocks_x_ct);
      if (e != cudaSuccess) { free_ctx_tables(c.get()); return fail(HFX_ERR_CUDA, "kernel setup: %s", cudaGetErrorString(e)); }
      auto tw = to_real_vec<float>(stage_twiddles(n));
      st = upload(&c->d_twct, tw.data(), tw.size() * sizeof(float));
      if (st != HFX_OK) { free_ctx_tables(c.get()); return st; }
      c->blocks_fwd_ct = std::max(1, c->blocks_fwd_ct);
      c->blocks_x_ct = std::max(1, c->blocks_x_ct);
      c->ct = f;
      // TMA needs the driver's tensor-map encoder; without it the dense pass copies per thread
      if (!encode_tiled()) c->dense_tma = false;
    }
  }
  if (mixed_tc) {
    const int n = grid[0];
    if (!c->ct || !dft::tc_edge(n))
      return fail(HFX_ERR_UNSUPPORTED_GRID,
                  "HFX_PREC_MIXED_TC needs a cubic grid of edge 32, 48, 64 or 96 (got %d x %d x %d)", (int)grid[0],
                  (int)grid[1], (int)grid[2]);
    e = dft::tc_prepare(n, &c->blocks_fwd_tc);
    if (e != cudaSuccess) { free_ctx_tables(c.get()); return fail(HFX_ERR_CUDA, "kernel setup: %s", cudaGetErrorString(e)); }
    const std::vector<uint32_t> tb = dft_tc_table(c->geo.d[2]);
    st = upload(&c->d_dftb, tb.data(), tb.size() * sizeof(uint32_t));
    if (st != HFX_OK) { free_ctx_tables(c.get()); return st; }
    c->blocks_fwd_tc = std::max(1, c->blocks_fwd_tc);
    c->tc_dft = true;
  }
  *out = c.release();
  return HFX_OK;
}

extern "C" void hfx_destroy(hfx_ctx* c) {
  if (!c) return;
  free_ctx_tables(c);
  delete c;
}

extern "C" const char* hfx_last_error(void) { return g_last_error.c_str(); }

extern "C" hfx_status hfx_set_workspace(hfx_ctx* c, void* dev_ptr, size_t bytes) {
  g_last_error.clear();
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
  if (bytes && !dev_ptr) return fail(HFX_ERR_INVALID_ARG, "workspace pointer is NULL");
  if (((uintptr_t)dev_ptr) % 256) return fail(HFX_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  c->ws = dev_ptr;
  c->ws_bytes = bytes;
  return HFX_OK;
}

// ------------------------------------------------------------------------------------
// workspace layout
// ------------------------------------------------------------------------------------

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static Schedule make_host_schedule(const hfx_ctx* c, int n_orb) {
  Schedule S;
  build_schedule(S, n_orb, c->bsize, c->transform_budget, (size_t)c->N * cplx_size(c), dense_available(c),
                 diag_available(c));
  return S;
}

// two transform buffers when the batches of a call are pipelined on the context's two streams
static bool two_buffers(const hfx_ctx* c, const Schedule& S) { return S.nbatches > 1 && c->side && c->pipeline; }

static Layout layout_of(const hfx_ctx* c, const Schedule& S, int n_orb, bool second_buffer) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
#ifdef HFX_DEBUG
    if (L.nguard < 8) L.guard[L.nguard++] = off;
    off += kGuardBytes;
#endif
    return o;
  };
  const size_t orb32_bytes = (c->prec == HFX_PREC_FP32) ? (size_t)n_orb * c->N * 4 : 0;
  L.orb32 = take(orb32_bytes);
  // FP32 path: the call's FP32 accumulator of V_x phi (widened into the caller's FP64 array once)
  L.v32 = take(c->prec == HFX_PREC_FP32 ? (size_t)n_orb * c->N * 4 : 0);
  L.W = take((size_t)S.max_batch_couples * c->N * cplx_size(c));
  // a second transform buffer when batches are pipelined on two streams
  L.W2 = take(second_buffer ? (size_t)S.max_batch_couples * c->N * cplx_size(c) : 0);
  L.epart = take((size_t)S.max_total_couples * eparts(c) * sizeof(double));
  L.eblk = take((size_t)64 * sizeof(double));  // per-block energy sums (kEnergyBlocks)
  L.couples = take((size_t)S.max_total_couples * sizeof(int4));
  L.total = off;
  return L;
}

extern "C" size_t hfx_workspace_bytes(const hfx_ctx* c, int32_t n_orb, int64_t n_pairs) {
  if (!c || n_orb <= 0 || n_pairs < 0) return 0;
  Schedule S = make_host_schedule(c, n_orb);
  (void)n_pairs;
  return layout_of(c, S, n_orb, two_buffers(c, S)).total;
}

static hfx_status get_schedule(hfx_ctx* c, int n_orb, Schedule** out) {
  auto it = c->sched.find(n_orb);
  if (it != c->sched.end()) { *out = it->second.get(); return HFX_OK; }
  std::unique_ptr<Schedule> S(new Schedule(make_host_schedule(c, n_orb)));
  auto up = [&](void** dst, const void* src, size_t bytes) -> hfx_status {
    if (bytes == 0) {  // an empty list still gets a valid (unused) device pointer
      cudaError_t e = dev_alloc(dst, 16);
      return e == cudaSuccess ? HFX_OK : fail(HFX_ERR_OOM, "cudaMalloc(16) failed: %s", cudaGetErrorString(e));
    }
    return upload(dst, src, bytes);
  };
  hfx_status st = up((void**)&S->d_slot_blocks, S->slot_blocks.data(), S->slot_blocks.size() * sizeof(int2));
  if (st == HFX_OK) st = up((void**)&S->d_slot_of_bp, S->slot_of_bp.data(), S->slot_of_bp.size() * sizeof(int));
  if (st == HFX_OK)
    st = up((void**)&S->d_slot_couple_base, S->slot_couple_base.data(), S->slot_couple_base.size() * sizeof(int));
  if (st == HFX_OK) st = up((void**)&S->d_dense_slots, S->dense_slots.data(), S->dense_slots.size() * sizeof(int));
  if (st == HFX_OK)
    st = up((void**)&S->d_generic_slots, S->generic_slots.data(), S->generic_slots.size() * sizeof(int));
  if (st == HFX_OK) st = up((void**)&S->d_diag_slots, S->diag_slots.data(), S->diag_slots.size() * sizeof(int));
  if (st != HFX_OK) {
    for (void* p : {(void*)S->d_slot_blocks, (void*)S->d_slot_of_bp, (void*)S->d_slot_couple_base,
                    (void*)S->d_dense_slots, (void*)S->d_generic_slots, (void*)S->d_diag_slots})
      dev_free(p);
    return st;
  }
  *out = S.get();
  c->sched[n_orb] = std::move(S);
  return HFX_OK;
}

// ------------------------------------------------------------------------------------
// pair-list staging kernels (validate, bucket by block pair and weight class, stable order)
// ------------------------------------------------------------------------------------
__global__ void k_cast_f32(const double* __restrict__ src, float* __restrict__ dst, long long n) {
  const long long n2 = n / 2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = reinterpret_cast<const double2*>(src)[i];
    reinterpret_cast<float2*>(dst)[i] = make_float2((float)v.x, (float)v.y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) dst[n - 1] = (float)src[n - 1];
}

// every listed pair goes to its fixed place in the canonical couple layout of its block pair;
// entries outside 0 <= i <= j < n_orb, and second copies of a pair, are flagged and skipped
__global__ void k_plan_place(const int2* __restrict__ pairs, long long P, int n_orb, int bsize, int nb,
                             const int* __restrict__ slot_of_bp, const int* __restrict__ slot_couple_base,
                             int4* __restrict__ couples, int* __restrict__ err) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    const int2 ij = pairs[p];
    const int i = ij.x, j = ij.y;
    if (!(i >= 0 && j < n_orb && i <= j)) { atomicOr(err, kErrBadPair); continue; }
    const int bi = i / bsize, bj = j / bsize;
    const int slot = slot_of_bp[bi * nb + bj];
    const int I0 = bi * bsize, J0 = bj * bsize;
    const int si = min(bsize, n_orb - I0), sj = min(bsize, n_orb - J0);
    int t, c;
    if (bi != bj) {
      t = (i - I0) * sj + (j - J0);
      c = t >> 1;
    } else if (i != j) {
      const int a = i - I0, b = j - I0;  // a < b
      t = a * si - a * (a + 1) / 2 + (b - a - 1);
      c = t >> 1;
    } else {
      const int noff = si * (si - 1) / 2;
      t = i - I0;
      c = (noff + 1) / 2 + (t >> 1);
    }
    int* cp = reinterpret_cast<int*>(couples + slot_couple_base[slot] + c) + 2 * (t & 1);
    if (atomicCAS(cp, -1, i) != -1) { atomicOr(err, kErrBadPair); continue; }
    cp[1] = j;
  }
}

// E_x = scale * sum_g w_g sum_y epart[g][y], in two deterministic launches: block b of
// k_energy_blocks sums couples [b*chunk, (b+1)*chunk) in a fixed order, k_energy_final sums the
// kEnergyBlocks block results in order and stores or accumulates E_x
constexpr int kEnergyBlocks = 64;

__global__ void __launch_bounds__(256) k_energy_blocks(const double* __restrict__ epart, const int4* __restrict__ couples,
                                                       int total, int n2, double* __restrict__ eblk) {
  __shared__ double red[32];
  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int g0 = blockIdx.x * chunk, g1 = min(total, g0 + chunk);
  double s = 0.0;
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const int4 cp = couples[g];
    if (couple_empty(cp)) continue;
    // both halves of a couple share a weight class: diagonal pairs count once, others twice
    const bool diag = cp.x >= 0 ? cp.x == cp.y : cp.z == cp.w;
    double t = 0.0;
    for (int y = 0; y < n2; ++y) t += epart[(long long)g * n2 + y];
    s += (diag ? 1.0 : 2.0) * t;
  }
  const double tot = block_sum(s, red);
  if (threadIdx.x == 0) eblk[blockIdx.x] = tot;
}

__global__ void k_energy_final(const double* __restrict__ eblk, int nb, double scale, int accumulate,
                               double* __restrict__ ex) {
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += eblk[b];
  ex[0] = (accumulate ? ex[0] : 0.0) + scale * t;
}

static void launch_energy(const double* epart, const int4* couples, int total, int n2, double* eblk, double scale,
                          bool accumulate, double* ex, cudaStream_t st) {
  k_energy_blocks<<<kEnergyBlocks, 256, 0, st>>>(epart, couples, total, n2, eblk);
  k_energy_final<<<1, 1, 0, st>>>(eblk, kEnergyBlocks, scale, accumulate ? 1 : 0, ex);
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }

// HFX_DEBUG builds: fill / check the workspace guard bands (up to 8 bands of kGuardBytes)
struct GuardSet {
  int n;
  size_t off[8];
};
__global__ void k_guard_fill(char* ws, GuardSet g) {
  for (int b = 0; b < g.n; ++b)
    for (int i = threadIdx.x; i < (int)(kGuardBytes / 4); i += blockDim.x)
      reinterpret_cast<uint32_t*>(ws + g.off[b])[i] = kGuardWord ^ (uint32_t)(b * 977 + i);
}
__global__ void k_guard_check(const char* ws, GuardSet g, int* err) {
  for (int b = 0; b < g.n; ++b)
    for (int i = threadIdx.x; i < (int)(kGuardBytes / 4); i += blockDim.x)
      if (reinterpret_cast<const uint32_t*>(ws + g.off[b])[i] != (kGuardWord ^ (uint32_t)(b * 977 + i)))
        atomicOr(err, kErrGuard);
}
// HFX_DEBUG builds: every placed couple holds pairs of its slot's block pair, at their canonical
// places (the layout the accumulate passes assume)
__global__ void k_check_couples(const int4* __restrict__ couples, const int* __restrict__ slot_couple_base,
                                const int2* __restrict__ slot_blocks, int nslots, int n_orb, int bsize,
                                int* err) {
  for (int s = blockIdx.x; s < nslots; s += gridDim.x) {
    const int2 bp = slot_blocks[s];
    const int I0 = bp.x * bsize, J0 = bp.y * bsize;
    const int si = min(bsize, n_orb - I0), sj = min(bsize, n_orb - J0);
    const int base = slot_couple_base[s], cap = slot_couple_base[s + 1] - base;
    for (int c = threadIdx.x; c < cap; c += blockDim.x) {
      const int4 cp = couples[base + c];
      for (int h = 0; h < 2; ++h) {
        const int i = h ? cp.z : cp.x, j = h ? cp.w : cp.y;
        if (i < 0) continue;
        bool ok = i <= j && i >= I0 && i < I0 + si && j >= J0 && j < J0 + sj;
        if (ok) {
          int t, cc;
          if (bp.x != bp.y) {
            t = (i - I0) * sj + (j - J0);
            cc = t >> 1;
          } else if (i != j) {
            const int a = i - I0, b = j - I0;
            t = a * si - a * (a + 1) / 2 + (b - a - 1);
            cc = t >> 1;
          } else {
            const int noff = si * (si - 1) / 2;
            t = i - I0;
            cc = (noff + 1) / 2 + (t >> 1);
          }
          ok = cc == c && (t & 1) == h;
        }
        if (!ok) atomicOr(err, kErrLayout);
      }
    }
  }
}
static GuardSet guard_set(const Layout& L) {
  GuardSet g;
  g.n = L.nguard;
  for (int k = 0; k < 8; ++k) g.off[k] = L.guard[k];
  return g;
}

// V_x phi (FP64) = (accumulate ? V_x phi : 0) + the call's FP32 accumulator, widened exactly with
// integer operations (FP32 subnormals flush to zero); n is a multiple of 4
__device__ __forceinline__ void widen_v4(const float* __restrict__ v32, double* __restrict__ v, long long i4,
                                         int accumulate) {
  const float4 a = __ldcs(reinterpret_cast<const float4*>(v32) + i4);
  double2 lo = make_double2(ct::widen_exact(a.x), ct::widen_exact(a.y));
  double2 hi = make_double2(ct::widen_exact(a.z), ct::widen_exact(a.w));
  double2* d = reinterpret_cast<double2*>(v) + 2 * i4;
  if (accumulate) {
    const double2 o0 = d[0], o1 = d[1];
    lo.x += o0.x; lo.y += o0.y; hi.x += o1.x; hi.y += o1.y;
  }
  d[0] = lo;
  d[1] = hi;
}
__global__ void k_widen_v(const float* __restrict__ v32, double* __restrict__ v, long long n, int accumulate) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n / 4; i += (long long)gridDim.x * blockDim.x)
    widen_v4(v32, v, i, accumulate);
}

// Small tables reach device memory as kernel arguments (8 KiB per launch): no host buffer has to
// outlive the call (it may be captured in a graph) and no pageable-memory copy is involved.
constexpr int kTableWords = 2048;
struct TableChunk { uint32_t w[kTableWords]; };
__global__ void k_put_words(uint32_t* __restrict__ dst, TableChunk chunk, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = chunk.w[i];
}
static hfx_status put_table(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  const uint32_t* s = (const uint32_t*)src;
  size_t words = bytes / 4;
  uint32_t* d = (uint32_t*)dst;
  while (words > 0) {
    const int n = (int)std::min<size_t>(words, kTableWords);
    TableChunk ch;
    std::memcpy(ch.w, s, (size_t)n * 4);
    k_put_words<<<1, 256, 0, st>>>(d, ch, n);
    HFX_CUDA_TRY(cudaGetLastError());
    s += n;
    d += n;
    words -= (size_t)n;
  }
  return HFX_OK;
}


// ------------------------------------------------------------------------------------
// apply
// ------------------------------------------------------------------------------------
// where one call's scratch lives and how its batches run: the workspace base, the second stream
// for pipelined batches (NULL: every batch on the caller's stream) and whether per-pass events
// are recorded
struct CallEnv {
  char* ws;
  cudaStream_t side;
  bool prof;
};

template <typename T>
static hfx_status run_passes(hfx_ctx* c, Schedule& S, const Layout& L, const CallEnv& env, const T* orb, int n_orb,
                             uint32_t flags, double* vxphi, cudaStream_t st) {
  char* ws = env.ws;
  using C = cx<T>;
  const bool pipe = S.nbatches > 1 && env.side != nullptr && c->pipeline;
  // what the accumulate passes add into: V_x phi itself (FP64), or the call's FP32 accumulator
  T* vacc = std::is_same<T, float>::value ? (T*)(ws + L.v32) : (T*)vxphi;
  auto mark = [&](cudaStream_t s) { return env.prof ? prof_mark(c, s) : nullptr; };
  auto close = [&](int slot, cudaEvent_t e, cudaStream_t s) { if (env.prof) prof_close(c, slot, e, s); };
  C* Wbuf[2] = {(C*)(ws + L.W), (C*)(ws + (pipe ? L.W2 : L.W))};
  int4* couples = (int4*)(ws + L.couples);
  double* epart = (double*)(ws + L.epart);
  const Geo& g = c->geo;
  const bool energy_only = (flags & HFX_ENERGY_ONLY) != 0;
  const double vscale = -c->alpha / (double)c->N;
  const int zc = zchunk(c);
  const int nzc = (g.n3 + zc - 1) / zc;
  const int pts = g.n2 * zc;
  const int dense_np = pts > 2 * DenseBounds<2>::threads ? 4 : 2;
  const int dense_threads = std::min(dense_np == 2 ? DenseBounds<2>::threads : DenseBounds<4>::threads,
                                     (((pts + dense_np - 1) / dense_np) + 31) / 32 * 32);
  // the tensor maps of the TMA dense accumulate pass (one per transform buffer)
  CUtensorMap tmW[2] = {}, tmOrb = {}, tmV = {};
  bool dense_tma = false;
  // (tensor maps need 16-byte row strides: FP32 orbital rows of an edge that is a multiple of 4)
  if (std::is_same<T, float>::value && c->ct && S.b == 8 && c->dense_tma && !energy_only && g.n1 % 4 == 0) {
    const int cpi = dense_rows_ct(g.n1) * (S.b / 2);
    dense_tma =
        encode_dense_maps(&tmW[0], Wbuf[0], S.max_batch_couples, cpi, &tmOrb, orb, &tmV, vacc, n_orb, g.n1) &&
        encode_dense_maps(&tmW[1], Wbuf[1], S.max_batch_couples, cpi, &tmOrb, orb, &tmV, vacc, n_orb, g.n1);
    // the buffers are 16-byte aligned and the edges multiples of 4, so the driver has no reason to refuse
    if (!dense_tma) return fail(HFX_ERR_CUDA, "cuTensorMapEncodeTiled refused the dense pass's tensor maps");
  }
  // forward and x passes on `fs`, accumulate passes on the caller's stream `st`
  cudaStream_t fs = pipe ? env.side : st;
  if (pipe) {
    HFX_CUDA_TRY(cudaEventRecord(c->ev_fork, st));
    HFX_CUDA_TRY(cudaStreamWaitEvent(fs, c->ev_fork, 0));
  }
  for (int b = 0; b < S.nbatches; ++b) {
    C* W = Wbuf[b & 1];
    // buffer b & 1 was last read by the accumulate pass of batch b - 2
    if (pipe && b >= 2) HFX_CUDA_TRY(cudaStreamWaitEvent(fs, c->ev_p3[b & 1], 0));
    const int s0 = S.batch_slot_begin[b], s1 = S.batch_slot_begin[b + 1];
    const int c0 = S.slot_couple_base[s0], c1 = S.slot_couple_base[s1];
    const long long items1 = (long long)(c1 - c0) * g.n1, items2 = (long long)(c1 - c0) * g.n2;
    const int grid1 = (int)std::min<long long>(items1, (long long)c->sm_count * c->blocks_fwd * 8);
    const int grid2 = (int)std::min<long long>(items2, (long long)c->sm_count * c->blocks_x * 8);
    const CtFns* ct = std::is_same<T, float>::value ? c->ct : nullptr;
    NvtxRange nv_batch("hfx batch: forward, x/Coulomb, accumulate passes");
    cudaEvent_t e0 = mark(fs);
    if (c->pencil) {
      const int nzc3 = g.n3 / zc, nrb = (g.n2 + c->rb - 1) / c->rb;
      const long long cap = (long long)c->sm_count * 16;
      const int gr = (int)std::max<long long>(1, std::min<long long>((long long)(c1 - c0) * g.n1 * nrb, cap));
      const int gy = (int)std::max<long long>(1, std::min<long long>((long long)(c1 - c0) * g.n1 * nzc3, cap));
      const int gx = (int)std::max<long long>(1, std::min<long long>((long long)(c1 - c0) * g.n2 * nzc3, cap));
      Passes<T>::fwd_z_rows(g, gr, smem_rows(c, c->rb), fs, orb, couples, c0, c1, c->rb, W, (const C*)c->d_tw[2]);
      Passes<T>::fwd_y_cols(g, gy, smem_cols(c, g.n2), fs, couples, c0, c1, W, (const C*)c->d_tw[1]);
      close(kProfFwd, e0, fs);
      e0 = mark(fs);
      Passes<T>::x_cols(g, gx, smem_cols(c, g.n1), fs, couples, c0, c1, W, (const T*)c->d_vtab,
                        (const C*)c->d_tw[0], epart, energy_only ? 1 : 0);
      if (!energy_only)
        Passes<T>::inv_z_rows(g, gr, smem_rows(c, c->rb), fs, couples, c0, c1, c->rb, W, (const C*)c->d_tw[2]);
      close(kProfX, e0, fs);
    } else {
      if (ct && c->tc_dft) {
        const int gt = (int)std::min<long long>(items1, (long long)c->sm_count * c->blocks_fwd_tc);
        dft::fwd_yz_tc(g.n1, std::max(gt, 1), fs, (const float*)orb, g.N, couples, c0, c1, (float2*)W,
                       (const unsigned char*)c->d_dftb, c->d_err);
      } else if (ct) {
        const int gct = (int)std::min<long long>(items1, (long long)c->sm_count * c->blocks_fwd_ct * c->ct_waves);
        ct->fwd_yz(std::max(gct, 1), smem_plane_ct(g.n1), fs, (const float*)orb, g.N, couples, c0, c1, (float2*)W,
                   (const float2*)c->d_twct, c->prefetch ? 1 : 0);
      } else {
        Passes<T>::fwd_yz(g, std::max(grid1, 1), smem_fwd(c), fs, orb, couples, c0, c1, W, (const C*)c->d_tw[1],
                          (const C*)c->d_tw[2]);
      }
      close(kProfFwd, e0, fs);
      e0 = mark(fs);
      if (ct) {
        const int gct = (int)std::min<long long>(items2, (long long)c->sm_count * c->blocks_x_ct * c->ct_waves);
        ct->x_coulomb(std::max(gct, 1), smem_plane_ct(g.n1), fs, couples, c0, c1, (float2*)W, (const float*)c->d_vtab,
                      (const float2*)c->d_twct, epart, energy_only ? 1 : 0, c->prefetch ? 1 : 0);
      } else {
        Passes<T>::x_coulomb(g, std::max(grid2, 1), smem_x(c), fs, couples, c0, c1, W, (const T*)c->d_vtab,
                             (const C*)c->d_tw[0], (const C*)c->d_tw[2], epart, energy_only ? 1 : 0);
      }
      close(kProfX, e0, fs);
    }
    if (pipe) {
      HFX_CUDA_TRY(cudaEventRecord(c->ev_p2, fs));
      HFX_CUDA_TRY(cudaStreamWaitEvent(st, c->ev_p2, 0));
    }
    if (!energy_only) {
      e0 = mark(st);
      const int nd = S.dense_begin[b + 1] - S.dense_begin[b];
      const int ng = S.generic_begin[b + 1] - S.generic_begin[b];
      if (nd > 0 && ct && S.b == 8 && dense_tma)  // [dense block pairs]
        ct->y_acc_dense_tma(dim3(nzc, g.n1, nd), smem_dense_tma_ct(g.n1), st, tmW[b & 1], tmOrb, tmV, couples,
                            S.d_dense_slots + S.dense_begin[b], S.d_slot_couple_base, S.d_slot_blocks, c0,
                            (const float2*)c->d_twct, vscale, c->d_err, (flags & HFX_TEST_STALL) ? 1 : 0);
      else if (nd > 0 && ct && S.b == 8)
        ct->y_acc_dense(dim3(nzc, g.n1, nd), smem_dense_ct(g.n1, 8), st, (const float*)orb, g.N, couples,
                        S.d_dense_slots + S.dense_begin[b], S.d_slot_couple_base, S.d_slot_blocks, c0,
                        (const float2*)W, (const float2*)c->d_twct, (float*)vacc, vscale);
      else if (nd > 0)
        Passes<T>::y_acc_dense(g, dim3(nzc, g.n1, nd), dense_threads, smem_dense(c), st, S.b, orb, couples,
                               S.d_dense_slots + S.dense_begin[b], S.d_slot_couple_base, S.d_slot_blocks, c0, W,
                               (const C*)c->d_tw[1], vacc, vscale);
      if (nd > 0) close(kProfAcc, e0, st);
      const int ndg = S.diag_begin[b + 1] - S.diag_begin[b];
      e0 = mark(st);
      if (ndg > 0)  // [full diagonal block pairs]; the generic pass takes whatever is left
        ct->y_acc_diag(dim3(nzc, g.n1, ndg), smem_diag_ct(g.n1, 8) + 128, st, (const float*)orb, g.N, couples,
                       S.d_diag_slots + S.diag_begin[b], S.d_slot_couple_base, S.d_slot_blocks, c0,
                       (const float2*)W, (const float2*)c->d_twct, (float*)vacc, vscale, tmV,
                       dense_tma ? 1 : 0);
      if (ndg > 0) close(kProfAccGeneric, e0, st);
      e0 = mark(st);
      if (ng > 0)
        Passes<T>::y_acc_generic(g, dim3(nzc, g.n1, ng), smem_acc(c), st, orb, couples,
                                 S.d_generic_slots + S.generic_begin[b], S.d_slot_couple_base, S.d_slot_blocks, S.b,
                                 n_orb, c0, W, (const C*)c->d_tw[1], vacc, vscale, c->gen_grp, c->gen_phi,
                                 gen_cap_max(c));
      if (ng > 0) close(kProfAccGeneric, e0, st);
    }
    if (pipe) HFX_CUDA_TRY(cudaEventRecord(c->ev_p3[b & 1], st));
  }
  if (std::is_same<T, float>::value && !energy_only) {
    const long long n = (long long)n_orb * g.N;
    const int blocks = (int)std::min<long long>((n / 4 + 255) / 256, (long long)c->sm_count * 16);
    k_widen_v<<<std::max(blocks, 1), 256, 0, st>>>((const float*)vacc, vxphi, n, (flags & HFX_ACCUMULATE) ? 1 : 0);
    HFX_CUDA_TRY(cudaGetLastError());
  }
  return HFX_OK;
}

// argument checks shared by every exchange entry point (host-visible errors, nothing enqueued)
static hfx_status check_apply_args(const hfx_ctx* c, const void* orbitals, int32_t n_orb, const int32_t* pairs,
                                   int64_t n_pairs, uint32_t flags, const double* ex_dev, const double* vxphi) {
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
  if (flags & ~(HFX_ENERGY_ONLY | HFX_ACCUMULATE | HFX_ORBITALS_F32 | HFX_TEST_STALL))
    return fail(HFX_ERR_INVALID_ARG, "unknown flag bits");
  if (n_orb <= 0) return fail(HFX_ERR_INVALID_ARG, "n_orb must be > 0");
  if (n_pairs < 0 || n_pairs > (int64_t)1 << 31) return fail(HFX_ERR_INVALID_ARG, "n_pairs out of range");
  if (!orbitals || !ex_dev) return fail(HFX_ERR_INVALID_ARG, "orbitals or ex_dev is NULL");
  if (n_pairs > 0 && !pairs) return fail(HFX_ERR_INVALID_ARG, "pairs is NULL");
  if (!(flags & HFX_ENERGY_ONLY) && !vxphi) return fail(HFX_ERR_INVALID_ARG, "vxphi is NULL without HFX_ENERGY_ONLY");
  if ((flags & HFX_ORBITALS_F32) && c->prec != HFX_PREC_FP32)
    return fail(HFX_ERR_INVALID_ARG, "HFX_ORBITALS_F32 needs HFX_PREC_FP32");
  if (((uintptr_t)orbitals | (uintptr_t)pairs | (uintptr_t)vxphi) % 16 || ((uintptr_t)ex_dev % 8))
    return fail(HFX_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
  return HFX_OK;
}

// an empty pair list: E_x = 0 and V_x phi = 0, or both left alone with HFX_ACCUMULATE
static hfx_status apply_empty(const hfx_ctx* c, int32_t n_orb, uint32_t flags, double* ex_dev, double* vxphi,
                              cudaStream_t st) {
  if (!(flags & HFX_ACCUMULATE)) {
    k_set_scalar<<<1, 1, 0, st>>>(ex_dev, 0.0);
    if (!(flags & HFX_ENERGY_ONLY))
      HFX_CUDA_TRY(cudaMemsetAsync(vxphi, 0, (size_t)n_orb * c->N * sizeof(double), st));
  }
  HFX_CUDA_TRY(cudaGetLastError());
  return HFX_OK;
}

// stage a1 of one evaluation: V cleared (unless accumulating or energy-only), the pair list placed
// in the canonical couple layout, the FP32 orbital copy; *orb_pass = the orbitals the passes read
static hfx_status stage_call(hfx_ctx* c, Schedule& S, const Layout& L, const CallEnv& env, const void* orbitals,
                             int32_t n_orb, const int32_t* pairs, int64_t n_pairs, uint32_t flags, double* vxphi,
                             cudaStream_t st, const void** orb_pass) {
  char* ws = env.ws;
  const bool accumulate = (flags & HFX_ACCUMULATE) != 0;
  const bool energy_only = (flags & HFX_ENERGY_ONLY) != 0;
  if (c->prec == HFX_PREC_FP32) {
    // the FP32 accumulator starts at zero; V_x phi itself is written (or added to) at the end
    if (!energy_only) HFX_CUDA_TRY(cudaMemsetAsync(ws + L.v32, 0, (size_t)n_orb * c->N * sizeof(float), st));
  } else if (!accumulate && !energy_only) {
    HFX_CUDA_TRY(cudaMemsetAsync(vxphi, 0, (size_t)n_orb * c->N * sizeof(double), st));
  }
  int4* couples = (int4*)(ws + L.couples);
  HFX_CUDA_TRY(cudaMemsetAsync(couples, 0xff, (size_t)S.max_total_couples * sizeof(int4), st));
  {
    const int threads = 256;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n_pairs + threads - 1) / threads,
                                                                        (long long)c->sm_count * 8));
    k_plan_place<<<blocks, threads, 0, st>>>((const int2*)pairs, n_pairs, n_orb, S.b, S.nb, S.d_slot_of_bp,
                                             S.d_slot_couple_base, couples, c->d_err);
  }
  HFX_CUDA_TRY(cudaGetLastError());
  *orb_pass = orbitals;
  if (c->prec == HFX_PREC_FP32 && !(flags & HFX_ORBITALS_F32)) {
    float* dst = (float*)(ws + L.orb32);
    const long long n = (long long)n_orb * c->N;
    const int blocks = (int)std::min<long long>((n / 2 + 255) / 256 + 1, (long long)c->sm_count * 16);
    k_cast_f32<<<blocks, 256, 0, st>>>((const double*)orbitals, dst, n);
    HFX_CUDA_TRY(cudaGetLastError());
    *orb_pass = dst;
  }
  return HFX_OK;
}

// one evaluation with its schedule tables on the device and its scratch at env.ws: stage a1, the
// passes of every batch, then the energy sum
static hfx_status apply_with(hfx_ctx* c, Schedule& S, const Layout& L, const CallEnv& env, const void* orbitals,
                             int32_t n_orb, const int32_t* pairs, int64_t n_pairs, uint32_t flags, double* ex_dev,
                             double* vxphi, cudaStream_t st) {
  char* ws = env.ws;
  const bool accumulate = (flags & HFX_ACCUMULATE) != 0;
#ifdef HFX_DEBUG
  k_guard_fill<<<1, 64, 0, st>>>(ws, guard_set(L));
  c->dbg_layout = L;
  c->dbg_ws = ws;
#endif
  cudaEvent_t e_stage = env.prof ? prof_mark(c, st) : nullptr;
  const void* orb = nullptr;
  hfx_status rs;
  {
    NvtxRange r("hfx stage: V clear, pair placement, FP32 copy");
    rs = stage_call(c, S, L, env, orbitals, n_orb, pairs, n_pairs, flags, vxphi, st, &orb);
  }
  if (rs != HFX_OK) return rs;
#ifdef HFX_DEBUG
  k_check_couples<<<std::max(1, std::min(S.nslots, c->sm_count * 4)), 128, 0, st>>>(
      (const int4*)(ws + L.couples), S.d_slot_couple_base, S.d_slot_blocks, S.nslots, n_orb, S.b, c->d_err);
#endif
  if (env.prof) prof_close(c, kProfStage, e_stage, st);
  if (c->prec == HFX_PREC_FP64) rs = run_passes<double>(c, S, L, env, (const double*)orb, n_orb, flags, vxphi, st);
  else rs = run_passes<float>(c, S, L, env, (const float*)orb, n_orb, flags, vxphi, st);
  if (rs != HFX_OK) return rs;
  const double scale = -0.5 * c->alpha * c->omega / ((double)c->N * (double)c->N);
  cudaEvent_t e_en = env.prof ? prof_mark(c, st) : nullptr;
  {
    NvtxRange r("hfx energy sum");
    launch_energy((const double*)(ws + L.epart), (const int4*)(ws + L.couples), (int)S.max_total_couples, eparts(c),
                  (double*)(ws + L.eblk), scale, accumulate, ex_dev, st);
  }
  if (env.prof) prof_close(c, kProfEnergy, e_en, st);
#ifdef HFX_DEBUG
  k_guard_check<<<1, 64, 0, st>>>(ws, guard_set(L), c->d_err);
#endif
  HFX_CUDA_TRY(cudaGetLastError());
  return HFX_OK;
}

extern "C" hfx_status hfx_debug_check_guards(hfx_ctx* c, void* cuda_stream) {
  g_last_error.clear();
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
#ifdef HFX_DEBUG
  if (!c->dbg_ws) return fail(HFX_ERR_INVALID_ARG, "no call has laid out the workspace yet");
  k_guard_check<<<1, 64, 0, (cudaStream_t)cuda_stream>>>(c->dbg_ws, guard_set(c->dbg_layout), c->d_err);
  HFX_CUDA_TRY(cudaGetLastError());
  return HFX_OK;
#else
  (void)cuda_stream;
  return fail(HFX_ERR_INVALID_ARG, "guard bands exist in HFX_DEBUG builds (libhfx_debug.so) only");
#endif
}

static hfx_status apply_impl(hfx_ctx* c, const void* orbitals, int32_t n_orb, const int32_t* pairs, int64_t n_pairs,
                             uint32_t flags, double* ex_dev, double* vxphi, cudaStream_t st) {
  hfx_status s = check_apply_args(c, orbitals, n_orb, pairs, n_pairs, flags, ex_dev, vxphi);
  if (s != HFX_OK) return s;
  if (n_pairs == 0) return apply_empty(c, n_orb, flags, ex_dev, vxphi, st);
  Schedule* S = nullptr;
  s = get_schedule(c, n_orb, &S);
  if (s != HFX_OK) return s;
  const Layout L = layout_of(c, *S, n_orb, two_buffers(c, *S));
  if (!c->ws || c->ws_bytes < L.total)
    return fail(HFX_ERR_OOM, "workspace too small: have %zu bytes, need %zu (hfx_workspace_bytes)", c->ws_bytes, L.total);
  const CallEnv env{(char*)c->ws, c->side, c->prof_on};
  return apply_with(c, *S, L, env, orbitals, n_orb, pairs, n_pairs, flags, ex_dev, vxphi, st);
}

extern "C" hfx_status hfx_apply(hfx_ctx* c, const void* orbitals, int32_t n_orb, const int32_t* pairs, int64_t n_pairs,
                                uint32_t flags, double* ex_dev, double* vxphi, void* cuda_stream) {
  g_last_error.clear();
  return apply_impl(c, orbitals, n_orb, pairs, n_pairs, flags, ex_dev, vxphi, (cudaStream_t)cuda_stream);
}

extern "C" hfx_status hfx_apply_sequential(hfx_ctx* const* ctxs, const hfx_apply_args* args, int32_t n,
                                           void* cuda_stream) {
  g_last_error.clear();
  if (n < 0 || (n > 0 && (!ctxs || !args))) return fail(HFX_ERR_INVALID_ARG, "bad batch arguments");
  for (int32_t k = 0; k < n; ++k) {
    const hfx_apply_args& a = args[k];
    if (a.flags & HFX_TEST_STALL) return fail(HFX_ERR_INVALID_ARG, "problem %d: HFX_TEST_STALL is for hfx_apply_batched", (int)k);
    hfx_status s = apply_impl(ctxs[k], a.orbitals, a.n_orb, a.pairs, a.n_pairs, a.flags, a.ex_dev, a.vxphi,
                              (cudaStream_t)cuda_stream);
    if (s != HFX_OK) {
      std::string m = g_last_error;
      return fail(s, "problem %d: %s", (int)k, m.c_str());
    }
  }
  return HFX_OK;
}

// The batch as one persistent launch (hfx_batch.cuh): per problem the staging launches (V cleared,
// pairs placed, FP32 copy), then one launch of k_batch_persistent over the tasks of all problems.
template <typename T>
static hfx_status batched_persistent(hfx_ctx* const* ctxs, const hfx_apply_args* args, int32_t n, cudaStream_t st) {
  hfx_ctx* lead = ctxs[0];
  std::vector<BatchProblem<T>> probs;
  std::vector<std::vector<BatchTask>> chains;
  std::vector<int> stall;
  size_t smem = 0;
  for (int32_t k = 0; k < n; ++k) {
    hfx_ctx* c = ctxs[k];
    const hfx_apply_args& a = args[k];
    if (c->pencil)
      return fail(HFX_ERR_UNSUPPORTED_GRID, "problem %d: planes exceed shared memory (use hfx_apply_sequential)", (int)k);
    if (a.n_pairs == 0) {
      hfx_status s = apply_empty(c, a.n_orb, a.flags, a.ex_dev, a.vxphi, st);
      if (s != HFX_OK) return s;
      continue;
    }
    Schedule* S = nullptr;
    hfx_status s = get_schedule(c, a.n_orb, &S);
    if (s != HFX_OK) return s;
    const Layout L = layout_of(c, *S, a.n_orb, false);
    if (!c->ws || c->ws_bytes < L.total)
      return fail(HFX_ERR_OOM, "problem %d: workspace too small: have %zu bytes, need %zu", (int)k, c->ws_bytes, L.total);
    const CallEnv env{(char*)c->ws, nullptr, false};
    const void* orb = nullptr;
    s = stage_call(c, *S, L, env, a.orbitals, a.n_orb, a.pairs, a.n_pairs, a.flags, a.vxphi, st, &orb);
    if (s != HFX_OK) return s;
    const bool eo = (a.flags & HFX_ENERGY_ONLY) != 0;
    BatchProblem<T> P;
    std::memset(&P, 0, sizeof(P));
    P.g = c->geo;
    P.orb = (const T*)orb;
    P.couples = (const int4*)(env.ws + L.couples);
    P.W = (cx<T>*)(env.ws + L.W);
    P.epart = (double*)(env.ws + L.epart);
    // the accumulate items add into V_x phi itself (FP64) or into the call's FP32 accumulator,
    // which a widening task then turns into V_x phi
    P.V = std::is_same<T, float>::value ? (T*)(env.ws + L.v32) : (T*)a.vxphi;
    P.V64 = a.vxphi;
    P.n_v = (long long)a.n_orb * c->N;
    P.ex = a.ex_dev;
    P.vtab = (const T*)c->d_vtab;
    P.tw1 = (const cx<T>*)c->d_tw[0];
    P.tw2 = (const cx<T>*)c->d_tw[1];
    P.tw3 = (const cx<T>*)c->d_tw[2];
    P.slot_couple_base = S->d_slot_couple_base;
    P.slot_blocks = S->d_slot_blocks;
    P.twct = (const cx<T>*)c->d_twct;
    P.ct_n = (std::is_same<T, float>::value && c->ct && (c->grid[0] == 48 || c->grid[0] == 64 || c->grid[0] == 72 ||
                                                        c->grid[0] == 80 || c->grid[0] == 90 || c->grid[0] == 96))
                 ? c->grid[0]
                 : 0;
    P.err = c->d_err;
    P.vscale = -c->alpha / (double)c->N;
    P.escale = -0.5 * c->alpha * c->omega / ((double)c->N * (double)c->N);
    P.n_orb = a.n_orb;
    P.bsize = S->b;
    P.grp = c->gen_grp;  // refitted below to the batch's shared-memory footprint
    P.phi_smem = c->gen_phi;
    P.cap_max = gen_cap_max(c);
    P.total_couples = (int)S->max_total_couples;
    P.accumulate = (a.flags & HFX_ACCUMULATE) ? 1 : 0;
    P.energy_only = eo ? 1 : 0;
    const int prob = (int)probs.size();
    probs.push_back(P);
    stall.push_back((a.flags & HFX_TEST_STALL) ? 1 : 0);
    std::vector<BatchTask> ch;
    auto add = [&](int kind, long long items, int a0, int a1, int cbase) {
      BatchTask t;
      std::memset(&t, 0, sizeof(t));
      t.items = (int)items;
      t.prob = prob;
      t.kind = kind;
      t.a0 = a0;
      t.a1 = a1;
      t.cbase = cbase;
      ch.push_back(t);
    };
    const int zc = zchunk(c), nzc = (c->grid[2] + zc - 1) / zc;
    for (int b = 0; b < S->nbatches; ++b) {
      const int s0 = S->batch_slot_begin[b], s1 = S->batch_slot_begin[b + 1];
      const int c0 = S->slot_couple_base[s0], c1 = S->slot_couple_base[s1];
      add(kTaskFwd, (long long)(c1 - c0) * c->grid[0], c0, c1, c0);
      add(kTaskX, (long long)(c1 - c0) * c->grid[1], c0, c1, c0);
      if (!eo) add(kTaskAcc, (long long)nzc * c->grid[0] * (s1 - s0), s0, s1, c0);
    }
    if (std::is_same<T, float>::value && !eo) add(kTaskWiden, (P.n_v + kWidenPerItem - 1) / kWidenPerItem, 0, 0, 0);
    add(kTaskEnergy, 1, 0, 0, 0);
    chains.push_back(ch);
    smem = std::max({smem, smem_fwd(c), smem_x(c)});
  }
  if (probs.empty()) return HFX_OK;
  // the accumulate tiles take at most the planes' footprint (largest couple group and orbital
  // tiles on chip that fit), so they do not lower the launch's resident blocks per SM
  {
    int p = 0;
    for (int32_t k = 0; k < n; ++k) {
      if (args[k].n_pairs == 0) continue;
      hfx_ctx* c = ctxs[k];
      BatchProblem<T>& P = probs[p++];
      if (P.energy_only) continue;
      bool fit = false;
      for (int grp : {4, 2, 1}) {
        for (int phi : {1, 0})
          if (smem_acc_cfg(c, grp, phi) <= smem) { P.grp = grp; P.phi_smem = phi; fit = true; break; }
        if (fit) break;
      }
      if (!fit) { P.grp = 1; P.phi_smem = 0; smem = std::max(smem, smem_acc_cfg(c, 1, 0)); }
    }
  }
  if (smem + 1024 > (size_t)lead->max_smem)  // the persistent kernel has 528 bytes of static shared memory
    return fail(HFX_ERR_UNSUPPORTED_GRID, "a batch tile needs %zu bytes of shared memory (limit %d)", smem, lead->max_smem);
  // interleave the chains level by level; each task waits for its predecessor in its own chain
  std::vector<BatchTask> tasks;
  std::vector<std::vector<int>> gidx(chains.size());
  size_t maxlen = 0;
  for (auto& ch : chains) maxlen = std::max(maxlen, ch.size());
  for (size_t lvl = 0; lvl < maxlen; ++lvl)
    for (size_t p = 0; p < chains.size(); ++p) {
      if (lvl >= chains[p].size()) continue;
      BatchTask t = chains[p][lvl];
      t.dep = lvl == 0 ? -1 : gidx[p][lvl - 1];
      t.extra = (lvl == 1 && stall[p]) ? 1 : 0;
      gidx[p].push_back((int)tasks.size());
      tasks.push_back(t);
    }
  long long total = 0;
  for (auto& t : tasks) { t.first = total; total += t.items; }
  const int ntasks = (int)tasks.size();
  // device tables: queue header and done counters, tasks, problems
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
  const size_t o_queue = take(sizeof(BatchQueue) + (size_t)ntasks * sizeof(int));
  const size_t o_tasks = take((size_t)ntasks * sizeof(BatchTask));
  const size_t o_probs = take(probs.size() * sizeof(BatchProblem<T>));
  if (lead->batch_bytes < off) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HFX_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(HFX_ERR_INVALID_ARG, "the first batched call of this size on its lead context must come before stream capture");
    if (lead->d_batch) { HFX_CUDA_TRY(cudaStreamSynchronize(st)); dev_free(lead->d_batch); }
    lead->d_batch = nullptr;
    lead->batch_bytes = 0;
    cudaError_t e = dev_alloc(&lead->d_batch, off);
    if (e != cudaSuccess) return fail(HFX_ERR_OOM, "cudaMalloc(%zu) for the batch tables failed: %s", off, cudaGetErrorString(e));
    lead->batch_bytes = off;
  }
  char* base = (char*)lead->d_batch;
  hfx_status s = put_table(base + o_tasks, tasks.data(), tasks.size() * sizeof(BatchTask), st);
  if (s == HFX_OK) s = put_table(base + o_probs, probs.data(), probs.size() * sizeof(BatchProblem<T>), st);
  if (s != HFX_OK) return s;
  HFX_CUDA_TRY(cudaMemsetAsync(base + o_queue, 0, sizeof(BatchQueue) + (size_t)ntasks * sizeof(int), st));
  int per_sm = 0;
  HFX_CUDA_TRY(Passes<T>::batch_occupancy(smem, &per_sm));
  const int grid = std::max(1, per_sm) * lead->sm_count;
  Passes<T>::batch(grid, smem, st, (const BatchProblem<T>*)(base + o_probs), (const BatchTask*)(base + o_tasks), ntasks,
                   total, (BatchQueue*)(base + o_queue), lead->wait_budget);
  HFX_CUDA_TRY(cudaGetLastError());
  return HFX_OK;
}

extern "C" hfx_status hfx_apply_batched(hfx_ctx* const* ctxs, const hfx_apply_args* args, int32_t n, void* cuda_stream) {
  g_last_error.clear();
  if (n < 0 || (n > 0 && (!ctxs || !args))) return fail(HFX_ERR_INVALID_ARG, "bad batch arguments");
  if (n == 0) return HFX_OK;
  for (int32_t k = 0; k < n; ++k) {
    const hfx_apply_args& a = args[k];
    hfx_status s = check_apply_args(ctxs[k], a.orbitals, a.n_orb, a.pairs, a.n_pairs, a.flags & ~HFX_TEST_STALL,
                                    a.ex_dev, a.vxphi);
    if (s != HFX_OK) {
      std::string m = g_last_error;
      return fail(s, "problem %d: %s", (int)k, m.c_str());
    }
    if (ctxs[k]->prec != ctxs[0]->prec || ctxs[k]->device != ctxs[0]->device)
      return fail(HFX_ERR_INVALID_ARG, "problem %d: every context of a batch needs the same precision and device", (int)k);
  }
  {  // one context per problem: problems of one batch run concurrently in their own workspaces
    std::vector<const hfx_ctx*> seen(ctxs, ctxs + n);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
      return fail(HFX_ERR_INVALID_ARG, "a context appears twice in the batch (each problem needs its own)");
  }
  hfx_status s = ctxs[0]->prec == HFX_PREC_FP64 ? batched_persistent<double>(ctxs, args, n, (cudaStream_t)cuda_stream)
                                                : batched_persistent<float>(ctxs, args, n, (cudaStream_t)cuda_stream);
  return s;
}

extern "C" hfx_status hfx_set_wait_budget(hfx_ctx* c, int64_t cycles) {
  g_last_error.clear();
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
  if (cycles < 0) return fail(HFX_ERR_INVALID_ARG, "cycles must be >= 0");
  c->wait_budget = cycles == 0 ? (1LL << 34) : cycles;
  return HFX_OK;
}

extern "C" hfx_status hfx_sync_status(hfx_ctx* c, void* cuda_stream) {
  g_last_error.clear();
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int h = 0;
  HFX_CUDA_TRY(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HFX_CUDA_TRY(cudaStreamSynchronize(st));
  if (h) {
    HFX_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    HFX_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (h & kErrGuard) return fail(HFX_ERR_CORRUPTION, "a guard band of the workspace was overwritten");
  if (h & kErrLayout) return fail(HFX_ERR_CORRUPTION, "a placed couple is off its canonical place in its block pair");
  if (h & kErrTimeout) return fail(HFX_ERR_TIMEOUT, "a device-side wait timed out");
  if (h & ace::kErrNotPosDef)
    return fail(HFX_ERR_NOT_POSITIVE_DEFINITE, "ACE construction: -(M + M^T)/2 is not positive definite; L and P are undefined");
  if (h & ace::kErrRankDeficient)
    return fail(HFX_ERR_RANK_DEFICIENT, "SCDM: no grid point with a positive residual norm was left to pick");
  if (h & kErrBadPair) return fail(HFX_ERR_BAD_PAIR_LIST, "pair list had entries outside 0 <= i <= j < n_orb or too many copies of a pair; they were skipped");
  return HFX_OK;
}

extern "C" hfx_status hfx_plan_stats(const hfx_ctx* c, int32_t n_orb, int64_t n_pairs, uint32_t flags, int64_t out[6]) {
  g_last_error.clear();
  if (!c || !out || n_orb <= 0 || n_pairs < 0) return fail(HFX_ERR_INVALID_ARG, "bad arguments");
  Schedule S = make_host_schedule(c, n_orb);
  const bool eo = (flags & HFX_ENERGY_ONLY) != 0;
  long long launches = 0;
  if (n_pairs > 0) {
    launches = 1 /* placement */ + 2 /* energy */ + (long long)S.nbatches * 2;
    if (!eo)
      for (int b = 0; b < S.nbatches; ++b)
        launches += (S.dense_begin[b + 1] > S.dense_begin[b]) + (S.generic_begin[b + 1] > S.generic_begin[b]) +
                    (S.diag_begin[b + 1] > S.diag_begin[b]);
    if (c->prec == HFX_PREC_FP32 && !(flags & HFX_ORBITALS_F32)) launches += 1; /* FP64 -> FP32 orbitals */
    if (c->prec == HFX_PREC_FP32 && !eo) launches += 1;                         /* FP32 V accumulator -> V */
  } else if (!(flags & HFX_ACCUMULATE)) {
    launches = 1;
  }
  out[0] = launches;
  out[1] = S.nbatches;
  out[2] = S.b;
  out[3] = S.max_batch_couples;
  out[4] = S.max_total_couples;
  long long dense = 0;
  for (int k : S.dense_slots) dense += S.slot_cap[k];
  out[5] = dense;
  return HFX_OK;
}

extern "C" hfx_status hfx_profile_enable(hfx_ctx* c, int on) {
  g_last_error.clear();
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
  c->prof_on = on != 0;
  return HFX_OK;
}

// waits for the recorded events and adds their times into the context's per-slot sums
static hfx_status prof_drain(hfx_ctx* c) {
  hfx_status st = HFX_OK;
  for (auto& pe : c->ev_pending) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(pe.second.second);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pe.second.first, pe.second.second);
    if (e != cudaSuccess && st == HFX_OK) st = fail(HFX_ERR_CUDA, "event timing failed: %s", cudaGetErrorString(e));
    c->prof_ms[pe.first] += t;
    c->prof_n[pe.first] += 1;
    c->ev_pool.push_back(pe.second.first);
    c->ev_pool.push_back(pe.second.second);
  }
  c->ev_pending.clear();
  return st;
}

static hfx_status prof_take(hfx_ctx* c, int first, int count, double* ms, int64_t* launches) {
  const hfx_status st = prof_drain(c);
  for (int k = 0; k < count; ++k) {
    ms[k] = c->prof_ms[first + k];
    launches[k] = c->prof_n[first + k];
    c->prof_ms[first + k] = 0.0;
    c->prof_n[first + k] = 0;
  }
  return st;
}

extern "C" hfx_status hfx_profile_read(hfx_ctx* c, double ms[6], int64_t launches[6]) {
  g_last_error.clear();
  if (!c || !ms || !launches) return fail(HFX_ERR_INVALID_ARG, "bad arguments");
  return prof_take(c, 0, kProfSlots, ms, launches);
}

extern "C" hfx_status hfx_ace_profile_read(hfx_ctx* c, double ms[3], int64_t launches[3]) {
  g_last_error.clear();
  if (!c || !ms || !launches) return fail(HFX_ERR_INVALID_ARG, "bad arguments");
  return prof_take(c, kProfAceGram, kProfAllSlots - kProfAceGram, ms, launches);
}

// ------------------------------------------------------------------------------------
// Allocation-free evaluation.
//
// Some callers cannot allocate device memory when they evaluate the exchange: code that runs
// inside a custom device allocator or memory-pool callback (re-entering cudaMalloc there would
// recurse or deadlock), a host whose CUDA allocations are owned by another framework that
// forbids side allocations, or a latency-critical loop where cudaMalloc's implicit device
// synchronisation is not acceptable.  hfx_apply_noalloc serves them: it runs the same kernels
// as hfx_apply, but its scratch (pair staging, per-batch transforms, energy partial sums, the
// FP32 orbital copy and the schedule tables) lives in the file-scope device array below, of
// kNoallocScratchBytes bytes, which every GPU that loads this library reserves until the
// process exits.  In host code the array's name only stands in for the symbol: its device
// address comes from cudaGetSymbolAddress, taken once per device on the first call there.
// ------------------------------------------------------------------------------------
constexpr size_t kNoallocScratchBytes = HFX_NOALLOC_SCRATCH_BYTES;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kNoallocMaxDevices = 64;
static void* g_noalloc_addr[kNoallocMaxDevices];  // device address of g_noalloc_scratch, per device
static std::mutex g_noalloc_mutex;

// device address of the scratch array on the current device (set up on first use there)
static hfx_status noalloc_scratch(void** out) {
  int dev = 0;
  HFX_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(HFX_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(HFX_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return HFX_OK;
}

extern "C" hfx_status hfx_apply_noalloc(hfx_ctx* c, const void* orbitals, int32_t n_orb, const int32_t* pairs,
                                        int64_t n_pairs, uint32_t flags, double* ex_dev, double* vxphi,
                                        void* cuda_stream) {
  g_last_error.clear();
  hfx_status s = check_apply_args(c, orbitals, n_orb, pairs, n_pairs, flags, ex_dev, vxphi);
  if (s != HFX_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (n_pairs == 0) return apply_empty(c, n_orb, flags, ex_dev, vxphi, st);

  // host schedule; its device tables go to the head of the scratch array, the workspace after
  // them.  The batches run on the caller's stream alone (one transform buffer), sized to the
  // space left: the schedule is rebuilt with that transform budget when the default one does
  // not fit, and the call is refused only when a single block pair's transforms do not.
  Schedule S = make_host_schedule(c, n_orb);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align256(std::max<size_t>(bytes, 16)); return o; };
  const size_t o_blocks = take(S.slot_blocks.size() * sizeof(int2));
  const size_t o_of_bp = take(S.slot_of_bp.size() * sizeof(int));
  const size_t o_base = take(S.slot_couple_base.size() * sizeof(int));
  const size_t o_dense = take(S.dense_slots.size() * sizeof(int));
  const size_t o_gen = take(S.generic_slots.size() * sizeof(int));
  const size_t o_diag = take(S.diag_slots.size() * sizeof(int));
  const size_t couple_bytes = (size_t)c->N * cplx_size(c);
  Layout L = layout_of(c, S, n_orb, false);
  if (off + L.total > kNoallocScratchBytes) {
    const size_t w_now = align256((size_t)S.max_batch_couples * couple_bytes);
    const size_t fixed = off + L.total - w_now;  // everything but the transform buffer
    int cap_max = 1;
    for (int k : S.slot_cap) cap_max = std::max(cap_max, k);
    const size_t room = fixed < kNoallocScratchBytes ? kNoallocScratchBytes - fixed : 0;
    if (room >= (size_t)cap_max * couple_bytes + 256) {
      build_schedule(S, n_orb, c->bsize, room - 256, couple_bytes, dense_available(c), diag_available(c));
      L = layout_of(c, S, n_orb, false);
    }
  }
  if (off + L.total > kNoallocScratchBytes)
    return fail(HFX_ERR_OOM,
                "problem needs %zu bytes of scratch; the allocation-free entry point holds %zu (use hfx_apply with a "
                "caller-owned workspace)",
                off + L.total, kNoallocScratchBytes);
  void* scratch = nullptr;
  s = noalloc_scratch(&scratch);
  if (s != HFX_OK) return s;
  char* base = (char*)scratch;
  const struct { size_t off; const void* src; size_t bytes; } tables[] = {
      {o_blocks, S.slot_blocks.data(), S.slot_blocks.size() * sizeof(int2)},
      {o_of_bp, S.slot_of_bp.data(), S.slot_of_bp.size() * sizeof(int)},
      {o_base, S.slot_couple_base.data(), S.slot_couple_base.size() * sizeof(int)},
      {o_dense, S.dense_slots.data(), S.dense_slots.size() * sizeof(int)},
      {o_gen, S.generic_slots.data(), S.generic_slots.size() * sizeof(int)},
      {o_diag, S.diag_slots.data(), S.diag_slots.size() * sizeof(int)}};
  for (const auto& t : tables) {
    s = put_table(base + t.off, t.src, t.bytes, st);
    if (s != HFX_OK) return s;
  }
  S.d_slot_blocks = (int2*)(base + o_blocks);
  S.d_slot_of_bp = (int*)(base + o_of_bp);
  S.d_slot_couple_base = (int*)(base + o_base);
  S.d_dense_slots = (int*)(base + o_dense);
  S.d_generic_slots = (int*)(base + o_gen);
  S.d_diag_slots = (int*)(base + o_diag);
  const CallEnv env{base + off, nullptr, false};
  return apply_with(c, S, L, env, orbitals, n_orb, pairs, n_pairs, flags, ex_dev, vxphi, st);
}

extern "C" hfx_status hfx_set_tuning(hfx_ctx* c, int32_t block, size_t batch_bytes, int32_t pipeline) {
  g_last_error.clear();
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
  if (block < 1 || block > 32) return fail(HFX_ERR_INVALID_ARG, "block must be in [1, 32]");
  if (batch_bytes == 0) return fail(HFX_ERR_INVALID_ARG, "batch_bytes must be > 0");
  const int old_b = c->bsize, old_grp = c->gen_grp, old_phi = c->gen_phi;
  c->bsize = block;
  if (!choose_generic(c) || smem_dense(c) + 512 > (size_t)c->max_smem) {
    c->bsize = old_b;
    c->gen_grp = old_grp;
    c->gen_phi = old_phi;
    return fail(HFX_ERR_INVALID_ARG, "block %d does not fit this grid's shared-memory tiles", (int)block);
  }
  c->transform_budget = batch_bytes;
  c->pipeline = pipeline != 0;
  // cached schedules depend on the block size and the budget: drop them (device tables freed after
  // the device is idle, since a call in flight may still read them)
  if (!c->sched.empty()) {
    cudaDeviceSynchronize();
    for (auto& kv : c->sched) {
      Schedule& S = *kv.second;
      for (void* p : {(void*)S.d_slot_blocks, (void*)S.d_slot_of_bp, (void*)S.d_slot_couple_base,
                      (void*)S.d_dense_slots, (void*)S.d_generic_slots, (void*)S.d_diag_slots})
        dev_free(p);
    }
    c->sched.clear();
  }
  return HFX_OK;
}

// ------------------------------------------------------------------------------------
// ACE operator and overlap screen (include/hfx_ace.h)
// ------------------------------------------------------------------------------------
static_assert(((ace::kErrNotPosDef | ace::kErrRankDeficient) & (kErrBadPair | kErrTimeout)) == 0 &&
                  (ace::kErrNotPosDef & ace::kErrRankDeficient) == 0,
              "device error bits overlap");

namespace {

constexpr size_t kAceAlign = 256;
size_t ace_round(size_t b) { return (b + kAceAlign - 1) / kAceAlign * kAceAlign; }

// workspace carve-up of one ACE / screen call; offsets in bytes from the workspace base
struct AceWs {
  size_t partials = 0, mat_a = 0, mat_b = 0, mat_c = 0, mat_d = 0, total = 0;
};

// build: partials | M | L | Cholesky work | L^-1
AceWs ace_ws_build(const hfx_ctx* c, int n) {
  AceWs w;
  const ace::GramPlan gp = ace::gram_plan(n, n, c->N, c->sm_count);
  const size_t sq = ace_round(((size_t)n * n + n) * sizeof(double));
  w.partials = 0;
  w.mat_a = ace_round(ace::gram_partial_bytes(gp, n, n));
  w.mat_b = w.mat_a + sq;
  w.mat_c = w.mat_b + sq;
  w.mat_d = w.mat_c + sq;
  w.total = w.mat_d + ace_round((size_t)n * ace::lmul_ldt(false, n) * sizeof(double));
  return w;
}
// apply: partials | X^T [n_orb][ldt(n_psi)]
AceWs ace_ws_apply(const hfx_ctx* c, int n_orb, int n_psi) {
  AceWs w;
  const ace::GramPlan gp = ace::gram_plan(n_psi, n_orb, c->N, c->sm_count);
  w.mat_a = ace_round(ace::gram_partial_bytes(gp, n_psi, n_orb));
  w.total = w.mat_a + ace_round((size_t)n_orb * ace::lmul_ldt(false, n_psi) * sizeof(double));
  return w;
}
// screen: partials | s | row offsets
AceWs ace_ws_screen(const hfx_ctx* c, int n) {
  AceWs w;
  const ace::GramPlan gp = ace::gram_plan(n, n, c->N, c->sm_count);
  w.mat_a = ace_round(ace::gram_partial_bytes(gp, n, n));
  w.mat_b = w.mat_a + ace_round((size_t)n * n * sizeof(double));
  w.total = w.mat_b + ace_round((size_t)(n + 1) * sizeof(int));
  return w;
}

bool misaligned8(const void* p) { return ((uintptr_t)p & 7u) != 0; }

hfx_status ace_check_ws(const void* ws, size_t have, size_t need) {
  if (!ws || have < need)
    return fail(HFX_ERR_OOM, "ACE workspace too small: have %zu bytes, need %zu (hfx_ace_workspace_bytes)", have, need);
  if (((uintptr_t)ws & (kAceAlign - 1)) != 0) return fail(HFX_ERR_INVALID_ARG, "ACE workspace must be 256-byte aligned");
  return HFX_OK;
}

}  // namespace

#define HFX_ACE_TRY(expr)                                                                           \
  do {                                                                                              \
    cudaError_t e_ = (expr);                                                                        \
    if (e_ != cudaSuccess) return fail(HFX_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

// the grid contractions of the ACE rows: tensor cores on FP32 contexts when the operands allow,
// the SIMT kernels otherwise (FP64 contexts always)
static cudaError_t ace_gram(hfx_ctx* c, bool fp32, bool absval, const double* x, long long ldx, int nx, const double* y,
                            long long ldy, int ny, long long K, const ace::GramPlan& gp, double* part, cudaStream_t st) {
  if (fp32 && c->ace_tc && ace::gram_tc_ok(x, ldx, y, ldy, K, gp))
    return ace::gram_tc(absval, x, ldx, nx, y, ldy, ny, K, gp, part, c->d_err, c->sm_count, st);
  return ace::gram(fp32, absval, x, ldx, nx, y, ldy, ny, K, gp, part, c->sm_count, st);
}
static cudaError_t ace_lmul(hfx_ctx* c, bool fp32, const void* tt, long long ldt, int m, int k, bool lower,
                            const double* y, long long ldy, long long n, bool accumulate, double* out, long long ldo,
                            cudaStream_t st) {
  if (fp32 && c->ace_tc && ace::lmul_tc_ok(tt, m, y, out))
    return ace::lmul_tc((const float*)tt, ldt, m, k, y, ldy, n, accumulate, out, ldo, c->d_err, c->sm_count, st);
  return ace::lmul(fp32, tt, ldt, m, k, lower, y, ldy, n, accumulate, out, ldo, c->sm_count, st);
}

extern "C" size_t hfx_ace_workspace_bytes(const hfx_ctx* c, int32_t n_orb, int32_t n_psi) {
  if (!c || n_orb < 1 || n_psi < 0) return 0;
  size_t need = std::max(ace_ws_build(c, n_orb).total, ace_ws_screen(c, n_orb).total);
  if (n_psi > 0) need = std::max(need, ace_ws_apply(c, n_orb, n_psi).total);
  return need;
}

extern "C" hfx_status hfx_ace_build(hfx_ctx* c, const double* orbitals, const double* w, int32_t n_orb, double* m,
                                    double* l, double* p, void* workspace, size_t workspace_bytes, void* cuda_stream) {
  g_last_error.clear();
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
  if (!orbitals || !w || !p) return fail(HFX_ERR_INVALID_ARG, "orbitals, w and p must be non-NULL");
  if (n_orb < 1) return fail(HFX_ERR_INVALID_ARG, "n_orb must be >= 1");
  if (misaligned8(orbitals) || misaligned8(w) || misaligned8(p) || misaligned8(m) || misaligned8(l))
    return fail(HFX_ERR_INVALID_ARG, "pointers must be 8-byte aligned");
  const AceWs lay = ace_ws_build(c, n_orb);
  if (hfx_status s = ace_check_ws(workspace, workspace_bytes, lay.total)) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  char* base = (char*)workspace;
  double* part = (double*)(base + lay.partials);
  double* M = m ? m : (double*)(base + lay.mat_a);
  double* L = l ? l : (double*)(base + lay.mat_b);
  double* work = (double*)(base + lay.mat_c);
  void* Linvt = base + lay.mat_d;
  const bool fp32 = c->prec == HFX_PREC_FP32;
  const long long N = c->N;
  const ace::GramPlan gp = ace::gram_plan(n_orb, n_orb, N, c->sm_count);
  // M_kl = <psi_k | W_l> = (Omega/N) sum_p psi_k(p) W_l(p)
  cudaEvent_t t0 = prof_mark(c, st);
  HFX_ACE_TRY(ace_gram(c, fp32, false, orbitals, N, n_orb, w, N, n_orb, N, gp, part, st));
  prof_close(c, kProfAceGram, t0, st);
  t0 = prof_mark(c, st);
  HFX_ACE_TRY(ace::gram_reduce(fp32, part, gp.splits, n_orb, n_orb, c->omega / (double)N, M, n_orb, nullptr, 0, st));
  // L L^T = -(M + M^T)/2, then P_rows = L^-1 W_rows (P = W L^-T)
  HFX_ACE_TRY(ace::cholesky_neg_sym(M, n_orb, n_orb, L, work, c->d_err, c->max_smem, st));
  const long long ldt = ace::lmul_ldt(fp32, n_orb);
  HFX_ACE_TRY(ace::tri_inverse(fp32, L, n_orb, Linvt, ldt, c->max_smem, st));
  prof_close(c, kProfAceSmall, t0, st);
  t0 = prof_mark(c, st);
  HFX_ACE_TRY(ace_lmul(c, fp32, Linvt, ldt, n_orb, n_orb, true, w, N, N, false, p, N, st));
  prof_close(c, kProfAceLmul, t0, st);
  return HFX_OK;
}

extern "C" hfx_status hfx_ace_apply(hfx_ctx* c, const double* p, int32_t n_orb, const double* psi, int32_t n_psi,
                                    uint32_t flags, double* out, void* workspace, size_t workspace_bytes,
                                    void* cuda_stream) {
  g_last_error.clear();
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
  if (!p || !psi || !out) return fail(HFX_ERR_INVALID_ARG, "p, psi and out must be non-NULL");
  if (n_orb < 1 || n_psi < 1) return fail(HFX_ERR_INVALID_ARG, "n_orb and n_psi must be >= 1");
  if (flags & ~HFX_ACCUMULATE) return fail(HFX_ERR_INVALID_ARG, "only HFX_ACCUMULATE is accepted in flags");
  if (misaligned8(p) || misaligned8(psi) || misaligned8(out)) return fail(HFX_ERR_INVALID_ARG, "pointers must be 8-byte aligned");
  const AceWs lay = ace_ws_apply(c, n_orb, n_psi);
  if (hfx_status s = ace_check_ws(workspace, workspace_bytes, lay.total)) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  char* base = (char*)workspace;
  double* part = (double*)(base + lay.partials);
  void* Xt = base + lay.mat_a;
  const bool fp32 = c->prec == HFX_PREC_FP32;
  const long long N = c->N;
  const ace::GramPlan gp = ace::gram_plan(n_psi, n_orb, N, c->sm_count);
  // X[i][k] = -<psi_i | P_k> (held transposed), then out_i (+)= sum_k X[i][k] P_k
  cudaEvent_t t0 = prof_mark(c, st);
  HFX_ACE_TRY(ace_gram(c, fp32, false, psi, N, n_psi, p, N, n_orb, N, gp, part, st));
  prof_close(c, kProfAceGram, t0, st);
  t0 = prof_mark(c, st);
  const long long ldt = ace::lmul_ldt(fp32, n_psi);
  HFX_ACE_TRY(ace::gram_reduce(fp32, part, gp.splits, n_psi, n_orb, -c->omega / (double)N, nullptr, 0, Xt, ldt, st));
  prof_close(c, kProfAceSmall, t0, st);
  t0 = prof_mark(c, st);
  HFX_ACE_TRY(ace_lmul(c, fp32, Xt, ldt, n_psi, n_orb, false, p, N, N, (flags & HFX_ACCUMULATE) != 0, out, N,
                        st));
  prof_close(c, kProfAceLmul, t0, st);
  return HFX_OK;
}

extern "C" hfx_status hfx_screen_pairs(hfx_ctx* c, const double* orbitals, int32_t n_orb, double cut, double* s,
                                       int32_t* pairs, int64_t* n_pairs, void* workspace, size_t workspace_bytes,
                                       void* cuda_stream) {
  g_last_error.clear();
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
  if (!orbitals || !pairs || !n_pairs) return fail(HFX_ERR_INVALID_ARG, "orbitals, pairs and n_pairs must be non-NULL");
  if (n_orb < 1) return fail(HFX_ERR_INVALID_ARG, "n_orb must be >= 1");
  if (!std::isfinite(cut) || cut < 0.0) return fail(HFX_ERR_INVALID_ARG, "cut must be finite and >= 0");
  if (misaligned8(orbitals) || misaligned8(s) || misaligned8(n_pairs) || ((uintptr_t)pairs & 3u))
    return fail(HFX_ERR_INVALID_ARG, "misaligned pointer");
  const AceWs lay = ace_ws_screen(c, n_orb);
  if (hfx_status st_ = ace_check_ws(workspace, workspace_bytes, lay.total)) return st_;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  char* base = (char*)workspace;
  double* part = (double*)(base + lay.partials);
  double* S = s ? s : (double*)(base + lay.mat_a);
  int* rowbuf = (int*)(base + lay.mat_b);
  const bool fp32 = c->prec == HFX_PREC_FP32;
  const long long N = c->N;
  const ace::GramPlan gp = ace::gram_plan(n_orb, n_orb, N, c->sm_count);
  cudaEvent_t t0 = prof_mark(c, st);
  HFX_ACE_TRY(ace_gram(c, fp32, true, orbitals, N, n_orb, orbitals, N, n_orb, N, gp, part, st));
  prof_close(c, kProfAceGram, t0, st);
  t0 = prof_mark(c, st);
  HFX_ACE_TRY(ace::gram_reduce(fp32, part, gp.splits, n_orb, n_orb, c->omega / (double)N, S, n_orb, nullptr, 0, st));
  HFX_ACE_TRY(ace::symmetrise(S, n_orb, n_orb, st));  // s_ij = s_ji exactly, whatever the summation order
  HFX_ACE_TRY(ace::screen_compact(S, n_orb, cut, pairs, n_pairs, rowbuf, st));
  prof_close(c, kProfAceSmall, t0, st);
  return HFX_OK;
}

// ------------------------------------------------------------------------------------
// SCDM localisation (include/hfx_ace.h)
// ------------------------------------------------------------------------------------
namespace {
constexpr int kScdmMaxOrb = 768;  // the pick kernel keeps 34 n values of the compute type on chip
size_t scdm_ws(const hfx_ctx* c, int n) {
  const bool fp32 = c->prec == HFX_PREC_FP32;
  return ace_round(ace::scdm_scratch_bytes(fp32, n, c->N, c->sm_count)) +
         ace_round((size_t)n * ace::lmul_ldt(fp32, n) * sizeof(double));
}
}  // namespace

extern "C" size_t hfx_scdm_workspace_bytes(const hfx_ctx* c, int32_t n_orb) {
  if (!c || n_orb < 1 || n_orb > kScdmMaxOrb || n_orb > c->N) return 0;
  return scdm_ws(c, n_orb);
}

extern "C" hfx_status hfx_scdm_localise(hfx_ctx* c, const double* orbitals, int32_t n_orb, int64_t* pivots, double* q,
                                        double* phi_loc, void* workspace, size_t workspace_bytes, void* cuda_stream) {
  g_last_error.clear();
  if (!c) return fail(HFX_ERR_INVALID_ARG, "ctx is NULL");
  if (!orbitals || !pivots || !phi_loc) return fail(HFX_ERR_INVALID_ARG, "orbitals, pivots and phi_loc must be non-NULL");
  if (n_orb < 1 || n_orb > kScdmMaxOrb || n_orb > c->N)
    return fail(HFX_ERR_INVALID_ARG, "n_orb must be in [1, min(N, %d)]", kScdmMaxOrb);
  if (misaligned8(orbitals) || misaligned8(pivots) || misaligned8(q) || misaligned8(phi_loc))
    return fail(HFX_ERR_INVALID_ARG, "pointers must be 8-byte aligned");
  const size_t need = scdm_ws(c, n_orb);
  if (hfx_status s = ace_check_ws(workspace, workspace_bytes, need)) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const bool fp32 = c->prec == HFX_PREC_FP32;
  const long long N = c->N;
  char* base = (char*)workspace;
  void* scratch = base;
  void* qt = base + ace_round(ace::scdm_scratch_bytes(fp32, n_orb, N, c->sm_count));
  const long long ldt = ace::lmul_ldt(fp32, n_orb);
  cudaEvent_t t0 = prof_mark(c, st);
  HFX_ACE_TRY(ace::scdm_pivots_q(fp32, orbitals, N, n_orb, scratch, (long long*)pivots, qt, ldt, q, c->d_err,
                                 c->sm_count, st));
  prof_close(c, kProfAceSmall, t0, st);
  t0 = prof_mark(c, st);
  HFX_ACE_TRY(ace_lmul(c, fp32, qt, ldt, n_orb, n_orb, false, orbitals, N, N, false, phi_loc, N, st));
  prof_close(c, kProfAceLmul, t0, st);
  return HFX_OK;
}

// ------------------------------------------------------------------------------------
// SIN(R) integrator updates (include/hfx_sinr.h)
// ------------------------------------------------------------------------------------
namespace {
hfx_status sinr_check(const hfx_sinr_params* p, int64_t n_dof, bool need_gamma, sinr::SinrArgs* a) {
  if (!p) return fail(HFX_ERR_INVALID_ARG, "params is NULL");
  if (n_dof < 0) return fail(HFX_ERR_INVALID_ARG, "n_dof must be >= 0");
  if (p->L < 1 || p->L > sinr::kMaxChain) return fail(HFX_ERR_INVALID_ARG, "L must be in [1, %d]", sinr::kMaxChain);
  if (!(p->kT > 0.0) || !(p->Q1 > 0.0) || !(p->Q2 > 0.0)) return fail(HFX_ERR_INVALID_ARG, "kT, Q1 and Q2 must be > 0");
  if (need_gamma && !(p->gamma > 0.0)) return fail(HFX_ERR_INVALID_ARG, "gamma must be > 0");
  a->kT = p->kT;
  a->Q1 = p->Q1;
  a->Q2 = p->Q2;
  a->gamma = p->gamma;
  a->L = p->L;
  return HFX_OK;
}
bool bad_ptr(const void* q, int64_t n_dof) { return n_dof > 0 && (!q || ((uintptr_t)q & 7u)); }
}  // namespace

extern "C" hfx_status hfx_sinr_update_n(const hfx_sinr_params* p, int64_t n_dof, double dt, int32_t n_res,
                                        int32_t n_sy, const double* mass, double* V, double* v1, double* v2,
                                        void* cuda_stream) {
  g_last_error.clear();
  sinr::SinrArgs a;
  if (hfx_status s = sinr_check(p, n_dof, false, &a)) return s;
  if (n_res < 1) return fail(HFX_ERR_INVALID_ARG, "n_res must be >= 1");
  sinr::SyWeights w{};
  if (n_sy == 1) {
    w.w[0] = 1.0;
  } else if (n_sy == 3) {
    const double w1 = 1.0 / (2.0 - std::pow(2.0, 1.0 / 3.0));
    w.w[0] = w1; w.w[1] = 1.0 - 2.0 * w1; w.w[2] = w1;
  } else if (n_sy == 5) {
    const double w1 = 1.0 / (4.0 - std::pow(4.0, 1.0 / 3.0));
    w.w[0] = w1; w.w[1] = w1; w.w[2] = 1.0 - 4.0 * w1; w.w[3] = w1; w.w[4] = w1;
  } else {
    return fail(HFX_ERR_INVALID_ARG, "n_sy must be 1, 3 or 5");
  }
  if (bad_ptr(mass, n_dof) || bad_ptr(V, n_dof) || bad_ptr(v1, n_dof) || bad_ptr(v2, n_dof))
    return fail(HFX_ERR_INVALID_ARG, "mass, V, v1 and v2 must be non-NULL 8-byte aligned device arrays");
  HFX_ACE_TRY(sinr::update_n(a, n_dof, dt, n_res, w, n_sy, mass, V, v1, v2, (cudaStream_t)cuda_stream));
  return HFX_OK;
}

extern "C" hfx_status hfx_sinr_update_v(const hfx_sinr_params* p, int64_t n_dof, double dt, const double* mass,
                                        const double* force, const double* force_extra, double* V, double* v1,
                                        void* cuda_stream) {
  g_last_error.clear();
  sinr::SinrArgs a;
  if (hfx_status s = sinr_check(p, n_dof, false, &a)) return s;
  if (bad_ptr(mass, n_dof) || bad_ptr(force, n_dof) || bad_ptr(V, n_dof) || bad_ptr(v1, n_dof) ||
      (force_extra && bad_ptr(force_extra, n_dof)))
    return fail(HFX_ERR_INVALID_ARG, "mass, force, V and v1 must be non-NULL 8-byte aligned device arrays");
  HFX_ACE_TRY(sinr::update_v(a, n_dof, dt, mass, force, force_extra, V, v1, (cudaStream_t)cuda_stream));
  return HFX_OK;
}

extern "C" hfx_status hfx_sinr_update_x(const hfx_sinr_params* p, int64_t n_dof, double dt, const double* V, double* X,
                                        double* v2, const double* R, void* cuda_stream) {
  g_last_error.clear();
  sinr::SinrArgs a;
  if (hfx_status s = sinr_check(p, n_dof, true, &a)) return s;
  if (bad_ptr(V, n_dof) || bad_ptr(X, n_dof) || bad_ptr(v2, n_dof) || bad_ptr(R, n_dof))
    return fail(HFX_ERR_INVALID_ARG, "V, X, v2 and R must be non-NULL 8-byte aligned device arrays");
  HFX_ACE_TRY(sinr::update_x(a, n_dof, dt, V, X, v2, R, (cudaStream_t)cuda_stream));
  return HFX_OK;
}
