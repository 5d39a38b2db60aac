// Internal interface between the host library (hfx_api.cu) and the per-precision pass
// launchers (hfx_passes_f32.cu / hfx_passes_f64.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include "hfx_batch.cuh"
#include "hfx_kernels.cuh"

namespace hfx {

template <typename T>
struct Passes {
  // opt the pass kernels into `bytes` of dynamic shared memory
  static cudaError_t set_smem_limit(int bytes);
  // resident blocks per SM of the two plane kernels at the given dynamic shared memory
  static cudaError_t occupancy(size_t smem_fwd, size_t smem_x, int* blocks_fwd, int* blocks_x);
  // true when a dense accumulation kernel exists for orbital blocks of size b
  static bool has_dense(int b);

  static void fwd_yz(const Geo& g, int grid, size_t smem, cudaStream_t st, const T* orb, const int4* couples, int c0,
                     int c1, cx<T>* W, const cx<T>* tw2, const cx<T>* tw3);
  static void x_coulomb(const Geo& g, int grid, size_t smem, cudaStream_t st, const int4* couples, int c0, int c1,
                        cx<T>* W, const T* vtab, const cx<T>* tw1, const cx<T>* tw3, double* epart, int energy_only);
  // pencil form of the forward/x passes (planes too large for shared memory)
  static void fwd_z_rows(const Geo& g, int grid, size_t smem, cudaStream_t st, const T* orb, const int4* couples, int c0,
                         int c1, int rb, cx<T>* W, const cx<T>* tw3);
  static void fwd_y_cols(const Geo& g, int grid, size_t smem, cudaStream_t st, const int4* couples, int c0, int c1,
                         cx<T>* W, const cx<T>* tw2);
  static void x_cols(const Geo& g, int grid, size_t smem, cudaStream_t st, const int4* couples, int c0, int c1,
                     cx<T>* W, const T* vtab, const cx<T>* tw1, double* epart, int energy_only);
  static void inv_z_rows(const Geo& g, int grid, size_t smem, cudaStream_t st, const int4* couples, int c0, int c1,
                         int rb, cx<T>* W, const cx<T>* tw3);
  static void y_acc_dense(const Geo& g, dim3 grid, int threads, size_t smem, cudaStream_t st, int b, const T* orb,
                          const int4* couples, const int* slot_list, const int* slot_couple_base,
                          const int2* slot_blocks, int c0, const cx<T>* W, const cx<T>* tw2, T* V, double vscale);
  // one persistent launch over the task list of a batch of problems (hfx_batch.cuh)
  static void batch(int grid, size_t smem, cudaStream_t st, const BatchProblem<T>* probs, const BatchTask* tasks,
                    int ntasks, long long total_items, BatchQueue* queue, long long budget);
  static cudaError_t batch_occupancy(size_t smem, int* blocks);
  static void y_acc_generic(const Geo& g, dim3 grid, size_t smem, cudaStream_t st, const T* orb, const int4* couples,
                            const int* slot_list, const int* slot_couple_base, const int2* slot_blocks, int bsize,
                            int n_orb, int c0, const cx<T>* W, const cx<T>* tw2, T* V, double vscale, int grp,
                            int phi_smem, int cap_max);
};

}  // namespace hfx

namespace hfx {

// couple tiles per ring slot of the diagonal-block accumulate pass (hfx_ct_diag.cuh): the 18
// couples of a full B = 8 diagonal block pair in 3 slots
constexpr int kDiagCouplesPerItCt = 6;

// Compile-time-geometry FP32 passes for cubic grids of edge N (hfx_ct.cuh), one translation unit
// per N; ct_fns(N) returns NULL for an edge without one.
struct CtFns {
  int n;
  int dense_threads;                    // threads per block of the dense accumulation pass (B = 8)
  cudaError_t (*prepare)(int max_dynamic_smem, size_t smem_plane, int* blocks_fwd, int* blocks_x);
  // prefetch != 0: each block sends the data of its next work item to L2 while it works on one
  void (*fwd_yz)(int grid, size_t smem, cudaStream_t st, const float* orb, long long Ntot, const int4* couples,
                 int c0, int c1, float2* W, const float2* tw, int prefetch);
  void (*x_coulomb)(int grid, size_t smem, cudaStream_t st, const int4* couples, int c0, int c1, float2* W,
                    const float* vtab, const float2* tw, double* epart, int energy_only, int prefetch);
  void (*y_acc_dense)(dim3 grid, size_t smem, cudaStream_t st, const float* orb, long long Ntot,
                      const int4* couples, const int* slot_list, const int* slot_couple_base,
                      const int2* slot_blocks, int c0, const float2* W, const float2* tw, float* V, double vscale);
  // the same pass with its tiles moved by TMA: tmW maps the batch's transform buffer (dimensions
  // z reals, couple, y, x), tmOrb the FP32 orbitals and tmV the FP32 accumulator V (both z, y,
  // orbital, x), into which the pass adds by tensor reduce-adds; boxes as k_y_acc_dense_tma reads
  // them, shared memory smem_dense_ct + 128; stall:
  // the HFX_TEST_STALL failure-detection test (each block's first wait runs out)
  void (*y_acc_dense_tma)(dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& tmW, const CUtensorMap& tmOrb,
                          const CUtensorMap& tmV, const int4* couples, const int* slot_list,
                          const int* slot_couple_base, const int2* slot_blocks, int c0, const float2* tw,
                          double vscale, int* err, int stall);
  // full diagonal block pairs (B = 8), same arguments and threads as the dense pass; tma_flush:
  // add the block's sums into V by one tensor reduce-add through tmV (else a read-modify-write);
  // shared memory smem_diag_ct + 128
  void (*y_acc_diag)(dim3 grid, size_t smem, cudaStream_t st, const float* orb, long long Ntot,
                     const int4* couples, const int* slot_list, const int* slot_couple_base,
                     const int2* slot_blocks, int c0, const float2* W, const float2* tw, float* V, double vscale,
                     const CUtensorMap& tmV, int tma_flush);
};

// Forward plane pass with the DFT stages on the tensor cores (hfx_dft_tc.cu): cubic FP32 grids of
// edge 32, 48, 64 or 96; `dftb` is the pre-split, pre-swizzled DFT matrix of the edge
// (tc_table_bytes(n) bytes, built by the host library).
namespace dft {
bool tc_edge(int n);
size_t tc_table_bytes(int n);
cudaError_t tc_prepare(int n, int* blocks_per_sm);
void fwd_yz_tc(int n, int grid, cudaStream_t st, const float* orb, long long Ntot, const int4* couples, int c0,
               int c1, float2* W, const unsigned char* dftb, int* err);
}  // namespace dft

#define HFX_CT_SIZES(X) X(32) X(48) X(64) X(72) X(80) X(90) X(96) X(128)
#define HFX_CT_DECLARE(NN) const CtFns* ct_fns_##NN();
HFX_CT_SIZES(HFX_CT_DECLARE)
#undef HFX_CT_DECLARE

inline const CtFns* ct_fns(int n) {
  switch (n) {
#define HFX_CT_CASE(NN) \
  case NN:              \
    return ct_fns_##NN();
    HFX_CT_SIZES(HFX_CT_CASE)
#undef HFX_CT_CASE
    default:
      return nullptr;
  }
}

}  // namespace hfx
