// Launchers of the passes for one real type `Real` (included by hfx_passes_f32.cu and
// hfx_passes_f64.cu, so the two precisions compile in parallel).
#include "hfx_internal.h"

namespace hfx {

template <>
cudaError_t Passes<Real>::set_smem_limit(int bytes) {
  const void* ks[] = {(const void*)k_fwd_yz<Real>,           (const void*)k_x_coulomb<Real>,
                      (const void*)k_y_acc_dense<Real, 4, 2>, (const void*)k_y_acc_dense<Real, 4, 4>,
                      (const void*)k_y_acc_dense<Real, 8, 2>, (const void*)k_y_acc_dense<Real, 8, 4>,
                      (const void*)k_y_acc_generic<Real>,      (const void*)k_fwd_z_rows<Real>,
                      (const void*)k_fwd_y_cols<Real>,         (const void*)k_x_cols<Real>,
                      (const void*)k_inv_z_rows<Real>,         (const void*)k_batch_persistent<Real>};
  for (const void* k : ks) {
    // `bytes` leaves 512 bytes of the per-block limit for static shared memory; a kernel with
    // more static shared memory gets correspondingly less dynamic memory
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    const int lim = fa.sharedSizeBytes > 512 ? bytes + 512 - (int)fa.sharedSizeBytes : bytes;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <>
cudaError_t Passes<Real>::occupancy(size_t smem_fwd, size_t smem_x, int* blocks_fwd, int* blocks_x) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_fwd, k_fwd_yz<Real>, kThreadsPlane, smem_fwd);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_x, k_x_coulomb<Real>, kThreadsPlane, smem_x);
}

template <>
bool Passes<Real>::has_dense(int b) { return b == 4 || b == 8; }

template <>
void Passes<Real>::fwd_yz(const Geo& g, int grid, size_t smem, cudaStream_t st, const Real* orb, const int4* couples,
                          int c0, int c1, cx<Real>* W, const cx<Real>* tw2, const cx<Real>* tw3) {
  k_fwd_yz<Real><<<grid, kThreadsPlane, smem, st>>>(g, orb, couples, c0, c1, W, tw2, tw3);
}

template <>
void Passes<Real>::x_coulomb(const Geo& g, int grid, size_t smem, cudaStream_t st, const int4* couples, int c0, int c1,
                             cx<Real>* W, const Real* vtab, const cx<Real>* tw1, const cx<Real>* tw3, double* epart,
                             int energy_only) {
  k_x_coulomb<Real><<<grid, kThreadsPlane, smem, st>>>(g, couples, c0, c1, W, vtab, tw1, tw3, epart, energy_only);
}

template <>
void Passes<Real>::y_acc_dense(const Geo& g, dim3 grid, int threads, size_t smem, cudaStream_t st, int b,
                               const Real* orb, const int4* couples, const int* slot_list, const int* slot_couple_base,
                               const int2* slot_blocks, int c0, const cx<Real>* W, const cx<Real>* tw2, Real* V,
                               double vscale) {
  // points per thread so that one block of at most kDenseMaxThreads threads covers the tile
  const int pts = g.n2 * ZChunk<Real>::value;
  const bool np4 = pts > 2 * DenseBounds<2>::threads;
#define HFX_DENSE(BB, NPP)                                                                                      \
  k_y_acc_dense<Real, BB, NPP><<<grid, threads, smem, st>>>(g, orb, couples, slot_list, slot_couple_base, slot_blocks, \
                                                            c0, W, tw2, V, vscale)
  if (b == 8) { if (np4) HFX_DENSE(8, 4); else HFX_DENSE(8, 2); }
  else { if (np4) HFX_DENSE(4, 4); else HFX_DENSE(4, 2); }
#undef HFX_DENSE
}

template <>
void Passes<Real>::y_acc_generic(const Geo& g, dim3 grid, size_t smem, cudaStream_t st, const Real* orb,
                                 const int4* couples, const int* slot_list, const int* slot_couple_base,
                                 const int2* slot_blocks, int bsize, int n_orb, int c0, const cx<Real>* W,
                                 const cx<Real>* tw2, Real* V, double vscale, int grp, int phi_smem, int cap_max) {
  k_y_acc_generic<Real><<<grid, kThreadsGen, smem, st>>>(g, orb, couples, slot_list, slot_couple_base, slot_blocks,
                                                        bsize, n_orb, c0, W, tw2, V, vscale, grp, phi_smem, cap_max);
}

template <>
void Passes<Real>::fwd_z_rows(const Geo& g, int grid, size_t smem, cudaStream_t st, const Real* orb, const int4* couples,
                              int c0, int c1, int rb, cx<Real>* W, const cx<Real>* tw3) {
  k_fwd_z_rows<Real><<<grid, kThreadsPencil, smem, st>>>(g, orb, couples, c0, c1, rb, W, tw3);
}

template <>
void Passes<Real>::fwd_y_cols(const Geo& g, int grid, size_t smem, cudaStream_t st, const int4* couples, int c0, int c1,
                              cx<Real>* W, const cx<Real>* tw2) {
  k_fwd_y_cols<Real><<<grid, kThreadsPencil, smem, st>>>(g, couples, c0, c1, W, tw2);
}

template <>
void Passes<Real>::x_cols(const Geo& g, int grid, size_t smem, cudaStream_t st, const int4* couples, int c0, int c1,
                          cx<Real>* W, const Real* vtab, const cx<Real>* tw1, double* epart, int energy_only) {
  k_x_cols<Real><<<grid, kThreadsPencil, smem, st>>>(g, couples, c0, c1, W, vtab, tw1, epart, energy_only);
}

template <>
void Passes<Real>::inv_z_rows(const Geo& g, int grid, size_t smem, cudaStream_t st, const int4* couples, int c0, int c1,
                              int rb, cx<Real>* W, const cx<Real>* tw3) {
  k_inv_z_rows<Real><<<grid, kThreadsPencil, smem, st>>>(g, couples, c0, c1, rb, W, tw3);
}

template <>
void Passes<Real>::batch(int grid, size_t smem, cudaStream_t st, const BatchProblem<Real>* probs, const BatchTask* tasks,
                         int ntasks, long long total_items, BatchQueue* queue, long long budget) {
  k_batch_persistent<Real><<<grid, kThreadsBatch, smem, st>>>(probs, tasks, ntasks, total_items, queue, budget);
}

template <>
cudaError_t Passes<Real>::batch_occupancy(size_t smem, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_batch_persistent<Real>, kThreadsBatch, smem);
}

template struct Passes<Real>;

}  // namespace hfx
