// Launchers of the three passes for one real type `Real` (included by hfx_passes_f32.cu and
// hfx_passes_f64.cu, so the two precisions compile in parallel).
#include "hfx_internal.h"

namespace hfx {

template <>
cudaError_t Passes<Real>::set_smem_limit(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_fwd_yz<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_x_coulomb<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_y_inv_acc<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <>
cudaError_t Passes<Real>::occupancy(size_t smem_fwd, size_t smem_x, int* blocks_fwd, int* blocks_x) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_fwd, k_fwd_yz<Real>, kThreadsPlane, smem_fwd);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_x, k_x_coulomb<Real>, kThreadsPlane, smem_x);
}

template <>
void Passes<Real>::fwd_yz(const Geo& g, int grid, size_t smem, cudaStream_t st, const Real* orb,
                          const int4* couples, const int* batch_begin, int batch, cx<Real>* W,
                          const cx<Real>* tw2, const cx<Real>* tw3) {
  k_fwd_yz<Real><<<grid, kThreadsPlane, smem, st>>>(g, orb, couples, batch_begin, batch, W, tw2, tw3);
}

template <>
void Passes<Real>::x_coulomb(const Geo& g, int grid, size_t smem, cudaStream_t st, const int* batch_begin,
                             int batch, cx<Real>* W, const Real* vtab, const cx<Real>* tw1,
                             const cx<Real>* tw3, double* epart, int energy_only) {
  k_x_coulomb<Real><<<grid, kThreadsPlane, smem, st>>>(g, batch_begin, batch, W, vtab, tw1, tw3, epart,
                                                       energy_only);
}

template <>
void Passes<Real>::y_inv_acc(const Geo& g, dim3 grid, size_t smem, cudaStream_t st, const Real* orb,
                             const int4* couples, const int* batch_begin, int batch, const int* slot_begin,
                             const int2* slot_blocks, int slot0, int bsize, int n_orb, const cx<Real>* W,
                             const cx<Real>* tw2, double* V, double vscale) {
  k_y_inv_acc<Real><<<grid, kThreadsAcc, smem, st>>>(g, orb, couples, batch_begin, batch, slot_begin,
                                                     slot_blocks, slot0, bsize, n_orb, W, tw2, V, vscale);
}

template struct Passes<Real>;

}  // namespace hfx
