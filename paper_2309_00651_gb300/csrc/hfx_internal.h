// Internal interface between the host library (hfx_api.cu) and the per-precision pass
// launchers (hfx_passes_f32.cu / hfx_passes_f64.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "hfx_kernels.cuh"

namespace hfx {

template <typename T>
struct Passes {
  // opt the three pass kernels into `bytes` of dynamic shared memory
  static cudaError_t set_smem_limit(int bytes);
  // resident blocks per SM of the two plane kernels at the given dynamic shared memory
  static cudaError_t occupancy(size_t smem_fwd, size_t smem_x, int* blocks_fwd, int* blocks_x);

  static void fwd_yz(const Geo& g, int grid, size_t smem, cudaStream_t st, const T* orb,
                     const int4* couples, const int* batch_begin, int batch, cx<T>* W,
                     const cx<T>* tw2, const cx<T>* tw3);
  static void x_coulomb(const Geo& g, int grid, size_t smem, cudaStream_t st, const int* batch_begin,
                        int batch, cx<T>* W, const T* vtab, const cx<T>* tw1, const cx<T>* tw3,
                        double* epart, int energy_only);
  static void y_inv_acc(const Geo& g, dim3 grid, size_t smem, cudaStream_t st, const T* orb,
                        const int4* couples, const int* batch_begin, int batch, const int* slot_begin,
                        const int2* slot_blocks, int slot0, int bsize, int n_orb, const cx<T>* W,
                        const cx<T>* tw2, double* V, double vscale);
};

}  // namespace hfx
