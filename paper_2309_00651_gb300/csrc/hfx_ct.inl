// Launchers of the compile-time-geometry FP32 passes for edge HFX_CT_N (one translation unit per
// edge, so the sizes compile in parallel).
#include "hfx_ct.cuh"
#include "hfx_ct_diag.cuh"
#include "hfx_internal.h"

namespace hfx {
namespace {

constexpr int kN = HFX_CT_N;
constexpr int kB = 8;
constexpr int kNT = ct::PlaneThreads<kN>::value;  // threads per block of the plane kernels

cudaError_t prepare(int max_dynamic_smem, size_t smem_plane, int* blocks_fwd, int* blocks_x) {
  const void* ks[] = {(const void*)ct::k_fwd_yz_ct<float, kN>, (const void*)ct::k_x_coulomb_ct<float, kN>,
                      (const void*)ct::k_y_acc_dense_ct<float, kN, kB>, (const void*)ct::k_y_acc_dense_tma<float, kN, kB>,
                      (const void*)ct::k_y_acc_diag_ct<float, kN, kB>};
  for (const void* k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dynamic_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_fwd, ct::k_fwd_yz_ct<float, kN>,
                                                                kNT, smem_plane);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_x, ct::k_x_coulomb_ct<float, kN>, kNT,
                                                       smem_plane);
}

void fwd_yz(int grid, size_t smem, cudaStream_t st, const float* orb, long long Ntot, const int4* couples, int c0,
            int c1, float2* W, const float2* tw, int prefetch) {
  ct::k_fwd_yz_ct<float, kN><<<grid, kNT, smem, st>>>(orb, Ntot, couples, c0, c1, W, tw, prefetch);
}

void x_coulomb(int grid, size_t smem, cudaStream_t st, const int4* couples, int c0, int c1, float2* W,
               const float* vtab, const float2* tw, double* epart, int energy_only, int prefetch) {
  ct::k_x_coulomb_ct<float, kN><<<grid, kNT, smem, st>>>(couples, c0, c1, W, vtab, tw, epart, energy_only,
                                                                    prefetch);
}

void y_acc_dense(dim3 grid, size_t smem, cudaStream_t st, const float* orb, long long Ntot, const int4* couples,
                 const int* slot_list, const int* slot_couple_base, const int2* slot_blocks, int c0, const float2* W,
                 const float2* tw, float* V, double vscale) {
  ct::k_y_acc_dense_ct<float, kN, kB><<<grid, ct::DenseGeo<float, kN>::NT, smem, st>>>(
      orb, Ntot, couples, slot_list, slot_couple_base, slot_blocks, c0, W, tw, V, vscale);
}

void y_acc_dense_tma(dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& tmW, const CUtensorMap& tmOrb,
                     const CUtensorMap& tmV, const int4* couples, const int* slot_list, const int* slot_couple_base,
                     const int2* slot_blocks, int c0, const float2* tw, double vscale, int* err, int stall) {
  ct::k_y_acc_dense_tma<float, kN, kB><<<grid, ct::DenseGeo<float, kN>::NT, smem, st>>>(
      tmW, tmOrb, tmV, couples, slot_list, slot_couple_base, slot_blocks, c0, tw, vscale, err, stall);
}

void y_acc_diag(dim3 grid, size_t smem, cudaStream_t st, const float* orb, long long Ntot, const int4* couples,
                const int* slot_list, const int* slot_couple_base, const int2* slot_blocks, int c0, const float2* W,
                const float2* tw, float* V, double vscale, const CUtensorMap& tmV, int tma_flush) {
  ct::k_y_acc_diag_ct<float, kN, kB><<<grid, ct::DenseGeo<float, kN>::NT, smem, st>>>(
      orb, Ntot, couples, slot_list, slot_couple_base, slot_blocks, c0, W, tw, V, vscale, tmV, tma_flush);
}

const CtFns kFns = {kN, ct::DenseGeo<float, kN>::NT, &prepare, &fwd_yz, &x_coulomb, &y_acc_dense,
                    &y_acc_dense_tma, &y_acc_diag};

}  // namespace

#define HFX_CT_JOIN2(a, b) a##b
#define HFX_CT_JOIN(a, b) HFX_CT_JOIN2(a, b)
const CtFns* HFX_CT_JOIN(ct_fns_, HFX_CT_N)() { return &kFns; }

}  // namespace hfx
