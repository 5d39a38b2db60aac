// Tensor-memory-accelerator (TMA) tile loads for the sm_100 family, written as inline PTX: one
// thread copies a whole box of a tensor -- described by a tensor map that the host encodes with
// cuTensorMapEncodeTiled -- from global into shared memory, and the copy completes its byte count
// on an mbarrier that the consuming threads wait on.  The box lands densely in shared memory,
// dimension 0 fastest; parts of the box outside the tensor read as zero.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "tc_sm100.cuh"

namespace hfx {
namespace tma {

// one arrival on `mbar` that also announces `bytes` of transactions still to come
__device__ __forceinline__ void expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(mbar)), "r"(bytes)
               : "memory");
}

// the 4-D box of `map` whose first element has coordinates (c0 innermost, c1, c2, c3) -> shared
// memory at `dst` (128-byte aligned); completes the box's bytes on `mbar`
__device__ __forceinline__ void load4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                       uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(tc::smem_u32(mbar))
      : "memory");
}

// the same box sent to L2 only (no shared memory, no mbarrier): a prefetch of data read later
__device__ __forceinline__ void prefetch4d(const CUtensorMap* map, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3)
               : "memory");
}

// element-wise add of the FP32 box at `src` (shared memory, 128-byte aligned, laid out as a load of
// the same box would land) into the tensor at coordinates (c0 .. c3), performed at L2; elements
// outside the tensor are skipped.  Completes in this thread's bulk group.
__device__ __forceinline__ void reduce_add4d(const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                             const void* src) {
  asm volatile("cp.reduce.async.bulk.tensor.4d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(tc::smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// until the shared-memory sources of this thread's committed bulk operations have been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

}  // namespace tma
}  // namespace hfx
