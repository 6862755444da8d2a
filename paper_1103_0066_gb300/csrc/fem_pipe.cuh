// fem_pipe.cuh -- asynchronous data movement used by the element kernels:
// per-lane cp.async (LDGSTS) gathers into shared memory, TMA 1D bulk stores
// (cp.async.bulk shared::cta -> global) and their completion waits.
//
// The element kernels run a software pipeline per warp over their tiles
// (32 consecutive elements): the connectivity of tile t+2 is loaded into
// registers, the vertex coordinates of tile t+1 are copied asynchronously into
// lane-private shared-memory slots, and tile t is computed from its slot.  The
// gather latency (HBM for the connectivity, L2 for the coordinates) is thus
// covered by the arithmetic of the previous tile instead of by occupancy.
#pragma once
#include <cstdint>

namespace fem {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Asynchronous global -> shared copies of 4, 8 or 16 bytes (cache in L1 for
// 4/8: neighbouring elements share vertices; bypass L1 for 16-byte streams).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "n"(BYTES)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (TMA) reads of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// TMA 1D bulk copy shared::cta -> global (both 16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_store(void* gmem, const void* smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gmem), "r"(smem_u32(smem)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// Waits until at most N bulk groups of this thread still READ shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
// Waits until at most N bulk groups of this thread are incomplete (writes done).
template <int N>
__device__ __forceinline__ void bulk_wait() {
  asm volatile("cp.async.bulk.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace fem
