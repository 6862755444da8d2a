// fem_pipe.cuh -- asynchronous data movement used by the element kernels:
// per-lane cp.async (LDGSTS) copies into shared memory, TMA bulk and tiled
// tensor stores (cp.async.bulk[.tensor]) with their bulk-group completion, and
// the host-side encoding of the tensor maps.
//
// Tiled tensor stores serve arrays of 64-byte rows (16 FP32: the 4x4 element
// matrices of P1 tetrahedra): one 2D box of 16 x 32 values is one warp's tile,
// staged in shared memory with the 64-byte swizzle, i.e. 16-byte chunk q of
// row l at chunk q ^ ((l >> 1) & 3), so that lane l writing its own row chunk
// by chunk hits eight distinct bank groups per quarter warp.  The swizzle is a
// function of the shared address, so such buffers are 1024-byte aligned.
// (A tensor load of the adjoint's dA tiles in the same layout was measured
// slower than per-lane 16-byte cp.async, 411 against 350 us at 128^3, and is
// not used.)
#pragma once
#include <cuda.h>  // CUtensorMap and its enums (types only; the driver is reached through the runtime)
#include <cuda_runtime.h>

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

// ------------------------------------------------------------------ TMA tensor copies

// 2D tiled store of box (x, y) from shared memory (bulk group of this thread);
// rows outside the tensor are not written.  The output is streamed (L2
// evict-first), like the per-lane evict-first stores it replaces.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
  asm volatile(
      "{\n .reg .b64 pol;\n createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n"
      " cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group.L2::cache_hint [%0, {%1, %2}], [%3], pol;\n}\n"
      ::"l"(map), "r"(x), "r"(y), "r"(src)
      : "memory");
}

// Host: tensor map of a row-major [rows][16] FP32 array (64-byte rows) with
// boxes of 16 x 32 values and the 64-byte shared-memory swizzle.  false when
// the array cannot be described (base not 16-byte aligned, too many rows, or
// no driver entry point).
bool encode_rows16_map(CUtensorMap* map, const void* base, int64_t rows);

}  // namespace fem
