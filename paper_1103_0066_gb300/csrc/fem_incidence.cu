// fem_incidence.cu -- vertex -> (element, local vertex) incidence CSR and the
// deterministic segmented reduction of the adjoint's per-element vertex
// contributions into dcoords.
//
// The CSR lists, for every vertex v, the slots s = e*(d+1) + k with
// conn[e][k] == v, sorted by s (i.e. by element, then local vertex).  The
// reduction adds scratch[s][0..d) over each segment in that order, so the
// result is bitwise reproducible run to run.  Built once per connectivity:
// count (atomics) -> exclusive scan -> fill (atomics) -> per-segment sort.
#include <cuda_runtime.h>

#include "fem_internal.h"

namespace fem {

namespace {

constexpr int kScanBlock = 1024;

__global__ void zero_i32(int32_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = 0;
}

__global__ void zero_f32(float* p, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = 0.f;
}

__global__ void count_kernel(const int32_t* conn, int64_t n_slots, int64_t n_vert, int32_t* cnt) {
  for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s < n_slots;
       s += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = conn[s];
    if (v >= 0 && v < n_vert) atomicAdd(cnt + v, 1);
  }
}

// Block-wide exclusive scan of one value per thread (blockDim.x == kScanBlock).
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t x) {
  __shared__ int32_t warp_tot[kScanBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int32_t t = warp_tot[lane];  // kScanBlock / 32 == 32 warps
    int32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    warp_tot[lane] = ti - t;
  }
  __syncthreads();
  const int32_t r = incl - x + warp_tot[warp];
  __syncthreads();  // warp_tot is reused by the next call
  return r;
}

__global__ void scan_partials_kernel(const int32_t* cnt, int64_t n, int32_t* partials) {
  __shared__ int32_t red[kScanBlock / 32];
  const int64_t i = blockIdx.x * int64_t(kScanBlock) + threadIdx.x;
  int32_t x = i < n ? cnt[i] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    int32_t y = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = y;
  }
}

// Exclusive scan of the block partials in place (one CTA, sequential over chunks).
__global__ void scan_top_kernel(int32_t* partials, int64_t nb) {
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += kScanBlock) {
    const int64_t i = base + threadIdx.x;
    const int32_t orig = i < nb ? partials[i] : 0;
    const int32_t x = block_exclusive_scan(orig);
    const int32_t c = carry;
    if (i < nb) partials[i] = x + c;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry = c + x + orig;
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[nb] = carry;
}

__global__ void scan_apply_kernel(const int32_t* cnt, int64_t n, const int32_t* partials, int64_t nb,
                                  int32_t* offsets) {
  const int64_t i = blockIdx.x * int64_t(kScanBlock) + threadIdx.x;
  const int32_t x = block_exclusive_scan(i < n ? cnt[i] : 0);
  if (i < n) offsets[i] = x + partials[blockIdx.x];
  if (blockIdx.x == 0 && threadIdx.x == 0) offsets[n] = partials[nb];
}

__global__ void fill_kernel(const int32_t* conn, int64_t n_slots, int64_t n_vert, const int32_t* offsets,
                            int32_t* cursor, int32_t* incidence) {
  for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s < n_slots;
       s += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = conn[s];
    if (v >= 0 && v < n_vert) incidence[offsets[v] + atomicAdd(cursor + v, 1)] = int32_t(s);
  }
}

// Sorts each vertex's segment (insertion sort: segments hold a few tens of slots).
__global__ void sort_segments_kernel(const int32_t* offsets, int64_t n_vert, int32_t* incidence) {
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n_vert;
       v += int64_t(gridDim.x) * blockDim.x) {
    const int32_t b = offsets[v], en = offsets[v + 1];
    for (int32_t i = b + 1; i < en; ++i) {
      const int32_t key = incidence[i];
      int32_t j = i - 1;
      while (j >= b && incidence[j] > key) {
        incidence[j + 1] = incidence[j];
        --j;
      }
      incidence[j + 1] = key;
    }
  }
}

template <int D>
__global__ void vertex_reduce_kernel(const int32_t* __restrict__ offsets, const int32_t* __restrict__ incidence,
                                     const float* __restrict__ scratch, int64_t n_vert,
                                     float* __restrict__ dcoords) {
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n_vert;
       v += int64_t(gridDim.x) * blockDim.x) {
    const int32_t b = __ldg(offsets + v), en = __ldg(offsets + v + 1);
    float s[D];
#pragma unroll
    for (int a = 0; a < D; ++a) s[a] = 0.f;
    for (int32_t i = b; i < en; ++i) {
      const int64_t slot = __ldg(incidence + i);
#pragma unroll
      for (int a = 0; a < D; ++a) s[a] += __ldcs(scratch + slot * D + a);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) dcoords[v * D + a] = s[a];
  }
}

unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  const int64_t cap = int64_t(device_sm_count()) * 32;
  if (g > cap) g = cap;
  return unsigned(g < 1 ? 1 : g);
}

}  // namespace

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t bwd_workspace_layout(int dim, int64_t n_elem, int64_t n_vert, bool with_scratch, void* base,
                            BwdWorkspace* ws) {
  const int64_t nv = dim + 1;
  const int64_t nb = (n_vert + kScanBlock - 1) / kScanBlock;
  size_t off = 0;
  const size_t o_offsets = off;
  off = align256(off + sizeof(int32_t) * size_t(n_vert + 1));
  const size_t o_inc = off;
  off = align256(off + sizeof(int32_t) * size_t(n_elem * nv));
  const size_t o_cursor = off;
  off = align256(off + sizeof(int32_t) * size_t(n_vert));
  const size_t o_part = off;
  off = align256(off + sizeof(int32_t) * size_t(nb + 1));
  const size_t o_scr = off;
  if (with_scratch) off = align256(off + sizeof(float) * size_t(n_elem * nv * dim));
  if (ws) {
    char* b = static_cast<char*>(base);
    ws->offsets = reinterpret_cast<int32_t*>(b + o_offsets);
    ws->incidence = reinterpret_cast<int32_t*>(b + o_inc);
    ws->cursor = reinterpret_cast<int32_t*>(b + o_cursor);
    ws->partials = reinterpret_cast<int32_t*>(b + o_part);
    ws->scratch = with_scratch ? reinterpret_cast<float*>(b + o_scr) : nullptr;
    ws->bytes = off;
  }
  return off;
}

cudaError_t launch_incidence_build(int dim, const int32_t* conn, int64_t n_elem, int64_t n_vert,
                                   const BwdWorkspace& ws, cudaStream_t stream) {
  const int64_t n_slots = n_elem * (dim + 1);
  const int64_t nb = (n_vert + kScanBlock - 1) / kScanBlock;
  zero_i32<<<grid_for(n_vert, 256), 256, 0, stream>>>(ws.cursor, n_vert);
  count_kernel<<<grid_for(n_slots, 256), 256, 0, stream>>>(conn, n_slots, n_vert, ws.cursor);
  if (nb > 0) scan_partials_kernel<<<unsigned(nb), kScanBlock, 0, stream>>>(ws.cursor, n_vert, ws.partials);
  scan_top_kernel<<<1, kScanBlock, 0, stream>>>(ws.partials, nb);
  scan_apply_kernel<<<unsigned(nb > 0 ? nb : 1), kScanBlock, 0, stream>>>(ws.cursor, n_vert, ws.partials, nb,
                                                                          ws.offsets);
  zero_i32<<<grid_for(n_vert, 256), 256, 0, stream>>>(ws.cursor, n_vert);
  fill_kernel<<<grid_for(n_slots, 256), 256, 0, stream>>>(conn, n_slots, n_vert, ws.offsets, ws.cursor,
                                                           ws.incidence);
  sort_segments_kernel<<<grid_for(n_vert, 128), 128, 0, stream>>>(ws.offsets, n_vert, ws.incidence);
  return cudaGetLastError();
}

cudaError_t launch_zero_f32(float* p, int64_t n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  zero_f32<<<grid_for(n, 256), 256, 0, stream>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_vertex_reduce(int dim, const BwdWorkspace& ws, int64_t n_vert, float* dcoords,
                                 cudaStream_t stream) {
  if (n_vert == 0) return cudaSuccess;
  const int block = 256;
  int64_t g = (n_vert + block - 1) / block;
  if (dim == 2)
    vertex_reduce_kernel<2><<<unsigned(g), block, 0, stream>>>(ws.offsets, ws.incidence, ws.scratch, n_vert,
                                                               dcoords);
  else
    vertex_reduce_kernel<3><<<unsigned(g), block, 0, stream>>>(ws.offsets, ws.incidence, ws.scratch, n_vert,
                                                               dcoords);
  return cudaGetLastError();
}

}  // namespace fem
