// fem_order.cu -- a locality numbering for unstructured meshes.
//
// The forward's coordinate gather and the adjoint's tile records both profit
// from elements that share vertices sitting in the same 32-element tile, and
// from vertices numbered near one another.  A mesh in random order (a mesher's
// output, a partitioner's slice) loses both.  fem_mesh_order numbers vertices
// along the Z-order (Morton) curve of their positions and elements along the
// curve of their centroids, quantised to a grid over the mesh's bounding box;
// ties keep the old numbering.  fem_mesh_renumber applies the two orders.
//
//   bbox   : per-axis min / max of the coordinates (order-independent atomics
//            on an order-preserving integer image of the floats)
//   keys   : Morton code of each vertex's / element centroid's grid cell
//   order  : counting sort by key, each bucket in increasing old number (the
//            incidence build's launch_key_csr), so the result is deterministic
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fem.h"
#include "fem_internal.h"

namespace fem {
namespace {

constexpr int kOrderBits3 = 7;   // grid cells per axis: 2^7 on tets (2^21 keys)
constexpr int kOrderBits2 = 10;  // 2^10 on triangles (2^20 keys)
// Largest bucket the order accepts: a bucket is put in increasing old number
// by one thread's insertion sort beyond 32 entries.
constexpr int kOrderMaxBucket = 1024;

int order_bits(int dim) { return dim == 3 ? kOrderBits3 : kOrderBits2; }
int64_t order_keys(int dim) { return int64_t(1) << (order_bits(dim) * dim); }

// Monotone map of floats to signed integers (and back): min / max commute with it.
__device__ __forceinline__ int f2ord(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

__global__ void bbox_init_kernel(int* box) {
  if (threadIdx.x < 3) box[threadIdx.x] = 0x7F800000;                      // +inf: minima
  if (threadIdx.x >= 3 && threadIdx.x < 6) box[threadIdx.x] = int(0x807FFFFFu);  // -inf: maxima
}

template <int D>
__global__ void bbox_kernel(const float* __restrict__ coords, int64_t n_vert, int* box) {
  float lo[D], hi[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    lo[a] = __int_as_float(0x7F800000);
    hi[a] = -__int_as_float(0x7F800000);
  }
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n_vert; v += int64_t(gridDim.x) * blockDim.x)
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const float x = __ldg(coords + v * D + a);
      lo[a] = fminf(lo[a], x);
      hi[a] = fmaxf(hi[a], x);
    }
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int a = 0; a < D; ++a) {
      atomicMin(box + a, f2ord(lo[a]));
      atomicMax(box + 3 + a, f2ord(hi[a]));
    }
}

// Spreads the low `bits` bits of x so that bit i lands on bit D * i.
template <int D>
__device__ __forceinline__ uint32_t spread_bits(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (D * i);
  return r;
}

// Morton key of point p: cell q_a = clamp(floor((p_a - lo_a) * s_a), 0, 2^bits - 1)
// with s_a = 2^bits / (hi_a - lo_a) (0 for a flat axis); NaN lands in cell 0.
template <int D>
__device__ __forceinline__ int32_t morton_key(const float (&p)[D], const int* box, int bits) {
  const float cells = float(1 << bits);
  uint32_t key = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const float lo = ord2f(box[a]), hi = ord2f(box[3 + a]);
    const float s = hi > lo ? cells / (hi - lo) : 0.f;
    const float q = fminf(fmaxf(floorf((p[a] - lo) * s), 0.f), cells - 1.f);
    key |= spread_bits<D>(uint32_t(q), bits) << a;
  }
  return int32_t(key);
}

template <int D>
__global__ void vertex_key_kernel(const float* __restrict__ coords, int64_t n_vert, const int* box, int bits,
                                  int32_t* keys) {
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n_vert;
       v += int64_t(gridDim.x) * blockDim.x) {
    float p[D];
#pragma unroll
    for (int a = 0; a < D; ++a) p[a] = __ldg(coords + v * D + a);
    keys[v] = morton_key<D>(p, box, bits);
  }
}

// Centroid key of each element; an element with a vertex number out of range
// takes key 0 (it still gets a position).
template <int D>
__global__ void element_key_kernel(const int32_t* __restrict__ conn, const float* __restrict__ coords,
                                   int64_t n_elem, int64_t n_vert, const int* box, int bits, int32_t* keys) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n_elem;
       e += int64_t(gridDim.x) * blockDim.x) {
    float c[D];
#pragma unroll
    for (int a = 0; a < D; ++a) c[a] = 0.f;
    bool ok = true;
#pragma unroll
    for (int k = 0; k <= D; ++k) {
      const int32_t v = __ldg(conn + e * (D + 1) + k);
      if (v < 0 || int64_t(v) >= n_vert) {
        ok = false;
        continue;
      }
#pragma unroll
      for (int a = 0; a < D; ++a) c[a] += __ldg(coords + int64_t(v) * D + a);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) c[a] *= 1.f / float(D + 1);
    keys[e] = ok ? morton_key<D>(c, box, bits) : 0;
  }
}

// The largest bucket: counts per key (cnt zeroed), then their maximum into *mx.
__global__ void bucket_count_kernel(const int32_t* __restrict__ keys, int64_t n, int32_t* cnt) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    atomicAdd(cnt + keys[i], 1);
}
__global__ void bucket_max_kernel(const int32_t* __restrict__ cnt, int64_t n, int* mx) {
  int m = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = max(m, cnt[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

__global__ void invert_kernel(const int32_t* __restrict__ perm, int64_t n, int32_t* inv) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x)
    inv[perm[j]] = int32_t(j);
}

template <int D>
__global__ void renumber_kernel(const float* __restrict__ coords, const int32_t* __restrict__ conn,
                                const int32_t* __restrict__ elem_perm, const int32_t* __restrict__ vert_perm,
                                const int32_t* __restrict__ inv, int64_t n_elem, int64_t n_vert,
                                float* __restrict__ coords_out, int32_t* __restrict__ conn_out) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n_vert; j += stride) {
    const int64_t v = __ldg(vert_perm + j);
#pragma unroll
    for (int a = 0; a < D; ++a) coords_out[j * D + a] = __ldg(coords + v * D + a);
  }
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n_elem; i += stride) {
    const int64_t e = __ldg(elem_perm + i);
#pragma unroll
    for (int k = 0; k <= D; ++k) {
      const int32_t v = __ldg(conn + e * (D + 1) + k);
      conn_out[i * (D + 1) + k] = (v >= 0 && int64_t(v) < n_vert) ? __ldg(inv + v) : v;
    }
  }
}

unsigned grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  const int64_t cap = int64_t(device_sm_count()) * 16;
  if (g > cap) g = cap;
  return unsigned(g < 1 ? 1 : g);
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace: keys [max(E, V)], offsets and cursor [n_keys + 1] each, scan
// partials, the bounding box (8 ints), the inverse vertex order [V].
struct OrderLayout {
  int32_t* keys;
  int32_t* off;
  int32_t* cursor;
  int32_t* partials;
  int* box;
  int32_t* inv;
  size_t bytes;
};

// Sorts n keys into perm (new position -> old number), after checking on the
// host that no bucket exceeds kOrderMaxBucket (FEM_ERR_UNSUPPORTED).
fem_status order_by_keys(const OrderLayout& L, int64_t n, int64_t nk, int32_t* perm, cudaStream_t st);

OrderLayout order_layout(const fem_mesh* m, void* base) {
  const int64_t nk = order_keys(m->dim), nmax = m->n_elem > m->n_vert ? m->n_elem : m->n_vert;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off = al256(off + b);
    return o;
  };
  const size_t o_keys = take(sizeof(int32_t) * size_t(nmax > 0 ? nmax : 1));
  const size_t o_off = take(sizeof(int32_t) * size_t(nk + 1));
  const size_t o_cur = take(sizeof(int32_t) * size_t(nk + 1));
  const size_t o_part = take(sizeof(int32_t) * scan_partials_count(nk));
  const size_t o_box = take(sizeof(int) * 8);
  const size_t o_inv = take(sizeof(int32_t) * size_t(m->n_vert > 0 ? m->n_vert : 1));
  OrderLayout L{};
  L.bytes = off;
  if (!base) return L;
  char* b = static_cast<char*>(base);
  L.keys = reinterpret_cast<int32_t*>(b + o_keys);
  L.off = reinterpret_cast<int32_t*>(b + o_off);
  L.cursor = reinterpret_cast<int32_t*>(b + o_cur);
  L.partials = reinterpret_cast<int32_t*>(b + o_part);
  L.box = reinterpret_cast<int*>(b + o_box);
  L.inv = reinterpret_cast<int32_t*>(b + o_inv);
  return L;
}

fem_status order_by_keys(const OrderLayout& L, int64_t n, int64_t nk, int32_t* perm, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(L.cursor, 0, sizeof(int32_t) * size_t(nk), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.box + 6, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    bucket_count_kernel<<<grid_of(n), 256, 0, st>>>(L.keys, n, L.cursor);
    bucket_max_kernel<<<grid_of(nk), 256, 0, st>>>(L.cursor, nk, L.box + 6);
    e = cudaGetLastError();
  }
  int mx = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&mx, L.box + 6, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error("fem_mesh_order: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  if (mx > kOrderMaxBucket) {
    set_last_error("fem_mesh_order: %d entries share one grid cell of the order (at most %d)", mx, kOrderMaxBucket);
    return FEM_ERR_UNSUPPORTED;
  }
  e = launch_key_csr(L.keys, n, nk, L.off, perm, L.cursor, L.partials, st);
  if (e != cudaSuccess) {
    set_last_error("fem_mesh_order: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  return FEM_OK;
}

}  // namespace
}  // namespace fem

namespace {

fem_status order_fail(fem_status s, const char* msg) {
  fem::set_last_error("%s", msg);
  return s;
}

fem_status order_check(const fem_mesh* m) {
  if (!m) return order_fail(FEM_ERR_ARG, "mesh is NULL");
  if ((m->dim != 2 && m->dim != 3) || m->n_elem < 0 || m->n_vert < 0 || m->n_vert > INT32_MAX ||
      m->n_elem > INT32_MAX)
    return order_fail(FEM_ERR_ARG, "invalid mesh (dim 2/3, counts 0..INT32_MAX)");
  if ((m->n_elem > 0 && !m->conn) || (m->n_vert > 0 && !m->coords))
    return order_fail(FEM_ERR_ARG, "conn / coords is NULL");
  if (m->coord_dtype != FEM_F32) return order_fail(FEM_ERR_UNSUPPORTED, "the mesh order takes FP32 coordinates");
  return FEM_OK;
}

}  // namespace

extern "C" {

fem_status fem_mesh_order_workspace_size(const fem_mesh* mesh, size_t* bytes) {
  fem_status s = order_check(mesh);
  if (s != FEM_OK) return s;
  if (!bytes) return order_fail(FEM_ERR_ARG, "bytes is NULL");
  *bytes = fem::order_layout(mesh, nullptr).bytes;
  return FEM_OK;
}

fem_status fem_mesh_order(const fem_mesh* mesh, void* ws, size_t ws_bytes, int32_t* elem_perm, int32_t* vert_perm,
                          void* stream) {
  fem_status s = order_check(mesh);
  if (s != FEM_OK) return s;
  if ((mesh->n_elem > 0 && !elem_perm) || (mesh->n_vert > 0 && !vert_perm))
    return order_fail(FEM_ERR_ARG, "elem_perm / vert_perm is NULL");
  const fem::OrderLayout L = fem::order_layout(mesh, ws);
  if (!ws || ws_bytes < L.bytes || reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return order_fail(FEM_ERR_WORKSPACE, "workspace too small or not 256-byte aligned (fem_mesh_order_workspace_size)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int d = mesh->dim, bits = fem::order_bits(d);
  const int64_t nk = fem::order_keys(d), V = mesh->n_vert, E = mesh->n_elem;
  const float* coords = static_cast<const float*>(mesh->coords);
  fem::bbox_init_kernel<<<1, 32, 0, st>>>(L.box);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && V > 0) {
    if (d == 3)
      fem::bbox_kernel<3><<<fem::grid_of(V), 256, 0, st>>>(coords, V, L.box);
    else
      fem::bbox_kernel<2><<<fem::grid_of(V), 256, 0, st>>>(coords, V, L.box);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && V > 0) {
    if (d == 3)
      fem::vertex_key_kernel<3><<<fem::grid_of(V), 256, 0, st>>>(coords, V, L.box, bits, L.keys);
    else
      fem::vertex_key_kernel<2><<<fem::grid_of(V), 256, 0, st>>>(coords, V, L.box, bits, L.keys);
    e = cudaGetLastError();
    if (e == cudaSuccess && (s = fem::order_by_keys(L, V, nk, vert_perm, st)) != FEM_OK) return s;
  }
  if (e == cudaSuccess && E > 0) {
    if (d == 3)
      fem::element_key_kernel<3><<<fem::grid_of(E), 256, 0, st>>>(mesh->conn, coords, E, V, L.box, bits, L.keys);
    else
      fem::element_key_kernel<2><<<fem::grid_of(E), 256, 0, st>>>(mesh->conn, coords, E, V, L.box, bits, L.keys);
    e = cudaGetLastError();
    if (e == cudaSuccess && (s = fem::order_by_keys(L, E, nk, elem_perm, st)) != FEM_OK) return s;
  }
  if (e != cudaSuccess) return order_fail(FEM_ERR_CUDA, cudaGetErrorString(e));
  return FEM_OK;
}

fem_status fem_mesh_renumber(const fem_mesh* mesh, const int32_t* elem_perm, const int32_t* vert_perm, void* ws,
                             size_t ws_bytes, float* coords_out, int32_t* conn_out, void* stream) {
  fem_status s = order_check(mesh);
  if (s != FEM_OK) return s;
  if ((mesh->n_elem > 0 && (!elem_perm || !conn_out)) || (mesh->n_vert > 0 && (!vert_perm || !coords_out)))
    return order_fail(FEM_ERR_ARG, "a permutation or an output is NULL");
  const fem::OrderLayout L = fem::order_layout(mesh, ws);
  if (!ws || ws_bytes < L.bytes || reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return order_fail(FEM_ERR_WORKSPACE, "workspace too small or not 256-byte aligned (fem_mesh_order_workspace_size)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t V = mesh->n_vert, E = mesh->n_elem;
  cudaError_t e = cudaSuccess;
  if (V > 0) {
    fem::invert_kernel<<<fem::grid_of(V), 256, 0, st>>>(vert_perm, V, L.inv);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && (V > 0 || E > 0)) {
    const int64_t n = V > E ? V : E;
    const float* coords = static_cast<const float*>(mesh->coords);
    if (mesh->dim == 3)
      fem::renumber_kernel<3><<<fem::grid_of(n), 256, 0, st>>>(coords, mesh->conn, elem_perm, vert_perm, L.inv, E, V,
                                                               coords_out, conn_out);
    else
      fem::renumber_kernel<2><<<fem::grid_of(n), 256, 0, st>>>(coords, mesh->conn, elem_perm, vert_perm, L.inv, E, V,
                                                               coords_out, conn_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return order_fail(FEM_ERR_CUDA, cudaGetErrorString(e));
  return FEM_OK;
}

}  // extern "C"
