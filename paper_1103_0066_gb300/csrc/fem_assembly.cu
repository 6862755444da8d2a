// fem_assembly.cu -- global sparse assembly of the element matrices, the step
// after the element integration: A = sum_e P_e^T A_e P_e over the vertex graph
// of the mesh, as CSR for the scalar P1 forms or as BSR with d x d blocks for
// P1 elasticity (node-major unknowns v*d + c; block (c, c') of entry (v, w)
// gathers A_e[(c, i), (c', j)] with conn[e][i] = v, conn[e][j] = w).
//
// Built once per connectivity (fem_assembly_build):
//   incidences : vertex -> (element, local vertex) list in increasing element
//                order (the same counting / scan / fill / segment-sort steps as
//                the adjoint's record CSR)
//   pattern    : one warp per row v gathers the vertices of its incident
//                elements, sorts them in shared memory (bitonic), keeps the
//                distinct ones (the row's columns, increasing), and stores for
//                every incidence t and local vertex j the position of
//                conn[e][j] among them (colpos, one byte)
// Assembly (fem_assemble): one thread per row walks its incidences in
// increasing element order and adds the element's row i into the row's
// columns, accumulating in shared memory (rows of up to kFastCols columns) or
// in place in the output.  Every matrix entry is thus the sum of its element
// contributions in increasing element order: bitwise reproducible.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fem.h"
#include "fem_internal.h"

namespace fem {

namespace {

constexpr int kRowCap = 512;    // candidate columns per row (incidences x (d+1))
constexpr int kMaxCols = 255;   // distinct columns per row (one-byte positions)
constexpr int kFastCols = 32;   // rows accumulated in shared memory
constexpr int kPatWarps = 4;
constexpr int kAsmThreads = 64;

enum : int { ASM_ROW_TOO_LONG = 1, ASM_BAD_VERTEX = 2 };

__global__ void check_conn_kernel(const int32_t* __restrict__ conn, int64_t n, int64_t n_vert, int32_t* flag) {
  int bad = 0;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
    bad |= uint32_t(conn[k]) >= uint32_t(n_vert);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, ASM_BAD_VERTEX);
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

template <int NV, bool WRITE>
__global__ void __launch_bounds__(kPatWarps * 32)
    row_pattern_kernel(const int32_t* __restrict__ conn, const int32_t* __restrict__ inc_off,
                       const int32_t* __restrict__ inc, int64_t n_vert, int32_t* row_len,
                       const int32_t* __restrict__ row_ptr, int32_t* col_idx, uint8_t* colpos, int32_t* flag) {
  __shared__ uint32_t keys_s[kPatWarps][kRowCap];
  __shared__ uint32_t uniq_s[kPatWarps][kRowCap];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* key = keys_s[warp];
  uint32_t* uniq = uniq_s[warp];
  const int64_t stride = int64_t(gridDim.x) * kPatWarps;
  for (int64_t v = int64_t(blockIdx.x) * kPatWarps + warp; v < n_vert; v += stride) {
    const int32_t b = inc_off[v];
    const int cnt = (inc_off[v + 1] - b) * NV;
    if (cnt > kRowCap) {  // warp-uniform
      if (lane == 0) {
        atomicOr(flag, ASM_ROW_TOO_LONG);
        if (!WRITE) row_len[v] = 0;
      }
      continue;
    }
    const int P = next_pow2(cnt);
    int bad = 0;
    for (int c = lane; c < P; c += 32) {
      uint32_t k = 0xFFFFFFFFu;
      if (c < cnt) {
        const int32_t s = inc[b + c / NV];  // e * NV + i
        const int32_t w = conn[int64_t(s / NV) * NV + c % NV];
        if (uint32_t(w) < uint32_t(n_vert))
          k = uint32_t(w);
        else
          bad = 1;
      }
      key[c] = k;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, ASM_BAD_VERTEX);
    __syncwarp();
    for (int k2 = 2; k2 <= P; k2 <<= 1)
      for (int jj = k2 >> 1; jj > 0; jj >>= 1) {
        for (int i = lane; i < P; i += 32) {
          const int ixj = i ^ jj;
          if (ixj > i) {
            const bool up = (i & k2) == 0;
            const uint32_t x = key[i], y = key[ixj];
            if ((x > y) == up) {
              key[i] = y;
              key[ixj] = x;
            }
          }
        }
        __syncwarp();
      }
    // distinct columns, in increasing order
    int nu = 0;
    for (int r = 0; r < cnt; r += 32) {
      const int i = r + lane;
      const bool head = i < cnt && key[i] != 0xFFFFFFFFu && (i == 0 || key[i] != key[i - 1]);
      const uint32_t bal = __ballot_sync(0xffffffffu, head);
      if (head) uniq[nu + __popc(bal & ((1u << lane) - 1u))] = key[i];
      nu += __popc(bal);
    }
    __syncwarp();
    if (nu > kMaxCols) {
      if (lane == 0) {
        atomicOr(flag, ASM_ROW_TOO_LONG);
        if (!WRITE) row_len[v] = 0;
      }
      continue;
    }
    if constexpr (!WRITE) {
      if (lane == 0) row_len[v] = nu;
    } else {
      const int32_t rp = row_ptr[v];
      for (int u = lane; u < nu; u += 32) col_idx[rp + u] = int32_t(uniq[u]);
      for (int c = lane; c < cnt; c += 32) {
        const int32_t s = inc[b + c / NV];
        const uint32_t w = uint32_t(conn[int64_t(s / NV) * NV + c % NV]);
        int lo = 0, hi = nu;  // first position with uniq >= w
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (uniq[mid] < w)
            lo = mid + 1;
          else
            hi = mid;
        }
        colpos[int64_t(b) * NV + c] = uint8_t(lo);
      }
    }
    __syncwarp();  // the buffers are refilled for the next row
  }
}

// N = rows of A_e = NV * B; local unknown (c, i) is row c * NV + i.
// Incidences are taken in groups of kAsmBatch: all their loads (incidence,
// column positions, element rows) are issued before the group's additions,
// which then run in increasing incidence order.  For tets the four column
// positions are one 4-byte load and an element row of a scalar form is one
// 16-byte load.
constexpr int kAsmBatch = 4;

template <int NV, int B>
__global__ void __launch_bounds__(kAsmThreads)
    assemble_kernel(const int32_t* __restrict__ inc_off, const int32_t* __restrict__ inc,
                    const uint8_t* __restrict__ colpos, const int32_t* __restrict__ row_ptr,
                    const float* __restrict__ A, int64_t n_vert, float* __restrict__ val, int vec_A) {
  constexpr int N = NV * B, BB = B * B;
  extern __shared__ float acc_s[];  // [kAsmThreads][kFastCols * BB + 1]
  float* acc = acc_s + threadIdx.x * (kFastCols * BB + 1);
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n_vert;
       v += int64_t(gridDim.x) * blockDim.x) {
    const int32_t rp = row_ptr[v];
    const int len = row_ptr[v + 1] - rp;
    const bool fast = len <= kFastCols;
    float* dst = fast ? acc : val + int64_t(rp) * BB;
    for (int q = 0; q < len * BB; ++q) dst[q] = 0.f;
    const int32_t t1 = inc_off[v + 1];
    for (int32_t t0 = inc_off[v]; t0 < t1; t0 += kAsmBatch) {
      int32_t s[kAsmBatch];
      uint8_t pos[kAsmBatch][NV];
      float a[kAsmBatch][B][B][NV];
#pragma unroll
      for (int u = 0; u < kAsmBatch; ++u) s[u] = t0 + u < t1 ? __ldg(inc + t0 + u) : 0;
#pragma unroll
      for (int u = 0; u < kAsmBatch; ++u) {
        const int32_t t = t0 + u < t1 ? t0 + u : t0;
        if constexpr (NV == 4) {
          const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(colpos) + t);
#pragma unroll
          for (int j = 0; j < 4; ++j) pos[u][j] = uint8_t(w >> (8 * j));
        } else {
#pragma unroll
          for (int j = 0; j < NV; ++j) pos[u][j] = __ldg(colpos + int64_t(t) * NV + j);
        }
        const int i = s[u] % NV;
        const float* Ae = A + int64_t(s[u] / NV) * (N * N);
#pragma unroll
        for (int c = 0; c < B; ++c)
#pragma unroll
          for (int c2 = 0; c2 < B; ++c2) {
            const float* src = Ae + (c * NV + i) * N + c2 * NV;
            if constexpr (NV == 4) {
              if (vec_A) {  // 16-byte aligned: (c*NV + i)*N + c2*NV is a multiple of 4
                const float4 q = __ldg(reinterpret_cast<const float4*>(src));
                a[u][c][c2][0] = q.x;
                a[u][c][c2][1] = q.y;
                a[u][c][c2][2] = q.z;
                a[u][c][c2][3] = q.w;
                continue;
              }
            }
#pragma unroll
            for (int j = 0; j < NV; ++j) a[u][c][c2][j] = __ldg(src + j);
          }
      }
#pragma unroll
      for (int u = 0; u < kAsmBatch; ++u) {
        if (t0 + u >= t1) break;
#pragma unroll
        for (int c = 0; c < B; ++c)
#pragma unroll
          for (int j = 0; j < NV; ++j)
#pragma unroll
            for (int c2 = 0; c2 < B; ++c2) dst[pos[u][j] * BB + c * B + c2] += a[u][c][c2][j];
      }
    }
    if (fast) {
      float* out = val + int64_t(rp) * BB;
      for (int q = 0; q < len * BB; ++q) out[q] = acc[q];
    }
  }
}

struct AsmLayout {
  int32_t *inc_off, *inc, *row_ptr, *col_idx, *cursor, *partials, *flag;
  uint8_t* colpos;
  size_t bytes;
};

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

AsmLayout asm_layout(int dim, int64_t n_elem, int64_t n_vert, void* base) {
  const int64_t nv = dim + 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = al256(off + bytes);
    return o;
  };
  const size_t o_inc_off = take(sizeof(int32_t) * size_t(n_vert + 1));
  const size_t o_inc = take(sizeof(int32_t) * size_t(n_elem * nv));
  const size_t o_colpos = take(size_t(n_elem * nv * nv));
  const size_t o_row_ptr = take(sizeof(int32_t) * size_t(n_vert + 1));
  const size_t o_col = take(sizeof(int32_t) * size_t(n_elem * nv * nv));  // capacity: every entry distinct
  const size_t o_cursor = take(sizeof(int32_t) * size_t(n_vert + 1));
  const size_t o_part = take(sizeof(int32_t) * scan_partials_count(n_vert + 1));
  const size_t o_flag = take(sizeof(int32_t) * 4);
  AsmLayout L{};
  char* b = static_cast<char*>(base);
  L.inc_off = reinterpret_cast<int32_t*>(b + o_inc_off);
  L.inc = reinterpret_cast<int32_t*>(b + o_inc);
  L.colpos = reinterpret_cast<uint8_t*>(b + o_colpos);
  L.row_ptr = reinterpret_cast<int32_t*>(b + o_row_ptr);
  L.col_idx = reinterpret_cast<int32_t*>(b + o_col);
  L.cursor = reinterpret_cast<int32_t*>(b + o_cursor);
  L.partials = reinterpret_cast<int32_t*>(b + o_part);
  L.flag = reinterpret_cast<int32_t*>(b + o_flag);
  L.bytes = off;
  return L;
}

unsigned grid_of(int64_t n, int per_block) {
  int64_t g = (n + per_block - 1) / per_block;
  const int64_t cap = int64_t(device_sm_count()) * 64;
  if (g > cap) g = cap;
  return unsigned(g < 1 ? 1 : g);
}

template <bool WRITE>
cudaError_t launch_pattern(int dim, const int32_t* conn, int64_t n_vert, const AsmLayout& L, cudaStream_t st) {
  const unsigned g = grid_of(n_vert, kPatWarps);
  if (dim == 2)
    row_pattern_kernel<3, WRITE><<<g, kPatWarps * 32, 0, st>>>(conn, L.inc_off, L.inc, n_vert, L.cursor, L.row_ptr,
                                                                L.col_idx, L.colpos, L.flag);
  else
    row_pattern_kernel<4, WRITE><<<g, kPatWarps * 32, 0, st>>>(conn, L.inc_off, L.inc, n_vert, L.cursor, L.row_ptr,
                                                                L.col_idx, L.colpos, L.flag);
  return cudaGetLastError();
}

template <int NV, int B>
cudaError_t launch_assemble_t(const AsmLayout& L, const float* A, int64_t n_vert, float* val, cudaStream_t st) {
  const size_t smem = size_t(kAsmThreads) * (kFastCols * B * B + 1) * sizeof(float);
  auto kern = assemble_kernel<NV, B>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  const int vec_A = reinterpret_cast<uintptr_t>(A) % 16 == 0;
  kern<<<grid_of(n_vert, kAsmThreads), kAsmThreads, smem, st>>>(L.inc_off, L.inc, L.colpos, L.row_ptr, A, n_vert,
                                                                 val, vec_A);
  return cudaGetLastError();
}

}  // namespace

}  // namespace fem

// ------------------------------------------------------------------ C ABI

namespace {

fem_status asm_fail(fem_status s, const char* msg) {
  fem::set_last_error("%s", msg);
  return s;
}

// Block size of the assembled matrix for a form: 1 (scalar P1 forms), d (P1
// elasticity), 0 (not assembled: P2 unknowns include the edges).
int asm_block(int form, int dim) {
  if (form == FEM_LAPLACE_P1 || form == FEM_LAPLACE_P1_W1 || form == FEM_LAPLACE_P1_ISO) return 1;
  if (form == FEM_ELASTIC_P1) return dim;
  return 0;
}

fem_status asm_check(const fem_mesh* mesh, int form) {
  if (!mesh) return asm_fail(FEM_ERR_ARG, "mesh is NULL");
  if ((mesh->dim != 2 && mesh->dim != 3) || mesh->n_elem < 0 || mesh->n_vert < 0 || mesh->n_vert > INT32_MAX ||
      (mesh->n_elem > 0 && !mesh->conn))
    return asm_fail(FEM_ERR_ARG, "invalid mesh (dim 2/3, counts, conn)");
  if (form < FEM_LAPLACE_P1 || form > FEM_LAPLACE_P2_ISO) return asm_fail(FEM_ERR_ARG, "form out of range");
  if (asm_block(form, mesh->dim) == 0)
    return asm_fail(FEM_ERR_UNSUPPORTED, "assembly serves the P1 forms (vertex unknowns)");
  if (mesh->n_elem * (mesh->dim + 1) * (mesh->dim + 1) > INT32_MAX)
    return asm_fail(FEM_ERR_UNSUPPORTED, "n_elem * (dim + 1)^2 exceeds the int32 entry range");
  return FEM_OK;
}

}  // namespace

extern "C" {

fem_status fem_assembly_workspace_size(const fem_mesh* mesh, int32_t form, size_t* bytes) {
  fem_status s = asm_check(mesh, form);
  if (s != FEM_OK) return s;
  if (!bytes) return asm_fail(FEM_ERR_ARG, "bytes is NULL");
  *bytes = fem::asm_layout(mesh->dim, mesh->n_elem, mesh->n_vert, nullptr).bytes;
  return FEM_OK;
}

fem_status fem_assembly_build(const fem_mesh* mesh, int32_t form, void* ws, size_t ws_bytes, int64_t* nnz,
                              void* stream) {
  fem_status s = asm_check(mesh, form);
  if (s != FEM_OK) return s;
  const fem::AsmLayout L = fem::asm_layout(mesh->dim, mesh->n_elem, mesh->n_vert, ws);
  if (!ws || ws_bytes < L.bytes || reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    fem::set_last_error("assembly workspace needs %zu bytes, 256-byte aligned (got %zu)", L.bytes, ws_bytes);
    return FEM_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nv = mesh->dim + 1;
  const int64_t V = mesh->n_vert;
  cudaError_t e = cudaMemsetAsync(L.flag, 0, sizeof(int32_t) * 4, st);
  if (e == cudaSuccess && mesh->n_elem > 0) {
    fem::check_conn_kernel<<<fem::grid_of(mesh->n_elem * nv, 256), 256, 0, st>>>(mesh->conn, mesh->n_elem * nv, V,
                                                                                  L.flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = fem::launch_key_csr(mesh->conn, mesh->n_elem * nv, V, L.inc_off, L.inc, L.cursor, L.partials, st);
  if (e == cudaSuccess && V > 0) e = fem::launch_pattern<false>(mesh->dim, mesh->conn, V, L, st);
  if (e == cudaSuccess) e = fem::launch_exclusive_scan(L.cursor, V, L.partials, L.row_ptr, st);
  if (e == cudaSuccess && V > 0) e = fem::launch_pattern<true>(mesh->dim, mesh->conn, V, L, st);
  int32_t host[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host[0], L.flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host[1], L.row_ptr + V, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    fem::set_last_error("fem_assembly_build: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  if (host[0] & fem::ASM_BAD_VERTEX) return asm_fail(FEM_ERR_ARG, "a connectivity entry is outside [0, n_vert)");
  if (host[0] & fem::ASM_ROW_TOO_LONG)
    return asm_fail(FEM_ERR_UNSUPPORTED, "a vertex has more than 128 incident elements or 255 neighbours");
  if (nnz) *nnz = host[1];
  return FEM_OK;
}

fem_status fem_assembly_pattern(const fem_mesh* mesh, int32_t form, const void* ws, size_t ws_bytes,
                                const int32_t** row_ptr, const int32_t** col_idx) {
  fem_status s = asm_check(mesh, form);
  if (s != FEM_OK) return s;
  const fem::AsmLayout L = fem::asm_layout(mesh->dim, mesh->n_elem, mesh->n_vert, const_cast<void*>(ws));
  if (!ws || ws_bytes < L.bytes) return asm_fail(FEM_ERR_WORKSPACE, "assembly workspace too small");
  if (row_ptr) *row_ptr = L.row_ptr;
  if (col_idx) *col_idx = L.col_idx;
  return FEM_OK;
}

fem_status fem_assemble(const fem_mesh* mesh, int32_t form, const float* A, const void* ws, size_t ws_bytes,
                        float* values, void* stream) {
  fem_status s = asm_check(mesh, form);
  if (s != FEM_OK) return s;
  const fem::AsmLayout L = fem::asm_layout(mesh->dim, mesh->n_elem, mesh->n_vert, const_cast<void*>(ws));
  if (!ws || ws_bytes < L.bytes || reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return asm_fail(FEM_ERR_WORKSPACE, "assembly workspace too small or unaligned");
  if (mesh->n_vert == 0) return FEM_OK;
  // without elements every row is empty and nothing is written
  if (mesh->n_elem > 0 && (!values || !A)) return asm_fail(FEM_ERR_ARG, "A or values is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int B = asm_block(form, mesh->dim);
  cudaError_t e;
  if (mesh->dim == 2)
    e = B == 1 ? fem::launch_assemble_t<3, 1>(L, A, mesh->n_vert, values, st)
               : fem::launch_assemble_t<3, 2>(L, A, mesh->n_vert, values, st);
  else
    e = B == 1 ? fem::launch_assemble_t<4, 1>(L, A, mesh->n_vert, values, st)
               : fem::launch_assemble_t<4, 3>(L, A, mesh->n_vert, values, st);
  if (e != cudaSuccess) {
    fem::set_last_error("fem_assemble: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  return FEM_OK;
}

}  // extern "C"
