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
// Scalar forms, tile records (built once per connectivity, after the pattern):
//   per 32-element tile (one warp): the tile's distinct vertices ("runs", R_t
//   of them) and every slot's run index (one byte); the distinct (row run,
//   column run) cells the tile touches, each one RECORD (records numbered in
//   tile order), the entry -> records CSR (eoff, rec_list) and its inverse,
//   every record's slot in entry order (rec_dest) -- the tile / record scheme
//   of the adjoint's reduction, keyed by matrix entry.
// Assembly of the scalar forms (fem_assemble):
//   1. one warp per tile reads its element matrices coalesced into shared
//      memory and adds them, element by element, into a dense R_t x R_t tile
//      matrix (an element's cells are distinct, so a step has no conflicts);
//      each cell is the sum of its contributions in element order.  Each cell
//      is written as a record to its slot in entry order (tiles with R_t above
//      kTileRuns take an exact per-record scan of the tile instead);
//   2. one thread per entry sums its records, which lie side by side in tile
//      order, so the pass reads them contiguously.
// Every entry is therefore a fixed-order sum, bitwise reproducible.
// P1 elasticity (d x d blocks) takes the row kernel: one thread per row walks
// its incidences in increasing element order and adds the element's rows into
// the row's columns, accumulating in shared memory (rows of up to kFastCols
// columns) or in place in the output.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fem.h"
#include "fem_internal.h"
#include "fem_pipe.cuh"

namespace fem {

namespace {

constexpr int kRowCap = 512;    // candidate columns per row (incidences x (d+1))
constexpr int kMaxCols = 255;   // distinct columns per row (one-byte positions)
constexpr int kFastCols = 32;   // rows accumulated in shared memory
constexpr int kPatWarps = 4;
constexpr int kAsmThreads = 64;
constexpr int kTileRuns = 36;  // dense tile matrix side (distinct vertices of a 32-element tile)
// Row stride of a tile's cells, cell = row run * stride + column run: at least
// kCellStride, so that the 16 cells of an element (4 runs x 4 runs) spread over
// the shared-memory banks (a stride of the run count itself, near 32 on a
// cell-major mesh, puts them in a few banks); the run count when it is larger.
// Cells ordered by value are in (row run, column run) order either way.
constexpr int kCellStride = 34;
__host__ __device__ __forceinline__ int cell_stride(int nr) { return nr > kCellStride ? nr : kCellStride; }
constexpr int kTileWarps = 1;  // warps per CTA of the tile pass (no CTA-wide barrier: finest sharing of shared memory)
constexpr int kTileCap = 128;  // slots of a 32-element tile (tets: 4 per element)
constexpr int kCellCap = 512;  // contributions of a 32-element tile (tets: 16 per element)
constexpr int kDestRegs = 8;   // record slots a lane of the tile pass holds in registers (tiles of up to 256 records)
constexpr int kHalvesDisjoint = 0x100;  // tile_runs flag: elements 0-15 and 16-31 share no cell

enum : int { ASM_ROW_TOO_LONG = 1, ASM_BAD_VERTEX = 2, ASM_REPEATED_VERTEX = 4 };

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
                    const float* __restrict__ A, int64_t n_vert, float* __restrict__ val, int vec_A,
                    const int32_t* __restrict__ n_rows_dev) {
  constexpr int N = NV * B, BB = B * B;
  extern __shared__ float acc_s[];  // [kAsmThreads][kFastCols * BB + 1]
  float* acc = acc_s + threadIdx.x * (kFastCols * BB + 1);
  if (n_rows_dev) n_vert = *n_rows_dev;  // rows known only on the device (P2 unknowns)
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

// ------------------------------------------------------------------ tile records (scalar forms)

// Sorts n_pow2 keys in shared memory (bitonic, one warp).
template <class K>
__device__ __forceinline__ void warp_bitonic(K* key, int P, int lane) {
  for (int k2 = 2; k2 <= P; k2 <<= 1)
    for (int jj = k2 >> 1; jj > 0; jj >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int ixj = i ^ jj;
        if (ixj > i) {
          const bool up = (i & k2) == 0;
          const K x = key[i], y = key[ixj];
          if ((x > y) == up) {
            key[i] = y;
            key[ixj] = x;
          }
        }
      }
      __syncwarp();
    }
}

// One warp per 32-element tile.  PASS 1 counts the tile's cells (records);
// PASS 2 writes the slot run indices, R_t, each record's cell (r_v * R_t + r_w)
// and its matrix entry (CSR position of (v, w)).
template <int NV, bool WRITE>
__global__ void __launch_bounds__(kPatWarps * 32)
    tile_cells_kernel(const int32_t* __restrict__ conn, int64_t n_elem, const int32_t* __restrict__ row_ptr,
                      const int32_t* __restrict__ col_idx, int32_t* tile_nrec, const int32_t* __restrict__ tile_rec,
                      uint32_t* run_word, uint16_t* tile_runs, uint16_t* rec_cell, int32_t* rec_entry, int32_t* flag) {
  __shared__ uint64_t skey_s[kPatWarps][kTileCap];
  __shared__ uint32_t ckey_s[kPatWarps][kCellCap];
  __shared__ int32_t runv_s[kPatWarps][kTileCap];
  __shared__ uint8_t runi_s[kPatWarps][kTileCap];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* skey = skey_s[warp];
  uint32_t* ckey = ckey_s[warp];
  int32_t* runv = runv_s[warp];
  uint8_t* runi = runi_s[warp];
  constexpr int NS = 32 * NV;                  // slots of a full tile
  constexpr int PS = NS <= 64 ? 64 : 128;      // power of two >= NS (and >= 32)
  constexpr int NC = 32 * NV * NV;             // contributions of a full tile
  constexpr int PC = NC <= 256 ? 256 : 512;
  const int64_t ntiles = (n_elem + 31) / 32;
  const int64_t stride = int64_t(gridDim.x) * kPatWarps;
  for (int64_t t = int64_t(blockIdx.x) * kPatWarps + warp; t < ntiles; t += stride) {
    const int64_t e0 = t * 32;
    const int ne = int(n_elem - e0 < 32 ? n_elem - e0 : 32);
    const int ns = ne * NV;
    // 1. slots sorted by (vertex, slot): runs and run index per slot
    for (int i = lane; i < PS; i += 32) {
      uint64_t k = ~0ull;
      if (i < ns) k = (uint64_t(uint32_t(conn[e0 * NV + i])) << 16) | uint64_t(i);
      skey[i] = k;
    }
    __syncwarp();
    warp_bitonic(skey, PS, lane);
    int nr = 0;
    for (int r = 0; r < ns; r += 32) {
      const int i = r + lane;
      const bool head = i < ns && (i == 0 || (skey[i] >> 16) != (skey[i - 1] >> 16));
      const uint32_t bal = __ballot_sync(0xffffffffu, head);
      const uint32_t upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);  // lanes <= this one
      const int run = nr + __popc(bal & upto) - 1;  // heads up to this position, minus one
      if (head) runv[run] = int32_t(skey[i] >> 16);
      if (i < ns) runi[int(skey[i] & 0xFFFF)] = uint8_t(run);
      nr += __popc(bal);
    }
    __syncwarp();
    // 2. cells of the tile's contributions, in (row run, column run) order; the
    //    key keeps the element (low 6 bits) to tell whether the two half-tiles
    //    (elements 0-15, 16-31) share a cell
    const int ncell = ne * NV * NV;
    int rep = 0;
    for (int c = lane; c < PC; c += 32) {
      uint32_t k = 0xFFFFFFFFu;
      if (c < ncell) {
        const int el = c / (NV * NV), ij = c % (NV * NV), i = ij / NV, j = ij % NV;
        const int ri = runi[el * NV + i], rj = runi[el * NV + j];
        if (i != j && ri == rj) rep = 1;  // an element repeats a vertex
        k = (uint32_t(ri * cell_stride(nr) + rj) << 6) | uint32_t(el);
      }
      ckey[c] = k;
    }
    if (__any_sync(0xffffffffu, rep) && lane == 0) atomicOr(flag, ASM_REPEATED_VERTEX);
    __syncwarp();
    warp_bitonic(ckey, PC, lane);
    int nu = 0, shared = 0;
    for (int r = 0; r < ncell; r += 32) {
      const int i = r + lane;
      const bool head = i < ncell && (i == 0 || (ckey[i] >> 6) != (ckey[i - 1] >> 6));
      // within a cell the elements ascend: the halves meet where a lower-half
      // element is followed by an upper-half one
      if (i + 1 < ncell && (ckey[i] >> 6) == (ckey[i + 1] >> 6) && (ckey[i] & 63u) < 16u && (ckey[i + 1] & 63u) >= 16u)
        shared = 1;
      const uint32_t bal = __ballot_sync(0xffffffffu, head);
      if constexpr (WRITE) {
        if (head) {
          const int32_t rec = tile_rec[t] + nu + __popc(bal & ((1u << lane) - 1u));
          const uint32_t cell = ckey[i] >> 6;
          const int32_t v = runv[cell / cell_stride(nr)], w = runv[cell % cell_stride(nr)];
          int lo = row_ptr[v], hi = row_ptr[v + 1];  // position of w in row v
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (col_idx[mid] < w)
              lo = mid + 1;
            else
              hi = mid;
          }
          rec_cell[t * kCellCap + (rec - tile_rec[t])] = uint16_t(cell);  // the tile's 512-entry slot
          rec_entry[rec] = lo;
        }
      }
      nu += __popc(bal);
    }
    shared = __any_sync(0xffffffffu, shared);
    if constexpr (!WRITE) {
      if (lane == 0) tile_nrec[t] = nu;
    } else {
      uint32_t wd = 0;
      if (lane < ne) {
#pragma unroll
        for (int k = 0; k < NV; ++k) wd |= uint32_t(runi[lane * NV + k]) << (8 * k);
      }
      run_word[t * 32 + lane] = wd;
      if (lane == 0) tile_runs[t] = uint16_t(nr | (shared ? 0 : kHalvesDisjoint));
    }
    __syncwarp();  // the buffers are refilled for the next tile
  }
}

// Step 1 of the scalar assembly: one warp per tile, pipelined over its tiles.
// The next tile's element matrices arrive by 16-byte cp.async into the other
// half of a double-buffered stage while this tile is summed.  Every lane
// first writes its element's cell indices (cells[l][ij], shared memory); the
// dense tile is zero at the start of every tile (zeroed once, and each record
// cell zeroed again as it is read out); then the contributions are added
// element by element (each element's cells are distinct) -- two elements per
// step, l and l + 16, when the tile's halves share no cell -- and the records
// are read out in tile order.
template <int NV>
struct TilePlan {
  static constexpr int NN = NV * NV;
  static constexpr int SST = NV == 4 ? 16 : NN;                      // stage row (floats)
  static constexpr size_t stage = size_t(32) * SST * 4;              // one tile of A
  static constexpr size_t rcell = size_t(kCellCap) * 2;              // one tile's record cells
  static constexpr size_t cells = size_t(32) * 17 * 4;               // u32 [32][17]: odd stride, no conflicts
  static constexpr size_t dense = size_t(kTileRuns) * kTileRuns * 4;
  static constexpr size_t per_warp = 2 * stage + 2 * rcell + cells + dense;
  static constexpr size_t smem = kTileWarps * per_warp;
};

template <int NV>
__device__ __forceinline__ void copy_tile_A(const float* A, int64_t n_elem, int64_t t, int lane, float* dst,
                                            int vec) {
  constexpr int NN = NV * NV;
  const int64_t e0 = t * 32;
  if (e0 >= n_elem) return;
  const int ne = int(n_elem - e0 < 32 ? n_elem - e0 : 32);
  const float* src = A + e0 * NN;
  if constexpr (NV == 4) {
    if (vec) {  // 64-byte rows of a 16-byte-aligned A: contiguous 16-byte chunks
      for (int q = lane; q < ne * 4; q += 32) cp_async<16>(dst + 4 * q, src + 4 * q);
      return;
    }
  }
  for (int q = lane; q < ne * NN; q += 32) cp_async<4>(dst + q, src + q);
}

// The first rn record cells of tile t (16-byte chunks of its 512-entry slot).
__device__ __forceinline__ void copy_tile_cells(const uint16_t* rec_cell, int64_t t, int rn, int lane, uint16_t* dst) {
  const uint16_t* src = rec_cell + t * kCellCap;
  for (int q = lane; q < (rn + 7) / 8; q += 32) cp_async<16>(dst + 8 * q, src + 8 * q);
}

template <int NV>
__global__ void __launch_bounds__(kTileWarps * 32)
    tile_assemble_kernel(const float* __restrict__ A, int64_t n_elem, const uint32_t* __restrict__ run_word,
                         const uint16_t* __restrict__ tile_runs, const int32_t* __restrict__ tile_rec,
                         const uint16_t* __restrict__ rec_cell, const int32_t* __restrict__ rec_dest,
                         float* __restrict__ records, int vec) {
  using TP = TilePlan<NV>;
  constexpr int NN = TP::NN, SST = TP::SST;
  extern __shared__ __align__(128) unsigned char tsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wb = tsm + size_t(warp) * TP::per_warp;
  float* stage = reinterpret_cast<float*>(wb);                                   // [2][32][SST]
  uint16_t* rcs = reinterpret_cast<uint16_t*>(wb + 2 * TP::stage);               // [2][512]
  uint32_t* cells = reinterpret_cast<uint32_t*>(wb + 2 * TP::stage + 2 * TP::rcell);
  float* dense = reinterpret_cast<float*>(wb + 2 * TP::stage + 2 * TP::rcell + TP::cells);
  const int64_t ntiles = (n_elem + 31) / 32;
  const int64_t S = int64_t(gridDim.x) * kTileWarps;
  int64_t t = int64_t(blockIdx.x) * kTileWarps + warp;
  if (t >= ntiles) return;
  // pipeline: tile metadata two tiles ahead, A / record cells / runs one tile ahead
  auto meta = [&](int64_t tt, int& tr, int32_t& rb, int32_t& rn) {
    tr = 0, rb = 0, rn = 0;
    if (tt < ntiles) {
      tr = __ldg(tile_runs + tt);
      rb = __ldg(tile_rec + tt);
      rn = __ldg(tile_rec + tt + 1) - rb;
    }
  };
  int trc, trn, tr2;
  int32_t rbc, rnc, rbn, rnn, rb2, rn2;
  meta(t, trc, rbc, rnc);
  meta(t + S, trn, rbn, rnn);
  copy_tile_A<NV>(A, n_elem, t, lane, stage, vec);
  copy_tile_cells(rec_cell, t, rnc, lane, rcs);
  cp_async_commit();
  uint32_t rwc = __ldg(run_word + t * 32 + lane);
  // the entry-order slots of a tile's first 32 * kDestRegs records, one tile ahead
  auto dests = [&](int32_t rb, int32_t rn, int32_t(&d)[kDestRegs]) {
#pragma unroll
    for (int q = 0; q < kDestRegs; ++q) d[q] = lane + 32 * q < rn ? __ldg(rec_dest + rb + lane + 32 * q) : 0;
  };
  int32_t dc[kDestRegs], dn[kDestRegs];
  dests(rbc, rnc, dc);
  for (int i = lane; i < kTileRuns * kTileRuns; i += 32) dense[i] = 0.f;
  for (int it = 0; t < ntiles; ++it, t += S) {
    const int sc = it & 1;
    const int64_t tn = t + S;
    meta(tn + S, tr2, rb2, rn2);
    uint32_t rwn = 0;
    if (tn < ntiles) {
      copy_tile_A<NV>(A, n_elem, tn, lane, stage + (sc ^ 1) * 32 * SST, vec);
      copy_tile_cells(rec_cell, tn, rnn, lane, rcs + (sc ^ 1) * kCellCap);
      rwn = __ldg(run_word + tn * 32 + lane);
    }
    dests(rbn, rnn, dn);  // rnn = 0 past the last tile
    cp_async_commit();
    const int64_t e0 = t * 32;
    const int ne = int(n_elem - e0 < 32 ? n_elem - e0 : 32);
    const int nr = trc & 0xFF;
    const bool halves = (trc & kHalvesDisjoint) && ne == 32;
    const float* st = stage + sc * 32 * SST;
    const uint16_t* rc = rcs + sc * kCellCap;
    const uint32_t ps = uint32_t(cell_stride(nr));
    if (nr <= kTileRuns && lane < ne) {
#pragma unroll
      for (int ij = 0; ij < NN; ++ij)
        cells[lane * 17 + ij] = ((rwc >> (8 * (ij / NV))) & 0xFFu) * ps + ((rwc >> (8 * (ij % NV))) & 0xFFu);
    }
    cp_async_wait<1>();
    __syncwarp();  // this tile's A and record cells (copied by every lane) and the cell indices are in place
    if (nr <= kTileRuns) {
      if (halves) {
        const int h = lane >> 4, ij = lane & 15;
        for (int l0 = 0; l0 < 16; ++l0) {
          const int l = l0 + 16 * h;
          if (ij < NN) dense[cells[l * 17 + ij]] += st[l * SST + ij];
          __syncwarp();
        }
      } else {
        for (int l = 0; l < ne; ++l) {  // element order
          if (lane < NN) dense[cells[l * 17 + lane]] += st[l * SST + lane];
          __syncwarp();
        }
      }
#pragma unroll
      for (int q = 0; q < kDestRegs; ++q)
        if (lane + 32 * q < rnc) {
          const int c = rc[lane + 32 * q];
          records[dc[q]] = dense[c];
          dense[c] = 0.f;
        }
      for (int r = lane + 32 * kDestRegs; r < rnc; r += 32) {
        const int c = rc[r];
        records[__ldg(rec_dest + rbc + r)] = dense[c];
        dense[c] = 0.f;
      }
    } else {
      // more distinct vertices than the dense tile holds: scan the tile per record
      for (int r0 = 0; r0 < rnc; r0 += 32) {  // warp-uniform, so the shuffles see every lane
        const int r = r0 + lane;
        const bool live = r < rnc;
        const int cell = live ? int(rc[r]) : -1;
        float acc = 0.f;
        for (int l = 0; l < ne; ++l) {
          const uint32_t w = __shfl_sync(0xffffffffu, rwc, l);
#pragma unroll
          for (int ij = 0; ij < NN; ++ij)
            if (int((w >> (8 * (ij / NV))) & 0xFFu) * int(ps) + int((w >> (8 * (ij % NV))) & 0xFFu) == cell)
              acc += st[l * SST + ij];
        }
        if (live) records[__ldg(rec_dest + rbc + r)] = acc;
      }
    }
    __syncwarp();  // the stage, record cells, cells and dense tile are refilled
    trc = trn, rbc = rbn, rnc = rnn, rwc = rwn;
#pragma unroll
    for (int q = 0; q < kDestRegs; ++q) dc[q] = dn[q];
    trn = tr2, rbn = rb2, rnn = rn2;
  }
  cp_async_wait<0>();
}

// Step 2: val[k] = sum of the records of entry k, records[eoff[k] .. eoff[k+1])
// in tile order: the tile pass wrote every record to its slot in entry order,
// so neighbouring threads read neighbouring runs.  A thread sums two entries
// at a time (k and k + S), four records of each loaded before they are added,
// while the bounds of its next two entries load.
__global__ void entry_reduce_kernel(const int32_t* __restrict__ eoff, const int32_t* __restrict__ nnz_ptr,
                                    const float* __restrict__ records, float* __restrict__ val) {
  const int64_t nnz = *nnz_ptr;  // row_ptr[n_vert]
  const int64_t S = int64_t(gridDim.x) * blockDim.x;
  auto bounds = [&](int64_t k, int32_t& b, int32_t& e) {
    b = 0, e = 0;
    if (k < nnz) b = __ldg(eoff + k), e = __ldg(eoff + k + 1);
  };
  int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  int32_t b0n, e0n, b1n, e1n;
  bounds(k, b0n, e0n);
  bounds(k + S, b1n, e1n);
  for (; k < nnz; k += 2 * S) {
    const int32_t b0 = b0n, e0 = e0n, b1 = b1n, e1 = e1n;
    bounds(k + 2 * S, b0n, e0n);
    bounds(k + 3 * S, b1n, e1n);
    const int32_t n0 = e0 - b0, n1 = e1 - b1;
    float acc0 = 0.f, acc1 = 0.f;
    for (int32_t m0 = 0; m0 < n0 || m0 < n1; m0 += 4) {
      float x0[4], x1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x0[u] = m0 + u < n0 ? __ldg(records + b0 + m0 + u) : 0.f;
        x1[u] = m0 + u < n1 ? __ldg(records + b1 + m0 + u) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (m0 + u < n0) acc0 += x0[u];
        if (m0 + u < n1) acc1 += x1[u];
      }
    }
    val[k] = acc0;
    if (k + S < nnz) val[k + S] = acc1;
  }
}

struct AsmLayout {
  int32_t *inc_off, *inc, *row_ptr, *col_idx, *cursor, *partials, *flag;
  uint8_t* colpos;
  // tile records (scalar forms)
  uint32_t* run_word;
  uint16_t* tile_runs;
  int32_t *tile_rec, *rec_entry, *rec_list, *eoff, *cursor2, *partials2;
  int32_t* rec_dest;  // the records' entry-order slots; shares rec_entry's storage, which the build no longer needs
  uint16_t* rec_cell;
  float* records;
  int64_t n_tiles, rec_cap;
  size_t bytes;
};

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

AsmLayout asm_layout(int dim, int64_t n_elem, int64_t n_vert, void* base) {
  const int64_t nv = dim + 1;
  const int64_t T = (n_elem + 31) / 32;
  const int64_t cap = n_elem * nv * nv;  // contributions: bounds the entries and the records
  const int64_t big = (T > cap ? T : cap) + 1;
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
  const size_t o_col = take(sizeof(int32_t) * size_t(cap));  // capacity: every entry distinct
  const size_t o_cursor = take(sizeof(int32_t) * size_t(n_vert + 1));
  const size_t o_part = take(sizeof(int32_t) * scan_partials_count(n_vert + 1));
  const size_t o_flag = take(sizeof(int32_t) * 4);
  const size_t o_run = take(sizeof(uint32_t) * size_t(T * 32));
  const size_t o_truns = take(sizeof(uint16_t) * size_t(T));
  const size_t o_trec = take(sizeof(int32_t) * size_t(T + 1));
  const size_t o_cell = take(sizeof(uint16_t) * size_t(T * kCellCap));  // 512 cells per tile, tile-strided
  const size_t o_rentry = take(sizeof(int32_t) * size_t(cap));
  const size_t o_rlist = take(sizeof(int32_t) * size_t(cap));
  const size_t o_eoff = take(sizeof(int32_t) * size_t(cap + 1));
  const size_t o_records = take(sizeof(float) * size_t(cap));
  const size_t o_cursor2 = take(sizeof(int32_t) * size_t(big));
  const size_t o_part2 = take(sizeof(int32_t) * scan_partials_count(big));
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
  L.run_word = reinterpret_cast<uint32_t*>(b + o_run);
  L.tile_runs = reinterpret_cast<uint16_t*>(b + o_truns);
  L.tile_rec = reinterpret_cast<int32_t*>(b + o_trec);
  L.rec_cell = reinterpret_cast<uint16_t*>(b + o_cell);
  L.rec_entry = reinterpret_cast<int32_t*>(b + o_rentry);
  L.rec_list = reinterpret_cast<int32_t*>(b + o_rlist);
  L.rec_dest = L.rec_entry;
  L.eoff = reinterpret_cast<int32_t*>(b + o_eoff);
  L.records = reinterpret_cast<float*>(b + o_records);
  L.cursor2 = reinterpret_cast<int32_t*>(b + o_cursor2);
  L.partials2 = reinterpret_cast<int32_t*>(b + o_part2);
  L.n_tiles = T;
  L.rec_cap = cap;
  L.bytes = off;
  return L;
}

// rec_dest[rec_list[p]] = p for the *n_rec records listed
__global__ void invert_list_kernel(const int32_t* __restrict__ rec_list, const int32_t* __restrict__ n_rec,
                                   int32_t* __restrict__ rec_dest) {
  const int64_t n = *n_rec;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x)
    rec_dest[rec_list[p]] = int32_t(p);
}

__global__ void fill_neg_kernel(int32_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = -1;
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

template <bool WRITE>
cudaError_t launch_tile_cells(int dim, const int32_t* conn, int64_t n_elem, const AsmLayout& L, cudaStream_t st) {
  const unsigned g = grid_of(L.n_tiles, kPatWarps);
  if (dim == 2)
    tile_cells_kernel<3, WRITE><<<g, kPatWarps * 32, 0, st>>>(conn, n_elem, L.row_ptr, L.col_idx, L.cursor2,
                                                               L.tile_rec, L.run_word, L.tile_runs, L.rec_cell,
                                                               L.rec_entry, L.flag);
  else
    tile_cells_kernel<4, WRITE><<<g, kPatWarps * 32, 0, st>>>(conn, n_elem, L.row_ptr, L.col_idx, L.cursor2,
                                                               L.tile_rec, L.run_word, L.tile_runs, L.rec_cell,
                                                               L.rec_entry, L.flag);
  return cudaGetLastError();
}

template <int NV>
cudaError_t launch_tile_assemble_t(const AsmLayout& L, const float* A, int64_t n_elem, int64_t n_vert, float* val,
                                   cudaStream_t st) {
  const size_t smem = TilePlan<NV>::smem;
  auto kern = tile_assemble_kernel<NV>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  kern<<<pipeline_grid(reinterpret_cast<const void*>(kern), kTileWarps, smem, n_elem, 0), kTileWarps * 32, smem, st>>>(
      A, n_elem, L.run_word, L.tile_runs, L.tile_rec, L.rec_cell, L.rec_dest, L.records,
      int(reinterpret_cast<uintptr_t>(A) % 16 == 0));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  entry_reduce_kernel<<<grid_of(L.rec_cap, 256), 256, 0, st>>>(L.eoff, L.row_ptr + n_vert, L.records, val);
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
                                                                 val, vec_A, nullptr);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ P2 unknowns (vertices, then edges)
//
// The P2 basis has one unknown per vertex and one per edge.  The edges are
// numbered from the vertex graph's pattern: row v's columns are sorted and
// contain v, so the edges with lower vertex v are its columns above v, and
// edge (v, w) gets V + eoff[v] + (position of w in row v) - (position of v) - 1
// with eoff the exclusive scan of those counts: the edges in increasing
// (lower vertex, higher vertex) order.  An element's unknowns (its vertices,
// then its edges in the local P2 order) form the connectivity of a second
// pattern, over the V + n_edges unknowns, which the row kernel assembles.

// Arrays of the P2 assembly: the vertex graph's incidences and pattern
// (positions per incidence), the edge offsets, the element unknowns, and the
// unknowns' incidences and pattern.
struct AsmP2Layout {
  AsmLayout g1;  // vertex graph (inc_off, inc, colpos, row_ptr, col_idx, cursor, partials, flag)
  AsmLayout g2;  // unknowns (same fields over up to V + E * n_edges rows)
  int32_t* eoff;   // [V + 1]
  int32_t* dofs;   // [E][n]
  int32_t* n_rows; // one word: V + n_edges
  int64_t rows_cap;
  size_t bytes;
};

AsmP2Layout asm_p2_layout(int dim, int64_t n_elem, int64_t n_vert, void* base) {
  const int64_t nv = dim + 1, ne = dim * (dim + 1) / 2, n = nv + ne;
  const int64_t rows_cap = n_vert + n_elem * ne;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = al256(off + bytes);
    return o;
  };
  char* b = static_cast<char*>(base);
  auto graph = [&](int64_t rows, int64_t per_elem, AsmLayout& G) {
    const int64_t cap = n_elem * per_elem * per_elem;
    const size_t o_inc_off = take(sizeof(int32_t) * size_t(rows + 1));
    const size_t o_inc = take(sizeof(int32_t) * size_t(n_elem * per_elem));
    const size_t o_colpos = take(size_t(cap));
    const size_t o_row_ptr = take(sizeof(int32_t) * size_t(rows + 1));
    const size_t o_col = take(sizeof(int32_t) * size_t(cap));
    const size_t o_cursor = take(sizeof(int32_t) * size_t(rows + 1));
    const size_t o_part = take(sizeof(int32_t) * scan_partials_count(rows + 1));
    G.inc_off = reinterpret_cast<int32_t*>(b + o_inc_off);
    G.inc = reinterpret_cast<int32_t*>(b + o_inc);
    G.colpos = reinterpret_cast<uint8_t*>(b + o_colpos);
    G.row_ptr = reinterpret_cast<int32_t*>(b + o_row_ptr);
    G.col_idx = reinterpret_cast<int32_t*>(b + o_col);
    G.cursor = reinterpret_cast<int32_t*>(b + o_cursor);
    G.partials = reinterpret_cast<int32_t*>(b + o_part);
  };
  AsmP2Layout L{};
  graph(n_vert, nv, L.g1);
  graph(rows_cap, n, L.g2);
  const size_t o_eoff = take(sizeof(int32_t) * size_t(n_vert + 1));
  const size_t o_dofs = take(sizeof(int32_t) * size_t(n_elem * n));
  const size_t o_flag = take(sizeof(int32_t) * 8);
  L.eoff = reinterpret_cast<int32_t*>(b + o_eoff);
  L.dofs = reinterpret_cast<int32_t*>(b + o_dofs);
  L.g1.flag = reinterpret_cast<int32_t*>(b + o_flag);
  L.g2.flag = L.g1.flag;
  L.n_rows = L.g1.flag + 4;
  L.rows_cap = rows_cap;
  L.bytes = off;
  return L;
}

// An element listing a vertex twice has no edge between the two: flagged.
template <int NV>
__global__ void check_repeat_kernel(const int32_t* __restrict__ conn, int64_t n_elem, int32_t* flag) {
  int bad = 0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n_elem; e += int64_t(gridDim.x) * blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
      for (int j = i + 1; j < NV; ++j) bad |= conn[e * NV + i] == conn[e * NV + j];
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, ASM_REPEATED_VERTEX);
}

// Position of v in its own (sorted) row, or -1 for an empty row.
__device__ __forceinline__ int diag_pos(const int32_t* __restrict__ col, int32_t b, int32_t e, int32_t v) {
  int lo = b, hi = e;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (col[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < e && col[lo] == v) ? lo - b : -1;
}

// n_up[v] = the columns of row v above v: the edges whose lower vertex is v.
__global__ void edge_count_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                  int64_t n_vert, int32_t* n_up) {
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n_vert; v += int64_t(gridDim.x) * blockDim.x) {
    const int32_t b = row_ptr[v], e = row_ptr[v + 1];
    const int d = diag_pos(col, b, e, int32_t(v));
    n_up[v] = d < 0 ? 0 : (e - b) - d - 1;
  }
}

// Element unknowns in the local P2 order: each incidence (e, i) of row v
// writes dofs[e][i] = v and, for every vertex w = conn[e][j] > v, the number
// of edge (v, w) into the slot of local edge (min(i, j), max(i, j)): every
// element edge is written once, by its lower vertex.
template <int NV>
__global__ void edge_dof_kernel(const int32_t* __restrict__ conn, const int32_t* __restrict__ inc_off,
                                const int32_t* __restrict__ inc, const uint8_t* __restrict__ colpos,
                                const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ eoff, int64_t n_vert, int32_t* __restrict__ dofs) {
  constexpr int NB = NV + NV * (NV - 1) / 2;
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n_vert; v += int64_t(gridDim.x) * blockDim.x) {
    const int d = diag_pos(col, row_ptr[v], row_ptr[v + 1], int32_t(v));
    const int64_t base = n_vert + eoff[v] - d - 1;
    for (int32_t t = inc_off[v]; t < inc_off[v + 1]; ++t) {
      const int32_t sl = inc[t];
      const int64_t el = sl / NV;
      const int i = sl % NV;
      dofs[el * NB + i] = int32_t(v);
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        if (j == i || conn[el * NV + j] <= v) continue;
        const int a = i < j ? i : j, c = i < j ? j : i;
        const int q = a * (2 * NV - a - 1) / 2 + (c - a - 1);
        dofs[el * NB + NV + q] = int32_t(base + colpos[int64_t(t) * NV + j]);
      }
    }
  }
}

__global__ void store_rows_kernel(const int32_t* __restrict__ eoff, int64_t n_vert, int32_t* n_rows) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_rows = int32_t(n_vert + eoff[n_vert]);
}

// The P2 build: vertex-graph pattern, edge numbers, element unknowns, then
// the unknowns' pattern.  Returns the unknown count and the flags (host).
template <int NV>
cudaError_t launch_p2_build(const int32_t* conn, int64_t n_elem, int64_t n_vert, const AsmP2Layout& L,
                            int32_t* rows_host, int32_t* flag_host, int32_t* nnz_host, cudaStream_t st) {
  constexpr int NB = NV + NV * (NV - 1) / 2;
  const AsmLayout& G1 = L.g1;
  const AsmLayout& G2 = L.g2;
  cudaError_t e = cudaMemsetAsync(G1.flag, 0, sizeof(int32_t) * 8, st);
  if (e == cudaSuccess && n_elem > 0) {
    check_conn_kernel<<<grid_of(n_elem * NV, 256), 256, 0, st>>>(conn, n_elem * NV, n_vert, G1.flag);
    check_repeat_kernel<NV><<<grid_of(n_elem, 256), 256, 0, st>>>(conn, n_elem, G1.flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(flag_host, G1.flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess || *flag_host) return e;
  const unsigned gv = grid_of(n_vert, kPatWarps);
  if (e == cudaSuccess) e = launch_key_csr(conn, n_elem * NV, n_vert, G1.inc_off, G1.inc, G1.cursor, G1.partials, st);
  if (e == cudaSuccess && n_vert > 0) {
    row_pattern_kernel<NV, false><<<gv, kPatWarps * 32, 0, st>>>(conn, G1.inc_off, G1.inc, n_vert, G1.cursor,
                                                                  G1.row_ptr, G1.col_idx, G1.colpos, G1.flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_exclusive_scan(G1.cursor, n_vert, G1.partials, G1.row_ptr, st);
  if (e == cudaSuccess && n_vert > 0) {
    row_pattern_kernel<NV, true><<<gv, kPatWarps * 32, 0, st>>>(conn, G1.inc_off, G1.inc, n_vert, G1.cursor,
                                                                 G1.row_ptr, G1.col_idx, G1.colpos, G1.flag);
    edge_count_kernel<<<grid_of(n_vert, 256), 256, 0, st>>>(G1.row_ptr, G1.col_idx, n_vert, G1.cursor);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_exclusive_scan(G1.cursor, n_vert, G1.partials, L.eoff, st);
  if (e == cudaSuccess && n_vert > 0) {
    edge_dof_kernel<NV><<<grid_of(n_vert, 256), 256, 0, st>>>(conn, G1.inc_off, G1.inc, G1.colpos, G1.row_ptr,
                                                               G1.col_idx, L.eoff, n_vert, L.dofs);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    store_rows_kernel<<<1, 32, 0, st>>>(L.eoff, n_vert, L.n_rows);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(rows_host, L.n_rows, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(flag_host, G1.flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess || *flag_host) return e;
  const int64_t R = *rows_host;
  const unsigned gr = grid_of(R, kPatWarps);
  e = launch_key_csr(L.dofs, n_elem * NB, R, G2.inc_off, G2.inc, G2.cursor, G2.partials, st);
  if (e == cudaSuccess && R > 0) {
    row_pattern_kernel<NB, false><<<gr, kPatWarps * 32, 0, st>>>(L.dofs, G2.inc_off, G2.inc, R, G2.cursor,
                                                                  G2.row_ptr, G2.col_idx, G2.colpos, G2.flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_exclusive_scan(G2.cursor, R, G2.partials, G2.row_ptr, st);
  if (e == cudaSuccess && R > 0) {
    row_pattern_kernel<NB, true><<<gr, kPatWarps * 32, 0, st>>>(L.dofs, G2.inc_off, G2.inc, R, G2.cursor,
                                                                 G2.row_ptr, G2.col_idx, G2.colpos, G2.flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(nnz_host, G2.row_ptr + R, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(flag_host, G1.flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// Rows of the P2 unknowns, 32 / NB of them per warp: lane group g (NB lanes)
// takes its own row, which accumulates in shared memory (at most kMaxCols
// columns).  For each incidence (e, i) of the row, in increasing element
// order, lane j of the group adds A_e[i][j] at the column position of the
// element's unknown j (distinct within an element); the group then stores the
// row, zeroing the buffer behind it.  Each entry is the sum of its
// contributions in element order.  The incidences' slots, positions and
// element rows are loaded NB incidences at a time before their additions.
constexpr int kRowWarps = 8;

template <int NB>
__global__ void __launch_bounds__(kRowWarps * 32)
    assemble_rows_kernel(const int32_t* __restrict__ inc_off, const int32_t* __restrict__ inc,
                         const uint8_t* __restrict__ colpos, const int32_t* __restrict__ row_ptr,
                         const float* __restrict__ A, const int32_t* __restrict__ n_rows_dev,
                         float* __restrict__ val) {
  constexpr int G = 32 / NB;  // rows per warp
  // row buffers 267 floats apart: the three rows of a warp start 11 banks apart
  constexpr int kRowStride = kMaxCols + 12;
  __shared__ float acc_s[kRowWarps][G][kRowStride];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / NB, j = lane - g * NB;
  const bool member = g < G;
  float* acc = acc_s[warp][member ? g : 0];
  // the row buffers are zero at the start of every row: zeroed once here, and
  // each column zeroed again as it is stored
  for (int c = lane; c < G * kRowStride; c += 32) (&acc_s[warp][0][0])[c] = 0.f;
  const int64_t n_rows = *n_rows_dev;
  for (int64_t r0 = (int64_t(blockIdx.x) * kRowWarps + warp) * G; r0 < n_rows;
       r0 += int64_t(gridDim.x) * kRowWarps * G) {
    const int64_t r = r0 + g;
    const bool live = member && r < n_rows;
    const int32_t rp = live ? row_ptr[r] : 0;
    const int len = live ? row_ptr[r + 1] - rp : 0;
    const int32_t tb = live ? inc_off[r] : 0;
    const int n_inc = live ? inc_off[r + 1] - tb : 0;
    __syncwarp();
    const int steps = __reduce_max_sync(0xffffffffu, n_inc);
    // NB incidences at a time: lane j of the group loads incidence k0 + j's
    // element slot and every incidence's column position j, then (after a
    // shuffle of the slots) the NB element rows, then the additions in order
    for (int k0 = 0; k0 < steps; k0 += NB) {
      const int32_t my_sl = (k0 + j < n_inc) ? __ldg(inc + tb + k0 + j) : 0;
      int pos[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) pos[u] = (k0 + u < n_inc) ? __ldg(colpos + (int64_t(tb) + k0 + u) * NB + j) : 0;
      float a[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int32_t sl = __shfl_sync(0xffffffffu, my_sl, (member ? g * NB : 0) + u);
        // slot sl = e * NB + i: row i of A_e starts at e * NB * NB + i * NB = sl * NB
        a[u] = (k0 + u < n_inc) ? __ldg(A + int64_t(sl) * NB + j) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        if (k0 + u < n_inc) acc[pos[u]] += a[u];
        __syncwarp();
      }
    }
    for (int c = j; c < len; c += NB) {
      __stcs(val + rp + c, acc[c]);
      acc[c] = 0.f;
    }
    __syncwarp();  // the row buffers are refilled for the next rows
  }
}

template <int NB>
cudaError_t launch_p2_assemble(const AsmP2Layout& L, const float* A, float* val, cudaStream_t st) {
  assemble_rows_kernel<NB><<<grid_of(L.rows_cap, kRowWarps * (32 / NB)), kRowWarps * 32, 0, st>>>(
      L.g2.inc_off, L.g2.inc, L.g2.colpos, L.g2.row_ptr, A, L.n_rows, val);
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

// Block size of the assembled matrix for a form: 1 (scalar forms), d (P1
// elasticity), 0 (not assembled: the coupling blocks are rectangular).
int asm_block(int form, int dim) {
  if (form == FEM_LAPLACE_P1 || form == FEM_LAPLACE_P1_W1 || form == FEM_LAPLACE_P1_ISO) return 1;
  if (form == FEM_LAPLACE_P2 || form == FEM_LAPLACE_P2_W1 || form == FEM_LAPLACE_P2_ISO) return 1;
  if (form == FEM_ELASTIC_P1) return dim;
  return 0;
}

// P2 forms: unknowns at the vertices and the edges.
bool asm_p2(int form) { return form == FEM_LAPLACE_P2 || form == FEM_LAPLACE_P2_W1 || form == FEM_LAPLACE_P2_ISO; }

fem_status asm_check(const fem_mesh* mesh, int form) {
  if (!mesh) return asm_fail(FEM_ERR_ARG, "mesh is NULL");
  if ((mesh->dim != 2 && mesh->dim != 3) || mesh->n_elem < 0 || mesh->n_vert < 0 || mesh->n_vert > INT32_MAX ||
      (mesh->n_elem > 0 && !mesh->conn))
    return asm_fail(FEM_ERR_ARG, "invalid mesh (dim 2/3, counts, conn)");
  if (form < FEM_LAPLACE_P1 || form > FEM_LAPLACE_P2_ISO) return asm_fail(FEM_ERR_ARG, "form out of range");
  if (asm_block(form, mesh->dim) == 0)
    return asm_fail(FEM_ERR_UNSUPPORTED, "assembly serves the square forms");
  const int64_t nodes = asm_p2(form) ? (mesh->dim + 1) * (mesh->dim + 2) / 2 : mesh->dim + 1;
  if (mesh->n_elem * nodes * nodes > INT32_MAX)
    return asm_fail(FEM_ERR_UNSUPPORTED, "n_elem * (nodes per element)^2 exceeds the int32 entry range");
  return FEM_OK;
}

// The P2 build (fem_assembly_build for the P2 forms).
fem_status p2_build(const fem_mesh* mesh, void* ws, size_t ws_bytes, int64_t* nnz, int64_t* n_records,
                    cudaStream_t st) {
  const fem::AsmP2Layout P = fem::asm_p2_layout(mesh->dim, mesh->n_elem, mesh->n_vert, ws);
  if (!ws || ws_bytes < P.bytes || reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    fem::set_last_error("assembly workspace needs %zu bytes, 256-byte aligned (got %zu)", P.bytes, ws_bytes);
    return FEM_ERR_WORKSPACE;
  }
  int32_t rows = 0, flag = 0, nz = 0;
  const cudaError_t e =
      mesh->dim == 2 ? fem::launch_p2_build<3>(mesh->conn, mesh->n_elem, mesh->n_vert, P, &rows, &flag, &nz, st)
                     : fem::launch_p2_build<4>(mesh->conn, mesh->n_elem, mesh->n_vert, P, &rows, &flag, &nz, st);
  if (e != cudaSuccess) {
    fem::set_last_error("fem_assembly_build: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  if (flag & fem::ASM_BAD_VERTEX) return asm_fail(FEM_ERR_ARG, "a connectivity entry is outside [0, n_vert)");
  if (flag & fem::ASM_REPEATED_VERTEX) return asm_fail(FEM_ERR_UNSUPPORTED, "an element repeats a vertex");
  if (flag & fem::ASM_ROW_TOO_LONG)
    return asm_fail(FEM_ERR_UNSUPPORTED, "an unknown has more than 255 neighbours or too many incident elements");
  if (nnz) *nnz = nz;
  if (n_records) *n_records = 0;
  return FEM_OK;
}

}  // namespace

extern "C" {

fem_status fem_assembly_workspace_size(const fem_mesh* mesh, int32_t form, size_t* bytes) {
  fem_status s = asm_check(mesh, form);
  if (s != FEM_OK) return s;
  if (!bytes) return asm_fail(FEM_ERR_ARG, "bytes is NULL");
  *bytes = asm_p2(form) ? fem::asm_p2_layout(mesh->dim, mesh->n_elem, mesh->n_vert, nullptr).bytes
                        : fem::asm_layout(mesh->dim, mesh->n_elem, mesh->n_vert, nullptr).bytes;
  return FEM_OK;
}

fem_status fem_assembly_build(const fem_mesh* mesh, int32_t form, void* ws, size_t ws_bytes, int64_t* nnz,
                              int64_t* n_records, void* stream) {
  fem_status s = asm_check(mesh, form);
  if (s != FEM_OK) return s;
  if (asm_p2(form)) return p2_build(mesh, ws, ws_bytes, nnz, n_records, static_cast<cudaStream_t>(stream));
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
  int32_t host[2] = {0, 0}, nrec = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host[0], L.flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host[1], L.row_ptr + V, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  // tile records of the scalar forms: cells per 32-element tile, entry-major records
  if (e == cudaSuccess && host[0] == 0 && asm_block(form, mesh->dim) == 1 && mesh->n_elem > 0) {
    e = fem::launch_tile_cells<false>(mesh->dim, mesh->conn, mesh->n_elem, L, st);
    if (e == cudaSuccess) e = fem::launch_exclusive_scan(L.cursor2, L.n_tiles, L.partials2, L.tile_rec, st);
    if (e == cudaSuccess) {
      fem::fill_neg_kernel<<<fem::grid_of(L.rec_cap, 256), 256, 0, st>>>(L.rec_entry, L.rec_cap);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = fem::launch_tile_cells<true>(mesh->dim, mesh->conn, mesh->n_elem, L, st);
    if (e == cudaSuccess)
      e = fem::launch_key_csr(L.rec_entry, L.rec_cap, host[1], L.eoff, L.rec_list, L.cursor2, L.partials2, st);
    if (e == cudaSuccess) {  // eoff[nnz] = the records
      fem::invert_list_kernel<<<fem::grid_of(L.rec_cap, 256), 256, 0, st>>>(L.rec_list, L.eoff + host[1], L.rec_dest);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host[0], L.flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nrec, L.tile_rec + L.n_tiles, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    fem::set_last_error("fem_assembly_build: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  if (host[0] & fem::ASM_BAD_VERTEX) return asm_fail(FEM_ERR_ARG, "a connectivity entry is outside [0, n_vert)");
  if (host[0] & fem::ASM_ROW_TOO_LONG)
    return asm_fail(FEM_ERR_UNSUPPORTED, "a vertex has more than 128 incident elements or 255 neighbours");
  if (host[0] & fem::ASM_REPEATED_VERTEX) return asm_fail(FEM_ERR_UNSUPPORTED, "an element repeats a vertex");
  if (nnz) *nnz = host[1];
  if (n_records) *n_records = nrec;
  return FEM_OK;
}

fem_status fem_assembly_pattern(const fem_mesh* mesh, int32_t form, const void* ws, size_t ws_bytes,
                                const int32_t** row_ptr, const int32_t** col_idx) {
  fem_status s = asm_check(mesh, form);
  if (s != FEM_OK) return s;
  if (asm_p2(form)) {
    const fem::AsmP2Layout P = fem::asm_p2_layout(mesh->dim, mesh->n_elem, mesh->n_vert, const_cast<void*>(ws));
    if (!ws || ws_bytes < P.bytes) return asm_fail(FEM_ERR_WORKSPACE, "assembly workspace too small");
    if (row_ptr) *row_ptr = P.g2.row_ptr;
    if (col_idx) *col_idx = P.g2.col_idx;
    return FEM_OK;
  }
  const fem::AsmLayout L = fem::asm_layout(mesh->dim, mesh->n_elem, mesh->n_vert, const_cast<void*>(ws));
  if (!ws || ws_bytes < L.bytes) return asm_fail(FEM_ERR_WORKSPACE, "assembly workspace too small");
  if (row_ptr) *row_ptr = L.row_ptr;
  if (col_idx) *col_idx = L.col_idx;
  return FEM_OK;
}

fem_status fem_assembly_unknowns(const fem_mesh* mesh, int32_t form, const void* ws, size_t ws_bytes,
                                 int64_t* n_rows, const int32_t** dofs) {
  fem_status s = asm_check(mesh, form);
  if (s != FEM_OK) return s;
  if (!asm_p2(form)) {
    if (n_rows) *n_rows = mesh->n_vert;
    if (dofs) *dofs = mesh->conn;
    return FEM_OK;
  }
  const fem::AsmP2Layout P = fem::asm_p2_layout(mesh->dim, mesh->n_elem, mesh->n_vert, const_cast<void*>(ws));
  if (!ws || ws_bytes < P.bytes) return asm_fail(FEM_ERR_WORKSPACE, "assembly workspace too small");
  if (n_rows) {
    int32_t r = 0;
    const cudaError_t e = cudaMemcpy(&r, P.n_rows, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      fem::set_last_error("fem_assembly_unknowns: %s", cudaGetErrorString(e));
      return FEM_ERR_CUDA;
    }
    *n_rows = r;
  }
  if (dofs) *dofs = P.dofs;
  return FEM_OK;
}

fem_status fem_assemble(const fem_mesh* mesh, int32_t form, const float* A, const void* ws, size_t ws_bytes,
                        float* values, void* stream) {
  fem_status s = asm_check(mesh, form);
  if (s != FEM_OK) return s;
  const fem::AsmLayout L = fem::asm_layout(mesh->dim, mesh->n_elem, mesh->n_vert, const_cast<void*>(ws));
  const size_t need = asm_p2(form) ? fem::asm_p2_layout(mesh->dim, mesh->n_elem, mesh->n_vert, nullptr).bytes : L.bytes;
  if (!ws || ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return asm_fail(FEM_ERR_WORKSPACE, "assembly workspace too small or unaligned");
  if (mesh->n_vert == 0) return FEM_OK;
  // without elements every row is empty and nothing is written
  if (mesh->n_elem > 0 && (!values || !A)) return asm_fail(FEM_ERR_ARG, "A or values is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int B = asm_block(form, mesh->dim);
  cudaError_t e;
  if (asm_p2(form)) {  // the row kernel over the vertex and edge unknowns
    const fem::AsmP2Layout P = fem::asm_p2_layout(mesh->dim, mesh->n_elem, mesh->n_vert, const_cast<void*>(ws));
    e = mesh->dim == 2 ? fem::launch_p2_assemble<6>(P, A, values, st) : fem::launch_p2_assemble<10>(P, A, values, st);
  } else if (B == 1 && mesh->n_elem > 0)  // scalar forms: tile records, then the per-entry sums
    e = mesh->dim == 2 ? fem::launch_tile_assemble_t<3>(L, A, mesh->n_elem, mesh->n_vert, values, st)
                       : fem::launch_tile_assemble_t<4>(L, A, mesh->n_elem, mesh->n_vert, values, st);
  else if (mesh->dim == 2)
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
