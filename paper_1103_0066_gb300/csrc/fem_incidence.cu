// fem_incidence.cu -- the deterministic vertex reduction of the adjoint:
// tile records, their vertex CSR, and the segmented sum into dcoords.
//
// The adjoint's element pass works on record tiles of kRecTile = 32
// consecutive elements, one per warp.  Within a tile the (d+1) vertex
// contributions of every element ("slots") that share a vertex are first
// summed in shared memory into one RECORD, in increasing slot order; a
// structured mesh in cell-major order has several times fewer records than
// slots, so only the records go to HBM.  The records of each vertex are then
// summed in increasing record order (= tile order).  Both orders are fixed by
// the mesh, so dcoords is bitwise reproducible.
//
// Built once per connectivity (fem_incidence_build), one warp per tile:
//   per tile : bitonic sort of (vertex, slot) keys -> the record count (pass
//              1); exclusive scan of the counts -> first record of each tile;
//              then (pass 2) every slot's stage position (one byte: the
//              element pass writes each contribution there, so a record is a
//              contiguous run), each record's span (start | length << 8) and
//              vertex.  On tets the runs start at positions congruent to 3r
//              mod 8 in a 256-position stage, which keeps the record loop's
//              shared reads free of bank conflicts.
//   global   : vertex -> records CSR (count, scan, fill, per-segment sort),
//              then each record's position in it (rec_dest): the element pass
//              writes record r straight to records[rec_dest[r]], so the
//              reduction reads each vertex's records as one contiguous run
#include <cuda_runtime.h>

#include <cstdint>

#include "fem_internal.h"
#include "fem_reduce.cuh"

namespace fem {

namespace {

constexpr int kScanBlock = 1024;

__global__ void fill_i32(int32_t* p, int64_t n, int32_t value) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = value;
}

__global__ void zero_f32(float* p, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = 0.f;
}

// cnt[key[i]] += 1 for every valid key
__global__ void count_kernel(const int32_t* keys, int64_t n, int64_t n_vert, int32_t* cnt) {
  for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = keys[s];
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

__global__ void fill_kernel(const int32_t* keys, int64_t n, int64_t n_vert, const int32_t* offsets,
                            int32_t* cursor, int32_t* list) {
  for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = keys[s];
    if (v >= 0 && v < n_vert) list[offsets[v] + atomicAdd(cursor + v, 1)] = int32_t(s);
  }
}

// Sorts each segment of a CSR list in increasing order: one warp per segment,
// each lane takes one entry and moves it to its rank (entries are distinct);
// segments longer than a warp fall back to an insertion sort by lane 0.
__global__ void sort_segments_kernel(const int32_t* offsets, int64_t n_seg, int32_t* list) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t v = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5); v < n_seg; v += warps) {
    const int32_t b = offsets[v], n = offsets[v + 1] - b;
    if (n <= 32) {
      const int32_t key = lane < n ? list[b + lane] : INT32_MAX;
      int rank = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) rank += (__shfl_sync(0xffffffffu, key, j) < key) ? 1 : 0;
      __syncwarp();
      if (lane < n) list[b + rank] = key;
    } else if (lane == 0) {
      for (int32_t i = b + 1; i < b + n; ++i) {
        const int32_t key = list[i];
        int32_t j = i - 1;
        while (j >= b && list[j] > key) {
          list[j + 1] = list[j];
          --j;
        }
        list[j + 1] = key;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- tile records

constexpr int kBuildThreads = 128;              // 4 warps, one record tile each
constexpr int kSortCap = 128;                   // power of two >= kRecTile * 4 slots
constexpr int kKeysPerLane = kSortCap / 32;
static_assert(kSortCap >= kRecTile * 4, "tile slot capacity");
constexpr uint64_t kNoVertex = 0xFFFFFFFFull;

// The warp's tile keys (vertex << 16 | slot), absent or invalid slots with the
// largest vertex, sorted in shared memory by a bitonic network (one warp).
__device__ void warp_sorted_keys(const int32_t* conn, int nv, int64_t n_elem, int64_t n_vert, int64_t tile,
                                 uint64_t* key) {
  const int lane = threadIdx.x & 31;
  const int ns = kRecTile * nv;
  const int64_t s0 = tile * kRecTile * nv;
  const int64_t smax = n_elem * nv;
#pragma unroll
  for (int q = 0; q < kKeysPerLane; ++q) {
    const int i = lane + 32 * q;
    uint64_t vtx = kNoVertex;
    if (i < ns && s0 + i < smax) {
      const int32_t v = conn[s0 + i];
      if (v >= 0 && v < n_vert) vtx = uint64_t(uint32_t(v));
    }
    key[i] = (vtx << 16) | uint64_t(i);
  }
  __syncwarp();
  for (int k = 2; k <= kSortCap; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int q = 0; q < kKeysPerLane; ++q) {
        const int i = lane + 32 * q;
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const uint64_t a = key[i], b = key[ixj];
          if ((a > b) == up) {
            key[i] = b;
            key[ixj] = a;
          }
        }
      }
      __syncwarp();
    }
}

__device__ __forceinline__ bool is_head(const uint64_t* key, int i) {
  const uint64_t v = key[i] >> 16;
  return v != kNoVertex && (i == 0 || (key[i - 1] >> 16) != v);
}

// Pass 1: the record count of each tile (its distinct vertices).
__global__ void __launch_bounds__(kBuildThreads)
    tile_sort_kernel(const int32_t* conn, int nv, int64_t n_elem, int64_t n_vert, int64_t n_tiles, int32_t* nrec) {
  __shared__ uint64_t keys[kBuildThreads / 32][kSortCap];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* key = keys[warp];
  const int ns = kRecTile * nv;
  const int64_t stride = int64_t(gridDim.x) * (kBuildThreads / 32);
  for (int64_t tile = blockIdx.x * int64_t(kBuildThreads / 32) + warp; tile < n_tiles; tile += stride) {
    warp_sorted_keys(conn, nv, n_elem, n_vert, tile, key);
    int c = 0;
#pragma unroll
    for (int q = 0; q < kKeysPerLane; ++q) {
      const int i = lane + 32 * q;
      if (i < ns) c += is_head(key, i) ? 1 : 0;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) nrec[tile] = c;
    __syncwarp();  // the key buffer is refilled for the next tile
  }
}

// Pass 2: per tile, its records (one per distinct vertex, in vertex order),
// the stage position (rank) of every slot, each record's span (start and
// length of its run in the stage) and vertex.  The slots of a record are
// consecutive positions in increasing slot order.  With pad = 8 the run of
// local record r starts at the first free position p with p = 3 r (mod 8): the
// adjoint sums record r in lane r, position by position, so the eight lanes of
// a quarter warp (eight consecutive records; 3 is odd) then read eight
// different 16-byte bank groups at every step.  The factor 3 rather than 1
// spreads the element lanes' stores of one slot over more bank groups (41.7
// against 34.6 store wavefronts per tile, simulated on the sliver cube).
// A tile whose padded stage would exceed cap positions, and every tile when
// pad = 0, packs the runs back to back.  Slots of absent elements (past
// n_elem) take the positions after the last run; zeros are written there and
// never read.
__global__ void __launch_bounds__(kBuildThreads)
    tile_records_kernel(const int32_t* conn, int nv, int64_t n_elem, int64_t n_vert, int64_t n_tiles,
                        const int32_t* tile_rec, int pad, int cap, uint8_t* rank, uint16_t* rec_span,
                        int32_t* rec_vertex) {
  __shared__ uint64_t keys[kBuildThreads / 32][kSortCap];
  __shared__ int16_t cstart[kBuildThreads / 32][kSortCap + 1];  // packed start of each record, + end
  __shared__ int16_t ostart[kBuildThreads / 32][kSortCap + 1];  // stage start of each record, + end
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* key = keys[warp];
  int16_t* cs = cstart[warp];
  int16_t* os = ostart[warp];
  const int ns = kRecTile * nv;
  const int64_t stride = int64_t(gridDim.x) * (kBuildThreads / 32);
  for (int64_t tile = blockIdx.x * int64_t(kBuildThreads / 32) + warp; tile < n_tiles; tile += stride) {
    warp_sorted_keys(conn, nv, n_elem, n_vert, tile, key);
    const int32_t rb = tile_rec[tile], rn = tile_rec[tile + 1] - rb;
    // lane owns the consecutive entries [kKeysPerLane * lane, kKeysPerLane * (lane + 1))
    int heads = 0, valid = 0;
#pragma unroll
    for (int q = 0; q < kKeysPerLane; ++q) {
      const int i = kKeysPerLane * lane + q;
      heads += is_head(key, i) ? 1 : 0;
      valid += (key[i] >> 16) != kNoVertex ? 1 : 0;
    }
    int incl = heads;  // inclusive warp scan of the head counts
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    const int n_valid = __reduce_add_sync(0xffffffffu, valid);
    const int lr0 = incl - heads - 1;  // local record of the entry before the lane's first
    int lr = lr0;
#pragma unroll
    for (int q = 0; q < kKeysPerLane; ++q) {
      const int i = kKeysPerLane * lane + q;
      if (is_head(key, i)) cs[++lr] = int16_t(i);
    }
    if (lane == 0) cs[rn] = int16_t(n_valid);
    __syncwarp();
    if (lane == 0) {  // stage starts: padded if they fit, else packed
      int o = 0;
      if (pad > 0) {
        for (int r = 0; r < rn; ++r) {
          o += (3 * r - o) & (pad - 1);
          os[r] = int16_t(o);
          o += cs[r + 1] - cs[r];
        }
      }
      if (pad == 0 || o + (ns - n_valid) > cap) {
        for (int r = 0; r < rn; ++r) os[r] = cs[r];
        o = n_valid;
      }
      os[rn] = int16_t(o);
    }
    __syncwarp();
    lr = lr0;
#pragma unroll
    for (int q = 0; q < kKeysPerLane; ++q) {
      const int i = kKeysPerLane * lane + q;
      if (i >= ns) continue;
      const uint64_t v = key[i] >> 16;
      const int slot = int(key[i] & 0xFFFF);
      int pos;
      if (v != kNoVertex) {
        if (is_head(key, i)) {
          ++lr;
          rec_vertex[rb + lr] = int32_t(v);
          rec_span[rb + lr] = uint16_t(os[lr] | ((cs[lr + 1] - cs[lr]) << 8));
        }
        pos = os[lr] + (i - cs[lr]);
      } else {
        pos = os[rn] + (i - n_valid);
      }
      // element slot / nv of the tile, local vertex slot % nv; 4 bytes per element
      rank[(tile * kRecTile + slot / nv) * 4 + slot % nv] = uint8_t(pos);
    }
    __syncwarp();  // the key and start buffers are refilled for the next tile
  }
}

// rec_dest[vrec[k]] = k for the R = voff[n_vert] records: the vertex-major
// position of every record (vrec[0, R) is a permutation of [0, R): every
// record has a valid vertex).
__global__ void dest_kernel(const int32_t* voff, int64_t n_vert, const int32_t* vrec, int32_t* rec_dest) {
  const int64_t R = voff[n_vert];
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < R; k += int64_t(gridDim.x) * blockDim.x)
    rec_dest[vrec[k]] = int32_t(k);
}

// Locality of the vertex-major layout: counts the records whose vertex-major
// row lies within kNearRows rows of the previous record's (record r - 1 of
// the same tile).  When most records are near, the element pass's record
// writes land in a few neighbouring sectors per tile; otherwise (elements in
// no spatial order, or vertices numbered at random) they scatter over the
// whole record array and every write is a partial-sector update.
constexpr int32_t kNearRows = 64;

__global__ void locality_kernel(const int32_t* tile_rec, int64_t n_tiles, const int32_t* rec_dest, int32_t* near) {
  int32_t c = 0;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n_tiles; t += int64_t(gridDim.x) * blockDim.x) {
    const int32_t rb = tile_rec[t], re = tile_rec[t + 1];
    for (int32_t r = rb + 1; r < re; ++r) {
      const int32_t d = rec_dest[r] - rec_dest[r - 1];
      c += (d >= -kNearRows && d <= kNearRows) ? 1 : 0;
    }
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(near, c);
}

// The layout decision, on the device: vertex-major when at least half of the
// records (beyond each tile's first) are near their predecessor, else tile
// order with rec_dest[r] = r.
__global__ void choose_layout_kernel(const int32_t* tile_rec, int64_t n_tiles, const int32_t* near, int32_t* mode,
                                     int32_t* rec_dest) {
  const int32_t R = tile_rec[n_tiles];
  const int32_t pairs = R - int32_t(n_tiles);
  const int32_t m = (2 * int64_t(*near) >= int64_t(pairs)) ? kRecVertexMajor : kRecTileOrder;
  if (blockIdx.x == 0 && threadIdx.x == 0) *mode = m;
  if (m == kRecTileOrder)
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < R; r += int64_t(gridDim.x) * blockDim.x)
      rec_dest[r] = int32_t(r);
}

// One thread per vertex; the per-vertex sums are fem_reduce.cuh's.  The
// layout word is read once; the branch is uniform over the grid.
template <int D, int NC>
__device__ __forceinline__ void reduce_direct(const int32_t* __restrict__ voff, const float* __restrict__ records,
                                              int64_t n_vert, float* __restrict__ dcoords, float* __restrict__ dcoef) {
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n_vert;
       v += int64_t(gridDim.x) * blockDim.x)
    reduce_vertex_direct<D, NC>(voff, records, v, dcoords, dcoef);
}

template <int D, int NC>
__device__ __forceinline__ void reduce_gather(const int32_t* __restrict__ voff, const int32_t* __restrict__ vrec,
                                              const float* __restrict__ records, int64_t n_vert,
                                              float* __restrict__ dcoords, float* __restrict__ dcoef) {
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n_vert;
       v += int64_t(gridDim.x) * blockDim.x)
    reduce_vertex_gather<D, NC>(voff, vrec, records, v, dcoords, dcoef);
}

template <int D, int NC>
__global__ void vertex_reduce_kernel(const int32_t* __restrict__ voff, const int32_t* __restrict__ vrec,
                                     const int32_t* __restrict__ mode, const float* __restrict__ records,
                                     int64_t n_vert, float* __restrict__ dcoords, float* __restrict__ dcoef) {
  if (__ldg(mode) == kRecTileOrder)
    reduce_gather<D, NC>(voff, vrec, records, n_vert, dcoords, dcoef);
  else
    reduce_direct<D, NC>(voff, records, n_vert, dcoords, dcoef);
}

unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  const int64_t cap = int64_t(device_sm_count()) * 32;
  if (g > cap) g = cap;
  return unsigned(g < 1 ? 1 : g);
}

// offsets[0..n] = exclusive prefix sums of cnt[0..n) (offsets[n] = total).
void exclusive_scan(const int32_t* cnt, int64_t n, int32_t* partials, int32_t* offsets, cudaStream_t stream) {
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  if (nb > 0) scan_partials_kernel<<<unsigned(nb), kScanBlock, 0, stream>>>(cnt, n, partials);
  scan_top_kernel<<<1, kScanBlock, 0, stream>>>(partials, nb);
  scan_apply_kernel<<<unsigned(nb > 0 ? nb : 1), kScanBlock, 0, stream>>>(cnt, n, partials, nb, offsets);
}

}  // namespace

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t bwd_workspace_layout(int dim, int64_t n_elem, int64_t n_vert, bool with_scratch, void* base,
                            BwdWorkspace* ws, int ncomp) {
  if (ncomp <= 0) ncomp = dim;
  const int64_t nv = dim + 1;
  const int64_t n_tiles = (n_elem + kRecTile - 1) / kRecTile;
  const int64_t r_max = n_elem * nv;  // at most one record per slot
  const int64_t n_cnt = n_vert > n_tiles ? n_vert : n_tiles;
  const int64_t nb = (n_cnt + kScanBlock - 1) / kScanBlock;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t o_tile_rec = take(sizeof(int32_t) * size_t(n_tiles + 1));
  const size_t o_rank = take(sizeof(uint32_t) * size_t(n_tiles * kRecTile));
  const size_t o_rec_span = take(sizeof(uint16_t) * size_t(r_max));
  const size_t o_rec_dest = take(sizeof(int32_t) * size_t(r_max));
  const size_t o_rec_vertex = take(sizeof(int32_t) * size_t(r_max));
  const size_t o_voff = take(sizeof(int32_t) * size_t(n_vert + 1));
  const size_t o_vrec = take(sizeof(int32_t) * size_t(r_max));
  const size_t o_cursor = take(sizeof(int32_t) * size_t(n_cnt + 1));
  const size_t o_part = take(sizeof(int32_t) * size_t(nb + 1));
  const size_t o_mode = take(sizeof(int32_t) * 2);  // layout word, locality count
  const size_t o_records = with_scratch ? take(sizeof(float) * size_t(r_max * ncomp)) : off;
  if (ws) {
    char* b = static_cast<char*>(base);
    ws->tile_rec = reinterpret_cast<int32_t*>(b + o_tile_rec);
    ws->rank = reinterpret_cast<uint32_t*>(b + o_rank);
    ws->rec_span = reinterpret_cast<uint16_t*>(b + o_rec_span);
    ws->rec_dest = reinterpret_cast<int32_t*>(b + o_rec_dest);
    ws->rec_vertex = reinterpret_cast<int32_t*>(b + o_rec_vertex);
    ws->voff = reinterpret_cast<int32_t*>(b + o_voff);
    ws->vrec = reinterpret_cast<int32_t*>(b + o_vrec);
    ws->cursor = reinterpret_cast<int32_t*>(b + o_cursor);
    ws->partials = reinterpret_cast<int32_t*>(b + o_part);
    ws->mode = reinterpret_cast<int32_t*>(b + o_mode);
    ws->records = with_scratch ? reinterpret_cast<float*>(b + o_records) : nullptr;
    ws->n_tiles = n_tiles;
    ws->ncomp = ncomp;
    ws->bytes = off;
  }
  return off;
}

size_t scan_partials_count(int64_t n) { return size_t((n + kScanBlock - 1) / kScanBlock + 1); }

cudaError_t launch_exclusive_scan(const int32_t* cnt, int64_t n, int32_t* partials, int32_t* offsets,
                                  cudaStream_t stream) {
  exclusive_scan(cnt, n, partials, offsets, stream);
  return cudaGetLastError();
}

cudaError_t launch_key_csr(const int32_t* keys, int64_t n_keys, int64_t n_seg, int32_t* off, int32_t* list,
                           int32_t* cursor, int32_t* partials, cudaStream_t stream) {
  fill_i32<<<grid_for(n_seg, 256), 256, 0, stream>>>(cursor, n_seg, 0);
  count_kernel<<<grid_for(n_keys, 256), 256, 0, stream>>>(keys, n_keys, n_seg, cursor);
  exclusive_scan(cursor, n_seg, partials, off, stream);
  fill_i32<<<grid_for(n_seg, 256), 256, 0, stream>>>(cursor, n_seg, 0);
  fill_kernel<<<grid_for(n_keys, 256), 256, 0, stream>>>(keys, n_keys, n_seg, off, cursor, list);
  sort_segments_kernel<<<grid_for((n_seg + 3) / 4, 128), 128, 0, stream>>>(off, n_seg, list);
  return cudaGetLastError();
}

cudaError_t launch_incidence_build(int dim, const int32_t* conn, int64_t n_elem, int64_t n_vert,
                                   const BwdWorkspace& ws, cudaStream_t stream) {
  const int nv = dim + 1;
  const int64_t n_tiles = ws.n_tiles;
  const int64_t r_max = n_elem * nv;
  const int64_t tb = (n_tiles + kBuildThreads / 32 - 1) / (kBuildThreads / 32);
  const unsigned tg = unsigned(tb < 4 * 65535 ? (tb > 0 ? tb : 1) : 4 * 65535);
  // tile records; record slots past the last record keep vertex -1
  tile_sort_kernel<<<tg, kBuildThreads, 0, stream>>>(conn, nv, n_elem, n_vert, n_tiles, ws.cursor);
  exclusive_scan(ws.cursor, n_tiles, ws.partials, ws.tile_rec, stream);
  fill_i32<<<grid_for(r_max, 256), 256, 0, stream>>>(ws.rec_vertex, r_max, -1);
  tile_records_kernel<<<tg, kBuildThreads, 0, stream>>>(conn, nv, n_elem, n_vert, n_tiles, ws.tile_rec,
                                                         dim == 3 ? 8 : 0, dim == 3 ? kStageCap3 : kRecTile * nv,
                                                         reinterpret_cast<uint8_t*>(ws.rank), ws.rec_span,
                                                         ws.rec_vertex);
  // vertex -> records CSR
  launch_key_csr(ws.rec_vertex, r_max, n_vert, ws.voff, ws.vrec, ws.cursor, ws.partials, stream);
  dest_kernel<<<grid_for(r_max, 256), 256, 0, stream>>>(ws.voff, n_vert, ws.vrec, ws.rec_dest);
  // record layout: vertex-major rows when the writes keep their locality, else tile order
  fill_i32<<<1, 32, 0, stream>>>(ws.mode + 1, 1, 0);
  locality_kernel<<<grid_for(n_tiles, 256), 256, 0, stream>>>(ws.tile_rec, n_tiles, ws.rec_dest, ws.mode + 1);
  choose_layout_kernel<<<grid_for(r_max, 256), 256, 0, stream>>>(ws.tile_rec, n_tiles, ws.mode + 1, ws.mode,
                                                                   ws.rec_dest);
  return cudaGetLastError();
}

cudaError_t launch_zero_f32(float* p, int64_t n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  zero_f32<<<grid_for(n, 256), 256, 0, stream>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_vertex_reduce(int dim, const BwdWorkspace& ws, int64_t n_vert, float* dcoords,
                                 cudaStream_t stream, float* dcoef) {
  if (n_vert == 0) return cudaSuccess;
  const int block = 256;
  const unsigned g = unsigned((n_vert + block - 1) / block);
  if (dim == 2) {
    if (ws.ncomp == 3)
      vertex_reduce_kernel<2, 3><<<g, block, 0, stream>>>(ws.voff, ws.vrec, ws.mode, ws.records, n_vert, dcoords,
                                                          dcoef);
    else
      vertex_reduce_kernel<2, 2><<<g, block, 0, stream>>>(ws.voff, ws.vrec, ws.mode, ws.records, n_vert, dcoords,
                                                          nullptr);
  } else {
    if (ws.ncomp == 4)
      vertex_reduce_kernel<3, 4><<<g, block, 0, stream>>>(ws.voff, ws.vrec, ws.mode, ws.records, n_vert, dcoords,
                                                          dcoef);
    else
      vertex_reduce_kernel<3, 3><<<g, block, 0, stream>>>(ws.voff, ws.vrec, ws.mode, ws.records, n_vert, dcoords,
                                                          nullptr);
  }
  return cudaGetLastError();
}

}  // namespace fem
