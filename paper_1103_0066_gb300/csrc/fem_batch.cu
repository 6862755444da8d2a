// fem_batch.cu -- many meshes of mixed forms in persistent launches.
//
// Single-kernel mode (FEM_BATCH_SINGLE).  Work items, in dispensing order:
//   [0, n_tile_items)        one 128-element tile of some mesh: forward A
//                            and/or the adjoint element pass with its records
//   [n_tile_items, n_total)  a range of vertices of some mesh: the deterministic
//                            reduction of that mesh's records into dcoords
// Persistent CTAs (4 warps, one tile each time) take `chunk` consecutive items
// per atomicAdd on a global counter.  A reduction item waits until every tile of
// its mesh has been counted done.  All tiles precede all reduction items in the
// dispensing order and a CTA holding a tile never waits, so every awaited tile
// is held by a running CTA and the wait ends; it is nevertheless bounded and
// reports FEM_DEVERR_TIMEOUT when it gives up.  The per-tile code is the
// per-mesh kernels' (fwd_compute_tile, bwd_compute_tile, warp_records).
//
// Per-item modes (FEM_BATCH_PER_ITEM, FEM_BATCH_PER_ITEM_CONCURRENT): every
// item through the single-mesh kernels, on the records this batch built; in
// order on one stream, or spread over kItemLanes streams (longest items first,
// each to the least loaded lane) so that small items fill the gaps of large
// ones.
//
// Grouped modes (FEM_BATCH_GROUPED, FEM_BATCH_GROUPED_CONCURRENT): the same
// item scheme per (dim, form) kind, one kind-specialised pipelined kernel per
// kind present, launched in order on one stream or forked onto side streams.
//
// Phased mode (FEM_BATCH_PHASED): per kind, the multi-mesh forward, adjoint
// element pass and vertex reduction of fem_multi.cuh, one launch each over
// all of the kind's meshes (kMultiMeshes at a time), the kinds forked onto
// side streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fem.h"
#include "fem_bwd.cuh"
#include "fem_fwd.cuh"
#include "fem_internal.h"
#include "fem_multi.cuh"

namespace fem {

struct BatchMesh {
  int32_t kind;   // (dim - 2) * 3 + form
  int32_t flags;  // BM_* bits
  int64_t n_elem, n_vert;
  const int32_t* conn;
  const float* coords;
  const float* coef;
  const float* dA;
  float* A;
  float* dcoords;
  float* dcoef;
  const int32_t* tile_rec;  // per 32-element record tile
  const uint32_t* rank;
  const uint16_t* rec_span;
  const int32_t* rec_dest;
  const int32_t* voff;
  const int32_t* vrec;  // records of each vertex (tile-order layout)
  const int32_t* rec_mode;  // record layout (kRecVertexMajor or kRecTileOrder)
  float* records;
  int64_t tile_begin, n_tiles;  // element tiles of this mesh in the item space (all meshes)
  int64_t wait_tiles;           // tiles counted done before the mesh's reduction items run (= n_tiles)
  int64_t red_begin, n_red;     // reduction items (all meshes)
  int64_t ktile_begin, kred_begin;  // the same within its kind group (grouped launches)
};
enum : int { BM_FWD = 1, BM_BWD = 2, BM_REC = 4 };

struct BatchCounters {
  unsigned long long next[8];  // [0]: single-kernel launch, [1 + kind]: grouped launches
  int32_t err;
  int32_t pad;
  int32_t done[1];  // [n_items] tiles completed per mesh
};

constexpr int kRedVerts = 2048;  // vertices per reduction item
constexpr int kItemLanes = 10;   // streams of the per-item concurrent mode (4: 2.14 ms, 6: 2.01, 10: 1.97, 16: 1.98 on the 96-mesh batch)
constexpr uint32_t kSpinLimit = 1u << 24;  // default bound of a reduction item's wait (about a second)

// Shared memory of one batch warp: a stage shared by the forward tile and the
// dA rows, then the slot stage of the warp's records (sized for tets).
template <int D, int FORM>
constexpr size_t batch_stage_bytes() {
  return std::max(FwdPlan<D, FORM, float, float>::per_warp, BwdPlan<D, FORM>::da_slot);
}
constexpr size_t kXsWarpBytes = BwdPlan<3, LAPLACE_P1>::xs_bytes;

__device__ __forceinline__ int find_mesh(const BatchMesh* desc, int n, int64_t item, bool red, bool local = false) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {  // last mesh whose range begins at or before `item`
    const int mid = (lo + hi + 1) >> 1;
    const int64_t b = local ? (red ? desc[mid].kred_begin : desc[mid].ktile_begin)
                            : (red ? desc[mid].red_begin : desc[mid].tile_begin);
    if (b <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Record range of the warp's 32-element tile t (rank word of its lane, first
// record, record count); zeros past the mesh.
struct WarpRec {
  uint32_t rk;
  int32_t rb, rn;
};

__device__ __forceinline__ WarpRec load_warp_rec(const BatchMesh& M, int64_t t, int lane) {
  WarpRec r{0u, 0, 0};
  if ((M.flags & BM_REC) && t * 32 < M.n_elem) {
    r.rk = __ldg(M.rank + t * 32 + lane);
    r.rb = __ldg(M.tile_rec + t);
    r.rn = __ldg(M.tile_rec + t + 1) - r.rb;
  }
  return r;
}

__device__ __forceinline__ BwdParams bwd_params(const BatchMesh& M, int vec_conn) {
  BwdParams bp;
  bp.conn = M.conn;
  bp.coords = M.coords;
  bp.coef = M.coef;
  bp.dA = M.dA;
  bp.tile_rec = (M.flags & BM_REC) ? M.tile_rec : nullptr;
  bp.rank = M.rank;
  bp.rec_span = M.rec_span;
  bp.rec_dest = M.rec_dest;
  bp.records = M.records;
  bp.dcoef = M.dcoef;
  bp.dcoords = nullptr;
  bp.n_elem = M.n_elem;
  bp.n_vert = M.n_vert;
  bp.dev_err = nullptr;
  bp.vec_conn = vec_conn;
  bp.vec_dA = reinterpret_cast<uintptr_t>(M.dA) % 16 == 0;
  return bp;
}

__device__ __forceinline__ FwdParams<float, float> fwd_params(const BatchMesh& M, int vec_conn) {
  FwdParams<float, float> fp;
  fp.conn = M.conn;
  fp.coords = M.coords;
  fp.coef = M.coef;
  fp.A = M.A;
  fp.n_elem = M.n_elem;
  fp.n_vert = M.n_vert;
  fp.dev_err = nullptr;
  fp.vec_conn = vec_conn;
  fp.vec_store = reinterpret_cast<uintptr_t>(M.A) % 16 == 0;
  return fp;
}

// Adjoint element pass of one warp's tile and its records (dA already staged in drow_base).
template <int D, int FORM>
__device__ __forceinline__ int warp_bwd(const BatchMesh& M, const BwdParams& bp, int64_t t, int lane, int f, float w,
                                        const float (&X)[D + 1][D], const int (&v)[D + 1], const float* dstage,
                                        float* xs, const WarpRec& wr) {
  const bool rec = (M.flags & BM_REC) != 0;
  const RecAhead ah = rec ? load_rec_ahead(M.rec_span, M.rec_dest, wr.rb, wr.rn, lane) : RecAhead{0u, 0};
  const int err = bwd_compute_tile<D, FORM, JAC_COMP, false>(bp, t, lane, f, Coef<1>{{w}}, X,
                                                            dstage + lane * BwdPlan<D, FORM>::DST, v,
                                                            rec ? xs : nullptr, wr.rk);
  if (rec) {
    __syncwarp();
    warp_records<D>(xs, M.rec_span, M.rec_dest, wr.rb, wr.rn, ah, M.records, lane);
  }
  return err;
}

template <int D, int FORM>
__device__ void batch_tile(const BatchMesh& M, int64_t T, int phases, unsigned char* smem, size_t stage_bytes,
                           int& err) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char* wbase = smem + size_t(warp) * (stage_bytes + kXsWarpBytes);
  float* wst = reinterpret_cast<float*>(wbase);
  float* xs = reinterpret_cast<float*>(wbase + stage_bytes);
  const int64_t t = T * 4 + warp, e = t * 32 + lane;
  const int vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(M.conn) % 16 == 0);
  int v[D + 1];
  float X[D + 1][D];
  load_conn<D>(M.conn, e, M.n_elem, vec_conn, v);
  const int f = gather_regs<D>(M.coords, M.n_vert, e, M.n_elem, v, X);
  const float w = (M.coef && e < M.n_elem) ? __ldg(M.coef + e) : 1.f;
  if ((phases & FEM_PHASE_FWD) && (M.flags & BM_FWD))
    err |= fwd_compute_tile<D, FORM, JAC_COMP, float, float>(fwd_params(M, vec_conn), t, lane, f, w, X, wst);
  if ((phases & FEM_PHASE_BWD) && (M.flags & BM_BWD)) {
    const BwdParams bp = bwd_params(M, vec_conn);
    const WarpRec wr = load_warp_rec(M, t, lane);
    __syncwarp();  // the forward tile's stage reads are done
    copy_dA_async<D, FORM>(bp, t, lane, wst);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    err |= warp_bwd<D, FORM>(M, bp, t, lane, f, w, X, v, wst, xs, wr);
  }
  __threadfence();  // every thread's records are visible device-wide before the tile is counted
  __syncthreads();  // (and the stages are reused by the next item)
}

template <int D>
__device__ void batch_reduce(const BatchMesh& M, int64_t r) {
  const int64_t v0 = r * kRedVerts;
  const int64_t v1 = v0 + kRedVerts < M.n_vert ? v0 + kRedVerts : M.n_vert;
  const bool gather = __ldg(M.rec_mode) == kRecTileOrder;
  for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    const int32_t b = M.voff[v], e = M.voff[v + 1];
    float acc[D];
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] = 0.f;
    for (int32_t k = b; k < e; ++k) {
      const int64_t row = gather ? M.vrec[k] : k;  // same increasing record order either way
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] += __ldcg(M.records + row * D + a);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) M.dcoords[v * D + a] = acc[a];
  }
}

__global__ void __launch_bounds__(kTileElems) fem_batch_kernel(const BatchMesh* __restrict__ desc, int n_items,
                                                               int64_t n_tile_items, int64_t n_total,
                                                               BatchCounters* ctr, int phases, int chunk,
                                                               size_t stage_bytes, uint32_t spin_limit) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long s_item;
  int err = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(&ctr->next[0], (unsigned long long)chunk);
    __syncthreads();
    const int64_t i0 = s_item;
    __syncthreads();  // s_item is rewritten at the next grab
    if (i0 >= n_total) break;
    const int64_t i1 = i0 + chunk < n_total ? i0 + chunk : n_total;
    for (int64_t it = i0; it < i1; ++it) {
      if (it < n_tile_items) {
        const int m = find_mesh(desc, n_items, it, false);
        const BatchMesh& M = desc[m];
        const int64_t T = it - M.tile_begin;
        switch (M.kind) {
          case 0: batch_tile<2, LAPLACE_P1>(M, T, phases, smem_raw, stage_bytes, err); break;
          case 1: batch_tile<2, LAPLACE_P2>(M, T, phases, smem_raw, stage_bytes, err); break;
          case 2: batch_tile<2, ELASTIC_P1>(M, T, phases, smem_raw, stage_bytes, err); break;
          case 3: batch_tile<3, LAPLACE_P1>(M, T, phases, smem_raw, stage_bytes, err); break;
          case 4: batch_tile<3, LAPLACE_P2>(M, T, phases, smem_raw, stage_bytes, err); break;
          default: batch_tile<3, ELASTIC_P1>(M, T, phases, smem_raw, stage_bytes, err); break;
        }
        if (threadIdx.x == 0) atomicAdd(&ctr->done[m], 1);
      } else {
        const int64_t ir = it - n_tile_items;
        const int m = find_mesh(desc, n_items, ir, true);
        const BatchMesh& M = desc[m];
        __shared__ int s_timeout;
        if (threadIdx.x == 0) {
          const volatile int32_t* done = ctr->done + m;
          uint32_t spins = 0;
          while (*done < M.wait_tiles && spins < spin_limit) {
            __nanosleep(64);
            ++spins;
          }
          s_timeout = *done < M.wait_tiles;
          __threadfence();
        }
        __syncthreads();
        if (s_timeout) {  // the mesh's records are incomplete: its dcoords are not written
          err |= DEVERR_TIMEOUT;
        } else if (M.kind < 3) {
          batch_reduce<2>(M, ir - M.red_begin);
        } else {
          batch_reduce<3>(M, ir - M.red_begin);
        }
        __syncthreads();
      }
    }
  }
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && (threadIdx.x & 31) == 0) atomicOr(&ctr->err, err);
}


// ------------------------------------------------------------------ grouped launches
// One persistent kernel per (dim, form) kind over that kind's meshes, with
// registers and shared memory sized for the kind, the forward and the adjoint
// element pass fused (one gather per element) and a two-deep item pipeline: the
// next item's connectivity, coordinates, slot ranks and record range
// (registers) and its dA (cp.async) are fetched while the current tile
// computes.

template <int D, int FORM>
struct KindPlan {
  using FP = FwdPlan<D, FORM, float, float>;
  using BP = BwdPlan<D, FORM>;
  static constexpr size_t da_slot = BP::da_slot;
  // Two dA slots beside the forward stage while that keeps two CTAs per SM;
  // otherwise (P2 and elasticity on tets) one slot that the forward stage
  // aliases, filled after the forward tile.
  static constexpr int DA_SLOTS = (4 * (FP::per_warp + 2 * da_slot + BP::xs_bytes) <= size_t(100) * 1024) ? 2 : 1;
  static constexpr size_t fst_bytes = DA_SLOTS == 2 ? FP::per_warp : 0;
  static constexpr size_t stage =
      DA_SLOTS == 2 ? FP::per_warp + 2 * da_slot : (FP::per_warp > da_slot ? FP::per_warp : da_slot);
  static constexpr size_t per_warp = stage + BP::xs_bytes;
  static constexpr size_t smem = 4 * per_warp;
};

template <int D>
struct KindItem {
  int m;       // mesh within the kind group
  int64_t T;   // CTA tile within the mesh
  int f;       // gather flags
  float w;
  int v[D + 1];
  float X[D + 1][D];
  WarpRec wr;
};

template <int D, int FORM>
__device__ __forceinline__ void kind_prefetch(const BatchMesh* desc, int n, int64_t item, int phases, int s,
                                              KindItem<D>& it, float* dslots) {
  using KP = KindPlan<D, FORM>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  it.m = find_mesh(desc, n, item, false, true);
  const BatchMesh& M = desc[it.m];
  it.T = item - M.ktile_begin;
  const int64_t t = it.T * 4 + warp, e = t * 32 + lane;
  const int vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(M.conn) % 16 == 0);
  load_conn<D>(M.conn, e, M.n_elem, vec_conn, it.v);
  it.f = gather_regs<D>(M.coords, M.n_vert, e, M.n_elem, it.v, it.X);
  it.w = (M.coef && e < M.n_elem) ? __ldg(M.coef + e) : 1.f;
  it.wr = WarpRec{0u, 0, 0};
  if ((phases & FEM_PHASE_BWD) && (M.flags & BM_BWD)) {
    if constexpr (KP::DA_SLOTS == 2) {
      BwdParams bp;
      bp.dA = M.dA;
      bp.n_elem = M.n_elem;
      bp.vec_dA = reinterpret_cast<uintptr_t>(M.dA) % 16 == 0;
      copy_dA_async<D, FORM>(bp, t, lane, dslots + s * (KP::da_slot / 4));
    }
    it.wr = load_warp_rec(M, t, lane);
  }
}

template <int D, int FORM>
__device__ __forceinline__ void kind_tile(const BatchMesh& M, const KindItem<D>& it, int phases, int s,
                                          float* fst, float* dslots, float* xs, int& err) {
  using KP = KindPlan<D, FORM>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t = it.T * 4 + warp;
  const int vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(M.conn) % 16 == 0);
  if ((phases & FEM_PHASE_FWD) && (M.flags & BM_FWD))
    err |= fwd_compute_tile<D, FORM, JAC_COMP, float, float>(fwd_params(M, vec_conn), t, lane, it.f, it.w, it.X,
                                                             fst);
  if ((phases & FEM_PHASE_BWD) && (M.flags & BM_BWD)) {
    const BwdParams bp = bwd_params(M, vec_conn);
    float* dslot = dslots + (KP::DA_SLOTS == 2 ? s : 0) * (KP::da_slot / 4);
    if constexpr (KP::DA_SLOTS == 1) {  // no room to prefetch: fetch now, into the forward stage
      __syncwarp();
      copy_dA_async<D, FORM>(bp, t, lane, dslot);
      cp_async_commit();
      cp_async_wait<0>();
      __syncwarp();
    }
    err |= warp_bwd<D, FORM>(M, bp, t, lane, it.f, it.w, it.X, it.v, dslot, xs, it.wr);
  }
  __threadfence();  // every thread's records are visible device-wide before the tile is counted
  __syncthreads();
}

template <int D, int FORM>
__global__ void __launch_bounds__(kTileElems)
    fem_batch_kind_kernel(const BatchMesh* __restrict__ desc, int n, int m_base, int64_t n_tile_items,
                          int64_t n_total, BatchCounters* ctr, int slot, int phases, int chunk,
                          uint32_t spin_limit) {
  using KP = KindPlan<D, FORM>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long s_next;
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned char* wbase = smem_raw + size_t(warp) * KP::per_warp;
  float* fst = reinterpret_cast<float*>(wbase);
  float* dslots = reinterpret_cast<float*>(wbase + KP::fst_bytes);
  float* xs = reinterpret_cast<float*>(wbase + KP::stage);
  int err = 0;
  auto grab = [&]() -> int64_t {
    if (tid == 0) s_next = (long long)atomicAdd(&ctr->next[slot], (unsigned long long)chunk);
    __syncthreads();
    const int64_t g = s_next;
    __syncthreads();
    return g;
  };
  int64_t cur = grab();
  int64_t cend = cur + chunk < n_total ? cur + chunk : n_total;
  KindItem<D> a, b;
  int s = 0;
  if (cur < n_tile_items) kind_prefetch<D, FORM>(desc, n, cur, phases, 0, a, dslots);
  cp_async_commit();
  while (cur < n_total) {
    int64_t nxt = cur + 1;
    if (nxt >= cend) {
      nxt = grab();
      cend = nxt + chunk < n_total ? nxt + chunk : n_total;
    }
    if (nxt < n_tile_items) kind_prefetch<D, FORM>(desc, n, nxt, phases, s ^ 1, b, dslots);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();  // the current item's dA rows (copied by the warp's lanes) are visible
    if (cur < n_tile_items) {
      kind_tile<D, FORM>(desc[a.m], a, phases, s, fst, dslots, xs, err);
      if (tid == 0) atomicAdd(&ctr->done[m_base + a.m], 1);
    } else {
      const int64_t ir = cur - n_tile_items;
      const int m = find_mesh(desc, n, ir, true, true);
      const BatchMesh& M = desc[m];
      __shared__ int s_timeout;
      if (tid == 0) {
        const volatile int32_t* done = ctr->done + m_base + m;
        uint32_t spins = 0;
        while (*done < M.wait_tiles && spins < spin_limit) {
          __nanosleep(64);
          ++spins;
        }
        s_timeout = *done < M.wait_tiles;
        __threadfence();
      }
      __syncthreads();
      if (s_timeout) {
        err |= DEVERR_TIMEOUT;
      } else {
        batch_reduce<D>(M, ir - M.kred_begin);
      }
      __syncthreads();
    }
    a = b;
    s ^= 1;
    cur = nxt;
  }
  cp_async_wait<0>();
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && (threadIdx.x & 31) == 0) atomicOr(&ctr->err, err);
}

size_t stage_bytes_for_kind(int kind) {
  switch (kind) {
    case 0: return batch_stage_bytes<2, LAPLACE_P1>();
    case 1: return batch_stage_bytes<2, LAPLACE_P2>();
    case 2: return batch_stage_bytes<2, ELASTIC_P1>();
    case 3: return batch_stage_bytes<3, LAPLACE_P1>();
    case 4: return batch_stage_bytes<3, LAPLACE_P2>();
    default: return batch_stage_bytes<3, ELASTIC_P1>();
  }
}

struct KindLaunch {
  const BatchMesh* desc;
  int n, m_base;
  int64_t n_tile_items, n_total;
  BatchCounters* ctr;
  int slot, phases, chunk;
  int64_t grid;
  uint32_t spin_limit;
};

template <int D, int FORM>
cudaError_t kind_setup_t(int* occ, size_t* smem) {
  using KP = KindPlan<D, FORM>;
  const void* fn = reinterpret_cast<const void*>(fem_batch_kind_kernel<D, FORM>);
  cudaError_t e = ensure_smem(fn, KP::smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fem_batch_kind_kernel<D, FORM>, kTileElems, KP::smem);
  *smem = KP::smem;
  return e;
}

template <int D, int FORM>
cudaError_t kind_launch_t(const KindLaunch& L, cudaStream_t st) {
  fem_batch_kind_kernel<D, FORM><<<unsigned(L.grid), kTileElems, KindPlan<D, FORM>::smem, st>>>(
      L.desc, L.n, L.m_base, L.n_tile_items, L.n_total, L.ctr, L.slot, L.phases, L.chunk, L.spin_limit);
  return cudaGetLastError();
}

cudaError_t kind_setup(int kind, int* occ, size_t* smem) {
  switch (kind) {
    case 0: return kind_setup_t<2, LAPLACE_P1>(occ, smem);
    case 1: return kind_setup_t<2, LAPLACE_P2>(occ, smem);
    case 2: return kind_setup_t<2, ELASTIC_P1>(occ, smem);
    case 3: return kind_setup_t<3, LAPLACE_P1>(occ, smem);
    case 4: return kind_setup_t<3, LAPLACE_P2>(occ, smem);
    default: return kind_setup_t<3, ELASTIC_P1>(occ, smem);
  }
}

cudaError_t kind_launch(int kind, const KindLaunch& L, cudaStream_t st) {
  switch (kind) {
    case 0: return kind_launch_t<2, LAPLACE_P1>(L, st);
    case 1: return kind_launch_t<2, LAPLACE_P2>(L, st);
    case 2: return kind_launch_t<2, ELASTIC_P1>(L, st);
    case 3: return kind_launch_t<3, LAPLACE_P1>(L, st);
    case 4: return kind_launch_t<3, LAPLACE_P2>(L, st);
    default: return kind_launch_t<3, ELASTIC_P1>(L, st);
  }
}

}  // namespace fem

// ------------------------------------------------------------------ host side

struct fem_batch {
  int n_items = 0;
  std::vector<fem::BatchMesh> desc;   // caller's order (single-kernel mode)
  std::vector<fem::BatchMesh> kdesc;  // grouped by kind, kind-local item ranges
  std::vector<int> kpos;              // position of each item's descriptor in kdesc (-1: in no group)
  std::vector<int> kitem;             // the item of each kdesc entry
  fem::BatchMesh* d_desc = nullptr;
  fem::BatchMesh* d_kdesc = nullptr;
  fem::BatchCounters* d_ctr = nullptr;
  size_t ctr_bytes = 0;
  int64_t n_tile_items = 0, n_total_fwd = 0, n_total = 0;
  size_t stage_bytes = 0, smem = 0;
  int ctas_per_sm = 0, chunk = 1, max_ctas_per_sm = 1, mode = FEM_BATCH_SINGLE;
  bool has_coupling = false;  // a coupling-block item: the per-item modes only
  uint32_t spin_limit = fem::kSpinLimit;  // bound of the reduction items' waits (fem_batch_inject_wait)
  struct Group {
    int kind, first, count;
    int64_t n_tile_items, n_total, work;
    int occ;
  };
  std::vector<Group> groups;  // non-empty kinds, largest work first
  std::vector<fem_batch_item> items;        // the caller's items (per-item mode)
  std::vector<fem::BwdWorkspace> item_ws;  // their record workspaces (valid when the item has records)
  std::vector<float*> item_det;            // det J from the forward for the adjoint (per-item mode), or null
  cudaStream_t aux[6] = {};
  cudaEvent_t fork = nullptr, join[6] = {};
  // per-item concurrent mode: lane of every item; lanes 1.. run on item_aux
  std::vector<int> item_lane;
  cudaStream_t item_aux[fem::kItemLanes - 1] = {};
  cudaEvent_t item_join[fem::kItemLanes - 1] = {};
  int n_lanes = 1;
  ~fem_batch() {
    for (cudaStream_t s : aux)
      if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : join)
      if (e) cudaEventDestroy(e);
    for (cudaStream_t s : item_aux)
      if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : item_join)
      if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
  }
};

namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

fem_status check_items(const fem_batch_item* items, int32_t n) {
  if (!items || n <= 0) {
    fem::set_last_error("items must be a non-empty array");
    return FEM_ERR_ARG;
  }
  for (int i = 0; i < n; ++i) {
    const fem_batch_item& it = items[i];
    const fem_mesh& m = it.mesh;
    if ((m.dim != 2 && m.dim != 3) || m.coord_dtype != FEM_F32 || m.n_elem < 0 || m.n_vert < 0 ||
        m.n_vert > INT32_MAX || (m.n_elem > 0 && (!m.conn || !m.coords))) {
      fem::set_last_error("batch item %d: invalid mesh (dim 2/3, FP32 coordinates, non-NULL arrays)", i);
      return FEM_ERR_ARG;
    }
    const bool form_ok = (it.form >= FEM_LAPLACE_P1 && it.form <= FEM_ELASTIC_P1) || it.form == FEM_DIV_P1P1 ||
                         it.form == FEM_DIV_P2P1;
    if (!form_ok || it.reserved != 0) {
      fem::set_last_error("batch item %d: invalid form or reserved field", i);
      return FEM_ERR_ARG;
    }
    if (m.n_elem * (m.dim + 1) > INT32_MAX) {
      fem::set_last_error("batch item %d: n_elem * (dim + 1) exceeds the int32 slot range", i);
      return FEM_ERR_UNSUPPORTED;
    }
  }
  return FEM_OK;
}

size_t item_ws_bytes(const fem_batch_item& it) {
  if (!it.dcoords) return 0;
  return fem::bwd_workspace_layout(it.mesh.dim, it.mesh.n_elem, it.mesh.n_vert, true, nullptr, nullptr);
}

// det J of every element, kept by the per-item forward for the per-item adjoint
// when an item has both.
size_t item_det_bytes(const fem_batch_item& it) {
  return (it.A && it.dA && (it.dcoords || it.dcoef)) ? sizeof(float) * size_t(it.mesh.n_elem) : 0;
}

// [descriptors, caller order][descriptors, grouped by kind][counters]
size_t head_bytes(int32_t n, size_t* kdesc_off, size_t* ctr_off, size_t* ctr_bytes) {
  const size_t desc_bytes = al256(sizeof(fem::BatchMesh) * size_t(n));
  *kdesc_off = desc_bytes;
  *ctr_off = 2 * desc_bytes;
  *ctr_bytes = al256(offsetof(fem::BatchCounters, done) + sizeof(int32_t) * size_t(n));
  return 2 * desc_bytes + *ctr_bytes;
}

int64_t grid_for(int ctas_per_sm, int64_t total, int chunk) {
  int64_t grid = int64_t(ctas_per_sm) * fem::device_sm_count();
  const int64_t need = (total + chunk - 1) / chunk;
  if (grid > need) grid = need;
  return grid < 1 ? 1 : grid;
}

cudaError_t launch_group(fem_batch* b, const fem_batch::Group& g, int phases, int ctas_per_sm, int chunk,
                         cudaStream_t st) {
  const int64_t total = (phases & FEM_PHASE_BWD) ? g.n_total : g.n_tile_items;
  if (total == 0) return cudaSuccess;
  fem::KindLaunch L;
  L.desc = b->d_kdesc + g.first;
  L.n = g.count;
  L.m_base = g.first;
  L.n_tile_items = g.n_tile_items;
  L.n_total = total;
  L.ctr = b->d_ctr;
  L.slot = 1 + g.kind;
  L.phases = phases;
  L.chunk = chunk;
  L.grid = grid_for(std::min(ctas_per_sm, g.occ), total, chunk);
  L.spin_limit = b->spin_limit;
  return fem::kind_launch(g.kind, L, st);
}

cudaError_t launch_per_item(fem_batch* b, int phases, cudaStream_t st0, bool concurrent) {
  cudaError_t e = cudaSuccess;
  const bool fan = concurrent && b->n_lanes > 1;
  if (fan) {  // fork: every lane starts after the work already on st0
    if ((e = cudaEventRecord(b->fork, st0)) != cudaSuccess) return e;
    for (int l = 1; l < b->n_lanes; ++l)
      if ((e = cudaStreamWaitEvent(b->item_aux[l - 1], b->fork, 0)) != cudaSuccess) return e;
  }
  for (size_t k = 0; k < b->items.size() && e == cudaSuccess; ++k) {
    const fem_batch_item& it = b->items[k];
    const fem::BatchMesh& M = b->desc[k];
    const int lane = fan ? b->item_lane[k] : 0;
    cudaStream_t st = lane == 0 ? st0 : b->item_aux[lane - 1];
    // both passes in this run: the forward keeps det J for the adjoint (same bits)
    float* det = ((phases & FEM_PHASE_FWD) && (phases & FEM_PHASE_BWD) && (M.flags & fem::BM_FWD) &&
                  (M.flags & fem::BM_BWD)) ? b->item_det[k] : nullptr;
    if (M.n_elem == 0) {
      if ((phases & FEM_PHASE_BWD) && (M.flags & fem::BM_REC) && M.n_vert > 0)
        e = fem::launch_zero_f32(it.dcoords, M.n_vert * it.mesh.dim, st);  // no element: dcoords = 0
      continue;
    }
    if ((phases & FEM_PHASE_FWD) && (M.flags & fem::BM_FWD)) {
      fem::FwdLaunch L{};
      L.dim = it.mesh.dim;
      L.form = it.form;
      L.jac = fem::JAC_COMP;
      L.conn = it.mesh.conn;
      L.coords = it.mesh.coords;
      L.coef = it.coef;
      L.A = it.A;
      L.n_elem = M.n_elem;
      L.n_vert = M.n_vert;
      L.dev_err = &b->d_ctr->err;
      L.warps = 0;  // the kernel's default
      L.stream = st;
      L.det_out = det;
      if (it.form == FEM_DIV_P1P1 || it.form == FEM_DIV_P2P1)
        e = fem::launch_div_fwd(L);
      else
        e = L.dim == 2 ? fem::launch_fwd_d2(L)
                       : (it.form == FEM_ELASTIC_P1 ? fem::launch_fwd_d3_ela(L) : fem::launch_fwd_d3_lap(L));
    }
    if (e == cudaSuccess && (phases & FEM_PHASE_BWD) && (M.flags & fem::BM_BWD)) {
      const bool rec = (M.flags & fem::BM_REC) != 0;
      const fem::BwdWorkspace& W = b->item_ws[k];
      fem::BwdLaunch L{};
      L.dim = it.mesh.dim;
      L.form = it.form;
      L.jac = fem::JAC_COMP;
      L.atomic = 0;
      L.conn = it.mesh.conn;
      L.coords = static_cast<const float*>(it.mesh.coords);
      L.coef = it.coef;
      L.dA = it.dA;
      L.dcoef = it.dcoef;
      L.tile_rec = rec ? W.tile_rec : nullptr;
      L.rank = rec ? W.rank : nullptr;
      L.rec_span = rec ? W.rec_span : nullptr;
      L.rec_dest = rec ? W.rec_dest : nullptr;
      L.records = rec ? W.records : nullptr;
      L.dcoords = it.dcoords;
      L.n_elem = M.n_elem;
      L.n_vert = M.n_vert;
      L.dev_err = &b->d_ctr->err;
      L.stream = st;
      L.det_in = det;
      e = (it.form == FEM_DIV_P1P1 || it.form == FEM_DIV_P2P1) ? fem::launch_div_bwd(L) : fem::launch_bwd_elem(L);
      if (e == cudaSuccess && rec) e = fem::launch_vertex_reduce(it.mesh.dim, W, M.n_vert, it.dcoords, st);
    }
  }
  if (fan && e == cudaSuccess) {  // join every lane back into st0
    for (int l = 1; l < b->n_lanes && e == cudaSuccess; ++l) {
      e = cudaEventRecord(b->item_join[l - 1], b->item_aux[l - 1]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st0, b->item_join[l - 1], 0);
    }
  }
  return e;
}

// One kind's three multi-mesh launches on stream st (FEM_BATCH_PHASED): the
// forward over the meshes that want A (keeping det J where the adjoint runs
// in the same call), the adjoint element pass (meshes with and without a
// saved det J in separate launches), then the vertex reduction.
cudaError_t launch_kind_phases(fem_batch* b, const fem_batch::Group& g, int phases, cudaStream_t st) {
  const int dim = g.kind / 3 + 2, form = g.kind % 3;
  const bool both = (phases & FEM_PHASE_FWD) && (phases & FEM_PHASE_BWD);
  int32_t* dev_err = &b->d_ctr->err;
  cudaError_t e = cudaSuccess;
  if (phases & FEM_PHASE_FWD) {
    fem::FwdMulti P;
    P.n = 0;
    P.dev_err = dev_err;
    P.tile_begin[0] = 0;
    auto flush = [&]() {
      if (P.n == 0 || e != cudaSuccess) return;
      e = dim == 2 ? fem::launch_fwd_multi_d2(form, P, st) : fem::launch_fwd_multi_d3(form, P, st);
      P.n = 0;
    };
    for (int j = g.first; j < g.first + g.count && e == cudaSuccess; ++j) {
      const int i = b->kitem[size_t(j)];
      const fem::BatchMesh& M = b->desc[size_t(i)];
      if (!(M.flags & fem::BM_FWD) || M.n_elem == 0) continue;
      fem::FwdParams<float, float>& p = P.p[P.n];
      p.conn = M.conn;
      p.coords = M.coords;
      p.coef = M.coef;
      p.A = M.A;
      p.n_elem = M.n_elem;
      p.n_vert = M.n_vert;
      p.dev_err = dev_err;
      p.vec_conn = (dim == 3) && (reinterpret_cast<uintptr_t>(M.conn) % 16 == 0);
      p.vec_store = reinterpret_cast<uintptr_t>(M.A) % 16 == 0;
      p.det_out = (both && (M.flags & fem::BM_BWD)) ? b->item_det[size_t(i)] : nullptr;
      P.tile_begin[P.n + 1] = P.tile_begin[P.n] + (M.n_elem + 31) / 32;
      if (++P.n == fem::kMultiMeshes) flush();
    }
    flush();
  }
  if (!(phases & FEM_PHASE_BWD) || e != cudaSuccess) return e;
  for (int saved = 0; saved < 2 && e == cudaSuccess; ++saved) {
    fem::BwdMulti P;
    P.n = 0;
    P.dev_err = dev_err;
    P.tile_begin[0] = 0;
    auto flush = [&]() {
      if (P.n == 0 || e != cudaSuccess) return;
      e = dim == 2 ? fem::launch_bwd_multi_d2(form, saved != 0, P, st)
                   : fem::launch_bwd_multi_d3(form, saved != 0, P, st);
      P.n = 0;
    };
    for (int j = g.first; j < g.first + g.count && e == cudaSuccess; ++j) {
      const int i = b->kitem[size_t(j)];
      const fem::BatchMesh& M = b->desc[size_t(i)];
      if (!(M.flags & fem::BM_BWD) || M.n_elem == 0) continue;
      const bool has_det = both && (M.flags & fem::BM_FWD);
      if (has_det != (saved != 0)) continue;
      const bool rec = (M.flags & fem::BM_REC) != 0;
      const fem::BwdWorkspace& W = b->item_ws[size_t(i)];
      fem::BwdParams& p = P.p[P.n];
      p.conn = M.conn;
      p.coords = M.coords;
      p.coef = M.coef;
      p.dA = M.dA;
      p.tile_rec = rec ? W.tile_rec : nullptr;
      p.rank = rec ? W.rank : nullptr;
      p.rec_span = rec ? W.rec_span : nullptr;
      p.rec_dest = rec ? W.rec_dest : nullptr;
      p.records = rec ? W.records : nullptr;
      p.dcoef = M.dcoef;
      p.dcoords = M.dcoords;
      p.n_elem = M.n_elem;
      p.n_vert = M.n_vert;
      p.dev_err = dev_err;
      p.vec_conn = (dim == 3) && (reinterpret_cast<uintptr_t>(M.conn) % 16 == 0);
      p.vec_dA = reinterpret_cast<uintptr_t>(M.dA) % 16 == 0;
      p.det = has_det ? b->item_det[size_t(i)] : nullptr;
      P.tile_begin[P.n + 1] = P.tile_begin[P.n] + (M.n_elem + 31) / 32;
      if (++P.n == fem::kMultiMeshes) flush();
    }
    flush();
  }
  fem::RedMulti R;
  R.n = 0;
  R.blk_begin[0] = 0;
  auto flush = [&]() {
    if (R.n == 0 || e != cudaSuccess) return;
    e = dim == 2 ? fem::launch_reduce_multi_d2(R, st) : fem::launch_reduce_multi_d3(R, st);
    R.n = 0;
  };
  for (int j = g.first; j < g.first + g.count && e == cudaSuccess; ++j) {
    const int i = b->kitem[size_t(j)];
    const fem::BatchMesh& M = b->desc[size_t(i)];
    if (!(M.flags & fem::BM_REC) || M.n_vert == 0) continue;
    if (M.n_elem == 0) {  // no element: dcoords = 0
      e = fem::launch_zero_f32(M.dcoords, M.n_vert * dim, st);
      continue;
    }
    const fem::BwdWorkspace& W = b->item_ws[size_t(i)];
    R.r[R.n] = fem::RedMesh{W.voff, W.vrec, W.mode, W.records, M.dcoords, M.n_vert};
    R.blk_begin[R.n + 1] = R.blk_begin[R.n] + (M.n_vert + fem::kMultiRedBlock - 1) / fem::kMultiRedBlock;
    if (++R.n == fem::kMultiMeshes) flush();
  }
  flush();
  return e;
}

// FEM_BATCH_PHASED: the largest kind on st, the others forked onto side
// streams and joined back.
cudaError_t launch_phased(fem_batch* b, int phases, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (b->groups.size() < 2) {
    for (const auto& g : b->groups)
      if ((e = launch_kind_phases(b, g, phases, st)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  if ((e = cudaEventRecord(b->fork, st)) != cudaSuccess) return e;
  for (size_t k = 1; k < b->groups.size(); ++k) {
    if ((e = cudaStreamWaitEvent(b->aux[k], b->fork, 0)) != cudaSuccess) return e;
    if ((e = launch_kind_phases(b, b->groups[k], phases, b->aux[k])) != cudaSuccess) return e;
    if ((e = cudaEventRecord(b->join[k], b->aux[k])) != cudaSuccess) return e;
  }
  if ((e = launch_kind_phases(b, b->groups[0], phases, st)) != cudaSuccess) return e;
  for (size_t k = 1; k < b->groups.size(); ++k)
    if ((e = cudaStreamWaitEvent(st, b->join[k], 0)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_batch(fem_batch* b, int phases, int ctas_per_sm, int chunk, int mode, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->d_ctr, 0, b->ctr_bytes, st);
  if (e != cudaSuccess) return e;
  if (mode == FEM_BATCH_PER_ITEM || mode == FEM_BATCH_PER_ITEM_CONCURRENT)
    return launch_per_item(b, phases, st, mode == FEM_BATCH_PER_ITEM_CONCURRENT);
  if (mode == FEM_BATCH_PHASED) return launch_phased(b, phases, st);
  if (mode == FEM_BATCH_SINGLE) {
    const int64_t total = (phases & FEM_PHASE_BWD) ? b->n_total : b->n_total_fwd;
    fem::fem_batch_kernel<<<unsigned(grid_for(ctas_per_sm, total, chunk)), fem::kTileElems, b->smem, st>>>(
        b->d_desc, b->n_items, b->n_tile_items, total, b->d_ctr, phases, chunk, b->stage_bytes, b->spin_limit);
    return cudaGetLastError();
  }
  if (mode == FEM_BATCH_GROUPED || b->groups.size() < 2) {
    for (const auto& g : b->groups)
      if ((e = launch_group(b, g, phases, ctas_per_sm, chunk, st)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  // concurrent: the largest group on `st`, the others forked onto side
  // streams and joined back, so one group's tail overlaps the next ones
  if ((e = cudaEventRecord(b->fork, st)) != cudaSuccess) return e;
  for (size_t k = 1; k < b->groups.size(); ++k) {
    if ((e = cudaStreamWaitEvent(b->aux[k], b->fork, 0)) != cudaSuccess) return e;
    if ((e = launch_group(b, b->groups[k], phases, ctas_per_sm, chunk, b->aux[k])) != cudaSuccess) return e;
    if ((e = cudaEventRecord(b->join[k], b->aux[k])) != cudaSuccess) return e;
  }
  if ((e = launch_group(b, b->groups[0], phases, ctas_per_sm, chunk, st)) != cudaSuccess) return e;
  for (size_t k = 1; k < b->groups.size(); ++k)
    if ((e = cudaStreamWaitEvent(st, b->join[k], 0)) != cudaSuccess) return e;
  return cudaSuccess;
}

bool valid_config(int ctas_per_sm, int chunk, int mode) {
  return mode >= FEM_BATCH_SINGLE && mode <= FEM_BATCH_PHASED && chunk >= 1 && chunk <= 64 &&
         ctas_per_sm >= 1 && ctas_per_sm <= 32;
}

}  // namespace

extern "C" {

fem_status fem_batch_workspace_size(const fem_batch_item* items, int32_t n_items, size_t* bytes) {
  fem_status s = check_items(items, n_items);
  if (s != FEM_OK) return s;
  if (!bytes) {
    fem::set_last_error("bytes is NULL");
    return FEM_ERR_ARG;
  }
  size_t ko, co, cb;
  size_t total = head_bytes(n_items, &ko, &co, &cb);
  for (int i = 0; i < n_items; ++i) total += al256(item_ws_bytes(items[i])) + al256(item_det_bytes(items[i]));
  *bytes = total;
  return FEM_OK;
}

fem_status fem_batch_create(const fem_batch_item* items, int32_t n_items, void* ws, size_t ws_bytes,
                            fem_batch** out, void* stream) {
  fem_status s = check_items(items, n_items);
  if (s != FEM_OK) return s;
  if (!out) {
    fem::set_last_error("out is NULL");
    return FEM_ERR_ARG;
  }
  size_t need = 0;
  fem_batch_workspace_size(items, n_items, &need);
  if (!ws || ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    fem::set_last_error("batch workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    return FEM_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  fem_batch* b = new (std::nothrow) fem_batch();
  if (!b) {
    fem::set_last_error("out of host memory");
    return FEM_ERR_ARG;
  }
  b->n_items = n_items;
  b->desc.resize(size_t(n_items));
  b->items.assign(items, items + n_items);
  b->item_ws.assign(size_t(n_items), fem::BwdWorkspace{});
  b->item_det.assign(size_t(n_items), nullptr);
  b->kpos.assign(size_t(n_items), -1);
  size_t kdesc_off = 0, ctr_off = 0;
  size_t off = head_bytes(n_items, &kdesc_off, &ctr_off, &b->ctr_bytes);
  char* base = static_cast<char*>(ws);
  b->d_desc = reinterpret_cast<fem::BatchMesh*>(base);
  b->d_kdesc = reinterpret_cast<fem::BatchMesh*>(base + kdesc_off);
  b->d_ctr = reinterpret_cast<fem::BatchCounters*>(base + ctr_off);
  int64_t tiles = 0, reds = 0;
  size_t stage = 0;
  for (int i = 0; i < n_items; ++i) {
    const fem_batch_item& it = items[i];
    fem::BatchMesh& M = b->desc[size_t(i)];
    std::memset(&M, 0, sizeof(M));
    // the persistent kernels serve the six square (dim, form) kinds; a coupling
    // block (kind -1) runs through the per-item modes only
    const bool cpl = it.form == FEM_DIV_P1P1 || it.form == FEM_DIV_P2P1;
    M.kind = cpl ? -1 : (it.mesh.dim - 2) * 3 + it.form;
    b->has_coupling |= cpl;
    M.n_elem = it.mesh.n_elem;
    M.n_vert = it.mesh.n_vert;
    M.conn = it.mesh.conn;
    M.coords = static_cast<const float*>(it.mesh.coords);
    M.coef = it.coef;
    M.dA = it.dA;
    M.A = it.A;
    M.dcoords = it.dcoords;
    M.dcoef = it.dcoef;
    M.flags = (it.A ? fem::BM_FWD : 0) | ((it.dA && (it.dcoords || it.dcoef)) ? fem::BM_BWD : 0) |
              ((it.dA && it.dcoords) ? fem::BM_REC : 0);
    M.n_tiles = (M.n_elem + fem::kTileElems - 1) / fem::kTileElems;
    M.wait_tiles = M.n_tiles;
    M.tile_begin = tiles;
    tiles += M.n_tiles;
    if (!cpl) stage = std::max(stage, fem::stage_bytes_for_kind(M.kind));
    const size_t wsb = item_ws_bytes(it);
    if (wsb) {
      fem::BwdWorkspace W{};
      fem::bwd_workspace_layout(it.mesh.dim, it.mesh.n_elem, it.mesh.n_vert, true, base + off, &W);
      cudaError_t e = fem::launch_incidence_build(it.mesh.dim, it.mesh.conn, it.mesh.n_elem, it.mesh.n_vert, W, st);
      if (e != cudaSuccess) {
        delete b;
        fem::set_last_error("batch item %d: incidence build: %s", i, cudaGetErrorString(e));
        return FEM_ERR_CUDA;
      }
      b->item_ws[size_t(i)] = W;
      M.tile_rec = W.tile_rec;
      M.rank = W.rank;
      M.rec_span = W.rec_span;
      M.rec_dest = W.rec_dest;
      M.voff = W.voff;
      M.vrec = W.vrec;
      M.rec_mode = W.mode;
      M.records = W.records;
      off += al256(wsb);
    }
    if (const size_t db = item_det_bytes(it)) {
      b->item_det[size_t(i)] = reinterpret_cast<float*>(base + off);
      off += al256(db);
    }
  }
  for (int i = 0; i < n_items; ++i) {  // reduction items follow all tiles
    fem::BatchMesh& M = b->desc[size_t(i)];
    M.n_red = (M.flags & fem::BM_REC) ? (M.n_vert + fem::kRedVerts - 1) / fem::kRedVerts : 0;
    M.red_begin = reds;
    reds += M.n_red;
  }
  b->n_tile_items = tiles;
  b->n_total_fwd = tiles;
  b->n_total = tiles + reds;
  b->stage_bytes = stage;
  b->smem = 4 * (stage + fem::kXsWarpBytes);
  // kind groups: the same descriptors ordered by kind, item ranges local to the kind
  cudaError_t e = cudaSuccess;
  for (int kind = 0; kind < 6 && e == cudaSuccess; ++kind) {
    fem_batch::Group g{kind, int(b->kdesc.size()), 0, 0, 0, 0, 1};
    int64_t kt = 0, kr = 0;
    for (size_t i = 0; i < b->desc.size(); ++i) {
      const fem::BatchMesh& M0 = b->desc[i];
      if (M0.kind != kind) continue;
      b->kpos[i] = int(b->kdesc.size());
      b->kitem.push_back(int(i));
      fem::BatchMesh M = M0;
      M.ktile_begin = kt;
      kt += M.n_tiles;
      b->kdesc.push_back(M);
      ++g.count;
      g.work += M.n_elem;
    }
    for (int j = g.first; j < g.first + g.count; ++j) {
      b->kdesc[size_t(j)].kred_begin = kr;
      kr += b->kdesc[size_t(j)].n_red;
    }
    if (g.count == 0 || kt + kr == 0) continue;  // (meshes without elements still get dcoords = 0)
    g.n_tile_items = kt;
    g.n_total = kt + kr;
    size_t ksmem = 0;
    e = fem::kind_setup(kind, &g.occ, &ksmem);
    g.occ = std::max(g.occ, 1);
    b->groups.push_back(g);
  }
  std::stable_sort(b->groups.begin(), b->groups.end(),
                   [](const fem_batch::Group& x, const fem_batch::Group& y) { return x.work > y.work; });
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  // per-item lanes: longest items first, each to the least loaded lane (bytes of
  // A or dA per element stand for an item's work)
  b->n_lanes = n_items > 1 ? std::min(n_items, fem::kItemLanes) : 1;
  for (int l = 1; l < b->n_lanes && e == cudaSuccess; ++l) {
    e = cudaStreamCreateWithFlags(&b->item_aux[l - 1], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->item_join[l - 1], cudaEventDisableTiming);
  }
  {
    std::vector<int> order(static_cast<size_t>(n_items));
    std::vector<double> work(static_cast<size_t>(n_items)), load(static_cast<size_t>(b->n_lanes), 0.0);
    for (int i = 0; i < n_items; ++i) {
      order[size_t(i)] = i;
      const int nv = items[i].mesh.dim + 1, d = nv - 1;
      int nn = 0;  // entries of one element block
      switch (items[i].form) {
        case FEM_LAPLACE_P1: nn = nv * nv; break;
        case FEM_LAPLACE_P2: nn = (nv * (nv + 1) / 2) * (nv * (nv + 1) / 2); break;
        case FEM_ELASTIC_P1: nn = d * nv * d * nv; break;
        case FEM_DIV_P1P1: nn = nv * d * nv; break;
        default: nn = nv * d * (nv * (nv + 1) / 2); break;
      }
      work[size_t(i)] = double(items[i].mesh.n_elem) * double(nn + 8);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[size_t(x)] > work[size_t(y)]; });
    b->item_lane.assign(size_t(n_items), 0);
    for (int i : order) {
      const int l = int(std::min_element(load.begin(), load.end()) - load.begin());
      b->item_lane[size_t(i)] = l;
      load[size_t(l)] += work[size_t(i)];
    }
  }
  for (size_t k = 1; k < b->groups.size() && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(fem::BatchMesh) * size_t(n_items), cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess && !b->kdesc.empty())
    e = cudaMemcpyAsync(b->d_kdesc, b->kdesc.data(), sizeof(fem::BatchMesh) * b->kdesc.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = fem::ensure_smem(reinterpret_cast<const void*>(fem::fem_batch_kernel), b->smem);
  int occ = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fem::fem_batch_kernel, fem::kTileElems, b->smem);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host tables must outlive the copies
  if (e != cudaSuccess) {
    delete b;
    fem::set_last_error("fem_batch_create: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  b->max_ctas_per_sm = occ > 0 ? occ : 1;
  for (const auto& g : b->groups) b->max_ctas_per_sm = std::max(b->max_ctas_per_sm, g.occ);
  b->ctas_per_sm = b->max_ctas_per_sm;
  b->chunk = 1;
  b->mode = b->has_coupling ? FEM_BATCH_PER_ITEM_CONCURRENT
            : b->groups.empty() ? FEM_BATCH_SINGLE : FEM_BATCH_PHASED;
  *out = b;
  return FEM_OK;
}

fem_status fem_batch_run(fem_batch* b, int32_t phases, void* stream) {
  if (!b || (phases & ~(FEM_PHASE_FWD | FEM_PHASE_BWD)) || !phases) {
    fem::set_last_error("fem_batch_run: bad batch or phases");
    return FEM_ERR_ARG;
  }
  cudaError_t e = launch_batch(b, phases, b->ctas_per_sm, b->chunk, b->mode, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    fem::set_last_error("fem_batch_run: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  return FEM_OK;
}

fem_status fem_batch_tune(fem_batch* b, int32_t phases, void* stream) {
  if (!b || (phases & ~(FEM_PHASE_FWD | FEM_PHASE_BWD)) || !phases) {
    fem::set_last_error("fem_batch_tune: bad batch or phases");
    return FEM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    fem::set_last_error("fem_batch_tune: event creation failed");
    return FEM_ERR_CUDA;
  }
  float best = 1e30f;
  int best_c = b->ctas_per_sm, best_k = b->chunk, best_m = b->mode;
  const int chunks[] = {1, 2, 4, 8};
  cudaError_t err = cudaSuccess;
  for (int mode = FEM_BATCH_SINGLE; mode <= FEM_BATCH_PHASED && err == cudaSuccess; ++mode) {
    const bool grouped = mode == FEM_BATCH_GROUPED || mode == FEM_BATCH_GROUPED_CONCURRENT || mode == FEM_BATCH_PHASED;
    const bool per_item = mode == FEM_BATCH_PER_ITEM || mode == FEM_BATCH_PER_ITEM_CONCURRENT;
    const bool fixed = per_item || mode == FEM_BATCH_PHASED;  // no grid or chunk to tune
    if (grouped && b->groups.empty()) continue;
    if (!per_item && b->has_coupling) continue;  // the persistent kernels serve the square kinds
    const int c_hi = fixed ? 1 : b->max_ctas_per_sm;
    for (int c = 1; c <= c_hi && err == cudaSuccess; ++c)
      for (int k : chunks) {
        if (fixed && k != 1) continue;
        err = launch_batch(b, phases, c, k, mode, st);  // warm-up
        float ms_best = 1e30f;
        for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
          cudaEventRecord(e0, st);
          err = launch_batch(b, phases, c, k, mode, st);
          cudaEventRecord(e1, st);
          if (err == cudaSuccess) err = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
          ms_best = std::min(ms_best, ms);
        }
        if (err != cudaSuccess) break;
        if (ms_best < best) {
          best = ms_best;
          best_c = c;
          best_k = k;
          best_m = mode;
        }
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    fem::set_last_error("fem_batch_tune: %s", cudaGetErrorString(err));
    return FEM_ERR_CUDA;
  }
  b->ctas_per_sm = best_c;
  b->chunk = best_k;
  b->mode = best_m;
  return FEM_OK;
}

fem_status fem_batch_config(const fem_batch* b, int32_t* ctas_per_sm, int32_t* chunk, int32_t* mode) {
  if (!b) {
    fem::set_last_error("batch is NULL");
    return FEM_ERR_ARG;
  }
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (chunk) *chunk = b->chunk;
  if (mode) *mode = b->mode;
  return FEM_OK;
}

fem_status fem_batch_set_config(fem_batch* b, int32_t ctas_per_sm, int32_t chunk, int32_t mode) {
  if (!b || !valid_config(ctas_per_sm, chunk, mode)) {
    fem::set_last_error("fem_batch_set_config: bad batch or configuration (ctas_per_sm 1..32, chunk 1..64, "
                        "mode FEM_BATCH_*)");
    return FEM_ERR_ARG;
  }
  if (b->has_coupling && mode != FEM_BATCH_PER_ITEM && mode != FEM_BATCH_PER_ITEM_CONCURRENT) {
    fem::set_last_error("fem_batch_set_config: a batch with a coupling-block item runs the per-item modes only");
    return FEM_ERR_UNSUPPORTED;
  }
  if ((mode == FEM_BATCH_GROUPED || mode == FEM_BATCH_GROUPED_CONCURRENT) && b->groups.empty())
    mode = FEM_BATCH_SINGLE;
  b->ctas_per_sm = ctas_per_sm;
  b->chunk = chunk;
  b->mode = mode;
  return FEM_OK;
}

fem_status fem_batch_errors(const fem_batch* b, int32_t* err_host, void* stream) {
  if (!b || !err_host) {
    fem::set_last_error("fem_batch_errors: NULL argument");
    return FEM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(err_host, &b->d_ctr->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    fem::set_last_error("fem_batch_errors: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  return FEM_OK;
}

fem_status fem_batch_inject_wait(fem_batch* b, int32_t item, int64_t extra_tiles, uint32_t spin_limit,
                                 void* stream) {
  if (!b || item < 0 || item >= b->n_items || extra_tiles < 0) {
    fem::set_last_error("fem_batch_inject_wait: bad batch, item or extra_tiles");
    return FEM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t want = b->desc[size_t(item)].n_tiles + extra_tiles;
  b->desc[size_t(item)].wait_tiles = want;
  if (b->kpos[size_t(item)] >= 0) b->kdesc[size_t(b->kpos[size_t(item)])].wait_tiles = want;
  b->spin_limit = spin_limit ? spin_limit : fem::kSpinLimit;
  cudaError_t e = cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(fem::BatchMesh) * b->desc.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !b->kdesc.empty())
    e = cudaMemcpyAsync(b->d_kdesc, b->kdesc.data(), sizeof(fem::BatchMesh) * b->kdesc.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host tables are reused by later calls
  if (e != cudaSuccess) {
    fem::set_last_error("fem_batch_inject_wait: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  return FEM_OK;
}

void fem_batch_destroy(fem_batch* b) { delete b; }

}  // extern "C"
