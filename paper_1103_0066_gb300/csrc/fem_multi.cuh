// fem_multi.cuh -- the forward, the adjoint element pass and the vertex
// reduction over many meshes of one (dim, form) kind, one launch each.
//
// The 32-element tiles of the kind's meshes are numbered one mesh after the
// other: mesh m holds tiles [tile_begin[m], tile_begin[m + 1]).  Warp w of the
// S resident warps takes tiles w, w + S, w + 2S, ... of that numbering, and
// the single-mesh kernels' software pipeline (connectivity two tiles ahead,
// coordinates and dA one tile ahead) keeps running across mesh boundaries:
// every pipeline stage carries the mesh of its tile and reads that mesh's
// parameters from the kernel's parameter block.  The per-tile code is the
// single-mesh kernels' (fwd_compute_tile, bwd_compute_tile, warp_records,
// reduce_vertex_*), so each mesh's results are those of its single-mesh
// launches, bit for bit.  A small mesh then takes a few warps' steps inside a
// launch that fills the GPU, instead of a launch of its own.
#pragma once

#include "fem_bwd.cuh"
#include "fem_fwd.cuh"
#include "fem_reduce.cuh"

namespace fem {

constexpr int kMultiMeshes = 32;  // meshes per launch (the parameter block stays below 8 KB)
constexpr int kMultiRedBlock = 256;

struct FwdMulti {
  int32_t n;
  int32_t* dev_err;
  int64_t tile_begin[kMultiMeshes + 1];
  FwdParams<float, float> p[kMultiMeshes];
};

struct BwdMulti {
  int32_t n;
  int32_t* dev_err;
  int64_t tile_begin[kMultiMeshes + 1];
  BwdParams p[kMultiMeshes];
};

struct RedMesh {
  const int32_t* voff;
  const int32_t* vrec;
  const int32_t* mode;
  const float* records;
  float* dcoords;
  int64_t n_vert;
};

struct RedMulti {
  int32_t n;
  int64_t blk_begin[kMultiMeshes + 1];  // kMultiRedBlock-vertex blocks
  RedMesh r[kMultiMeshes];
};

// The mesh of tile g, searching forward from mesh m (g never decreases along
// a warp's tiles).  Past the last tile: the last mesh, whose local tile index
// is then beyond its elements, so every load of that stage is masked.
__device__ __forceinline__ int multi_mesh_at(const int64_t* tile_begin, int n, int m, int64_t g) {
  while (m < n - 1 && g >= tile_begin[m + 1]) ++m;
  return m;
}

// One pipeline step of the multi-mesh forward: connectivity of tile g + 2S,
// coordinates and coefficient of tile g + S, then tile g computed and stored.
template <int D, int FORM, int JAC>
__device__ __forceinline__ void fwd_multi_step(const FwdMulti& P, int64_t g, int64_t S, int lane, int& m0, int& m1,
                                               const int (&vnext)[D + 1], int (&vload)[D + 1],
                                               const float (&Xcur)[D + 1][D], float (&Xnext)[D + 1][D], int fcur,
                                               const Coef<FormTraits<D, FORM>::NW>& wcur, int& fnext,
                                               Coef<FormTraits<D, FORM>::NW>& wnext, float* st, int& err) {
  const int m2 = multi_mesh_at(P.tile_begin, P.n, m1, g + 2 * S);
  {
    const FwdParams<float, float>& p = P.p[m2];
    load_conn<D>(p.conn, (g + 2 * S - P.tile_begin[m2]) * 32 + lane, p.n_elem, p.vec_conn, vload);
  }
  {
    const FwdParams<float, float>& p = P.p[m1];
    const int64_t en = (g + S - P.tile_begin[m1]) * 32 + lane;
    fnext = gather_regs<D>(p.coords, p.n_vert, en, p.n_elem, vnext, Xnext);
    load_coef<D, FORM>(p.coef, en, p.n_elem, p.n_vert, vnext, wnext);
  }
  err |= fwd_compute_tile<D, FORM, JAC, float, float, false>(P.p[m0], g - P.tile_begin[m0], lane, fcur, wcur, Xcur,
                                                             st);
  m0 = m1;
  m1 = m2;
}

template <int D, int FORM, int JAC>
__global__ void __launch_bounds__(FwdShape<D, FORM, JAC, float, float>::threads,
                                  FwdShape<D, FORM, JAC, float, float>::min_ctas)
    fem_fwd_multi_kernel(const __grid_constant__ FwdMulti P) {
  using PL = FwdPlan<D, FORM, float, float>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  float* st = reinterpret_cast<float*>(smem_raw + size_t(warp) * PL::per_warp);
  const int64_t T = P.tile_begin[P.n];
  const int64_t S = int64_t(gridDim.x) * nwarps;
  int64_t g = int64_t(blockIdx.x) * nwarps + warp;
  if (g >= T) return;  // warp-uniform
  int err = 0;
  int va[D + 1], vb[D + 1];
  float Xa[D + 1][D], Xb[D + 1][D];
  int fa, fb;
  Coef<FormTraits<D, FORM>::NW> wa, wb;
  int m0 = multi_mesh_at(P.tile_begin, P.n, 0, g);
  int m1 = multi_mesh_at(P.tile_begin, P.n, m0, g + S);
  {  // prologue: tile g gathered, tile g + S's connectivity in flight
    const FwdParams<float, float>& p = P.p[m0];
    const int64_t e = (g - P.tile_begin[m0]) * 32 + lane;
    load_conn<D>(p.conn, e, p.n_elem, p.vec_conn, va);
    fa = gather_regs<D>(p.coords, p.n_vert, e, p.n_elem, va, Xa);
    load_coef<D, FORM>(p.coef, e, p.n_elem, p.n_vert, va, wa);
  }
  {
    const FwdParams<float, float>& p = P.p[m1];
    load_conn<D>(p.conn, (g + S - P.tile_begin[m1]) * 32 + lane, p.n_elem, p.vec_conn, va);
  }
  for (;;) {
    fwd_multi_step<D, FORM, JAC>(P, g, S, lane, m0, m1, va, vb, Xa, Xb, fa, wa, fb, wb, st, err);
    if ((g += S) >= T) break;
    fwd_multi_step<D, FORM, JAC>(P, g, S, lane, m0, m1, vb, va, Xb, Xa, fb, wb, fa, wa, st, err);
    if ((g += S) >= T) break;
  }
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && P.dev_err) atomicOr(P.dev_err, err);
}

// The multi-mesh adjoint element pass: the single-mesh kernel's pipeline with
// a mesh per stage (tile g computes with mesh m0; tile g + S, mesh m1, has its
// coordinates, dA, coefficient, saved det J and record range in flight; tile
// g + 2S, mesh m2, its connectivity).  A mesh without records (no dcoords
// wanted) skips the record stage, as its single-mesh launch does.
template <int D, int FORM, int JAC>
__global__ void __launch_bounds__(BwdShape<D, FORM, JAC>::threads, BwdShape<D, FORM, JAC>::min_ctas)
    fem_bwd_multi_kernel(const __grid_constant__ BwdMulti P) {
  using PL = BwdPlan<D, FORM>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  unsigned char* wbase = smem_raw + size_t(warp) * PL::per_warp;
  auto dslot = [&](int s) { return reinterpret_cast<float*>(wbase + size_t(s) * (PL::da_slot + PL::xs_over)); };
  auto xstage = [&](int s) { return reinterpret_cast<float*>(wbase + size_t(s) * PL::da_slot); };
  const int64_t T = P.tile_begin[P.n];
  const int64_t S = int64_t(gridDim.x) * nwarps;
  int64_t g = int64_t(blockIdx.x) * nwarps + warp;
  if (g >= T) return;  // warp-uniform: the kernel has no CTA-wide barrier
  int err = 0;
  int v1[D + 1], v2[D + 1], vc[D + 1];
  float Xc[D + 1][D], Xn[D + 1][D];
  Coef<FormTraits<D, FORM>::NW> wcur, wnext;
  float dcur = 0.f;
  uint32_t rkcur = 0;
  int32_t rb = 0, rn = 0;
  int fcur;
  int m0 = multi_mesh_at(P.tile_begin, P.n, 0, g);
  {
    const BwdParams& p = P.p[m0];
    const int64_t t = g - P.tile_begin[m0], e = t * 32 + lane;
    load_conn<D>(p.conn, e, p.n_elem, p.vec_conn, v1);
    fcur = gather_regs<D>(p.coords, p.n_vert, e, p.n_elem, v1, Xc);
    copy_dA_async<D, FORM>(p, t, lane, dslot(0));
    load_coef<D, FORM>(p.coef, e, p.n_elem, p.n_vert, v1, wcur);
    if constexpr (JAC == JAC_SAVED) dcur = e < p.n_elem ? __ldg(p.det + e) : 0.f;
    if (p.tile_rec) {
      rkcur = __ldg(p.rank + e);
      rb = __ldg(p.tile_rec + t);
      rn = __ldg(p.tile_rec + t + 1) - rb;
    }
  }
  cp_async_commit();
#pragma unroll
  for (int k = 0; k <= D; ++k) vc[k] = v1[k];
  int m1 = multi_mesh_at(P.tile_begin, P.n, m0, g + S);
  {
    const BwdParams& p = P.p[m1];
    load_conn<D>(p.conn, (g + S - P.tile_begin[m1]) * 32 + lane, p.n_elem, p.vec_conn, v1);
  }
  for (int i = 0; g < T; ++i, g += S) {
    const int sn = (i + 1) & 1, sc = i & 1;
    const int m2 = multi_mesh_at(P.tile_begin, P.n, m1, g + 2 * S);
    {
      const BwdParams& p = P.p[m2];
      load_conn<D>(p.conn, (g + 2 * S - P.tile_begin[m2]) * 32 + lane, p.n_elem, p.vec_conn, v2);
    }
    int fnext;
    float dnext = 0.f;
    uint32_t rknext = 0;
    int32_t rbn = 0, rnn = 0;
    {
      const BwdParams& p = P.p[m1];
      const int64_t tn = g + S - P.tile_begin[m1], en = tn * 32 + lane;
      fnext = gather_regs<D>(p.coords, p.n_vert, en, p.n_elem, v1, Xn);
      copy_dA_async<D, FORM>(p, tn, lane, dslot(sn));
      load_coef<D, FORM>(p.coef, en, p.n_elem, p.n_vert, v1, wnext);
      if constexpr (JAC == JAC_SAVED) dnext = en < p.n_elem ? __ldg(p.det + en) : 0.f;
      if (p.tile_rec && tn * 32 < p.n_elem) {
        rknext = __ldg(p.rank + en);
        rbn = __ldg(p.tile_rec + tn);
        rnn = __ldg(p.tile_rec + tn + 1) - rbn;
      }
    }
    const BwdParams& p = P.p[m0];
    const bool rec = p.tile_rec != nullptr;
    // this tile's record ends and destinations: in flight while the element math runs
    const RecAhead ah = rec ? load_rec_ahead(p.rec_span, p.rec_dest, rb, rn, lane) : RecAhead{0u, 0};
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();  // dA rows were copied by other lanes
    float* xs = xstage(sc);
    err |= bwd_compute_tile<D, FORM, JAC, false>(p, g - P.tile_begin[m0], lane, fcur, wcur, Xc,
                                                 dslot(sc) + lane * PL::DST, vc, rec ? xs : nullptr, rkcur, dcur);
    if (rec) {
      __syncwarp();  // every lane's contributions are staged
      warp_records<D, PL::NC>(xs, p.rec_span, p.rec_dest, rb, rn, ah, p.records, lane);
    }
    __syncwarp();  // the next tile's dA copy may overwrite this tile's stage
    fcur = fnext;
    wcur = wnext;
    dcur = dnext;
    rkcur = rknext;
    rb = rbn;
    rn = rnn;
    m0 = m1;
    m1 = m2;
#pragma unroll
    for (int k = 0; k <= D; ++k) {
      vc[k] = v1[k];
      v1[k] = v2[k];
#pragma unroll
      for (int a = 0; a < D; ++a) Xc[k][a] = Xn[k][a];
    }
  }
  cp_async_wait<0>();
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && P.dev_err) atomicOr(P.dev_err, err);
}

// The multi-mesh vertex reduction: one block per kMultiRedBlock vertices of
// one mesh (blocks numbered one mesh after the other), the mesh found by a
// binary search of the block offsets; each vertex summed as in the
// single-mesh reduction.
template <int D>
__global__ void __launch_bounds__(kMultiRedBlock) vertex_reduce_multi_kernel(const __grid_constant__ RedMulti P) {
  const int64_t b = blockIdx.x;
  int lo = 0, hi = P.n - 1;  // the last mesh whose first block is <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.blk_begin[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  const RedMesh& R = P.r[lo];
  const int64_t v = (b - P.blk_begin[lo]) * kMultiRedBlock + threadIdx.x;
  if (v >= R.n_vert) return;
  if (__ldg(R.mode) == kRecTileOrder)
    reduce_vertex_gather<D, D>(R.voff, R.vrec, R.records, v, R.dcoords, nullptr);
  else
    reduce_vertex_direct<D, D>(R.voff, R.records, v, R.dcoords, nullptr);
}

// Host launchers, one translation unit per dimension (fem_multi_d2.cu,
// fem_multi_d3.cu): the forms LAPLACE_P1, LAPLACE_P2 and ELASTIC_P1; the
// adjoint with det J saved by the forward (saved_det) or recomputed.
cudaError_t launch_fwd_multi_d2(int form, const FwdMulti& P, cudaStream_t st);
cudaError_t launch_fwd_multi_d3(int form, const FwdMulti& P, cudaStream_t st);
cudaError_t launch_bwd_multi_d2(int form, bool saved_det, const BwdMulti& P, cudaStream_t st);
cudaError_t launch_bwd_multi_d3(int form, bool saved_det, const BwdMulti& P, cudaStream_t st);
cudaError_t launch_reduce_multi_d2(const RedMulti& P, cudaStream_t st);
cudaError_t launch_reduce_multi_d3(const RedMulti& P, cudaStream_t st);

// Launch geometry shared by both dimensions (host).
template <int D, int FORM, int JAC>
cudaError_t launch_fwd_multi_t(const FwdMulti& P, cudaStream_t st) {
  using PL = FwdPlan<D, FORM, float, float>;
  using SH = FwdShape<D, FORM, JAC, float, float>;
  const int64_t T = P.tile_begin[P.n];
  if (T == 0) return cudaSuccess;
  auto kern = fem_fwd_multi_kernel<D, FORM, JAC>;
  const int warps = clamp_warps(SH::default_warps, PL::per_warp);
  const size_t smem = size_t(warps) * PL::per_warp;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = pipeline_grid(reinterpret_cast<const void*>(kern), warps, smem, T * 32, 0);
  kern<<<grid, warps * 32, smem, st>>>(P);
  return cudaGetLastError();
}

template <int D, int FORM, int JAC>
cudaError_t launch_bwd_multi_t(const BwdMulti& P, cudaStream_t st) {
  using PL = BwdPlan<D, FORM>;
  const int64_t T = P.tile_begin[P.n];
  if (T == 0) return cudaSuccess;
  auto kern = fem_bwd_multi_kernel<D, FORM, JAC>;
  const int warps = clamp_warps(BwdShape<D, FORM, JAC>::threads / 32, PL::per_warp);
  const size_t smem = size_t(warps) * PL::per_warp;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = pipeline_grid(reinterpret_cast<const void*>(kern), warps, smem, T * 32, 0);
  kern<<<grid, warps * 32, smem, st>>>(P);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_reduce_multi_t(const RedMulti& P, cudaStream_t st) {
  const int64_t blocks = P.blk_begin[P.n];
  if (blocks == 0) return cudaSuccess;
  vertex_reduce_multi_kernel<D><<<unsigned(blocks), kMultiRedBlock, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace fem
