// fem_fwd.cuh -- forward element integration kernel (Knepley & Terrel, Sec. 4).
//
// Work decomposition (GB300 design, not the paper's GTX285 thread-per-entry
// mapping): a warp owns a tile of 32 consecutive elements, one element per
// lane.  Each lane gathers its connectivity (one 16-byte load for a tet) and
// vertex coordinates (L2-resident), builds the Jacobian, the geometric tensor
// and the sparse contraction with K as immediates, and writes its element
// matrix into a per-warp shared-memory stage (odd row stride: conflict-free).
// The warp then streams the tile's 32 * n^2 contiguous outputs to HBM with
// coalesced 16-byte evict-first stores -- the paper's "fully coalesced write"
// of element matrices (Sec. 4.3), done for a whole warp tile at once.  Warps
// walk the tile space grid-stride; the grid is sized from the SM count.
// Every element is integrated: the final tile is partial (no dropped tail).
#pragma once
#include <cuda_runtime.h>

#include "fem_core.cuh"
#include "fem_internal.h"

namespace fem {

template <class CT, class OT>
struct FwdParams {
  const int32_t* conn;
  const CT* coords;
  const float* coef;
  OT* A;
  int64_t n_elem;
  int64_t n_vert;
  int32_t* dev_err;
  int vec_conn;   // conn rows are 16-byte aligned int4 (tets)
  int vec_store;  // A is 16-byte aligned and n^2 % 4 == 0
};

template <int NN>
constexpr int stage_stride() {
  return NN | 1;
}

template <int N, int SST, class OT>
struct StageSink {
  OT* row;
  template <int I, int J>
  __device__ __forceinline__ void put(OT v) {
    row[I * N + J] = v;
    if constexpr (I != J) row[J * N + I] = v;
  }
};

template <int D>
__device__ __forceinline__ void load_conn(const int32_t* conn, int64_t e, int vec, int (&v)[D + 1]) {
  if constexpr (D == 3) {
    if (vec) {
      int4 c = __ldcs(reinterpret_cast<const int4*>(conn) + e);
      v[0] = c.x;
      v[1] = c.y;
      v[2] = c.z;
      v[3] = c.w;
      return;
    }
  }
#pragma unroll
  for (int k = 0; k <= D; ++k) v[k] = __ldcs(conn + e * (D + 1) + k);
}

template <int D, class CT>
__device__ __forceinline__ bool gather(const CT* coords, int64_t n_vert, const int (&v)[D + 1],
                                       CT (&X)[D + 1][D]) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k <= D; ++k) ok &= (v[k] >= 0) & (int64_t(v[k]) < n_vert);
  if (!ok) return false;
#pragma unroll
  for (int k = 0; k <= D; ++k)
#pragma unroll
    for (int a = 0; a < D; ++a) X[k][a] = __ldg(coords + int64_t(v[k]) * D + a);
  return true;
}

// One warp tile: returns the device error bits of its elements.
template <int D, int FORM, int JAC, class CT, class OT>
__device__ __forceinline__ int fwd_warp_tile(const FwdParams<CT, OT>& p, int64_t tile, int lane,
                                             OT* st) {
  using FT = FormTraits<D, FORM>;
  using GT = typename std::conditional<JAC == JAC_F64, double, float>::type;
  constexpr int NN = FT::NN;
  constexpr int SST = stage_stride<NN>();
  const int64_t e = tile * 32 + lane;
  int err = 0;
  OT Gf[FT::NG];
#pragma unroll
  for (int g = 0; g < FT::NG; ++g) Gf[g] = OT(0);
  if (e < p.n_elem) {
    int v[D + 1];
    CT X[D + 1][D];
    load_conn<D>(p.conn, e, p.vec_conn, v);
    if (!gather<D>(p.coords, p.n_vert, v, X)) {
      err |= DEVERR_CONN;
    } else {
      Jac<D, GT> jac;
      if (!jacobian<D, JAC>(X, jac)) {
        err |= DEVERR_DEGENERATE;
      } else {
        GT w = p.coef ? GT(__ldg(p.coef + e)) : GT(1);
        GT scale = w / (dev_abs(jac.det) * GT(FT::DEN));
        GT Gt[FT::NG];
        geometric_tensor<D, FORM>(jac.adj, scale, Gt);
#pragma unroll
        for (int g = 0; g < FT::NG; ++g) Gf[g] = OT(Gt[g]);
      }
    }
  }
  StageSink<FT::N, SST, OT> sink{st + lane * SST};
  contract<D, FORM>(Gf, sink);
  __syncwarp();
  const int64_t e0 = tile * 32;
  const int cnt = int(p.n_elem - e0 < 32 ? p.n_elem - e0 : 32);
  OT* dst = p.A + e0 * NN;
  bool done = false;
  if constexpr (sizeof(OT) == 4 && NN % 4 == 0) {
    if (p.vec_store) {
      const int nq = cnt * (NN / 4);
      for (int q = lane; q < nq; q += 32) {
        const int idx = 4 * q;
        const int el = idx / NN;
        const OT* s = st + el * SST + (idx - el * NN);
        __stcs(reinterpret_cast<float4*>(dst) + q, make_float4(s[0], s[1], s[2], s[3]));
      }
      done = true;
    }
  }
  if (!done) {
    const int nw = cnt * NN;
    for (int idx = lane; idx < nw; idx += 32) {
      const int el = idx / NN;
      __stcs(dst + idx, st[el * SST + (idx - el * NN)]);
    }
  }
  __syncwarp();
  return err;
}

template <int D, int FORM, int JAC, class CT, class OT>
__global__ void __launch_bounds__(512) fem_fwd_kernel(FwdParams<CT, OT> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int SST = stage_stride<FormTraits<D, FORM>::NN>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  OT* st = reinterpret_cast<OT*>(smem_raw) + warp * 32 * SST;
  const int64_t ntiles = (p.n_elem + 31) / 32;
  int err = 0;
  for (int64_t t = int64_t(blockIdx.x) * nwarps + warp; t < ntiles; t += int64_t(gridDim.x) * nwarps)
    err |= fwd_warp_tile<D, FORM, JAC>(p, t, lane, st);
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

template <int D, int FORM, int JAC, class CT, class OT>
cudaError_t launch_fwd_t(const FwdLaunch& L) {
  using FT = FormTraits<D, FORM>;
  FwdParams<CT, OT> p;
  p.conn = L.conn;
  p.coords = static_cast<const CT*>(L.coords);
  p.coef = L.coef;
  p.A = static_cast<OT*>(L.A);
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(L.conn) % 16 == 0);
  p.vec_store = (reinterpret_cast<uintptr_t>(L.A) % 16 == 0);
  auto kern = fem_fwd_kernel<D, FORM, JAC, CT, OT>;
  const int warps = clamp_warps(L.warps, size_t(32) * stage_stride<FT::NN>() * sizeof(OT));
  const size_t smem = size_t(warps) * 32 * stage_stride<FT::NN>() * sizeof(OT);
  cudaError_t st = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (st != cudaSuccess) return st;
  const int64_t ntiles = (L.n_elem + 31) / 32;
  int64_t grid = (ntiles + warps - 1) / warps;
  if (L.ctas_per_sm > 0) {
    int64_t cap = int64_t(L.ctas_per_sm) * device_sm_count();
    if (grid > cap) grid = cap;
  }
  if (grid < 1) grid = 1;
  kern<<<unsigned(grid), warps * 32, smem, L.stream>>>(p);
  return cudaGetLastError();
}

// Dispatch one (D, FORM) over the precision combinations the ABI accepts.
template <int D, int FORM>
cudaError_t launch_fwd_form(const FwdLaunch& L) {
  if (!L.coord_f64) {
    if (!L.out_f64) {
      switch (L.jac) {
        case JAC_COMP: return launch_fwd_t<D, FORM, JAC_COMP, float, float>(L);
        case JAC_F64: return launch_fwd_t<D, FORM, JAC_F64, float, float>(L);
        case JAC_F32: return launch_fwd_t<D, FORM, JAC_F32, float, float>(L);
        default: return cudaErrorInvalidValue;
      }
    }
    return launch_fwd_t<D, FORM, JAC_F64, float, double>(L);
  }
  if (!L.out_f64) return launch_fwd_t<D, FORM, JAC_F64, double, float>(L);
  return launch_fwd_t<D, FORM, JAC_F64, double, double>(L);
}

}  // namespace fem
