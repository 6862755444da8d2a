// fem_bwd.cu -- adjoint (reverse mode) of the element integration, element part.
//
// For L = sum_e <dA_e, A_e> with A_e = G_e : K (Eq. 6) and
// G_e = (w_e / (|det J| DEN)) * products of adj(J) (Eq. 8 / Eq. 15 with the
// symmetric-gradient reading), each lane of a warp handles one element:
//   1. dG[g]   = sum_{i<=j} s_ij K'[g][i][j],  s_ii = dA_ii, s_ij = dA_ij + dA_ji
//                (transpose of the sparse contraction, K' as immediates)
//   2. dw_e    = sum_g dG[g] G0[g]             (G0 = G without w; A is linear in w)
//   3. L_e     = w_e dw_e,  c = w_e / (|det J| DEN)
//      Laplacian   d adj_{rho a} = 2c sum_nu S_{rho nu} adj_{nu a}
//      elasticity  d adj_p      = 2c sum_q S_pq adj_q          (p = (mu a) flattened)
//      with S the symmetric matrix of dG (off-diagonal entries halved)
//   4. |det J| enters as 1/|det J|:  d e_mu += -(L_e / det J) adj_mu   (d det / d e_mu = adj_mu)
//   5. adj_mu = e_{mu+1} x e_{mu+2} (3D; rotated edges in 2D) is pulled back to the
//      edge vectors, then x_{mu+1} += d e_mu and x_0 -= sum_mu d e_mu.
// The per-vertex contributions go either to a per-element scratch buffer
// [E][d+1][d] (deterministic segmented reduction afterwards) or straight into
// dcoords with red.global.add (atomic variant).  dA is read through the same
// per-warp shared-memory stage as the forward stores, with coalesced 16-byte loads.
#include "fem_core.cuh"
#include "fem_fwd.cuh"
#include "fem_internal.h"

namespace fem {

template <int T, int N>
struct TriIdx {
  static constexpr int i = tri_row(T, N);
  static constexpr int j = tri_col(T, N);
};

template <int NT>
struct SymVals {
  float s[NT];
  template <int T>
  __device__ __forceinline__ float get() const {
    return s[T];
  }
};

template <int N, int... Ts>
__device__ __forceinline__ void load_sym(const float* row, float* s, std::integer_sequence<int, Ts...>) {
  ((s[Ts] = (TriIdx<Ts, N>::i == TriIdx<Ts, N>::j)
                ? row[TriIdx<Ts, N>::i * N + TriIdx<Ts, N>::j]
                : row[TriIdx<Ts, N>::i * N + TriIdx<Ts, N>::j] + row[TriIdx<Ts, N>::j * N + TriIdx<Ts, N>::i]),
   ...);
}

struct BwdParams {
  const int32_t* conn;
  const float* coords;
  const float* coef;
  const float* dA;
  float* dcoef;
  float* xbar;
  float* dcoords;
  int64_t n_elem;
  int64_t n_vert;
  int32_t* dev_err;
  int vec_conn;
  int vec_dA;
  int vec_xbar;
};

template <int D, int FORM, int JAC, bool ATOMIC>
__device__ __forceinline__ int bwd_warp_tile(const BwdParams& p, int64_t tile, int lane, float* st) {
  using FT = FormTraits<D, FORM>;
  using GT = typename std::conditional<JAC == JAC_F64, double, float>::type;
  constexpr int N = FT::N, NN = FT::NN, NV = FT::NV;
  constexpr int SST = stage_stride<NN>();
  constexpr int NX = NV * D;
  constexpr int SSX = NX | 1;
  const int64_t e0 = tile * 32;
  const int cnt = int(p.n_elem - e0 < 32 ? p.n_elem - e0 : 32);
  // 1. stage the tile's upstream dA (contiguous cnt * NN floats)
  {
    const float* src = p.dA + e0 * NN;
    bool done = false;
    if constexpr (NN % 4 == 0) {
      if (p.vec_dA) {
        const int nq = cnt * (NN / 4);
        for (int q = lane; q < nq; q += 32) {
          float4 v = __ldcs(reinterpret_cast<const float4*>(src) + q);
          const int idx = 4 * q;
          const int el = idx / NN;
          float* d = st + el * SST + (idx - el * NN);
          d[0] = v.x;
          d[1] = v.y;
          d[2] = v.z;
          d[3] = v.w;
        }
        done = true;
      }
    }
    if (!done) {
      const int nw = cnt * NN;
      for (int idx = lane; idx < nw; idx += 32) {
        const int el = idx / NN;
        st[el * SST + (idx - el * NN)] = __ldcs(src + idx);
      }
    }
  }
  __syncwarp();
  const int64_t e = e0 + lane;
  int err = 0;
  float xb[NV][D];
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int a = 0; a < D; ++a) xb[k][a] = 0.f;
  float dcoef = 0.f;
  int v[D + 1];
  bool ok = false;
  if (e < p.n_elem) {
    float X[D + 1][D];
    load_conn<D>(p.conn, e, p.vec_conn, v);
    if (!gather<D>(p.coords, p.n_vert, v, X)) {
      err |= DEVERR_CONN;
    } else {
      Jac<D, GT> jac;
      if (!jacobian<D, JAC>(X, jac)) {
        err |= DEVERR_DEGENERATE;
      } else {
        ok = true;
        float adj[D][D], ed[D][D];
#pragma unroll
        for (int mu = 0; mu < D; ++mu)
#pragma unroll
          for (int a = 0; a < D; ++a) {
            adj[mu][a] = float(jac.adj[mu][a]);
            ed[mu][a] = float(jac.e[mu][a]);
          }
        const float det = float(jac.det);
        const float scale0 = 1.f / (dev_abs(det) * float(FT::DEN));
        float G0[FT::NG];
        geometric_tensor<D, FORM>(adj, scale0, G0);
        // 1. dG = transpose of the contraction applied to sym(dA)
        SymVals<FT::NT> sym;
        load_sym<N>(st + lane * SST, sym.s, std::make_integer_sequence<int, FT::NT>{});
        float dG[FT::NG];
        contract_adjoint<D, FORM>(sym, dG);
        // 2. coefficient gradient
#pragma unroll
        for (int g = 0; g < FT::NG; ++g) dcoef = fmaf(dG[g], G0[g], dcoef);
        const float w = p.coef ? __ldg(p.coef + e) : 1.f;
        const float L = w * dcoef;
        const float c2 = 2.f * w * scale0;
        // 3. adjoint of G with respect to adj(J)
        float adjb[D][D];
        if constexpr (FORM != ELASTIC_P1) {
#pragma unroll
          for (int r = 0; r < D; ++r)
#pragma unroll
            for (int a = 0; a < D; ++a) {
              float acc = 0.f;
#pragma unroll
              for (int nu = 0; nu < D; ++nu) {
                const float Srn = (r == nu) ? dG[pair_index(r, nu, D)]
                                            : 0.5f * dG[pair_index(r < nu ? r : nu, r < nu ? nu : r, D)];
                acc = fmaf(Srn, adj[nu][a], acc);
              }
              adjb[r][a] = c2 * acc;
            }
        } else {
          constexpr int NP = FT::NP;
#pragma unroll
          for (int pp = 0; pp < NP; ++pp) {
            float acc = 0.f;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
              const float Spq = (pp == q) ? dG[pair_index(pp, q, NP)]
                                          : 0.5f * dG[pair_index(pp < q ? pp : q, pp < q ? q : pp, NP)];
              acc = fmaf(Spq, adj[q / D][q % D], acc);
            }
            adjb[pp / D][pp % D] = c2 * acc;
          }
        }
        // 4. |det J| term and 5. adjugate pulled back to the edge vectors
        float eb[D][D];
        const float Ld = -L / det;
#pragma unroll
        for (int mu = 0; mu < D; ++mu)
#pragma unroll
          for (int a = 0; a < D; ++a) eb[mu][a] = Ld * adj[mu][a];
        if constexpr (D == 3) {
#pragma unroll
          for (int mu = 0; mu < 3; ++mu) {
            const int i1 = (mu + 1) % 3, i2 = (mu + 2) % 3;
            const float* a = ed[i1];
            const float* b = ed[i2];
            const float* cb = adjb[mu];
            // d a += b x cb ; d b += cb x a
            eb[i1][0] += b[1] * cb[2] - b[2] * cb[1];
            eb[i1][1] += b[2] * cb[0] - b[0] * cb[2];
            eb[i1][2] += b[0] * cb[1] - b[1] * cb[0];
            eb[i2][0] += cb[1] * a[2] - cb[2] * a[1];
            eb[i2][1] += cb[2] * a[0] - cb[0] * a[2];
            eb[i2][2] += cb[0] * a[1] - cb[1] * a[0];
          }
        } else {
          eb[1][1] += adjb[0][0];
          eb[1][0] -= adjb[0][1];
          eb[0][1] -= adjb[1][0];
          eb[0][0] += adjb[1][1];
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float s = 0.f;
#pragma unroll
          for (int mu = 0; mu < D; ++mu) {
            xb[mu + 1][a] = eb[mu][a];
            s += eb[mu][a];
          }
          xb[0][a] = -s;
        }
      }
    }
    if (p.dcoef) __stcs(p.dcoef + e, dcoef);
  }
  if constexpr (ATOMIC) {
    if (ok) {
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int a = 0; a < D; ++a) atomicAdd(p.dcoords + int64_t(v[k]) * D + a, xb[k][a]);
    }
    __syncwarp();
  } else if (p.xbar) {
    __syncwarp();  // every lane has read its dA row: reuse the stage for xbar
    float* row = st + lane * SSX;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int a = 0; a < D; ++a) row[k * D + a] = xb[k][a];
    __syncwarp();
    float* dst = p.xbar + e0 * NX;
    bool done = false;
    if constexpr (NX % 4 == 0) {
      if (p.vec_xbar) {
        const int nq = cnt * (NX / 4);
        for (int q = lane; q < nq; q += 32) {
          const int idx = 4 * q;
          const int el = idx / NX;
          const float* s = st + el * SSX + (idx - el * NX);
          reinterpret_cast<float4*>(dst)[q] = make_float4(s[0], s[1], s[2], s[3]);
        }
        done = true;
      }
    }
    if (!done) {
      const int nw = cnt * NX;
      for (int idx = lane; idx < nw; idx += 32) {
        const int el = idx / NX;
        dst[idx] = st[el * SSX + (idx - el * NX)];
      }
    }
    __syncwarp();
  }
  return err;
}

template <int D, int FORM, int JAC, bool ATOMIC>
__global__ void __launch_bounds__(512) fem_bwd_elem_kernel(BwdParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using FT = FormTraits<D, FORM>;
  constexpr int SST = stage_stride<FT::NN>() > ((FT::NV * D) | 1) ? stage_stride<FT::NN>()
                                                                   : ((FT::NV * D) | 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  float* st = reinterpret_cast<float*>(smem_raw) + warp * 32 * SST;
  const int64_t ntiles = (p.n_elem + 31) / 32;
  int err = 0;
  for (int64_t t = int64_t(blockIdx.x) * nwarps + warp; t < ntiles; t += int64_t(gridDim.x) * nwarps)
    err |= bwd_warp_tile<D, FORM, JAC, ATOMIC>(p, t, lane, st);
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

template <int D, int FORM, int JAC, bool ATOMIC>
static cudaError_t launch_bwd_t(const BwdLaunch& L) {
  using FT = FormTraits<D, FORM>;
  constexpr int SST = stage_stride<FT::NN>() > ((FT::NV * D) | 1) ? stage_stride<FT::NN>()
                                                                   : ((FT::NV * D) | 1);
  BwdParams p;
  p.conn = L.conn;
  p.coords = L.coords;
  p.coef = L.coef;
  p.dA = L.dA;
  p.dcoef = L.dcoef;
  p.xbar = L.xbar;
  p.dcoords = L.dcoords;
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(L.conn) % 16 == 0);
  p.vec_dA = reinterpret_cast<uintptr_t>(L.dA) % 16 == 0;
  p.vec_xbar = reinterpret_cast<uintptr_t>(L.xbar) % 16 == 0;
  auto kern = fem_bwd_elem_kernel<D, FORM, JAC, ATOMIC>;
  const int warps = clamp_warps(L.warps, size_t(32) * SST * sizeof(float));
  const size_t smem = size_t(warps) * 32 * SST * sizeof(float);
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

template <int D, int FORM>
static cudaError_t launch_bwd_form(const BwdLaunch& L) {
  switch (L.jac) {
    case JAC_COMP:
      return L.atomic ? launch_bwd_t<D, FORM, JAC_COMP, true>(L) : launch_bwd_t<D, FORM, JAC_COMP, false>(L);
    case JAC_F64:
      return L.atomic ? launch_bwd_t<D, FORM, JAC_F64, true>(L) : launch_bwd_t<D, FORM, JAC_F64, false>(L);
    case JAC_F32:
      return L.atomic ? launch_bwd_t<D, FORM, JAC_F32, true>(L) : launch_bwd_t<D, FORM, JAC_F32, false>(L);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_bwd_elem(const BwdLaunch& L) {
  if (L.dim == 2) {
    switch (L.form) {
      case LAPLACE_P1: return launch_bwd_form<2, LAPLACE_P1>(L);
      case LAPLACE_P2: return launch_bwd_form<2, LAPLACE_P2>(L);
      case ELASTIC_P1: return launch_bwd_form<2, ELASTIC_P1>(L);
    }
  } else {
    switch (L.form) {
      case LAPLACE_P1: return launch_bwd_form<3, LAPLACE_P1>(L);
      case LAPLACE_P2: return launch_bwd_form<3, LAPLACE_P2>(L);
      case ELASTIC_P1: return launch_bwd_form<3, ELASTIC_P1>(L);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace fem
