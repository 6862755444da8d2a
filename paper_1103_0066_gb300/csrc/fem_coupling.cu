// fem_coupling.cu -- the coupling block of a multiphysics pair and its adjoint.
//
// Sec. 6 of Knepley & Terrel plans systems of equations from multiphysics
// problems, with the weak form broken into blocks.  The off-diagonal block of
// a (scalar field q in P1, vector field v in [P1]^d or [P2]^d) pair is
//   B_{i,(c,j)} = int_T w phi_i d psi_j / d x_c = sum_mu G^{mu c} K^{ij}_mu
//   G^{mu c}    = w |J| J^{-1}_{mu c} = w sgn(det J) adj(J)_{mu c}
//   K^{ij}_mu   = int_ref lambda_i d_mu psi_j          (fem_forms.cuh: DivRef)
// -- Eq. 1 with a basis-function value and a derivative in K.  Rows i = 0..d,
// columns c * NBV + j.  G needs det J only for its sign, so the element
// matrix carries no 1/det J: the compensated determinant only decides the
// sign on slivers, and adj(J) (exact products of the FP32 edge vectors,
// rounded once) sets the accuracy.
//
// Forward: each warp walks 32-element tiles grid-stride with the affine
// kernel's pipeline (connectivity two tiles ahead, coordinates one tile ahead
// in registers); a lane forms its element's block, writes it as one row of a
// per-warp shared stage, and the warp stores the tile's contiguous rows with
// coalesced evict-first 16-byte stores.
//
// Adjoint, for an upstream dB: T^{mu c} = sum_{i,j} dB_{i,(c,j)} K^{ij}_mu,
//   dw      = sgn sum_{mu,c} T^{mu c} adj_{mu c}
//   d adj   = w sgn T           (no det J term: sgn is piecewise constant)
// then adj(J) is pulled back to the edge vectors and the vertices as in the
// Laplacian adjoint, and the vertex contributions go through the same
// deterministic record reduction (or red.global.add).
#include <cuda_runtime.h>

#include <utility>

#include "../../include/fem.h"
#include "fem_bwd.cuh"
#include "fem_core.cuh"
#include "fem_fwd.cuh"
#include "fem_internal.h"
#include "fem_pipe.cuh"

namespace fem {

namespace {

template <int D, int VDEG>
struct DivPlan {
  using T = DivTraits<D, VDEG>;
  static constexpr int NN = T::NN;
  static constexpr bool VEC = NN % 4 == 0;
  // A lane's row in the stage: 16-byte aligned rows of stride NN + 4 floats
  // (a quarter warp's 16-byte row accesses then hit eight different 16-byte
  // bank groups), or an odd stride for scalar rows.
  static constexpr int SST = VEC ? NN + 4 : (NN | 1);
  static constexpr size_t row_stage = align_up(size_t(32) * SST * 4, 128);
  static constexpr int XCAP = D == 3 ? kStageCap3 : kRecTile * (D + 1);
  static constexpr int XP = D == 3 ? 4 : 2;
  static constexpr size_t xs_bytes = align_up(size_t(XCAP) * XP * 4, 128);
  static constexpr size_t fwd_per_warp = row_stage;
  static constexpr size_t bwd_per_warp = 2 * row_stage + xs_bytes;
  static constexpr int threads = 128;  // four warps, no CTA-wide barrier
};

struct DivParams {
  const int32_t* conn;
  const float* coords;
  const float* coef;
  float* B;             // forward output [E][NN]
  float* det_out;       // forward: det J saved for the adjoint, or null
  const float* dB;      // adjoint input [E][NN]
  const float* det_in;  // adjoint: det J saved by the forward, or null
  float* dcoef;
  float* dcoords;  // atomic adjoint
  const int32_t* tile_rec;
  const uint32_t* rank;
  const uint16_t* rec_span;
  const int32_t* rec_dest;
  float* records;
  int64_t n_elem, n_vert;
  int32_t* dev_err;
  int vec_conn, vec_io;
};

// ---------------------------------------------------------------- contraction with K as immediates

template <int D, int VDEG, int T>
struct DivIdx {
  static constexpr int NBV = DivTraits<D, VDEG>::NBV;
  static constexpr int NCOL = DivTraits<D, VDEG>::NCOL;
  static constexpr int I = T / NCOL;
  static constexpr int C = (T % NCOL) / NBV;
  static constexpr int J = T % NBV;
};

template <int D, int VDEG, int I, int C, int J, int MU>
__device__ __forceinline__ void div_term(float& acc, const float (&sa)[D][D]) {
  constexpr int k = DivRef<D, VDEG>::K.v[MU][I][J];
  if constexpr (k == 1) {
    acc += sa[MU][C];
  } else if constexpr (k == -1) {
    acc -= sa[MU][C];
  } else if constexpr (k != 0) {
    acc = fmaf(sa[MU][C], float(k), acc);
  }
}

template <int D, int VDEG, int T, int... MUs>
__device__ __forceinline__ float div_entry(const float (&sa)[D][D], std::integer_sequence<int, MUs...>) {
  using X = DivIdx<D, VDEG, T>;
  float acc = 0.f;
  (div_term<D, VDEG, X::I, X::C, X::J, MUs>(acc, sa), ...);
  return acc;
}

// out[t] = B entry t (row-major) for sa[mu][c] = (w sgn / DEN) adj[mu][c]
template <int D, int VDEG, int... Ts>
__device__ __forceinline__ void div_contract(const float (&sa)[D][D], float* out, std::integer_sequence<int, Ts...>) {
  ((out[Ts] = div_entry<D, VDEG, Ts>(sa, std::make_integer_sequence<int, D>{})), ...);
}

// T^{MU C} = sum_{i,j} dB_{i,(C,j)} K^{ij}_MU, for the row dB
template <int D, int VDEG, int MU, int C, int IJ>
__device__ __forceinline__ void div_adj_term(float& acc, const float* row) {
  constexpr int NBV = DivTraits<D, VDEG>::NBV, NCOL = DivTraits<D, VDEG>::NCOL;
  constexpr int I = IJ / NBV, J = IJ % NBV;
  constexpr int k = DivRef<D, VDEG>::K.v[MU][I][J];
  if constexpr (k == 1) {
    acc += row[I * NCOL + C * NBV + J];
  } else if constexpr (k == -1) {
    acc -= row[I * NCOL + C * NBV + J];
  } else if constexpr (k != 0) {
    acc = fmaf(row[I * NCOL + C * NBV + J], float(k), acc);
  }
}

template <int D, int VDEG, int MC, int... IJs>
__device__ __forceinline__ float div_adj_entry(const float* row, std::integer_sequence<int, IJs...>) {
  float acc = 0.f;
  (div_adj_term<D, VDEG, MC / D, MC % D, IJs>(acc, row), ...);
  return acc;
}

template <int D, int VDEG, int... MCs>
__device__ __forceinline__ void div_contract_adjoint(const float* row, float (&Tg)[D][D],
                                                     std::integer_sequence<int, MCs...>) {
  constexpr int NIJ = (D + 1) * DivTraits<D, VDEG>::NBV;
  ((Tg[MCs / D][MCs % D] = div_adj_entry<D, VDEG, MCs>(row, std::make_integer_sequence<int, NIJ>{})), ...);
}

// ---------------------------------------------------------------- geometry

// Edge vectors, adj(J) and det J of one element (compensated det, or det as
// saved by the forward); false for det J == 0.
template <int D, bool SAVED>
__device__ __forceinline__ bool div_geometry(const float (&X)[D + 1][D], float det_saved, Jac<D, float>& jac) {
  if constexpr (SAVED)
    return jacobian_saved<D>(X, det_saved, jac);
  else
    return jacobian<D, JAC_COMP>(X, jac);
}

// ---------------------------------------------------------------- forward

template <int D, int VDEG>
__global__ void __launch_bounds__(DivPlan<D, VDEG>::threads) fem_div_fwd_kernel(DivParams p) {
  using PL = DivPlan<D, VDEG>;
  using TR = DivTraits<D, VDEG>;
  constexpr int NN = TR::NN, SST = PL::SST;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  float* st = reinterpret_cast<float*>(smem_raw + size_t(warp) * PL::fwd_per_warp);
  const int64_t ntiles = (p.n_elem + 31) / 32;
  const int64_t S = int64_t(gridDim.x) * nwarps;
  int64_t t = int64_t(blockIdx.x) * nwarps + warp;
  if (t >= ntiles) return;  // warp-uniform
  int err = 0;
  int v1[D + 1], v2[D + 1];
  float Xc[D + 1][D], Xn[D + 1][D];
  load_conn<D>(p.conn, t * 32 + lane, p.n_elem, p.vec_conn, v1);
  int fcur = gather_regs<D>(p.coords, p.n_vert, t * 32 + lane, p.n_elem, v1, Xc);
  float wcur = (p.coef && t * 32 + lane < p.n_elem) ? __ldg(p.coef + t * 32 + lane) : 1.f;
  load_conn<D>(p.conn, (t + S) * 32 + lane, p.n_elem, p.vec_conn, v1);
  for (; t < ntiles; t += S) {
    const int64_t en = (t + S) * 32 + lane;
    load_conn<D>(p.conn, (t + 2 * S) * 32 + lane, p.n_elem, p.vec_conn, v2);
    const int fnext = gather_regs<D>(p.coords, p.n_vert, en, p.n_elem, v1, Xn);
    const float wnext = (p.coef && en < p.n_elem) ? __ldg(p.coef + en) : 1.f;
    // this tile: geometry and the block, into the lane's stage row
    float sa[D][D];
#pragma unroll
    for (int mu = 0; mu < D; ++mu)
#pragma unroll
      for (int c = 0; c < D; ++c) sa[mu][c] = 0.f;
    const int64_t e = t * 32 + lane;
    if (fcur & GF_OK) {
      Jac<D, float> jac;
      const bool nondeg = div_geometry<D, false>(Xc, 0.f, jac);
      err |= nondeg ? 0 : DEVERR_DEGENERATE;
      if (p.det_out) __stcs(p.det_out + e, jac.det);
      const float scale = nondeg ? (jac.det > 0.f ? wcur : -wcur) * (1.f / float(TR::DEN)) : 0.f;
#pragma unroll
      for (int mu = 0; mu < D; ++mu)
#pragma unroll
        for (int c = 0; c < D; ++c) sa[mu][c] = scale * jac.adj[mu][c];
    } else if (fcur & GF_ELEM) {
      err |= DEVERR_CONN;
      if (p.det_out) __stcs(p.det_out + e, 0.f);
    }
    float out[NN];
    div_contract<D, VDEG>(sa, out, std::make_integer_sequence<int, NN>{});
    float* row = st + lane * SST;
    if constexpr (PL::VEC) {
#pragma unroll
      for (int q = 0; q < NN / 4; ++q)
        reinterpret_cast<float4*>(row)[q] = make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
    } else {
#pragma unroll
      for (int q = 0; q < NN; ++q) row[q] = out[q];
    }
    __syncwarp();
    const int64_t e0 = t * 32;
    const int cnt = int(p.n_elem - e0 < 32 ? p.n_elem - e0 : 32);
    float* dst = p.B + e0 * NN;
    if (PL::VEC && p.vec_io) {
      const int nq = cnt * (NN / 4);
      for (int q = lane; q < nq; q += 32) {
        const int el = q / (NN / 4);
        const float4 v = *reinterpret_cast<const float4*>(st + el * SST + 4 * (q - el * (NN / 4)));
        __stcs(reinterpret_cast<float4*>(dst) + q, v);
      }
    } else {
      const int nw = cnt * NN;
      for (int idx = lane; idx < nw; idx += 32) {
        const int el = idx / NN;
        __stcs(dst + idx, st[el * SST + (idx - el * NN)]);
      }
    }
    __syncwarp();  // the stage is rewritten next tile
    fcur = fnext;
    wcur = wnext;
#pragma unroll
    for (int k = 0; k <= D; ++k) {
      v1[k] = v2[k];
#pragma unroll
      for (int a = 0; a < D; ++a) Xc[k][a] = Xn[k][a];
    }
  }
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

// ---------------------------------------------------------------- adjoint

template <int D, int VDEG>
__device__ __forceinline__ void copy_dB_async(const DivParams& p, int64_t tile, int lane, float* dslot) {
  using PL = DivPlan<D, VDEG>;
  constexpr int NN = PL::NN;
  const int64_t e0 = tile * 32;
  if (e0 >= p.n_elem) return;
  const int cnt = int(p.n_elem - e0 < 32 ? p.n_elem - e0 : 32);
  const float* src = p.dB + e0 * NN;
  if constexpr (PL::VEC) {
    if (p.vec_io) {
      constexpr int Q = NN / 4;
      for (int q = lane; q < cnt * Q; q += 32) {
        const int el = q / Q;
        cp_async<16>(dslot + el * PL::SST + 4 * (q - el * Q), src + 4 * q);
      }
      return;
    }
  }
  for (int idx = lane; idx < cnt * NN; idx += 32) {
    const int el = idx / NN;
    cp_async<4>(dslot + el * PL::SST + (idx - el * NN), src + idx);
  }
}

template <int D, int VDEG, bool SAVED, bool ATOMIC>
__global__ void __launch_bounds__(DivPlan<D, VDEG>::threads) fem_div_bwd_kernel(DivParams p) {
  using PL = DivPlan<D, VDEG>;
  constexpr int NV = D + 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned char* wbase = smem_raw + size_t(warp) * PL::bwd_per_warp;
  float* dslots = reinterpret_cast<float*>(wbase);                       // [2][32][SST]
  float* xs = reinterpret_cast<float*>(wbase + 2 * PL::row_stage);       // [XCAP][XP]
  const bool rec = !ATOMIC && p.tile_rec != nullptr;
  const int64_t ntiles = (p.n_elem + 31) / 32;
  const int64_t S = int64_t(gridDim.x) * nwarps;
  int64_t t = int64_t(blockIdx.x) * nwarps + warp;
  if (t >= ntiles) return;  // warp-uniform
  int err = 0;
  int v1[D + 1], v2[D + 1], vc[D + 1];
  float Xc[D + 1][D], Xn[D + 1][D];
  load_conn<D>(p.conn, t * 32 + lane, p.n_elem, p.vec_conn, v1);
  int fcur = gather_regs<D>(p.coords, p.n_vert, t * 32 + lane, p.n_elem, v1, Xc);
  copy_dB_async<D, VDEG>(p, t, lane, dslots);
  float wcur = (p.coef && t * 32 + lane < p.n_elem) ? __ldg(p.coef + t * 32 + lane) : 1.f;
  float dcur = (SAVED && t * 32 + lane < p.n_elem) ? __ldg(p.det_in + t * 32 + lane) : 0.f;
  uint32_t rkcur = 0;
  int32_t rb = 0, rn = 0;
  if (rec) {
    rkcur = __ldg(p.rank + t * 32 + lane);
    rb = __ldg(p.tile_rec + t);
    rn = __ldg(p.tile_rec + t + 1) - rb;
  }
  cp_async_commit();
#pragma unroll
  for (int k = 0; k <= D; ++k) vc[k] = v1[k];
  load_conn<D>(p.conn, (t + S) * 32 + lane, p.n_elem, p.vec_conn, v1);
  for (int i = 0; t < ntiles; ++i, t += S) {
    const int64_t tn = t + S, en = tn * 32 + lane;
    const int sn = (i + 1) & 1, sc = i & 1;
    load_conn<D>(p.conn, (tn + S) * 32 + lane, p.n_elem, p.vec_conn, v2);
    const int fnext = gather_regs<D>(p.coords, p.n_vert, en, p.n_elem, v1, Xn);
    copy_dB_async<D, VDEG>(p, tn, lane, dslots + sn * 32 * PL::SST);
    const float wnext = (p.coef && en < p.n_elem) ? __ldg(p.coef + en) : 1.f;
    const float dnext = (SAVED && en < p.n_elem) ? __ldg(p.det_in + en) : 0.f;
    uint32_t rknext = 0;
    int32_t rbn = 0, rnn = 0;
    if (rec && tn < ntiles) {
      rknext = __ldg(p.rank + en);
      rbn = __ldg(p.tile_rec + tn);
      rnn = __ldg(p.tile_rec + tn + 1) - rbn;
    }
    const RecAhead ah = rec ? load_rec_ahead(p.rec_span, p.rec_dest, rb, rn, lane) : RecAhead{0u, 0};
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();  // dB rows were copied by other lanes
    // ---- this tile: one element per lane
    const int64_t e = t * 32 + lane;
    float xb[NV][D];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int a = 0; a < D; ++a) xb[k][a] = 0.f;
    float dcoef = 0.f;
    bool ok = false;
    if (fcur & GF_OK) {
      Jac<D, float> jac;
      const bool nondeg = div_geometry<D, SAVED>(Xc, dcur, jac);
      if (!nondeg) {
        err |= DEVERR_DEGENERATE;
      } else {
        ok = true;
        const float sgn = jac.det > 0.f ? 1.f : -1.f;
        float Tg[D][D];
        div_contract_adjoint<D, VDEG>(dslots + (sc * 32 + lane) * PL::SST, Tg,
                                      std::make_integer_sequence<int, D * D>{});
        const float inv = 1.f / float(DivTraits<D, VDEG>::DEN);
        float dw = 0.f;
        float adjb[D][D];
#pragma unroll
        for (int mu = 0; mu < D; ++mu)
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const float tv = Tg[mu][c] * inv;
            dw = fmaf(tv, jac.adj[mu][c], dw);
            adjb[mu][c] = wcur * sgn * tv;
          }
        dcoef = sgn * dw;
        // adj(J) pulled back to the edge vectors (as in the Laplacian adjoint)
        float eb[D][D];
#pragma unroll
        for (int mu = 0; mu < D; ++mu)
#pragma unroll
          for (int a = 0; a < D; ++a) eb[mu][a] = 0.f;
        if constexpr (D == 3) {
#pragma unroll
          for (int mu = 0; mu < 3; ++mu) {
            const int i1 = (mu + 1) % 3, i2 = (mu + 2) % 3;
            const float* a = jac.e[i1];
            const float* b = jac.e[i2];
            const float* cb = adjb[mu];
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
    } else if (fcur & GF_ELEM) {
      err |= DEVERR_CONN;
    }
    if (fcur & GF_ELEM) {
      if (p.dcoef) __stcs(p.dcoef + e, dcoef);
      if constexpr (ATOMIC) {
        if (ok) {
#pragma unroll
          for (int k = 0; k < NV; ++k)
#pragma unroll
            for (int a = 0; a < D; ++a) atomicAdd(p.dcoords + int64_t(vc[k]) * D + a, xb[k][a]);
        }
      }
    }
    if (rec) {  // slot contributions at their stage positions (zeros for skipped elements), then the records
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        float* d = xs + ((rkcur >> (8 * k)) & 0xFFu) * PL::XP;
        if constexpr (D == 3)
          *reinterpret_cast<float4*>(d) = make_float4(xb[k][0], xb[k][1], xb[k][2], 0.f);
        else
          *reinterpret_cast<float2*>(d) = make_float2(xb[k][0], xb[k][1]);
      }
      __syncwarp();
      warp_records<D>(xs, p.rec_span, p.rec_dest, rb, rn, ah, p.records, lane);
    }
    __syncwarp();  // the slot stage is rewritten next tile, the dB slot two tiles later
    fcur = fnext;
    wcur = wnext;
    dcur = dnext;
    rkcur = rknext;
    rb = rbn;
    rn = rnn;
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
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

// ---------------------------------------------------------------- launchers

template <class K>
cudaError_t launch_pipeline(K kern, size_t per_warp, int64_t n_elem, int ctas_per_sm, cudaStream_t st,
                            const DivParams& p, int threads) {
  const int warps = threads / 32;
  const size_t smem = size_t(warps) * per_warp;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = pipeline_grid(reinterpret_cast<const void*>(kern), warps, smem, n_elem, ctas_per_sm);
  kern<<<grid, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int D, int VDEG>
cudaError_t div_fwd_t(const DivParams& p, int ctas_per_sm, cudaStream_t st) {
  using PL = DivPlan<D, VDEG>;
  return launch_pipeline(fem_div_fwd_kernel<D, VDEG>, PL::fwd_per_warp, p.n_elem, ctas_per_sm, st, p, PL::threads);
}

template <int D, int VDEG>
cudaError_t div_bwd_t(const DivParams& p, bool saved, bool atomic, int ctas_per_sm, cudaStream_t st) {
  using PL = DivPlan<D, VDEG>;
  if (atomic)
    return saved ? launch_pipeline(fem_div_bwd_kernel<D, VDEG, true, true>, PL::bwd_per_warp, p.n_elem, ctas_per_sm,
                                   st, p, PL::threads)
                 : launch_pipeline(fem_div_bwd_kernel<D, VDEG, false, true>, PL::bwd_per_warp, p.n_elem,
                                   ctas_per_sm, st, p, PL::threads);
  return saved ? launch_pipeline(fem_div_bwd_kernel<D, VDEG, true, false>, PL::bwd_per_warp, p.n_elem, ctas_per_sm,
                                 st, p, PL::threads)
               : launch_pipeline(fem_div_bwd_kernel<D, VDEG, false, false>, PL::bwd_per_warp, p.n_elem, ctas_per_sm,
                                 st, p, PL::threads);
}

}  // namespace

cudaError_t launch_div_fwd(const FwdLaunch& L) {
  if (L.coord_f64 || L.out_f64) return cudaErrorInvalidValue;
  DivParams p{};
  p.conn = L.conn;
  p.coords = static_cast<const float*>(L.coords);
  p.coef = L.coef;
  p.B = static_cast<float*>(L.A);
  p.det_out = L.det_out;
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = (L.dim == 3) && (reinterpret_cast<uintptr_t>(L.conn) % 16 == 0);
  p.vec_io = reinterpret_cast<uintptr_t>(L.A) % 16 == 0;
  const bool p2 = L.form == DIV_P2P1;
  if (L.dim == 3) return p2 ? div_fwd_t<3, 2>(p, L.ctas_per_sm, L.stream) : div_fwd_t<3, 1>(p, L.ctas_per_sm, L.stream);
  return p2 ? div_fwd_t<2, 2>(p, L.ctas_per_sm, L.stream) : div_fwd_t<2, 1>(p, L.ctas_per_sm, L.stream);
}

cudaError_t launch_div_bwd(const BwdLaunch& L) {
  DivParams p{};
  p.conn = L.conn;
  p.coords = L.coords;
  p.coef = L.coef;
  p.dB = L.dA;
  p.det_in = L.det_in;
  p.dcoef = L.dcoef;
  p.dcoords = L.atomic ? L.dcoords : nullptr;
  p.tile_rec = L.tile_rec;
  p.rank = L.rank;
  p.rec_span = L.rec_span;
  p.rec_dest = L.rec_dest;
  p.records = L.records;
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = (L.dim == 3) && (reinterpret_cast<uintptr_t>(L.conn) % 16 == 0);
  p.vec_io = reinterpret_cast<uintptr_t>(L.dA) % 16 == 0;
  const bool p2 = L.form == DIV_P2P1, saved = L.det_in != nullptr, atomic = L.atomic != 0;
  if (L.dim == 3)
    return p2 ? div_bwd_t<3, 2>(p, saved, atomic, L.ctas_per_sm, L.stream)
              : div_bwd_t<3, 1>(p, saved, atomic, L.ctas_per_sm, L.stream);
  return p2 ? div_bwd_t<2, 2>(p, saved, atomic, L.ctas_per_sm, L.stream)
            : div_bwd_t<2, 1>(p, saved, atomic, L.ctas_per_sm, L.stream);
}

}  // namespace fem
