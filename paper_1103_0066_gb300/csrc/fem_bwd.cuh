// fem_bwd.cuh -- adjoint (reverse mode) of the element integration, element part.
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
// A CTA of 4 warps owns a tile of 128 consecutive elements.  Each warp runs
// the forward kernel's three-stage pipeline over its 32 elements (connectivity
// two tiles ahead, coordinates one tile ahead in registers) and copies its
// upstream dA (contiguous) with 16-byte cp.async into a padded stage.  In the
// deterministic mode the CTA stages the (d+1) vertex contributions of its 128
// elements in shared memory and writes one RECORD per distinct vertex of the
// tile, summed in slot order (the tile's sorted slot list, built once per
// mesh); the segmented reduction then adds the few records of each vertex.  The
// atomic variant adds each contribution into dcoords with red.global.add.
#pragma once
#include "fem_core.cuh"
#include "fem_fwd.cuh"
#include "fem_internal.h"
#include "fem_pipe.cuh"

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
  const int32_t* tile_rec;  // first record of each tile (null: no coordinate records)
  const uint16_t* sorted;   // per tile: slots sorted by (vertex, slot)
  const uint16_t* rec_end;  // per record: end of its run in the tile's sorted list
  float* records;           // [R][D]
  float* dcoef;
  float* dcoords;  // atomic mode
  int64_t n_elem;
  int64_t n_vert;
  int32_t* dev_err;
  int vec_conn;
  int vec_dA;
};

template <int D, int FORM>
struct BwdPlan {
  static constexpr int NN = FormTraits<D, FORM>::NN;
  static constexpr bool VEC = (NN % 4 == 0);
  static constexpr int DST = VEC ? NN + 4 : (NN | 1);  // dA row stride in the stage
  static constexpr int NV = D + 1;
  static constexpr int NS = kTileElems * NV;  // slots per CTA tile
  static constexpr int XP = D == 3 ? 4 : 2;     // padded floats per staged slot (one vector store)
  static constexpr int WARPS = kTileElems / 32;
  static constexpr size_t da_bytes = align_up(size_t(2) * 32 * DST * 4, 128);  // per warp
  static constexpr size_t xs_bytes = align_up(size_t(NS) * XP * 4, 128);        // per CTA
  static constexpr size_t sorted_bytes = align_up(size_t(2) * NS * 2, 128);     // per CTA
  static constexpr int ENDS = NS + 16;  // record ends of a tile (<= NS) plus alignment slack
  static constexpr size_t ends_bytes = align_up(size_t(2) * ENDS * 2, 128);     // per CTA
  static constexpr size_t smem = WARPS * da_bytes + xs_bytes + sorted_bytes + ends_bytes;
};

// Asynchronous copy of a tile's contiguous dA into the padded stage slot.
template <int D, int FORM>
__device__ __forceinline__ void copy_dA_async(const BwdParams& p, int64_t tile, int lane, float* dslot) {
  using PL = BwdPlan<D, FORM>;
  constexpr int NN = PL::NN;
  const int64_t e0 = tile * 32;
  if (e0 >= p.n_elem) return;
  const int cnt = int(p.n_elem - e0 < 32 ? p.n_elem - e0 : 32);
  const float* src = p.dA + e0 * NN;
  if constexpr (PL::VEC) {
    if (p.vec_dA) {
      constexpr int Q = NN / 4;
      const int nq = cnt * Q;
      for (int q = lane; q < nq; q += 32) {
        const int el = q / Q;
        cp_async<16>(dslot + el * PL::DST + 4 * (q - el * Q), src + 4 * q);
      }
      return;
    }
  }
  const int nw = cnt * NN;
  for (int idx = lane; idx < nw; idx += 32) {
    const int el = idx / NN;
    cp_async<4>(dslot + el * PL::DST + (idx - el * NN), src + idx);
  }
}

// Asynchronous copy of tile `tile`'s sorted slot list (NS u16) by the CTA.
template <int NS>
__device__ __forceinline__ void copy_sorted(const uint16_t* sorted, int64_t tile, int tid, uint16_t* dst) {
  static_assert((NS * 2) % 16 == 0, "sorted slot list in 16-byte chunks");
  constexpr int NCH = NS * 2 / 16;
  const uint16_t* src = sorted + tile * NS;
  for (int c = tid; c < NCH; c += kTileElems) cp_async<16>(dst + 8 * c, src + 8 * c);
}

// Asynchronous copy of the record ends rec_end[rb, rb + rn) of a tile into
// dst[0, ...), starting at the 16-byte chunk that holds entry rb; returns the
// offset of entry rb in dst.  The workspace pads rec_end so the last chunk
// never leaves the array.
template <int ENDS>
__device__ __forceinline__ int copy_ends(const uint16_t* rec_end, int32_t rb, int32_t rn, int tid, uint16_t* dst) {
  const int32_t c0 = rb & ~7;
  const int nch = (rb + rn - c0 + 7) >> 3;
  for (int c = tid; c < nch; c += kTileElems) cp_async<16>(dst + 8 * c, rec_end + c0 + 8 * c);
  return rb - c0;
}

// Position of slot (element el of the CTA tile, local vertex k) in the padded
// stage: the slot order within an element is rotated by (el >> 1), which keeps
// the 16-byte writes of a quarter warp on distinct bank groups.
template <int NV>
__device__ __forceinline__ int stage_slot(int el, int k) {
  if constexpr (NV == 4)
    return el * 4 + ((k + (el >> 1)) & 3);
  else
    return el * NV + k;
}

// Upper triangle of sym(dA) from a staged row: 16-byte reads when the row is
// 16-byte aligned and small enough to hold in registers, scalar reads otherwise.
template <int D, int FORM>
__device__ __forceinline__ void stage_sym(const float* drow, float (&s)[FormTraits<D, FORM>::NT]) {
  using FT = FormTraits<D, FORM>;
  constexpr int N = FT::N, NN = FT::NN;
  if constexpr (NN % 4 == 0 && NN <= 36) {
    float r[NN];
#pragma unroll
    for (int q = 0; q < NN / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(drow)[q];
      r[4 * q] = v.x;
      r[4 * q + 1] = v.y;
      r[4 * q + 2] = v.z;
      r[4 * q + 3] = v.w;
    }
    load_sym<N>(r, s, std::make_integer_sequence<int, FT::NT>{});
  } else {
    load_sym<N>(drow, s, std::make_integer_sequence<int, FT::NT>{});
  }
}

// Record phase of a CTA tile: record r (r < rn) sums the staged contributions
// of its slots srt[ends[r-1] .. ends[r]) in order and writes records[rb + r].
template <int D>
__device__ __forceinline__ void write_records(const uint16_t* srt, const uint16_t* ends, const float* xs, int32_t rb,
                                              int32_t rn, float* records, int tid) {
  constexpr int NV = D + 1, XP = D == 3 ? 4 : 2;
  for (int r = tid; r < rn; r += kTileElems) {
    const int beg = r == 0 ? 0 : int(ends[r - 1]);
    const int end = int(ends[r]);
    float acc[D];
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] = 0.f;
    for (int j = beg; j < end; ++j) {
      const int slot = srt[j];
      const float* x = xs + stage_slot<NV>(slot / NV, slot % NV) * XP;
      if constexpr (D == 3) {
        const float4 v = *reinterpret_cast<const float4*>(x);
        acc[0] += v.x;
        acc[1] += v.y;
        acc[2] += v.z;
      } else {
        const float2 v = *reinterpret_cast<const float2*>(x);
        acc[0] += v.x;
        acc[1] += v.y;
      }
    }
    float* dst = records + int64_t(rb + r) * D;
#pragma unroll
    for (int a = 0; a < D; ++a) dst[a] = acc[a];
  }
}

// Stage 3 of the adjoint for one element per lane.
template <int D, int FORM, int JAC, bool ATOMIC>
__device__ __forceinline__ int bwd_compute_tile(const BwdParams& p, int64_t tile, int lane, int flags, float w,
                                                const float (&X)[D + 1][D], const float* drow,
                                                const int (&vc)[D + 1], float* xs, int el) {
  using FT = FormTraits<D, FORM>;
  using GT = typename std::conditional<JAC == JAC_F64, double, float>::type;
  constexpr int N = FT::N, NV = FT::NV;
  const int64_t e = tile * 32 + lane;
  int err = 0;
  float xb[NV][D];
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int a = 0; a < D; ++a) xb[k][a] = 0.f;
  float dcoef = 0.f;
  bool ok = false;
  if (flags & GF_OK) {
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
      const float scale0 = __frcp_rn(dev_abs(det) * float(FT::DEN));
      float G0[FT::NG];
      geometric_tensor<D, FORM>(adj, scale0, G0);
      // 1. dG = transpose of the contraction applied to sym(dA)
      SymVals<FT::NT> sym;
      stage_sym<D, FORM>(drow, sym.s);
      float dG[FT::NG];
      contract_adjoint<D, FORM>(sym, dG);
      // 2. coefficient gradient
#pragma unroll
      for (int g = 0; g < FT::NG; ++g) dcoef = fmaf(dG[g], G0[g], dcoef);
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
      const float Ld = -__fdividef(L, det);
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
  } else if (flags & GF_ELEM) {
    err |= DEVERR_CONN;
  }
  if (flags & GF_ELEM) {
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
  if constexpr (!ATOMIC) {
    if (xs) {  // the element's slot contributions (zeros when it is skipped)
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        float* d = xs + stage_slot<NV>(el, k) * (D == 3 ? 4 : 2);
        if constexpr (D == 3)
          *reinterpret_cast<float4*>(d) = make_float4(xb[k][0], xb[k][1], xb[k][2], 0.f);
        else
          *reinterpret_cast<float2*>(d) = make_float2(xb[k][0], xb[k][1]);
      }
    }
  }
  return err;
}

template <int D, int FORM, int JAC, bool ATOMIC>
__global__ void __launch_bounds__(kTileElems) fem_bwd_elem_kernel(BwdParams p) {
  using PL = BwdPlan<D, FORM>;
  constexpr int W = PL::WARPS, NS = PL::NS, NV = PL::NV;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* dslots = reinterpret_cast<float*>(smem_raw + size_t(warp) * PL::da_bytes);  // [2][32][DST]
  float* xs = reinterpret_cast<float*>(smem_raw + W * PL::da_bytes);                 // [NS][XP]
  uint16_t* sbuf = reinterpret_cast<uint16_t*>(smem_raw + W * PL::da_bytes + PL::xs_bytes);  // [2][NS]
  uint16_t* ebuf = reinterpret_cast<uint16_t*>(smem_raw + W * PL::da_bytes + PL::xs_bytes +
                                               PL::sorted_bytes);  // [2][ENDS]
  const bool rec = !ATOMIC && p.tile_rec != nullptr;
  const int64_t nct = (p.n_elem + kTileElems - 1) / kTileElems;
  const int64_t G = gridDim.x;
  int64_t T = blockIdx.x;
  if (T >= nct) return;  // CTA-uniform
  const int el = warp * 32 + lane;  // element within the CTA tile
  int eoff = 0;                     // position of the tile's first record end in its ebuf slot
  int err = 0;
  int v1[D + 1], v2[D + 1], vc[D + 1];
  float Xc[D + 1][D], Xn[D + 1][D];
  int64_t t = T * W + warp;  // this warp's 32-element sub-tile
  load_conn<D>(p.conn, t * 32 + lane, p.n_elem, p.vec_conn, v1);
  int fcur = gather_regs<D>(p.coords, p.n_vert, t * 32 + lane, p.n_elem, v1, Xc);
  copy_dA_async<D, FORM>(p, t, lane, dslots);
  if (rec) copy_sorted<NS>(p.sorted, T, tid, sbuf);
  float wcur = (p.coef && t * 32 + lane < p.n_elem) ? __ldg(p.coef + t * 32 + lane) : 1.f;
  int32_t rb = 0, rn = 0;  // first record and record count of tile T
  if (rec) {
    rb = __ldg(p.tile_rec + T);
    rn = __ldg(p.tile_rec + T + 1) - rb;
    eoff = copy_ends<PL::ENDS>(p.rec_end, rb, rn, tid, ebuf);
  }
  cp_async_commit();
#pragma unroll
  for (int k = 0; k <= D; ++k) vc[k] = v1[k];
  load_conn<D>(p.conn, (t + W * G) * 32 + lane, p.n_elem, p.vec_conn, v1);
  for (int i = 0; T < nct; ++i, T += G, t += W * G) {
    const int64_t tn = t + W * G, en = tn * 32 + lane;
    const int sn = (i + 1) & 1, sc = i & 1;
    load_conn<D>(p.conn, (tn + W * G) * 32 + lane, p.n_elem, p.vec_conn, v2);
    const int fnext = gather_regs<D>(p.coords, p.n_vert, en, p.n_elem, v1, Xn);
    copy_dA_async<D, FORM>(p, tn, lane, dslots + sn * 32 * PL::DST);
    const bool has_next = T + G < nct;
    if (rec && has_next) copy_sorted<NS>(p.sorted, T + G, tid, sbuf + sn * NS);
    const float wnext = (p.coef && en < p.n_elem) ? __ldg(p.coef + en) : 1.f;
    int32_t rbn = 0, rnn = 0, eoffn = 0;
    if (rec && has_next) {
      rbn = __ldg(p.tile_rec + T + G);
      rnn = __ldg(p.tile_rec + T + G + 1) - rbn;
      eoffn = copy_ends<PL::ENDS>(p.rec_end, rbn, rnn, tid, ebuf + sn * PL::ENDS);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();  // dA rows were copied by other lanes
    err |= bwd_compute_tile<D, FORM, JAC, ATOMIC>(p, t, lane, fcur, wcur, Xc, dslots + (sc * 32 + lane) * PL::DST,
                                                  vc, rec ? xs : nullptr, el);
    if (rec) {
      __syncthreads();  // every warp's contributions and the sorted list are in shared memory
      write_records<D>(sbuf + sc * NS, ebuf + sc * PL::ENDS + eoff, xs, rb, rn, p.records, tid);
      __syncthreads();  // xs and the sorted slot buffer are refilled next
    } else {
      __syncwarp();  // the dA slot is refilled two tiles later
    }
    fcur = fnext;
    wcur = wnext;
    rb = rbn;
    rn = rnn;
    eoff = eoffn;
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

}  // namespace fem
