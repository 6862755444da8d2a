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
// Each warp runs the forward kernel's three-stage pipeline over tiles of 32
// elements (connectivity two tiles ahead; coordinates, slot ranks and the
// tile's record range one tile ahead in registers) and copies its upstream dA
// (contiguous) with 16-byte cp.async into a stage.  In the deterministic mode
// each lane writes the (d+1) vertex contributions of its element into the
// warp's slot stage at their stage positions (built once per mesh): the
// contributions to one vertex form a contiguous run, the runs follow the
// tile's vertex order, and on tets each run starts at a position congruent to
// its record index mod 8.  Lane r then sums run r in order into RECORD r of
// the tile, and the segmented reduction adds the few records of each vertex.
// Warps never wait for one another.  The atomic variant adds each
// contribution into dcoords with red.global.add.
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
  const int32_t* tile_rec;  // first record of each 32-element tile (null: no coordinate records)
  const uint32_t* rank;     // per element: byte k = stage position of slot k (runs in (vertex, slot) order)
  const uint16_t* rec_span; // per record: start | length << 8 of its run in the stage
  const int32_t* rec_dest;  // per record: its row in the records array (the identity in tile order)
  float* records;           // [R][D]
  float* dcoef;
  float* dcoords;  // atomic mode
  int64_t n_elem;
  int64_t n_vert;
  int32_t* dev_err;
  int vec_conn;
  int vec_dA;
  const float* det = nullptr;  // [n_elem] det J saved by the forward (JAC_SAVED)
};

template <int D, int FORM>
struct BwdPlan {
  static constexpr int NN = FormTraits<D, FORM>::NN;
  static constexpr bool VEC = (NN % 4 == 0);
  // 4x4 rows: unpadded, 16-byte chunk c of row r at chunk c ^ ((r >> 1) & 3),
  // so that both the copy (four lanes per row) and the row reads (a lane per
  // row) are free of bank conflicts.  Other rows of 16-byte chunks: a stride of
  // an odd number of chunks, so that the eight lanes of a 16-byte read phase
  // (lane per row) reach eight different bank groups; odd-sized rows: an odd
  // stride in words.
  static constexpr bool SWZ = (NN == 16);
  static constexpr int DST = SWZ ? 16 : (VEC ? ((NN / 4) % 2 ? NN : NN + 4) : (NN | 1));  // dA row stride
  static constexpr int NV = D + 1;
  static constexpr int NSW = kRecTile * NV;  // slots per record tile (one warp)
  static constexpr int XCAP = D == 3 ? kStageCap3 : NSW;  // stage positions (aligned runs on tets)
  // components of a slot contribution: the vertex gradient, plus the
  // coefficient gradient for the P1-coefficient forms (Eqs. 20-23)
  static constexpr int NC = D + (FormTraits<D, FORM>::W1 ? 1 : 0);
  static constexpr int XP = NC > 2 ? 4 : 2;  // padded floats per staged slot (one vector store)
  static constexpr size_t da_slot = align_up(size_t(32) * DST * 4, 128);    // one tile of dA rows
  static constexpr size_t da_bytes = 2 * da_slot;                           // double buffered
  static constexpr size_t xs_bytes = align_up(size_t(XCAP) * XP * 4, 128);  // slot stage of one tile
  // Per warp of the single-mesh kernel: [dA slot 0][xs_over][dA slot 1].  A
  // tile's slot stage overlays its own dA slot once every lane has read its
  // dA row -- from slot 0's base, or ending at slot 1's end -- and never
  // reaches the other slot, where the next tile's dA is arriving.  On P1 tets
  // that is 6 KB per warp instead of 8 (2 KB dA slots, a 4 KB stage).
  static constexpr size_t xs_over = xs_bytes > da_slot ? xs_bytes - da_slot : 0;
  static constexpr size_t per_warp = 2 * da_slot + xs_over;
};

// CTA shape of the adjoint element kernel.  The kernel has no CTA-wide
// barrier, so the CTA size only sets how finely the register file and shared
// memory are shared out.  On tets every form runs one-warp CTAs: the P2
// Laplacian's 30 KB per warp then packs 7 warps per SM instead of one 4-warp
// CTA.  The compensated 3D P1 Laplacian also asks for at least 28 resident
// per SM, which holds it to 72 registers without spills: 28 warps per SM
// (7 KB of shared memory each with the reserved 1 KB), against 20 at its
// natural 93 registers.  Triangles keep 4-warp CTAs.
template <int D, int FORM, int JAC>
struct BwdShape {
  static constexpr bool tight = (D == 3 && FORM == LAPLACE_P1 && (JAC == JAC_COMP || JAC == JAC_SAVED));
  static constexpr int threads = D == 3 ? 32 : kTileElems;
  static constexpr int min_ctas = tight ? 28 : 1;
};

// Asynchronous copy of a tile's contiguous dA into the stage slot.
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
      if constexpr (PL::SWZ) {
        if (cnt == 32) {  // chunk lane + 32 i: row lane / 4 + 8 i, chunk lane % 4, swizzle (lane >> 3) & 3
          float* d = dslot + (lane >> 2) * 16 + 4 * ((lane & 3) ^ ((lane >> 3) & 3));
          const float* s = src + 4 * lane;
#pragma unroll
          for (int i = 0; i < 4; ++i) cp_async<16>(d + i * 128, s + 128 * i);
          return;
        }
        for (int q = lane; q < cnt * 4; q += 32) {
          const int el = q >> 2;
          cp_async<16>(dslot + el * 16 + 4 * ((q & 3) ^ ((el >> 1) & 3)), src + 4 * q);
        }
        return;
      }
      if constexpr (32 % Q == 0) {
        if (cnt == 32) {  // full tile: chunk lane + 32 i is chunk lane % Q of row lane / Q + i (32 / Q)
          constexpr int RPI = 32 / Q;
          float* d = dslot + (lane / Q) * PL::DST + 4 * (lane % Q);
          const float* s = src + 4 * lane;
#pragma unroll
          for (int i = 0; i < Q; ++i) cp_async<16>(d + i * RPI * PL::DST, s + 128 * i);
          return;
        }
      }
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
    int w = idx - el * NN;
    if constexpr (PL::SWZ) w = 4 * ((w >> 2) ^ ((el >> 1) & 3)) + (w & 3);
    cp_async<4>(dslot + el * PL::DST + w, src + idx);
  }
}

// Upper triangle of sym(dA) from a staged row (row = lane): 16-byte reads when
// the row is 16-byte aligned (small rows whole into registers; larger ones a
// chunk at a time, each entry going to its triangle slot: an upper entry
// comes first in the row, so an off-diagonal slot is upper + lower, as
// load_sym forms it), scalar reads otherwise.
template <int N, int Q, int... Us>
__device__ __forceinline__ void sym_chunk(const float4 v, float* s, std::integer_sequence<int, Us...>) {
  const float x[4] = {v.x, v.y, v.z, v.w};
  (
      [&] {
        constexpr int i = (4 * Q + Us) / N, j = (4 * Q + Us) % N;
        constexpr int lo = i < j ? i : j, hi = i < j ? j : i;
        constexpr int T = pair_index(lo, hi, N);
        static_assert(TriIdx<T, N>::i == lo && TriIdx<T, N>::j == hi, "triangle index");
        if constexpr (i <= j)
          s[T] = x[Us];
        else
          s[T] += x[Us];
      }(),
      ...);
}

template <int N, int... Qs>
__device__ __forceinline__ void sym_chunks(const float* drow, float* s, std::integer_sequence<int, Qs...>) {
  (sym_chunk<N, Qs>(reinterpret_cast<const float4*>(drow)[Qs], s, std::make_integer_sequence<int, 4>{}), ...);
}

template <int D, int FORM>
__device__ __forceinline__ void stage_sym(const float* drow, float (&s)[FormTraits<D, FORM>::NT]) {
  using FT = FormTraits<D, FORM>;
  constexpr int N = FT::N, NN = FT::NN;
  if constexpr (NN % 4 == 0 && NN <= 36) {
    float r[NN];
    const int sw = BwdPlan<D, FORM>::SWZ ? ((threadIdx.x & 31) >> 1) & 3 : 0;
#pragma unroll
    for (int q = 0; q < NN / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(drow)[q ^ sw];
      r[4 * q] = v.x;
      r[4 * q + 1] = v.y;
      r[4 * q + 2] = v.z;
      r[4 * q + 3] = v.w;
    }
    load_sym<N>(r, s, std::make_integer_sequence<int, FT::NT>{});
  } else if constexpr (NN % 4 == 0) {
    sym_chunks<N>(drow, s, std::make_integer_sequence<int, NN / 4>{});
  } else {
    load_sym<N>(drow, s, std::make_integer_sequence<int, FT::NT>{});
  }
}

// Records of one warp's 32-element tile.  Record r (r < rn) sums the staged
// contributions of its run -- the slots of its vertex, in increasing slot
// order, at stage positions [start, start + length) -- and writes row
// rec_dest[rb + r] of the vertex-major records.  span0 = rec_span[rb + lane]
// and dest0 = rec_dest[rb + lane] for lane < rn (loaded ahead by the caller),
// anything for the other lanes.
struct RecAhead {
  uint32_t span0;
  int dest0;
};

__device__ __forceinline__ RecAhead load_rec_ahead(const uint16_t* rec_span, const int32_t* rec_dest, int32_t rb,
                                                   int32_t rn, int lane) {
  RecAhead a{0u, 0};
  if (lane < rn) {
    a.span0 = __ldg(rec_span + rb + lane);
    a.dest0 = __ldg(rec_dest + rb + lane);
  }
  return a;
}

template <int D, int NC = D>
__device__ __forceinline__ void warp_records(const float* xs, const uint16_t* rec_span, const int32_t* rec_dest,
                                             int32_t rb, int32_t rn, RecAhead ah, float* records, int lane) {
  constexpr int XP = NC > 2 ? 4 : 2;
  for (int r0 = 0; r0 < rn; r0 += 32) {
    const int r = r0 + lane;
    const bool live = r < rn;
    const uint32_t span = r0 == 0 ? ah.span0 : (live ? uint32_t(__ldg(rec_span + rb + r)) : 0u);
    const int dest = r0 == 0 ? ah.dest0 : (live ? __ldg(rec_dest + rb + r) : 0);
    const int beg = int(span & 0xFFu);
    // Runs have different lengths; the warp steps to its longest run in
    // blocks of 8 predicated loads, so the loads of a lane are in flight
    // together.  Each run is still summed in increasing position order.
    const int len = live ? int(span >> 8) : 0;
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    float acc[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) acc[a] = 0.f;
    for (int m0 = 0; m0 < maxlen; m0 += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (m0 + u < len) {
          const float* x = xs + (beg + m0 + u) * XP;
          if constexpr (XP == 4) {
            const float4 v = *reinterpret_cast<const float4*>(x);
            acc[0] += v.x;
            acc[1] += v.y;
            acc[2] += v.z;
            if constexpr (NC == 4) acc[3] += v.w;
          } else {
            const float2 v = *reinterpret_cast<const float2*>(x);
            acc[0] += v.x;
            acc[1] += v.y;
          }
        }
      }
    }
    if (live) {
      float* dst = records + int64_t(dest) * NC;
#pragma unroll
      for (int a = 0; a < NC; ++a) dst[a] = acc[a];
    }
  }
}

// Stage 3 of the adjoint for one element per lane.
// For the P1-coefficient forms (Eqs. 20-23) the contraction's slots are
// w_k G_g (slot k * NGB + g): with dGw its adjoint, the base form's adjoint
// runs on dG_g = sum_k w_k dGw_kg with w = 1, and the coefficient's vertex
// value k collects wb_k = sum_g dGw_kg G_g, staged beside the vertex gradient.
template <int D, int FORM, int JAC, bool ATOMIC>
__device__ __forceinline__ int bwd_compute_tile(const BwdParams& p, int64_t tile, int lane, int flags,
                                                const Coef<FormTraits<D, FORM>::NW>& wv,
                                                const float (&X)[D + 1][D], const float* drow,
                                                const int (&vc)[D + 1], float* xs, uint32_t rk,
                                                float det_saved = 0.f) {
  using FT = FormTraits<D, FORM>;
  using BT = FormTraits<D, FT::BASE>;
  using GT = typename std::conditional<JAC == JAC_F64, double, float>::type;
  constexpr int N = FT::N, NV = FT::NV;
  constexpr bool W1 = FT::W1;
  const int64_t e = tile * 32 + lane;
  int err = 0;
  float xb[NV][D];
  float wb[NV];  // P1 coefficient: gradient of the element's vertex values
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    wb[k] = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) xb[k][a] = 0.f;
  }
  float dcoef = 0.f;
  bool ok = false;
  if (flags & GF_OK) {
    Jac<D, GT> jac;
    bool nondeg;
    if constexpr (JAC == JAC_SAVED)
      nondeg = jacobian_saved<D>(X, det_saved, jac);
    else
      nondeg = jacobian<D, JAC>(X, jac);
    if (!nondeg) {
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
      float G0[BT::NG];
      geometric_tensor<D, FT::BASE>(adj, scale0, G0);
      // 1. dG = transpose of the contraction applied to sym(dA)
      SymVals<FT::NT> sym;
      stage_sym<D, FORM>(drow, sym.s);
      float dGw[FT::NG];
      contract_adjoint<D, FORM>(sym, dGw);
      // 2. coefficient gradient
      float dG[BT::NG];
      float w = 1.f;
      if constexpr (W1) {
#pragma unroll
        for (int g = 0; g < BT::NG; ++g) {
          float acc = wv.v[0] * dGw[g];
#pragma unroll
          for (int k = 1; k < NV; ++k) acc = fmaf(wv.v[k], dGw[k * BT::NG + g], acc);
          dG[g] = acc;
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          float acc = 0.f;
#pragma unroll
          for (int g = 0; g < BT::NG; ++g) acc = fmaf(dGw[k * BT::NG + g], G0[g], acc);
          wb[k] = acc;
        }
      } else {
        w = wv.v[0];
#pragma unroll
        for (int g = 0; g < BT::NG; ++g) dG[g] = dGw[g];
      }
#pragma unroll
      for (int g = 0; g < BT::NG; ++g) dcoef = fmaf(dG[g], G0[g], dcoef);
      const float L = w * dcoef;
      const float c2 = 2.f * w * scale0;
      // 3. adjoint of G with respect to adj(J): adjb = c2 S adj, with S the
      // symmetric matrix of dG (off-diagonal entries halved); c2 is folded
      // into S once
      float adjb[D][D];
      if constexpr (FT::BASE != ELASTIC_P1) {
        float Sc[D][D];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int nu = r; nu < D; ++nu) {
            Sc[r][nu] = (r == nu ? c2 : 0.5f * c2) * dG[pair_index(r, nu, D)];
            Sc[nu][r] = Sc[r][nu];
          }
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int a = 0; a < D; ++a) {
            float acc = Sc[r][0] * adj[0][a];
#pragma unroll
            for (int nu = 1; nu < D; ++nu) acc = fmaf(Sc[r][nu], adj[nu][a], acc);
            adjb[r][a] = acc;
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
      if constexpr (D == 3) {
        // adj_mu = e_{mu+1} x e_{mu+2}, so edge nu collects
        //   d e_nu = Ld adj_nu + e_{nu+1} x adjb_{nu+2} + adjb_{nu+1} x e_{nu+2}
        // (indices mod 3), each component as one chain of fused multiply-adds
#pragma unroll
        for (int nu = 0; nu < 3; ++nu) {
          const float* ea = ed[(nu + 1) % 3];
          const float* eb2 = ed[(nu + 2) % 3];
          const float* ga = adjb[(nu + 2) % 3];
          const float* gb = adjb[(nu + 1) % 3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int c1 = (c + 1) % 3, c2i = (c + 2) % 3;
            float t = Ld * adj[nu][c];
            t = fmaf(ea[c1], ga[c2i], t);
            t = fmaf(-ea[c2i], ga[c1], t);
            t = fmaf(gb[c1], eb2[c2i], t);
            t = fmaf(-gb[c2i], eb2[c1], t);
            eb[nu][c] = t;
          }
        }
      } else {
#pragma unroll
        for (int mu = 0; mu < D; ++mu)
#pragma unroll
          for (int a = 0; a < D; ++a) eb[mu][a] = Ld * adj[mu][a];
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
    if (!W1 && p.dcoef) __stcs(p.dcoef + e, dcoef);  // W1: dcoef holds vertex values (records / atomics)
    if constexpr (ATOMIC) {
      if (ok) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          if (p.dcoords)
#pragma unroll
            for (int a = 0; a < D; ++a) atomicAdd(p.dcoords + int64_t(vc[k]) * D + a, xb[k][a]);
          if (W1 && p.dcoef) atomicAdd(p.dcoef + vc[k], wb[k]);
        }
      }
    }
  }
  if constexpr (!ATOMIC) {
    __syncwarp();  // every lane has read its dA row (the stage overlays it)
    if (xs) {  // the element's slot contributions at their ranks (zeros when it is skipped)
      constexpr int XP = BwdPlan<D, FORM>::XP;
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        float* d = xs + ((rk >> (8 * k)) & 0xFFu) * XP;
        if constexpr (XP == 4) {
          const float c2v = D == 3 ? xb[k][D - 1] : (W1 ? wb[k] : 0.f);
          const float c3v = (D == 3 && W1) ? wb[k] : 0.f;
          *reinterpret_cast<float4*>(d) = make_float4(xb[k][0], xb[k][1], c2v, c3v);
        } else {
          *reinterpret_cast<float2*>(d) = make_float2(xb[k][0], xb[k][1]);
        }
      }
    }
  }
  return err;
}

template <int D, int FORM, int JAC, bool ATOMIC>
__global__ void __launch_bounds__(BwdShape<D, FORM, JAC>::threads, BwdShape<D, FORM, JAC>::min_ctas)
    fem_bwd_elem_kernel(BwdParams p) {
  using PL = BwdPlan<D, FORM>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  unsigned char* wbase = smem_raw + size_t(warp) * PL::per_warp;
  // dA slot s and the slot stage of a tile whose dA is in slot s (BwdPlan)
  auto dslot = [&](int s) { return reinterpret_cast<float*>(wbase + size_t(s) * (PL::da_slot + PL::xs_over)); };
  auto xstage = [&](int s) { return reinterpret_cast<float*>(wbase + size_t(s) * PL::da_slot); };
  const bool rec = !ATOMIC && p.tile_rec != nullptr;
  const int64_t ntiles = (p.n_elem + 31) / 32;
  const int64_t S = int64_t(gridDim.x) * nwarps;  // warp-tile stride
  int64_t t = int64_t(blockIdx.x) * nwarps + warp;
  if (t >= ntiles) return;  // warp-uniform: the kernel has no CTA-wide barrier
  int err = 0;
  int v1[D + 1], v2[D + 1], vc[D + 1];
  float Xc[D + 1][D], Xn[D + 1][D];
  load_conn<D>(p.conn, t * 32 + lane, p.n_elem, p.vec_conn, v1);
  int fcur = gather_regs<D>(p.coords, p.n_vert, t * 32 + lane, p.n_elem, v1, Xc);
  copy_dA_async<D, FORM>(p, t, lane, dslot(0));
  Coef<FormTraits<D, FORM>::NW> wcur, wnext;
  load_coef<D, FORM>(p.coef, t * 32 + lane, p.n_elem, p.n_vert, v1, wcur);
  float dcur = 0.f;  // saved det J (JAC_SAVED)
  if constexpr (JAC == JAC_SAVED) dcur = t * 32 + lane < p.n_elem ? __ldg(p.det + t * 32 + lane) : 0.f;
  uint32_t rkcur = 0;
  int32_t rb = 0, rn = 0;  // first record and record count of tile t
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
    copy_dA_async<D, FORM>(p, tn, lane, dslot(sn));
    load_coef<D, FORM>(p.coef, en, p.n_elem, p.n_vert, v1, wnext);
    float dnext = 0.f;
    if constexpr (JAC == JAC_SAVED) dnext = en < p.n_elem ? __ldg(p.det + en) : 0.f;
    uint32_t rknext = 0;
    int32_t rbn = 0, rnn = 0;
    if (rec && tn < ntiles) {
      rknext = __ldg(p.rank + en);
      rbn = __ldg(p.tile_rec + tn);
      rnn = __ldg(p.tile_rec + tn + 1) - rbn;
    }
    // this tile's record ends and destinations: in flight while the element math runs
    const RecAhead ah = rec ? load_rec_ahead(p.rec_span, p.rec_dest, rb, rn, lane) : RecAhead{0u, 0};
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();  // dA rows were copied by other lanes
    float* xs = xstage(sc);
    err |= bwd_compute_tile<D, FORM, JAC, ATOMIC>(p, t, lane, fcur, wcur, Xc, dslot(sc) + lane * PL::DST,
                                                  vc, rec ? xs : nullptr, rkcur, dcur);
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

// Launch of one instantiation of the adjoint element kernel (host).
template <int D, int FORM, int JAC, bool ATOMIC>
cudaError_t launch_bwd_t(const BwdLaunch& L) {
  using PL = BwdPlan<D, FORM>;
  BwdParams p;
  p.conn = L.conn;
  p.coords = L.coords;
  p.coef = L.coef;
  p.dA = L.dA;
  p.tile_rec = ATOMIC ? nullptr : L.tile_rec;
  p.rank = L.rank;
  p.rec_span = L.rec_span;
  p.rec_dest = L.rec_dest;
  p.records = L.records;
  p.dcoef = L.dcoef;
  p.dcoords = L.dcoords;
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(L.conn) % 16 == 0);
  p.vec_dA = reinterpret_cast<uintptr_t>(L.dA) % 16 == 0;
  p.det = L.det_in;
  auto kern = fem_bwd_elem_kernel<D, FORM, JAC, ATOMIC>;
  constexpr int max_warps = BwdShape<D, FORM, JAC>::threads / 32;  // the kernel's launch bounds
  const int want = L.warps > 0 ? L.warps : max_warps;
  const int warps = clamp_warps(want < max_warps ? want : max_warps, PL::per_warp);
  const size_t smem = size_t(warps) * PL::per_warp;
  cudaError_t st = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (st != cudaSuccess) return st;
  const unsigned grid = pipeline_grid(reinterpret_cast<const void*>(kern), warps, smem, L.n_elem, L.ctas_per_sm);
  kern<<<grid, warps * 32, smem, L.stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_bwd_elem_w1(const BwdLaunch& L);  // fem_bwd_w1.cu

}  // namespace fem
