// fem_bwd_iso.cu -- adjoint of the non-affine (quadratic-geometry) forward,
// Eqs. 16-19: the gradients of L = sum dA : A with respect to the vertex
// coordinates, the edge-midpoint nodes and the per-element coefficient.
//
// The forward forms, per element, J^{-1} at every vertex (ji[k] = adj(e_k) /
// det(e_k) with e_k the edge-vector matrix of the geometry map at vertex k,
// e_k[mu][al] = d x_al / d xi_mu), scale = w |det J_c| / DEN at the centroid
// (J_c = the mean of the vertex Jacobians, the map being quadratic), and
//   A_T = scale * sum_g K'[g][T] H_g,   H_g = sum_a ji[k][mu][a] ji[l][nu][a]
// over the folded slot pairs g = ((k mu), (l nu)).  Per lane, in reverse:
//   1. s_g = sum_T K'[g][T] sym(dA)_T (the contraction's adjoint, K' as
//      immediates, one g at a time), dscale += s_g H_g and
//      dji[k][mu] += scale s_g ji[l][nu] (and symmetrically);
//   2. dw = dscale |det J_c| / DEN, d det(e_c) = sgn w dscale / (DEN (d+1)^d),
//      d e_c = d det(e_c) adj(e_c), added to every d e_k;
//   3. ji = e^{-T}: d e_k = -ji[k] dji[k]^T ji[k] + d e_c;
//   4. the nodes (relative to vertex 0): d nd_a = sum_k sum_mu dpsi_a/dxi_mu(vertex
//      k) d e_k[mu], vertex 0 gets minus their sum.
// The vertex gradients take the affine adjoint's path (slot stage, tile
// records, deterministic reduction; or red.add); the edge-node and
// coefficient gradients are per element.  The tile's edge nodes come in, and
// their gradients go out, through a shared-memory stage as contiguous 16-byte
// pieces (an element's 18 floats are not 16-byte aligned on their own).
#include "fem_iso_adj.cuh"

namespace fem {

namespace {

// CTA shape: one-warp CTAs on tets (no CTA-wide barrier), each holding the
// four inverse Jacobians, their adjoints and sym(dA) in registers.
template <int D, int FORM>
struct IsoBwdShape {
  static constexpr int threads = D == 3 ? 32 : kTileElems;
  static constexpr int min_ctas = D == 3 ? (FORM == LAPLACE_P1_ISO ? 16 : 8) : 1;
};

// Per warp: [dA slot][slot stage][edge nodes of the tile, then their gradients].
template <int D, int FORM>
struct IsoBwdPlan {
  using PL = BwdPlan<D, FORM>;
  static constexpr int NEF = D * D * (D + 1) / 2;  // edge-node floats per element
  static constexpr size_t mid_bytes = align_up(size_t(32) * NEF * 4, 128);
  static constexpr size_t per_warp = PL::da_slot + PL::xs_bytes + mid_bytes;
};

template <int D, int FORM, bool ATOMIC>
__global__ void __launch_bounds__(IsoBwdShape<D, FORM>::threads, IsoBwdShape<D, FORM>::min_ctas)
    fem_bwd_iso_kernel(BwdParams p, const float* __restrict__ mid, float* __restrict__ dmid) {
  using FT = FormTraits<D, FORM>;
  using PL = BwdPlan<D, FORM>;
  constexpr int NV = D + 1, NE = D * (D + 1) / 2, NG = n_geo(D);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned char* wbase = smem_raw + size_t(warp) * IsoBwdPlan<D, FORM>::per_warp;
  float* dslot = reinterpret_cast<float*>(wbase);
  float* xs = reinterpret_cast<float*>(wbase + PL::da_slot);
  float* ms = reinterpret_cast<float*>(wbase + PL::da_slot + PL::xs_bytes);  // [32][NE * D]
  const bool rec = !ATOMIC && p.tile_rec != nullptr;
  const int64_t ntiles = (p.n_elem + 31) / 32;
  int err = 0;
  for (int64_t t = int64_t(blockIdx.x) * nwarps + warp; t < ntiles; t += int64_t(gridDim.x) * nwarps) {
    const int64_t e = t * 32 + lane;
    const int cnt = int(p.n_elem - t * 32 < 32 ? p.n_elem - t * 32 : 32);
    copy_dA_async<D, FORM>(p, t, lane, dslot);
    tile_load_async(ms, mid + t * 32 * (NE * D), cnt * (NE * D), lane);
    cp_async_commit();
    int v[NV];
    float X[NV][D];
    load_conn<D>(p.conn, e, p.n_elem, p.vec_conn, v);
    const int flags = gather_regs<D>(p.coords, p.n_vert, e, p.n_elem, v, X);
    uint32_t rk = 0;
    int32_t rb = 0, rn = 0;
    if (rec) {
      rk = __ldg(p.rank + e);  // T * 32 entries: the tail lanes' slots too
      rb = __ldg(p.tile_rec + t);
      rn = __ldg(p.tile_rec + t + 1) - rb;
    }
    const RecAhead ah = rec ? load_rec_ahead(p.rec_span, p.rec_dest, rb, rn, lane) : RecAhead{0u, 0};
    float xb[NV][D], mb[NE][D];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int a = 0; a < D; ++a) xb[k][a] = 0.f;
#pragma unroll
    for (int q = 0; q < NE; ++q)
#pragma unroll
      for (int a = 0; a < D; ++a) mb[q][a] = 0.f;
    float dw = 0.f;
    bool ok = false;
    cp_async_wait<0>();
    __syncwarp();  // the tile's dA rows were copied by other lanes
    if (flags & GF_OK) {
      const float w = (p.coef && e < p.n_elem) ? __ldg(p.coef + e) : 1.f;
      // geometry as the forward forms it: nodes relative to vertex 0, J^{-1}
      // at the vertices, the centroid's edge vectors and adjugate
      float nd[NG][D];
#pragma unroll
      for (int a = 0; a <= D; ++a)
#pragma unroll
        for (int al = 0; al < D; ++al) nd[a][al] = X[a][al] - X[0][al];
      const float* me = ms + lane * (NE * D);
#pragma unroll
      for (int q = 0; q < NE; ++q)
#pragma unroll
        for (int al = 0; al < D; ++al) nd[D + 1 + q][al] = me[q * D + al] - X[0][al];
      float ji[NV][D][D], ec[D][D], adjc[D][D];
      ok = all_vertex_jinv<D>(nd, ji, ec, std::make_integer_sequence<int, NV>{});
      const float detc = det_adj<D>(ec, adjc) * (D == 2 ? (1.f / 9.f) : (1.f / 64.f));
      ok &= detc != 0.f;
      if (!ok) {
        err |= DEVERR_DEGENERATE;
      } else {
        const float absdet = fabsf(detc);
        const float sc = w * absdet * (1.f / float(FT::DEN));
        // 1. the contraction's adjoint, one folded slot pair at a time
        float dji[NV][D][D];
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int mu = 0; mu < D; ++mu)
#pragma unroll
            for (int a = 0; a < D; ++a) dji[k][mu][a] = 0.f;
        float dsc = 0.f;
        {
          SymVals<FT::NT> sym;
          stage_sym<D, FORM>(dslot + lane * PL::DST, sym.s);
          iso_adj_all<D, FORM>(sym, ji, sc, dji, dsc, std::make_integer_sequence<int, FT::NG>{});
        }
        // 2. coefficient and centroid determinant
        dw = dsc * absdet * (1.f / float(FT::DEN));
        const float ddet = (detc > 0.f ? 1.f : -1.f) * dsc * w * (1.f / float(FT::DEN)) *
                           (D == 2 ? (1.f / 9.f) : (1.f / 64.f));
        float dec[D][D];
#pragma unroll
        for (int mu = 0; mu < D; ++mu)
#pragma unroll
          for (int al = 0; al < D; ++al) dec[mu][al] = ddet * adjc[mu][al];
        // 3.-4. inverse Jacobians and the centroid term pulled back to the nodes
        float dnd[NG][D];
#pragma unroll
        for (int a = 0; a < NG; ++a)
#pragma unroll
          for (int al = 0; al < D; ++al) dnd[a][al] = 0.f;
        all_vertex_pullback<D>(ji, dji, dec, dnd, std::make_integer_sequence<int, NV>{});
#pragma unroll
        for (int al = 0; al < D; ++al) {
          float s = 0.f;
#pragma unroll
          for (int a = 1; a < NG; ++a) s += dnd[a][al];
          xb[0][al] = -s;
        }
#pragma unroll
        for (int k = 1; k <= D; ++k)
#pragma unroll
          for (int al = 0; al < D; ++al) xb[k][al] = dnd[k][al];
#pragma unroll
        for (int q = 0; q < NE; ++q)
#pragma unroll
          for (int al = 0; al < D; ++al) mb[q][al] = dnd[D + 1 + q][al];
      }
    } else if (flags & GF_ELEM) {
      err |= DEVERR_CONN;
    }
    if (flags & GF_ELEM) {
      if (p.dcoef) __stcs(p.dcoef + e, dw);

      if constexpr (ATOMIC) {
        if (ok && p.dcoords)
#pragma unroll
          for (int k = 0; k < NV; ++k)
#pragma unroll
            for (int a = 0; a < D; ++a) atomicAdd(p.dcoords + int64_t(v[k]) * D + a, xb[k][a]);
      }
    }
    if (rec) {  // the element's vertex contributions at their stage positions (zeros when skipped)
      constexpr int XP = PL::XP;
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        float* d = xs + ((rk >> (8 * k)) & 0xFFu) * XP;
        if constexpr (XP == 4)
          *reinterpret_cast<float4*>(d) = make_float4(xb[k][0], xb[k][1], D == 3 ? xb[k][D - 1] : 0.f, 0.f);
        else
          *reinterpret_cast<float2*>(d) = make_float2(xb[k][0], xb[k][1]);
      }
      __syncwarp();  // every lane's contributions are staged
      warp_records<D, PL::NC>(xs, p.rec_span, p.rec_dest, rb, rn, ah, p.records, lane);
    }
    if (dmid) {  // the tile's edge-node gradients through the stage, stored coalesced
      __syncwarp();  // every lane has read its edge nodes
#pragma unroll
      for (int q = 0; q < NE; ++q)
#pragma unroll
        for (int al = 0; al < D; ++al) ms[lane * (NE * D) + q * D + al] = mb[q][al];
      __syncwarp();
      tile_store(dmid + t * 32 * (NE * D), ms, cnt * (NE * D), lane);
    }
    __syncwarp();  // the stages and the dA slot are rewritten next tile
  }
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

template <int D, int FORM, bool ATOMIC>
cudaError_t launch_bwd_iso_t(const BwdLaunch& L, const float* mid, float* dmid) {
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
  auto kern = fem_bwd_iso_kernel<D, FORM, ATOMIC>;
  const int warps = IsoBwdShape<D, FORM>::threads / 32;
  const size_t smem = size_t(warps) * IsoBwdPlan<D, FORM>::per_warp;
  cudaError_t st = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (st != cudaSuccess) return st;
  const unsigned grid = pipeline_grid(reinterpret_cast<const void*>(kern), warps, smem, L.n_elem, L.ctas_per_sm);
  kern<<<grid, warps * 32, smem, L.stream>>>(p, mid, dmid);
  return cudaGetLastError();
}

template <int D, int FORM>
cudaError_t launch_bwd_iso_form(const BwdLaunch& L, const float* mid, float* dmid) {
  return L.atomic ? launch_bwd_iso_t<D, FORM, true>(L, mid, dmid) : launch_bwd_iso_t<D, FORM, false>(L, mid, dmid);
}

}  // namespace

cudaError_t launch_bwd_iso(const BwdLaunch& L, const float* mid, float* dmid) {
  if (L.dim == 2) {
    if (L.form == LAPLACE_P1_ISO) return launch_bwd_iso_form<2, LAPLACE_P1_ISO>(L, mid, dmid);
    if (L.form == LAPLACE_P2_ISO) return launch_bwd_iso_form<2, LAPLACE_P2_ISO>(L, mid, dmid);
  } else {
    if (L.form == LAPLACE_P1_ISO) return launch_bwd_iso_form<3, LAPLACE_P1_ISO>(L, mid, dmid);
    if (L.form == LAPLACE_P2_ISO) return launch_bwd_iso_form<3, LAPLACE_P2_ISO>(L, mid, dmid);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fem
